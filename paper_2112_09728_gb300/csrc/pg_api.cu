// C ABI of the guide pass (include/pg.h): context, argument checks, launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/pg.h"
#include "pg_launch.h"

struct pg_ctx {
    pg_config cfg;
    cudaStream_t stream = nullptr;
    int device = 0;
    void* gam[2] = {nullptr, nullptr};
    int cur = 0;
    size_t gam_bytes = 0;
    float4* work = nullptr;   // binary32 work copy of the staged pass
    int phase = 0;            // 1 between pg_reproject and pg_update
    int* d_err = nullptr;     // device flag: non-finite Gamma stored
    pgk::Params base;         // configuration part of the launch parameters
    std::string err;
};

namespace {

pg_status fail(pg_ctx* c, pg_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

pg_status cuda_fail(pg_ctx* c, cudaError_t e, const char* where) {
    return fail(c, PG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Gauss-Legendre rule on [-1, 1]: nodes are the roots of P_n found by Newton
// iteration from Chebyshev-like starting points, weights 2/((1-x^2) P_n'(x)^2).
void gauss_legendre(int n, float* x_out, float* w_out) {
    for (int i = 0; i < n; ++i) {
        double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        x_out[i] = (float)x;
        w_out[i] = (float)(2.0 / ((1.0 - x * x) * dp * dp));
    }
}

pg_status check_config(const pg_config* c, std::string& why) {
    char buf[160];
    if (c->width < 1 || c->width > 32768 || c->height < 1 || c->height > 32768) {
        std::snprintf(buf, sizeof buf, "width/height %d x %d outside [1, 32768]", c->width, c->height);
        why = buf;
        return PG_ERR_ARG;
    }
    if ((int64_t)c->width * c->height > (int64_t)1 << 30) { why = "more than 2^30 pixels"; return PG_ERR_ARG; }
    if (c->spp < 1 || c->spp > 1024) { why = "spp outside [1, 1024]"; return PG_ERR_ARG; }
    if (c->gamma_dtype < PG_F32 || c->gamma_dtype > PG_BF16) { why = "unknown gamma_dtype"; return PG_ERR_ARG; }
    if (c->k_max < 0 || c->k_max > 1 << 20) { why = "k_max outside [0, 2^20]"; return PG_ERR_ARG; }
    if (!(c->pi_min >= 0.0f && c->pi_min <= c->pi_max && c->pi_max <= 1.0f)) {
        why = "need 0 <= pi_min <= pi_max <= 1";
        return PG_ERR_ARG;
    }
    if (!(c->pi_reinit >= 0.0f && c->pi_reinit <= 1.0f) || !(c->init_pi >= 0.0f && c->init_pi <= 1.0f)) {
        why = "pi_reinit / init_pi outside [0, 1]";
        return PG_ERR_ARG;
    }
    if (!(c->sigma2_min > 0.0f) || !(c->rho_max >= 0.0f && c->rho_max < 1.0f)) {
        why = "need sigma2_min > 0 and 0 <= rho_max < 1";
        return PG_ERR_ARG;
    }
    if (!(c->depth_tol >= 0.0f) || !std::isfinite(c->normal_tol) || !std::isfinite(c->rough_min)) {
        why = "bad depth_tol / normal_tol / rough_min";
        return PG_ERR_ARG;
    }
    if (!(c->init_sigma[0] > 0.0f && c->init_sigma[1] > 0.0f) ||
        !(c->init_sigma[2] * c->init_sigma[2] < c->init_sigma[0] * c->init_sigma[1]) ||
        !(c->init_mu[0] >= 0.0f && c->init_mu[0] <= 1.0f && c->init_mu[1] >= 0.0f && c->init_mu[1] <= 1.0f)) {
        why = "initial guide must have mu in [0,1]^2 and a positive definite covariance";
        return PG_ERR_ARG;
    }
    return PG_OK;
}

pg_status fill_camera(pg_ctx* c, const pg_camera& cam, pgk::Params& P) {
    if (cam.kind != 0 && cam.kind != 1) return fail(c, PG_ERR_ARG, "camera kind must be 0 or 1");
    P.cam_kind = cam.kind;
    for (int k = 0; k < 3; ++k) {
        P.cam_o[k] = cam.origin[k];
        P.cam_f[k] = cam.fwd[k];
        P.cam_r[k] = cam.right[k];
        P.cam_u[k] = cam.up[k];
    }
    P.cam_ps = cam.pixel_size;
    P.cam_tan = cam.tan_half_fov;
    P.cam_aspect = (float)P.W / (float)P.H;
    return PG_OK;
}

pg_status fill_field(pg_ctx* c, const pg_field* f, pgk::Params& P) {
    if (!f) return fail(c, PG_ERR_ARG, "field is NULL");
    if (f->n_lobes < 0 || f->n_lobes > 8) return fail(c, PG_ERR_ARG, "n_lobes outside [0, 8]");
    if (f->mask_kind != 0 && f->mask_kind != 1) return fail(c, PG_ERR_ARG, "mask_kind must be 0 or 1");
    P.n_lobes = f->n_lobes;
    for (int j = 0; j < 8; ++j) {
        for (int k = 0; k < 3; ++k) P.lobe_dir[j][k] = j < f->n_lobes ? f->dir[j][k] : 0.0f;
        if (j < f->n_lobes) {
            const double kap = f->kappa[j];
            if (!(kap > 0.0) || !std::isfinite(kap)) return fail(c, PG_ERR_ARG, "lobe kappa must be > 0");
            // normalised vMF on the sphere: kappa / (2 pi (1 - exp(-2 kappa)))
            P.lobe_kappa[j] = (float)kap;
            P.lobe_scale[j] = (float)((double)f->amp[j] * kap / (2.0 * M_PI * -std::expm1(-2.0 * kap)));
        } else {
            P.lobe_kappa[j] = 0.0f;
            P.lobe_scale[j] = 0.0f;
        }
    }
    P.field_const = f->constant;
    P.mask_kind = f->mask_kind;
    for (int k = 0; k < 3; ++k) P.mask[k] = f->mask[k];
    return PG_OK;
}

pg_status check_gbuffer(pg_ctx* c, const pg_gbuffer* g) {
    if (!g || !g->g0 || !g->g1) return fail(c, PG_ERR_ARG, "G-buffer or one of its planes is NULL");
    if (!aligned16(g->g0) || !aligned16(g->g1)) return fail(c, PG_ERR_ARG, "G-buffer planes must be 16-byte aligned");
    return PG_OK;
}

size_t hw_of(const pg_ctx* c) { return (size_t)c->cfg.width * c->cfg.height; }

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const char *pa = (const char*)a, *pb = (const char*)b;
    return a && b && pa < pb + nb && pb < pa + na;
}

pg_status ensure_work(pg_ctx* c) {
    if (c->work) return PG_OK;
    cudaError_t e = cudaMalloc(&c->work, 2 * hw_of(c) * sizeof(float4));
    if (e != cudaSuccess) {
        c->work = nullptr;
        cudaGetLastError();
        return fail(c, PG_ERR_OOM, "cannot allocate the staged work copy");
    }
    return PG_OK;
}

}  // namespace

extern "C" {

void pg_config_default(pg_config* c, int32_t width, int32_t height) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->width = width;
    c->height = height;
    c->spp = 1;
    c->gamma_dtype = PG_F32;
    c->seed = 0;
    c->k_max = 32;
    c->pi_min = 0.05f;
    c->pi_max = 0.95f;
    c->pi_reinit = 0.05f;
    c->depth_tol = 0.1f;
    c->normal_tol = 0.9f;
    c->rough_min = 0.1f;
    c->sigma2_min = 1e-4f;
    c->rho_max = 0.9f;
    c->init_mu[0] = c->init_mu[1] = 0.5f;
    c->init_sigma[0] = c->init_sigma[1] = 0.1f;
    c->init_sigma[2] = 0.0f;
    c->init_pi = 0.5f;
}

pg_status pg_create(const pg_config* cfg, void* stream, pg_ctx** out) {
    if (!out) return PG_ERR_ARG;
    *out = nullptr;
    if (!cfg) return PG_ERR_ARG;
    std::string why;
    if (check_config(cfg, why) != PG_OK) {
        std::fprintf(stderr, "pg_create: %s\n", why.c_str());
        return PG_ERR_ARG;
    }
    pg_ctx* c = new (std::nothrow) pg_ctx();
    if (!c) return PG_ERR_OOM;
    c->cfg = *cfg;
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    const size_t hw = hw_of(c);
    c->gam_bytes = hw * (cfg->gamma_dtype == PG_F32 ? 32 : 16);

    pgk::Params& P = c->base;
    std::memset(&P, 0, sizeof P);
    P.W = cfg->width;
    P.H = cfg->height;
    P.spp = cfg->spp;
    P.k_max = cfg->k_max;
    P.key0 = (uint32_t)(cfg->seed & 0xffffffffu);
    P.key1 = (uint32_t)(cfg->seed >> 32);
    P.pi_min = cfg->pi_min;
    P.pi_max = cfg->pi_max;
    P.pi_reinit = cfg->pi_reinit;
    P.depth_tol = cfg->depth_tol;
    P.normal_tol = cfg->normal_tol;
    P.rough_min = cfg->rough_min;
    P.sigma2_min = cfg->sigma2_min;
    P.rho_max = cfg->rho_max;
    const double mx = cfg->init_mu[0], my = cfg->init_mu[1];
    P.init_raw[0] = (float)mx;
    P.init_raw[1] = (float)my;
    P.init_raw[2] = (float)(cfg->init_sigma[0] + mx * mx);
    P.init_raw[3] = (float)(cfg->init_sigma[1] + my * my);
    P.init_raw[4] = (float)(cfg->init_sigma[2] + mx * my);
    P.init_c[0] = cfg->init_sigma[0];
    P.init_c[1] = cfg->init_sigma[1];
    P.init_c[2] = cfg->init_sigma[2];
    gauss_legendre(4, P.gl_x, P.gl_w);
    gauss_legendre(6, P.gl_x + 4, P.gl_w + 4);
    gauss_legendre(8, P.gl_x + 10, P.gl_w + 10);

    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&c->gam[b], c->gam_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        pg_destroy(c);
        return PG_ERR_OOM;
    }
    e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = pgk::launch_init(cfg->gamma_dtype, P, c->gam[0], cfg->init_pi, c->stream);
    if (e != cudaSuccess) {
        std::fprintf(stderr, "pg_create: %s\n", cudaGetErrorString(e));
        pg_destroy(c);
        return PG_ERR_CUDA;
    }
    *out = c;
    return PG_OK;
}

pg_status pg_set_stream(pg_ctx* c, void* stream) {
    if (!c) return PG_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    return PG_OK;
}

pg_status pg_reproject(pg_ctx* c, const pg_gbuffer* cur, const float* d_g0_prev, uint8_t* d_accept) {
    if (!c) return PG_ERR_ARG;
    if (c->phase != 0) return fail(c, PG_ERR_STATE, "pg_reproject: a staged frame is already in progress");
    pg_status s = check_gbuffer(c, cur);
    if (s != PG_OK) return s;
    if (!d_g0_prev || !aligned16(d_g0_prev)) return fail(c, PG_ERR_ARG, "d_g0_prev NULL or not 16-byte aligned");
    if ((s = ensure_work(c)) != PG_OK) return s;
    pgk::Params P = c->base;
    if ((s = fill_camera(c, cur->camera, P)) != PG_OK) return s;
    cudaError_t e = pgk::launch_reproject(c->cfg.gamma_dtype, P, c->gam[c->cur], c->work, (const float4*)cur->g0,
                                          (const float4*)cur->g1, (const float4*)d_g0_prev, d_accept, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_reproject");
    c->phase = 1;
    return PG_OK;
}

pg_status pg_sample(pg_ctx* c, const pg_gbuffer* cur, const pg_field* field, uint32_t frame,
                    const pg_samples* d_out, float* d_img) {
    if (!c) return PG_ERR_ARG;
    if (c->phase != 1) return fail(c, PG_ERR_STATE, "pg_sample: call pg_reproject first");
    pg_status s = check_gbuffer(c, cur);
    if (s != PG_OK) return s;
    pgk::Params P = c->base;
    if ((s = fill_camera(c, cur->camera, P)) != PG_OK || (s = fill_field(c, field, P)) != PG_OK) return s;
    pgk::SamplePlanes o{};
    if (d_out) {
        o.wx = d_out->wx; o.wy = d_out->wy; o.wz = d_out->wz;
        o.radiance = d_out->radiance; o.pdf = d_out->pdf; o.mis = d_out->mis;
        o.estimate = d_out->estimate; o.strategy = d_out->strategy;
        if ((o.wx != nullptr) != (o.wy != nullptr) || (o.wx != nullptr) != (o.wz != nullptr))
            return fail(c, PG_ERR_ARG, "pg_sample: wx, wy, wz must be all set or all NULL");
    }
    cudaError_t e = pgk::launch_sample(c->cfg.gamma_dtype, P, c->work, (const float4*)cur->g0, (const float4*)cur->g1,
                                       frame, o, d_img, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_sample");
    return PG_OK;
}

pg_status pg_update(pg_ctx* c, const pg_gbuffer* cur, const pg_samples* d_in) {
    if (!c) return PG_ERR_ARG;
    if (c->phase != 1) return fail(c, PG_ERR_STATE, "pg_update: call pg_reproject first");
    pg_status s = check_gbuffer(c, cur);
    if (s != PG_OK) return s;
    if (!d_in || !d_in->wx || !d_in->wy || !d_in->wz || !d_in->radiance || !d_in->strategy)
        return fail(c, PG_ERR_ARG, "pg_update: wx, wy, wz, radiance and strategy are required");
    pgk::Params P = c->base;
    if ((s = fill_camera(c, cur->camera, P)) != PG_OK) return s;
    pgk::SamplePlanes in{d_in->wx, d_in->wy, d_in->wz, d_in->radiance, nullptr, nullptr, nullptr, d_in->strategy};
    cudaError_t e = pgk::launch_update(c->cfg.gamma_dtype, P, c->work, (const float4*)cur->g0,
                                       (const float4*)cur->g1, in, c->gam[c->cur ^ 1], c->d_err, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_update");
    c->cur ^= 1;
    c->phase = 0;
    return PG_OK;
}

pg_status pg_frame(pg_ctx* c, const pg_gbuffer* cur, const float* d_g0_prev, const pg_field* field,
                   uint32_t frame, float* d_img) {
    if (!c) return PG_ERR_ARG;
    if (c->phase != 0) return fail(c, PG_ERR_STATE, "pg_frame: a staged frame is in progress");
    pg_status s = check_gbuffer(c, cur);
    if (s != PG_OK) return s;
    if (!d_g0_prev || !aligned16(d_g0_prev)) return fail(c, PG_ERR_ARG, "d_g0_prev NULL or not 16-byte aligned");
    const size_t hw = hw_of(c);
    if (overlaps(d_img, hw * 4, c->gam[0], c->gam_bytes) || overlaps(d_img, hw * 4, c->gam[1], c->gam_bytes))
        return fail(c, PG_ERR_ARG, "d_img overlaps Gamma");
    pgk::Params P = c->base;
    if ((s = fill_camera(c, cur->camera, P)) != PG_OK || (s = fill_field(c, field, P)) != PG_OK) return s;
    cudaError_t e = pgk::launch_frame(c->cfg.gamma_dtype, P, c->gam[c->cur], c->gam[c->cur ^ 1],
                                      (const float4*)cur->g0, (const float4*)cur->g1, (const float4*)d_g0_prev,
                                      d_img, frame, c->d_err, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_frame");
    c->cur ^= 1;
    return PG_OK;
}

pg_status pg_eval(pg_ctx* c, const pg_gbuffer* cur, const pg_field* field, int32_t n_dirs, const float* d_dirs,
                  float* d_out) {
    if (!c) return PG_ERR_ARG;
    pg_status s = check_gbuffer(c, cur);
    if (s != PG_OK) return s;
    if (n_dirs < 0 || n_dirs > 1 << 16) return fail(c, PG_ERR_ARG, "pg_eval: n_dirs outside [0, 65536]");
    if (n_dirs == 0) return PG_OK;
    if (!d_dirs || !d_out) return fail(c, PG_ERR_ARG, "pg_eval: d_dirs and d_out are required");
    pgk::Params P = c->base;
    if ((s = fill_camera(c, cur->camera, P)) != PG_OK || (s = fill_field(c, field, P)) != PG_OK) return s;
    const bool work = c->phase == 1;
    cudaError_t e = pgk::launch_eval(c->cfg.gamma_dtype, P, work ? (const void*)c->work : c->gam[c->cur], work,
                                     (const float4*)cur->g0, (const float4*)cur->g1, n_dirs, d_dirs, d_out,
                                     c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_eval");
    return PG_OK;
}

size_t pg_gamma_bytes(const pg_ctx* c) { return c ? c->gam_bytes : 0; }

pg_status pg_get_gamma(pg_ctx* c, void* dst, int32_t dst_is_host) {
    if (!c || !dst) return fail(c, PG_ERR_ARG, "pg_get_gamma: NULL argument");
    cudaError_t e = cudaMemcpyAsync(dst, c->gam[c->cur], c->gam_bytes,
                                    dst_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && dst_is_host) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_get_gamma");
    return PG_OK;
}

pg_status pg_set_gamma(pg_ctx* c, const void* src, int32_t src_is_host) {
    if (!c || !src) return fail(c, PG_ERR_ARG, "pg_set_gamma: NULL argument");
    if (c->phase != 0) return fail(c, PG_ERR_STATE, "pg_set_gamma: a staged frame is in progress");
    cudaError_t e = cudaMemcpyAsync(c->gam[c->cur], src, c->gam_bytes,
                                    src_is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && src_is_host) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_set_gamma");
    return PG_OK;
}

pg_status pg_gamma_to_f32(pg_ctx* c, float* d_dst) {
    if (!c || !d_dst || !aligned16(d_dst)) return fail(c, PG_ERR_ARG, "pg_gamma_to_f32: NULL or unaligned");
    cudaError_t e = pgk::launch_to_f32(c->cfg.gamma_dtype, c->base, c->gam[c->cur], false, (float4*)d_dst, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_gamma_to_f32");
    return PG_OK;
}

pg_status pg_gamma_from_f32(pg_ctx* c, const float* d_src) {
    if (!c || !d_src || !aligned16(d_src)) return fail(c, PG_ERR_ARG, "pg_gamma_from_f32: NULL or unaligned");
    if (c->phase != 0) return fail(c, PG_ERR_STATE, "pg_gamma_from_f32: a staged frame is in progress");
    cudaError_t e = pgk::launch_from_f32(c->cfg.gamma_dtype, c->base, (const float4*)d_src, c->gam[c->cur], c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_gamma_from_f32");
    return PG_OK;
}

pg_status pg_get_reprojected(pg_ctx* c, float* d_dst) {
    if (!c || !d_dst || !aligned16(d_dst)) return fail(c, PG_ERR_ARG, "pg_get_reprojected: NULL or unaligned");
    if (c->phase != 1) return fail(c, PG_ERR_STATE, "pg_get_reprojected: call pg_reproject first");
    cudaError_t e = pgk::launch_to_f32(c->cfg.gamma_dtype, c->base, c->work, true, (float4*)d_dst, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_get_reprojected");
    return PG_OK;
}

pg_status pg_check(pg_ctx* c) {
    if (!c) return PG_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_check");
    int flag = 0;
    e = cudaMemcpy(&flag, c->d_err, sizeof flag, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_check");
    if (flag) {
        cudaMemset(c->d_err, 0, sizeof(int));
        return fail(c, PG_ERR_NUMERIC, "a kernel stored a non-finite Gamma");
    }
    return PG_OK;
}

pg_status pg_philox(const uint32_t* d_ctr, const uint32_t key[2], int64_t n, uint32_t* d_out, int32_t use_curand,
                    void* stream) {
    if (n < 0 || n > ((int64_t)1 << 31) * 256) return PG_ERR_ARG;
    if (n == 0) return PG_OK;
    if (!d_ctr || !key || !d_out || !aligned16(d_ctr) || !aligned16(d_out)) return PG_ERR_ARG;
    cudaError_t e = pgk::launch_philox(d_ctr, key[0], key[1], n, d_out, use_curand != 0, (cudaStream_t)stream);
    return e == cudaSuccess ? PG_OK : PG_ERR_CUDA;
}

const char* pg_last_error(const pg_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

void pg_destroy(pg_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int b = 0; b < 2; ++b)
        if (c->gam[b]) cudaFree(c->gam[b]);
    if (c->work) cudaFree(c->work);
    if (c->d_err) cudaFree(c->d_err);
    delete c;
}

}  // extern "C"
