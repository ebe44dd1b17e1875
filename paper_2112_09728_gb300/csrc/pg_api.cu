// C ABI of the guide pass (include/pg.h): context, argument checks, launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/pg.h"
#include "pg_launch.h"
#include "pg_params.h"

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
    uint32_t sample_frame = 0;  // frame of the last pg_sample (rounding bits of pg_update)
    // Adam moments of theta (allocated on first use): binary32 [6][H*W] planes
    // in adam_m and adam_v, or BF16 records of 24 bytes per pixel in adam_m alone
    void* adam_m = nullptr;
    void* adam_v = nullptr;
    float4* vpl = nullptr;    // neighbour reuse: one VPL per sample {world direction, radiance}
    float* vpl_pb = nullptr;  //   and the density of its BRDF draw (0: does not train)
    float2* hand = nullptr;   //   and each pixel's handover record {Z, reprojection outcome} between the passes
    // pg_frames_host: device rings for the G-buffer and the image, upload and
    // read-back streams, and per-step events (created on first use)
    cudaStream_t hs_up = nullptr, hs_down = nullptr;
    float4* hg0[3] = {nullptr, nullptr, nullptr};
    float4* hg1[2] = {nullptr, nullptr};
    float* himg[2] = {nullptr, nullptr};
    cudaEvent_t ev_up[4] = {}, ev_ran[4] = {}, ev_down[4] = {};
    bool host_ready = false;
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

using pgk::aligned16;

pg_status fill_camera(pg_ctx* c, const pg_camera& cam, pgk::Params& P) {
    std::string why;
    const pg_status s = pgk::camera_params(cam, P, why);
    return s == PG_OK ? s : fail(c, s, why);
}

pg_status fill_field(pg_ctx* c, const pg_field* f, pgk::Params& P) {
    std::string why;
    const pg_status s = pgk::field_params(f, P, why);
    return s == PG_OK ? s : fail(c, s, why);
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

// Frees the host pipeline's streams, events and device rings (any subset may
// exist after a failed set-up) and clears the pointers.
void release_host(pg_ctx* c) {
    for (int k = 0; k < 3; ++k) {
        if (c->hg0[k]) cudaFree(c->hg0[k]);
        c->hg0[k] = nullptr;
    }
    for (int k = 0; k < 2; ++k) {
        if (c->hg1[k]) cudaFree(c->hg1[k]);
        if (c->himg[k]) cudaFree(c->himg[k]);
        c->hg1[k] = nullptr;
        c->himg[k] = nullptr;
    }
    for (int k = 0; k < 4; ++k) {
        if (c->ev_up[k]) cudaEventDestroy(c->ev_up[k]);
        if (c->ev_ran[k]) cudaEventDestroy(c->ev_ran[k]);
        if (c->ev_down[k]) cudaEventDestroy(c->ev_down[k]);
        c->ev_up[k] = c->ev_ran[k] = c->ev_down[k] = nullptr;
    }
    if (c->hs_up) cudaStreamDestroy(c->hs_up);
    if (c->hs_down) cudaStreamDestroy(c->hs_down);
    c->hs_up = c->hs_down = nullptr;
    c->host_ready = false;
}

pg_status ensure_host(pg_ctx* c) {
    if (c->host_ready) return PG_OK;
    const size_t hw = hw_of(c);
    cudaError_t e = cudaStreamCreateWithFlags(&c->hs_up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->hs_down, cudaStreamNonBlocking);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&c->ev_up[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_ran[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_down[k], cudaEventDisableTiming);
    }
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMalloc(&c->hg0[k], hw * sizeof(float4));
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMalloc(&c->hg1[k], hw * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc(&c->himg[k], 3 * hw * sizeof(float));   // room for three planes
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        release_host(c);   // a later call starts from nothing
        return fail(c, PG_ERR_OOM, std::string("pg_frames_host: cannot set up the host pipeline: ") +
                                       cudaGetErrorString(e));
    }
    c->host_ready = true;
    return PG_OK;
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
    c->ggx_f0 = 1.0f;
}

pg_status pg_create(const pg_config* cfg, void* stream, pg_ctx** out) {
    if (!out) return PG_ERR_ARG;
    *out = nullptr;
    if (!cfg) return PG_ERR_ARG;
    std::string why;
    if (pgk::check_config(cfg, why) != PG_OK) {
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
    pgk::config_params(*cfg, P);

    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&c->gam[b], c->gam_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int));
    if (e == cudaSuccess && cfg->reuse_radius > 0) {
        const size_t n = hw * (size_t)cfg->spp;
        e = cudaMalloc(&c->vpl, n * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc(&c->vpl_pb, n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&c->hand, hw * sizeof(float2));
    }
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
    if (c->cfg.reuse_radius > 0) return fail(c, PG_ERR_ARG, "pg_reproject: neighbour reuse runs in pg_frame only");
    pg_status s = check_gbuffer(c, cur);
    if (s != PG_OK) return s;
    if (!d_g0_prev || !aligned16(d_g0_prev)) return fail(c, PG_ERR_ARG, "d_g0_prev NULL or not 16-byte aligned");
    if ((s = ensure_work(c)) != PG_OK) return s;
    pgk::Params P = c->base;
    if ((s = fill_camera(c, cur->camera, P)) != PG_OK) return s;
    cudaError_t e = pgk::launch_reproject(c->cfg.gamma_dtype, P, c->gam[c->cur], c->work, (const float4*)cur->g0,
                                          (const float4*)cur->g1, (const float4*)d_g0_prev, d_accept, c->d_err,
                                          c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_reproject");
    c->phase = 1;
    c->sample_frame = 0;
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
    c->sample_frame = frame;
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
    P.sr_frame = c->sample_frame;
    pgk::SamplePlanes in{d_in->wx, d_in->wy, d_in->wz, d_in->radiance, nullptr, nullptr, nullptr, d_in->strategy};
    cudaError_t e = pgk::launch_update(c->cfg.gamma_dtype, P, c->work, (const float4*)cur->g0,
                                       (const float4*)cur->g1, in, c->gam[c->cur ^ 1], c->d_err, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_update");
    c->cur ^= 1;
    c->phase = 0;
    return PG_OK;
}

}  // extern "C"

namespace {

// The launches of one frame on the context's stream (arguments checked by the caller).
pg_status frame_impl(pg_ctx* c, const pg_gbuffer* cur, const float* d_g0_prev, const pg_field* field,
                     uint32_t frame, float* d_img) {
    pg_status s;
    pgk::Params P = c->base;
    if ((s = fill_camera(c, cur->camera, P)) != PG_OK || (s = fill_field(c, field, P)) != PG_OK) return s;
    const float4 *g0 = (const float4*)cur->g0, *g1 = (const float4*)cur->g1, *g0p = (const float4*)d_g0_prev;
    cudaError_t e;
    if (c->cfg.reuse_radius > 0) {
        // the paper's two passes: path tracing writes the VPLs, training reads them
        e = pgk::launch_pt(c->cfg.gamma_dtype, P, c->gam[c->cur], g0, g1, g0p, d_img, frame, c->vpl, c->vpl_pb,
                           c->hand, c->d_err, c->stream);
        if (e == cudaSuccess)
            e = pgk::launch_train(c->cfg.gamma_dtype, P, c->gam[c->cur], c->gam[c->cur ^ 1], g0, g1, g0p, frame,
                                  c->vpl, c->vpl_pb, c->hand, c->d_err, c->stream);
    } else {
        e = pgk::launch_frame(c->cfg.gamma_dtype, P, c->gam[c->cur], c->gam[c->cur ^ 1], g0, g1, g0p, d_img, frame,
                              c->d_err, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_frame");
    c->cur ^= 1;
    return PG_OK;
}

}  // namespace

extern "C" {

pg_status pg_frame(pg_ctx* c, const pg_gbuffer* cur, const float* d_g0_prev, const pg_field* field,
                   uint32_t frame, float* d_img) {
    if (!c) return PG_ERR_ARG;
    if (c->phase != 0) return fail(c, PG_ERR_STATE, "pg_frame: a staged frame is in progress");
    pg_status s = check_gbuffer(c, cur);
    if (s != PG_OK) return s;
    if (!d_g0_prev || !aligned16(d_g0_prev)) return fail(c, PG_ERR_ARG, "d_g0_prev NULL or not 16-byte aligned");
    const size_t ib = hw_of(c) * 4 * (field && field->rgb ? 3 : 1);
    if (overlaps(d_img, ib, c->gam[0], c->gam_bytes) || overlaps(d_img, ib, c->gam[1], c->gam_bytes))
        return fail(c, PG_ERR_ARG, "d_img overlaps Gamma");
    return frame_impl(c, cur, d_g0_prev, field, frame, d_img);
}

pg_status pg_frames_host(pg_ctx* c, int32_t n_frames, const float* h_g0, const float* h_g1,
                         const pg_camera* cameras, const pg_field* field, uint32_t frame0, const float* h_g0_prev,
                         float* h_img) {
    if (!c) return PG_ERR_ARG;
    if (c->phase != 0) return fail(c, PG_ERR_STATE, "pg_frames_host: a staged frame is in progress");
    if (n_frames < 1 || n_frames > (1 << 20)) return fail(c, PG_ERR_ARG, "pg_frames_host: n_frames outside [1, 2^20]");
    if (!h_g0 || !h_g1 || !cameras) return fail(c, PG_ERR_ARG, "pg_frames_host: h_g0, h_g1 and cameras are required");
    if (!field) return fail(c, PG_ERR_ARG, "pg_frames_host: field is NULL");
    pg_status s = ensure_host(c);
    if (s != PG_OK) return s;
    const size_t planes = field->rgb ? 3 : 1;
    const size_t hw = hw_of(c), gbytes = hw * sizeof(float4), ibytes = planes * hw * sizeof(float);
    cudaError_t e = cudaSuccess;
    // step t: upload into g0 slot t % 3 and g1 slot t % 2, once step t-2 (the
    // last reader of both slots) has run; run once the upload is in and step
    // t-2's image has been read back; read back once the step has run.
    if (h_g0_prev) e = cudaMemcpyAsync(c->hg0[2], h_g0_prev, gbytes, cudaMemcpyHostToDevice, c->hs_up);
    for (int32_t t = 0; t < n_frames && e == cudaSuccess; ++t) {
        const int a = t % 3, b = t % 2, k = t % 4, k2 = (t + 2) % 4;   // k2: the events of step t - 2
        if (t >= 2) e = cudaStreamWaitEvent(c->hs_up, c->ev_ran[k2], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->hg0[a], h_g0 + (size_t)t * hw * 4, gbytes, cudaMemcpyHostToDevice, c->hs_up);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->hg1[b], h_g1 + (size_t)t * hw * 4, gbytes, cudaMemcpyHostToDevice, c->hs_up);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_up[k], c->hs_up);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_up[k], 0);
        if (e == cudaSuccess && t >= 2 && h_img) e = cudaStreamWaitEvent(c->stream, c->ev_down[k2], 0);
        if (e != cudaSuccess) break;
        pg_gbuffer gb;
        gb.g0 = reinterpret_cast<const float*>(c->hg0[a]);
        gb.g1 = reinterpret_cast<const float*>(c->hg1[b]);
        gb.camera = cameras[t];
        const float4* prev = t > 0 ? c->hg0[(t + 2) % 3] : (h_g0_prev ? c->hg0[2] : c->hg0[a]);
        s = frame_impl(c, &gb, reinterpret_cast<const float*>(prev), field, frame0 + (uint32_t)t,
                       h_img ? c->himg[b] : nullptr);
        if (s != PG_OK) {
            cudaStreamSynchronize(c->hs_up);
            cudaStreamSynchronize(c->stream);
            cudaStreamSynchronize(c->hs_down);
            return s;
        }
        e = cudaEventRecord(c->ev_ran[k], c->stream);
        if (e == cudaSuccess && h_img) {
            e = cudaStreamWaitEvent(c->hs_down, c->ev_ran[k], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_img + (size_t)t * planes * hw, c->himg[b], ibytes, cudaMemcpyDeviceToHost,
                                    c->hs_down);
            if (e == cudaSuccess) e = cudaEventRecord(c->ev_down[k], c->hs_down);
        }
    }
    const cudaError_t e1 = cudaStreamSynchronize(c->hs_up);
    const cudaError_t e2 = cudaStreamSynchronize(c->stream);
    const cudaError_t e3 = cudaStreamSynchronize(c->hs_down);
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_frames_host");
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
        if (flag & PG_ERR_BIT_BOUNDS)
            return fail(c, PG_ERR_BOUNDS, "an index of the bounds-checked build fell outside its buffer");
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

pg_status pg_grad(pg_ctx* c, const pg_gbuffer* cur, const pg_field* field, uint32_t frame, int32_t n_samples,
                  const float* d_theta, float* d_loss, float* d_grad) {
    if (!c) return PG_ERR_ARG;
    if (c->phase != 0) return fail(c, PG_ERR_STATE, "pg_grad: a staged frame is in progress");
    pg_status s = check_gbuffer(c, cur);
    if (s != PG_OK) return s;
    if (n_samples < 1 || n_samples > 1 << 16) return fail(c, PG_ERR_ARG, "pg_grad: n_samples outside [1, 65536]");
    if (!d_loss || !d_grad) return fail(c, PG_ERR_ARG, "pg_grad: d_loss and d_grad are required");
    pgk::Params P = c->base;
    if ((s = fill_camera(c, cur->camera, P)) != PG_OK || (s = fill_field(c, field, P)) != PG_OK) return s;
    cudaError_t e = pgk::launch_grad(c->cfg.gamma_dtype, P, c->gam[c->cur], d_theta, (const float4*)cur->g0,
                                     (const float4*)cur->g1, frame, n_samples, d_loss, d_grad, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_grad");
    return PG_OK;
}

static bool adam_bf16(const pg_ctx* c) { return c->cfg.adam_dtype == PG_BF16; }

static pg_status ensure_adam(pg_ctx* c, const char* where) {
    if (c->adam_m) return PG_OK;
    const size_t bytes = 6 * hw_of(c) * sizeof(float);   // one plane set, or both BF16 moments
    bool ok = cudaMalloc(&c->adam_m, bytes) == cudaSuccess;
    if (ok && !adam_bf16(c)) ok = cudaMalloc(&c->adam_v, bytes) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (c->adam_m) cudaFree(c->adam_m);
        c->adam_m = c->adam_v = nullptr;
        return fail(c, PG_ERR_OOM, where);
    }
    return PG_OK;
}

pg_status pg_adam_step(pg_ctx* c, const float* d_grad, float lr, float beta1, float beta2, float eps, int32_t step) {
    if (!c) return PG_ERR_ARG;
    if (c->phase != 0) return fail(c, PG_ERR_STATE, "pg_adam_step: a staged frame is in progress");
    if (!d_grad) return fail(c, PG_ERR_ARG, "pg_adam_step: d_grad is required");
    if (step < 1 || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f) ||
        !std::isfinite(lr))
        return fail(c, PG_ERR_ARG, "pg_adam_step: need step >= 1, 0 <= beta < 1, eps > 0, finite lr");
    pg_status s = ensure_adam(c, "pg_adam_step: cannot allocate the Adam moments");
    if (s != PG_OK) return s;
    const size_t bytes = 6 * hw_of(c) * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (step == 1) {   // a new run of steps starts from zero moments
        e = cudaMemsetAsync(c->adam_m, 0, bytes, c->stream);
        if (e == cudaSuccess && c->adam_v) e = cudaMemsetAsync(c->adam_v, 0, bytes, c->stream);
    }
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, step)));
    if (e == cudaSuccess) {
        if (adam_bf16(c))
            e = pgk::launch_adam_bf16(c->cfg.gamma_dtype, c->base, c->gam[c->cur], d_grad, c->adam_m, lr, beta1,
                                      beta2, eps, c1, c2, (uint32_t)step, c->stream);
        else
            e = pgk::launch_adam(c->cfg.gamma_dtype, c->base, c->gam[c->cur], d_grad, (float*)c->adam_m,
                                 (float*)c->adam_v, lr, beta1, beta2, eps, c1, c2, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_adam_step");
    return PG_OK;
}

pg_status pg_get_adam_state(pg_ctx* c, float* d_m, float* d_v) {
    if (!c) return PG_ERR_ARG;
    if (!d_m || !d_v || d_m == d_v) return fail(c, PG_ERR_ARG, "pg_get_adam_state: need two distinct buffers");
    if (!c->adam_m) return fail(c, PG_ERR_STATE, "pg_get_adam_state: no Adam step has run");
    const size_t bytes = 6 * hw_of(c) * sizeof(float);
    cudaError_t e;
    if (adam_bf16(c)) {
        e = pgk::launch_adam_rec_get(c->base, c->adam_m, d_m, d_v, c->stream);
    } else {
        e = cudaMemcpyAsync(d_m, c->adam_m, bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_v, c->adam_v, bytes, cudaMemcpyDeviceToDevice, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_get_adam_state");
    return PG_OK;
}

pg_status pg_set_adam_state(pg_ctx* c, const float* d_m, const float* d_v) {
    if (!c) return PG_ERR_ARG;
    if (!d_m || !d_v) return fail(c, PG_ERR_ARG, "pg_set_adam_state: NULL argument");
    pg_status s = ensure_adam(c, "pg_set_adam_state: cannot allocate the Adam moments");
    if (s != PG_OK) return s;
    const size_t bytes = 6 * hw_of(c) * sizeof(float);
    cudaError_t e;
    if (adam_bf16(c)) {
        e = pgk::launch_adam_rec_set(c->base, d_m, d_v, c->adam_m, c->stream);
    } else {
        e = cudaMemcpyAsync(c->adam_m, d_m, bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->adam_v, d_v, bytes, cudaMemcpyDeviceToDevice, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_set_adam_state");
    return PG_OK;
}

pg_status pg_theta_from_gamma(pg_ctx* c, float* d_theta) {
    if (!c || !d_theta) return fail(c, PG_ERR_ARG, "pg_theta_from_gamma: NULL argument");
    cudaError_t e = pgk::launch_theta_get(c->cfg.gamma_dtype, c->base, c->gam[c->cur], d_theta, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_theta_from_gamma");
    return PG_OK;
}

pg_status pg_theta_to_gamma(pg_ctx* c, const float* d_theta) {
    if (!c || !d_theta) return fail(c, PG_ERR_ARG, "pg_theta_to_gamma: NULL argument");
    if (c->phase != 0) return fail(c, PG_ERR_STATE, "pg_theta_to_gamma: a staged frame is in progress");
    cudaError_t e = pgk::launch_theta_set(c->cfg.gamma_dtype, c->base, c->gam[c->cur], d_theta, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pg_theta_to_gamma");
    return PG_OK;
}

const char* pg_last_error(const pg_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

void pg_destroy(pg_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int b = 0; b < 2; ++b)
        if (c->gam[b]) cudaFree(c->gam[b]);
    if (c->work) cudaFree(c->work);
    if (c->d_err) cudaFree(c->d_err);
    if (c->adam_m) cudaFree(c->adam_m);
    if (c->adam_v) cudaFree(c->adam_v);
    if (c->vpl) cudaFree(c->vpl);
    if (c->vpl_pb) cudaFree(c->vpl_pb);
    if (c->hand) cudaFree(c->hand);
    if (c->hs_up) cudaStreamSynchronize(c->hs_up);
    if (c->hs_down) cudaStreamSynchronize(c->hs_down);
    release_host(c);
    delete c;
}

}  // extern "C"
