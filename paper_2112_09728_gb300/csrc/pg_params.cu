// Host-side construction and validation of the launch parameters.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "pg_params.h"

namespace pgk {

namespace {

// The rule of Z's corner integrals on [0, rho] in s = sin t (nodes rho c,
// weights rho w), six nodes fitted to the integrands the kernels evaluate by
// fit_corner_rule.py, whose output these are.
constexpr float kZRuleC[kZNodes] = {6.453754298e-02f, 2.967437484e-01f, 5.753261929e-01f,
                                    7.920209216e-01f, 9.232052864e-01f, 9.863174196e-01f};
constexpr float kZRuleW[kZNodes] = {1.604145295e-01f, 2.797993463e-01f, 2.581585785e-01f,
                                    1.724387613e-01f, 9.353107058e-02f, 3.565772626e-02f};

}  // namespace

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

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
    if (c->reuse_radius < 0 || c->reuse_radius > 8) { why = "reuse_radius outside [0, 8]"; return PG_ERR_ARG; }
    if (c->reuse_radius > 0 && c->k_max < 1) { why = "neighbour reuse needs k_max >= 1"; return PG_ERR_ARG; }
    if (c->stochastic_round != 0 && c->stochastic_round != 1) { why = "stochastic_round must be 0 or 1"; return PG_ERR_ARG; }
    if (!(c->ggx_f0 >= 0.0f && c->ggx_f0 <= 1.0f)) { why = "ggx_f0 outside [0, 1]"; return PG_ERR_ARG; }
    if (c->transparent != 0 && c->transparent != 1) { why = "transparent must be 0 or 1"; return PG_ERR_ARG; }
    if (c->adam_dtype != PG_F32 && c->adam_dtype != PG_BF16) {
        why = "adam_dtype must be PG_F32 or PG_BF16";
        return PG_ERR_ARG;
    }
    return PG_OK;
}

void config_params(const pg_config& cfg, Params& P) {
    std::memset(&P, 0, sizeof P);
    P.W = cfg.width;
    P.H = cfg.height;
    P.spp = cfg.spp;
    P.k_max = cfg.k_max;
    P.key0 = (uint32_t)(cfg.seed & 0xffffffffu);
    P.key1 = (uint32_t)(cfg.seed >> 32);
    for (int r = 0; r < 10; ++r) {          // Philox4x32-10 round keys (Weyl increments)
        P.rk[2 * r] = P.key0 + (uint32_t)r * 0x9E3779B9u;
        P.rk[2 * r + 1] = P.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    P.pi_min = cfg.pi_min;
    P.pi_max = cfg.pi_max;
    P.pi_reinit = cfg.pi_reinit;
    P.depth_tol = cfg.depth_tol;
    P.normal_tol = cfg.normal_tol;
    P.rough_min = cfg.rough_min;
    P.sigma2_min = cfg.sigma2_min;
    P.rho_max = cfg.rho_max;
    const double mx = cfg.init_mu[0], my = cfg.init_mu[1];
    P.init_raw[0] = (float)mx;
    P.init_raw[1] = (float)my;
    P.init_raw[2] = (float)(cfg.init_sigma[0] + mx * mx);
    P.init_raw[3] = (float)(cfg.init_sigma[1] + my * my);
    P.init_raw[4] = (float)(cfg.init_sigma[2] + mx * my);
    P.init_c[0] = cfg.init_sigma[0];
    P.init_c[1] = cfg.init_sigma[1];
    P.init_c[2] = cfg.init_sigma[2];
    for (int i = 0; i < kZNodes; ++i) {
        P.zq_c[i] = kZRuleC[i];
        P.zq_w[i] = kZRuleW[i];
    }
    // neighbour reuse: C candidates, walked with the smallest stride >= 0.618 C
    // that is coprime with C (so N <= C picks are distinct)
    P.sr = cfg.stochastic_round;
    P.f0 = cfg.ggx_f0;
    P.glass = cfg.transparent;
    P.reuse_r = cfg.reuse_radius;
    if (cfg.reuse_radius > 0) {
        const int d = 2 * cfg.reuse_radius + 1;
        const int64_t c = (int64_t)(d * d - 1) * cfg.spp;
        int64_t t = (618 * c + 999) / 1000;
        if (t < 1) t = 1;
        auto gcd = [](int64_t a, int64_t b) { while (b) { const int64_t r = a % b; a = b; b = r; } return a; };
        while (gcd(t, c) != 1) ++t;
        P.reuse_c = (int)c;
        P.reuse_stride = (int)t;
        P.reuse_inv_spp = 1.0f / (float)cfg.spp;
        P.reuse_inv_dw = 1.0f / (float)d;
    }
}

pg_status camera_params(const pg_camera& cam, Params& P, std::string& why) {
    if (cam.kind != 0 && cam.kind != 1) {
        why = "camera kind must be 0 or 1";
        return PG_ERR_ARG;
    }
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

pg_status field_params(const pg_field* f, Params& P, std::string& why) {
    if (!f) { why = "field is NULL"; return PG_ERR_ARG; }
    if (f->n_lobes < 0 || f->n_lobes > 8) { why = "n_lobes outside [0, 8]"; return PG_ERR_ARG; }
    if (f->mask_kind != 0 && f->mask_kind != 1) { why = "mask_kind must be 0 or 1"; return PG_ERR_ARG; }
    if (f->rgb != 0 && f->rgb != 1) { why = "rgb must be 0 or 1"; return PG_ERR_ARG; }
    // Rec. 709 luminance of a colour
    auto lum = [](const float* c) { return 0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2]; };
    P.n_lobes = f->n_lobes;
    P.rgb = f->rgb;
    for (int j = 0; j < 8; ++j) {
        for (int k = 0; k < 3; ++k) P.lobe_dir[j][k] = j < f->n_lobes ? f->dir[j][k] : 0.0f;
        if (j < f->n_lobes) {
            const double kap = f->kappa[j];
            if (!(kap > 0.0) || !std::isfinite(kap)) { why = "lobe kappa must be > 0"; return PG_ERR_ARG; }
            // normalised vMF on the sphere: kappa / (2 pi (1 - exp(-2 kappa)))
            const double norm = kap / (2.0 * M_PI * -std::expm1(-2.0 * kap));
            P.lobe_kappa[j] = (float)kap;
            P.lobe_scale[j] = (float)((f->rgb ? lum(f->amp_rgb[j]) : (double)f->amp[j]) * norm);
            for (int c = 0; c < 3; ++c) P.lobe_rgb[j][c] = f->rgb ? (float)((double)f->amp_rgb[j][c] * norm) : 0.0f;
            P.lobe_e2[j] = (float)(-0.5 * kap / std::log(2.0));
        } else {
            P.lobe_kappa[j] = 0.0f;
            P.lobe_scale[j] = 0.0f;
            P.lobe_e2[j] = 0.0f;
            for (int c = 0; c < 3; ++c) P.lobe_rgb[j][c] = 0.0f;
        }
    }
    for (int jp = 0; jp < 4; ++jp) {
        const int a = 2 * jp, b = 2 * jp + 1;
        P.lobe_pnx[jp] = make_float2(-P.lobe_dir[a][0], -P.lobe_dir[b][0]);
        P.lobe_pny[jp] = make_float2(-P.lobe_dir[a][1], -P.lobe_dir[b][1]);
        P.lobe_pnz[jp] = make_float2(-P.lobe_dir[a][2], -P.lobe_dir[b][2]);
        P.lobe_pe2[jp] = make_float2(P.lobe_e2[a], P.lobe_e2[b]);
    }
    P.field_const = f->rgb ? (float)lum(f->constant_rgb) : f->constant;
    for (int c = 0; c < 3; ++c) P.field_const_rgb[c] = f->rgb ? f->constant_rgb[c] : 0.0f;
    P.mask_kind = f->mask_kind;
    for (int k = 0; k < 3; ++k) P.mask[k] = f->mask[k];
    return PG_OK;
}

}  // namespace pgk
