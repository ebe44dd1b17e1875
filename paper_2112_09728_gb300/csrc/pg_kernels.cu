// Kernels of the guide pass (Derevyannykh, arXiv 2112.09728, Sec. 3).
//
// k_frame is the hot path: one thread per pixel does reprojection (Sec. 3.1),
// guided sampling with the mixture pdf and MIS (Eq. 2), the analytic radiance
// that stands in for the traced ray, and one weighted online EM step
// (Sec. 3.2), reading Gamma(t-1) and the G-buffer once and writing Gamma(t)
// and the pixel estimate once. Samples never touch memory. The staged kernels
// split the same per-pixel code at the paper's pass boundary (Fig. 2): the
// path-tracing pass writes per-sample records (the VPL texture Pi), the
// training pass reads them back.
#include <curand_kernel.h>

#include "pg_launch.h"

namespace pgk {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ bool same_normal(float4 a, float4 b) {
    return __float_as_uint(a.x) == __float_as_uint(b.x) && __float_as_uint(a.y) == __float_as_uint(b.y) &&
           __float_as_uint(a.z) == __float_as_uint(b.z);
}

__device__ __forceinline__ bool gated(const Params& P, bool reinit, float4 g1) {
    // guiding is off for fresh history (Sec. 3.1), near-mirror GGX and
    // transparent surfaces (Sec. 5)
    return reinit || (g1.z >= 0.0f && g1.z < P.rough_min) || (P.glass && g1.z <= -1.5f);
}

template <int DT>
__global__ void __launch_bounds__(kBlock) k_init(const Params P, void* __restrict__ gam, float init_pi) {
    const size_t hw = (size_t)P.W * P.H;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
    Gam g = init_gam(P);
    g.pi = init_pi;
    Store<DT>::store(gam, hw, i, g);
}

// Reprojection of one pixel: Gamma(t-1) at the motion-compensated pixel, or a
// re-initialised guide. Returns true for a re-initialised pixel.
template <int DT>
__device__ __forceinline__ bool reproject_pixel(const Params& P, int x, int y, float4 a0, float4 a1,
                                                const void* __restrict__ gin, const float4* __restrict__ g0p,
                                                size_t hw, Gam& g) {
    float4 gp;
    const int j = reproject_index(P, x, y, a0, a1, g0p, &gp);
    if (j < 0) {
        g = init_gam(P);
        return true;
    }
    g = Store<DT>::load(gin, hw, (size_t)j);
    if (!same_normal(gp, a0)) change_frame(g, make_float3(gp.x, gp.y, gp.z), make_float3(a0.x, a0.y, a0.z));
    return false;
}

// ONE: one sample per pixel, known at compile time (no sample loop, no Kahan
// compensation state). GLASS: the transparent material compiled in (launched
// when the configuration enables it; without it the kernel carries none of
// its code).
// RGB: a coloured field; the image gets three planes [3][H*W].
template <int DT, bool ONE, bool GLASS, bool RGB>
__global__ void __launch_bounds__(kBlock, 5) k_frame(const Params P, const void* __restrict__ gin,
                                                     void* __restrict__ gout, const float4* __restrict__ g0,
                                                     const float4* __restrict__ g1, const float4* __restrict__ g0p,
                                                     float* __restrict__ img, uint32_t frame, int* __restrict__ err) {
    const size_t hw = (size_t)P.W * P.H;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if ((size_t)i >= hw) return;
    const int y = i / P.W, x = i - y * P.W;
    const float4 a0 = __ldcs(g0 + i), a1 = __ldcs(g1 + i);
    Gam g;
    const bool reinit = reproject_pixel<DT>(P, x, y, a0, a1, gin, g0p, hw, g);
    const Surf s = make_surf<GLASS>(P, x, y, a0, a1);
    const Guide d = derive_guide(P, g, gated(P, reinit, a1));
    Stats st;
    Kahan f, fr, fg, fb;
    const int spp = ONE ? 1 : P.spp;
    for (int si = 0; si < spp; ++si) {
        const Smp o = draw_sample<RGB>(P, d, s, (uint32_t)i, frame, (uint32_t)si);
        if (si == 0) {
            f.set(o.F);
            if (RGB) {
                fr.set(o.wgt * o.Lrgb.x);
                fg.set(o.wgt * o.Lrgb.y);
                fb.set(o.wgt * o.Lrgb.z);
            }
        } else {
            f.add(o.F);
            if (RGB) {
                fr.add(o.wgt * o.Lrgb.x);
                fg.add(o.wgt * o.Lrgb.y);
                fb.add(o.wgt * o.Lrgb.z);
            }
        }
        st.add_train(d, g, o);
    }
    m_step(P, g, st);
    if (!gam_finite(g)) atomicOr(err, 1);
    store_step<DT>(P, gout, hw, (size_t)i, g, frame);
    if (img) {
        if (RGB) {
            __stcs(img + i, ONE ? fr.s : fdiv(fr.s, (float)spp));
            __stcs(img + hw + i, ONE ? fg.s : fdiv(fg.s, (float)spp));
            __stcs(img + 2 * hw + i, ONE ? fb.s : fdiv(fb.s, (float)spp));
        } else {
            __stcs(img + i, ONE ? f.s : fdiv(f.s, (float)spp));
        }
    }
}

// Neighbour-VPL reuse, pass 1 (path tracing, Fig. 2): the frame's samples
// and image as in k_frame, plus one VPL per sample in the buffer Pi: world
// direction and radiance in vpl, and in pb_src the density of the pixel's
// BRDF draw for a BRDF-strategy sample (0 for samples that do not train).
// The guide's rectangle mass Z goes to zbuf for the training pass.
template <int DT, bool ONE, bool RGB>
__global__ void __launch_bounds__(kBlock, 5) k_pt(const Params P, const void* __restrict__ gin,
                                                  const float4* __restrict__ g0, const float4* __restrict__ g1,
                                                  const float4* __restrict__ g0p, float* __restrict__ img,
                                                  uint32_t frame, float4* __restrict__ vpl,
                                                  float* __restrict__ pb_src, float* __restrict__ zbuf) {
    const size_t hw = (size_t)P.W * P.H;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if ((size_t)i >= hw) return;
    const int y = i / P.W, x = i - y * P.W;
    const float4 a0 = __ldcs(g0 + i), a1 = __ldcs(g1 + i);
    Gam g;
    const bool reinit = reproject_pixel<DT>(P, x, y, a0, a1, gin, g0p, hw, g);
    const Surf s = make_surf(P, x, y, a0, a1);
    const Guide d = derive_guide(P, g, gated(P, reinit, a1));
    zbuf[i] = d.Z;
    Kahan f, fr, fg, fb;
    const int spp = ONE ? 1 : P.spp;
    for (int si = 0; si < spp; ++si) {
        const Smp o = draw_sample<RGB>(P, d, s, (uint32_t)i, frame, (uint32_t)si);
        if (si == 0) {
            f.set(o.F);
            if (RGB) {
                fr.set(o.wgt * o.Lrgb.x);
                fg.set(o.wgt * o.Lrgb.y);
                fb.set(o.wgt * o.Lrgb.z);
            }
        } else {
            f.add(o.F);
            if (RGB) {
                fr.add(o.wgt * o.Lrgb.x);
                fg.add(o.wgt * o.Lrgb.y);
                fb.add(o.wgt * o.Lrgb.z);
            }
        }
        const float3 ww = to_world(s.f, o.wl);
        const size_t q = (size_t)si * hw + i;
        vpl[q] = make_float4(ww.x, ww.y, ww.z, o.L);
        pb_src[q] = (o.strat == ST_BRDF && o.pb > 0.0f) ? o.pb : 0.0f;
    }
    if (img) {
        if (RGB) {
            __stcs(img + i, ONE ? fr.s : fdiv(fr.s, (float)spp));
            __stcs(img + hw + i, ONE ? fg.s : fdiv(fg.s, (float)spp));
            __stcs(img + 2 * hw + i, ONE ? fb.s : fdiv(fb.s, (float)spp));
        } else {
            __stcs(img + i, ONE ? f.s : fdiv(f.s, (float)spp));
        }
    }
}

// Neighbour-VPL reuse, pass 2 (training, Sec. 3.2 and 4.2): the pixel's own
// BRDF-strategy VPLs and N picks of its window, each weighted f / p_src, then
// the M-step. N = 5 + floor(15 (k_max - k) / k_max) (at most the window's C
// candidates); the picks walk the candidates from a Philox start by a stride
// coprime with C, so they are distinct. Reprojection is recomputed (same
// inputs, same result as pass 1) rather than stored; Z comes from pass 1.
//
// Each thread walks its own picks to the next one that trains (inside the
// image, drawn by the BRDF strategy) before the warp evaluates a VPL, so a
// warp runs as many evaluations as its busiest lane has training VPLs, not
// one per pick.
template <int DT, bool ONE>
__global__ void __launch_bounds__(kBlock, 4) k_train(const Params P, const void* __restrict__ gin,
                                                     void* __restrict__ gout, const float4* __restrict__ g0,
                                                     const float4* __restrict__ g1,
                                                     const float4* __restrict__ g0p, uint32_t frame,
                                                     const float4* __restrict__ vpl,
                                                     const float* __restrict__ pb_src,
                                                     const float* __restrict__ zbuf, int* __restrict__ err) {
    const size_t hw = (size_t)P.W * P.H;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if ((size_t)i >= hw) return;
    const int y = i / P.W, x = i - y * P.W;
    const float4 a0 = __ldcs(g0 + i), a1 = __ldcs(g1 + i);
    Gam g;
    const bool reinit = reproject_pixel<DT>(P, x, y, a0, a1, gin, g0p, hw, g);
    const Surf s = make_surf(P, x, y, a0, a1);
    Guide d = derive_guide_shape(P, g, gated(P, reinit, a1));
    d.Z = __ldcs(zbuf + i);
    const int spp = ONE ? 1 : P.spp;
    const int kc = (int)fminf(fmaxf(g.k, 0.0f), (float)P.k_max);
    const int n = min(5 + (15 * (P.k_max - kc)) / P.k_max, P.reuse_c);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, frame, 0u, 4u), P.rk);
    int o = (int)(((uint64_t)r.x * (uint64_t)P.reuse_c) >> 32);
    const int dw = 2 * P.reuse_r + 1, center = (dw * dw - 1) / 2;
    int j = -spp;   // own samples first (j < 0), then the picks
    Stats st;
    while (true) {
        // this lane's next VPL that trains
        float pb = 0.0f;
        size_t q = 0;
        while (j < n) {
            if (j < 0) {
                q = (size_t)(j + spp) * hw + i;
            } else {
                // candidate o: pixel cell o / spp of the window (p itself skipped), sample o mod spp;
                // the floor divisions are exact in binary32 for these small integers
                const int cell0 = ONE ? o : (int)(((float)o + 0.5f) * P.reuse_inv_spp);
                const int sj = o - cell0 * spp;
                const int cell = cell0 + (cell0 >= center ? 1 : 0);
                const int ry = (int)(((float)cell + 0.5f) * P.reuse_inv_dw);
                const int qx = x + cell - ry * dw - P.reuse_r, qy = y + ry - P.reuse_r;
                o += P.reuse_stride;
                if (o >= P.reuse_c) o -= P.reuse_c;
                if (qx < 0 || qx >= P.W || qy < 0 || qy >= P.H) {
                    ++j;
                    continue;
                }
                q = (size_t)sj * hw + (size_t)qy * P.W + qx;
            }
            ++j;
            pb = pb_src[q];
            if (pb > 0.0f) break;
        }
        if (!(pb > 0.0f)) break;
        const float4 v = vpl[q];
        st.add_vpl(d, g, s, make_float3(v.x, v.y, v.z), v.w, pb, P.f0);
    }
    m_step(P, g, st);
    if (!gam_finite(g)) atomicOr(err, 1);
    store_step<DT>(P, gout, hw, (size_t)i, g, frame);
}

template <int DT>
__global__ void __launch_bounds__(kBlock) k_reproject(const Params P, const void* __restrict__ gin,
                                                      float4* __restrict__ work, const float4* __restrict__ g0,
                                                      const float4* __restrict__ g1,
                                                      const float4* __restrict__ g0p, uint8_t* __restrict__ accept) {
    const size_t hw = (size_t)P.W * P.H;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if ((size_t)i >= hw) return;
    const int y = i / P.W, x = i - y * P.W;
    const float4 a0 = g0[i], a1 = g1[i];
    Gam g;
    const bool reinit = reproject_pixel<DT>(P, x, y, a0, a1, gin, g0p, hw, g);
    if (reinit) g.k = -1.0f;  // marks "fresh history, BRDF only" for the next stages
    Work<DT>::store(work, hw, (size_t)i, g);
    if (accept) accept[i] = reinit ? 0 : 1;
}

template <int DT>
__global__ void __launch_bounds__(kBlock) k_sample(const Params P, const float4* __restrict__ work,
                                                   const float4* __restrict__ g0, const float4* __restrict__ g1,
                                                   uint32_t frame, SamplePlanes out, float* __restrict__ img) {
    const size_t hw = (size_t)P.W * P.H;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if ((size_t)i >= hw) return;
    const int y = i / P.W, x = i - y * P.W;
    const float4 a0 = g0[i], a1 = g1[i];
    const Gam g = Work<DT>::load(work, hw, (size_t)i);
    const Surf s = make_surf(P, x, y, a0, a1);
    const Guide d = derive_guide(P, g, gated(P, g.k < 0.0f, a1));
    Kahan f, fr, fg, fb;
    for (int si = 0; si < P.spp; ++si) {
        const Smp o = draw_sample<true>(P, d, s, (uint32_t)i, frame, (uint32_t)si);
        f.add(o.F);
        fr.add(o.wgt * o.Lrgb.x);
        fg.add(o.wgt * o.Lrgb.y);
        fb.add(o.wgt * o.Lrgb.z);
        const size_t q = (size_t)si * hw + i;
        if (out.wx) {
            const float3 ww = to_world(s.f, o.wl);
            out.wx[q] = ww.x;
            out.wy[q] = ww.y;
            out.wz[q] = ww.z;
        }
        if (out.radiance) out.radiance[q] = o.L;
        if (out.pdf) out.pdf[q] = o.pmix;
        if (out.mis) out.mis[q] = o.mis;
        if (out.estimate) out.estimate[q] = o.F;
        if (out.strategy) out.strategy[q] = (uint8_t)o.strat;
    }
    if (img) {
        if (P.rgb) {
            img[i] = fdiv(fr.s, (float)P.spp);
            img[hw + i] = fdiv(fg.s, (float)P.spp);
            img[2 * hw + i] = fdiv(fb.s, (float)P.spp);
        } else {
            img[i] = fdiv(f.s, (float)P.spp);
        }
    }
}

// Training pass on given samples (Sec. 3.2): the E-step re-evaluates each
// BRDF draw from the G-buffer and the guide (the paper's training pass reads
// material parameters from the G-buffer and the VPL from Pi).
template <int DT>
__global__ void __launch_bounds__(kBlock) k_update(const Params P, const float4* __restrict__ work,
                                                   const float4* __restrict__ g0, const float4* __restrict__ g1,
                                                   SamplePlanes in, void* __restrict__ gout, int* __restrict__ err) {
    const size_t hw = (size_t)P.W * P.H;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if ((size_t)i >= hw) return;
    const int y = i / P.W, x = i - y * P.W;
    const float4 a0 = g0[i], a1 = g1[i];
    Gam g = Work<DT>::load(work, hw, (size_t)i);
    const Surf s = make_surf(P, x, y, a0, a1);
    const Guide d = derive_guide(P, g, gated(P, g.k < 0.0f, a1));
    Stats st;
    for (int si = 0; si < P.spp; ++si) {
        const size_t q = (size_t)si * hw + i;
        Smp o;
        o.strat = in.strategy[q];
        if (o.strat != ST_BRDF) continue;
        o.wl = to_local(s.f, make_float3(in.wx[q], in.wy[q], in.wz[q]));
        float fr;
        brdf_eval(s, o.wl, fr, o.pb, P.f0);
        if (!(o.pb > 0.0f)) continue;
        o.fcos = in.radiance[q] * fr;
        const float2 u = hemi_to_square(o.wl);
        o.ux = u.x;
        o.uy = u.y;
        o.pg = guide_pdf(d, o.ux, o.uy);
        o.pmix = d.pi_eff * o.pg + (1.0f - d.pi_eff * d.Z) * o.pb;
        st.add_train(d, g, o);
    }
    m_step(P, g, st);
    if (!gam_finite(g)) atomicOr(err, 1);
    store_step<DT>(P, gout, hw, (size_t)i, g, P.sr_frame);
}

template <int DT, bool WORK>
__device__ __forceinline__ Gam load_any(const void* src, size_t hw, size_t i) {
    if (WORK) return Work<DT>::load(reinterpret_cast<const float4*>(src), hw, i);
    Gam g = Store<DT>::load(src, hw, i);
    return g;
}

template <int DT, bool WORK>
__global__ void __launch_bounds__(kBlock) k_eval(const Params P, const void* __restrict__ src,
                                                 const float4* __restrict__ g0, const float4* __restrict__ g1,
                                                 int n_dirs, const float* __restrict__ dirs, float* __restrict__ out) {
    const size_t hw = (size_t)P.W * P.H;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if ((size_t)i >= hw) return;
    const int y = i / P.W, x = i - y * P.W;
    const float4 a0 = g0[i], a1 = g1[i];
    const Gam g = load_any<DT, WORK>(src, hw, (size_t)i);
    const Surf s = make_surf(P, x, y, a0, a1);
    const Guide d = derive_guide(P, g, gated(P, WORK && g.k < 0.0f, a1));
    const size_t tot = (size_t)n_dirs * hw;
    for (int si = 0; si < n_dirs; ++si) {
        const size_t q = (size_t)si * hw + i;
        const float3 ww = make_float3(dirs[3 * q], dirs[3 * q + 1], dirs[3 * q + 2]);
        const float3 wl = to_local(s.f, ww);
        const float L = radiance(P, s.pos, ww);
        float fr, pb, pg = 0.0f;
        brdf_eval(s, wl, fr, pb, P.f0);
        if (wl.z > 0.0f) {
            const float2 u = hemi_to_square(wl);
            pg = guide_pdf(d, u.x, u.y);
        }
        const float wgs = d.pi_eff * pg, wbs = (1.0f - d.pi_eff * d.Z) * pb;
        const float pmix = wgs + wbs;
        out[0 * tot + q] = pg;
        out[1 * tot + q] = pb;
        out[2 * tot + q] = pmix;
        out[3 * tot + q] = pmix > 0.0f ? wgs / pmix : 0.0f;
        out[4 * tot + q] = pmix > 0.0f ? wbs / pmix : 0.0f;
        out[5 * tot + q] = L * fr;
        out[6 * tot + q] = L;
    }
}

template <int DT, bool WORK>
__global__ void __launch_bounds__(kBlock) k_to_f32(const Params P, const void* __restrict__ src,
                                                   float4* __restrict__ dst) {
    const size_t hw = (size_t)P.W * P.H;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
    const Gam g = load_any<DT, WORK>(src, hw, i);
    dst[i] = make_float4(g.ex, g.ey, g.exx, g.eyy);
    dst[hw + i] = make_float4(g.exy, g.pi, g.k, g.W);
}

template <int DT>
__global__ void __launch_bounds__(kBlock) k_from_f32(const Params P, const float4* __restrict__ src,
                                                     void* __restrict__ dst) {
    const size_t hw = (size_t)P.W * P.H;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
    const float4 a = src[i], b = src[hw + i];
    Gam g;
    g.ex = a.x; g.ey = a.y; g.exx = a.z; g.eyy = a.w;
    g.exy = b.x; g.pi = b.y; g.k = b.z; g.W = b.w;
    central_from_raw(g);
    Store<DT>::store(dst, hw, i, g);
}

__global__ void __launch_bounds__(kBlock) k_philox(const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1,
                                                   int64_t n, uint4* __restrict__ out, bool use_curand) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (use_curand) {
        out[i] = curand_Philox4x32_10(ctr[i], make_uint2(k0, k1));
    } else {
        out[i] = philox4x32_10(ctr[i], k0, k1);
    }
}

// ---------------------------------------------------------------------------
// The differentiable form: the gradient of the per-pixel second-moment loss
// l(theta) = 1/n sum f_i^2 / (p_theta(w_i) p_theta0(w_i)) at theta = theta0,
// with the n directions drawn from the guide itself (Philox streams 2 and 3):
//   l = 1/n sum f^2 / p^2,  dl/dtheta = -1/n sum f^2 (dp/dtheta) / p^3,
//   dp/dpi = g - Z p_b,  dp/dmu = pi (g Sigma^-1 d - p_b dZ/dmu),
//   dp/dSigma = pi (g/2 (Sigma^-1 d d^T Sigma^-1 - Sigma^-1) - p_b dZ/dSigma)
// for theta = (mu_x, mu_y, s_xx, s_yy, s_xy, pi), s_xy a single parameter.
// ---------------------------------------------------------------------------
template <int DT, bool THETA>
__global__ void __launch_bounds__(kBlock) k_grad(const Params P, const void* __restrict__ gam,
                                                 const float* __restrict__ theta, const float4* __restrict__ g0,
                                                 const float4* __restrict__ g1, uint32_t frame, int n,
                                                 float* __restrict__ loss, float* __restrict__ grad) {
    const size_t hw = (size_t)P.W * P.H;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if ((size_t)i >= hw) return;
    const int y = i / P.W, x = i - y * P.W;
    const float4 a0 = g0[i], a1 = g1[i];
    Gam g;
    if (THETA) {
        g.ex = theta[i]; g.ey = theta[hw + i];
        g.sxx = theta[2 * hw + i]; g.syy = theta[3 * hw + i]; g.sxy = theta[4 * hw + i];
        g.pi = theta[5 * hw + i]; g.k = 0.0f; g.W = 0.0f;
    } else {
        g = Store<DT>::load(gam, hw, (size_t)i);
    }
    const Surf s = make_surf(P, x, y, a0, a1);
    const Guide d = derive_guide(P, g, gated(P, false, a1));
    float dz[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    const bool guided = d.pi_eff > 0.0f;
    if (guided) rect_mass_grad(d, dz);
    const float det = fmaf(d.sxx, d.syy, -d.sxy * d.sxy), idet = fdiv(1.0f, det);
    Kahan l, gs[6];
    for (int si = 0; si < n; ++si) {
        const Smp o = draw_sample(P, d, s, (uint32_t)i, frame, (uint32_t)si, 2u);
        if ((o.strat & ST_INVALID) || o.fcos == 0.0f || !(o.pmix > 0.0f)) continue;
        const float ip = fdiv(1.0f, o.pmix), f2 = o.fcos * o.fcos;
        l.add(f2 * ip * ip);
        if (!guided) continue;
        const float dx = o.ux - d.mx, dy = o.uy - d.my;
        const float ix = (d.syy * dx - d.sxy * dy) * idet, iy = (d.sxx * dy - d.sxy * dx) * idet;
        const float c = -f2 * ip * ip * ip, pe = d.pi_eff;
        gs[0].add(c * pe * (o.pg * ix - o.pb * dz[0]));
        gs[1].add(c * pe * (o.pg * iy - o.pb * dz[1]));
        gs[2].add(c * pe * (o.pg * 0.5f * (ix * ix - d.syy * idet) - o.pb * dz[2]));
        gs[3].add(c * pe * (o.pg * 0.5f * (iy * iy - d.sxx * idet) - o.pb * dz[3]));
        gs[4].add(c * pe * (o.pg * (ix * iy + d.sxy * idet) - o.pb * dz[4]));
        gs[5].add(c * (o.pg - d.Z * o.pb));
    }
    const float in = 1.0f / (float)n;
    loss[i] = l.s * in;
#pragma unroll
    for (int k = 0; k < 6; ++k) grad[k * hw + i] = gs[k].s * in;
}

// Regularised guide parameters theta = (mu_x, mu_y, s_xx, s_yy, s_xy) and the
// stored pi of a Gamma pixel.
__device__ __forceinline__ void theta_of(const Params& P, const Gam& g, float th[6]) {
    th[0] = fminf(fmaxf(g.ex, 0.0f), 1.0f);
    th[1] = fminf(fmaxf(g.ey, 0.0f), 1.0f);
    th[2] = fmaxf(g.sxx, P.sigma2_min);
    th[3] = fmaxf(g.syy, P.sigma2_min);
    const float lim = P.rho_max * sqrtf(th[2] * th[3]);
    th[4] = fminf(fmaxf(g.sxy, -lim), lim);
    th[5] = g.pi;
}

// theta projected onto the guide's domain and written into Gamma as moments
// (k and W are kept).
__device__ __forceinline__ void set_theta(const Params& P, Gam& g, const float th[6]) {
    g.ex = fminf(fmaxf(th[0], 0.0f), 1.0f);
    g.ey = fminf(fmaxf(th[1], 0.0f), 1.0f);
    g.sxx = fmaxf(th[2], P.sigma2_min);
    g.syy = fmaxf(th[3], P.sigma2_min);
    const float lim = P.rho_max * sqrtf(g.sxx * g.syy);
    g.sxy = fminf(fmaxf(th[4], -lim), lim);
    g.pi = fminf(fmaxf(th[5], P.pi_min), P.pi_max);
    raw_from_central(g);
}

// One Adam step (Kingma & Ba 2015) on theta with projection; c1, c2 are the
// bias corrections 1/(1 - b1^t), 1/(1 - b2^t) of step t.
// One projected Adam step on theta of a pixel from its gradient and the old
// moments (binary32 arithmetic); returns the new moments in mk, vk.
template <int DT>
__device__ __forceinline__ void adam_pixel(const Params& P, void* gam, size_t hw, size_t i, const float gk[6],
                                           const float mo[6], const float vo[6], float mk[6], float vk[6], float lr,
                                           float b1, float b2, float eps, float c1, float c2) {
    Gam g = Store<DT>::load(gam, hw, i);
    float th[6];
    theta_of(P, g, th);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        mk[k] = fmaf(b1, mo[k], (1.0f - b1) * gk[k]);
        vk[k] = fmaf(b2, vo[k], (1.0f - b2) * gk[k] * gk[k]);
        th[k] -= lr * fdiv(mk[k] * c1, sqrtf(vk[k] * c2) + eps);
    }
    set_theta(P, g, th);
    Store<DT>::store(gam, hw, i, g);
}

// Binary32 moments: [6][H*W] planes each, one pixel per thread.
template <int DT>
__global__ void __launch_bounds__(kBlock) k_adam(const Params P, void* __restrict__ gam,
                                                 const float* __restrict__ grad, float* __restrict__ m,
                                                 float* __restrict__ v, float lr, float b1, float b2, float eps,
                                                 float c1, float c2) {
    const size_t hw = (size_t)P.W * P.H;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
    Gam g = Store<DT>::load(gam, hw, i);
    float th[6];
    theta_of(P, g, th);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const size_t q = k * hw + i;
        const float gk = grad[q];
        const float mk = fmaf(b1, m[q], (1.0f - b1) * gk);
        const float vk = fmaf(b2, v[q], (1.0f - b2) * gk * gk);
        m[q] = mk;
        v[q] = vk;
        th[k] -= lr * fdiv(mk * c1, sqrtf(vk * c2) + eps);
    }
    set_theta(P, g, th);
    Store<DT>::store(gam, hw, i, g);
}

// BF16 moments: one 24-byte record per pixel {m_0..m_5, v_0..v_5} (three
// 8-byte words), read and written whole; each moment is stored stochastically
// with 16 bits of the Philox calls at (pixel, step, 0, 6) and (pixel, step, 1, 6)
// (moment n: word n/2, bits 16 (n mod 2) and up). A thread steps two pixels,
// i and i + ceil(H*W / 2), for more loads in flight.
template <int DT>
__device__ __forceinline__ void adam_pixel_bf16(const Params& P, void* gam, const float* grad, uint2* rec,
                                                size_t hw, size_t i, float lr, float b1, float b2, float eps,
                                                float c1, float c2, uint32_t step) {
    const uint2 r0 = rec[3 * i], r1 = rec[3 * i + 1], r2 = rec[3 * i + 2];
    const uint32_t w[6] = {r0.x, r0.y, r1.x, r1.y, r2.x, r2.y};
    float gk[6], mo[6], vo[6], mk[6], vk[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        gk[k] = grad[k * hw + i];
        mo[k] = __uint_as_float((w[k >> 1] >> (16 * (k & 1))) << 16);
        vo[k] = __uint_as_float((w[(k + 6) >> 1] >> (16 * (k & 1))) << 16);
    }
    adam_pixel<DT>(P, gam, hw, i, gk, mo, vo, mk, vk, lr, b1, b2, eps, c1, c2);
    const uint4 ra = philox4x32_10(make_uint4((uint32_t)i, step, 0u, 6u), P.rk);
    const uint4 rb = philox4x32_10(make_uint4((uint32_t)i, step, 1u, 6u), P.rk);
    const uint32_t rw[6] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y};
    uint32_t o[12];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        o[k] = sr_pack_bf16(mk[k], rw[k >> 1] >> (16 * (k & 1)));
        o[k + 6] = sr_pack_bf16(vk[k], rw[(k + 6) >> 1] >> (16 * (k & 1)));
    }
    rec[3 * i] = make_uint2(o[0] | (o[1] << 16), o[2] | (o[3] << 16));
    rec[3 * i + 1] = make_uint2(o[4] | (o[5] << 16), o[6] | (o[7] << 16));
    rec[3 * i + 2] = make_uint2(o[8] | (o[9] << 16), o[10] | (o[11] << 16));
}

template <int DT>
__global__ void __launch_bounds__(kBlock) k_adam_bf16(const Params P, void* __restrict__ gam,
                                                      const float* __restrict__ grad, uint2* __restrict__ rec,
                                                      float lr, float b1, float b2, float eps, float c1, float c2,
                                                      uint32_t step) {
    const size_t hw = (size_t)P.W * P.H, half = (hw + 1) / 2;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= half) return;
    adam_pixel_bf16<DT>(P, gam, grad, rec, hw, i, lr, b1, b2, eps, c1, c2, step);
    if (i + half < hw) adam_pixel_bf16<DT>(P, gam, grad, rec, hw, i + half, lr, b1, b2, eps, c1, c2, step);
}

// BF16 moment records <-> binary32 [6][H*W] planes (checkpoint and resume;
// the planes are rounded to nearest).
__global__ void k_adam_rec_get(const uint16_t* __restrict__ rec, float* __restrict__ m, float* __restrict__ v,
                               size_t hw) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        m[k * hw + i] = __uint_as_float((uint32_t)rec[12 * i + k] << 16);
        v[k * hw + i] = __uint_as_float((uint32_t)rec[12 * i + 6 + k] << 16);
    }
}

__global__ void k_adam_rec_set(const float* __restrict__ m, const float* __restrict__ v, uint16_t* __restrict__ rec,
                               size_t hw) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        rec[12 * i + k] = __bfloat16_as_ushort(__float2bfloat16_rn(m[k * hw + i]));
        rec[12 * i + 6 + k] = __bfloat16_as_ushort(__float2bfloat16_rn(v[k * hw + i]));
    }
}

template <int DT>
__global__ void __launch_bounds__(kBlock) k_theta_get(const Params P, const void* __restrict__ gam,
                                                      float* __restrict__ theta) {
    const size_t hw = (size_t)P.W * P.H;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
    const Gam g = Store<DT>::load(gam, hw, i);
    float th[6];
    theta_of(P, g, th);
#pragma unroll
    for (int k = 0; k < 6; ++k) theta[k * hw + i] = th[k];
}

template <int DT>
__global__ void __launch_bounds__(kBlock) k_theta_set(const Params P, void* __restrict__ gam,
                                                      const float* __restrict__ theta) {
    const size_t hw = (size_t)P.W * P.H;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
    Gam g = Store<DT>::load(gam, hw, i);
    float th[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) th[k] = theta[k * hw + i];
    set_theta(P, g, th);
    Store<DT>::store(gam, hw, i, g);
}

inline dim3 grid_for(const Params& P) {
    const size_t hw = (size_t)P.W * P.H;
    return dim3((unsigned)((hw + kBlock - 1) / kBlock));
}

}  // namespace

#define PG_DISPATCH(dt, CALL)                 \
    switch (dt) {                             \
        case DT_F32: { constexpr int D = DT_F32; CALL; break; }   \
        case DT_F16: { constexpr int D = DT_F16; CALL; break; }   \
        default: { constexpr int D = DT_BF16; CALL; break; }      \
    }

cudaError_t launch_init(int dt, const Params& P, void* gam, float init_pi, cudaStream_t st) {
    PG_DISPATCH(dt, (k_init<D><<<grid_for(P), kBlock, 0, st>>>(P, gam, init_pi)));
    return cudaGetLastError();
}

cudaError_t launch_frame(int dt, const Params& P, const void* gin, void* gout, const float4* g0,
                         const float4* g1, const float4* g0p, float* img, uint32_t frame, int* err,
                         cudaStream_t st) {
    const dim3 grid = grid_for(P);
#define PG_FRAME(ONE, GLASS, RGB) \
    PG_DISPATCH(dt, (k_frame<D, ONE, GLASS, RGB><<<grid, kBlock, 0, st>>>(P, gin, gout, g0, g1, g0p, img, frame, err)))
    const int v = (P.spp == 1 ? 4 : 0) + (P.glass ? 2 : 0) + (P.rgb ? 1 : 0);
    switch (v) {
        case 0: PG_FRAME(false, false, false); break;
        case 1: PG_FRAME(false, false, true); break;
        case 2: PG_FRAME(false, true, false); break;
        case 3: PG_FRAME(false, true, true); break;
        case 4: PG_FRAME(true, false, false); break;
        case 5: PG_FRAME(true, false, true); break;
        case 6: PG_FRAME(true, true, false); break;
        default: PG_FRAME(true, true, true); break;
    }
#undef PG_FRAME
    return cudaGetLastError();
}

cudaError_t launch_pt(int dt, const Params& P, const void* gin, const float4* g0, const float4* g1,
                      const float4* g0p, float* img, uint32_t frame, float4* vpl, float* pb_src, float* zbuf,
                      cudaStream_t st) {
    const dim3 grid = grid_for(P);
#define PG_PT(ONE, RGB) \
    PG_DISPATCH(dt, (k_pt<D, ONE, RGB><<<grid, kBlock, 0, st>>>(P, gin, g0, g1, g0p, img, frame, vpl, pb_src, zbuf)))
    if (P.spp == 1 && P.rgb) {
        PG_PT(true, true);
    } else if (P.spp == 1) {
        PG_PT(true, false);
    } else if (P.rgb) {
        PG_PT(false, true);
    } else {
        PG_PT(false, false);
    }
#undef PG_PT
    return cudaGetLastError();
}

cudaError_t launch_train(int dt, const Params& P, const void* gin, void* gout, const float4* g0, const float4* g1,
                         const float4* g0p, uint32_t frame, const float4* vpl, const float* pb_src, const float* zbuf,
                         int* err, cudaStream_t st) {
    if (P.spp == 1) {
        PG_DISPATCH(dt, (k_train<D, true><<<grid_for(P), kBlock, 0, st>>>(P, gin, gout, g0, g1, g0p, frame, vpl,
                                                                          pb_src, zbuf, err)));
    } else {
        PG_DISPATCH(dt, (k_train<D, false><<<grid_for(P), kBlock, 0, st>>>(P, gin, gout, g0, g1, g0p, frame, vpl,
                                                                           pb_src, zbuf, err)));
    }
    return cudaGetLastError();
}

cudaError_t launch_reproject(int dt, const Params& P, const void* gin, float4* work, const float4* g0,
                             const float4* g1, const float4* g0p, uint8_t* accept, cudaStream_t st) {
    PG_DISPATCH(dt, (k_reproject<D><<<grid_for(P), kBlock, 0, st>>>(P, gin, work, g0, g1, g0p, accept)));
    return cudaGetLastError();
}

cudaError_t launch_sample(int dt, const Params& P, const float4* work, const float4* g0, const float4* g1,
                          uint32_t frame, SamplePlanes out, float* img, cudaStream_t st) {
    PG_DISPATCH(dt, (k_sample<D><<<grid_for(P), kBlock, 0, st>>>(P, work, g0, g1, frame, out, img)));
    return cudaGetLastError();
}

cudaError_t launch_update(int dt, const Params& P, const float4* work, const float4* g0, const float4* g1,
                          SamplePlanes in, void* gout, int* err, cudaStream_t st) {
    PG_DISPATCH(dt, (k_update<D><<<grid_for(P), kBlock, 0, st>>>(P, work, g0, g1, in, gout, err)));
    return cudaGetLastError();
}

cudaError_t launch_eval(int dt, const Params& P, const void* src, bool src_is_work, const float4* g0,
                        const float4* g1, int n_dirs, const float* dirs, float* out, cudaStream_t st) {
    if (src_is_work) {
        PG_DISPATCH(dt, (k_eval<D, true><<<grid_for(P), kBlock, 0, st>>>(P, src, g0, g1, n_dirs, dirs, out)));
    } else {
        PG_DISPATCH(dt, (k_eval<D, false><<<grid_for(P), kBlock, 0, st>>>(P, src, g0, g1, n_dirs, dirs, out)));
    }
    return cudaGetLastError();
}

cudaError_t launch_to_f32(int dt, const Params& P, const void* src, bool src_is_work, float4* dst,
                          cudaStream_t st) {
    if (src_is_work) {
        PG_DISPATCH(dt, (k_to_f32<D, true><<<grid_for(P), kBlock, 0, st>>>(P, src, dst)));
    } else {
        PG_DISPATCH(dt, (k_to_f32<D, false><<<grid_for(P), kBlock, 0, st>>>(P, src, dst)));
    }
    return cudaGetLastError();
}

cudaError_t launch_from_f32(int dt, const Params& P, const float4* src, void* dst, cudaStream_t st) {
    PG_DISPATCH(dt, (k_from_f32<D><<<grid_for(P), kBlock, 0, st>>>(P, src, dst)));
    return cudaGetLastError();
}

cudaError_t launch_grad(int dt, const Params& P, const void* gam, const float* theta, const float4* g0,
                        const float4* g1, uint32_t frame, int n, float* loss, float* grad, cudaStream_t st) {
    if (theta) {
        PG_DISPATCH(dt, (k_grad<D, true><<<grid_for(P), kBlock, 0, st>>>(P, gam, theta, g0, g1, frame, n, loss, grad)));
    } else {
        PG_DISPATCH(dt, (k_grad<D, false><<<grid_for(P), kBlock, 0, st>>>(P, gam, theta, g0, g1, frame, n, loss, grad)));
    }
    return cudaGetLastError();
}

cudaError_t launch_adam(int dt, const Params& P, void* gam, const float* grad, float* m, float* v, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t st) {
    PG_DISPATCH(dt, (k_adam<D><<<grid_for(P), kBlock, 0, st>>>(P, gam, grad, m, v, lr, b1, b2, eps, c1, c2)));
    return cudaGetLastError();
}

cudaError_t launch_adam_bf16(int dt, const Params& P, void* gam, const float* grad, void* rec, float lr, float b1,
                             float b2, float eps, float c1, float c2, uint32_t step, cudaStream_t st) {
    const size_t half = ((size_t)P.W * P.H + 1) / 2;
    const dim3 grid((unsigned)((half + kBlock - 1) / kBlock));
    PG_DISPATCH(dt, (k_adam_bf16<D><<<grid, kBlock, 0, st>>>(P, gam, grad, reinterpret_cast<uint2*>(rec), lr, b1, b2,
                                                              eps, c1, c2, step)));
    return cudaGetLastError();
}

cudaError_t launch_adam_rec_get(const Params& P, const void* rec, float* m, float* v, cudaStream_t st) {
    k_adam_rec_get<<<grid_for(P), kBlock, 0, st>>>(reinterpret_cast<const uint16_t*>(rec), m, v,
                                                     (size_t)P.W * P.H);
    return cudaGetLastError();
}

cudaError_t launch_adam_rec_set(const Params& P, const float* m, const float* v, void* rec, cudaStream_t st) {
    k_adam_rec_set<<<grid_for(P), kBlock, 0, st>>>(m, v, reinterpret_cast<uint16_t*>(rec), (size_t)P.W * P.H);
    return cudaGetLastError();
}

cudaError_t launch_theta_get(int dt, const Params& P, const void* gam, float* theta, cudaStream_t st) {
    PG_DISPATCH(dt, (k_theta_get<D><<<grid_for(P), kBlock, 0, st>>>(P, gam, theta)));
    return cudaGetLastError();
}

cudaError_t launch_theta_set(int dt, const Params& P, void* gam, const float* theta, cudaStream_t st) {
    PG_DISPATCH(dt, (k_theta_set<D><<<grid_for(P), kBlock, 0, st>>>(P, gam, theta)));
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out, bool curand,
                          cudaStream_t st) {
    const unsigned blocks = (unsigned)((n + kBlock - 1) / kBlock);
    k_philox<<<blocks, kBlock, 0, st>>>(reinterpret_cast<const uint4*>(ctr), k0, k1, n, reinterpret_cast<uint4*>(out),
                                        curand);
    return cudaGetLastError();
}

}  // namespace pgk
