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

#include "pg_common.cuh"

namespace pgk {

namespace {

template <int DT>
__global__ void __launch_bounds__(kBlock) k_init(const Params P, void* __restrict__ gam, float init_pi) {
    const size_t hw = (size_t)P.W * P.H;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hw) return;
    Gam g = init_gam(P);
    g.pi = init_pi;
    Store<DT>::store(gam, hw, i, g);
}

// ONE: one sample per pixel, known at compile time (no sample loop, no Kahan
// compensation state). GLASS: the transparent material compiled in (launched
// when the configuration enables it; without it the kernel carries none of
// its code).
// RGB: a coloured field; the image gets three planes [3][H*W].
template <int DT, bool ONE, bool GLASS, bool RGB>
__global__ void __launch_bounds__(kFrameBlock, ONE ? 10 : 8) k_frame(const Params P, const void* __restrict__ gin,
                                                     void* __restrict__ gout, const float4* __restrict__ g0,
                                                     const float4* __restrict__ g1, const float4* __restrict__ g0p,
                                                     float* __restrict__ img, uint32_t frame, int* __restrict__ err) {
    const size_t hw = (size_t)P.W * P.H;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if ((size_t)i >= hw) return;
    const int y = i / P.W, x = i - y * P.W;
    const float4 a0 = __ldcs(g0 + i), a1 = __ldcs(g1 + i);
    Gam g;
    const bool reinit = reproject_pixel<DT>(P, x, y, a0, a1, gin, g0p, hw, g, err);
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
    m_step<ONE>(P, g, st);
    if (!gam_finite(g)) atomicOr(err, PG_ERR_BIT_NUMERIC);
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

template <int DT>
__global__ void __launch_bounds__(kBlock) k_reproject(const Params P, const void* __restrict__ gin,
                                                      float4* __restrict__ work, const float4* __restrict__ g0,
                                                      const float4* __restrict__ g1,
                                                      const float4* __restrict__ g0p, uint8_t* __restrict__ accept,
                                                      int* __restrict__ err) {
    const size_t hw = (size_t)P.W * P.H;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if ((size_t)i >= hw) return;
    const int y = i / P.W, x = i - y * P.W;
    const float4 a0 = g0[i], a1 = g1[i];
    Gam g;
    const bool reinit = reproject_pixel<DT>(P, x, y, a0, a1, gin, g0p, hw, g, err);
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
    if (!gam_finite(g)) atomicOr(err, PG_ERR_BIT_NUMERIC);
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

}  // namespace

cudaError_t launch_init(int dt, const Params& P, void* gam, float init_pi, cudaStream_t st) {
    PG_DISPATCH(dt, (k_init<D><<<grid_for(P), kBlock, 0, st>>>(P, gam, init_pi)));
    return cudaGetLastError();
}

cudaError_t launch_frame(int dt, const Params& P, const void* gin, void* gout, const float4* g0,
                         const float4* g1, const float4* g0p, float* img, uint32_t frame, int* err,
                         cudaStream_t st) {
    const dim3 grid = grid_for(P, kFrameBlock);
#define PG_FRAME(ONE, GLASS, RGB) \
    PG_DISPATCH(dt, (k_frame<D, ONE, GLASS, RGB><<<grid, kFrameBlock, 0, st>>>(P, gin, gout, g0, g1, g0p, img, frame, \
                                                                                 err)))
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

cudaError_t launch_reproject(int dt, const Params& P, const void* gin, float4* work, const float4* g0,
                             const float4* g1, const float4* g0p, uint8_t* accept, int* err, cudaStream_t st) {
    PG_DISPATCH(dt, (k_reproject<D><<<grid_for(P), kBlock, 0, st>>>(P, gin, work, g0, g1, g0p, accept, err)));
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

cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out, bool curand,
                          cudaStream_t st) {
    const unsigned blocks = (unsigned)((n + kBlock - 1) / kBlock);
    k_philox<<<blocks, kBlock, 0, st>>>(reinterpret_cast<const uint4*>(ctr), k0, k1, n, reinterpret_cast<uint4*>(out),
                                        curand);
    return cudaGetLastError();
}

}  // namespace pgk
