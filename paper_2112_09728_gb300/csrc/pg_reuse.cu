// Neighbour-VPL reuse (Sec. 3.2, 4.2): the frame as the paper's two passes.
// k_pt reprojects, samples and writes one VPL per sample (world direction,
// radiance and, for a BRDF-strategy draw, its BRDF density), and per pixel a
// handover record {Z, outcome of the reprojection}; k_train takes the
// reprojected guide from that record (no second reprojection) and trains it
// on its own samples and N picks among its window's samples.
#include "pg_common.cuh"

namespace pgk {

namespace {

// Neighbour-VPL reuse, pass 1 (path tracing, Fig. 2): the frame's samples
// and image as in k_frame, plus one VPL per sample in the buffer Pi: world
// direction and radiance in vpl, and in pb_src the density of the pixel's
// BRDF draw for a BRDF-strategy sample (0 for samples that do not train).
// Each pixel's handover record, {Z, reprojection record}, goes to hand for
// the training pass (reproject_pixel_rec).
template <int DT, bool ONE, bool RGB>
__global__ void __launch_bounds__(kBlock, 5) k_pt(const Params P, const void* __restrict__ gin,
                                                  const float4* __restrict__ g0, const float4* __restrict__ g1,
                                                  const float4* __restrict__ g0p, float* __restrict__ img,
                                                  uint32_t frame, float4* __restrict__ vpl,
                                                  float* __restrict__ pb_src, float2* __restrict__ hand,
                                                  int* __restrict__ err) {
    const size_t hw = (size_t)P.W * P.H;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if ((size_t)i >= hw) return;
    const int y = i / P.W, x = i - y * P.W;
    const float4 a0 = __ldcs(g0 + i), a1 = __ldcs(g1 + i);
    Gam g;
    uint32_t rec;
    const bool reinit = reproject_pixel_rec<DT>(P, x, y, a0, a1, gin, g0p, hw, g, rec, err);
    const Surf s = make_surf(P, x, y, a0, a1);
    const Guide d = derive_guide(P, g, gated(P, reinit, a1));
    hand[i] = make_float2(d.Z, __uint_as_float(rec));
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
// coprime with C, so they are distinct. The reprojected guide and Z come
// from pass 1's handover record.
//
// Each thread first classifies its N picks in a loop of the same length on
// every lane (decode, on screen, drawn by the BRDF strategy), keeping a bit
// per training pick, then evaluates only those. A warp thus runs as many
// evaluations as its busiest lane has training VPLs, with no lane waiting on
// another's search for its next one. The own samples come first, then the
// picks in pick order: the order of the compensated sums is the pick order.
//
// TILED (the VPL preload of Sec. 4.2): a block covers kTileW x kTileH pixels
// and first copies the window tile of its pixels' candidates, (kTileW + 2R) x
// (kTileH + 2R) pixels x spp samples of VPLs and densities, into shared memory
// (zeros off the screen); the picks then read the tile. Launched when the tile
// fits kTileBytes.
constexpr int kTileW = 32, kTileH = 8;
constexpr int kTileBytes = 24 * 1024;

template <int DT, bool ONE, bool TILED>
__global__ void __launch_bounds__(kBlock, 4) k_train(const Params P, const void* __restrict__ gin,
                                                     void* __restrict__ gout, const float4* __restrict__ g0,
                                                     const float4* __restrict__ g1,
                                                     const float4* __restrict__ g0p, uint32_t frame,
                                                     const float4* __restrict__ vpl,
                                                     const float* __restrict__ pb_src,
                                                     const float2* __restrict__ hand, int* __restrict__ err) {
    const size_t hw = (size_t)P.W * P.H;
    const int spp = ONE ? 1 : P.spp;
    int x, y;
    bool inside;
    if (TILED) {
        x = blockIdx.x * kTileW + (int)(threadIdx.x % kTileW);
        y = blockIdx.y * kTileH + (int)(threadIdx.x / kTileW);
        inside = x < P.W && y < P.H;
    } else {
        const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
        inside = (size_t)i0 < hw;
        y = inside ? i0 / P.W : 0;
        x = inside ? i0 - y * P.W : 0;
    }
    // TILED: the block's window tile, VPLs [spp][th][tw] then densities
    extern __shared__ float4 s_vpl[];
    const int tw = kTileW + 2 * P.reuse_r, th = kTileH + 2 * P.reuse_r, tn = tw * th;
    const int x0 = (int)blockIdx.x * kTileW - P.reuse_r, y0 = (int)blockIdx.y * kTileH - P.reuse_r;
    float* s_pb = reinterpret_cast<float*>(s_vpl + (TILED ? tn * spp : 0));
    if (TILED) {
        for (int k = threadIdx.x; k < tn * spp; k += blockDim.x) {
            const int sj = k / tn, rem = k - sj * tn, ty = rem / tw, tx = rem - ty * tw;
            const int gx = x0 + tx, gy = y0 + ty;
            float pb = 0.0f;
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (gx >= 0 && gx < P.W && gy >= 0 && gy < P.H) {
                const size_t q = (size_t)sj * hw + (size_t)gy * P.W + gx;
                if (PG_IN_BOUNDS(q, (size_t)spp * hw, err)) {
                    pb = pb_src[q];
                    v = vpl[q];
                }
            }
            s_pb[k] = pb;
            s_vpl[k] = v;
        }
        __syncthreads();
    }
    if (!inside) return;
    const int i = y * P.W + x;
    const float4 a0 = __ldcs(g0 + i), a1 = __ldcs(g1 + i);
    const float2 hv = __ldcs(hand + i);
    Gam g;
    const bool reinit = replay_reprojection<DT>(P, __float_as_uint(hv.y), a0, gin, g0p, hw, g, err);
    const Surf s = make_surf(P, x, y, a0, a1);
    Guide d = derive_guide_shape(P, g, gated(P, reinit, a1));
    d.Z = hv.x;
    const int kc = (int)fminf(fmaxf(g.k, 0.0f), (float)P.k_max);
    const int n = min(5 + (15 * (P.k_max - kc)) / P.k_max, P.reuse_c);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, frame, 0u, 4u), P.rk);
    const int o0 = (int)(((uint64_t)r.x * (uint64_t)P.reuse_c) >> 32);
    const int dw = 2 * P.reuse_r + 1, center = (dw * dw - 1) / 2;
    // index of sample sj of pixel (qx, qy): in the tile (TILED) or in the
    // sample-major buffers
    auto slot = [&](int qx, int qy, int sj) -> size_t {
        if (TILED) return (size_t)((sj * th + (qy - y0)) * tw + (qx - x0));
        return (size_t)sj * hw + (size_t)qy * P.W + qx;
    };
    auto pb_at = [&](size_t q) { return TILED ? s_pb[q] : pb_src[q]; };
    auto vpl_at = [&](size_t q) { return TILED ? s_vpl[q] : vpl[q]; };
    const size_t n_slots = TILED ? (size_t)tn * spp : (size_t)spp * hw;
    (void)n_slots;                               // read by the bounds-checked build only
    // candidate o: pixel cell o / spp of the window (p itself skipped), sample
    // o mod spp; the floor divisions are exact in binary32 for these small
    // integers. False for a cell off the screen.
    auto candidate = [&](int o, size_t& q) {
        const int cell0 = ONE ? o : (int)(((float)o + 0.5f) * P.reuse_inv_spp);
        const int sj = o - cell0 * spp;
        const int cell = cell0 + (cell0 >= center ? 1 : 0);
        const int ry = (int)(((float)cell + 0.5f) * P.reuse_inv_dw);
        const int qx = x + cell - ry * dw - P.reuse_r, qy = y + ry - P.reuse_r;
        if (qx < 0 || qx >= P.W || qy < 0 || qy >= P.H) return false;
        q = slot(qx, qy, sj);
        return PG_IN_BOUNDS(q, n_slots, err);
    };
    // pick j (j < n <= 20) trains iff bit j of mask is set
    uint32_t mask = 0u;
#pragma unroll 4
    for (int j = 0, o = o0; j < n; ++j) {
        size_t q;
        if (candidate(o, q) && pb_at(q) > 0.0f) mask |= 1u << j;
        o += P.reuse_stride;
        if (o >= P.reuse_c) o -= P.reuse_c;
    }
    Stats st;
    for (int si = 0; si < spp; ++si) {           // the pixel's own samples
        const size_t q = slot(x, y, si);
        const float pb = pb_at(q);
        if (pb > 0.0f) {
            const float4 v = vpl_at(q);
            st.add_vpl(d, g, s, make_float3(v.x, v.y, v.z), v.w, pb, P.f0);
        }
    }
    while (mask) {                               // the training picks, in pick order
        const int j = __ffs(mask) - 1;
        mask &= mask - 1u;
        // o_j = (o_0 + j stride) mod C; below 2^32 since C, stride < 2^19 and j < 20
        const int o = (int)(((uint32_t)o0 + (uint32_t)j * (uint32_t)P.reuse_stride) % (uint32_t)P.reuse_c);
        size_t q = 0;
        candidate(o, q);
        const float pb = pb_at(q);
        const float4 v = vpl_at(q);
        st.add_vpl(d, g, s, make_float3(v.x, v.y, v.z), v.w, pb, P.f0);
    }
    m_step(P, g, st);
    if (!gam_finite(g)) atomicOr(err, PG_ERR_BIT_NUMERIC);
    store_step<DT>(P, gout, hw, (size_t)i, g, frame);
}

}  // namespace

cudaError_t launch_pt(int dt, const Params& P, const void* gin, const float4* g0, const float4* g1,
                      const float4* g0p, float* img, uint32_t frame, float4* vpl, float* pb_src, float2* hand, int* err,
                      cudaStream_t st) {
    const dim3 grid = grid_for(P);
#define PG_PT(ONE, RGB) \
    PG_DISPATCH(dt, (k_pt<D, ONE, RGB><<<grid, kBlock, 0, st>>>(P, gin, g0, g1, g0p, img, frame, vpl, pb_src, hand, err)))
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
                         const float4* g0p, uint32_t frame, const float4* vpl, const float* pb_src, const float2* hand,
                         int* err, cudaStream_t st) {
    const int tn = (kTileW + 2 * P.reuse_r) * (kTileH + 2 * P.reuse_r);
    const size_t tile_bytes = (size_t)tn * P.spp * (sizeof(float4) + sizeof(float));
    static_assert(kTileW * kTileH == kBlock, "a tile is one block of pixels");
    if (tile_bytes <= (size_t)kTileBytes) {
        const dim3 grid((unsigned)((P.W + kTileW - 1) / kTileW), (unsigned)((P.H + kTileH - 1) / kTileH));
#define PG_TRAIN_TILED(ONE) \
    PG_DISPATCH(dt, (k_train<D, ONE, true><<<grid, kBlock, tile_bytes, st>>>(P, gin, gout, g0, g1, g0p, frame, vpl, \
                                                                             pb_src, hand, err)))
        if (P.spp == 1) {
            PG_TRAIN_TILED(true);
        } else {
            PG_TRAIN_TILED(false);
        }
#undef PG_TRAIN_TILED
    } else if (P.spp == 1) {
        PG_DISPATCH(dt, (k_train<D, true, false><<<grid_for(P), kBlock, 0, st>>>(P, gin, gout, g0, g1, g0p, frame,
                                                                                 vpl, pb_src, hand, err)));
    } else {
        PG_DISPATCH(dt, (k_train<D, false, false><<<grid_for(P), kBlock, 0, st>>>(P, gin, gout, g0, g1, g0p, frame,
                                                                                  vpl, pb_src, hand, err)));
    }
    return cudaGetLastError();
}

}  // namespace pgk
