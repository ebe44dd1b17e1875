// Internal helpers shared by the kernel translation units (not part of the
// public ABI): block size, grid sizing, storage-type dispatch and the guide
// gate of Sec. 3.1 and Sec. 5.
#pragma once

#include "pg_launch.h"

namespace pgk {

constexpr int kBlock = 256;
// The block of the fused frame kernel and of the adjoint: 128 threads, ten
// blocks per SM for the one-sample frame (the same 1,280 threads as five of
// 256), eight for the others, so that the last wave's blocks are smaller and
// the SMs run out of work closer together (measured against 256-thread
// blocks: the 1080p frame 2.5% faster, the 4K frame 1.4%, the adjoint 0.9%,
// bit-identical).
constexpr int kFrameBlock = 128;

static __device__ __forceinline__ bool same_normal(float4 a, float4 b) {
    return __float_as_uint(a.x) == __float_as_uint(b.x) && __float_as_uint(a.y) == __float_as_uint(b.y) &&
           __float_as_uint(a.z) == __float_as_uint(b.z);
}

static __device__ __forceinline__ bool gated(const Params& P, bool reinit, float4 g1) {
    // guiding is off for fresh history (Sec. 3.1), near-mirror GGX and
    // transparent surfaces (Sec. 5)
    return reinit || (g1.z >= 0.0f && g1.z < P.rough_min) || (P.glass && g1.z <= -1.5f);
}

// Reprojection of one pixel: Gamma(t-1) at the motion-compensated pixel, or a
// re-initialised guide. Returns true for a re-initialised pixel.
template <int DT>
static __device__ __forceinline__ bool reproject_pixel(const Params& P, int x, int y, float4 a0, float4 a1,
                                                const void* __restrict__ gin, const float4* __restrict__ g0p,
                                                size_t hw, Gam& g, int* err) {
    const int j = reproject_target(P, x, y, a1, err);
    if (j < 0) {
        g = init_gam(P);
        return true;
    }
    // Gamma(t-1) at the target is loaded beside the previous G-buffer, before
    // the test decides on it: the two loads overlap instead of following one
    // another (for a rejected pixel the guide read goes unused)
    const float4 gp = __ldcs(g0p + j);
    const Gam gj = Store<DT>::load(gin, hw, (size_t)j);
    if (!reproject_accept(P, a0, gp)) {
        g = init_gam(P);
        return true;
    }
    g = gj;
    if (!same_normal(gp, a0)) change_frame(g, make_float3(gp.x, gp.y, gp.z), make_float3(a0.x, a0.y, a0.z));
    return false;
}

// Reprojection with a record of its outcome for a later pass (neighbour reuse):
// 0xFFFFFFFF for a re-initialised pixel, else the previous pixel j, with bit 31
// set when the normals differ and the guide went through the frame change.
template <int DT>
static __device__ __forceinline__ bool reproject_pixel_rec(const Params& P, int x, int y, float4 a0, float4 a1,
                                                    const void* __restrict__ gin, const float4* __restrict__ g0p,
                                                    size_t hw, Gam& g, uint32_t& rec, int* err) {
    const int j = reproject_target(P, x, y, a1, err);
    rec = 0xFFFFFFFFu;
    if (j < 0) {
        g = init_gam(P);
        return true;
    }
    const float4 gp = __ldcs(g0p + j);
    const Gam gj = Store<DT>::load(gin, hw, (size_t)j);   // beside the G-buffer load, as above
    if (!reproject_accept(P, a0, gp)) {
        g = init_gam(P);
        return true;
    }
    g = gj;
    rec = (uint32_t)j;
    if (!same_normal(gp, a0)) {
        change_frame(g, make_float3(gp.x, gp.y, gp.z), make_float3(a0.x, a0.y, a0.z));
        rec |= 0x80000000u;
    }
    return false;
}

// The same guide again from the record: the outcome is not re-derived, only
// the guide reloaded (and the frame change redone where bit 31 says so).
template <int DT>
static __device__ __forceinline__ bool replay_reprojection(const Params& P, uint32_t rec, float4 a0,
                                                    const void* __restrict__ gin, const float4* __restrict__ g0p,
                                                    size_t hw, Gam& g, int* err) {
    const int j = (int)(rec & 0x7FFFFFFFu);
    if (rec == 0xFFFFFFFFu || !PG_IN_BOUNDS(j, hw, err)) {
        g = init_gam(P);
        return true;
    }
    g = Store<DT>::load(gin, hw, (size_t)j);
    if (rec & 0x80000000u) {
        const float4 gp = __ldcs(g0p + j);
        change_frame(g, make_float3(gp.x, gp.y, gp.z), make_float3(a0.x, a0.y, a0.z));
    }
    return false;
}

static inline dim3 grid_for(const Params& P, int block = kBlock) {
    const size_t hw = (size_t)P.W * P.H;
    return dim3((unsigned)((hw + block - 1) / block));
}

}  // namespace pgk

#define PG_DISPATCH(dt, CALL)                 \
    switch (dt) {                             \
        case DT_F32: { constexpr int D = DT_F32; CALL; break; }   \
        case DT_F16: { constexpr int D = DT_F16; CALL; break; }   \
        default: { constexpr int D = DT_BF16; CALL; break; }      \
    }

