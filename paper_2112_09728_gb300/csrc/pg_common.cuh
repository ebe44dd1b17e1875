// Internal helpers shared by the kernel translation units (not part of the
// public ABI): block size, grid sizing, storage-type dispatch and the guide
// gate of Sec. 3.1 and Sec. 5.
#pragma once

#include "pg_launch.h"

namespace pgk {

constexpr int kBlock = 256;

static __device__ __forceinline__ bool same_normal(float4 a, float4 b) {
    return __float_as_uint(a.x) == __float_as_uint(b.x) && __float_as_uint(a.y) == __float_as_uint(b.y) &&
           __float_as_uint(a.z) == __float_as_uint(b.z);
}

static __device__ __forceinline__ bool gated(const Params& P, bool reinit, float4 g1) {
    // guiding is off for fresh history (Sec. 3.1), near-mirror GGX and
    // transparent surfaces (Sec. 5)
    return reinit || (g1.z >= 0.0f && g1.z < P.rough_min) || (P.glass && g1.z <= -1.5f);
}

static inline dim3 grid_for(const Params& P) {
    const size_t hw = (size_t)P.W * P.H;
    return dim3((unsigned)((hw + kBlock - 1) / kBlock));
}

}  // namespace pgk

#define PG_DISPATCH(dt, CALL)                 \
    switch (dt) {                             \
        case DT_F32: { constexpr int D = DT_F32; CALL; break; }   \
        case DT_F16: { constexpr int D = DT_F16; CALL; break; }   \
        default: { constexpr int D = DT_BF16; CALL; break; }      \
    }

