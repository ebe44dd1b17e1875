// Device functions of the guide pass (binary32), shared by the fused frame
// kernel and the staged kernels. Sections and equations refer to Derevyannykh,
// "Real-Time Path-Guiding Based on Parametric Mixture Models" (2112.09728).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pgk {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kInvPi = 0.318309886183790671538f;
constexpr float kInv2Pi = 0.159154943091895335769f;
constexpr float kInv4Pi2 = 0.0253302959105844428f;   // 1 / (4 pi^2)
constexpr float k4OverPi = 1.27323954473516268615f;
// Nodes of the Phi_2 correction: one 6-node rule in s = sin t fitted to the
// corner integrals the kernels evaluate (fit_corner_rule.py), whose worst
// corner error is 1.3e-8 up to |rho| = 0.9, about that of the 8-node
// Gauss-Legendre rule in t (8e-9; the 6-node one's is 3.5e-7). One rule serves
// every pixel: pixels of one warp on different rules would run each rule's
// nodes in turn (on trained guides a warp then ran 11 to 14 node steps where
// one common 8-node rule ran 8).
constexpr int kZNodes = 6;

enum { DT_F32 = 0, DT_F16 = 1, DT_BF16 = 2 };

// Index checks of the debug build (compiled with PG_BOUNDS_CHECK): an index
// that depends on the data (the reprojected pixel, a reused neighbour's
// sample) and falls outside its buffer sets bit 2 of the context's error word
// (pg_check reports PG_ERR_BOUNDS) and the access is skipped. In the normal
// build the check is the constant true and costs nothing.
#define PG_ERR_BIT_NUMERIC 1
#define PG_ERR_BIT_BOUNDS 2
#ifdef PG_BOUNDS_CHECK
__device__ __forceinline__ bool pg_in_bounds(long long i, long long n, int* err) {
    if (i >= 0 && i < n) return true;
    if (err) atomicOr(err, PG_ERR_BIT_BOUNDS);
    return false;
}
#define PG_IN_BOUNDS(i, n, err) pg_in_bounds((long long)(i), (long long)(n), (err))
#else
#define PG_IN_BOUNDS(i, n, err) true
#endif
enum { ST_BRDF = 0, ST_GUIDE = 1, ST_FALLBACK = 2, ST_DELTA = 3, ST_INVALID = 4 };

// Everything a launch needs besides its pointers; passed by value (kernel
// parameter space), so concurrent contexts never share constant memory.
struct Params {
    int W, H, spp, k_max;
    uint32_t key0, key1;
    uint32_t rk[20];     // Philox round keys: (key0 + r W0, key1 + r W1) for rounds r = 0..9
    float pi_min, pi_max, pi_reinit;
    float depth_tol, normal_tol, rough_min, sigma2_min, rho_max;
    float init_raw[5];   // E[X], E[Y], E[X^2], E[Y^2], E[XY] of a re-initialised guide
    float init_c[3];     // its central moments s_xx, s_yy, s_xy
    // camera of the current frame
    int cam_kind;
    float cam_o[3], cam_f[3], cam_r[3], cam_u[3];
    float cam_ps, cam_tan, cam_aspect;
    // analytic radiance field
    int n_lobes, mask_kind;
    float lobe_dir[8][3], lobe_kappa[8], lobe_scale[8];  // scale = amp * vMF normaliser
    float lobe_e2[8];                                     // -kappa log2(e) / 2: exponent per |w - d|^2 in base 2
    // the same lobes in pairs (2i, 2i+1) for paired arithmetic: negated
    // direction components and exponent factors (zero beyond n_lobes)
    float2 lobe_pnx[4], lobe_pny[4], lobe_pnz[4], lobe_pe2[4];
    float field_const, mask[3];
    // coloured field: per-lobe scale of each channel and the constant's
    // channels (lobe_scale and field_const then hold the luminance)
    int rgb;
    float lobe_rgb[8][3], field_const_rgb[3];
    // the rule of Z's corner integrals on [0, rho]: nodes s = rho c, weights rho w
    float zq_c[kZNodes], zq_w[kZNodes];
    // neighbour-VPL reuse: window radius (0 = off), number of candidates
    // ((2R+1)^2 - 1) spp, and the stride of the walk through them
    int reuse_r, reuse_c, reuse_stride;
    float reuse_inv_spp, reuse_inv_dw;   // 1/spp and 1/(2R+1), for exact floor divisions of small integers
    float f0;                            // Schlick reflectance of GGX at normal incidence (1: F = 1)
    int glass;                           // roughness codes <= -1.5 are transparent (else Lambertian)
    int sr;                              // stochastic rounding of the 16-bit EM stores
    uint32_t sr_frame;                   // frame index of the staged update's rounding bits
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), counter-based: ten rounds of two
// 32x32->64 multiplies with the key bumped by the Weyl constants in between.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t k0, uint32_t k1) {
    // one 32x32 -> 64 product per multiplier gives both halves
    const uint64_t p0 = (uint64_t)c.x * 0xD2511F53u, p1 = (uint64_t)c.z * 0xCD9E8D57u;
    return make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
}
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        c = philox_round(c, k0, k1);
    }
    return c;
}
// the same with the round keys precomputed on the host (Params::rk)
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const uint32_t* rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) c = philox_round(c, rk[2 * r], rk[2 * r + 1]);
    return c;
}
// top 24 bits -> [0, 1) and (0, 1]; both exact in binary32
__device__ __forceinline__ float unit24(uint32_t w) { return (float)(w >> 8) * 5.9604644775390625e-8f; }
__device__ __forceinline__ float unit24_open0(uint32_t w) {
    return (float)((w >> 8) + 1u) * 5.9604644775390625e-8f;
}

// x / y for y > 0 by the hardware reciprocal (2 ulp). Below 1e-30 both
// operands are first scaled by 2^64 (exactly), so that 1/y stays a normal
// number; the scale is a select, not a branch to a slow division, which
// would split the straight-line code around every call (measured: the reuse
// frame 7% and the 4K frame 2% faster without it, bit-identical on both).
__device__ __forceinline__ float fdiv(float x, float y) {
    const float sc = y > 1e-30f ? 1.0f : 18446744073709551616.0f;
    return __fdividef(x * sc, y * sc);
}

// Pairs of binary32 values: sm_100's paired FMA, multiply and add issue once
// for both halves, each half rounded as the scalar operation would round it,
// so code written on pairs gives the scalar code's bits in half the issue
// slots of its arithmetic.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// 2^x by the hardware approximation (relative error below 2^-22 over the
// normal range; results below the smallest normal flush to zero).
__device__ __forceinline__ float exp2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Square root by the hardware approximation (sqrt.approx.f32), for the
// per-sample geometry where a correctly rounded root buys nothing: a few ulp
// of a direction component are far below the parity tolerances.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sin and cos of 2 pi x for x in [0, 1): shifted by half a turn into [-pi, pi),
// where the hardware approximation holds its 2^-21.4 absolute accuracy.
__device__ __forceinline__ void sincos_turn(float x, float* s, float* c) {
    float sn, cs;
    __sincosf(6.28318530717958648f * (x - 0.5f), &sn, &cs);
    *s = -sn;
    *c = -cs;
}

// ---------------------------------------------------------------------------
// Small vector helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 f3(const float* p) { return make_float3(p[0], p[1], p[2]); }

// Orthonormal basis around n: Duff et al., "Building an Orthonormal Basis,
// Revisited" (JCGT 2017), the same construction on both sides of the pass.
struct Basis {
    float3 t, b, n;
};
__device__ __forceinline__ Basis make_basis(float3 n) {
    const float sg = copysignf(1.0f, n.z);
    const float a = __fdividef(-1.0f, sg + n.z);   // sg + n.z in [1, 2] for a unit normal
    const float c = n.x * n.y * a;
    Basis f;
    f.n = n;
    f.t = make_float3(1.0f + sg * n.x * n.x * a, sg * c, -sg * n.x);
    f.b = make_float3(c, sg + n.y * n.y * a, -n.y);
    return f;
}
__device__ __forceinline__ float3 to_world(const Basis& f, float3 l) {
    return make_float3(l.x * f.t.x + l.y * f.b.x + l.z * f.n.x, l.x * f.t.y + l.y * f.b.y + l.z * f.n.y,
                       l.x * f.t.z + l.y * f.b.z + l.z * f.n.z);
}
__device__ __forceinline__ float3 to_local(const Basis& f, float3 w) {
    return make_float3(dot3(w, f.t), dot3(w, f.b), dot3(w, f.n));
}

// ---------------------------------------------------------------------------
// Shirley-Chiu map M (Eq. 2): concentric square->disk, equal-area lift.
// z = 1 - r^2 is formed as 4 m (1 - m), m the distance of the dominant
// coordinate to the square's edge, so grazing directions keep their relative
// precision in binary32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 square_to_hemi(float u, float v) {
    const float a = 2.0f * u - 1.0f, b = 2.0f * v - 1.0f;
    if (a == 0.0f && b == 0.0f) return make_float3(0.0f, 0.0f, 1.0f);
    // either dominant axis by the same instructions (no divergent sincos sites)
    const bool xd = fabsf(a) > fabsf(b);
    const float r = xd ? a : b;
    const float m = xd ? fminf(u, 1.0f - u) : fminf(v, 1.0f - v);
    float s, c;
    __sincosf(0.78539816339744831f * __fdividef(xd ? b : a, r), &s, &c);
    const float z = 4.0f * m * (1.0f - m);
    const float lift = sqrt_approx(1.0f + z);
    const float2 d = mul2(mul2(dup2(r), xd ? make_float2(c, s) : make_float2(s, c)), dup2(lift));
    return make_float3(d.x, d.y, z);
}

// (4/pi) atan(t) for t in [-1, 1]: t P(t^2) with P of degree 7, this
// library's own fit (fit_atan.py; absolute error 5e-8, 1.7e-7 in binary32).
__device__ __forceinline__ float atan_unit(float t) {
    const float t2 = t * t;
    float p = -5.160561652e-03f;
    p = fmaf(p, t2, 2.782882500e-02f);
    p = fmaf(p, t2, -7.117607943e-02f);
    p = fmaf(p, t2, 1.227560273e-01f);
    p = fmaf(p, t2, -1.770841680e-01f);
    p = fmaf(p, t2, 2.539659938e-01f);
    p = fmaf(p, t2, -4.243687760e-01f);
    p = fmaf(p, t2, 1.273238691e+00f);
    return p * t;
}

// Inverse map: disk point d = w_xy / sqrt(1 + z); the dominant disk axis gives
// the square coordinate of radius |d|, the other one follows from the
// arctangent of the component ratio (within [-1, 1]), for either axis by the
// same instructions.
__device__ __forceinline__ float2 hemi_to_square(float3 w) {
    const float z = fmaxf(w.z, 0.0f);
    const float inv = rsqrtf(1.0f + z);
    const float dx = w.x * inv, dy = w.y * inv;
    const float r = sqrt_approx(dx * dx + dy * dy);
    if (r < 1e-30f) return make_float2(0.5f, 0.5f);   // the pole (to within 1e-30)
    const bool xdom = fabsf(dx) >= fabsf(dy);
    const float lead = xdom ? dx : dy, other = xdom ? dy : dx;
    const float m = copysignf(r, lead);                 // the dominant coordinate
    const float n = m * atan_unit(__fdividef(other, lead));
    const float a = xdom ? m : n, b = xdom ? n : m;
    return make_float2(0.5f * (a + 1.0f), 0.5f * (b + 1.0f));
}

// ---------------------------------------------------------------------------
// Guide state (one pixel of Gamma) in registers.
// ---------------------------------------------------------------------------
struct Gam {
    float ex, ey;             // mean (stored, not clamped)
    float exx, eyy, exy;      // raw second moments (binary32 storage only)
    float sxx, syy, sxy;      // central second moments (not regularised)
    float pi, k, W;      // mixing weight, epoch count, running luminance mass
};

__device__ __forceinline__ void central_from_raw(Gam& g) {
    g.sxx = fmaf(-g.ex, g.ex, g.exx);
    g.syy = fmaf(-g.ey, g.ey, g.eyy);
    g.sxy = fmaf(-g.ex, g.ey, g.exy);
}
__device__ __forceinline__ void raw_from_central(Gam& g) {
    g.exx = fmaf(g.ex, g.ex, g.sxx);
    g.eyy = fmaf(g.ey, g.ey, g.syy);
    g.exy = fmaf(g.ex, g.ey, g.sxy);
}

// Storage codecs. F32: two float4 planes {E[X],E[Y],E[X^2],E[Y^2]},
// {E[XY],pi,k,W}. F16/BF16: one uint4 of 8 halves {mu, s_xx, s_yy, s_xy, pi, k, W}.
template <int DT>
struct Store;

template <>
struct Store<DT_F32> {
    static __device__ __forceinline__ Gam load(const void* base, size_t hw, size_t i) {
        const float4* p = reinterpret_cast<const float4*>(base);
        const float4 a = __ldcs(p + i), b = __ldcs(p + hw + i);
        Gam g;
        g.ex = a.x; g.ey = a.y; g.exx = a.z; g.eyy = a.w;
        g.exy = b.x; g.pi = b.y; g.k = b.z; g.W = b.w;
        central_from_raw(g);
        return g;
    }
    static __device__ __forceinline__ void store(void* base, size_t hw, size_t i, const Gam& g) {
        float4* p = reinterpret_cast<float4*>(base);
        __stcs(p + i, make_float4(g.ex, g.ey, g.exx, g.eyy));
        __stcs(p + hw + i, make_float4(g.exy, g.pi, g.k, g.W));
    }
};

template <typename H>
struct HalfStore {
    static __device__ __forceinline__ float cvt(uint16_t v);
    static __device__ __forceinline__ uint16_t pack(float v);
    // two fields at once, lo in the low half: the same rounding as pack
    static __device__ __forceinline__ uint32_t pack2(float lo, float hi);
};
template <>
__device__ __forceinline__ float HalfStore<__half>::cvt(uint16_t v) { return __half2float(__ushort_as_half(v)); }
// FP16 saturates at +-65504 rather than overflowing to infinity: the mass W
// can pass it under neighbour reuse, whose importance weights f / p_src are
// unbounded. (The finiteness check runs on the binary32 values before the
// store, so a NaN is still reported.)
template <>
__device__ __forceinline__ uint16_t HalfStore<__half>::pack(float v) {
    return __half_as_ushort(__float2half_rn(fminf(fmaxf(v, -65504.0f), 65504.0f)));
}
// the pair conversion with saturation to the largest finite value: for a
// finite input the same bits as the clamp-then-round of pack
template <>
__device__ __forceinline__ uint32_t HalfStore<__half>::pack2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
template <>
__device__ __forceinline__ float HalfStore<__nv_bfloat16>::cvt(uint16_t v) {
    return __bfloat162float(__ushort_as_bfloat16(v));
}
template <>
__device__ __forceinline__ uint16_t HalfStore<__nv_bfloat16>::pack(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
template <>
__device__ __forceinline__ uint32_t HalfStore<__nv_bfloat16>::pack2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Stochastic rounding of a binary32 value to the storage type, from 16
// random bits r: rounds to one of the two neighbours of v with probabilities
// proportional to proximity, so the stored value is v in expectation (an EM
// update below half a storage ulp still moves the guide on average).
// FP16: |v| + u ulp16(|v|), u = (r >> 3) / 2^13, then toward zero; the sum is
// exact in binary32 (u ulp16 is a multiple of binary32's ulp at |v|), and
// rounding toward zero saturates at 65504 like the nearest-rounding store.
// BF16: the random bits are added below bf16's last kept bit, then the low
// half is dropped (a carry rounds the magnitude up).
__device__ __forceinline__ uint16_t sr_pack_f16(float v, uint32_t r) {
    if (!isfinite(v)) return __half_as_ushort(__float2half_rn(v));
    const float a = fabsf(v);
    const int e = max((int)(__float_as_uint(a) >> 23) - 127, -14);   // fp16 binade (subnormals: -14)
    const float ulp = __uint_as_float((uint32_t)(e - 10 + 127) << 23);
    const float b = __fmaf_rn((float)((r & 0xFFFFu) >> 3) * (1.0f / 8192.0f), ulp, a);
    return __half_as_ushort(__float2half_rz(copysignf(b, v)));
}
__device__ __forceinline__ uint16_t sr_pack_bf16(float v, uint32_t r) {
    if (!isfinite(v)) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    return (uint16_t)((__float_as_uint(v) + (r & 0xFFFFu)) >> 16);
}

template <typename H>
struct SrPack;
template <>
struct SrPack<__half> {
    static __device__ __forceinline__ uint16_t pack(float v, uint32_t r) { return sr_pack_f16(v, r); }
};
template <>
struct SrPack<__nv_bfloat16> {
    static __device__ __forceinline__ uint16_t pack(float v, uint32_t r) { return sr_pack_bf16(v, r); }
};

template <typename H>
struct Store16 {
    static __device__ __forceinline__ Gam load(const void* base, size_t, size_t i) {
        const uint4 q = __ldcs(reinterpret_cast<const uint4*>(base) + i);
        Gam g;
        g.ex = HalfStore<H>::cvt(q.x & 0xffffu); g.ey = HalfStore<H>::cvt(q.x >> 16);
        g.sxx = HalfStore<H>::cvt(q.y & 0xffffu); g.syy = HalfStore<H>::cvt(q.y >> 16);
        g.sxy = HalfStore<H>::cvt(q.z & 0xffffu); g.pi = HalfStore<H>::cvt(q.z >> 16);
        g.k = HalfStore<H>::cvt(q.w & 0xffffu); g.W = HalfStore<H>::cvt(q.w >> 16);
        raw_from_central(g);
        return g;
    }
    static __device__ __forceinline__ void store(void* base, size_t, size_t i, const Gam& g) {
        __stcs(reinterpret_cast<uint4*>(base) + i,
               make_uint4(HalfStore<H>::pack2(g.ex, g.ey), HalfStore<H>::pack2(g.sxx, g.syy),
                          HalfStore<H>::pack2(g.sxy, g.pi), HalfStore<H>::pack2(g.k, g.W)));
    }
    // stochastic rounding: field j takes the 16 bits (r[j / 2] >> 16 (j mod 2)) & 0xFFFF
    static __device__ __forceinline__ void store_sr(void* base, size_t, size_t i, const Gam& g, uint4 r) {
        auto pk = [](float lo, float hi, uint32_t w) {
            return (uint32_t)SrPack<H>::pack(lo, w) | ((uint32_t)SrPack<H>::pack(hi, w >> 16) << 16);
        };
        __stcs(reinterpret_cast<uint4*>(base) + i,
               make_uint4(pk(g.ex, g.ey, r.x), pk(g.sxx, g.syy, r.y), pk(g.sxy, g.pi, r.z), pk(g.k, g.W, r.w)));
    }
};
template <>
struct Store<DT_F16> : Store16<__half> {};
template <>
struct Store<DT_BF16> : Store16<__nv_bfloat16> {};

// Work copy of the staged pass: binary32, two float4 planes. For F32 storage
// it holds the raw moments (bit-identical to storage); for F16/BF16 it holds
// the mean and central moments, so no precision is lost between the stages.
template <int DT>
struct Work {
    static __device__ __forceinline__ Gam load(const float4* w, size_t hw, size_t i) {
        const float4 a = w[i], b = w[hw + i];
        Gam g;
        g.ex = a.x; g.ey = a.y;
        if (DT == DT_F32) {
            g.exx = a.z; g.eyy = a.w; g.exy = b.x;
            central_from_raw(g);
        } else {
            g.sxx = a.z; g.syy = a.w; g.sxy = b.x;
            raw_from_central(g);
        }
        g.pi = b.y; g.k = b.z; g.W = b.w;
        return g;
    }
    static __device__ __forceinline__ void store(float4* w, size_t hw, size_t i, const Gam& g) {
        if (DT == DT_F32) {
            w[i] = make_float4(g.ex, g.ey, g.exx, g.eyy);
            w[hw + i] = make_float4(g.exy, g.pi, g.k, g.W);
        } else {
            w[i] = make_float4(g.ex, g.ey, g.sxx, g.syy);
            w[hw + i] = make_float4(g.sxy, g.pi, g.k, g.W);
        }
    }
};

// The store of an EM step: round to nearest, or with stochastic_round set and
// a 16-bit storage type, stochastic rounding from Philox at counter (pixel,
// frame, 0, 5).
template <int DT>
__device__ __forceinline__ void store_step(const Params& P, void* base, size_t hw, size_t i, const Gam& g,
                                           uint32_t frame) {
    if constexpr (DT != DT_F32) {
        if (P.sr) {
            Store<DT>::store_sr(base, hw, i, g, philox4x32_10(make_uint4((uint32_t)i, frame, 0u, 5u), P.rk));
            return;
        }
    }
    Store<DT>::store(base, hw, i, g);
}

__device__ __forceinline__ Gam init_gam(const Params& P) {
    Gam g;
    g.ex = P.init_raw[0]; g.ey = P.init_raw[1];
    g.exx = P.init_raw[2]; g.eyy = P.init_raw[3]; g.exy = P.init_raw[4];
    g.sxx = P.init_c[0]; g.syy = P.init_c[1]; g.sxy = P.init_c[2];
    g.pi = P.pi_reinit; g.k = 0.0f; g.W = 0.0f;
    return g;
}

__device__ __forceinline__ bool gam_finite(const Gam& g) {
    return isfinite(g.ex) && isfinite(g.ey) && isfinite(g.sxx) && isfinite(g.syy) && isfinite(g.sxy) &&
           isfinite(g.pi) && isfinite(g.k) && isfinite(g.W);
}

// ---------------------------------------------------------------------------
// Reprojection (Sec. 3.1). The previous pixel and the acceptance test are
// taken in binary32 with explicit round-to-nearest operations in a fixed
// order (no contraction), so the decision is reproducible bit for bit.
// Returns the linear index of the previous pixel, or -1 for a rejection.
// ---------------------------------------------------------------------------
// The motion-compensated previous pixel of (x, y), or -1 off the screen.
__device__ __forceinline__ int reproject_target(const Params& P, int x, int y, float4 g1, int* err) {
    const float fx = __fadd_rn(__fadd_rn((float)x, 0.5f), g1.x);
    const float fy = __fadd_rn(__fadd_rn((float)y, 0.5f), g1.y);
    if (!(fx >= 0.0f && fx < (float)P.W && fy >= 0.0f && fy < (float)P.H)) return -1;
    const int qx = (int)floorf(fx), qy = (int)floorf(fy);
    const int j = qy * P.W + qx;
    if (!PG_IN_BOUNDS(j, (long long)P.W * P.H, err)) return -1;
    return j;
}

// The depth and normal test between the current surface g0 and the previous
// surface gp at the target pixel.
__device__ __forceinline__ bool reproject_accept(const Params& P, float4 g0, float4 gp) {
    const float dd = fabsf(__fsub_rn(gp.w, g0.w));
    const float dl = __fmul_rn(P.depth_tol, g0.w);
    const float nd = __fadd_rn(__fadd_rn(__fmul_rn(gp.x, g0.x), __fmul_rn(gp.y, g0.y)), __fmul_rn(gp.z, g0.z));
    return dd <= dl && nd >= P.normal_tol;
}

__device__ __forceinline__ int reproject_index(const Params& P, int x, int y, float4 g0, float4 g1,
                                               const float4* __restrict__ g0_prev, float4* g0p_out, int* err) {
    const int j = reproject_target(P, x, y, g1, err);
    if (j < 0) return -1;
    const float4 gp = __ldcs(g0_prev + j);
    *g0p_out = gp;
    return reproject_accept(P, g0, gp) ? j : -1;
}

// Frame change between the previous and the current surface (Sec. 3.1): the
// guide's mean direction goes through world space into the new frame (held
// at the horizon if it falls below), the covariance is kept.
__device__ __forceinline__ void change_frame(Gam& g, float3 np, float3 nc) {
    const float mx = fminf(fmaxf(g.ex, 0.0f), 1.0f), my = fminf(fmaxf(g.ey, 0.0f), 1.0f);
    const float3 wl = square_to_hemi(mx, my);
    const float3 ww = to_world(make_basis(np), wl);
    float3 wn = to_local(make_basis(nc), ww);
    if (wn.z < 0.0f) {
        const float r = sqrtf(wn.x * wn.x + wn.y * wn.y);
        wn.z = 0.0f;
        if (r > 0.0f) {
            wn.x /= r;
            wn.y /= r;
        } else {
            wn.x = 1.0f;
            wn.y = 0.0f;
        }
    }
    const float2 u = hemi_to_square(wn);
    g.ex = u.x;
    g.ey = u.y;
    raw_from_central(g);
}

// ---------------------------------------------------------------------------
// Derived guide (Eq. 2): clamped mean, regularised covariance, its Cholesky
// factor, and Z = mass of N(mu, Sigma) on [0,1]^2.
// ---------------------------------------------------------------------------
struct Guide {
    float mx, my, sxx, syy, sxy;
    float l11, l21, l22, il11, il22, pnorm;  // pnorm = 1/(4 pi^2 l11 l22): per-steradian factor
    float Z, pi_eff;
};

// Upper tail 1 - Phi(h) = erfc(h / sqrt 2) / 2 for h >= 0; below 8e-9 past
// h = 5.66, where it is dropped. erfc(x) ~ t exp(-x^2 + Q(t - 0.66)) with
// t = 1 / (1 + x/2) and Q of degree 9, fitted by this library
// (fit_normal_tail.py): relative error of the fit 6e-9; in binary32 with the
// hardware exp2 the tail is within 2e-7 absolute, about erfcf's own accuracy,
// and the 1080p frame is 6% shorter than with erfcf.
__device__ __forceinline__ float normal_tail(float h) {
    if (!(h < 5.66f)) return 0.0f;
    const float x = h * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.5f, x, 1.0f)), s = t - 0.66f;
    float q = 1.351362865e-02f;
    q = fmaf(q, s, 1.648487823e-01f);
    q = fmaf(q, s, -1.294304248e-01f);
    q = fmaf(q, s, -1.525244650e-01f);
    q = fmaf(q, s, 2.444149027e-01f);
    q = fmaf(q, s, 7.020706726e-02f);
    q = fmaf(q, s, -4.014188533e-01f);
    q = fmaf(q, s, -2.941247197e-03f);
    q = fmaf(q, s, 1.375446506e+00f);
    q = fmaf(q, s, -4.533098012e-01f);
    return 0.5f * t * exp2_approx(fmaf(-x, x, q) * 1.44269504088896341f);
}

// normal_tail of two arguments at once: the same operations on each half.
__device__ __forceinline__ float2 normal_tail2(float2 h) {
    const float2 x = mul2(h, dup2(0.70710678118654752f));
    const float2 den = fma2(dup2(0.5f), x, dup2(1.0f));
    const float2 t = make_float2(__fdividef(1.0f, den.x), __fdividef(1.0f, den.y));
    const float2 s = add2(t, dup2(-0.66f));
    float2 q = dup2(1.351362865e-02f);
    q = fma2(q, s, dup2(1.648487823e-01f));
    q = fma2(q, s, dup2(-1.294304248e-01f));
    q = fma2(q, s, dup2(-1.525244650e-01f));
    q = fma2(q, s, dup2(2.444149027e-01f));
    q = fma2(q, s, dup2(7.020706726e-02f));
    q = fma2(q, s, dup2(-4.014188533e-01f));
    q = fma2(q, s, dup2(-2.941247197e-03f));
    q = fma2(q, s, dup2(1.375446506e+00f));
    q = fma2(q, s, dup2(-4.533098012e-01f));
    const float2 e = mul2(fma2(neg2(x), x, q), dup2(1.44269504088896341f));
    const float2 v = mul2(mul2(dup2(0.5f), t), make_float2(exp2_approx(e.x), exp2_approx(e.y)));
    return make_float2(h.x < 5.66f ? v.x : 0.0f, h.y < 5.66f ? v.y : 0.0f);
}

// Z by four corners of the bivariate normal cdf in the Drezner-Wesolowsky form
//   Phi_2(h,k;rho) = Phi(h)Phi(k) + 1/(2 pi) int_0^asin(rho) exp(-(h^2+k^2-2hk sin t)/(2 cos^2 t)) dt,
// so Z = (Phi(h1)-Phi(h0)) (Phi(k1)-Phi(k0)) + signed sum of the four corner
// integrals, each by the fitted 6-node rule in s = sin t on [0, rho] (abs.
// error below 1.4e-8 up to |rho| = 0.9; dt = ds / cos t, cos^2 t = 1 - s^2,
// so a node needs no sine and rho no arcsine). As (h^2+k^2-2hks)/cos^2 t >=
// max(h^2, k^2), and >= h^2 + k^2 when hk rho <= 0, a corner whose bound
// exceeds 36 contributes below e^-18 (times asin(rho)/(2 pi) < 0.18) and is
// skipped.
// Every operation of Z is an explicitly rounded one (the paired intrinsics,
// fmaf, __fmul_rn, __fadd_rn), none left to the compiler to contract, so
// that every kernel (fused, staged, adjoint, reuse) computes the same Z bit
// for bit from the same guide.
__device__ __forceinline__ float rect_mass(const Params& P, float mx, float my, float isx, float isy, float rho) {
    const float h0 = __fmul_rn(-mx, isx), h1 = __fmul_rn(__fsub_rn(1.0f, mx), isx);
    const float k0 = __fmul_rn(-my, isy), k1 = __fmul_rn(__fsub_rn(1.0f, my), isy);
    // the tails of both axes in pairs: (T(-h0), T(-k0)) and (T(h1), T(k1))
    const float2 ta = normal_tail2(make_float2(-h0, -k0)), tb = normal_tail2(make_float2(h1, k1));
    const float2 dp = sub2(sub2(dup2(1.0f), ta), tb);
    float z = __fmul_rn(dp.x, dp.y);
    const float h0s = __fmul_rn(h0, h0), h1s = __fmul_rn(h1, h1), k0s = __fmul_rn(k0, k0), k1s = __fmul_rn(k1, k1);
    // a corner contributes below e^-18 when its exponent bound exceeds 18:
    // (h^2 + k^2)/2 if h k rho <= 0 (the cross term only adds), else max(h^2, k^2)/2
    auto live = [&](float h, float k, float hs, float ks) {
        const float bound = (__fmul_rn(__fmul_rn(h, k), rho) <= 0.0f) ? __fadd_rn(hs, ks) : fmaxf(hs, ks);
        return bound <= 36.0f;
    };
    const bool c00 = live(h0, k0, h0s, k0s), c10 = live(h1, k0, h1s, k0s);
    const bool c01 = live(h0, k1, h0s, k1s), c11 = live(h1, k1, h1s, k1s);
    if (rho != 0.0f && (c00 || c10 || c01 || c11)) {
        // exponent of corner (h, k) in base 2: (2hk s - h^2 - k^2) log2(e) / (2 cos^2 t)
        const float l2 = 0.72134752044448170f;                  // log2(e) / 2
        auto a_of = [&](float hs, float ks) { return __fmul_rn(__fadd_rn(hs, ks), l2); };
        auto b_of = [&](float h, float k) { return __fmul_rn(__fmul_rn(__fmul_rn(2.0f, h), k), l2); };
        const float a00 = a_of(h0s, k0s), b00 = b_of(h0, k0);
        const float a11 = a_of(h1s, k1s), b11 = b_of(h1, k1);
        const float a10 = a_of(h1s, k0s), b10 = b_of(h1, k0);
        const float a01 = a_of(h0s, k1s), b01 = b_of(h0, k1);
        auto corner = [](float b, float a, float2 s, float2 q) {
            const float2 e = mul2(fma2(dup2(b), s, dup2(-a)), q);
            return make_float2(exp2_approx(e.x), exp2_approx(e.y));
        };
        float acc = 0.0f;
        // two nodes at a time, each half of a pair one node: s = rho c,
        // cos^2 t = 1 - s^2 >= 0.19, q = 1 / cos^2 t, the weight w / cos t
#pragma unroll
        for (int i = 0; i < kZNodes; i += 2) {
            const float2 s = mul2(dup2(rho), make_float2(P.zq_c[i], P.zq_c[i + 1]));
            const float2 om = fma2(neg2(s), s, dup2(1.0f));
            const float2 q = make_float2(__fdividef(1.0f, om.x), __fdividef(1.0f, om.y));
            const float2 wr = mul2(make_float2(P.zq_w[i], P.zq_w[i + 1]), make_float2(rsqrtf(om.x), rsqrtf(om.y)));
            float2 v = dup2(0.0f);
            if (c00) v = add2(v, corner(b00, a00, s, q));
            if (c11) v = add2(v, corner(b11, a11, s, q));
            if (c10) v = sub2(v, corner(b10, a10, s, q));
            if (c01) v = sub2(v, corner(b01, a01, s, q));
            acc = fmaf(wr.x, v.x, acc);
            acc = fmaf(wr.y, v.y, acc);
        }
        z = fmaf(acc, __fmul_rn(rho, kInv2Pi), z);
    }
    return z;
}

// Everything of the derived guide but Z (left at 1).
__device__ __forceinline__ Guide derive_guide_shape(const Params& P, const Gam& g, bool gated) {
    Guide d;
    d.mx = fminf(fmaxf(g.ex, 0.0f), 1.0f);
    d.my = fminf(fmaxf(g.ey, 0.0f), 1.0f);
    d.sxx = fmaxf(g.sxx, P.sigma2_min);
    d.syy = fmaxf(g.syy, P.sigma2_min);
    const float isy = rsqrtf(d.syy);
    d.il11 = rsqrtf(d.sxx);
    const float lim = P.rho_max * d.sxx * d.il11 * d.syy * isy;   // rho_max sqrt(sxx syy)
    d.sxy = fminf(fmaxf(g.sxy, -lim), lim);
    d.l11 = d.sxx * d.il11;
    d.l21 = d.sxy * d.il11;
    const float c22 = fmaf(-d.l21, d.l21, d.syy);
    d.il22 = rsqrtf(c22);
    d.l22 = c22 * d.il22;
    d.pnorm = kInv4Pi2 * d.il11 * d.il22;
    d.pi_eff = gated ? 0.0f : g.pi;
    d.Z = 1.0f;
    return d;
}

__device__ __forceinline__ Guide derive_guide(const Params& P, const Gam& g, bool gated) {
    Guide d = derive_guide_shape(P, g, gated);
    if (d.pi_eff > 0.0f) {
        const float isy = rsqrtf(d.syy);
        d.Z = rect_mass(P, d.mx, d.my, d.il11, isy, d.sxy * d.il11 * isy);
    }
    return d;
}

// Guide density per steradian at square point u: N(u; mu, Sigma) / (2 pi).
__device__ __forceinline__ float guide_pdf(const Guide& d, float ux, float uy) {
    const float y1 = (ux - d.mx) * d.il11;
    const float y2 = (uy - d.my - d.l21 * y1) * d.il22;
    return __expf(-0.5f * (y1 * y1 + y2 * y2)) * d.pnorm;
}

// ---------------------------------------------------------------------------
// Surface: basis, view direction, material (Eq. 1's f_r). The roughness slot
// codes the material: >= 0 GGX, in (-1.5, 0) Lambertian, <= -1.5 transparent.
// Lambert: f_r = albedo / pi, cosine-weighted draws.
// GGX (Walter et al. 2007): alpha = roughness^2 (>= 1e-4), separable Smith
// shadowing, Schlick's Fresnel F0 + (1 - F0)(1 - o.h)^5 (F0 = 1: F = 1); the
// draw picks h ~ D(h) cos(theta_h) and reflects w_o.
// Transparent (Sec. 5, guiding off): a smooth dielectric of index 1.5 that
// reflects w_o with its Fresnel reflectance and refracts it otherwise; its
// draws are deltas, with no finite f_r or density.
// ---------------------------------------------------------------------------
struct Surf {
    Basis f;
    float3 wo;      // local view direction
    float3 pos;     // world shading point
    float a2;       // alpha^2 (GGX)
    float albedo;
    float go;       // GGX: albedo G1(w_o) / (4 cos theta_o), 0 when back-facing
    int mat;        // MAT_GGX, MAT_LAMBERT or MAT_GLASS
};
enum { MAT_GGX = 0, MAT_LAMBERT = 1, MAT_GLASS = 2 };

// Unpolarised Fresnel reflectance of the index-1.5 dielectric for light from
// outside at cosine ci > 0.
__device__ __forceinline__ float dielectric_fresnel(float ci) {
    const float n = 1.5f, ct = sqrtf(1.0f - (1.0f - ci * ci) * (1.0f / (n * n)));
    const float rs = fdiv(ci - n * ct, ci + n * ct), rp = fdiv(n * ci - ct, n * ci + ct);
    return 0.5f * (rs * rs + rp * rp);
}


// GLASS = false compiles the transparent material out (its code is then
// Lambertian, as without P.glass); the kernels that always support it pass
// true and honour P.glass at run time.
template <bool GLASS = true>
__device__ __forceinline__ Surf make_surf(const Params& P, int x, int y, float4 g0, float4 g1) {
    Surf s;
    float3 o, d;
    if (P.cam_kind == 0) {
        const float sx = ((float)x + 0.5f) * P.cam_ps, sy = ((float)y + 0.5f) * P.cam_ps;
        o = make_float3(P.cam_o[0] + sx * P.cam_r[0] + sy * P.cam_u[0], P.cam_o[1] + sx * P.cam_r[1] + sy * P.cam_u[1],
                        P.cam_o[2] + sx * P.cam_r[2] + sy * P.cam_u[2]);
        d = f3(P.cam_f);
    } else {
        const float sx = (2.0f * ((float)x + 0.5f) / (float)P.W - 1.0f) * P.cam_tan * P.cam_aspect;
        const float sy = (1.0f - 2.0f * ((float)y + 0.5f) / (float)P.H) * P.cam_tan;
        float3 v = make_float3(P.cam_f[0] + sx * P.cam_r[0] + sy * P.cam_u[0], P.cam_f[1] + sx * P.cam_r[1] + sy * P.cam_u[1],
                               P.cam_f[2] + sx * P.cam_r[2] + sy * P.cam_u[2]);
        const float il = rsqrtf(dot3(v, v));
        d = make_float3(v.x * il, v.y * il, v.z * il);
        o = f3(P.cam_o);
    }
    s.pos = make_float3(o.x + g0.w * d.x, o.y + g0.w * d.y, o.z + g0.w * d.z);
    s.f = make_basis(make_float3(g0.x, g0.y, g0.z));
    s.wo = to_local(s.f, make_float3(-d.x, -d.y, -d.z));
    s.mat = g1.z >= 0.0f ? MAT_GGX : ((GLASS && P.glass && g1.z <= -1.5f) ? MAT_GLASS : MAT_LAMBERT);
    const float a = fmaxf(g1.z * g1.z, 1e-4f);
    s.a2 = a * a;
    s.albedo = g1.w;
    // albedo G1(w_o) / (4 cos_o) with Smith's G1(c) = 2c / (c + sqrt(a^2 + (1 - a^2) c^2)):
    // the cosines cancel, leaving albedo / (2 (c + e)), e >= alpha >= 1e-4
    s.go = s.wo.z > 0.0f
               ? __fdividef(0.5f * g1.w, s.wo.z + sqrt_approx(fmaf(1.0f - s.a2, s.wo.z * s.wo.z, s.a2)))
               : 0.0f;
    return s;
}

// GGX f_r cos(theta_i) and its draw's density at local wi, from the cosines
// of the unit half vector h: ct = n.h, st2 = 1 - (n.h)^2, oh = w_o.h (> 0).
// With D = a^2 / (pi t^2), t = a^2 ct^2 + st2 (= (n.h)^2 (a^2 - 1) + 1, free
// of cancellation), Smith's G1(w_i) = 2 c / e, e = c + sqrt(a^2 + (1 - a^2) c^2):
//   f_r cos = D G1(w_i) go F,  p_b = D ct / (4 oh),
// both through one reciprocal r = 1 / (pi t^2 e oh).
__device__ __forceinline__ void ggx_eval(const Surf& s, float wiz, float ct, float st2, float oh, float& fcos,
                                         float& pb, float f0) {
    const float t = fmaf(s.a2, ct * ct, st2);
    const float e = wiz + sqrt_approx(fmaf(1.0f - s.a2, wiz * wiz, s.a2));
    const float den = kPi * t * t * e * oh;
    const float sc = den > 1e-30f ? 1.0f : 18446744073709551616.0f;   // as fdiv
    const float r = __fdividef(sc, den * sc);
    const float a2r = s.a2 * r;
    fcos = a2r * 2.0f * wiz * oh * s.go;
    if (f0 < 1.0f) {
        const float m = 1.0f - oh, m2 = m * m;
        fcos *= fmaf(1.0f - f0, m2 * m2 * m, f0);
    }
    pb = a2r * ct * e * 0.25f;
}

// The half vector's cosines of a direction pair: h = w_o + w_i normalised.
// (Near a grazing mirror pair w_i ~ -w_o reflected, h's components cancel in
// binary32: a direction the GGX sampler drew carries its own h instead.)
__device__ __forceinline__ void half_cosines(const Surf& s, float3 wi, float& ct, float& st2, float& oh) {
    const float3 h = make_float3(s.wo.x + wi.x, s.wo.y + wi.y, s.wo.z + wi.z);
    const float hz2 = h.z * h.z, hxy2 = h.x * h.x + h.y * h.y, hl2 = hz2 + hxy2;
    const float ihl = rsqrtf(hl2);
    ct = h.z * ihl;
    st2 = hxy2 * ihl * ihl;
    oh = dot3(s.wo, h) * ihl;
}

// f_r cos(theta_i) and the BRDF draw's density (per steradian) at local wi.
// f0: Schlick reflectance of the GGX lobe at normal incidence (1: F = 1).
__device__ __forceinline__ void brdf_eval(const Surf& s, float3 wi, float& fcos, float& pb, float f0) {
    if (!(wi.z > 0.0f) || s.mat == MAT_GLASS) {
        fcos = 0.0f;
        pb = 0.0f;
        return;
    }
    if (s.mat == MAT_LAMBERT) {
        pb = wi.z * kInvPi;
        fcos = s.wo.z > 0.0f ? s.albedo * pb : 0.0f;
        return;
    }
    float ct, st2, oh;
    half_cosines(s, wi, ct, st2, oh);
    if (!(s.wo.z > 0.0f) || !(oh > 0.0f)) {
        fcos = 0.0f;
        pb = 0.0f;
        return;
    }
    ggx_eval(s, wi.z, ct, st2, oh, fcos, pb, f0);
}

// The draw of a transparent surface: reflection when x1 < F, refraction (into
// the lower hemisphere) otherwise; viewed from below it wastes the draw.
__device__ __forceinline__ bool glass_sample(const Surf& s, float x1, float3& wi) {
    const float ci = s.wo.z;
    if (!(ci > 0.0f)) {
        wi = make_float3(0.0f, 0.0f, 1.0f);
        return false;
    }
    if (x1 < dielectric_fresnel(ci)) {
        wi = make_float3(-s.wo.x, -s.wo.y, ci);
    } else {
        const float eta = 1.0f / 1.5f, ct = sqrtf(1.0f - eta * eta * (1.0f - ci * ci));
        wi = make_float3(-eta * s.wo.x, -eta * s.wo.y, -ct);
    }
    return true;
}

// BRDF draw from a uniform x1 and the sine and cosine of a uniform turn x2
// (Lambertian or GGX); false for a wasted draw (below the horizon). A GGX
// draw also returns its half vector's cosines ct = n.h, st2 = 1 - (n.h)^2
// and oh = w_o.h, with which it is evaluated (see half_cosines).
__device__ __forceinline__ bool brdf_sample_sc(const Surf& s, float x1, float sn, float cs, float3& wi, float& hct,
                                               float& hst2, float& hoh) {
    if (s.mat == MAT_LAMBERT) {
        const float r = sqrt_approx(x1);
        wi = make_float3(r * cs, r * sn, sqrt_approx(1.0f - x1));
        return true;
    }
    const float id = __fdividef(1.0f, (1.0f - x1) + s.a2 * x1);
    const float st2 = s.a2 * x1 * id;
    const float ct = sqrt_approx((1.0f - x1) * id), st = sqrt_approx(st2);
    const float3 h = make_float3(st * cs, st * sn, ct);
    const float oh = dot3(s.wo, h);
    wi = make_float3(2.0f * oh * h.x - s.wo.x, 2.0f * oh * h.y - s.wo.y, 2.0f * oh * h.z - s.wo.z);
    hct = ct;
    hst2 = st2;
    hoh = oh;
    return oh > 0.0f && wi.z > 0.0f;
}

// ---------------------------------------------------------------------------
// Analytic incident radiance (stand-in for the traced ray of Fig. 2).
// Each lobe is amp * C_k exp(-k |w - d|^2 / 2) (= amp * C_k exp(k (d.w - 1))
// for unit vectors, in a form that keeps its precision near the peak).
// ---------------------------------------------------------------------------
// sqrt(2) sin(pi x / 2) for each half of x in [0, 1/2]: x P(x^2) with P of
// degree 3, this library's own fit (fit_mask_sine.py; relative error 3e-9,
// 1.3e-7 in binary32). Its square is 1 - cos(pi x) to 3.2e-7 relative.
__device__ __forceinline__ float2 sqrt2_sin_half_pi(float2 x) {
    const float2 x2 = mul2(x, x);
    float2 p = dup2(-6.507568864e-03f);
    p = fma2(p, x2, dup2(1.126845176e-01f));
    p = fma2(p, x2, dup2(-9.135302789e-01f));
    p = fma2(p, x2, dup2(2.221441462e+00f));
    return mul2(p, x);
}

// The occlusion mask m = (1 + sin(pi A) cos(pi B)) / 2, A and B in
// half-turns. Both phases are reduced exactly to [-1, 1] (A - 2 rint(A/2) is
// representable), then written through the distance e of A to the nearest
// half-integer and the distance d of B to the nearest integer:
// |sin(pi A)| = 1 - vs, |cos(pi B)| = 1 - vc with vs = 1 - cos(pi e) and
// vc = 1 - cos(pi d), each from the fitted sine without cancellation. Where
// the product is negative m = (vs + vc - vs vc) / 2, so m keeps its relative
// precision as it approaches 0; elsewhere m = (1 + (1 - vs)(1 - vc)) / 2.
__device__ __forceinline__ float occlusion_mask(float A, float B) {
    const float2 ab = make_float2(A, B);
    const float2 h = mul2(ab, dup2(0.5f));
    const float2 r = fma2(dup2(-2.0f), make_float2(rintf(h.x), rintf(h.y)), ab);
    const float ar = fabsf(r.x), br = fabsf(r.y);
    const float e = fabsf(0.5f - ar);      // exact for ar >= 1/4 (Sterbenz)
    const float d = fminf(br, 1.0f - br);  // exact
    const float2 q = sqrt2_sin_half_pi(make_float2(e, d));
    const float2 v = mul2(q, q);           // (vs, vc)
    const bool neg = (r.x < 0.0f) != (br > 0.5f);
    return neg ? 0.5f * fmaf(-v.x, v.y, v.x + v.y) : 0.5f * fmaf(1.0f - v.x, 1.0f - v.y, 1.0f);
}

// The first 2 NP lobes, two per paired operation (each half the scalar
// operations of one lobe), summed in lobe order into s (and the channels).
// A lobe beyond n_lobes has scale 0 and exponent 0: it adds exactly 0.
template <int NP, bool RGB>
__device__ __forceinline__ void lobe_sums(const Params& P, float3 w, float& s, float& sr, float& sg, float& sb) {
    const float2 wx = dup2(w.x), wy = dup2(w.y), wz = dup2(w.z);
#pragma unroll
    for (int jp = 0; jp < NP; ++jp) {
        const int j = 2 * jp;
        const float2 dx = add2(wx, P.lobe_pnx[jp]), dy = add2(wy, P.lobe_pny[jp]), dz = add2(wz, P.lobe_pnz[jp]);
        const float2 q = mul2(P.lobe_pe2[jp], fma2(dx, dx, fma2(dy, dy, mul2(dz, dz))));
        const float e0 = exp2_approx(q.x), e1 = exp2_approx(q.y);
        s = fmaf(P.lobe_scale[j], e0, s);
        s = fmaf(P.lobe_scale[j + 1], e1, s);
        if (RGB) {
            sr = fmaf(P.lobe_rgb[j][0], e0, sr);
            sg = fmaf(P.lobe_rgb[j][1], e0, sg);
            sb = fmaf(P.lobe_rgb[j][2], e0, sb);
            sr = fmaf(P.lobe_rgb[j + 1][0], e1, sr);
            sg = fmaf(P.lobe_rgb[j + 1][1], e1, sg);
            sb = fmaf(P.lobe_rgb[j + 1][2], e1, sb);
        }
    }
}

// Returns the radiance's luminance (the field itself when monochrome); with
// RGB, *rgb receives its three channels (coloured fields). One branch on the
// field's lobe count (the same for every lane) picks straight-line code for
// 2, 4 or 8 lobes: a branch per lobe pair costs more than the pairs it skips
// (measured: the 8-lobe 4K frame 5% faster without them).
template <bool RGB = false>
__device__ __forceinline__ float radiance(const Params& P, float3 pos, float3 w, float3* rgb = nullptr) {
    float s = 0.0f, sr = 0.0f, sg = 0.0f, sb = 0.0f;
    if (P.n_lobes > 4) {
        lobe_sums<4, RGB>(P, w, s, sr, sg, sb);
    } else if (P.n_lobes > 2) {
        lobe_sums<2, RGB>(P, w, s, sr, sg, sb);
    } else if (P.n_lobes > 0) {
        lobe_sums<1, RGB>(P, w, s, sr, sg, sb);
    }
    if (P.mask_kind == 1) {
        const float m = occlusion_mask(2.0f * (P.mask[0] * pos.x + P.mask[2] * w.x),
                                       2.0f * (P.mask[1] * pos.y + P.mask[2] * w.y));
        s *= m;
        if (RGB) {
            sr *= m;
            sg *= m;
            sb *= m;
        }
    }
    if (RGB) *rgb = make_float3(sr + P.field_const_rgb[0], sg + P.field_const_rgb[1], sb + P.field_const_rgb[2]);
    return s + P.field_const;
}

// ---------------------------------------------------------------------------
// One sample of the path-tracing pass (Sec. 3.1, Eq. 2): strategy choice,
// Box-Muller guide draw through the Cholesky factor and M, fallback to the
// BRDF outside the square, evaluation of radiance, pdfs and the estimate.
// ---------------------------------------------------------------------------
struct Smp {
    float3 wl;        // local direction
    float ux, uy;     // square coordinate of wl
    float L, fcos;    // radiance (luminance) and L f_r cos
    float pg, pb, pmix, F, mis;
    int strat;        // ST_* | ST_INVALID
    float3 Lrgb;      // coloured fields: the radiance's channels
    float wgt;        // coloured fields: the estimate per unit radiance (F = wgt L per channel)
    bool hs;          // a GGX BRDF draw: its half vector's cosines hct, hst2, hoh
    float hct, hst2, hoh;
};

template <bool RGB = false>
__device__ __forceinline__ void eval_sample(const Params& P, const Guide& d, const Surf& s, Smp& o, bool have_u) {
    const float3 ww = to_world(s.f, o.wl);
    o.L = radiance<RGB>(P, s.pos, ww, &o.Lrgb);
    o.wgt = 0.0f;
    if (o.strat & ST_INVALID) {
        o.fcos = o.pg = o.pb = o.pmix = o.F = o.mis = 0.0f;
        return;
    }
    if (o.strat == ST_DELTA) {
        // the Fresnel weight of the chosen branch cancels its probability
        o.fcos = o.pg = o.pb = o.pmix = 0.0f;
        o.ux = o.uy = -1.0f;
        o.F = s.albedo * o.L;
        o.wgt = s.albedo;
        o.mis = 1.0f;
        return;
    }
    float fr;
    if (s.mat == MAT_GGX && o.wl.z > 0.0f && s.wo.z > 0.0f) {
        // the draw's own half vector, or w_o + w_i for a direction the guide drew
        if (!o.hs) half_cosines(s, o.wl, o.hct, o.hst2, o.hoh);
        if (o.hoh > 0.0f) {
            ggx_eval(s, o.wl.z, o.hct, o.hst2, o.hoh, fr, o.pb, P.f0);
        } else {
            fr = 0.0f;
            o.pb = 0.0f;
        }
    } else {
        brdf_eval(s, o.wl, fr, o.pb, P.f0);
    }
    o.fcos = o.L * fr;
    if (!have_u) {
        const float2 u = hemi_to_square(o.wl);
        o.ux = u.x;
        o.uy = u.y;
    }
    o.pg = guide_pdf(d, o.ux, o.uy);
    const float wb = (1.0f - d.pi_eff * d.Z) * o.pb;
    const float wg = d.pi_eff * o.pg;
    o.pmix = wg + wb;
    if (o.pmix > 0.0f) {
        o.F = fdiv(o.fcos, o.pmix);
        if (RGB) o.wgt = fdiv(fr, o.pmix);
        o.mis = fdiv((o.strat & 3) == ST_GUIDE ? wg : wb, o.pmix);
    } else {
        o.F = 0.0f;
        o.mis = 0.0f;
    }
}

// Random numbers: one Philox call per sample, at counter (pixel, frame,
// sample, stream0) with stream0 = 0 for the pass and 2 for the adjoint's
// draws. The top 24 bits of word 0 pick the strategy; those of words 1 and 2
// drive Box-Muller for a guide draw or the BRDF draw otherwise (independent
// of word 0, hence still uniform given the choice); a guide draw that left
// the square takes its BRDF draw from word 3 and the low bytes of words 0-2.
template <bool RGB = false>
__device__ __forceinline__ Smp draw_sample(const Params& P, const Guide& d, const Surf& s, uint32_t pix,
                                           uint32_t frame, uint32_t si, uint32_t stream0 = 0u) {
    Smp o;
    const uint4 r0 = philox4x32_10(make_uint4(pix, frame, si, stream0), P.rk);
    const float zeta = unit24(r0.x);
    bool have_u = false, valid = false, brdf = false;
    o.hs = false;
    // word 2's turn is the Box-Muller angle of a guide draw and the azimuth of
    // a BRDF draw: one sincos serves the lanes of either strategy
    float sn, cs, x1 = unit24(r0.y);
    sincos_turn(unit24(r0.z), &sn, &cs);
    if (s.mat == MAT_GLASS) {
        // a transparent surface (always gated): one of its two deltas
        o.strat = ST_DELTA;
        valid = glass_sample(s, x1, o.wl);
    } else if (zeta < d.pi_eff) {
        const float rr = sqrt_approx(-2.0f * __logf(unit24_open0(r0.y)));
        const float z1 = rr * cs, z2 = rr * sn;
        o.ux = fmaf(d.l11, z1, d.mx);
        o.uy = fmaf(d.l22, z2, fmaf(d.l21, z1, d.my));
        if (o.ux >= 0.0f && o.ux <= 1.0f && o.uy >= 0.0f && o.uy <= 1.0f) {
            o.strat = ST_GUIDE;
            o.wl = square_to_hemi(o.ux, o.uy);
            valid = o.wl.z > 0.0f;
            have_u = true;
        } else {
            o.strat = ST_FALLBACK;
            // fresh uniforms from bits the draw has not used: word 3 and the
            // low bytes of words 0-2 (independent of their top 24 bits)
            const uint32_t spare = (r0.x & 0xFFu) | ((r0.y & 0xFFu) << 8) | ((r0.z & 0xFFu) << 16);
            x1 = unit24(r0.w);
            sincos_turn((float)spare * 5.9604644775390625e-8f, &sn, &cs);
            brdf = true;
        }
    } else {
        o.strat = ST_BRDF;
        brdf = true;
    }
    // the BRDF draw of both the BRDF strategy and a fallback, at one site
    if (brdf) {
        valid = brdf_sample_sc(s, x1, sn, cs, o.wl, o.hct, o.hst2, o.hoh);
        o.hs = s.mat == MAT_GGX;
    }
    if (!valid) o.strat |= ST_INVALID;
    eval_sample<RGB>(P, d, s, o, have_u);
    return o;
}

// ---------------------------------------------------------------------------
// Gradient of Z with respect to (mu_x, mu_y, s_xx, s_yy, s_xy), from the
// corner form of Z and the bivariate normal cdf's derivatives
//   dPhi2/dh = phi(h) Phi((k - rho h)/sqrt(1-rho^2)),
//   dPhi2/dk = phi(k) Phi((h - rho k)/sqrt(1-rho^2)),
//   dPhi2/drho = exp(-(h^2 - 2 rho h k + k^2)/(2(1-rho^2))) / (2 pi sqrt(1-rho^2)),
// chained through h = (a - mu_x)/s_x, k = (b - mu_y)/s_y, rho = s_xy/(s_x s_y).
// ---------------------------------------------------------------------------
// Phi(x) of both halves from the fitted upper tail (normal_tail2): within
// 2e-7 absolute.
__device__ __forceinline__ float2 normal_cdf2(float2 x) {
    const float2 t = normal_tail2(make_float2(fabsf(x.x), fabsf(x.y)));
    return make_float2(x.x >= 0.0f ? 1.0f - t.x : t.x, x.y >= 0.0f ? 1.0f - t.y : t.y);
}

// exp(x) of both halves as 2^(x log2 e) by the hardware approximation.
__device__ __forceinline__ float2 exp2x(float2 x) {
    const float2 e = mul2(x, dup2(1.44269504088896341f));
    return make_float2(exp2_approx(e.x), exp2_approx(e.y));
}

// The two axes of each corner go in pairs: (h, k), (dPhi2/dh, dPhi2/dk) and
// the (s_xx, s_yy) and (mu_x, mu_y) components of the gradient.
__device__ __forceinline__ void rect_mass_grad(const Guide& d, float dz[5]) {
    const float isx = d.il11, isy = rsqrtf(d.syy);
    const float rho = d.sxy * isx * isy;
    const float om = fmaf(-rho, rho, 1.0f), ir1 = rsqrtf(om);
    const float c0 = 0.398942280401432678f;      // 1 / sqrt(2 pi)
    const float2 is = make_float2(isx, isy);
    const float2 is2h = mul2(mul2(is, is), dup2(0.5f));
    float2 dmu = dup2(0.0f), dsg = dup2(0.0f);
    float dxy = 0.0f;
#pragma unroll
    for (int cn = 0; cn < 4; ++cn) {
        const float a = (float)(cn & 1), b = (float)(cn >> 1);
        const float sg = (cn == 0 || cn == 3) ? 1.0f : -1.0f;
        const float2 hk = mul2(make_float2(a - d.mx, b - d.my), is);          // (h, k)
        const float2 kh = make_float2(hk.y, hk.x);
        // (dPhi2/dh, dPhi2/dk) = phi(h) Phi((k - rho h)/sqrt(1 - rho^2)), and with h, k swapped
        const float2 dhk = mul2(mul2(dup2(c0), exp2x(mul2(dup2(-0.5f), mul2(hk, hk)))),
                                normal_cdf2(mul2(fma2(dup2(-rho), hk, kh), dup2(ir1))));
        const float h = hk.x, k = hk.y;
        const float dr = kInv2Pi * ir1 * __expf(-0.5f * (h * h - 2.0f * rho * h * k + k * k) / om);
        dmu = fma2(dup2(-sg), mul2(dhk, is), dmu);
        dsg = fma2(dup2(-sg), mul2(fma2(dhk, hk, dup2(dr * rho)), is2h), dsg);
        dxy = fmaf(sg * dr, isx * isy, dxy);
    }
    dz[0] = dmu.x;
    dz[1] = dmu.y;
    dz[2] = dsg.x;
    dz[3] = dsg.y;
    dz[4] = dxy;
}

// ---------------------------------------------------------------------------
// Weighted online EM (Sec. 3.2). Statistics over BRDF-strategy draws only, in
// binary32: the masses a = sum w g and b = sum w with Kahan compensation, and
// the batch's weighted mean and second central moment by West's incremental
// update (West 1979: each draw moves the mean by its weight's share of the
// running mass and adds its share of the spread), with w = f / p_b the
// luminance weight of the draw and g = pi p_g / p_mix its posterior for the
// guide. Unlike sums of (u - c)(u - c)^T about a fixed point c, from which the
// covariance follows only as a difference, no step of this update cancels,
// however unequal the weights (a bright draw after a dim one at another place
// leaves a batch covariance far below the square of their distance).
// ---------------------------------------------------------------------------
struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v) {
        const float y = __fsub_rn(v, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    // the first term of a sum is exact: no compensation to carry
    __device__ __forceinline__ void set(float v) { s = v; }
};

// Two Kahan sums advanced together, each half as Kahan::add.
struct Kahan2 {
    float2 s = {0.0f, 0.0f}, c = {0.0f, 0.0f};
    __device__ __forceinline__ void add(float2 v) {
        const float2 y = sub2(v, c);
        const float2 t = add2(s, y);
        c = sub2(sub2(t, s), y);
        s = t;
    }
    __device__ __forceinline__ void set(float2 v) { s = v; }
};

struct Stats {
    Kahan2 ab;          // (a, b)
    float2 m = {0.0f, 0.0f};   // weighted mean of the batch's square coordinates (weights w g)
    Kahan2 c2;          // weighted second central moments (M_xx, M_yy), times a
    Kahan c2xy;         // M_xy times a
    bool empty = true;
    __device__ __forceinline__ void add_train(const Guide& d, const Gam& g, const Smp& o) {
        if (o.strat != ST_BRDF || !(o.pb > 0.0f)) return;
        // w = f / p_b and gamma = pi p_g / p_mix through one reciprocal of
        // p_b p_mix (> 0: p_mix >= (1 - pi Z) p_b) while it is a normal number
        const float den = o.pb * o.pmix;
        float w, gam;
        if (den > 1e-30f && den < 1e30f) {
            const float r = __fdividef(1.0f, den);
            w = o.fcos * o.pmix * r;
            gam = d.pi_eff * o.pg * o.pb * r;
        } else {
            w = fdiv(o.fcos, o.pb);
            gam = o.pmix > 0.0f ? fdiv(d.pi_eff * o.pg, o.pmix) : 0.0f;
        }
        add(g, w, gam, o.ux, o.uy);
    }
    // One reused VPL (Sec. 3.2): world direction ww and radiance L of a
    // BRDF-strategy draw whose own pixel's BRDF drew it with density pb_src.
    // It enters with the importance weight f / pb_src and this pixel's
    // posterior, the own samples of the reuse path included.
    __device__ __forceinline__ void add_vpl(const Guide& d, const Gam& g, const Surf& s, float3 ww, float L,
                                            float pb_src, float f0) {
        const float3 wl = to_local(s.f, ww);
        if (!(wl.z > 0.0f) || !(pb_src > 0.0f)) return;
        float fr, pb;
        brdf_eval(s, wl, fr, pb, f0);
        const float2 u = hemi_to_square(wl);
        const float pg = guide_pdf(d, u.x, u.y);
        const float pmix = d.pi_eff * pg + (1.0f - d.pi_eff * d.Z) * pb;
        // w = L f_r / p_src and gamma = pi p_g / p_mix through one reciprocal
        // of p_src p_mix while that product is a normal number
        const float den = pb_src * pmix;
        float w, gam;
        if (den > 1e-30f && den < 1e30f) {
            const float r = __fdividef(1.0f, den);
            w = L * fr * pmix * r;
            gam = d.pi_eff * pg * pb_src * r;
        } else {
            w = fdiv(L * fr, pb_src);
            gam = pmix > 0.0f ? fdiv(d.pi_eff * pg, pmix) : 0.0f;
        }
        add(g, w, gam, u.x, u.y);
    }
    __device__ __forceinline__ void add(const Gam&, float w, float gam, float ux, float uy) {
        const float v = w * gam;
        if (empty) {
            ab.set(make_float2(v, w));
            m = make_float2(ux, uy);
            c2.set(dup2(0.0f));
            c2xy.set(0.0f);
            empty = false;
            return;
        }
        const float a0 = ab.s.x;
        ab.add(make_float2(v, w));
        const float a1 = ab.s.x;
        if (!(v > 0.0f) || !(a1 > 0.0f)) return;
        // t = v / a1, the draw's share of the mass; f = v a0 / a1
        const float t = fdiv(v, a1), f = t * a0;
        const float2 d = sub2(make_float2(ux, uy), m);
        m = fma2(d, dup2(t), m);
        const float2 fd = mul2(dup2(f), d);
        c2.add(mul2(fd, d));
        c2xy.add(fd.x * d.y);
    }
};

// M-step: a luminance-weighted running average filtered by the epoch count
// k (Sec. 3.2, 4.2). With eta = 1/(min(k, k_max) + 2) and the stored guide
// carrying mass M0 = W (for an untrained guide, the frame's own mass b):
//   A = (1-eta) pi M0 + eta a,  B = (1-eta) M0 + eta b,
//   E <- ((1-eta) pi M0 E + eta S) / A,  pi <- clamp(A/B),  W <- B,  k <- k+1.
// The moments are updated as a mixture of the stored guide and the frame's
// batch, with lambda = eta a / A and 1 - lambda = (1-eta) pi M0 / A:
//   mu' = mu + lambda delta,
//   Sigma' = (1-lambda) Sigma + lambda (C + (1-lambda) delta delta^T),
// delta = the batch mean minus mu, C = the batch covariance about its own
// mean. It is the same update in exact arithmetic, and every term of it is
// free of cancellation in binary32, also as lambda -> 1 (a frame whose mass
// dwarfs the stored guide's), where 1 - lambda formed as a difference, or
// lambda M2 - (lambda delta)^2 from moments about mu, would lose the small
// covariance that remains. ONE: at most one training sample (C = 0). A frame
// with b = 0 changes nothing.
template <bool ONE = false>
__device__ __forceinline__ void m_step(const Params& P, Gam& g, const Stats& st) {
    const float k = fmaxf(g.k, 0.0f);
    const float a = st.ab.s.x, b = st.ab.s.y;
    g.k = k;
    if (!(b > 0.0f)) return;
    const float eta = __fdividef(1.0f, fminf(k, (float)P.k_max) + 2.0f);   // an integer in [2, k_max + 2]
    const float m0 = (k > 0.0f && g.W > 0.0f) ? g.W : b;
    const float e1 = 1.0f - eta;
    const float keep = e1 * g.pi * m0;
    const float A = fmaf(eta, a, keep);
    const float B = fmaf(eta, b, e1 * m0);
    if (a > 0.0f && A > 0.0f) {
        // lambda and 1 - lambda by one hardware reciprocal of A while A is
        // normal (2 ulp, as fdiv's fast path), by correctly rounded divisions
        // for a subnormal A; the same for C over a
        float lam, l1, cxy = 0.0f;
        float2 c = dup2(0.0f);
        if (A > 1e-30f) {
            const float rA = __fdividef(1.0f, A);
            lam = eta * a * rA;
            l1 = keep * rA;
        } else {
            lam = __fdiv_rn(eta * a, A);
            l1 = __fdiv_rn(keep, A);
        }
        if (!ONE) {
            if (a > 1e-30f) {
                const float ra = __fdividef(1.0f, a);
                c = mul2(st.c2.s, dup2(ra));
                cxy = st.c2xy.s * ra;
            } else {
                c = make_float2(__fdiv_rn(st.c2.s.x, a), __fdiv_rn(st.c2.s.y, a));
                cxy = __fdiv_rn(st.c2xy.s, a);
            }
        }
        const float2 dl = sub2(st.m, make_float2(g.ex, g.ey));   // delta
        const float2 l1d = mul2(dup2(l1), dl);
        const float2 q = fma2(l1d, dl, c);             // C + (1 - lambda) delta delta^T
        const float qxy = fmaf(l1d.x, dl.y, cxy);
        const float2 sd = fma2(dup2(l1), make_float2(g.sxx, g.syy), mul2(dup2(lam), q));
        g.sxx = sd.x;
        g.syy = sd.y;
        g.sxy = fmaf(l1, g.sxy, lam * qxy);
        const float2 e = fma2(dup2(lam), dl, make_float2(g.ex, g.ey));
        g.ex = e.x;
        g.ey = e.y;
        raw_from_central(g);
    }
    g.pi = fminf(fmaxf(fdiv(A, B), P.pi_min), P.pi_max);
    g.W = B;
    g.k = fminf(k + 1.0f, (float)P.k_max);
}

}  // namespace pgk
