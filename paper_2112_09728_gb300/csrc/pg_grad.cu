// Kernels of the differentiable form (not in the paper): the adjoint of the
// per-pixel second-moment loss, the projected Adam step on the guide's
// parameters theta with binary32 or BF16 moments, and theta <-> Gamma.
#include "pg_common.cuh"

namespace pgk {

namespace {

// ---------------------------------------------------------------------------
// The differentiable form: the gradient of the per-pixel second-moment loss
// l(theta) = 1/n sum f_i^2 / (p_theta(w_i) p_theta0(w_i)) at theta = theta0,
// with the n directions drawn from the guide itself (Philox stream 2):
//   l = 1/n sum f^2 / p^2,  dl/dtheta = -1/n sum f^2 (dp/dtheta) / p^3,
//   dp/dpi = g - Z p_b,  dp/dmu = pi (g Sigma^-1 d - p_b dZ/dmu),
//   dp/dSigma = pi (g/2 (Sigma^-1 d d^T Sigma^-1 - Sigma^-1) - p_b dZ/dSigma)
// for theta = (mu_x, mu_y, s_xx, s_yy, s_xy, pi), s_xy a single parameter.
// ---------------------------------------------------------------------------
// The sums over the draws are factored so that nothing of Z's derivative is
// live in the loop: with c = -f^2/p^3 and cg = c p_g,
//   dl/dmu    ~ pi (sum cg Sigma^-1 d - dZ/dmu sum c p_b),
//   dl/dSigma ~ pi (1/2 (sum cg (Sigma^-1 d)(Sigma^-1 d)^T - Sigma^-1 sum cg) - dZ/dSigma sum c p_b),
//   dl/dpi    ~ sum cg - Z sum c p_b,
// eight binary32 sums (the loss, five of cg times a monomial of Sigma^-1 d,
// sum cg and sum c p_b); dZ/dtheta is taken once, after the loop.
// Eight blocks of 128 threads per SM (64 registers, no spills): 0.69 ms for
// the 3840x2160 orbit step at 4 draws. When the bound was chosen, the
// register count the compiler picks unbounded (two blocks of 256 per SM) ran
// a third slower, and five blocks of 256 (48 registers, more spills) a
// quarter slower, than four blocks of 256 with these 64 registers; blocks of
// 128 then gained 1% over blocks of 256 (a smaller last wave).
template <int DT, bool THETA>
__global__ void __launch_bounds__(kFrameBlock, 8) k_grad(const Params P, const void* __restrict__ gam,
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
    const bool guided = d.pi_eff > 0.0f;
    // Sigma^-1 = [[qxx, -qxy], [-qxy, qyy]]
    const float idet = fdiv(1.0f, fmaf(d.sxx, d.syy, -d.sxy * d.sxy));
    const float qxx = d.syy * idet, qyy = d.sxx * idet, qxy = d.sxy * idet;
    // plain binary32 sums: at most a few hundred draws of one pixel, whose
    // rounding (~n 2^-24 of the summed magnitudes) is far inside the
    // adjoint's 1e-3 parity bound; compensation cost ~5% of the kernel
    // (x, y) components in pairs: a = sum cg Sigma^-1 d, aa = sum cg (Sigma^-1 d)^2
    float l = 0.0f, axy = 0.0f, sg = 0.0f, sb = 0.0f;
    float2 a = dup2(0.0f), aa = dup2(0.0f);
    for (int si = 0; si < n; ++si) {
        const Smp o = draw_sample(P, d, s, (uint32_t)i, frame, (uint32_t)si, 2u);
        if ((o.strat & ST_INVALID) || o.fcos == 0.0f || !(o.pmix > 0.0f)) continue;
        const float ip = fdiv(1.0f, o.pmix), f2ip2 = o.fcos * o.fcos * ip * ip;
        l += f2ip2;
        if (!guided) continue;
        const float2 dd = sub2(make_float2(o.ux, o.uy), make_float2(d.mx, d.my));
        // Sigma^-1 d = (qxx dx - qxy dy, qyy dy - qxy dx)
        const float2 id = fma2(make_float2(qxx, qyy), dd, mul2(dup2(-qxy), make_float2(dd.y, dd.x)));
        const float c = -f2ip2 * ip, cg = c * o.pg;
        const float2 cid = mul2(dup2(cg), id);
        a = add2(a, cid);
        aa = fma2(cid, id, aa);
        axy = fmaf(cid.x, id.y, axy);
        sg += cg;
        sb = fmaf(c, o.pb, sb);
    }
    const float ax = a.x, ay = a.y, axx = aa.x, ayy = aa.y;
    const float in = 1.0f / (float)n;
    loss[i] = l * in;
    float gs[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (guided) {
        float dz[5];
        rect_mass_grad(d, dz);
        const float pe = d.pi_eff;
        gs[0] = pe * fmaf(-sb, dz[0], ax);
        gs[1] = pe * fmaf(-sb, dz[1], ay);
        gs[2] = pe * fmaf(-sb, dz[2], 0.5f * fmaf(-qxx, sg, axx));
        gs[3] = pe * fmaf(-sb, dz[3], 0.5f * fmaf(-qyy, sg, ayy));
        gs[4] = pe * fmaf(-sb, dz[4], fmaf(qxy, sg, axy));
        gs[5] = fmaf(-d.Z, sb, sg);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) grad[k * hw + i] = gs[k] * in;
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

}  // namespace

cudaError_t launch_grad(int dt, const Params& P, const void* gam, const float* theta, const float4* g0,
                        const float4* g1, uint32_t frame, int n, float* loss, float* grad, cudaStream_t st) {
    const dim3 grid = grid_for(P, kFrameBlock);
    if (theta) {
        PG_DISPATCH(dt, (k_grad<D, true><<<grid, kFrameBlock, 0, st>>>(P, gam, theta, g0, g1, frame, n, loss, grad)));
    } else {
        PG_DISPATCH(dt, (k_grad<D, false><<<grid, kFrameBlock, 0, st>>>(P, gam, theta, g0, g1, frame, n, loss, grad)));
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

}  // namespace pgk
