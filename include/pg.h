/*
 * pg.h - C ABI of the GB300 guide pass for screen-space path guiding with
 * parametric mixture models (Derevyannykh, "Real-Time Path-Guiding Based on
 * Parametric Mixture Models", arXiv 2112.09728).
 *
 * Each pixel keeps the 8-parameter texture Gamma (abstract; Sec. 3.1) of a
 * mixture (Eq. 2) of a 2D normal distribution on the Shirley-Chiu square and
 * the surface BRDF. Per frame the pass
 *   (a) reprojects last frame's Gamma by motion vectors with depth/normal
 *       rejection (Sec. 3.1),
 *   (b) draws guided directions with their mixture pdf and balance-heuristic
 *       MIS weight (Eq. 2, Sec. 3.1), and
 *   (c) runs one weighted online EM step from the BRDF-strategy samples
 *       (Sec. 3.2).
 * The traced incident radiance of the paper's path-tracing pass is replaced by
 * an analytic field (pg_field), evaluated in the kernel.
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are CUDA device pointers owned by the caller; the
 *    library never frees them. The context owns only Gamma (two buffers), a
 *    binary32 work copy for the staged calls, and the Adam moments.
 *  - All work is enqueued on the context's stream and is asynchronous; a call
 *    returns after the launch, not after the kernel finishes.
 *  - Arrays are row-major over pixels, index i = y * width + x. Per-sample
 *    arrays are sample-major: element (s, i) is at s * width * height + i.
 *  - Every call returns a pg_status and never aborts or throws. On an error the
 *    context keeps its previous Gamma, and pg_last_error() describes it.
 *  - The library does no host<->device synchronisation except in
 *    pg_get_gamma / pg_set_gamma with host buffers and in pg_check.
 */
#ifndef PG_H
#define PG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pg_ctx pg_ctx;

typedef enum {
    PG_OK = 0,
    PG_ERR_ARG = 1,      /* a null pointer, a bad size, a bad enum, aliasing buffers */
    PG_ERR_CUDA = 2,     /* a CUDA runtime error (launch or copy) */
    PG_ERR_OOM = 3,      /* device allocation failed */
    PG_ERR_STATE = 4,    /* call out of order (e.g. pg_update without pg_reproject) */
    PG_ERR_TIMEOUT = 5,  /* reserved for bounded device waits; no call waits today */
    PG_ERR_NUMERIC = 6,  /* the device flagged a non-finite Gamma (pg_check) */
    PG_ERR_BOUNDS = 7    /* bounds-checked build only (libpg_bounds.so): an index that depends on
                            the data fell outside its buffer; the access was skipped (pg_check) */
} pg_status;

/* Storage type of Gamma. PG_F32 stores the paper's raw moments
 * E[X], E[Y], E[X^2], E[Y^2], E[XY] (Sec. 3.1) as two float4 planes
 * {E[X], E[Y], E[X^2], E[Y^2]} and {E[XY], pi, k, W} (32 bytes per pixel);
 * W is the running luminance-weight mass that weighs a new frame's samples
 * against the stored moments (the paper's unnamed eighth parameter).
 * PG_F16 / PG_BF16 store one 16-byte record per pixel of eight halves
 * {mu_x, mu_y, s_xx, s_yy, s_xy, pi, k, W}: the mean and the CENTRAL second
 * moments, because raw second moments lose the covariance to cancellation at
 * 11 (8) significand bits. All arithmetic is binary32; only storage differs. */
typedef enum { PG_F32 = 0, PG_F16 = 1, PG_BF16 = 2 } pg_dtype;

/* Pass configuration. Values the paper fixes: pi_min = 0.05, pi_max = 0.95
 * (clamp, Sec. 3.2), pi_reinit = 0.05 and k = 0 for invalid history
 * (Sec. 3.1), k_max (Sec. 4.2). The others are this library's readings of
 * passages the paper leaves open (defaults in brackets):
 *   depth_tol  [0.1]  accept iff |d_prev - d_cur| <= depth_tol * d_cur (Sec. 3.1)
 *   normal_tol [0.9]  accept iff n_prev . n_cur >= normal_tol           (Sec. 3.1)
 *   rough_min  [0.1]  GGX pixels below this roughness use the BRDF only (Sec. 5)
 *   sigma2_min [1e-4] variance floor of the guide on the square
 *   rho_max    [0.9]  correlation clamp of the guide
 *   k_max      [32]   cap of the epoch counter; the EM step is 1/(min(k,k_max)+2)
 * init_mu / init_sigma (xx, yy, xy) / init_pi give the Gamma that pg_create
 * writes to every pixel; a rejected pixel is re-initialised with the same
 * mean and covariance but pi = pi_reinit, k = 0, W = 0.
 * reuse_radius [0] neighbour-VPL reuse (Sec. 3.2, 4.2), R in [0, 8]: with
 * R > 0 each pixel also trains on N = 5 + floor(15 (k_max - k) / k_max)
 * distinct BRDF-strategy samples of the (2R+1)^2 window around it (see
 * pg_frame). 0 turns reuse off.
 * stochastic_round [0] with FP16/BF16 storage, 1 rounds the Gamma written by
 * an EM step stochastically instead of to nearest: each field goes to one of
 * its two neighbours in the storage type with probability proportional to
 * proximity (unbiased), using 16 bits of Philox at counter (pixel, frame, 0,
 * 5) per field (field j: word j/2, bits 16 (j mod 2) and up). An update
 * smaller than half a storage ulp then still moves the guide on average.
 * pg_update takes `frame` from the pg_sample of its staged frame (0 without
 * one). Values
 * that are already representable are stored exactly either way.
 * ggx_f0 [1] Schlick reflectance of the GGX lobe at normal incidence, in
 * [0, 1]: f_r carries F = F0 + (1 - F0)(1 - o.h)^5; 1 gives F = 1.
 * transparent [0] 1 enables the transparent material (roughness codes
 * <= -1.5, see pg_gbuffer); with 0 every negative roughness code is
 * Lambertian and the fused kernel carries none of the transparent code.
 * adam_dtype [PG_F32] storage of the Adam moments m and v of pg_adam_step:
 * PG_F32, or PG_BF16 (12 bytes per pixel per moment instead of 24). BF16
 * moments are rounded stochastically when stored (round to nearest would
 * freeze v, whose update with beta2 = 0.999 is a thousandth of its value,
 * well below BF16's half ulp of 2^-9); the arithmetic is binary32 either
 * way. PG_F16 is refused (g^2 leaves its range). */
typedef struct {
    int32_t width, height;   /* screen size in pixels, each in [1, 32768] */
    int32_t spp;             /* samples per pixel per frame, in [1, 1024] */
    int32_t gamma_dtype;     /* pg_dtype */
    uint64_t seed;           /* Philox4x32-10 key: (low word, high word) */
    int32_t k_max;
    float pi_min, pi_max, pi_reinit;
    float depth_tol, normal_tol, rough_min, sigma2_min, rho_max;
    float init_mu[2], init_sigma[3], init_pi;
    int32_t reuse_radius;
    int32_t stochastic_round;
    float ggx_f0;
    int32_t transparent;
    int32_t adam_dtype;      /* pg_dtype: PG_F32 or PG_BF16 */
} pg_config;

/* Camera of one frame: the primary ray of pixel (x, y). Orthographic (kind 0):
 * origin + (x+0.5)*pixel_size*right + (y+0.5)*pixel_size*up, direction fwd.
 * Pinhole (kind 1): from origin along normalize(fwd + sx*right + sy*up), with
 * sx = (2(x+0.5)/W - 1) * tan_half_fov * W/H, sy = (1 - 2(y+0.5)/H) * tan_half_fov.
 * The view direction w_o (Eq. 1) is the reversed ray; the shading point is
 * ray origin + depth * ray direction. */
typedef struct {
    int32_t kind;
    float origin[3], fwd[3], right[3], up[3];
    float pixel_size, tan_half_fov;
} pg_camera;

/* The rasterised G-buffer of the current frame (Sec. 3.1): device float4
 * arrays of width*height elements, 16-byte aligned.
 *   g0[i] = {n_x, n_y, n_z, depth}   unit world normal, distance along the ray
 *   g1[i] = {mv_x, mv_y, roughness, albedo}
 * mv is the previous minus the current screen position in pixels. The
 * roughness slot codes the material: >= 0 GGX with alpha = roughness^2; in
 * (-1.5, 0) Lambertian (-1 by convention); <= -1.5, with the configuration's
 * `transparent` set, transparent (-2 by convention; Lambertian otherwise):
 * a smooth dielectric of index 1.5 that reflects or refracts the
 * view direction with its Fresnel reflectance. Guiding is off on transparent
 * surfaces (Sec. 5); their draws are deltas (strategy 3) that do not train,
 * their estimate is albedo * L along the chosen direction, and pg_eval and
 * pg_grad give them no finite f_r, density, loss or gradient (all 0). */
typedef struct {
    const float *g0;
    const float *g1;
    pg_camera camera;
} pg_gbuffer;

/* Analytic incident radiance standing in for the ray traced in the
 * path-tracing pass (Fig. 2): sum over lobes of amp * vMF(w; dir, kappa)
 * (normalised on the sphere), times the occlusion mask
 * 0.5 + 0.5 sin(2 pi (mask[0] x + mask[2] w_x)) cos(2 pi (mask[1] y + mask[2] w_y))
 * when mask_kind = 1 (x, y: world position of the shading point), plus
 * constant.
 * With rgb = 1 the field is coloured: lobe j carries amp_rgb[j] and the
 * constant is constant_rgb (amp and constant are ignored). The pass then
 * weighs its EM samples by the luminance of the radiance (Sec. 3.1),
 * Y = 0.2126 R + 0.7152 G + 0.0722 B (Rec. 709): sampling, densities, MIS
 * and training see the field's luminance, and the per-pixel estimates
 * written to d_img become three planes [3][H*W] (R, G, B). Per-sample
 * records (pg_samples) and pg_eval report the luminance. */
typedef struct {
    int32_t n_lobes;         /* 0..8 */
    float dir[8][3];
    float kappa[8];          /* > 0 */
    float amp[8];
    float constant;
    int32_t mask_kind;       /* 0 none, 1 sinusoidal mask */
    float mask[4];
    int32_t rgb;             /* 0 monochrome, 1 coloured (amp_rgb, constant_rgb) */
    float amp_rgb[8][3];
    float constant_rgb[3];
} pg_field;

/* Per-sample record of the path-tracing pass, the counterpart of the paper's
 * VPL texture Pi (Fig. 2): device planes of spp*width*height elements each.
 * Any plane may be NULL in pg_sample (not written); pg_update reads wx, wy,
 * wz, radiance and strategy. strategy: 0 BRDF draw, 1 guide draw,
 * 2 guide draw that left the square and fell back to a BRDF draw; +4 marks a
 * wasted draw (GGX reflection below the horizon), which carries no energy. */
typedef struct {
    float *wx, *wy, *wz;     /* world direction */
    float *radiance;         /* L_i(x, w) */
    float *pdf;              /* mixture pdf p_mix(w), per steradian */
    float *mis;              /* balance weight of the strategy that drew it */
    float *estimate;         /* F = L_i f_r cos / p_mix */
    uint8_t *strategy;
} pg_samples;

/* Fill *cfg with the defaults above for a width x height screen. */
void pg_config_default(pg_config *cfg, int32_t width, int32_t height);

/* Create a context: validates *cfg, allocates Gamma (2 buffers of
 * width*height*(32 or 16) bytes) on the current device and writes the initial
 * Gamma on `stream` (a cudaStream_t; NULL = legacy default stream).
 * Returns PG_ERR_ARG (bad config), PG_ERR_OOM, PG_ERR_CUDA. *out is NULL on
 * failure. */
pg_status pg_create(const pg_config *cfg, void *stream, pg_ctx **out);

/* Use another stream for subsequent calls. */
pg_status pg_set_stream(pg_ctx *ctx, void *stream);

/* Staged pass, step (a) (Sec. 3.1): reproject Gamma by the motion vectors of
 * `cur` into the binary32 work copy; d_g0_prev is last frame's g0.
 * d_accept (nullable, uint8 per pixel) receives 1 for reused history, 0 for a
 * re-initialised pixel. Must be followed by pg_sample and/or pg_update. */
pg_status pg_reproject(pg_ctx *ctx, const pg_gbuffer *cur, const float *d_g0_prev,
                       uint8_t *d_accept);

/* Staged pass, step (b) (Eq. 2, Sec. 3.1): draw spp guided directions per
 * pixel from the reprojected guide with Philox4x32-10 (counter = (pixel,
 * frame, sample, stream)), evaluate the analytic radiance, the mixture pdf,
 * the MIS weight and the estimate. d_img (nullable) receives the per-pixel
 * mean estimate. Requires a preceding pg_reproject. */
pg_status pg_sample(pg_ctx *ctx, const pg_gbuffer *cur, const pg_field *field, uint32_t frame,
                    const pg_samples *d_out, float *d_img);

/* Staged pass, step (c) (Sec. 3.2): one weighted online EM step from the
 * given samples (only BRDF-strategy draws train), written as the new Gamma:
 * with eta = 1/(min(k,k_max)+2), luminance weights w = f/p_b, posteriors
 * g = pi p_guide / p_mix, a = sum w g, b = sum w, S = sum w g (u, u u^T) and
 * prior mass M0 = W (b for an untrained guide): A = (1-eta) pi M0 + eta a,
 * B = (1-eta) M0 + eta b, E <- ((1-eta) pi M0 E + eta S)/A,
 * pi <- clamp(A/B, pi_min, pi_max), W <- B, k <- min(k+1, k_max).
 * Requires a preceding pg_reproject; ends the staged frame. */
pg_status pg_update(pg_ctx *ctx, const pg_gbuffer *cur, const pg_samples *d_in);

/* The whole frame, steps (a)-(c) fused in one kernel: reads Gamma(t-1), the
 * G-buffer and last frame's g0, writes Gamma(t) and d_img (per-pixel mean
 * estimate, nullable). Requires no staged frame in progress.
 * With reuse_radius R > 0 the frame runs as the paper's two passes (Fig. 2):
 * the path-tracing pass writes one VPL per sample into a buffer the context
 * owns (world direction, radiance, and the density of the pixel's BRDF draw
 * for a BRDF-strategy sample); the training pass then trains each pixel on
 * its own BRDF-strategy VPLs and on N picks of its window: N = 5 +
 * floor(15 (k_max - k) / k_max) for the reprojected k (at most the window's
 * ((2R+1)^2 - 1) spp candidates), the candidates (s + j t) mod C for
 * j < N, s = floor(r C / 2^32) with r word 0 of Philox at counter (pixel,
 * frame, 0, 4), t the smallest integer >= 0.618 C coprime with C; picks
 * off the screen are dropped. A reused VPL weighs f / p_src (f = L f_r cos at
 * this pixel, p_src the density of the draw at its own pixel). The staged
 * calls and pg_frame_noalloc do not reuse: they return PG_ERR_ARG when
 * reuse_radius > 0. */
pg_status pg_frame(pg_ctx *ctx, const pg_gbuffer *cur, const float *d_g0_prev,
                   const pg_field *field, uint32_t frame, float *d_img);

/* A run of whole frames from HOST memory (the end-to-end form of pg_frame;
 * the paper has no counterpart: it is this library's host pipeline). Frame t
 * (t < n_frames, frame index frame0 + t) reads h_g0 + t*H*W*4 and
 * h_g1 + t*H*W*4 (float4 per pixel, as in pg_gbuffer) with cameras[t], its
 * previous g0 being frame t-1's (for t = 0: h_g0_prev, or its own g0 when
 * NULL), and writes its per-pixel estimate to h_img + t*H*W (nullable; with a
 * coloured field three planes, at h_img + t*3*H*W). The
 * uploads, the frames and the read-backs run on three streams so that
 * neighbouring frames overlap; device rings of three g0, two g1 and two image
 * buffers are reused only after the frames that read them have finished.
 * The call returns when every frame's image is in host memory. Host buffers
 * should be page-locked (cudaHostAlloc / cudaHostRegister) for the copies to
 * overlap; pageable memory works but serialises them. Buffers, streams and
 * events are the context's, created on the first call (PG_ERR_OOM if that
 * fails). Requires no staged frame in progress. */
pg_status pg_frames_host(pg_ctx *ctx, int32_t n_frames, const float *h_g0, const float *h_g1,
                         const pg_camera *cameras, const pg_field *field, uint32_t frame0,
                         const float *h_g0_prev, float *h_img);

/* Evaluate the current guide (Eq. 2) at n_dirs caller-given world directions
 * per pixel, d_dirs [n_dirs][H*W][3]. d_out [7][n_dirs*H*W] receives p_guide,
 * p_brdf, p_mix (per steradian), the two balance weights, f_r cos and the
 * radiance. Uses the work copy between pg_reproject and pg_update, else
 * Gamma. */
pg_status pg_eval(pg_ctx *ctx, const pg_gbuffer *cur, const pg_field *field, int32_t n_dirs,
                  const float *d_dirs, float *d_out);

/* The differentiable form of the guide (not in the paper; a per-pixel
 * variance objective beside the EM step of Sec. 3.2). With theta =
 * (mu_x, mu_y, s_xx, s_yy, s_xy, pi) the guide's regularised mean,
 * covariance and mixing weight, n_samples directions w_i are drawn from the
 * guide at theta (Philox stream 2 of `frame`) and the loss is the Monte
 * Carlo second moment of the estimator, l = 1/n sum f_i^2 / p(w_i)^2; its
 * gradient with the draws held fixed is
 *   dl/dtheta = -1/n sum f_i^2 (dp/dtheta)(w_i) / p(w_i)^3,
 * including the dependence of the mixture pdf on Z. s_xy is one parameter
 * (its derivative covers both off-diagonal entries). A pixel whose guide is
 * gated off has a loss and a zero gradient.
 *   d_theta  [6][H*W] planes (nullable: theta of the current Gamma)
 *   d_loss   [H*W];  d_grad [6][H*W] planes. */
pg_status pg_grad(pg_ctx *ctx, const pg_gbuffer *cur, const pg_field *field, uint32_t frame,
                  int32_t n_samples, const float *d_theta, float *d_loss, float *d_grad);

/* One Adam step (Kingma & Ba) on theta of every pixel from d_grad
 * ([6][H*W]), projected back onto the guide's domain (mean in [0,1]^2,
 * variances >= sigma2_min, |rho| <= rho_max, pi in [pi_min, pi_max]) and
 * written into Gamma as moments; k and W are kept. The context owns the
 * moments (allocated on first use: binary32 [6][H*W] planes, or with BF16 one
 * 24-byte record {m_0..m_5, v_0..v_5} per pixel); step = 1 restarts them
 * from zero. The new m and v are formed in binary32 and the step uses them
 * before they are stored; with BF16 moments, moment n (m_0..m_5, then
 * v_0..v_5) of pixel i is stored stochastically with the 16 bits of Philox
 * word n/2 (of the 8 words of the calls at counters (i, step, 0, 6) and
 * (i, step, 1, 6)) at bit 16 (n mod 2) and up, as Gamma is under
 * stochastic_round. */
pg_status pg_adam_step(pg_ctx *ctx, const float *d_grad, float lr, float beta1, float beta2, float eps,
                       int32_t step);

/* The Adam moments m and v as binary32 [6][H*W] device planes: checkpoint
 * (get) and resume (set; BF16 moments are rounded to nearest, so values got
 * from a BF16 context are restored exactly). Resume by setting Gamma and the
 * moments, then calling pg_adam_step with the next step number. get fails
 * with PG_ERR_STATE before the first pg_adam_step or pg_set_adam_state. */
pg_status pg_get_adam_state(pg_ctx *ctx, float *d_m, float *d_v);
pg_status pg_set_adam_state(pg_ctx *ctx, const float *d_m, const float *d_v);

/* theta of every pixel ([6][H*W] planes) from Gamma, and back (projected as
 * in pg_adam_step; k and W are kept). */
pg_status pg_theta_from_gamma(pg_ctx *ctx, float *d_theta);
pg_status pg_theta_to_gamma(pg_ctx *ctx, const float *d_theta);

/* A whole staged frame (pg_reproject + pg_sample + pg_update) without a
 * context and without allocating any device memory, for callers that cannot
 * call cudaMalloc (an engine whose device memory is handed out by its own
 * allocator, code that must not allocate while frames are in flight). The
 * paper has no counterpart: it is a deployment variant of the staged pass.
 *   cfg          validated as in pg_create; width*height must not exceed
 *                262144 pixels (PG_ERR_ARG and a message on stderr otherwise)
 *   d_gamma_in   Gamma(t-1) in cfg->gamma_dtype's storage layout (read)
 *   d_gamma_out  Gamma(t), same layout (written); may equal d_gamma_in but
 *                must not otherwise overlap it
 *   d_samples    per-sample records as for pg_sample; wx, wy, wz, radiance
 *                and strategy are required, the other planes may be NULL
 *   d_img        per-pixel mean estimate (nullable); stream: a cudaStream_t
 * The work copy of Gamma lives in a fixed 8 MiB device array inside the
 * library, which every GPU that loads the library holds until the process
 * exits. The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and should come before any stream capture; the
 * address is kept for the life of the process, so after a cudaDeviceReset of
 * that device the entry point must not be called again. All
 * calls share the array and overwrite it, so calls whose work overlaps on the
 * GPU (different streams, different threads) race: order them on one stream.
 * A non-finite Gamma is not reported (there is no context to hold the flag). */
pg_status pg_frame_noalloc(const pg_config *cfg, const pg_gbuffer *cur, const float *d_g0_prev,
                           const pg_field *field, uint32_t frame, const void *d_gamma_in,
                           void *d_gamma_out, const pg_samples *d_samples, float *d_img,
                           void *stream);

/* Raw Gamma in its storage layout (pg_gamma_bytes bytes): checkpoint and
 * resume. Copies are stream-ordered; with a host buffer the call waits. */
size_t pg_gamma_bytes(const pg_ctx *ctx);
pg_status pg_get_gamma(pg_ctx *ctx, void *dst, int32_t dst_is_host);
pg_status pg_set_gamma(pg_ctx *ctx, const void *src, int32_t src_is_host);

/* Gamma as binary32 raw moments in the PG_F32 two-plane layout
 * (2 * H*W float4), whatever the storage type; the setter rounds to storage. */
pg_status pg_gamma_to_f32(pg_ctx *ctx, float *d_dst);
pg_status pg_gamma_from_f32(pg_ctx *ctx, const float *d_src);

/* The reprojected guide of a staged frame (between pg_reproject and
 * pg_update) as binary32 raw moments in the PG_F32 two-plane layout; k = -1
 * marks a re-initialised pixel, which samples from the BRDF alone. */
pg_status pg_get_reprojected(pg_ctx *ctx, float *d_dst);

/* Wait for the stream and read the device error flag: PG_ERR_NUMERIC if a
 * kernel stored a non-finite Gamma since the last check; in the
 * bounds-checked build (libpg_bounds.so, compiled with PG_BOUNDS_CHECK),
 * PG_ERR_BOUNDS if an index that depends on the data (the reprojected pixel,
 * a reused neighbour's sample) fell outside its buffer. The flag is cleared. */
pg_status pg_check(pg_ctx *ctx);

/* Philox4x32-10 (Salmon et al., SC'11), the counter-based generator behind
 * every random number of the pass: d_out[4i..4i+3] = Philox(d_ctr[4i..4i+3],
 * key) for i < n. use_curand != 0 computes the same words with cuRAND's
 * header implementation (a cross-check). No context needed; enqueued on
 * `stream`. */
pg_status pg_philox(const uint32_t *d_ctr, const uint32_t key[2], int64_t n, uint32_t *d_out,
                    int32_t use_curand, void *stream);

const char *pg_last_error(const pg_ctx *ctx);
void pg_destroy(pg_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* PG_H */
