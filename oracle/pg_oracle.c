/*
 * FP64 CPU oracle for the per-pixel guide pass of
 *   M. Derevyannykh, "Real-Time Path-Guiding Based on Parametric Mixture
 *   Models" (arXiv 2112.09728).
 *
 * TEST INFRASTRUCTURE ONLY. This is the slow, plain statement of what the
 * guide pass computes, written in double precision, one pixel at a time, in
 * the order the paper describes it. Only the test-suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it. It shares no code, header,
 * constant table or helper with the CUDA implementation, and it never reads
 * anything the CUDA implementation produced.
 *
 * Where the paper fixes a step, the comment names the section or equation.
 * Where the paper is silent, the function states the reading it implements.
 *
 * Decisions that turn floating-point values into integers (the reprojected
 * pixel index and the depth/normal acceptance test) are taken in IEEE binary32
 * with a fixed operation order, because the GPU kernel takes them in binary32.
 * This file must be compiled with -ffp-contract=off so those expressions are
 * not fused.
 *
 * Parity status per function is recorded beside each one ("pinned by ..." or
 * "parity unpinned").
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Public structs (mirrored by ctypes in oracle/__init__.py).               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t width, height, spp, k_max;
    uint32_t seed_lo, seed_hi;
    double pi_min, pi_max, pi_reinit;
    double depth_tol, normal_tol, rough_min, sigma2_min, rho_max;
    double init_mu[2], init_sigma[3];
    int32_t reuse_radius;    /* neighbour-VPL reuse window radius R (0: off) */
    double ggx_f0;           /* Schlick reflectance of GGX at normal incidence (1: F = 1) */
    int32_t transparent;     /* 1: roughness codes <= -1.5 are transparent, 0: Lambertian */
} or_config;

typedef struct {
    int32_t kind;            /* 0 orthographic, 1 pinhole */
    double origin[3], fwd[3], right[3], up[3];
    double pixel_size;       /* orthographic: world units per pixel */
    double tan_half_fov;     /* pinhole: tan of half the vertical field of view */
} or_camera;

typedef struct {
    int32_t n_lobes;
    double dir[8][3], kappa[8], amp[8];
    double constant;
    int32_t mask_kind;       /* 0 none, 1 sinusoidal occlusion mask */
    double mask[4];          /* f1, f2, g, unused */
    int32_t rgb;             /* 1: coloured lobes amp_rgb and constant constant_rgb */
    double amp_rgb[8][3];
    double constant_rgb[3];
} or_field;

/* Per-sample outputs of the sampling step, sample-major [s*HW + i]. */
typedef struct {
    double *wx, *wy, *wz;    /* world direction */
    double *radiance;        /* L_i(x, w) */
    double *pdf;             /* mixture pdf p_mix(w), solid angle */
    double *mis;             /* balance-heuristic weight of the drawing strategy */
    double *estimate;        /* F = L f_r cos / p_mix (0 for an invalid draw) */
    uint8_t *strategy;       /* 0 BRDF, 1 guide, 2 guide draw outside the square -> BRDF, 3 transparent delta */
    double *pg, *pb;         /* guide and BRDF pdfs (solid angle) at w */
    double *ux, *uy;         /* square coordinates used for the guide pdf */
    double *margin;          /* distance of the sample's own decisions to their thresholds */
} or_samples;

/* strategy byte: low two bits name the strategy, bit 2 marks a wasted draw
 * (a GGX reflection below the horizon), which contributes nothing */
enum { S_BRDF = 0, S_GUIDE = 1, S_FALLBACK = 2, S_DELTA = 3, S_INVALID = 4 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11): a Feistel-like network of 10 rounds; each      */
/* round multiplies words 0 and 2 by two odd constants, keeps hi and lo     */
/* halves, xors the high halves with the other words and the round key;    */
/* the key is advanced by two Weyl increments between rounds.               */
/* Pinned by the published known-answer vectors (tests/golden).             */
/* ------------------------------------------------------------------------ */
void or_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint64_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += weyl0; k1 += weyl1; }
        uint64_t p0 = mul0 * (uint64_t)c0;
        uint64_t p1 = mul1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void or_philox_many(int64_t n, const uint32_t *ctr, const uint32_t key[2], uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i) or_philox(ctr + 4 * i, key, out + 4 * i);
}

/* 24-bit uniform in [0, 1): top 24 bits of the word times 2^-24 (exact in
 * binary32 and binary64). */
static double unif(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }
/* 24-bit uniform in (0, 1], for the logarithm of Box-Muller. */
static double unif_open0(uint32_t w) { return (double)((w >> 8) + 1u) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------ */
/* Shirley-Chiu concentric map M (Eq. 2: the area-preserving map of        */
/* Shirley and Chiu): unit square -> unit disk by concentric squares, the   */
/* equal-area lift of the disk to the hemisphere, so dw = 2*pi du dv.       */
/* Pinned by: round trip, constant Jacobian 2*pi, boundary -> horizon,      */
/* centre -> pole, moments of the uniform hemisphere.                       */
/* ------------------------------------------------------------------------ */
void or_square_to_hemi(const double u[2], double w[3])
{
    double a = 2.0 * u[0] - 1.0, b = 2.0 * u[1] - 1.0;
    double r, phi;
    if (a == 0.0 && b == 0.0) { w[0] = 0.0; w[1] = 0.0; w[2] = 1.0; return; }
    if (fabs(a) > fabs(b)) { r = a; phi = (M_PI / 4.0) * (b / a); }
    else { r = b; phi = M_PI / 2.0 - (M_PI / 4.0) * (a / b); }
    double dx = r * cos(phi), dy = r * sin(phi);
    double r2 = r * r;
    double s = sqrt(2.0 - r2);
    w[0] = dx * s; w[1] = dy * s; w[2] = 1.0 - r2;
}

void or_hemi_to_square(const double w[3], double u[2])
{
    double z = w[2] < 0.0 ? 0.0 : w[2];
    double inv = 1.0 / sqrt(1.0 + z);
    double dx = w[0] * inv, dy = w[1] * inv;
    double r = sqrt(dx * dx + dy * dy);
    double a, b;
    if (r == 0.0) { u[0] = 0.5; u[1] = 0.5; return; }
    double phi = atan2(dy, dx);
    if (phi < -M_PI / 4.0) phi += 2.0 * M_PI;
    if (phi < M_PI / 4.0) { a = r; b = (4.0 / M_PI) * phi * r; }
    else if (phi < 3.0 * M_PI / 4.0) { b = r; a = -(4.0 / M_PI) * (phi - M_PI / 2.0) * r; }
    else if (phi < 5.0 * M_PI / 4.0) { a = -r; b = -(4.0 / M_PI) * (phi - M_PI) * r; }
    else { b = -r; a = (4.0 / M_PI) * (phi - 3.0 * M_PI / 2.0) * r; }
    u[0] = 0.5 * (a + 1.0); u[1] = 0.5 * (b + 1.0);
}

/* ------------------------------------------------------------------------ */
/* Orthonormal basis around the surface normal. The paper does not fix one; */
/* this is the branchless construction of Duff et al., "Building an         */
/* Orthonormal Basis, Revisited" (JCGT 2017).                               */
/* ------------------------------------------------------------------------ */
void or_basis(const double n[3], double t[3], double b[3])
{
    double sg = copysign(1.0, n[2]);
    double a = -1.0 / (sg + n[2]);
    double c = n[0] * n[1] * a;
    t[0] = 1.0 + sg * n[0] * n[0] * a; t[1] = sg * c; t[2] = -sg * n[0];
    b[0] = c; b[1] = sg + n[1] * n[1] * a; b[2] = -n[1];
}

/* The G-buffer's unit normal at g (binary32, unit only to ~6e-8),
 * normalised in FP64: the local frame is an orthonormal basis about it, so
 * a direction taken to the world and back is unchanged to FP64 rounding.
 * (With the binary32 vector as it stands the frame is orthonormal only to
 * ~6e-8, and a sample re-derived from its world direction moves by that
 * much: enough, for a GGX mirror reflection of a grazing view, where the half
 * vector w_o + w_i nearly cancels, to move its weight by percents.) */
static void unit_normal(const float *g, double n[3])
{
    double l = sqrt((double)g[0] * g[0] + (double)g[1] * g[1] + (double)g[2] * g[2]);
    for (int k = 0; k < 3; ++k) n[k] = g[k] / l;
}

static void to_world(const double n[3], const double l[3], double w[3])
{
    double t[3], b[3];
    or_basis(n, t, b);
    for (int i = 0; i < 3; ++i) w[i] = l[0] * t[i] + l[1] * b[i] + l[2] * n[i];
}

static void to_local(const double n[3], const double w[3], double l[3])
{
    double t[3], b[3];
    or_basis(n, t, b);
    l[0] = w[0] * t[0] + w[1] * t[1] + w[2] * t[2];
    l[1] = w[0] * b[0] + w[1] * b[1] + w[2] * b[2];
    l[2] = w[0] * n[0] + w[1] * n[1] + w[2] * n[2];
}

/* ------------------------------------------------------------------------ */
/* Normal distribution on the square and its mass Z on [0,1]^2.             */
/* ------------------------------------------------------------------------ */
typedef struct { double mx, my, sxx, syy, sxy; } gauss2;

/* N(u; mu, Sigma), plain bivariate normal density. */
double or_gauss_pdf(const double g5[5], const double u[2])
{
    double sxx = g5[2], syy = g5[3], sxy = g5[4];
    double det = sxx * syy - sxy * sxy;
    double dx = u[0] - g5[0], dy = u[1] - g5[1];
    double q = (syy * dx * dx - 2.0 * sxy * dx * dy + sxx * dy * dy) / det;
    return exp(-0.5 * q) / (2.0 * M_PI * sqrt(det));
}

typedef double (*fn1)(double x, const void *ctx);

static double simpson_rec(fn1 f, const void *c, double a, double b, double fa, double fm,
                          double fb, double whole, double eps, int depth)
{
    double m = 0.5 * (a + b), lm = 0.5 * (a + m), rm = 0.5 * (m + b);
    double flm = f(lm, c), frm = f(rm, c);
    double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
    double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
    double delta = left + right - whole;
    /* stop at the requested absolute error, or at 1e-14 of the piece itself:
     * binary64 cannot resolve less, and a smaller target never converges */
    double tol = 15.0 * eps, floor_rel = 1e-14 * fabs(left + right);
    if (tol < floor_rel) tol = floor_rel;
    if (depth <= 0 || fabs(delta) <= tol) return left + right + delta / 15.0;
    return simpson_rec(f, c, a, m, fa, flm, fm, left, 0.5 * eps, depth - 1) +
           simpson_rec(f, c, m, b, fm, frm, fb, right, 0.5 * eps, depth - 1);
}

/* Adaptive Simpson on [a,b]. */
static double simpson(fn1 f, const void *c, double a, double b, double eps)
{
    if (!(b > a)) return 0.0;
    double fa = f(a, c), fb = f(b, c), m = 0.5 * (a + b), fm = f(m, c);
    double whole = (b - a) / 6.0 * (fa + 4.0 * fm + fb);
    return simpson_rec(f, c, a, b, fa, fm, fb, whole, eps, 30);
}

/* Integral over [0,1] of a function with a Gaussian-shaped peak of scale s at
 * c: [c-14s, c+14s] is cut into pieces of width s/2 so the adaptive rule
 * cannot step over the peak; the rest of [0,1] is integrated in one piece
 * each side. */
static double integrate_peaked(fn1 f, const void *ctx, double c, double s)
{
    double lo = c - 14.0 * s, hi = c + 14.0 * s;
    double a = lo < 0.0 ? 0.0 : lo, b = hi > 1.0 ? 1.0 : hi;
    double total = 0.0;
    if (a > 0.0) total += simpson(f, ctx, 0.0, a, 1e-16);
    if (b < 1.0) total += simpson(f, ctx, b, 1.0, 1e-16);
    if (b > a) {
        int pieces = (int)ceil((b - a) / (0.5 * s));
        if (pieces < 1) pieces = 1;
        if (pieces > 4096) pieces = 4096;
        double h = (b - a) / pieces;
        for (int i = 0; i < pieces; ++i)
            total += simpson(f, ctx, a + i * h, a + (i + 1) * h, 1e-16);
    }
    return total;
}

/* x-marginal density times P(0 <= Y <= 1 | X = x). */
static double z_integrand(double x, const void *ctx)
{
    const gauss2 *g = (const gauss2 *)ctx;
    double sx = sqrt(g->sxx);
    double px = exp(-0.5 * (x - g->mx) * (x - g->mx) / g->sxx) / (sqrt(2.0 * M_PI) * sx);
    double cm = g->my + g->sxy / g->sxx * (x - g->mx);
    double cs = sqrt(g->syy - g->sxy * g->sxy / g->sxx);
    double hi = (1.0 - cm) / cs, lo = (0.0 - cm) / cs;
    double p;
    if (lo > 0.0) p = 0.5 * (erfc(lo / sqrt(2.0)) - erfc(hi / sqrt(2.0)));
    else if (hi < 0.0) p = 0.5 * (erfc(-hi / sqrt(2.0)) - erfc(-lo / sqrt(2.0)));
    else p = 1.0 - 0.5 * erfc(-lo / sqrt(2.0)) - 0.5 * erfc(hi / sqrt(2.0));
    return px * p;
}

/* Z = integral over [0,1]^2 of N(u; mu, Sigma): the guide's mass inside the
 * square (the guide's draws outside it fall back to the BRDF). Written as the
 * textbook conditioning identity: marginal of X times the conditional
 * probability of Y, integrated over x by adaptive quadrature.
 * Pinned by: brute-force 2D midpoint sums, the diagonal-Sigma product of 1D
 * normal cdfs, the orthant probability 1/4 + asin(rho)/(2 pi). */
double or_rect_mass(const double g5[5])
{
    gauss2 g = {g5[0], g5[1], g5[2], g5[3], g5[4]};
    return integrate_peaked(z_integrand, &g, g.mx, sqrt(g.sxx));
}

/* Edge integrals for dZ/dtheta, from differentiating under the integral:
 *   dZ/dmu_x   = int_0^1 [N(0,y) - N(1,y)] dy
 *   dZ/ds_xx   = 1/2 int_0^1 [dN/dx(1,y) - dN/dx(0,y)] dy
 *   dZ/ds_xy   = N(1,1) - N(1,0) - N(0,1) + N(0,0)
 * (dN/dSigma_ij = 1/2 d2N/dmu_i dmu_j, and dN/dmu = -dN/du). The symmetric
 * off-diagonal entry is one parameter, so its derivative carries both
 * off-diagonal slots. Pinned by central finite differences of or_rect_mass. */
typedef struct { const double *g5; int axis; double fixed; int deriv; } edge_ctx;

static double edge_integrand(double t, const void *ctx)
{
    const edge_ctx *e = (const edge_ctx *)ctx;
    double u[2];
    if (e->axis == 0) { u[0] = e->fixed; u[1] = t; } else { u[0] = t; u[1] = e->fixed; }
    double n = or_gauss_pdf(e->g5, u);
    if (!e->deriv) return n;
    /* dN/du_axis = -N * (Sigma^-1 (u - mu))_axis */
    double sxx = e->g5[2], syy = e->g5[3], sxy = e->g5[4];
    double det = sxx * syy - sxy * sxy;
    double dx = u[0] - e->g5[0], dy = u[1] - e->g5[1];
    double ix = (syy * dx - sxy * dy) / det, iy = (-sxy * dx + sxx * dy) / det;
    return -n * (e->axis == 0 ? ix : iy);
}

static double edge_integral(const double g5[5], int axis, double fixed, int deriv)
{
    /* The density restricted to the edge is Gaussian in t with the
     * conditional mean and spread of the other coordinate. */
    double mx = g5[0], my = g5[1], sxx = g5[2], syy = g5[3], sxy = g5[4];
    double c, s;
    if (axis == 0) { c = my + sxy / sxx * (fixed - mx); s = sqrt(syy - sxy * sxy / sxx); }
    else { c = mx + sxy / syy * (fixed - my); s = sqrt(sxx - sxy * sxy / syy); }
    edge_ctx e = {g5, axis, fixed, deriv};
    return integrate_peaked(edge_integrand, &e, c, s);
}

void or_rect_mass_grad(const double g5[5], double out[5])
{
    double u00[2] = {0, 0}, u01[2] = {0, 1}, u10[2] = {1, 0}, u11[2] = {1, 1};
    out[0] = edge_integral(g5, 0, 0.0, 0) - edge_integral(g5, 0, 1.0, 0);
    out[1] = edge_integral(g5, 1, 0.0, 0) - edge_integral(g5, 1, 1.0, 0);
    out[2] = 0.5 * (edge_integral(g5, 0, 1.0, 1) - edge_integral(g5, 0, 0.0, 1));
    out[3] = 0.5 * (edge_integral(g5, 1, 1.0, 1) - edge_integral(g5, 1, 0.0, 1));
    out[4] = or_gauss_pdf(g5, u11) - or_gauss_pdf(g5, u10) - or_gauss_pdf(g5, u01) +
             or_gauss_pdf(g5, u00);
}

void or_rect_mass_many(int64_t n, const double *g5, double *z)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) z[i] = or_rect_mass(g5 + 5 * i);
}

void or_rect_mass_grad_many(int64_t n, const double *g5, double *dz)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) or_rect_mass_grad(g5 + 5 * i, dz + 5 * i);
}

/* ------------------------------------------------------------------------ */
/* Materials (Eq. 1's f_r). The paper does not define its BRDFs; the        */
/* synthetic scenes use a Lambertian surface (f_r = albedo/pi), a GGX       */
/* microfacet surface (Walter et al. 2007: alpha = roughness^2, separable   */
/* Smith shadowing, Schlick's Fresnel F = F0 + (1 - F0)(1 - o.h)^5 with F0  */
/* from the configuration, F0 = 1 giving F = 1; visible normals not used;   */
/* the draw picks the half vector with density D(h) cos(theta_h) and        */
/* reflects the view direction about it) and a transparent surface (Sec. 5: */
/* guiding is off for transparent materials): a smooth dielectric of index  */
/* 1.5 that reflects or refracts the view direction, choosing reflection    */
/* with its exact unpolarised Fresnel reflectance, tinted by the albedo.    */
/* The roughness slot codes the material: >= 0 GGX, in (-1.5, 0) Lambertian */
/* (-1 by convention), <= -1.5 transparent (-2 by convention).              */
/* All directions are in the local frame (normal = +z).                     */
/* Pinned by: the Lambertian pdf normalised and consistent with its         */
/* sampler; the GGX distribution normalised, its sampler against its pdf,   */
/* reciprocity and the energy bound (tests/test_oracle_pins.py); the        */
/* dielectric Fresnel against the sine/tangent form, Snell's law, Schlick's */
/* limits and the Fresnel-weighted lobe against its sampler                 */
/* (tests/test_oracle_materials.py).                                        */
/* ------------------------------------------------------------------------ */
static int is_transparent(double rough) { return rough <= -1.5; }
static int is_lambert(double rough) { return rough < 0.0 && rough > -1.5; }

#define DIELECTRIC_IOR 1.5

/* Unpolarised Fresnel reflectance of a smooth dielectric for light arriving
 * from outside at cosine ci > 0 (no total reflection from the outside). */
double or_dielectric_fresnel(double ci)
{
    double n = DIELECTRIC_IOR, si2 = 1.0 - ci * ci, ct = sqrt(1.0 - si2 / (n * n));
    double rs = (ci - n * ct) / (ci + n * ct), rp = (n * ci - ct) / (n * ci + ct);
    return 0.5 * (rs * rs + rp * rp);
}

static double ggx_alpha(double rough) { double a = rough * rough; return a < 1e-4 ? 1e-4 : a; }

static double ggx_d(double a2, double nh)
{
    double t = nh * nh * (a2 - 1.0) + 1.0;
    return a2 / (M_PI * t * t);
}

static double smith_g1(double a2, double c)
{
    return 2.0 * c / (c + sqrt(a2 + (1.0 - a2) * c * c));
}

/* f_r * cos(theta_i) with GGX reflectance f0 at normal incidence (0 for a
 * transparent surface: its BSDF is a pair of deltas). */
double or_brdf_cos_f0(double rough, double albedo, double f0, const double wo[3], const double wi[3])
{
    if (wi[2] <= 0.0 || wo[2] <= 0.0 || is_transparent(rough)) return 0.0;
    if (rough < 0.0) return albedo / M_PI * wi[2];
    double a = ggx_alpha(rough), a2 = a * a;
    double h[3] = {wo[0] + wi[0], wo[1] + wi[1], wo[2] + wi[2]};
    double hl = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    double nh = h[2] / hl;
    double oh = (wo[0] * h[0] + wo[1] * h[1] + wo[2] * h[2]) / hl;
    double m = 1.0 - oh, fr = f0 + (1.0 - f0) * m * m * m * m * m;
    return albedo * fr * ggx_d(a2, nh) * smith_g1(a2, wi[2]) * smith_g1(a2, wo[2]) / (4.0 * wo[2]);
}

double or_brdf_cos(double rough, double albedo, const double wo[3], const double wi[3])
{
    return or_brdf_cos_f0(rough, albedo, 1.0, wo, wi);
}

/* Density of the BRDF draw at wi (solid angle). */
double or_brdf_pdf(double rough, const double wo[3], const double wi[3])
{
    if (wi[2] <= 0.0 || is_transparent(rough)) return 0.0;
    if (rough < 0.0) return wi[2] / M_PI;
    if (wo[2] <= 0.0) return 0.0;
    double a = ggx_alpha(rough), a2 = a * a;
    double h[3] = {wo[0] + wi[0], wo[1] + wi[1], wo[2] + wi[2]};
    double hl = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    double hn[3] = {h[0] / hl, h[1] / hl, h[2] / hl};
    double oh = wo[0] * hn[0] + wo[1] * hn[1] + wo[2] * hn[2];
    if (oh <= 0.0) return 0.0;
    return ggx_d(a2, hn[2]) * hn[2] / (4.0 * oh);
}

/* BRDF draw from two uniforms in [0,1). Returns 1 for a draw in the upper
 * hemisphere, 0 for a wasted draw; *margin receives how far the validity
 * decision was from its threshold. A transparent surface reflects when
 * x1 < F (the Fresnel reflectance at the view direction) and refracts
 * otherwise, into the lower hemisphere; a view from below wastes the draw. */
int or_brdf_sample(double rough, const double wo[3], double x1, double x2, double wi[3],
                   double *margin)
{
    if (is_transparent(rough)) {
        double ci = wo[2];
        if (ci <= 0.0) {
            wi[0] = wi[1] = 0.0; wi[2] = 1.0;
            *margin = fabs(ci);
            return 0;
        }
        double fr = or_dielectric_fresnel(ci), eta = 1.0 / DIELECTRIC_IOR;
        *margin = fabs(x1 - fr) < ci ? fabs(x1 - fr) : ci;
        if (x1 < fr) {
            wi[0] = -wo[0]; wi[1] = -wo[1]; wi[2] = ci;
        } else {
            double ct = sqrt(1.0 - eta * eta * (1.0 - ci * ci));
            wi[0] = -eta * wo[0]; wi[1] = -eta * wo[1]; wi[2] = -ct;
        }
        return 1;
    }
    if (rough < 0.0) {
        /* cosine-weighted: radius sqrt(x1) on the disk, lifted */
        double r = sqrt(x1), phi = 2.0 * M_PI * x2;
        wi[0] = r * cos(phi); wi[1] = r * sin(phi); wi[2] = sqrt(1.0 - x1);
        *margin = 1.0;
        return 1;
    }
    double a = ggx_alpha(rough), a2 = a * a;
    double den = (1.0 - x1) + a2 * x1;
    double ct = sqrt((1.0 - x1) / den), st = sqrt(a2 * x1 / den);
    double phi = 2.0 * M_PI * x2;
    double h[3] = {st * cos(phi), st * sin(phi), ct};
    double oh = wo[0] * h[0] + wo[1] * h[1] + wo[2] * h[2];
    for (int i = 0; i < 3; ++i) wi[i] = 2.0 * oh * h[i] - wo[i];
    double m1 = oh, m2 = wi[2];
    *margin = fabs(m1) < fabs(m2) ? fabs(m1) : fabs(m2);
    return (oh > 0.0 && wi[2] > 0.0) ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Analytic incident radiance, standing in for the traced ray of the path-  */
/* tracing pass: a sum of normalised von Mises-Fisher lobes                 */
/*   vMF(w; d, k) = k / (2 pi (1 - exp(-2k))) exp(k (d.w - 1)),             */
/* optionally times a smooth occlusion mask of the world position and the   */
/* direction, plus a constant.                                              */
/* Pinned by: each normalised lobe integrating to 1 over the sphere         */
/* (tests/test_oracle_pins.py); the coloured field training exactly as the  */
/* monochrome field of its luminances (tests/test_oracle_colour.py).        */
/* ------------------------------------------------------------------------ */
/* The coloured field's channels (a monochrome field gives its value in all three). */
void or_radiance_rgb(const or_field *f, const double x[3], const double w[3], double out[3])
{
    double s[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < f->n_lobes; ++j) {
        double k = f->kappa[j];
        double dot = f->dir[j][0] * w[0] + f->dir[j][1] * w[1] + f->dir[j][2] * w[2];
        double v = k / (2.0 * M_PI * (1.0 - exp(-2.0 * k))) * exp(k * (dot - 1.0));
        for (int c = 0; c < 3; ++c) s[c] += (f->rgb ? f->amp_rgb[j][c] : f->amp[j]) * v;
    }
    double m = 1.0;
    if (f->mask_kind == 1)
        m = 0.5 + 0.5 * sin(2.0 * M_PI * (f->mask[0] * x[0] + f->mask[2] * w[0])) *
                  cos(2.0 * M_PI * (f->mask[1] * x[1] + f->mask[2] * w[1]));
    for (int c = 0; c < 3; ++c) out[c] = s[c] * m + (f->rgb ? f->constant_rgb[c] : f->constant);
}

/* The radiance the pass works with: the field's value, or for a coloured
 * field its luminance (Sec. 3.1 weighs by the radiance's luminance), with the
 * Rec. 709 weights Y = 0.2126 R + 0.7152 G + 0.0722 B. */
double or_radiance(const or_field *f, const double x[3], const double w[3])
{
    if (f->rgb) {
        double c[3];
        or_radiance_rgb(f, x, w, c);
        return 0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2];
    }
    double s = 0.0;
    for (int j = 0; j < f->n_lobes; ++j) {
        double k = f->kappa[j];
        double dot = f->dir[j][0] * w[0] + f->dir[j][1] * w[1] + f->dir[j][2] * w[2];
        s += f->amp[j] * k / (2.0 * M_PI * (1.0 - exp(-2.0 * k))) * exp(k * (dot - 1.0));
    }
    if (f->mask_kind == 1) {
        double m = 0.5 + 0.5 * sin(2.0 * M_PI * (f->mask[0] * x[0] + f->mask[2] * w[0])) *
                             cos(2.0 * M_PI * (f->mask[1] * x[1] + f->mask[2] * w[1]));
        s *= m;
    }
    return s + f->constant;
}

/* ------------------------------------------------------------------------ */
/* Camera: primary ray of pixel (x, y); the view direction w_o is the       */
/* reversed ray and the shading point is origin + depth * dir.              */
/* Orthographic: from origin + (x+0.5) s right + (y+0.5) s up along fwd      */
/* (s the pixel size). Pinhole: from origin along fwd + sx right + sy up,   */
/* normalised, sx = (2 (x+0.5)/W - 1) tan(fov_v/2) W/H, sy = (1 - 2 (y+0.5)/H)*/
/* tan(fov_v/2): row 0 at the top, the image's horizontal half-angle at     */
/* atan(tan(fov_v/2) W/H).                                                  */
/* Pinned by: shading points landing on the synthetic scenes' surfaces (the */
/* panned heightfield, the orbit's ground and quads), the centre pixel's    */
/* ray along fwd and the horizontal field of view at the screen's edge      */
/* (tests/test_oracle_ground_truth.py).                                     */
/* ------------------------------------------------------------------------ */
void or_camera_ray(const or_camera *c, int W, int H, int x, int y, double o[3], double d[3])
{
    if (c->kind == 0) {
        double sx = (x + 0.5) * c->pixel_size, sy = (y + 0.5) * c->pixel_size;
        for (int i = 0; i < 3; ++i) {
            o[i] = c->origin[i] + sx * c->right[i] + sy * c->up[i];
            d[i] = c->fwd[i];
        }
    } else {
        double aspect = (double)W / (double)H;
        double sx = (2.0 * (x + 0.5) / W - 1.0) * c->tan_half_fov * aspect;
        double sy = (1.0 - 2.0 * (y + 0.5) / H) * c->tan_half_fov;
        double v[3];
        for (int i = 0; i < 3; ++i) v[i] = c->fwd[i] + sx * c->right[i] + sy * c->up[i];
        double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int i = 0; i < 3; ++i) { o[i] = c->origin[i]; d[i] = v[i] / l; }
    }
}

/* ------------------------------------------------------------------------ */
/* Gamma: 8 parameters per pixel (abstract; Sec. 3.1), in the order         */
/*   E[X], E[Y], E[X^2], E[Y^2], E[XY], pi, k, W                             */
/* where [X, Y] = M^-1(w), the moments are weighted by the luminance of the  */
/* samples (Sec. 3.1), pi is the guide's mixing weight, k the number of     */
/* training epochs, and W the running luminance-weight mass of a frame's    */
/* training samples. The paper names seven of its eight parameters; the     */
/* eighth is read as W, the quantity a weighted running average of the      */
/* moments needs in order to weigh a new frame against the stored ones.    */
/* ------------------------------------------------------------------------ */
enum { G_EX = 0, G_EY, G_EXX, G_EYY, G_EXY, G_PI, G_K, G_W };

/* Mean and regularised covariance of the guide from stored moments:
 * mean clamped to the square, variances floored, correlation clamped. */
static void derive_gauss(const or_config *cfg, const double *gm, double g5[5])
{
    double ex = gm[G_EX], ey = gm[G_EY];
    double sxx = gm[G_EXX] - ex * ex, syy = gm[G_EYY] - ey * ey, sxy = gm[G_EXY] - ex * ey;
    if (sxx < cfg->sigma2_min) sxx = cfg->sigma2_min;
    if (syy < cfg->sigma2_min) syy = cfg->sigma2_min;
    double lim = cfg->rho_max * sqrt(sxx * syy);
    if (sxy > lim) sxy = lim;
    if (sxy < -lim) sxy = -lim;
    g5[0] = ex < 0.0 ? 0.0 : (ex > 1.0 ? 1.0 : ex);
    g5[1] = ey < 0.0 ? 0.0 : (ey > 1.0 ? 1.0 : ey);
    g5[2] = sxx; g5[3] = syy; g5[4] = sxy;
}

void or_derive_many(const or_config *cfg, int64_t n, const double *gam, double *g5)
{
    for (int64_t i = 0; i < n; ++i) derive_gauss(cfg, gam + 8 * i, g5 + 5 * i);
}

static void init_gamma(const or_config *cfg, double pi, double *gm)
{
    double mx = cfg->init_mu[0], my = cfg->init_mu[1];
    gm[G_EX] = mx; gm[G_EY] = my;
    gm[G_EXX] = cfg->init_sigma[0] + mx * mx;
    gm[G_EYY] = cfg->init_sigma[1] + my * my;
    gm[G_EXY] = cfg->init_sigma[2] + mx * my;
    gm[G_PI] = pi; gm[G_K] = 0.0; gm[G_W] = 0.0;
}

void or_init_gamma(const or_config *cfg, double pi, int64_t n, double *gam)
{
    for (int64_t i = 0; i < n; ++i) init_gamma(cfg, pi, gam + 8 * i);
}

/* ------------------------------------------------------------------------ */
/* Reprojection (Sec. 3.1): fetch last frame's Gamma at the pixel the       */
/* motion vector points to, nearest neighbour; reject on depth and normal   */
/* differences (SVGF-style); account for the change of hemisphere frame     */
/* between the old and the new surface; re-initialise rejected pixels with  */
/* pi = pi_reinit, k = 0, and mark them to sample from the BRDF alone.      */
/*                                                                          */
/* Readings (paper silent): mv = previous minus current screen position in  */
/* pixels; q = floor(p + 0.5 + mv); accept iff q on screen and              */
/* |d_prev - d_cur| <= depth_tol * d_cur and n_prev . n_cur >= normal_tol,  */
/* all evaluated in binary32 in this order. Frame change when the normals   */
/* differ: the guide's mean direction is carried through the world into the */
/* new frame (clamped to the horizon), the covariance is kept.              */
/* Pinned by: identity motion copying Gamma exactly, an integer pan         */
/* shifting it with exactly the newly exposed columns rejected, the depth,  */
/* normal and off-screen rejections, and the frame change keeping the       */
/* mean's world direction (tests/test_oracle_pins.py).                      */
/* ------------------------------------------------------------------------ */
static void frame_change(const double np_[3], const double nc[3], double *gm)
{
    double ex = gm[G_EX], ey = gm[G_EY];
    double sxx = gm[G_EXX] - ex * ex, syy = gm[G_EYY] - ey * ey, sxy = gm[G_EXY] - ex * ey;
    double mu[2] = {ex < 0.0 ? 0.0 : (ex > 1.0 ? 1.0 : ex), ey < 0.0 ? 0.0 : (ey > 1.0 ? 1.0 : ey)};
    double wl[3], ww[3], wn[3], mu2[2];
    or_square_to_hemi(mu, wl);
    to_world(np_, wl, ww);
    to_local(nc, ww, wn);
    if (wn[2] < 0.0) {
        double r = sqrt(wn[0] * wn[0] + wn[1] * wn[1]);
        wn[2] = 0.0;
        if (r > 0.0) { wn[0] /= r; wn[1] /= r; } else { wn[0] = 1.0; wn[1] = 0.0; }
    }
    or_hemi_to_square(wn, mu2);
    gm[G_EX] = mu2[0]; gm[G_EY] = mu2[1];
    gm[G_EXX] = sxx + mu2[0] * mu2[0];
    gm[G_EYY] = syy + mu2[1] * mu2[1];
    gm[G_EXY] = sxy + mu2[0] * mu2[1];
}

/* One pixel of the reprojection step. Returns accept; writes q (-1 if off
 * screen) and the reprojected / re-initialised Gamma. */
static int reproject_pixel_s(const or_config *cfg, int x, int y, const float *g0, const float *g1,
                             const float *g0p, const double *gam_prev, int64_t gstride, double *out, int32_t *q)
{
    int W = cfg->width, H = cfg->height;
    int64_t i = (int64_t)y * W + x;
    float mvx = g1[4 * i + 0], mvy = g1[4 * i + 1];
    volatile float fx = ((float)x + 0.5f) + mvx;
    volatile float fy = ((float)y + 0.5f) + mvy;
    int acc = 0;
    *q = -1;
    if (fx >= 0.0f && fx < (float)W && fy >= 0.0f && fy < (float)H) {
        int qx = (int)floorf(fx), qy = (int)floorf(fy);
        int64_t j = (int64_t)qy * W + qx;
        *q = (int32_t)j;
        float dc = g0[4 * i + 3], dp = g0p[4 * j + 3];
        volatile float dd = dp - dc;
        volatile float dlim = (float)cfg->depth_tol * dc;
        volatile float n0 = g0p[4 * j + 0] * g0[4 * i + 0];
        volatile float n1 = g0p[4 * j + 1] * g0[4 * i + 1];
        volatile float n2 = g0p[4 * j + 2] * g0[4 * i + 2];
        volatile float ndot = (n0 + n1) + n2;
        acc = (fabsf(dd) <= dlim) && (ndot >= (float)cfg->normal_tol);
        if (acc) {
            memcpy(out, gam_prev + gstride * j, 8 * sizeof(double));
            int same = memcmp(&g0p[4 * j], &g0[4 * i], 3 * sizeof(float)) == 0;
            if (!same) {
                double np_[3], nc[3];
                unit_normal(g0p + 4 * j, np_);
                unit_normal(g0 + 4 * i, nc);
                frame_change(np_, nc, out);
            }
        }
    }
    if (!acc) init_gamma(cfg, cfg->pi_reinit, out);
    return acc;
}

static int reproject_pixel(const or_config *cfg, int x, int y, const float *g0, const float *g1,
                           const float *g0p, const double *gam_prev, double *out, int32_t *q)
{
    return reproject_pixel_s(cfg, x, y, g0, g1, g0p, gam_prev, 8, out, q);
}

void or_reproject(const or_config *cfg, const float *g0, const float *g1, const float *g0p,
                  const double *gam_prev, double *gam_out, uint8_t *accept, int32_t *qidx)
{
    int W = cfg->width, H = cfg->height;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t i = (int64_t)y * W + x;
            accept[i] = (uint8_t)reproject_pixel(cfg, x, y, g0, g1, g0p, gam_prev, gam_out + 8 * i,
                                                 &qidx[i]);
        }
}

/* ------------------------------------------------------------------------ */
/* Guided sampling, mixture pdf and MIS (Eq. 2, Sec. 3.1).                  */
/*                                                                          */
/* D(w) = pi N(M^-1(w); mu, Sigma) + (1 - pi) f_r. The guide draw takes two */
/* N(0,1) variates by Box-Muller, maps them through the Cholesky factor of  */
/* Sigma and then through M. Reading (paper silent on the square's edge):   */
/* a guide draw that lands outside [0,1]^2 is replaced by a BRDF draw, so   */
/* the density of the procedure is exactly                                   */
/*   p_mix(w) = pi N(u)/(2 pi) + (1 - pi Z) p_b(w),  u = M^-1(w_local),     */
/* and the one-sample balance-heuristic MIS estimate is F = f / p_mix.      */
/* Random numbers: Philox4x32-10, key = seed, counter = (pixel, frame,      */
/* sample, stream). The top 24 bits of word 0 pick the strategy; those of   */
/* words 1 and 2 drive either Box-Muller (guide) or the BRDF draw (they are */
/* independent of word 0, so still uniform given the choice); a guide draw  */
/* that left the square takes its BRDF draw from word 3 and from the low    */
/* bytes of words 0-2, bits the decision has not looked at.                 */
/* Pinned by: the mixture pdf integrating to 1 (Lambert) and to the valid   */
/* BRDF mass (GGX), the MIS weights at the samples, unbiased estimates of   */
/* closed-form integrals (constant radiance, a lobe on the normal, GGX      */
/* albedo) and BRDF-only draws on re-initialised pixels                     */
/* (tests/test_oracle_pins.py).                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    double g5[5], chol[3], Z, pi_eff;
    double n[3], wo_l[3], pos[3];
    double rough, albedo, f0;
} pixel_ctx;

static void cholesky(const double g5[5], double c[3])
{
    c[0] = sqrt(g5[2]);
    c[1] = g5[4] / c[0];
    c[2] = sqrt(g5[3] - c[1] * c[1]);
}

/* The surface of pixel (x, y): normal, shading point, local view direction
 * and material. */
static void surface_setup(const or_config *cfg, const or_camera *cam, int x, int y,
                          const float *g0, const float *g1, pixel_ctx *p)
{
    int W = cfg->width, H = cfg->height;
    int64_t i = (int64_t)y * W + x;
    double o[3], d[3];
    or_camera_ray(cam, W, H, x, y, o, d);
    double depth = g0[4 * i + 3];
    double wo[3] = {-d[0], -d[1], -d[2]};
    unit_normal(g0 + 4 * i, p->n);
    for (int k = 0; k < 3; ++k) p->pos[k] = o[k] + depth * d[k];
    to_local(p->n, wo, p->wo_l);
    p->rough = g1[4 * i + 2];
    if (!cfg->transparent && is_transparent(p->rough)) p->rough = -1.0;   /* the code is Lambertian then */
    p->albedo = g1[4 * i + 3];
    p->f0 = cfg->ggx_f0;
}

static void pixel_setup(const or_config *cfg, const or_camera *cam, int x, int y,
                        const float *g0, const float *g1, const double *gm, int reinit,
                        pixel_ctx *p)
{
    surface_setup(cfg, cam, x, y, g0, g1, p);
    derive_gauss(cfg, gm, p->g5);
    cholesky(p->g5, p->chol);
    p->Z = or_rect_mass(p->g5);
    /* Guiding is off on a re-initialised pixel (Sec. 3.1), on near-mirror
     * surfaces (Sec. 5; threshold rough_min is this build's reading) and on
     * transparent surfaces (Sec. 5). */
    int gated = reinit || (p->rough >= 0.0 && p->rough < cfg->rough_min) || is_transparent(p->rough);
    p->pi_eff = gated ? 0.0 : gm[G_PI];
}

/* Evaluate the pieces of the estimator at a local direction; u is the square
 * coordinate to use for the guide density (NULL: compute M^-1(wl)). */
static void eval_local(const or_field *fld, const pixel_ctx *p, const double wl[3],
                       const double *u_in, double *fcos, double *pg, double *pb, double *pmix,
                       double *rad, double u_out[2])
{
    double ww[3];
    to_world(p->n, wl, ww);
    *rad = or_radiance(fld, p->pos, ww);
    if (wl[2] <= 0.0) {
        *fcos = 0.0; *pg = 0.0; *pb = 0.0; *pmix = 0.0;
        u_out[0] = u_out[1] = -1.0;
        return;
    }
    double u[2];
    if (u_in) { u[0] = u_in[0]; u[1] = u_in[1]; } else or_hemi_to_square(wl, u);
    u_out[0] = u[0]; u_out[1] = u[1];
    *fcos = *rad * or_brdf_cos_f0(p->rough, p->albedo, p->f0, p->wo_l, wl);
    *pb = or_brdf_pdf(p->rough, p->wo_l, wl);
    *pg = or_gauss_pdf(p->g5, u) / (2.0 * M_PI);
    *pmix = p->pi_eff * *pg + (1.0 - p->pi_eff * p->Z) * *pb;
}

/* One direction drawn from the mixture of pixel p from the four words of
 * Philox at counter (pixel, frame, sample, stream0): word 0 picks the
 * strategy, words 1-2 drive Box-Muller or the BRDF draw, and a fallback draws
 * from word 3 and the low bytes of words 0-2. Returns the strategy; writes the local
 * direction, whether it is valid, the square point when the guide drew it,
 * and the distance of the draw's decisions to their thresholds. */
static int draw_direction(const pixel_ctx *p, const uint32_t key[2], uint32_t pix, uint32_t frame,
                          uint32_t s, uint32_t stream0, double wl[3], double u[2], int *have_u,
                          int *valid, double *margin)
{
    uint32_t c0[4] = {pix, frame, s, stream0}, r0[4];
    float pi_dec = (float)p->pi_eff; /* the strategy decision is taken in binary32 */
    or_philox(c0, key, r0);
    double zeta = unif(r0[0]);
    int strat;
    *have_u = 0;
    *margin = fabs(zeta - (double)pi_dec);
    if (zeta < (double)pi_dec) {
        double x1 = unif_open0(r0[1]), x2 = unif(r0[2]);
        double rr = sqrt(-2.0 * log(x1));
        double z1 = rr * cos(2.0 * M_PI * x2), z2 = rr * sin(2.0 * M_PI * x2);
        u[0] = p->g5[0] + p->chol[0] * z1;
        u[1] = p->g5[1] + p->chol[1] * z1 + p->chol[2] * z2;
        double m = fmin(fmin(fabs(u[0]), fabs(1.0 - u[0])), fmin(fabs(u[1]), fabs(1.0 - u[1])));
        if (m < *margin) *margin = m;
        if (u[0] >= 0.0 && u[0] <= 1.0 && u[1] >= 0.0 && u[1] <= 1.0) {
            strat = S_GUIDE;
            or_square_to_hemi(u, wl);
            *valid = wl[2] > 0.0;
            *have_u = 1;
        } else {
            strat = S_FALLBACK;
            /* fresh uniforms from the bits the draw has not used: word 3, and
             * the low bytes of words 0-2 (independent of their top 24 bits) */
            uint32_t spare = (r0[0] & 0xFFu) | ((r0[1] & 0xFFu) << 8) | ((r0[2] & 0xFFu) << 16);
            double mb;
            *valid = or_brdf_sample(p->rough, p->wo_l, unif(r0[3]), (double)spare * (1.0 / 16777216.0), wl,
                                    &mb);
            if (mb < *margin) *margin = mb;
        }
    } else {
        /* a transparent surface (always gated) draws one of its two deltas */
        strat = is_transparent(p->rough) ? S_DELTA : S_BRDF;
        double mb;
        *valid = or_brdf_sample(p->rough, p->wo_l, unif(r0[1]), unif(r0[2]), wl, &mb);
        if (mb < *margin) *margin = mb;
    }
    return strat;
}

/* Sampling of pixel (x, y); its outputs go to slot `slot` of planes of
 * `stride` entries (the whole frame: slot = pixel index, stride = W H). */
static void sample_pixel_s(const or_config *cfg, const or_camera *cam, const or_field *fld,
                           uint32_t frame, int x, int y, const float *g0, const float *g1,
                           const double *gm, int reinit, or_samples *S, double *img, int64_t slot,
                           int64_t stride)
{
    int W = cfg->width, spp = cfg->spp;
    int64_t i = (int64_t)y * W + x;
    pixel_ctx p;
    pixel_setup(cfg, cam, x, y, g0, g1, gm, reinit, &p);
    uint32_t key[2] = {cfg->seed_lo, cfg->seed_hi};
    double sum = 0.0, sum_rgb[3] = {0.0, 0.0, 0.0};
    for (int s = 0; s < spp; ++s) {
        int64_t o = (int64_t)s * stride + slot;
        double wl[3], u[2], margin;
        int valid, have_u;
        int strat = draw_direction(&p, key, (uint32_t)i, frame, (uint32_t)s, 0u, wl, u, &have_u, &valid,
                                   &margin);
        double wgt = 0.0;   /* the estimate per unit radiance, for the colour channels */
        double fcos = 0, pg = 0, pb = 0, pmix = 0, rad, uo[2] = {-1.0, -1.0};
        double F = 0.0, mis = 0.0;
        if (valid && strat == S_DELTA) {
            /* a delta of the transparent surface: the Fresnel weight of the
             * chosen branch cancels its probability, leaving the tint */
            double wwi[3];
            to_world(p.n, wl, wwi);
            rad = or_radiance(fld, p.pos, wwi);
            F = p.albedo * rad;
            wgt = p.albedo;
            mis = 1.0;
        } else if (valid) {
            eval_local(fld, &p, wl, have_u ? u : NULL, &fcos, &pg, &pb, &pmix, &rad, uo);
            if (pmix > 0.0) {
                F = fcos / pmix;
                wgt = (wl[2] > 0.0 ? or_brdf_cos_f0(p.rough, p.albedo, p.f0, p.wo_l, wl) : 0.0) / pmix;
                mis = strat == S_GUIDE ? p.pi_eff * pg / pmix : (1.0 - p.pi_eff * p.Z) * pb / pmix;
            }
        } else {
            double wwi[3];
            to_world(p.n, wl, wwi);
            rad = or_radiance(fld, p.pos, wwi);
            strat |= S_INVALID;
        }
        double ww[3];
        to_world(p.n, wl, ww);
        if (S->wx) { S->wx[o] = ww[0]; S->wy[o] = ww[1]; S->wz[o] = ww[2]; }
        if (S->radiance) S->radiance[o] = rad;
        if (S->pdf) S->pdf[o] = pmix;
        if (S->mis) S->mis[o] = mis;
        if (S->estimate) S->estimate[o] = F;
        if (S->strategy) S->strategy[o] = (uint8_t)strat;
        if (S->pg) S->pg[o] = pg;
        if (S->pb) S->pb[o] = pb;
        if (S->ux) { S->ux[o] = uo[0]; S->uy[o] = uo[1]; }
        if (S->margin) S->margin[o] = margin;
        sum += F;
        if (fld->rgb) {
            double c[3];
            or_radiance_rgb(fld, p.pos, ww, c);
            for (int k = 0; k < 3; ++k) sum_rgb[k] += wgt * c[k];
        }
    }
    if (fld->rgb) {
        for (int k = 0; k < 3; ++k) img[k * stride + slot] = sum_rgb[k] / spp;
    } else {
        img[slot] = sum / spp;
    }
}

static void sample_pixel(const or_config *cfg, const or_camera *cam, const or_field *fld,
                         uint32_t frame, int x, int y, const float *g0, const float *g1,
                         const double *gm, int reinit, or_samples *S, double *img)
{
    sample_pixel_s(cfg, cam, fld, frame, x, y, g0, g1, gm, reinit, S, img, (int64_t)y * cfg->width + x,
                   (int64_t)cfg->width * cfg->height);
}

void or_sample(const or_config *cfg, const or_camera *cam, const or_field *fld, uint32_t frame,
               const float *g0, const float *g1, const double *gam, const uint8_t *reinit,
               or_samples *S, double *img)
{
    int W = cfg->width, H = cfg->height;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t i = (int64_t)y * W + x;
            sample_pixel(cfg, cam, fld, frame, x, y, g0, g1, gam + 8 * i, reinit ? reinit[i] : 0, S,
                         img);
        }
}

/* ------------------------------------------------------------------------ */
/* Training (Sec. 3.2): weighted online EM from this frame's samples.       */
/*                                                                          */
/* Only samples drawn by the BRDF strategy train (Sec. 3.2; using all of    */
/* them drives pi to 1). For each: weight w = f / p_b (the importance       */
/* weight of the luminance of L f_r cos under the BRDF draw), E-step        */
/* posterior gamma = pi N / p_mix. Frame statistics a = sum w gamma,        */
/* b = sum w, S1 = sum w gamma u, S2 = sum w gamma u u^T.                   */
/* M-step as a weighted running average filtered by the epoch count k       */
/* (Sec. 3.2, 4.2), the stepwise EM of the parametric-mixture guiding the   */
/* paper builds on: with eta = 1 / (min(k, kMax) + 2) and the stored guide  */
/* carrying luminance mass M0 = W (or, for a guide not yet trained, the     */
/* mass b of this frame), when b > 0:                                       */
/*   A = (1 - eta) pi M0 + eta a          new guide mass                    */
/*   B = (1 - eta) M0 + eta b             new total mass                    */
/*   E <- ((1 - eta) pi M0 E + eta S) / A  for the five moments              */
/*   pi <- clamp(A / B, 0.05, 0.95), k <- min(k + 1, kMax), W <- B.         */
/* A frame without BRDF-strategy energy (b = 0) leaves Gamma unchanged.     */
/* Pinned by: the population fixed point, a convex move toward the sample,  */
/* continuity and luminance weighting, scale invariance, guide and wasted   */
/* samples not training, and recovery of a known mixture from its samples   */
/* (tests/test_oracle_pins.py); reuse weighting and the pick law            */
/* (tests/test_oracle_reuse.py).                                            */
/* ------------------------------------------------------------------------ */
static void em_step(const or_config *cfg, double *gm, double a, double b, double s1x, double s1y,
                    double s2xx, double s2yy, double s2xy);
static void update_pixel_s(const or_config *cfg, const or_camera *cam, int x, int y,
                           const float *g0, const float *g1, double *gm, int reinit,
                           const double *wx, const double *wy, const double *wz,
                           const double *rad, const uint8_t *strat, int64_t slot, int64_t stride);

static void update_pixel(const or_config *cfg, const or_camera *cam, int x, int y,
                         const float *g0, const float *g1, double *gm, int reinit,
                         const double *wx, const double *wy, const double *wz,
                         const double *rad, const uint8_t *strat)
{
    int64_t i = (int64_t)y * cfg->width + x;
    update_pixel_s(cfg, cam, x, y, g0, g1, gm, reinit, wx, wy, wz, rad, strat, i,
                   (int64_t)cfg->width * cfg->height);
}

static void update_pixel_s(const or_config *cfg, const or_camera *cam, int x, int y,
                           const float *g0, const float *g1, double *gm, int reinit,
                           const double *wx, const double *wy, const double *wz,
                           const double *rad, const uint8_t *strat, int64_t slot, int64_t stride)
{
    int spp = cfg->spp;
    pixel_ctx p;
    pixel_setup(cfg, cam, x, y, g0, g1, gm, reinit, &p);
    double a = 0, b = 0, s1x = 0, s1y = 0, s2xx = 0, s2yy = 0, s2xy = 0;
    for (int s = 0; s < spp; ++s) {
        int64_t o = (int64_t)s * stride + slot;
        if (strat[o] != S_BRDF) continue; /* guide draws, fallbacks and wasted draws do not train */
        double ww[3] = {wx[o], wy[o], wz[o]}, wl[3];
        to_local(p.n, ww, wl);
        if (wl[2] <= 0.0) continue;
        double u[2];
        or_hemi_to_square(wl, u);
        double fcos = rad[o] * or_brdf_cos_f0(p.rough, p.albedo, p.f0, p.wo_l, wl);
        double pb = or_brdf_pdf(p.rough, p.wo_l, wl);
        if (!(pb > 0.0)) continue;
        double pg = or_gauss_pdf(p.g5, u) / (2.0 * M_PI);
        double pmix = p.pi_eff * pg + (1.0 - p.pi_eff * p.Z) * pb;
        double w = fcos / pb;
        double gam = pmix > 0.0 ? p.pi_eff * pg / pmix : 0.0;
        a += w * gam; b += w;
        s1x += w * gam * u[0]; s1y += w * gam * u[1];
        s2xx += w * gam * u[0] * u[0]; s2yy += w * gam * u[1] * u[1]; s2xy += w * gam * u[0] * u[1];
    }
    em_step(cfg, gm, a, b, s1x, s1y, s2xx, s2yy, s2xy);
}

/* The M-step of one pixel from its frame statistics (see above). */
static void em_step(const or_config *cfg, double *gm, double a, double b, double s1x, double s1y,
                    double s2xx, double s2yy, double s2xy)
{
    double k = gm[G_K] < 0.0 ? 0.0 : gm[G_K];
    if (b > 0.0) {
        double kc = k < cfg->k_max ? k : cfg->k_max;
        double eta = 1.0 / (kc + 2.0);
        double m0 = (k > 0.0 && gm[G_W] > 0.0) ? gm[G_W] : b;
        double keep = (1.0 - eta) * gm[G_PI] * m0;
        double A = keep + eta * a;
        double B = (1.0 - eta) * m0 + eta * b;
        if (A > 0.0) {
            gm[G_EX] = (keep * gm[G_EX] + eta * s1x) / A;
            gm[G_EY] = (keep * gm[G_EY] + eta * s1y) / A;
            gm[G_EXX] = (keep * gm[G_EXX] + eta * s2xx) / A;
            gm[G_EYY] = (keep * gm[G_EYY] + eta * s2yy) / A;
            gm[G_EXY] = (keep * gm[G_EXY] + eta * s2xy) / A;
        }
        double pi = A / B;
        gm[G_PI] = pi < cfg->pi_min ? cfg->pi_min : (pi > cfg->pi_max ? cfg->pi_max : pi);
        gm[G_W] = B;
        k = k + 1.0;
        if (k > cfg->k_max) k = cfg->k_max;
    }
    gm[G_K] = k;
}

void or_update(const or_config *cfg, const or_camera *cam, const float *g0, const float *g1,
               double *gam, const uint8_t *reinit, const double *wx, const double *wy,
               const double *wz, const double *rad, const uint8_t *strat)
{
    int W = cfg->width, H = cfg->height;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t i = (int64_t)y * W + x;
            update_pixel(cfg, cam, x, y, g0, g1, gam + 8 * i, reinit ? reinit[i] : 0, wx, wy, wz,
                         rad, strat);
        }
}

/* ------------------------------------------------------------------------ */
/* Neighbour-VPL reuse (Sec. 3.2: the VPLs of nearby pixels also train a    */
/* pixel's guide, which speeds up convergence without bias; Sec. 4.2: N     */
/* close VPLs per pixel, N = (1 - k/kMax) 15 + 5).                          */
/*                                                                          */
/* Readings (the paper gives no more than the above):                       */
/* - A VPL is one sample of the sampling step: its world direction w, the   */
/*   radiance L it brought back and, for a BRDF-strategy draw, the density  */
/*   p_src(w) with which its own pixel's BRDF drew it. The radiance field   */
/*   is distant, so a VPL reused at pixel p keeps its direction and its L.  */
/* - Candidates: the samples of the pixels of the (2R+1)^2 window around p, */
/*   p excluded, C = ((2R+1)^2 - 1) spp of them, enumerated row by row      */
/*   (dy, then dx, from -R), each pixel's samples consecutively.            */
/* - N = 5 + floor(15 (kMax - k) / kMax) for the reprojected epoch count k  */
/*   (clamped to [0, kMax]; a re-initialised pixel has k = 0), at most C.   */
/* - The N picks are distinct: candidate (start + j stride) mod C for       */
/*   j < N, start = floor(r C / 2^32) for word 0 r of Philox at counter     */
/*   (pixel, frame, 0, 4), stride the smallest integer >= 0.618 C coprime   */
/*   with C. Picks outside the image are dropped.                           */
/* - Only BRDF-strategy VPLs train (the rule for the pixel's own samples,   */
/*   Sec. 3.2). Each enters p's statistics with the importance weight       */
/*   w = f_p(w) / p_src(w) (f_p = L f_r cos at p), the density that drew it  */
/*   being its own pixel's BRDF: the sums stay unbiased estimates of the    */
/*   integrals of f_p over the directions p_src covers. The posterior is    */
/*   p's: gamma = pi N / p_mix at p. Own samples enter the same way.        */
/* Pinned by: the pick law (count, distinctness, window, uniform offsets), */
/* the exact statistics of a constant field over equal Lambertian pixels,  */
/* and unbiasedness of the weights across tilted neighbours (statistical).  */
/* ------------------------------------------------------------------------ */
static int64_t gcd64(int64_t a, int64_t b) { while (b) { int64_t t = a % b; a = b; b = t; } return a; }

static int64_t reuse_candidates(const or_config *cfg)
{
    int64_t d = 2 * (int64_t)cfg->reuse_radius + 1;
    return (d * d - 1) * (int64_t)cfg->spp;
}

static int64_t reuse_stride(int64_t c)
{
    int64_t s = (618 * c + 999) / 1000;   /* ceil(0.618 c) */
    if (s < 1) s = 1;
    while (gcd64(s, c) != 1) ++s;
    return s;
}

/* The picks of pixel pix in frame `frame` for reprojected epoch count k:
 * window offsets and sample index of each; returns their number N. */
int or_reuse_picks(const or_config *cfg, double k, uint32_t pix, uint32_t frame, int32_t *dx,
                   int32_t *dy, int32_t *sample)
{
    if (cfg->reuse_radius <= 0) return 0;
    int64_t c = reuse_candidates(cfg), stride = reuse_stride(c);
    int64_t kc = k < 0.0 ? 0 : (k > cfg->k_max ? cfg->k_max : (int64_t)k);
    int64_t n = 5 + (15 * (cfg->k_max - kc)) / cfg->k_max;
    if (n > c) n = c;
    uint32_t ctr[4] = {pix, frame, 0u, 4u}, key[2] = {cfg->seed_lo, cfg->seed_hi}, r[4];
    or_philox(ctr, key, r);
    int64_t start = (int64_t)(((uint64_t)r[0] * (uint64_t)c) >> 32);
    int32_t d = 2 * cfg->reuse_radius + 1, center = (d * d - 1) / 2;
    for (int64_t j = 0; j < n; ++j) {
        int64_t o = (start + j * stride) % c;
        int32_t cell = (int32_t)(o / cfg->spp);
        if (cell >= center) ++cell;   /* skip p itself */
        dy[j] = cell / d - cfg->reuse_radius;
        dx[j] = cell % d - cfg->reuse_radius;
        sample[j] = (int32_t)(o % cfg->spp);
    }
    return (int)n;
}

/* Adds one VPL (world direction ww, radiance L, source BRDF density pb_src)
 * to pixel p's statistics acc = {a, b, s1x, s1y, s2xx, s2yy, s2xy}. */
static void vpl_stats(const pixel_ctx *p, const double ww[3], double L, double pb_src, double acc[7])
{
    double wl[3];
    to_local(p->n, ww, wl);
    if (wl[2] <= 0.0 || !(pb_src > 0.0)) return;
    double u[2];
    or_hemi_to_square(wl, u);
    double fcos = L * or_brdf_cos_f0(p->rough, p->albedo, p->f0, p->wo_l, wl);
    double pb = or_brdf_pdf(p->rough, p->wo_l, wl);
    double pg = or_gauss_pdf(p->g5, u) / (2.0 * M_PI);
    double pmix = p->pi_eff * pg + (1.0 - p->pi_eff * p->Z) * pb;
    double w = fcos / pb_src;
    double gam = pmix > 0.0 ? p->pi_eff * pg / pmix : 0.0;
    acc[0] += w * gam; acc[1] += w;
    acc[2] += w * gam * u[0]; acc[3] += w * gam * u[1];
    acc[4] += w * gam * u[0] * u[0]; acc[5] += w * gam * u[1] * u[1]; acc[6] += w * gam * u[0] * u[1];
}

static void update_pixel_reuse(const or_config *cfg, const or_camera *cam, uint32_t frame, int x, int y,
                               const float *g0, const float *g1, double *gm, int reinit,
                               const or_samples *S)
{
    int W = cfg->width, H = cfg->height, spp = cfg->spp;
    int64_t i = (int64_t)y * W + x, HW = (int64_t)W * H;
    pixel_ctx p;
    pixel_setup(cfg, cam, x, y, g0, g1, gm, reinit, &p);
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int s = 0; s < spp; ++s) {
        int64_t o = (int64_t)s * HW + i;
        if (S->strategy[o] != S_BRDF) continue;
        double ww[3] = {S->wx[o], S->wy[o], S->wz[o]};
        vpl_stats(&p, ww, S->radiance[o], S->pb[o], acc);
    }
    int64_t cmax = reuse_candidates(cfg);
    int32_t *dx = malloc(sizeof(int32_t) * 3 * (size_t)(cmax > 0 ? cmax : 1));
    int32_t *dy = dx + cmax, *sm = dy + cmax;
    int n = or_reuse_picks(cfg, gm[G_K], (uint32_t)i, frame, dx, dy, sm);
    for (int j = 0; j < n; ++j) {
        int qx = x + dx[j], qy = y + dy[j];
        if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
        int64_t o = (int64_t)sm[j] * HW + (int64_t)qy * W + qx;
        if (S->strategy[o] != S_BRDF) continue;
        double ww[3] = {S->wx[o], S->wy[o], S->wz[o]};
        vpl_stats(&p, ww, S->radiance[o], S->pb[o], acc);
    }
    free(dx);
    em_step(cfg, gm, acc[0], acc[1], acc[2], acc[3], acc[4], acc[5], acc[6]);
}

/* Chosen pixels (xs[k], ys[k]) of one frame, each computed alone (no
 * neighbour reuse): reprojection against the previous Gamma, sampling and
 * training. The previous Gamma is either a whole frame (gstride = 8: row q
 * at gam_prev + 8 q, gathered at the reprojected pixel q, e.g. the state
 * another implementation reached) or one row shared by every pixel
 * (gstride = 0: a screen's first frame). Writes each pixel's new Gamma
 * (gam_out[8k..]), its estimate (img[k * planes + c], planes = 3 for a
 * coloured field, else 1), the smallest decision margin of its draws and,
 * when accept is not NULL, whether its history was reused. For parity
 * checks of full-size frames on a sample of their pixels. Pinned by
 * equality, exact, with or_frame on the same pixels
 * (tests/test_oracle_pixels.py). */
void or_frame_pixels(const or_config *cfg, const or_camera *cam, const or_field *fld, uint32_t frame,
                     const float *g0, const float *g1, const float *g0p, const double *gam_prev,
                     int64_t gstride, int64_t n, const int32_t *xs, const int32_t *ys, double *gam_out,
                     double *img, double *margin, uint8_t *accept)
{
    int spp = cfg->spp, planes = fld->rgb ? 3 : 1;
#pragma omp parallel
    {
        double *buf = malloc(sizeof(double) * 12 * (size_t)spp);
        uint8_t *strat = malloc((size_t)spp);
        or_samples S = {.wx = buf, .wy = buf + spp, .wz = buf + 2 * spp, .radiance = buf + 3 * spp,
                        .pdf = buf + 4 * spp, .mis = buf + 5 * spp, .estimate = buf + 6 * spp,
                        .strategy = strat, .pg = buf + 7 * spp, .pb = buf + 8 * spp, .ux = buf + 9 * spp,
                        .uy = buf + 10 * spp, .margin = buf + 11 * spp};
#pragma omp for schedule(dynamic, 16)
        for (int64_t k = 0; k < n; ++k) {
            int x = xs[k], y = ys[k];
            int32_t q;
            double *gm = gam_out + 8 * k, im[3];
            int acc = reproject_pixel_s(cfg, x, y, g0, g1, g0p, gam_prev, gstride, gm, &q);
            if (accept) accept[k] = (uint8_t)acc;
            sample_pixel_s(cfg, cam, fld, frame, x, y, g0, g1, gm, !acc, &S, im, 0, 1);
            update_pixel_s(cfg, cam, x, y, g0, g1, gm, !acc, S.wx, S.wy, S.wz, S.radiance, S.strategy, 0, 1);
            double m = 1.0;
            for (int t = 0; t < spp; ++t) m = S.margin[t] < m ? S.margin[t] : m;
            margin[k] = m;
            for (int c = 0; c < planes; ++c) img[k * planes + c] = im[c];
        }
        free(buf);
        free(strat);
    }
}

/* One whole frame: reprojection, sampling and training, pixel by pixel.
 * gam_prev and gam_out are HW x 8; samples S may have NULL planes except the
 * ones the training step reads (wx, wy, wz, radiance, strategy). A
 * composition of the steps above, each pinned where it is defined; the reuse,
 * material and colour forms of the frame are pinned in their own tests. */
void or_frame(const or_config *cfg, const or_camera *cam, const or_field *fld, uint32_t frame,
              const float *g0, const float *g1, const float *g0p, const double *gam_prev,
              double *gam_out, uint8_t *accept, or_samples *S, double *img)
{
    int W = cfg->width, H = cfg->height;
    if (cfg->reuse_radius <= 0) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int64_t i = (int64_t)y * W + x;
                int32_t q;
                int acc = reproject_pixel(cfg, x, y, g0, g1, g0p, gam_prev, gam_out + 8 * i, &q);
                if (accept) accept[i] = (uint8_t)acc;
                sample_pixel(cfg, cam, fld, frame, x, y, g0, g1, gam_out + 8 * i, !acc, S, img);
                update_pixel(cfg, cam, x, y, g0, g1, gam_out + 8 * i, !acc, S->wx, S->wy, S->wz,
                             S->radiance, S->strategy);
            }
        return;
    }
    /* with reuse, training needs every pixel's samples of this frame: the
     * paper's two passes (path tracing, then training), Fig. 2 */
    int64_t HW = (int64_t)W * H;
    uint8_t *acc_all = malloc((size_t)HW);
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t i = (int64_t)y * W + x;
            int32_t q;
            acc_all[i] = (uint8_t)reproject_pixel(cfg, x, y, g0, g1, g0p, gam_prev, gam_out + 8 * i, &q);
            sample_pixel(cfg, cam, fld, frame, x, y, g0, g1, gam_out + 8 * i, !acc_all[i], S, img);
        }
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t i = (int64_t)y * W + x;
            update_pixel_reuse(cfg, cam, frame, x, y, g0, g1, gam_out + 8 * i, !acc_all[i], S);
        }
    if (accept) memcpy(accept, acc_all, (size_t)HW);
    free(acc_all);
}

/* Evaluate the mixture at caller-given world directions: for each pixel and
 * each of n directions, the pieces p_g, p_b, p_mix, the two balance weights,
 * f_r cos and the radiance. Output layout [k][n*HW + i] for k = 0..6.
 * Pinned by the mixture-pdf integrals and the MIS weights at the samples,
 * which read it (tests/test_oracle_pins.py). */
void or_eval(const or_config *cfg, const or_camera *cam, const or_field *fld, const float *g0,
             const float *g1, const double *gam, const uint8_t *reinit, int n,
             const double *dirs /* [n*HW][3] */, double *out)
{
    int W = cfg->width, H = cfg->height;
    int64_t HW = (int64_t)W * H, tot = (int64_t)n * HW;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t i = (int64_t)y * W + x;
            pixel_ctx p;
            pixel_setup(cfg, cam, x, y, g0, g1, gam + 8 * i, reinit ? reinit[i] : 0, &p);
            for (int s = 0; s < n; ++s) {
                int64_t o = (int64_t)s * HW + i;
                double wl[3], fcos, pg, pb, pmix, rad, uo[2];
                to_local(p.n, dirs + 3 * o, wl);
                eval_local(fld, &p, wl, NULL, &fcos, &pg, &pb, &pmix, &rad, uo);
                double wg = pmix > 0 ? p.pi_eff * pg / pmix : 0.0;
                double wb = pmix > 0 ? (1.0 - p.pi_eff * p.Z) * pb / pmix : 0.0;
                out[0 * tot + o] = pg;
                out[1 * tot + o] = pb;
                out[2 * tot + o] = pmix;
                out[3 * tot + o] = wg;
                out[4 * tot + o] = wb;
                out[5 * tot + o] = fcos;
                out[6 * tot + o] = rad;
            }
        }
}

/* Per-pixel derived guide: mu, Sigma (regularised), Z, pi_eff. out [HW][8]:
 * mx, my, sxx, syy, sxy, Z, pi_eff, 0. Z as pinned in or_rect_mass. */
void or_derive_pixels(const or_config *cfg, const or_camera *cam, const float *g0,
                      const float *g1, const double *gam, const uint8_t *reinit, double *out)
{
    int W = cfg->width, H = cfg->height;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t i = (int64_t)y * W + x;
            pixel_ctx p;
            pixel_setup(cfg, cam, x, y, g0, g1, gam + 8 * i, reinit ? reinit[i] : 0, &p);
            for (int k = 0; k < 5; ++k) out[8 * i + k] = p.g5[k];
            out[8 * i + 5] = p.Z; out[8 * i + 6] = p.pi_eff; out[8 * i + 7] = 0.0;
        }
}

/* ------------------------------------------------------------------------ */
/* Second-moment loss and its gradient: the differentiable form of the      */
/* guide (not in the paper). theta = (mu_x, mu_y, s_xx, s_yy, s_xy, pi) of  */
/* a pixel's guide, regularised as in the pass. n directions w_i are drawn  */
/* from the guide at theta0 (Philox stream 2) and held fixed, so           */
/*   l(theta) = 1/n sum_i f_i^2 / (p_theta(w_i) p_theta0(w_i)),              */
/* which at theta = theta0 is the Monte Carlo second moment of the          */
/* estimator F = f / p, and                                                  */
/*   dl/dtheta = -1/n sum_i f_i^2 (dp_theta/dtheta) / (p_theta^2 p_theta0).  */
/* With p = pi g + (1 - pi Z) p_b and g = N(u; mu, Sigma)/(2 pi):            */
/*   dp/dpi = g - Z p_b,                                                     */
/*   dp/dmu = pi (g Sigma^-1 d - p_b dZ/dmu),  d = u - mu,                  */
/*   dp/dSigma = pi (g/2 (Sigma^-1 d d^T Sigma^-1 - Sigma^-1) - p_b dZ/dSigma),*/
/* the symmetric off-diagonal entry being one parameter (counted twice).    */
/* A gated pixel (pi_eff = 0) has a loss but no gradient.                   */
/* Pinned by central differences of l and by the quadrature of f^2 / p.     */
/* ------------------------------------------------------------------------ */
static void theta_to_gamma(const double th[6], double gm[8])
{
    gm[G_EX] = th[0]; gm[G_EY] = th[1];
    gm[G_EXX] = th[2] + th[0] * th[0];
    gm[G_EYY] = th[3] + th[1] * th[1];
    gm[G_EXY] = th[4] + th[0] * th[1];
    gm[G_PI] = th[5]; gm[G_K] = 0.0; gm[G_W] = 0.0;
}

static void second_moment_pixel(const or_config *cfg, const or_camera *cam, const or_field *fld,
                                uint32_t frame, int n, int x, int y, const float *g0, const float *g1,
                                const double th0[6], const double th[6], double *loss, double grad[6],
                                double *margin_out)
{
    int W = cfg->width;
    int64_t i = (int64_t)y * W + x;
    double gm0[8], gm[8];
    theta_to_gamma(th0, gm0);
    theta_to_gamma(th, gm);
    pixel_ctx p0, p;
    pixel_setup(cfg, cam, x, y, g0, g1, gm0, 0, &p0);
    pixel_setup(cfg, cam, x, y, g0, g1, gm, 0, &p);
    double dZ[5];
    or_rect_mass_grad(p.g5, dZ);
    double sxx = p.g5[2], syy = p.g5[3], sxy = p.g5[4], det = sxx * syy - sxy * sxy;
    uint32_t key[2] = {cfg->seed_lo, cfg->seed_hi};
    double l = 0.0, gsum[6] = {0, 0, 0, 0, 0, 0}, mmin = 1.0;
    for (int s = 0; s < n; ++s) {
        double wl[3], u[2], margin;
        int valid, have_u;
        draw_direction(&p0, key, (uint32_t)i, frame, (uint32_t)s, 2u, wl, u, &have_u, &valid, &margin);
        if (margin < mmin) mmin = margin;
        if (!valid) continue;
        double fcos0, pg0, pb, pmix0, rad, uo[2], fcos, pg, pmix;
        eval_local(fld, &p0, wl, have_u ? u : NULL, &fcos0, &pg0, &pb, &pmix0, &rad, uo);
        eval_local(fld, &p, wl, uo, &fcos, &pg, &pb, &pmix, &rad, uo);
        if (!(fcos != 0.0) || !(pmix > 0.0) || !(pmix0 > 0.0)) continue;
        double f2 = fcos * fcos;
        l += f2 / (pmix * pmix0);
        if (!(p.pi_eff > 0.0)) continue;
        double dx = uo[0] - p.g5[0], dy = uo[1] - p.g5[1];
        double ix = (syy * dx - sxy * dy) / det, iy = (-sxy * dx + sxx * dy) / det;
        double dp[6];
        dp[0] = p.pi_eff * (pg * ix - pb * dZ[0]);
        dp[1] = p.pi_eff * (pg * iy - pb * dZ[1]);
        dp[2] = p.pi_eff * (pg * 0.5 * (ix * ix - syy / det) - pb * dZ[2]);
        dp[3] = p.pi_eff * (pg * 0.5 * (iy * iy - sxx / det) - pb * dZ[3]);
        dp[4] = p.pi_eff * (pg * (ix * iy + sxy / det) - pb * dZ[4]);
        dp[5] = pg - p.Z * pb;
        double c = f2 / (pmix * pmix * pmix0);
        for (int k = 0; k < 6; ++k) gsum[k] -= c * dp[k];
    }
    *loss = l / n;
    for (int k = 0; k < 6; ++k) grad[k] = gsum[k] / n;
    *margin_out = mmin;
}

/* theta0, theta: [HW][6]; theta may be NULL (= theta0). Outputs loss [HW],
 * grad [HW][6] and the smallest decision margin of each pixel's draws. */
void or_second_moment(const or_config *cfg, const or_camera *cam, const or_field *fld, uint32_t frame,
                      int n, const float *g0, const float *g1, const double *theta0, const double *theta,
                      double *loss, double *grad, double *margin)
{
    int W = cfg->width, H = cfg->height;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t i = (int64_t)y * W + x;
            const double *t0 = theta0 + 6 * i, *t = theta ? theta + 6 * i : t0;
            second_moment_pixel(cfg, cam, fld, frame, n, x, y, g0, g1, t0, t, loss + i, grad + 6 * i,
                                margin + i);
        }
}

/* ------------------------------------------------------------------------ */
/* One Adam step on theta (Kingma & Ba 2015) with projection back onto the  */
/* guide's domain (mean in the square, variances floored, correlation       */
/* clamped, pi clamped), written back to Gamma as moments; k and W are kept.*/
/* gam [HW][8] in/out, grad, m, v [HW][6] (m, v in/out). c1 = 1/(1-b1^t),   */
/* c2 = 1/(1-b2^t) are the bias corrections of step t.                     */
/* Pinned by Adam's first step in closed form and the projection onto     */
/* the guide's domain (tests/test_oracle_pins.py).                         */
/* ------------------------------------------------------------------------ */
void or_adam(const or_config *cfg, int64_t n, double *gam, const double *grad, double *m, double *v,
             double lr, double b1, double b2, double eps, double c1, double c2)
{
    for (int64_t i = 0; i < n; ++i) {
        double *gm = gam + 8 * i, g5[5], th[6];
        derive_gauss(cfg, gm, g5);
        for (int k = 0; k < 5; ++k) th[k] = g5[k];
        th[5] = gm[G_PI];
        for (int k = 0; k < 6; ++k) {
            double g = grad[6 * i + k];
            m[6 * i + k] = b1 * m[6 * i + k] + (1.0 - b1) * g;
            v[6 * i + k] = b2 * v[6 * i + k] + (1.0 - b2) * g * g;
            th[k] -= lr * (m[6 * i + k] * c1) / (sqrt(v[6 * i + k] * c2) + eps);
        }
        th[0] = th[0] < 0.0 ? 0.0 : (th[0] > 1.0 ? 1.0 : th[0]);
        th[1] = th[1] < 0.0 ? 0.0 : (th[1] > 1.0 ? 1.0 : th[1]);
        if (th[2] < cfg->sigma2_min) th[2] = cfg->sigma2_min;
        if (th[3] < cfg->sigma2_min) th[3] = cfg->sigma2_min;
        double lim = cfg->rho_max * sqrt(th[2] * th[3]);
        th[4] = th[4] > lim ? lim : (th[4] < -lim ? -lim : th[4]);
        th[5] = th[5] < cfg->pi_min ? cfg->pi_min : (th[5] > cfg->pi_max ? cfg->pi_max : th[5]);
        double k = gm[G_K], wmass = gm[G_W];
        theta_to_gamma(th, gm);
        gm[G_K] = k; gm[G_W] = wmass;
    }
}

/* ------------------------------------------------------------------------ */
/* Ground truth of a pixel (Eq. 1): the reflected radiance                  */
/*   I(p) = int_H L_i(x, w) f_r(w_o, w) cos(theta) dw,                      */
/* the value whose estimate F the pass returns. FP64 adaptive cubature in   */
/* the polar coordinates of the disk that M lifts to the hemisphere:        */
/*   w_local = (r cos phi sqrt(2 - r^2), r sin phi sqrt(2 - r^2), 1 - r^2),  */
/*   dw = 2 r dr dphi  (the equal-area lift doubles areas),                 */
/* r in [0, 1], phi in [0, 2 pi): the horizon is the edge r = 1, so the     */
/* integrand is smooth inside the domain. Each cell carries a tensor        */
/* Gauss-Legendre rule of GT_NG x GT_NG nodes and an error: how far its     */
/* rule is from the sum over its halves along r, or along phi, whichever is */
/* further. Globally adaptive: the cell with the largest error is halved    */
/* until the summed error is within tol_rel of the result; before that,     */
/* whatever the error, every cell that is large against its distance to a   */
/* known peak of the integrand is halved: each vMF lobe (width 1/sqrt(kappa);*/
/* a lobe below the horizon at its horizon point) and the GGX mirror        */
/* direction (width 2 alpha), so that no peak can hide between nodes.      */
/* A transparent surface sends the view along two deltas:                   */
/*   I = albedo (F L(w_r) + (1 - F) L(w_t)),  F the Fresnel reflectance.     */
/* A coloured field has one integral per channel.                           */
/* Pinned by: constant radiance (I = albedo c), a lobe on the normal and a  */
/* lobe away from the horizon in closed form, the GGX directional albedo by */
/* an independent quadrature over half vectors, a masked field against a    */
/* brute-force grid on the square, and the mean of the pass's own estimator */
/* on workload pixels (tests/test_oracle_ground_truth.py).                  */
/* ------------------------------------------------------------------------ */
#define GT_NG 6
/* integrand evaluations per pixel after which cells are accepted as they are
 * (their differences still enter the reported error): a tolerance below the
 * integrand's own rounding, e.g. 1e-10 at a GGX peak of alpha = 1e-4, where
 * D loses ~1e-8 of its relative precision, would refine without end */
#define GT_MAX_EVALS 4000000L
#define GT_MAX_PEAKS 9

typedef struct {
    const or_field *fld;
    pixel_ctx p;                        /* surface only: normal, position, view, material */
    double t[3], b[3];                  /* basis around the normal */
    int planes;
    int n_peaks;
    double peak[GT_MAX_PEAKS][3], width[GT_MAX_PEAKS];
    double gx[GT_NG], gw[GT_NG];        /* Gauss-Legendre nodes and weights on [-1, 1] */
    double tol_rel;                     /* relative tolerance of the whole integral */
    long evals;                         /* integrand evaluations so far */
} gt_ctx;

/* Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on the
 * Legendre polynomial P_n from the usual cosine starting points, with P_n and
 * its derivative from the three-term recurrence. */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static void gt_dir(double r, double phi, double wl[3])
{
    double s = sqrt(2.0 - r * r);
    wl[0] = r * cos(phi) * s; wl[1] = r * sin(phi) * s; wl[2] = 1.0 - r * r;
}

/* Integrand times the Jacobian 2 r at (r, phi). */
static void gt_eval(const gt_ctx *c, double r, double phi, double out[3])
{
    double wl[3], ww[3];
    gt_dir(r, phi, wl);
    double fc = or_brdf_cos_f0(c->p.rough, c->p.albedo, c->p.f0, c->p.wo_l, wl);
    out[0] = out[1] = out[2] = 0.0;
    if (fc == 0.0) return;
    for (int i = 0; i < 3; ++i) ww[i] = wl[0] * c->t[i] + wl[1] * c->b[i] + wl[2] * c->p.n[i];
    if (c->planes == 3) {
        double L[3];
        or_radiance_rgb(c->fld, c->p.pos, ww, L);
        for (int k = 0; k < 3; ++k) out[k] = L[k] * fc * 2.0 * r;
    } else {
        out[0] = or_radiance(c->fld, c->p.pos, ww) * fc * 2.0 * r;
    }
}

/* The tensor rule on [r0, r1] x [p0, p1]. */
static void gt_rule(gt_ctx *c, double r0, double r1, double p0, double p1, double q[3])
{
    c->evals += GT_NG * GT_NG;
    double hr = 0.5 * (r1 - r0), hp = 0.5 * (p1 - p0), mr = 0.5 * (r0 + r1), mp = 0.5 * (p0 + p1);
    q[0] = q[1] = q[2] = 0.0;
    for (int i = 0; i < GT_NG; ++i)
        for (int j = 0; j < GT_NG; ++j) {
            double v[3];
            gt_eval(c, mr + hr * c->gx[i], mp + hp * c->gx[j], v);
            for (int k = 0; k < 3; ++k) q[k] += c->gw[i] * c->gw[j] * v[k];
        }
    for (int k = 0; k < 3; ++k) q[k] *= hr * hp;
}

/* Whether a cell is large against its distance to a peak: its radius (the
 * largest chord from its centre to a corner or an edge midpoint) above a
 * quarter of max(distance, width). */
static int gt_must_split(const gt_ctx *c, double r0, double r1, double p0, double p1)
{
    double ctr[3], pts[8][3];
    gt_dir(0.5 * (r0 + r1), 0.5 * (p0 + p1), ctr);
    double rs[3] = {r0, 0.5 * (r0 + r1), r1}, ps[3] = {p0, 0.5 * (p0 + p1), p1};
    int m = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (a != 1 || b != 1) gt_dir(rs[a], ps[b], pts[m++]);
    double rad = 0.0;
    for (int k = 0; k < 8; ++k) {
        double dx = pts[k][0] - ctr[0], dy = pts[k][1] - ctr[1], dz = pts[k][2] - ctr[2];
        double d = sqrt(dx * dx + dy * dy + dz * dz);
        if (d > rad) rad = d;
    }
    for (int j = 0; j < c->n_peaks; ++j) {
        double dx = c->peak[j][0] - ctr[0], dy = c->peak[j][1] - ctr[1], dz = c->peak[j][2] - ctr[2];
        double dist = sqrt(dx * dx + dy * dy + dz * dz) - rad;
        if (dist < 0.0) dist = 0.0;
        double scale = dist > c->width[j] ? dist : c->width[j];
        if (rad > 0.25 * scale) return 1;
    }
    return 0;
}

/* One cell of the adaptive cubature: its bounds, its rule's halves along r
 * (ra, rb) and along phi (pa, pb), its estimate (the halves' sum along its
 * worse axis), that axis, its error (the larger difference between its rule
 * and the sum of its halves along either axis, so an error along either axis
 * shows) and whether a peak forces its split. */
typedef struct {
    double r0, r1, p0, p1;
    double ra[3], rb[3], pa[3], pb[3];
    double est[3], err;
    int along_r, forced;
} gt_cellrec;

static void gt_make_cell(gt_ctx *c, double r0, double r1, double p0, double p1, const double q[3], gt_cellrec *e)
{
    double rm = 0.5 * (r0 + r1), pm = 0.5 * (p0 + p1), dr = 0.0, dp = 0.0;
    e->r0 = r0; e->r1 = r1; e->p0 = p0; e->p1 = p1;
    gt_rule(c, r0, rm, p0, p1, e->ra);
    gt_rule(c, rm, r1, p0, p1, e->rb);
    gt_rule(c, r0, r1, p0, pm, e->pa);
    gt_rule(c, r0, r1, pm, p1, e->pb);
    double sr[3], sp[3];
    for (int k = 0; k < 3; ++k) {
        sr[k] = e->ra[k] + e->rb[k];
        sp[k] = e->pa[k] + e->pb[k];
        if (fabs(sr[k] - q[k]) > dr) dr = fabs(sr[k] - q[k]);
        if (fabs(sp[k] - q[k]) > dp) dp = fabs(sp[k] - q[k]);
    }
    for (int k = 0; k < 3; ++k) e->est[k] = dr >= dp ? sr[k] : sp[k];
    e->err = dr > dp ? dr : dp;
    e->forced = gt_must_split(c, r0, r1, p0, p1);
    /* a forced split cuts the longer side (radial extent ~ sqrt(2) dr,
     * azimuthal ~ sqrt(2) r1 dphi: a cell at the pole is cut in r, not into
     * ever thinner wedges); any other split cuts the worse axis */
    e->along_r = e->forced ? (r1 - r0) >= r1 * (p1 - p0) : dr >= dp;
}

/* max-heap of cells: forced splits first, then by error */
static int gt_before(const gt_cellrec *a, const gt_cellrec *b)
{
    if (a->forced != b->forced) return a->forced > b->forced;
    return a->err > b->err;
}

static void gt_push(gt_cellrec *h, long *n, const gt_cellrec *e)
{
    long i = (*n)++;
    h[i] = *e;
    while (i > 0) {
        long up = (i - 1) / 2;
        if (!gt_before(&h[i], &h[up])) break;
        gt_cellrec t = h[i]; h[i] = h[up]; h[up] = t;
        i = up;
    }
}

static void gt_pop(gt_cellrec *h, long *n, gt_cellrec *out)
{
    *out = h[0];
    h[0] = h[--(*n)];
    long i = 0;
    for (;;) {
        long l = 2 * i + 1, r = l + 1, m = i;
        if (l < *n && gt_before(&h[l], &h[m])) m = l;
        if (r < *n && gt_before(&h[r], &h[m])) m = r;
        if (m == i) break;
        gt_cellrec t = h[i]; h[i] = h[m]; h[m] = t;
        i = m;
    }
}

/* Global adaptive cubature over the disk from a base grid of 4 x 16 cells:
 * the cell first in the heap is split while a peak forces a split or the
 * summed error exceeds tol_rel times the summed estimate, within
 * GT_MAX_EVALS evaluations. The sums are kept as the cells change and
 * summed afresh every 1024 splits and at the end. */
static void gt_sums(const gt_cellrec *h, long n, double tot[3], double *terr)
{
    tot[0] = tot[1] = tot[2] = 0.0;
    *terr = 0.0;
    for (long i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) tot[k] += h[i].est[k];
        *terr += h[i].err;
    }
}

static void gt_integrate(gt_ctx *c, double out[3], double *err)
{
    long cap = GT_MAX_EVALS / (4 * GT_NG * GT_NG) + 256, n = 0;
    gt_cellrec *h = malloc(sizeof(gt_cellrec) * (size_t)cap);
    c->evals = 0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 16; ++b) {
            double r0 = 0.25 * a, r1 = 0.25 * (a + 1), p0 = 2.0 * M_PI * b / 16.0, p1 = 2.0 * M_PI * (b + 1) / 16.0;
            double q[3];
            gt_cellrec e;
            gt_rule(c, r0, r1, p0, p1, q);
            gt_make_cell(c, r0, r1, p0, p1, q, &e);
            gt_push(h, &n, &e);
        }
    double tot[3], terr;
    gt_sums(h, n, tot, &terr);
    for (long it = 1;; ++it) {
        double mag = 0.0;
        for (int k = 0; k < 3; ++k) mag = fabs(tot[k]) > mag ? fabs(tot[k]) : mag;
        if (!(h[0].forced || terr > c->tol_rel * mag) || c->evals > GT_MAX_EVALS || n + 2 > cap) break;
        gt_cellrec e, ca, cb;
        gt_pop(h, &n, &e);
        if (e.along_r) {
            double rm = 0.5 * (e.r0 + e.r1);
            gt_make_cell(c, e.r0, rm, e.p0, e.p1, e.ra, &ca);
            gt_make_cell(c, rm, e.r1, e.p0, e.p1, e.rb, &cb);
        } else {
            double pm = 0.5 * (e.p0 + e.p1);
            gt_make_cell(c, e.r0, e.r1, e.p0, pm, e.pa, &ca);
            gt_make_cell(c, e.r0, e.r1, pm, e.p1, e.pb, &cb);
        }
        gt_push(h, &n, &ca);
        gt_push(h, &n, &cb);
        for (int k = 0; k < 3; ++k) tot[k] += ca.est[k] + cb.est[k] - e.est[k];
        terr += ca.err + cb.err - e.err;
        if (it % 1024 == 0) gt_sums(h, n, tot, &terr);
    }
    gt_sums(h, n, out, err);
    free(h);
}

static void gt_add_peak(gt_ctx *c, const double l[3], double width)
{
    if (c->n_peaks >= GT_MAX_PEAKS) return;
    double v[3] = {l[0], l[1], l[2]};
    if (v[2] < 0.0) {   /* below the horizon: the integrand peaks at the nearest horizon point */
        double h = sqrt(v[0] * v[0] + v[1] * v[1]);
        if (h == 0.0) return;
        v[0] /= h; v[1] /= h; v[2] = 0.0;
    }
    for (int k = 0; k < 3; ++k) c->peak[c->n_peaks][k] = v[k];
    c->width[c->n_peaks] = width;
    ++c->n_peaks;
}

/* Ground truth of pixels (xs[k], ys[k]): out[k * planes + c] (planes = 3 for
 * a coloured field, else 1); err[k] (nullable) receives the sum of the
 * accepted cells' differences, a bound on the error of the result. */
void or_ground_truth(const or_config *cfg, const or_camera *cam, const or_field *fld, const float *g0,
                     const float *g1, int64_t n, const int32_t *xs, const int32_t *ys, double tol_rel,
                     double *out, double *err)
{
    double gx[GT_NG], gw[GT_NG];
    gauss_legendre(GT_NG, gx, gw);
    int planes = fld->rgb ? 3 : 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n; ++k) {
        gt_ctx c;
        memset(&c, 0, sizeof(c));
        c.fld = fld;
        c.planes = planes;
        memcpy(c.gx, gx, sizeof(gx));
        memcpy(c.gw, gw, sizeof(gw));
        surface_setup(cfg, cam, xs[k], ys[k], g0, g1, &c.p);
        or_basis(c.p.n, c.t, c.b);
        double res[3] = {0.0, 0.0, 0.0}, e = 0.0;
        if (is_transparent(c.p.rough)) {
            /* the two deltas of the dielectric (Fresnel-weighted, tinted) */
            double ci = c.p.wo_l[2];
            if (ci > 0.0) {
                double fr = or_dielectric_fresnel(ci), eta = 1.0 / DIELECTRIC_IOR;
                double ct = sqrt(1.0 - eta * eta * (1.0 - ci * ci));
                double lr[3] = {-c.p.wo_l[0], -c.p.wo_l[1], ci};
                double lt[3] = {-eta * c.p.wo_l[0], -eta * c.p.wo_l[1], -ct};
                double wr[3], wt[3], Lr[3], Lt[3];
                to_world(c.p.n, lr, wr);
                to_world(c.p.n, lt, wt);
                if (planes == 3) {
                    or_radiance_rgb(fld, c.p.pos, wr, Lr);
                    or_radiance_rgb(fld, c.p.pos, wt, Lt);
                } else {
                    Lr[0] = or_radiance(fld, c.p.pos, wr);
                    Lt[0] = or_radiance(fld, c.p.pos, wt);
                }
                for (int q = 0; q < planes; ++q) res[q] = c.p.albedo * (fr * Lr[q] + (1.0 - fr) * Lt[q]);
            }
        } else {
            for (int j = 0; j < fld->n_lobes; ++j) {
                double dl[3];
                to_local(c.p.n, fld->dir[j], dl);
                gt_add_peak(&c, dl, 1.0 / sqrt(fld->kappa[j]));
            }
            if (c.p.rough >= 0.0) {
                double mir[3] = {-c.p.wo_l[0], -c.p.wo_l[1], c.p.wo_l[2]};
                double w = 2.0 * ggx_alpha(c.p.rough);
                gt_add_peak(&c, mir, w);
            }
            c.tol_rel = tol_rel;
            gt_integrate(&c, res, &e);
        }
        for (int q = 0; q < planes; ++q) out[k * planes + q] = res[q];
        if (err) err[k] = e;
    }
}

/* Threads of the oracle's parallel loops (OpenMP): for timing it on a
 * stated number of host cores. Changes no result: every pixel is computed
 * alone, in the same order of operations, whatever thread runs it. */
void or_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int or_max_threads(void) { return omp_get_max_threads(); }
