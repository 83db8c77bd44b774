/*
 * glint_oracle.c -- plain, slow CPU oracle for per-pixel glint shading under
 * an environment map (Kneiphof & Klein, "Real-Time Image-based Lighting of
 * Glints", EGSR 2025, arXiv 2507.02674).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The CUDA library never
 * links, calls or executes it, and the two share no code, header or table.
 *
 * Precision.  Everything is FP64, with one exception: the quantities that
 * decide an integer before any probability enters -- the footprint area |P|,
 * the microfacet count N_P, the grid level, the grid vertices and the
 * dithering of N_P -- are computed with correctly rounded IEEE single
 * precision operations in a fixed order.  The paper's method is an FP32
 * method (Sec. 5 "Numeric Gating Issues"; its bias constant is tuned for
 * FP32), so those integer decisions are taken in the paper's precision on
 * both sides.  Compile with -ffp-contract=off so that no multiply-add is
 * fused behind our back.
 *
 * Decisions that depend on probabilities (the gating comparisons of Alg. 1
 * and the rounding of the Gaussian count) cannot be reproduced bit for bit by
 * an FP32 kernel.  For each such decision the oracle evaluates how far its
 * threshold can move under a stated relative error of the FP32 inputs
 * (tie model, see or_shade) and, when the uniform number falls inside that
 * band, keeps every outcome as a valid alternative.  A tree therefore yields
 * a small set of valid count vectors; the GPU result must be one of them.
 *
 * Readings of the paper that this file makes (the paper is silent or the
 * source is garbled) are marked "Reading:".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_MAXK 16
#define OR_NV 6 /* grid samples per pixel: 2 levels x 3 triangle vertices */

/* --------------------------------------------------------------------------
 * Hashing and uniform numbers.
 * The paper stores random seeds theta_i at the grid vertices (Sec. 3.3,
 * Eq. anisogrid) but does not name a generator.  Reading: pcg4d of
 * Jarzynski & Olano, "Hash Functions for GPU Rendering", JCGT 9(3), 2020,
 * applied to (vertex x, vertex y, level | call << 16, user seed).  Call 1
 * gives xi0 (the root's dither, word 0) and node 1's xi1 (gating) and xi2
 * (Gaussian) in words 1 and 2; the sibling nodes 2m and 2m+1 of the balanced
 * tree share call m + 1, node 2m taking words 0, 1 and node 2m+1 words 2, 3.
 * ------------------------------------------------------------------------ */
void or_pcg4d(const uint32_t in[4], uint32_t out[4])
{
    uint32_t x = in[0] * 1664525u + 1013904223u;
    uint32_t y = in[1] * 1664525u + 1013904223u;
    uint32_t z = in[2] * 1664525u + 1013904223u;
    uint32_t w = in[3] * 1664525u + 1013904223u;
    x += y * w; y += z * x; z += x * y; w += y * z;
    x ^= x >> 16; y ^= y >> 16; z ^= z >> 16; w ^= w >> 16;
    x += y * w; y += z * x; z += x * y; w += y * z;
    out[0] = x; out[1] = y; out[2] = z; out[3] = w;
}

/* Uniform number in (0,1) from a hash word: the top 23 bits, centred,
 * (2m+1) * 2^-24.  Exactly representable in FP32 and FP64, never 0 or 1,
 * and 1 - xi is exact as well. */
double or_xi(uint32_t h)
{
    return (2.0 * (double)(h >> 9) + 1.0) * 0x1p-24;
}

/* Where tree node `node` (heap order, 1 .. K-1) of the vertex keyed
 * (key0, key1, key2) takes its two uniforms xi1, xi2: the hash call index
 * (`call`, put in bits 16+ of the third key word) and the first of the two
 * consecutive output words (`word`).  Node 1: call 1, words 1 and 2 (word 0
 * is the root's dither); siblings 2m and 2m+1 share call m + 1, words 0, 1
 * and 2, 3. */
void or_node_stream(int node, int *call, int *word)
{
    *call = (node == 1) ? 1 : 1 + node / 2;
    *word = (node == 1) ? 1 : (node & 1) ? 2 : 0;
}

void or_node_uniforms(uint32_t key0, uint32_t key1, uint32_t key2, uint32_t seed, int node, double xi[2])
{
    int call, word;
    or_node_stream(node, &call, &word);
    uint32_t in[4] = {key0, key1, key2 | ((uint32_t)call << 16), seed}, h[4];
    or_pcg4d(in, h);
    xi[0] = or_xi(h[word]);
    xi[1] = or_xi(h[word + 1]);
}

/* Standard normal quantile Phi^-1(p) in FP64.  Starting value from
 * Abramowitz & Stegun 26.2.23 (absolute error < 4.5e-4), refined by Newton
 * steps on Phi(x) = erfc(-x/sqrt 2)/2 from the C library. */
double or_ndtri(double p)
{
    if (!(p > 0.0)) return -INFINITY;
    if (!(p < 1.0)) return INFINITY;
    if (p > 0.5) return -or_ndtri(1.0 - p); /* 1 - p is exact on (0.5, 1) */
    double t = sqrt(-2.0 * log(p));
    double x = -(t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                         (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t));
    for (int it = 0; it < 8; ++it) {
        double f = 0.5 * erfc(-x / sqrt(2.0)) - p;
        double d = exp(-0.5 * x * x) / sqrt(2.0 * OR_PI);
        double dx = f / d;
        x -= dx;
        if (fabs(dx) <= 1e-17 * (1.0 + fabs(x))) break;
    }
    return x;
}

/* --------------------------------------------------------------------------
 * Binomial approximations (Sec. 5).
 * ------------------------------------------------------------------------ */

/* Bias constant of the small-p fix: eps = 10^-3.54 (Sec. 5, "Numeric Gating
 * Issues"). */
double or_eps(void) { return pow(10.0, -3.54); }

/* Thresholds of the dual-gated Gaussian (Alg. 1) for N trials and success
 * probability p, as the four numbers xi1 is compared with:
 *   T[0] = P_{n=N}                       (B_{n=N}      = xi1 <  T[0])
 *   T[1] = P_{n=N} + P_{n=1}             (B_{n in 1,N} = xi1 <  T[1])
 *   T[2] = 1 - P_{nbar=N}                (B_{nbar=N}   = T[2] <= xi1)
 *   T[3] = 1 - P_{nbar=N} - P_{nbar=1}   (B_{nbar in 1,N} = T[3] <= xi1)
 * and the mean and deviation of the Gaussian part.
 * Reading: for p = 0 the bias factor c = max(1, eps/p) is infinite and
 * (1 - c p)^(N/c) is taken at its limit 1. */
void or_dualgated_thresholds(double N, double p, double T[4], double *mu, double *sigma)
{
    double eps = or_eps();
    double N2 = fmax(2.0, N);
    double a = fmin(fmax(N - 1.0, 0.0), 1.0);           /* clamp_[0,1](N-1) */
    double Pall = a * pow(p, N2);
    double Pallneg;
    if (p > 0.0) {
        double c = fmax(1.0, eps / p);
        Pallneg = a * pow(1.0 - c * p, N2 / c);
    } else {
        Pallneg = a;
    }
    double b = fmax(0.0, 1.0 - fabs(1.0 - N));         /* max(0, 1-|1-N|) */
    double Pone = b * p, Poneneg = b * (1.0 - p);
    T[0] = Pall;
    T[1] = Pall + Pone;
    T[2] = 1.0 - Pallneg;
    T[3] = 1.0 - Pallneg - Poneneg;
    *mu = 1.0 + (N2 - 2.0) * p;
    *sigma = sqrt(fmax((N2 - 2.0) * p * (1.0 - p), 0.0));
}

/* Dual-gated Gaussian b_dualgated(N, p, xi1, xi2) -> (n, nbar), Alg. 1,
 * written out step by step.
 * Reading: the clamp interval of G, garbled in the source, is the closed
 * interval [1, N_{>=2} - 1]; Phi^-1(xi; mu, sigma^2) = mu + sigma Phi^-1(xi)
 * (equal to mu when sigma = 0).
 * integer_mode = 0: the paper's real-valued counts.
 * integer_mode = 1 (Reading of "dithered to the nearest integer", Sec. 5):
 * N is an integer, the Gaussian part is rounded half up,
 * G = clamp(floor(mu + sigma z + 1/2), 1, N_{>=2} - 1), and nbar = N - n, which
 * equals Alg. 1's nbar whenever the thresholds partition [0,1) (always, in
 * exact arithmetic) and keeps sum_k n_k = N under rounding. */
void or_dualgated(double N, double p, double xi1, double xi2, int integer_mode,
                  double *n, double *nbar)
{
    double T[4], mu, sigma;
    or_dualgated_thresholds(N, p, T, &mu, &sigma);
    double N2 = fmax(2.0, N);
    double B_all = xi1 < T[0];
    double B_allone = xi1 < T[1];
    double B_allneg = T[2] <= xi1;
    double B_alloneneg = T[3] <= xi1;
    double B_G = (N > 1.0) * (1.0 - B_allone) * (1.0 - B_alloneneg);
    double z = or_ndtri(xi2);
    double G = (sigma > 0.0) ? mu + sigma * z : mu;
    if (integer_mode) G = floor(G + 0.5);
    G = fmin(fmax(G, 1.0), N2 - 1.0);
    double Gbar = N2 - G;
    *n = B_all * (N2 - 1.0) + B_allone + B_G * G;
    if (integer_mode)
        *nbar = N - *n;
    else
        *nbar = B_allneg * (N2 - 1.0) + B_alloneneg + B_G * Gbar;
}

/* Alg. 1 over arrays of uniforms (test convenience). */
void or_dualgated_many(double N, double p, const double *xi1, const double *xi2, long count, int integer_mode,
                       double *n, double *nbar)
{
    for (long i = 0; i < count; ++i) or_dualgated(N, p, xi1[i], xi2[i], integer_mode, n + i, nbar + i);
}

/* Single-gated Gaussian of prior work, Eq. oldgated:
 * floor(chi(xi1 < P_{n>=1}) * clamp_[1,N](Phi^-1(xi2; mu, sigma^2))),
 * mu = 1 + (N-1) p, sigma^2 = (N-1) p (1-p), P_{n>=1} = 1 - (1-p)^N. */
double or_singlegated_old(double N, double p, double xi1, double xi2)
{
    double Pany = 1.0 - pow(1.0 - p, N);
    double mu = 1.0 + (N - 1.0) * p;
    double s2 = (N - 1.0) * p * (1.0 - p);
    double G = mu + sqrt(fmax(s2, 0.0)) * or_ndtri(xi2);
    G = fmin(fmax(G, 1.0), N);
    return floor((xi1 < Pany) * G);
}

/* Generalised single gating for real N >= 0, Eq. gated:
 * chi(xi1 < min(N p, P_{n>=1})) * clamp_[1, max(N,1)](Phi^-1(xi2; mu, sigma^2)). */
double or_singlegated(double N, double p, double xi1, double xi2)
{
    double Pany = 1.0 - pow(1.0 - p, N);
    double gate = fmin(N * p, Pany);
    double mu = 1.0 + (N - 1.0) * p;
    double s2 = (N - 1.0) * p * (1.0 - p);
    double G = (s2 > 0.0) ? mu + sqrt(s2) * or_ndtri(xi2) : mu;
    G = fmin(fmax(G, 1.0), fmax(N, 1.0));
    return (xi1 < gate) * G;
}

/* --------------------------------------------------------------------------
 * Microfacet model (Sec. 3.1, Sec. 6: isotropic GGX, Smith, Schlick).
 * ------------------------------------------------------------------------ */

/* Isotropic GGX NDF as a function of cos(theta_h). */
double or_ggx_d(double cos_h, double alpha)
{
    if (cos_h <= 0.0) return 0.0;
    double c2 = cos_h * cos_h;
    double a2 = alpha * alpha;
    double d = c2 * (a2 - 1.0) + 1.0;
    return a2 / (OR_PI * d * d);
}

/* Smith Lambda for GGX at a direction with cos(theta) = mu. */
static double smith_lambda(double mu, double alpha)
{
    if (mu >= 1.0) return 0.0;
    double t2 = (1.0 - mu * mu) / (mu * mu);
    return 0.5 * (-1.0 + sqrt(1.0 + alpha * alpha * t2));
}

/* Look-up tables over (mu_o, sqrt(alpha)) on an n x n grid of texel centres
 * mu_i = (i+1/2)/n, s_j = (j+1/2)/n, alpha = s_j^2.  Four channels per node:
 *   V = E_D(w_o) / D_H   (visible reflecting microfacet area over the total
 *                         microfacet area, Sec. 4 Eq. rtiblndf and Sec. 3.2)
 *   U = 1 - V            (masked fraction, integrated on its own)
 *   A, B                 (split-sum directional albedo E_rho = F0 A + B,
 *                         Sec. 3.4 Eq. rtibl; Schlick F, height-correlated
 *                         Smith G2 -- Reading of "Smith")
 * Integrals over microfacet normals h:  int f(h) D(h) dh.
 * Quadrature: the GGX projected-area distribution gives
 * D(h) dh = 2 sqrt(a^2 + (1-a^2) s^2) ds dphi/(2 pi) in the variable
 * s = sqrt(1 - u), u the CDF of theta_h (the integrand is bounded there);
 * phi over [0, pi) by the mirror symmetry of the configuration.  V and U
 * integrate the validity indicator over phi in closed form and use a Q*Q
 * point midpoint rule in s; A and B use a Q x Q midpoint rule in (s, phi).
 * E_D(w_o) = int D(h) 1[h.w_o > 0] 1[n.w_i(h) > 0] dh, w_i = reflect(w_o, h)
 * (change of variables of Sec. 3.2).  D_H = int D(h) dh.
 * A = int (1-Fc) G2 D (v.h)/(n.v) dh over valid h, B the same with Fc,
 * Fc = (1 - v.h)^5. */
void or_lut_point(double mu, double alpha, int Q, double out[4])
{
    double a2 = alpha * alpha;
    double sv = sqrt(fmax(1.0 - mu * mu, 0.0));
    /* V and U: for fixed theta_h the valid normals form the arc
     * cos(phi) > c* = -(mu / sin theta_o) cot(2 theta_h) (the condition
     * n.w_i > 0, which implies h.w_o > 0), whose share of [0, pi] is
     * acos(clamp(c*)) / pi; midpoint rule with Q*Q points in s. */
    int ns = Q * Q;
    double sw = 0.0, sv_valid = 0.0, sv_invalid = 0.0;
    for (int a = 0; a < ns; ++a) {
        double s = (a + 0.5) / ns;
        double root2 = a2 + (1.0 - a2) * s * s;
        double w = 2.0 * sqrt(root2);
        double cos2t = (s * s - a2 * (1.0 - s * s)) / root2;
        double sin2t = 2.0 * s * alpha * sqrt(1.0 - s * s) / root2;
        double m;
        if (sv > 0.0) {
            double cstar = -(mu / sv) * cos2t / sin2t;
            m = acos(fmin(fmax(cstar, -1.0), 1.0));
        } else {
            m = (cos2t > 0.0) ? OR_PI : 0.0;
        }
        sw += w;
        sv_valid += w * m;
        sv_invalid += w * (OR_PI - m);
    }
    out[0] = sv_valid / (OR_PI * sw);
    out[1] = sv_invalid / (OR_PI * sw);
    /* A, B: Q x Q midpoint rule in (s, phi in [0, pi)); the integrand vanishes
     * on the boundary of the valid set (G2 -> 0 as n.w_i -> 0). */
    double sA = 0.0, sB = 0.0;
    double lam_o = smith_lambda(mu, alpha);
    for (int a = 0; a < Q; ++a) {
        double s = (a + 0.5) / Q;
        double root = sqrt(a2 + (1.0 - a2) * s * s);
        double w = 2.0 * root;
        double cos_h = s / root;
        double sin_h = alpha * sqrt(1.0 - s * s) / root;
        for (int b = 0; b < Q; ++b) {
            double phi = OR_PI * (b + 0.5) / Q;
            double vh = sv * sin_h * cos(phi) + mu * cos_h;
            double li_z = 2.0 * vh * cos_h - mu;
            if (vh > 0.0 && li_z > 0.0) {
                double G2 = 1.0 / (1.0 + lam_o + smith_lambda(li_z, alpha));
                double Fc = pow(1.0 - vh, 5.0);
                double g = G2 * vh / mu;
                sA += w * (1.0 - Fc) * g;
                sB += w * Fc * g;
            }
        }
    }
    double norm = 1.0 / ((double)Q * (double)Q);
    out[2] = sA * norm;
    out[3] = sB * norm;
}

void or_lut(int n, int Q, double *out)
{
    for (int j = 0; j < n; ++j) {
        double s_tex = (j + 0.5) / n;
        for (int i = 0; i < n; ++i) or_lut_point((i + 0.5) / n, s_tex * s_tex, Q, out + 4 * (j * n + i));
    }
}

/* Quadrature of int D(h) cos(theta_h) dh with the weights of or_lut; the GGX
 * projected microfacet area is exactly 1 (Sec. 3.2). */
double or_projected_area(double alpha, int Q)
{
    double a2 = alpha * alpha, sum = 0.0;
    for (int a = 0; a < Q; ++a) {
        double s = (a + 0.5) / Q;
        double root = sqrt(a2 + (1.0 - a2) * s * s);
        sum += 2.0 * root * (s / root);
    }
    return sum / Q;
}

/* Total microfacet area D_H(alpha) = int D(h) dh by the same quadrature as
 * or_lut (Sec. 3.2: the normaliser of the microfacet distribution). */
double or_total_area(double alpha, int Q)
{
    double a2 = alpha * alpha, sum = 0.0;
    for (int a = 0; a < Q; ++a) {
        double s = (a + 0.5) / Q;
        sum += 2.0 * sqrt(a2 + (1.0 - a2) * s * s);
    }
    return sum / Q;
}

/* Bilinear look-up in the (mu, sqrt alpha) table with texel-centre nodes and
 * clamp-to-edge addressing. */
static void lut_fetch(const double *lut, int n, double mu, double s, double out[4])
{
    double x = mu * n - 0.5, y = s * n - 0.5;
    x = fmin(fmax(x, 0.0), n - 1.0);
    y = fmin(fmax(y, 0.0), n - 1.0);
    int x0 = (int)floor(x), y0 = (int)floor(y);
    int x1 = x0 + 1 < n ? x0 + 1 : n - 1, y1 = y0 + 1 < n ? y0 + 1 : n - 1;
    double fx = x - x0, fy = y - y0;
    for (int c = 0; c < 4; ++c) {
        double v00 = lut[4 * (y0 * n + x0) + c], v01 = lut[4 * (y0 * n + x1) + c];
        double v10 = lut[4 * (y1 * n + x0) + c], v11 = lut[4 * (y1 * n + x1) + c];
        out[c] = (1.0 - fy) * ((1.0 - fx) * v00 + fx * v01) + fy * ((1.0 - fx) * v10 + fx * v11);
    }
}

/* --------------------------------------------------------------------------
 * Environment map: equirectangular, texel (x, y) of a W x H image is centred
 * on phi = 2 pi (x+1/2)/W, theta = pi (y+1/2)/H, direction
 * d(theta, phi) = (sin th cos ph, cos th, sin th sin ph)  (y up).
 * ------------------------------------------------------------------------ */

/* Radiance levels and fuzzy weights, Sec. 4 "Discrete Radiance Levels" and
 * "Fuzzy Indicator Functions", Eq. wkdefpractice.
 *   Y = 0.2126 R + 0.7152 G + 0.0722 B          (Reading: Rec. 709 luminance
 *                                                  as the scalar brightness)
 *   lo = max(min Y, ell), hi = max(max Y, lo)
 *   L_1 = 0, L_k = exp(lerp(ln lo, ln hi, (k-1)/(K-1))) for k >= 2
 *   w_j = 1 - t, w_{j+1} = t, t = (Y - L_j)/(L_{j+1} - L_j), with j the
 *   largest index in [1, K-1] such that L_j <= Y; Y >= L_K gives w_K = 1.
 * rgba: H x W x 4 floats (stored radiance, multiplied by `scale`).
 * ch0: H x W x (3+K) output, channels (R, G, B, w_1 .. w_K). */
void or_env_decompose(const float *rgba, int W, int H, double scale, int K, double ell,
                      double *L, double *lohi, double *ch0, int log_space)
{
    long n = (long)W * H;
    double ymin = INFINITY, ymax = -INFINITY;
    for (long t = 0; t < n; ++t) {
        double R = rgba[4 * t] * scale, G = rgba[4 * t + 1] * scale, B = rgba[4 * t + 2] * scale;
        double Y = fmax(0.2126 * R + 0.7152 * G + 0.0722 * B, 0.0);
        ymin = fmin(ymin, Y);
        ymax = fmax(ymax, Y);
    }
    double lo = fmax(ymin, ell);
    double hi = fmax(ymax, lo);
    lohi[0] = lo;
    lohi[1] = hi;
    L[0] = 0.0;
    for (int k = 2; k <= K; ++k) {
        double a = (double)(k - 1) / (double)(K - 1);
        L[k - 1] = exp(log(lo) + (log(hi) - log(lo)) * a);
    }
    int C = 3 + K;
    for (long t = 0; t < n; ++t) {
        double R = rgba[4 * t] * scale, G = rgba[4 * t + 1] * scale, B = rgba[4 * t + 2] * scale;
        double Y = fmax(0.2126 * R + 0.7152 * G + 0.0722 * B, 0.0);
        double *o = ch0 + C * t;
        o[0] = R; o[1] = G; o[2] = B;
        for (int k = 0; k < K; ++k) o[3 + k] = 0.0;
        if (Y >= L[K - 1]) {
            o[3 + K - 1] = 1.0;
        } else {
            int j = 0; /* 0-based: L[j] <= Y < L[j+1] */
            for (int k = 1; k < K - 1; ++k)
                if (L[k] <= Y) j = k;
            /* Sec. 7 "Linear vs Logarithmic Radiance": the paper assigns weights in
             * linear space; log_space interpolates ln Y between ln L_j and
             * ln L_{j+1} instead, except below L_2 where L_1 = 0 has no logarithm. */
            double tt = (log_space && j > 0) ? (log(Y) - log(L[j])) / (log(L[j + 1]) - log(L[j]))
                                             : (Y - L[j]) / (L[j + 1] - L[j]);
            o[3 + j] = 1.0 - tt;
            o[3 + j + 1] = tt;
        }
    }
}

/* Number of levels of the mip pyramid of a W x H (W = 2H, H a power of two)
 * equirect image, down to 2 x 1. */
int or_mip_count(int H)
{
    int m = 1;
    while ((H >> (m - 1)) > 1) ++m;
    return m;
}

/* Mip pyramid of the (3+K) channels.  Reading: each texel of level m+1 is the
 * solid-angle weighted mean of its 2 x 2 children; the weight of a row of
 * texels spanning [theta0, theta1] is cos(theta0) - cos(theta1).
 * out: all levels concatenated, level m of size (H>>m) x (W>>m) x C. */
void or_env_mips(const double *ch0, int W, int H, int C, double *out)
{
    int M = or_mip_count(H);
    memcpy(out, ch0, sizeof(double) * (size_t)W * H * C);
    const double *src = out;
    double *dst = out + (size_t)W * H * C;
    for (int m = 1; m < M; ++m) {
        int Ws = W >> (m - 1), Hs = H >> (m - 1);
        int Wd = Ws / 2, Hd = Hs / 2;
        for (int y = 0; y < Hd; ++y) {
            double w0 = cos(OR_PI * (2 * y) / Hs) - cos(OR_PI * (2 * y + 1) / Hs);
            double w1 = cos(OR_PI * (2 * y + 1) / Hs) - cos(OR_PI * (2 * y + 2) / Hs);
            for (int x = 0; x < Wd; ++x) {
                for (int c = 0; c < C; ++c) {
                    double a = src[((size_t)(2 * y) * Ws + 2 * x) * C + c] +
                               src[((size_t)(2 * y) * Ws + 2 * x + 1) * C + c];
                    double b = src[((size_t)(2 * y + 1) * Ws + 2 * x) * C + c] +
                               src[((size_t)(2 * y + 1) * Ws + 2 * x + 1) * C + c];
                    dst[((size_t)y * Wd + x) * C + c] = (w0 * a + w1 * b) / (2.0 * (w0 + w1));
                }
            }
        }
        src = dst;
        dst += (size_t)Wd * Hd * C;
    }
}

/* Bilinear look-up on level m of the pyramid: wrap in phi, clamp in theta. */
static void env_bilinear(const double *lev, int Wm, int Hm, int C, const double d[3], double *out)
{
    double th = acos(fmin(fmax(d[1], -1.0), 1.0));
    double ph = atan2(d[2], d[0]);
    if (ph < 0.0) ph += 2.0 * OR_PI;
    double x = ph / (2.0 * OR_PI) * Wm - 0.5;
    double y = th / OR_PI * Hm - 0.5;
    double fx0 = floor(x), fy0 = floor(y);
    double fx = x - fx0, fy = y - fy0;
    long x0 = (long)fx0, y0 = (long)fy0;
    long xa = ((x0 % Wm) + Wm) % Wm, xb = (((x0 + 1) % Wm) + Wm) % Wm;
    long ya = y0 < 0 ? 0 : (y0 > Hm - 1 ? Hm - 1 : y0);
    long yb = y0 + 1 < 0 ? 0 : (y0 + 1 > Hm - 1 ? Hm - 1 : y0 + 1);
    for (int c = 0; c < C; ++c) {
        double v00 = lev[(ya * Wm + xa) * C + c], v01 = lev[(ya * Wm + xb) * C + c];
        double v10 = lev[(yb * Wm + xa) * C + c], v11 = lev[(yb * Wm + xb) * C + c];
        out[c] = (1.0 - fy) * ((1.0 - fx) * v00 + fx * v01) + fy * ((1.0 - fx) * v10 + fx * v11);
    }
}

static size_t mip_offset(int W, int H, int C, int m)
{
    size_t off = 0;
    for (int k = 0; k < m; ++k) off += (size_t)(W >> k) * (H >> k) * C;
    return off;
}

/* Sample table of the environment filter.
 * Sec. 3.4 Eq. rtibl: the map is filtered with p_{L_i}(w_i) proportional to
 * rho~(w_i, w_r) under n = v = r.  Reading: F = G = 1, so p is proportional
 * to D(h), h = normalize(w_i + r), on w_i . r > 0.  The filter is evaluated
 * by filtered importance sampling (the technique of the real-time IBL works
 * the paper cites, Karis 2013 / Lagarde 2014; Colbert & Krivanek, GPU Gems 3
 * ch. 20): S Hammersley points u1 = (j+1/2)/S, u2 = radical inverse of j,
 * cos^2 theta_h = (1-u1)/(1 + (a^2-1) u1), phi_h = 2 pi u2; the reflected
 * direction in the frame (e1, e2, r) is
 * w_i = sin 2th cos ph e1 + sin 2th sin ph e2 + cos 2th r,
 * valid iff cos 2th > 0.  Sampling h with density D cos(theta_h) gives w_i the
 * density D(h)/4 when n = r, so the importance weight p/pdf is constant and
 * the estimate is the plain mean over valid samples.  Each sample reads the
 * pyramid at lod = 0.5 log2(Omega_s / Omega_0) + b, clamped to [0, M-1], with
 * Omega_s = 4 / (S D(h)) and Omega_0 = 4 pi / (W H).  Reading of the bias: the
 * cited works use b = +1; on maps with bright suns b = -1/2 keeps the result
 * closest to the exact convolution (or_prefilter_exact) among b in {+1, +1/2,
 * 0, -1/2, -1} at 64 samples (median luminance error 3-10% instead of 18-25%),
 * so b = -1/2.
 * Levels r = 0..R-1: sqrt(alpha_r) spaced evenly on [s_min, s_max].
 * table: R x S x 4 (e1 weight, e2 weight, r weight, lod; zeros where
 * invalid); nvalid: R; valid samples come first in each level. */
void or_prefilter_table(int R, int S, double s_min, double s_max, int W, int H, double *table, int *nvalid)
{
    int M = or_mip_count(H);
    double omega0 = 4.0 * OR_PI / ((double)W * H);
    for (int r = 0; r < R; ++r) {
        double sr = (R > 1) ? s_min + (s_max - s_min) * r / (R - 1) : s_min;
        double alpha = sr * sr, a2 = alpha * alpha;
        int nv = 0;
        for (int j = 0; j < S; ++j) {
            double u1 = (j + 0.5) / S;
            uint32_t bits = (uint32_t)j, rev = 0;
            for (int b = 0; b < 32; ++b) { rev = (rev << 1) | (bits & 1u); bits >>= 1; }
            double u2 = rev * 0x1p-32;
            double c2 = (1.0 - u1) / (1.0 + (a2 - 1.0) * u1);
            double cos2t = 2.0 * c2 - 1.0;
            if (!(cos2t > 0.0)) continue;
            double c = sqrt(c2), s = sqrt(1.0 - c2);
            double sin2t = 2.0 * s * c;
            double ph = 2.0 * OR_PI * u2;
            double D = or_ggx_d(c, alpha);
            double omega_s = 4.0 / (S * D);
            double lod = 0.5 * log2(omega_s / omega0) - 0.5;
            lod = fmin(fmax(lod, 0.0), (double)(M - 1));
            double *o = table + 4 * ((size_t)r * S + nv);
            o[0] = sin2t * cos(ph);
            o[1] = sin2t * sin(ph);
            o[2] = cos2t;
            o[3] = lod;
            ++nv;
        }
        for (int j = nv; j < S; ++j) {
            double *o = table + 4 * ((size_t)r * S + j);
            o[0] = o[1] = o[2] = o[3] = 0.0;
        }
        nvalid[r] = nv;
    }
}

/* Width of filtered level r (height = width / 2).  Reading: the real-time
 * IBL technique the paper cites (Sec. 3.4, Sec. 4) stores each roughness
 * level as a mip of decreasing resolution; we give level r the power of two
 * nearest (in log2) to 2 pi / alpha_r texels around the equator, i.e. texels
 * of about alpha_r radians, clamped to [min(8, Wmax), Wmax]. */
void or_filtered_widths(int R, double s_min, double s_max, int Wmax, int *widths)
{
    int lo = Wmax < 8 ? Wmax : 8;
    for (int r = 0; r < R; ++r) {
        double sr = (R > 1) ? s_min + (s_max - s_min) * r / (R - 1) : s_min;
        double alpha = sr * sr;
        double e = floor(log2(2.0 * OR_PI / alpha) + 0.5);
        double w = e > 30.0 ? 1073741824.0 : pow(2.0, e);
        if (w > Wmax) w = Wmax;
        if (w < lo) w = lo;
        widths[r] = (int)w;
    }
}

/* Filtered environment: for level r, output texel (y, x) of a W_r x W_r/2
 * equirect grid, the mean over the level's valid samples of the trilinear
 * pyramid look-up (bilinear on levels floor(lod) and floor(lod)+1, linear
 * between) at the sample's reflected direction.
 * Levels are concatenated (level r starts after levels 0..r-1).
 * mips: from or_env_mips.  idx: optional list of `count` flat texel indices
 * into the concatenation (NULL = all texels); out: one C-vector per listed
 * texel. */
void or_prefilter(const double *mips, int W, int H, int C, const double *table, const int *nvalid,
                  int R, int S, const int *widths, const long *idx, long count, double *out)
{
    int M = or_mip_count(H);
    double tmp0[3 + OR_MAXK], tmp1[3 + OR_MAXK];
    long start[65];
    start[0] = 0;
    for (int r = 0; r < R; ++r) start[r + 1] = start[r] + (long)widths[r] * (widths[r] / 2);
    long total = idx ? count : start[R];
#pragma omp parallel for schedule(dynamic, 256) private(tmp0, tmp1)
    for (long q = 0; q < total; ++q) {
        long id = idx ? idx[q] : q;
        int r = 0;
        while (r + 1 < R && id >= start[r + 1]) ++r;
        int Wo = widths[r], Ho = widths[r] / 2;
        long t = id - start[r];
        int y = (int)(t / Wo);
        int x = (int)(t % Wo);
        double th = OR_PI * (y + 0.5) / Ho, ph = 2.0 * OR_PI * (x + 0.5) / Wo;
        double st = sin(th), ct = cos(th), sp = sin(ph), cp = cos(ph);
        double rr[3] = {st * cp, ct, st * sp};
        double e1[3] = {ct * cp, -st, ct * sp};
        double e2[3] = {-sp, 0.0, cp};
        double acc[3 + OR_MAXK];
        for (int c = 0; c < C; ++c) acc[c] = 0.0;
        int nv = nvalid[r];
        for (int j = 0; j < nv; ++j) {
            const double *tb = table + 4 * ((size_t)r * S + j);
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = tb[0] * e1[k] + tb[1] * e2[k] + tb[2] * rr[k];
            double lod = tb[3];
            int m0 = (int)floor(lod);
            double f = lod - m0;
            int m1 = m0 + 1 < M ? m0 + 1 : M - 1;
            env_bilinear(mips + mip_offset(W, H, C, m0), W >> m0, H >> m0, C, d, tmp0);
            env_bilinear(mips + mip_offset(W, H, C, m1), W >> m1, H >> m1, C, d, tmp1);
            for (int c = 0; c < C; ++c) acc[c] += (1.0 - f) * tmp0[c] + f * tmp1[c];
        }
        for (int c = 0; c < C; ++c) out[q * C + c] = nv > 0 ? acc[c] / nv : 0.0;
    }
}

/* Exact filter for comparison: the same kernel p ~ D(h) 1[w_i.r > 0] summed
 * over every texel of level 0 with its solid angle, normalised by the sum of
 * kernel times solid angle (Sec. 3.4 Eq. rtibl as a plain quadrature). */
void or_prefilter_exact(const double *ch0, int W, int H, int C, double alpha, const double *dirs, long count,
                        double *out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (long q = 0; q < count; ++q) {
        const double *r = dirs + 3 * q;
        double acc[3 + OR_MAXK], norm = 0.0;
        for (int c = 0; c < C; ++c) acc[c] = 0.0;
        for (int y = 0; y < H; ++y) {
            double th = OR_PI * (y + 0.5) / H;
            double dOmega = (cos(OR_PI * y / H) - cos(OR_PI * (y + 1) / H)) * 2.0 * OR_PI / W;
            for (int x = 0; x < W; ++x) {
                double ph = 2.0 * OR_PI * (x + 0.5) / W;
                double d[3] = {sin(th) * cos(ph), cos(th), sin(th) * sin(ph)};
                double cd = d[0] * r[0] + d[1] * r[1] + d[2] * r[2];
                if (!(cd > 0.0)) continue;
                double hx = d[0] + r[0], hy = d[1] + r[1], hz = d[2] + r[2];
                double hl = sqrt(hx * hx + hy * hy + hz * hz);
                double cos_h = (hx * r[0] + hy * r[1] + hz * r[2]) / hl;
                double k = or_ggx_d(cos_h, alpha) * dOmega;
                norm += k;
                for (int c = 0; c < C; ++c) acc[c] += k * ch0[((size_t)y * W + x) * C + c];
            }
        }
        for (int c = 0; c < C; ++c) out[q * C + c] = norm > 0.0 ? acc[c] / norm : 0.0;
    }
}

/* --------------------------------------------------------------------------
 * E2: reflection probabilities of an anisotropic GGX footprint by quadrature.
 *
 * Eq. probhk without the n = v = r approximation of Eq. rtiblndf:
 *   p_k = int D(h) 1[n.w_i(h) > 0] w_k(w_i(h)) dh / int D(h) dh      (k >= 2)
 *   p_1 = (int D(h) 1[n.w_i <= 0] dh + int D(h) 1[n.w_i > 0] w_1 dh) / int D(h) dh
 * with w_i(h) = reflect(w_o, h) (Sec. 3.2 change of variables) and the
 * masked mass in bin 1 as in the E1 path.  Quadrature (Reading; the paper only
 * treats the isotropic case): the GGX projected-area slope distribution with
 * u1 = 1 - s^2 (the CDF of the standard slope radius), so r = sqrt(1-s^2)/s,
 * slope = (a_x r cos phi, a_y r sin phi), phi = 2 pi u2, h' = (-slope, 1) in
 * the frame (t, b = n x t, n).  Since D(h) dh = (D cos dh)/cos and
 * du1 = 2 s ds, a point carries the bounded weight
 * 2 s / cos(theta_h) = 2 sqrt(s^2 + rho^2 (1 - s^2)), rho^2 = a_x^2 cos^2 phi +
 * a_y^2 sin^2 phi; S x S midpoint points in (s, u2).  A point is valid iff
 * 2 (w_o . h') > mu_o |h'|^2 (<=> n . w_i > 0).  The weights w_k(w_i) are read
 * bilinearly from pyramid level m, the coarsest level whose texel (pi / H_m
 * radians) is at most 4 min(a_x, a_y) / S; the comparison is made in FP32 as
 * (float)H_m * (min(a_x, a_y) * (4/S)) >= (float)pi, exact for powers of two.
 * Returns the number of points whose validity margin is below 1e-5 of its
 * scale (FP32 may classify those either way). */
int or_e2_pk(const double wo[3], const double nn[3], const double tg[3], float ax, float ay, int S,
             const double *mips, int W, int H, int C, int K, double *pk)
{
    int M = or_mip_count(H);
    float x = fminf(ax, ay) * (4.0f / (float)S);
    int m = 0;
    for (int k = 0; k < M; ++k)
        if ((float)(H >> k) * x >= (float)OR_PI) m = k;
    const double *lev = mips + mip_offset(W, H, C, m);
    int Wm = W >> m, Hm = H >> m;
    /* frame: tangent made orthogonal to n */
    double tn = tg[0] * nn[0] + tg[1] * nn[1] + tg[2] * nn[2];
    double t[3] = {tg[0] - tn * nn[0], tg[1] - tn * nn[1], tg[2] - tn * nn[2]};
    double tl = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    for (int i = 0; i < 3; ++i) t[i] /= tl;
    double b[3] = {nn[1] * t[2] - nn[2] * t[1], nn[2] * t[0] - nn[0] * t[2], nn[0] * t[1] - nn[1] * t[0]};
    double mu = wo[0] * nn[0] + wo[1] * nn[1] + wo[2] * nn[2];
    double ot = wo[0] * t[0] + wo[1] * t[1] + wo[2] * t[2];
    double ob = wo[0] * b[0] + wo[1] * b[1] + wo[2] * b[2];
    double sum_all = 0.0, sum_inv = 0.0, acc[OR_MAXK];
    double ch[3 + OR_MAXK];
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    int flagged = 0;
    for (int a = 0; a < S; ++a) {
        double sv = (a + 0.5) / S;
        double r = sqrt(1.0 - sv * sv) / sv;
        for (int c = 0; c < S; ++c) {
            double u2 = (c + 0.5) / S;
            double cp = cos(2.0 * OR_PI * u2), sp = sin(2.0 * OR_PI * u2);
            double sx = ax * r * cp, sy = ay * r * sp;
            double rho2 = (double)ax * ax * cp * cp + (double)ay * ay * sp * sp;
            double wgt = 2.0 * sqrt(sv * sv + rho2 * (1.0 - sv * sv));
            double hl2 = 1.0 + sx * sx + sy * sy;
            double hl = sqrt(hl2);
            double oh = -sx * ot - sy * ob + mu; /* w_o . h' */
            double margin = 2.0 * oh - mu * hl2;
            double scale = 2.0 * fabs(oh) + fabs(mu) * hl2;
            if (fabs(margin) < 1e-5 * scale) ++flagged;
            sum_all += wgt;
            if (!(margin > 0.0)) {
                sum_inv += wgt;
                continue;
            }
            /* w_i = 2 (w_o . h) h - w_o, h = h'/|h'| */
            double hw[3];
            for (int i = 0; i < 3; ++i) hw[i] = (-sx * t[i] - sy * b[i] + nn[i]) / hl;
            double oh_n = oh / hl;
            double wi[3];
            for (int i = 0; i < 3; ++i) wi[i] = 2.0 * oh_n * hw[i] - wo[i];
            env_bilinear(lev, Wm, Hm, C, wi, ch);
            for (int k = 0; k < K; ++k) acc[k] += wgt * ch[3 + k];
        }
    }
    pk[0] = (sum_inv + acc[0]) / sum_all;
    for (int k = 1; k < K; ++k) pk[k] = acc[k] / sum_all;
    return flagged;
}

/* --------------------------------------------------------------------------
 * Inputs of the p_k surrogate (the learned part has no counterpart in the
 * paper; this is the definition the library documents).  Per pixel row of
 * the G-buffer (16 floats) and tangent (4 floats):
 *   x[0..K)      p_k of E1 (Eq. rtiblndf: V W_k, p_1 = U + V W_1)
 *   x[K..6K)     W_k of the filtered maps at roughness parameter
 *                s = sqrt(min(a_x, a_y)) in five directions: w_r, then
 *                normalize(w_r + a_x J_t), normalize(w_r - a_x J_t),
 *                normalize(w_r + a_y J_b), normalize(w_r - a_y J_b), with
 *                J_t = 2 (-(w_o.t) n - mu_o t) the derivative of the mirror
 *                direction with respect to the slope along t (tangent made
 *                orthogonal to n), J_b likewise for b = n x t
 *   x[6K..6K+3)  mu_o, sqrt a_x, sqrt a_y;  x[6K+3..64) = 0
 *   lp[k]        log max(p_k^E1, 1e-6)
 * Background rows (N_0 <= 0) are all zero.  dirs (optional, npix x 5 x 3):
 * the five unit directions.
 * ------------------------------------------------------------------------ */
static void filtered_at(const double *pref, int R, const int *widths, int C, double s_min, double s_max,
                        double s, const double d[3], double *cc)
{
    double tl = (R > 1) ? (s - s_min) / (s_max - s_min) * (R - 1) : 0.0;
    tl = fmin(fmax(tl, 0.0), (double)(R - 1));
    int r0 = (int)floor(tl);
    int r1 = r0 + 1 < R ? r0 + 1 : R - 1;
    double ft = tl - r0;
    size_t off0 = 0, off1 = 0;
    for (int r = 0; r < r0; ++r) off0 += (size_t)widths[r] * (widths[r] / 2) * C;
    for (int r = 0; r < r1; ++r) off1 += (size_t)widths[r] * (widths[r] / 2) * C;
    double c0[3 + OR_MAXK], c1[3 + OR_MAXK];
    env_bilinear(pref + off0, widths[r0], widths[r0] / 2, C, d, c0);
    env_bilinear(pref + off1, widths[r1], widths[r1] / 2, C, d, c1);
    for (int i = 0; i < C; ++i) cc[i] = (1.0 - ft) * c0[i] + ft * c1[i];
}

/* --------------------------------------------------------------------------
 * Anisotropic E1 by multi-tap prefiltered look-ups (the multiple filtered
 * look-ups along an anisotropic lobe that the paper's related work and its
 * limitations section point to for anisotropic materials).
 * Reading: the lobe of reflected directions w_i is taken as an ellipse whose
 * axes are the images of the slope axes t and b: J_t a_x and J_b a_y, with
 * J_t = 2 (-(w_o.t) n - mu_o t), J_b likewise, the derivatives of the mirror
 * direction with respect to the slope (t made orthogonal to n, b = n x t).
 * With L_t = |J_t| a_x, L_b = |J_b| a_y, L_min <= L_max and u the unit
 * direction of the longer one, the filtered maps are read at roughness
 * a_l = L_min / 2 (the isotropic lobe of the minor axis; |J| = 2 at normal
 * incidence) at the five nodes x_j of the Gauss-Hermite rule (weights w_j)
 * along u: d_j = normalize(w_r + x_j sigma u), sigma^2 = 0.4 (L_max^2 -
 * L_min^2) (the factor measured against E2 on a 1080p scene other than the
 * benchmark frame, from 0.25 .. 0.6), and W_k = sum_j w_j W_k(d_j, a_l).
 * p_k = V W_k (k >= 2), p_1 = U + V W_1 with V, U as E1 (table at
 * sqrt(a_x a_y)).  An isotropic material seen head-on gives sigma = 0 and
 * a_l = alpha: E1 exactly.
 * ------------------------------------------------------------------------ */
static const double OR_GH5_X[5] = {0.0, -1.3556261799742659, 1.3556261799742659, -2.8569700138728056,
                                   2.8569700138728056};
static const double OR_GH5_W[5] = {0.53333333333333333, 0.22207592200561265, 0.22207592200561265,
                                   0.011257411327720690, 0.011257411327720690};

static void or_e1a_weights(const double wo[3], const double n[3], const double tg[3], double ax, double ay,
                           const double *pref, int R, const int *widths, int C, double s_min, double s_max, double *W)
{
    double mu = n[0] * wo[0] + n[1] * wo[1] + n[2] * wo[2];
    double wr[3], t[3], b[3], Jt[3], Jb[3];
    for (int i = 0; i < 3; ++i) wr[i] = 2.0 * mu * n[i] - wo[i];
    double tn = tg[0] * n[0] + tg[1] * n[1] + tg[2] * n[2];
    for (int i = 0; i < 3; ++i) t[i] = tg[i] - tn * n[i];
    double tl = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    for (int i = 0; i < 3; ++i) t[i] /= tl;
    b[0] = n[1] * t[2] - n[2] * t[1];
    b[1] = n[2] * t[0] - n[0] * t[2];
    b[2] = n[0] * t[1] - n[1] * t[0];
    double ot = wo[0] * t[0] + wo[1] * t[1] + wo[2] * t[2];
    double ob = wo[0] * b[0] + wo[1] * b[1] + wo[2] * b[2];
    for (int i = 0; i < 3; ++i) {
        Jt[i] = 2.0 * (-ot * n[i] - mu * t[i]);
        Jb[i] = 2.0 * (-ob * n[i] - mu * b[i]);
    }
    double nt = sqrt(Jt[0] * Jt[0] + Jt[1] * Jt[1] + Jt[2] * Jt[2]);
    double nb = sqrt(Jb[0] * Jb[0] + Jb[1] * Jb[1] + Jb[2] * Jb[2]);
    double Lt = nt * ax, Lb = nb * ay;
    double Lmin = fmin(Lt, Lb), Lmax = fmax(Lt, Lb);
    double u[3];
    for (int i = 0; i < 3; ++i) u[i] = (Lt >= Lb) ? Jt[i] / nt : Jb[i] / nb;
    double a_l = fmin(fmax(0.5 * Lmin, 1e-4), 1.0);
    double s = sqrt(a_l);
    double sigma = sqrt(0.4 * (Lmax * Lmax - Lmin * Lmin));
    double cc[3 + OR_MAXK];
    for (int c = 0; c < C - 3; ++c) W[c] = 0.0;
    for (int j = 0; j < 5; ++j) {
        double d[3];
        for (int i = 0; i < 3; ++i) d[i] = wr[i] + OR_GH5_X[j] * sigma * u[i];
        double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int i = 0; i < 3; ++i) d[i] /= dl;
        filtered_at(pref, R, widths, C, s_min, s_max, s, d, cc);
        for (int c = 0; c < C - 3; ++c) W[c] += OR_GH5_W[j] * cc[3 + c];
    }
}

void or_mlp_features(const float *gb, const float *tangents, long npix, const double *pref, int R, const int *widths,
                     int C, double s_min, double s_max, const double *lut, int nlut, int K, double *x, double *lp,
                     double *dirs)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (long q = 0; q < npix; ++q) {
        const float *g = gb + 16 * q;
        double *xq = x + 64 * q;
        for (int i = 0; i < 64; ++i) xq[i] = 0.0;
        for (int k = 0; k < K; ++k) lp[q * K + k] = 0.0;
        if (!(g[3] > 0.0f)) continue;
        double wo[3] = {g[0], g[1], g[2]}, n[3] = {g[4], g[5], g[6]};
        double ax = g[10], ay = g[11];
        double mu = n[0] * wo[0] + n[1] * wo[1] + n[2] * wo[2];
        double wr[3];
        for (int i = 0; i < 3; ++i) wr[i] = 2.0 * mu * n[i] - wo[i];
        /* E1 */
        double s_iso = sqrt(sqrt(ax * ay));
        double tab[4], cc[3 + OR_MAXK];
        lut_fetch(lut, nlut, fmin(fmax(mu, 1e-4), 1.0), s_iso, tab);
        filtered_at(pref, R, widths, C, s_min, s_max, s_iso, wr, cc);
        xq[0] = tab[1] + tab[0] * cc[3];
        for (int k = 1; k < K; ++k) xq[k] = tab[0] * cc[3 + k];
        for (int k = 0; k < K; ++k) lp[q * K + k] = log(fmax(xq[k], 1e-6));
        /* lobe axes */
        const float *tg = tangents + 4 * q;
        double tn = tg[0] * n[0] + tg[1] * n[1] + tg[2] * n[2];
        double t[3] = {tg[0] - tn * n[0], tg[1] - tn * n[1], tg[2] - tn * n[2]};
        double tl = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        for (int i = 0; i < 3; ++i) t[i] /= tl;
        double b[3] = {n[1] * t[2] - n[2] * t[1], n[2] * t[0] - n[0] * t[2], n[0] * t[1] - n[1] * t[0]};
        double ot = wo[0] * t[0] + wo[1] * t[1] + wo[2] * t[2];
        double ob = wo[0] * b[0] + wo[1] * b[1] + wo[2] * b[2];
        double Jt[3], Jb[3];
        for (int i = 0; i < 3; ++i) {
            Jt[i] = 2.0 * (-ot * n[i] - mu * t[i]);
            Jb[i] = 2.0 * (-ob * n[i] - mu * b[i]);
        }
        double s_tap = sqrt(fmin(ax, ay));
        for (int tap = 0; tap < 5; ++tap) {
            double d[3];
            for (int i = 0; i < 3; ++i) {
                double off = 0.0;
                if (tap == 1) off = ax * Jt[i];
                if (tap == 2) off = -ax * Jt[i];
                if (tap == 3) off = ay * Jb[i];
                if (tap == 4) off = -ay * Jb[i];
                d[i] = wr[i] + off;
            }
            double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            for (int i = 0; i < 3; ++i) d[i] /= dl;
            if (dirs)
                for (int i = 0; i < 3; ++i) dirs[(q * 5 + tap) * 3 + i] = d[i];
            filtered_at(pref, R, widths, C, s_min, s_max, s_tap, d, cc);
            for (int k = 0; k < K; ++k) xq[K + tap * K + k] = cc[3 + k];
        }
        xq[6 * K] = mu;
        xq[6 * K + 1] = sqrt(ax);
        xq[6 * K + 2] = sqrt(ay);
    }
}

/* --------------------------------------------------------------------------
 * Per-pixel shading.
 * ------------------------------------------------------------------------ */

/* |P| = |du/dx dv/dy - du/dy dv/dx| in FP32: the 2 x 2 determinant with one
 * fused multiply-add correction (Kahan), then N_P = N_0 |P| (Sec. 3.2: the
 * microfacets are stratified, so N_P equals its expectation). */
static float f32_footprint_area(float dudx, float dvdx, float dudy, float dvdy)
{
    float w = dudy * dvdx;
    float e = fmaf(-dudy, dvdx, w);
    float f = fmaf(dudx, dvdy, -w);
    return fabsf(f + e);
}

/* Grid level: l0 = floor(log2(sqrt|P|)) from the FP32 exponent of |P|
 * (exact), f = log2(sqrt|P|) - l0 in FP64.  Reading (the grid of Sec. 3.3 is
 * a black box in the paper): one level per octave of footprint size, cells as
 * large as the footprint, l0 clamped to [-24, 23]. */
static void grid_level(float area, int *l0, double *frac)
{
    int e;
    float m = frexpf(area, &e); /* area = m 2^e, m in [1/2, 1) */
    int ep = e - 1;             /* area = (2m) 2^ep, 2m in [1, 2) */
    int l = (ep >= 0) ? ep / 2 : -((-ep + 1) / 2);
    double f = 0.5 * ((double)(ep - 2 * l) + log2(2.0 * (double)m));
    if (l < -24) { l = -24; f = 0.0; }
    if (l > 23) { l = 23; f = 1.0; }
    *l0 = l;
    *frac = f;
}

/* Triangle grid vertices at one level (Sec. 3.3: "a triangle grid in the
 * space of uv coordinates").  Reading: the equilateral lattice of 2-D simplex
 * noise; the point (u,v) 2^-l is skewed by F = (sqrt 3 - 1)/2 (FP32 constant
 * 0x3EBB67AF), the skewed cell (i, j) is split along its diagonal, and the
 * barycentric weights of the three corners are taken in skewed coordinates.
 * The skew and the vertex choice use FP32 operations in this order. */
static void lattice_vertices(float x, float y, int64_t vx[3], int64_t vy[3], double b[3])
{
    const float F2 = 0x1.76cf5ep-2f; /* (sqrt(3)-1)/2 rounded to FP32 */
    float t = x + y;
    float s = t * F2;
    float xs = x + s, ys = y + s;
    float fi = floorf(xs), fj = floorf(ys);
    float fx = xs - fi, fy = ys - fj;
    int64_t i = (int64_t)fi, j = (int64_t)fj;
    vx[0] = i; vy[0] = j;
    vx[2] = i + 1; vy[2] = j + 1;
    if (fx > fy) {
        vx[1] = i + 1; vy[1] = j;
        b[0] = 1.0 - (double)fx; b[1] = (double)fx - (double)fy; b[2] = (double)fy;
    } else {
        vx[1] = i; vy[1] = j + 1;
        b[0] = 1.0 - (double)fy; b[1] = (double)fy - (double)fx; b[2] = (double)fx;
    }
}

static void grid_vertices(float u, float v, int l, int64_t vx[3], int64_t vy[3], double b[3])
{
    lattice_vertices(ldexpf(u, -l), ldexpf(v, -l), vx, vy, b);
}

/* Anisotropic grid (our reading of the anisotropic grids Sec. 3.3 builds on:
 * cells over the footprint's length, anisotropy factor and orientation).  The footprint
 * ellipse of the uv Jacobian J = [du/dx du/dy; dv/dx dv/dy] has eigenvalues
 * lam1 >= lam2 of J J^T = [a b; b c].  Coordinates: the level L = l0 + fl
 * (log2 sqrt|P|, as grid_level), the anisotropy A = (log2 lam1 - log2 |P|)/2
 * = log2(sqrt(lam1/lam2))/2 clamped to [0, 2], and the orientation
 * O = (4/pi) atan2(b, (a - c)/2) in [0, 8) (the major axis at O pi/8),
 * periodic.  N_P is spread over the Freudenthal tetrahedron of the cell:
 * fractions sorted in decreasing order (ties: L, A, O) give the unit steps
 * and the weights 1 - f1, f1 - f2, f2 - f3, f3; vertices with a = 0 take
 * o = 0.  Returns 1 when a decision (a floor or the order of two fractions)
 * lies within reach of an FP32 evaluation of the same quantities. */
static int footprint_cell(const float *g, float area, int l0, double fl, int tl[4], int ta[4], int to[4],
                          double tw[4])
{
    double dudx = g[12], dvdx = g[13], dudy = g[14], dvdy = g[15];
    double ea = dudx * dudx + dudy * dudy, ec = dvdx * dvdx + dvdy * dvdy, eb = dudx * dvdx + dudy * dvdy;
    double hd = 0.5 * (ea - ec);
    double rr = sqrt(hd * hd + eb * eb);
    double lam1 = 0.5 * (ea + ec) + rr;
    double Araw = 0.5 * (log2(lam1) - log2((double)area));
    double A = fmin(fmax(Araw, 0.0), 2.0);
    double O = atan2(eb, hd) * (4.0 / OR_PI);
    if (O < 0.0) O += 8.0;
    if (O >= 8.0) O -= 8.0;
    int a0 = (A >= 2.0) ? 2 : (int)floor(A);
    double fa = A - a0;
    int o0 = (int)floor(O);
    if (o0 > 7) o0 = 7;
    double fo = O - o0;
    double f[3] = {fl, fa, fo};
    int ord[3] = {0, 1, 2};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2 - i; ++j)
            if (f[ord[j + 1]] > f[ord[j]]) { int t = ord[j]; ord[j] = ord[j + 1]; ord[j + 1] = t; }
    int cl = l0, ca = a0, co = o0;
    for (int v = 0; v < 4; ++v) {
        if (v > 0) {
            int ax = ord[v - 1];
            if (ax == 0) ++cl; else if (ax == 1) ++ca; else co = (co + 1) & 7;
        }
        tl[v] = cl;
        ta[v] = ca;
        to[v] = (ca == 0) ? 0 : co;
        double hi = (v == 0) ? 1.0 : f[ord[v - 1]];
        double lo = (v == 3) ? 0.0 : f[ord[v]];
        tw[v] = hi - lo;
    }
    /* reach of the FP32 evaluation: log2 and sqrt of values ~2^+-60 carry a
     * few 1e-6 absolute; the orientation's angle is ill-conditioned when the
     * footprint is nearly round (rr small against a + c) */
    const double tau = 4e-5;
    double tauO = tau + (4.0 / OR_PI) * 1e-6 * (ea + ec) / fmax(2.0 * rr, 1e-300);
    int flag = 0;
    if (Araw > tau && Araw < 2.0 - tau && fabs(A - floor(A + 0.5)) < tau) flag = 1;  /* floor of A */
    double dO = fabs(O - floor(O + 0.5));
    if (dO < tauO || 8.0 - O < tauO) flag = 1;                                          /* floor of O */
    double tf[3] = {tau, tau, tauO};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (fabs(f[i] - f[j]) < tf[i] + tf[j]) flag = 1;                          /* step order */
    return flag;
}

/* FP32 cos and sin of the orientations o pi / 8 of the anisotropic grid,
 * built from cos(pi/8), sin(pi/8) and sqrt(2)/2 rounded to FP32. */
static void orient_table(float cs[8], float sn[8])
{
    const float c1 = (float)cos(OR_PI / 8.0), s1 = (float)sin(OR_PI / 8.0), h = (float)(sqrt(2.0) / 2.0);
    const float cc[8] = {1.0f, c1, h, s1, 0.0f, -s1, -h, -c1};
    const float ss[8] = {0.0f, s1, h, c1, 1.0f, c1, h, s1};
    for (int k = 0; k < 8; ++k) { cs[k] = cc[k]; sn[k] = ss[k]; }
}

/* Tie model of the FP32 kernel, used to decide when a decision is too close
 * to call:  tie[0] = e_P  relative error bound of each subtree probability
 *                         mass (prefilter, look-up tables, interpolation)
 *           tie[1] = e_z  relative error bound of the FP32 normal quantile
 *           tie[2] = e_f  relative error bound of an FP32 exp2/log2 chain
 *           tie[3] = d_a  absolute floor of every threshold tolerance
 *           tie[4] = a_P  absolute error bound of each subtree mass (E2 reads
 *                         single pyramid texels per quadrature point) */
typedef struct {
    int K, integer_mode;
    int draw; /* 0 dual-gated (Alg. 1), 1 single-gated (Eq. gated), 2 Eq. oldgated */
    uint32_t key0, key1, key2, seed;
    double P[2 * OR_MAXK];
    double tie[5];
    int max_cand, n_out, overflow, flagged;
    double *out;     /* max_cand x K leaf counts */
    double *out_err; /* max_cand x K leaf count tolerance */
} tree_ctx;

/* Probability of no positive trial among N, in the small-p biased form of
 * Sec. 5: (1 - c p)^(N/c), c = max(1, eps/p) (exactly (1-p)^N for p >= eps). */
static double single_pnone(double N, double p)
{
    if (!(p > 0.0)) return 1.0;
    if (p >= 1.0) return N > 0.0 ? 0.0 : 1.0;
    double c = fmax(1.0, or_eps() / p);
    return pow(1.0 - c * p, N / c);
}

static double thr_eval_err(double T, double a, double e_f)
{
    /* FP32 evaluation of a * exp2(X): relative error ~ (|X ln 2| + 1) e_f */
    if (!(T > 0.0)) return 0.0;
    double lx = (a > 0.0) ? fabs(log(T / a)) : 0.0;
    return T * (lx + 2.0) * e_f;
}

typedef struct { double n, nb, en, eb; } outcome;

/* Append an outcome unless an identical one is already listed. */
static int push_outcome(outcome *list, int cnt, double n, double nb, double en, double eb)
{
    for (int i = 0; i < cnt; ++i)
        if (list[i].n == n && list[i].nb == nb) return cnt;
    list[cnt].n = n; list[cnt].nb = nb; list[cnt].en = en; list[cnt].eb = eb;
    return cnt + 1;
}

/* Evaluate node `node` of the multinomial tree (heap order) for the trials
 * N[node] (tolerance dN[node]) and recurse; every valid outcome is listed,
 * the nominal FP64 outcome first. */
static void tree_rec(tree_ctx *t, int node, double *N, double *dN);

/* One tree node with a single-gated Gaussian (Sec. 5: Eq. gated, or with
 * draw 2 Eq. oldgated).  The gate opens when 1 - xi1 > (1 - c p)^(N/c) (at
 * least one positive trial) and, for Eq. gated with real N, also xi1 < N p;
 * an open gate gives the Gaussian N(1 + (N-1) p, (N-1) p (1-p)) clamped to
 * [1, max(N, 1)] (rounded half up for integer counts; Eq. oldgated takes the
 * floor), a closed one 0; the right child gets max(N - n, 0).  Decisions
 * within the tie model's reach enumerate both outcomes, as for Alg. 1. */
static void tree_single(tree_ctx *t, int node, double *N, double *dN, double Nn, double dNn, double PL, double PR,
                        double p, double xi1, double xi2, int use_tie)
{
    int old = t->draw == 2;
    double e_P = t->tie[0], e_z = t->tie[1], e_f = t->tie[2], d_a = t->tie[3], a_P = t->tie[4];
    double xi1c = 1.0 - xi1;
    double Pn = single_pnone(Nn, p);
    double mu = 1.0 + (Nn - 1.0) * p, s2 = (Nn - 1.0) * p * (1.0 - p);
    double sigma = s2 > 0.0 ? sqrt(s2) : 0.0;
    double z = or_ndtri(xi2);
    double G = mu + sigma * z;
    double Np = Nn * p;
    double tauP = 0.0, tauG = 0.0, tauN = 0.0;
    if (use_tie) {
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            double pp = p;
            if (PL + PR > 0.0) {
                double pl = fmax(PL * (1.0 + sgn * e_P) + sgn * a_P, 0.0);
                double pr = fmax(PR * (1.0 - sgn * e_P) - sgn * a_P, 0.0);
                if (pl + pr > 0.0) pp = pl / (pl + pr);
            }
            for (int sn = -1; sn <= 1; sn += 2) {
                double Nq = fmax(Nn + sn * dNn, 0.0);
                tauP = fmax(tauP, fabs(single_pnone(Nq, pp) - Pn));
                double s22 = (Nq - 1.0) * pp * (1.0 - pp);
                double G2 = 1.0 + (Nq - 1.0) * pp + (s22 > 0.0 ? sqrt(s22) : 0.0) * z;
                tauG = fmax(tauG, fabs(G2 - G));
                tauN = fmax(tauN, fabs(Nq * pp - Np));
            }
        }
        tauP += thr_eval_err(Pn, 1.0, e_f) + d_a;
        tauG += sigma * (fabs(z) * e_z + 0x1p-22) + fabs(G) * 0x1p-22 + 0x1p-24;
        tauN += Np * 0x1p-22 + d_a;
    }
    int real_gate = !t->integer_mode && !old;
    int open_nom = (xi1c > Pn) && (!real_gate || xi1 < Np);
    int can_open = (xi1c > Pn - tauP) && (!real_gate || xi1 < Np + tauN);
    int can_close = (xi1c <= Pn + tauP) || (real_gate && xi1 >= Np - tauN);
    double Nmax = fmax(Nn, 1.0);
    outcome list[64];
    int cnt = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int open = 1; open >= 0; --open) {
            if (pass == 0 ? open != open_nom : !(open ? can_open : can_close)) continue;
            if (!open) {
                cnt = push_outcome(list, cnt, 0.0, Nn, 0.0, dNn);
                continue;
            }
            if (t->integer_mode) {
                if (Nn <= 1.0 && dNn <= 0.0) {  /* one trial: the gate decides */
                    cnt = push_outcome(list, cnt, 1.0, Nn - 1.0, 0.0, 0.0);
                    continue;
                }
                double r = old ? floor(G) : floor(G + 0.5);
                double gn = fmin(fmax(r, 1.0), Nn);
                double glo = fmin(fmax(old ? floor(G - tauG) : floor(G - tauG + 0.5), 1.0), Nn);
                double ghi = fmin(fmax(old ? floor(G + tauG) : floor(G + tauG + 0.5), 1.0), Nn);
                int interval = (dNn > 0.0) || (ghi - glo > 2.0);
                /* the kernel rounds (or floors) some G' with |G' - G| <= tauG: its count
                 * lies within tauG + 1/2 of G, so within tauG + 1 of round(G) */
                double eG = interval ? tauG + 1.0 : 0.0;
                cnt = push_outcome(list, cnt, gn, Nn - gn, eG, dNn + eG);
                if (pass == 1 && !interval)
                    for (double g = glo; g <= ghi; g += 1.0) cnt = push_outcome(list, cnt, g, Nn - g, 0.0, 0.0);
            } else {
                double g = fmin(fmax(G, 1.0), Nmax);
                double n = old ? floor(g) : g;
                double en = old ? 1.0 : tauG;
                if (old && floor(g - tauG) == floor(g + tauG)) en = 0.0;
                cnt = push_outcome(list, cnt, n, fmax(Nn - n, 0.0), en, en + dNn);
            }
        }
    }
    if (cnt > 1) t->flagged++;
    for (int i = 0; i < cnt; ++i) {
        N[2 * node] = list[i].n;
        N[2 * node + 1] = list[i].nb;
        dN[2 * node] = list[i].en;
        dN[2 * node + 1] = list[i].eb;
        tree_rec(t, node + 1, N, dN);
    }
}

static void tree_rec(tree_ctx *t, int node, double *N, double *dN)
{
    int K = t->K;
    if (node == K) {
        if (t->n_out >= t->max_cand) { t->overflow = 1; return; }
        for (int k = 0; k < K; ++k) {
            t->out[t->n_out * K + k] = N[K + k];
            t->out_err[t->n_out * K + k] = dN[K + k];
        }
        t->n_out++;
        return;
    }
    double Nn = N[node], dNn = dN[node];
    if (Nn <= 0.0 && dNn <= 0.0) { /* no trials: Alg. 1 gives (0, 0) */
        N[2 * node] = N[2 * node + 1] = 0.0;
        dN[2 * node] = dN[2 * node + 1] = 0.0;
        tree_rec(t, node + 1, N, dN);
        return;
    }
    double xi[2];
    or_node_uniforms(t->key0, t->key1, t->key2, t->seed, node, xi);
    double xi1 = xi[0], xi2 = xi[1];
    double PL = t->P[2 * node], PR = t->P[2 * node + 1];
    double p = (PL + PR > 0.0) ? PL / (PL + PR) : 0.0;
    double e_P = t->tie[0], e_z = t->tie[1], e_f = t->tie[2], d_a = t->tie[3], a_P = t->tie[4];
    int use_tie = (e_P > 0.0 || e_z > 0.0 || e_f > 0.0 || d_a > 0.0 || a_P > 0.0);

    if (t->draw == 1 || t->draw == 2) {
        tree_single(t, node, N, dN, Nn, dNn, PL, PR, p, xi1, xi2, use_tie);
        return;
    }
    double T[4], mu, sigma;
    or_dualgated_thresholds(Nn, p, T, &mu, &sigma);
    double z = or_ndtri(xi2);
    double G = (sigma > 0.0) ? mu + sigma * z : mu;
    double N2 = fmax(2.0, Nn);

    /* tolerance of each threshold and of G: inputs perturbed by the tie model */
    double tau[4] = {0, 0, 0, 0}, tauG = 0.0;
    if (use_tie) {
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            double pp = p;
            if (PL + PR > 0.0) {
                double pl = fmax(PL * (1.0 + sgn * e_P) + sgn * a_P, 0.0);
                double pr = fmax(PR * (1.0 - sgn * e_P) - sgn * a_P, 0.0);
                if (pl + pr > 0.0) pp = pl / (pl + pr);
            }
            for (int sn = -1; sn <= 1; sn += 2) {
                double Np = fmax(Nn + sn * dNn, 0.0);
                double T2[4], mu2, sg2;
                or_dualgated_thresholds(Np, pp, T2, &mu2, &sg2);
                for (int i = 0; i < 4; ++i) tau[i] = fmax(tau[i], fabs(T2[i] - T[i]));
                double G2 = (sg2 > 0.0) ? mu2 + sg2 * z : mu2;
                tauG = fmax(tauG, fabs(G2 - G));
            }
        }
        double a = fmin(fmax(Nn - 1.0, 0.0), 1.0);
        double Pall = T[0], Pallneg = 1.0 - T[2];
        tau[0] += thr_eval_err(Pall, a, e_f) + d_a;
        tau[1] += thr_eval_err(Pall, a, e_f) + (T[1] - T[0]) * e_f + d_a;
        tau[2] += thr_eval_err(Pallneg, a, e_f) + d_a;
        tau[3] += thr_eval_err(Pallneg, a, e_f) + (T[2] - T[3]) * e_f + d_a;
        tauG += sigma * (fabs(z) * e_z + 0x1p-22) + fabs(G) * 0x1p-22 + 0x1p-24;
    }

    outcome list[64];
    int cnt = 0;
    if (t->integer_mode) {
        /* n is decided by the region of xi1 among T0 <= T1 <= T3:
         * [0,T0): N   [T0,T1): 1   [T1,T3): G (only if N > 1)   [T3,1): 0.
         * When the rounding of G cannot be called exactly (more than 3
         * integers within its tolerance, or the trials themselves carry a
         * tolerance), G is kept as one outcome with a count tolerance that the
         * subtree propagates. */
        int nominal = (xi1 < T[0]) ? 0 : (xi1 < T[1]) ? 1 : (xi1 < T[3]) ? 2 : 3;
        if (nominal == 2 && !(Nn > 1.0)) nominal = 3;
        int poss[4] = {0, 0, 0, 0};
        if (T[0] > 0.0 && xi1 < T[0] + tau[0]) poss[0] = 1;
        if (T[1] > T[0] && xi1 >= T[0] - tau[0] && xi1 < T[1] + tau[1]) poss[1] = 1;
        if (Nn > 1.0 && xi1 >= T[1] - tau[1] && xi1 < T[3] + tau[3]) poss[2] = 1;
        if (xi1 >= T[3] - tau[3]) poss[3] = 1;
        double Gn = fmin(fmax(floor(G + 0.5), 1.0), N2 - 1.0);
        double glo = fmin(fmax(floor(G - tauG + 0.5), 1.0), N2 - 1.0);
        double ghi = fmin(fmax(floor(G + tauG + 0.5), 1.0), N2 - 1.0);
        int interval = (dNn > 0.0) || (ghi - glo > 2.0);
        /* the kernel rounds some G' with |G' - G| <= tauG: its count lies
         * within tauG + 1/2 of G, so within tauG + 1 of Gn = round(G) */
        double eG = interval ? tauG + 1.0 : 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int reg = 0; reg < 4; ++reg) {
                if (pass == 0 ? reg != nominal : !poss[reg]) continue;
                if (reg == 2) {
                    cnt = push_outcome(list, cnt, Gn, Nn - Gn, eG, dNn + eG);
                    if (pass == 1 && !interval)
                        for (double g = glo; g <= ghi; g += 1.0) cnt = push_outcome(list, cnt, g, Nn - g, 0.0, 0.0);
                } else {
                    double n = (reg == 0) ? N2 : (reg == 1) ? 1.0 : 0.0;
                    double en = (reg == 0) ? dNn : 0.0;
                    cnt = push_outcome(list, cnt, n, Nn - n, en, dNn - en);
                }
            }
        }
    } else {
        /* Real-valued counts (Alg. 1 as printed): n and nbar from their own
         * masks.  n side: [0,T0): N2  [T0,T1): 1  [T1,1): G or 0;
         * nbar side: [T2,1): N2  [T3,T2): 1  [0,T3): Gbar or 0; the Gaussian
         * is used only when N > 1 and neither one-or-all gate fired. */
        int nom_n = (xi1 < T[0]) ? 0 : (xi1 < T[1]) ? 1 : 2;
        int nom_b = (T[2] <= xi1) ? 0 : (T[3] <= xi1) ? 1 : 2;
        int pn[3] = {0, 0, 0}, pb[3] = {0, 0, 0};
        if (T[0] > 0.0 && xi1 < T[0] + tau[0]) pn[0] = 1;
        if (T[1] > T[0] && xi1 >= T[0] - tau[0] && xi1 < T[1] + tau[1]) pn[1] = 1;
        if (xi1 >= T[1] - tau[1]) pn[2] = 1;
        if (T[2] < 1.0 && xi1 >= T[2] - tau[2]) pb[0] = 1;
        if (T[3] < T[2] && xi1 >= T[3] - tau[3] && xi1 < T[2] + tau[2]) pb[1] = 1;
        if (xi1 < T[3] + tau[3]) pb[2] = 1;
        double Gc = fmin(fmax(G, 1.0), N2 - 1.0);
        for (int pass = 0; pass < 2; ++pass) {
            for (int rn = 0; rn < 3; ++rn) {
                for (int rb = 0; rb < 3; ++rb) {
                    if (pass == 0 ? (rn != nom_n || rb != nom_b) : (!pn[rn] || !pb[rb])) continue;
                    int gauss = (Nn > 1.0) && rn == 2 && rb == 2;
                    double n = (rn == 0) ? N2 : (rn == 1) ? 1.0 : (gauss ? Gc : 0.0);
                    double nb = (rb == 0) ? N2 : (rb == 1) ? 1.0 : (gauss ? N2 - Gc : 0.0);
                    double en = gauss ? tauG : ((rn == 0) ? dNn : 0.0);
                    double eb = gauss ? tauG : ((rb == 0) ? dNn : 0.0);
                    cnt = push_outcome(list, cnt, n, nb, en, eb);
                }
            }
        }
    }
    if (cnt > 1) t->flagged++;
    for (int i = 0; i < cnt; ++i) {
        N[2 * node] = list[i].n;
        N[2 * node + 1] = list[i].nb;
        dN[2 * node] = list[i].en;
        dN[2 * node + 1] = list[i].eb;
        tree_rec(t, node + 1, N, dN);
    }
}

/* Shade npix pixels (Sec. 4, Eq. iblglints:fin; Sec. 3.3 Eq. anisogrid;
 * Alg. 1; Sec. 5 hierarchical multinomial).
 *
 * G-buffer, 16 floats per pixel:
 *   [0..2] w_o, unit vector towards the viewer; [3] N_0, microfacets per unit
 *   uv area (<= 0 marks a background pixel, shaded black);
 *   [4..6] n, unit shading normal; [7] F0 (Schlick);
 *   [8..9] (u, v); [10] alpha_x; [11] alpha_y;
 *   [12] du/dx, [13] dv/dx, [14] du/dy, [15] dv/dy (screen-space derivatives).
 * pref: the R filtered levels concatenated, level r of widths[r] x
 * widths[r]/2 texels x C (C = 3+K: RGB, W_1..W_K), sqrt(alpha) of the levels
 * evenly spaced in [s_min, s_max]; lut: nlut x nlut x 4 (V, U, A, B).
 * L: the K radiance levels.
 *
 * Per pixel:
 *  - smooth radiance L_o = prefRGB(w_r, alpha) (F0 A + B) (Eq. rtibl), with
 *    w_r = 2 (n.w_o) n - w_o, alpha = sqrt(alpha_x alpha_y) (the paper's
 *    method is isotropic), mu_o = clamp(n.w_o, 1e-4, 1) for the tables;
 *  - p_k = V W_k for k >= 2 and p_1 = U + V W_1: Eq. probhk with Eq.
 *    rtiblndf, D^(k) ~ E_D int p_{L_i} w_k; the masked mass 1 - V goes to the
 *    dummy light, merged with k = 1 whose radiance is 0 (Sec. 4);
 *  - N_P and the six grid samples (w_i, vertex, level);
 *  - per sample, the multinomial M(N_i, p) by a balanced binary tree over the
 *    K bins in heap order (Reading of "hierarchical sampling of binomial
 *    distributions"), node probability P_left / (P_left + P_right) (0 if the
 *    node has no mass), left child takes n, right child nbar; integer mode
 *    dithers the root: N_i = floor(N_P) + chi(xi0 < N_P - floor(N_P)) with
 *    xi0 from the root's hash; real mode uses N_i = N_P;
 *  - M_k = sum_i w_i n_k(i), L^_o = L_o sum_k L_k M_k / (N_P sum_k L_k p_k)
 *    (0 when the denominator is 0).
 *
 * evaluator = 2 takes p_k from pk_in (npix x K) as given; evaluator = 3
 * takes them from the anisotropic multi-tap E1 (or_e1a_weights; tangents
 * needed).
 * draw selects the binomial approximation at the tree nodes: 0 dual-gated
 * (Alg. 1), 1 single-gated (Eq. gated), 2 Eq. oldgated, 3 the Wang 2020
 * comparison of Sec. 7 (one single-gated count per sample with probability
 * gamma, independent of the map; counts (glints, rest) in bins 1 and 2;
 * L^_o = L_o M_1 / (N_P gamma)).
 * grid = 1 spreads N_P over the anisotropic grid (footprint_cell: 4 cell
 * vertices x 3 lattice vertices = 12 samples per pixel; the per-sample arrays
 * then hold 12 entries per pixel and vert's third entry is the packed
 * (level, anisotropy, orientation) key); grid_flags (optional) marks pixels
 * whose cell decisions are too close to call.
 * evaluator = 1 replaces p_k by the E2 quadrature (or_e2_pk) of the
 * anisotropic footprint, with per-pixel tangents (npix x 4) and the pyramid
 * (mips, W x H level 0); e2_flags counts its near-boundary points.
 *
 * Outputs (all per pixel): rgb (3, nominal outcome at every decision),
 * lo (3), pk (K), np (1, FP32 N_P), vert (6 x 3: x, y, level), wv (6),
 * nroot (6), ncand (6: number of valid count vectors of each tree, -1 when
 * the enumeration overflowed), cand (6 x max_cand x K), cand_err (same
 * shape, tolerance of each count in real mode), flags (decisions that were
 * too close to call).  Returns the number of background pixels. */
long or_shade(const float *gb, long npix, const double *pref, int R, const int *widths, int C, double s_min,
              double s_max, const double *lut, int nlut, const double *L, int K, uint32_t seed, int integer_mode,
              const double *tie, int max_cand, double *rgb, double *lo, double *pk, float *np, int64_t *vert,
              double *wv, double *nroot, int32_t *ncand, double *cand, double *cand_err, int32_t *flags,
              int evaluator, const float *tangents, int e2_S, const double *mips, int W, int H, int32_t *e2_flags,
              const double *pk_in, int draw, double gamma, int grid, int32_t *grid_flags)
{
    const int nv = grid ? 12 : OR_NV; /* grid samples per pixel */
    float ocs[8], osn[8];
    orient_table(ocs, osn);
    long nbg = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : nbg)
    for (long q = 0; q < npix; ++q) {
        const float *g = gb + 16 * q;
        for (int c = 0; c < 3; ++c) rgb[3 * q + c] = lo[3 * q + c] = 0.0;
        for (int k = 0; k < K; ++k) pk[q * K + k] = 0.0;
        np[q] = 0.0f;
        flags[q] = 0;
        if (grid_flags) grid_flags[q] = 0;
        for (int v = 0; v < nv; ++v) {
            wv[q * nv + v] = 0.0;
            nroot[q * nv + v] = 0.0;
            ncand[q * nv + v] = 0;
            for (int k = 0; k < 3; ++k) vert[(q * nv + v) * 3 + k] = 0;
        }
        if (!(g[3] > 0.0f)) { ++nbg; continue; }

        /* smooth radiance and reflection probabilities (E1) */
        double wo[3] = {g[0], g[1], g[2]}, nn[3] = {g[4], g[5], g[6]};
        double F0 = g[7];
        double mu_o = nn[0] * wo[0] + nn[1] * wo[1] + nn[2] * wo[2];
        double wr[3];
        for (int k = 0; k < 3; ++k) wr[k] = 2.0 * mu_o * nn[k] - wo[k];
        double mu_c = fmin(fmax(mu_o, 1e-4), 1.0);
        double alpha = sqrt((double)g[10] * (double)g[11]);
        double s = sqrt(alpha);
        double tab[4];
        lut_fetch(lut, nlut, mu_c, s, tab);
        double V = tab[0], U = tab[1], A = tab[2], B = tab[3];
        double tl = (R > 1) ? (s - s_min) / (s_max - s_min) * (R - 1) : 0.0;
        tl = fmin(fmax(tl, 0.0), (double)(R - 1));
        int r0 = (int)floor(tl);
        int r1 = r0 + 1 < R ? r0 + 1 : R - 1;
        double ft = tl - r0;
        double c0[3 + OR_MAXK], c1[3 + OR_MAXK], cc[3 + OR_MAXK];
        size_t off0 = 0, off1 = 0;
        for (int r = 0; r < r0; ++r) off0 += (size_t)widths[r] * (widths[r] / 2) * C;
        for (int r = 0; r < r1; ++r) off1 += (size_t)widths[r] * (widths[r] / 2) * C;
        env_bilinear(pref + off0, widths[r0], widths[r0] / 2, C, wr, c0);
        env_bilinear(pref + off1, widths[r1], widths[r1] / 2, C, wr, c1);
        for (int c = 0; c < C; ++c) cc[c] = (1.0 - ft) * c0[c] + ft * c1[c];
        double Eb = F0 * A + B;
        double Lo[3] = {cc[0] * Eb, cc[1] * Eb, cc[2] * Eb};
        double p[OR_MAXK];
        p[0] = U + V * cc[3];
        for (int k = 1; k < K; ++k) p[k] = V * cc[3 + k];
        if (evaluator == 1) {
            double tg[3] = {tangents[4 * q], tangents[4 * q + 1], tangents[4 * q + 2]};
            e2_flags[q] = or_e2_pk(wo, nn, tg, g[10], g[11], e2_S, mips, W, H, C, K, p);
        } else if (e2_flags) {
            e2_flags[q] = 0;
        }
        if (evaluator == 2)
            for (int k = 0; k < K; ++k) p[k] = pk_in[q * K + k];
        if (evaluator == 3) {
            double tg[3] = {tangents[4 * q], tangents[4 * q + 1], tangents[4 * q + 2]};
            double Wa[OR_MAXK];
            or_e1a_weights(wo, nn, tg, g[10], g[11], pref, R, widths, C, s_min, s_max, Wa);
            p[0] = U + V * Wa[0];
            for (int k = 1; k < K; ++k) p[k] = V * Wa[k];
        }
        for (int c = 0; c < 3; ++c) lo[3 * q + c] = Lo[c];
        for (int k = 0; k < K; ++k) pk[q * K + k] = p[k];

        /* footprint and microfacet count (FP32) */
        /* Reading: counts are uint32, so N_P saturates at the largest FP32 value
         * below 2^32; the radiance uses the same saturated N_P. */
        float area = f32_footprint_area(g[12], g[13], g[14], g[15]);
        float NP = fminf(g[3] * area, 4294967040.0f);
        np[q] = NP;
        if (!(area > 0.0f) || !(NP > 0.0f)) continue;

        /* grid samples */
        int l0;
        double fl;
        grid_level(area, &l0, &fl);
        tree_ctx t;
        memset(&t, 0, sizeof(t));
        t.K = K;
        t.integer_mode = integer_mode;
        t.seed = seed;
        for (int i = 0; i < 5; ++i) t.tie[i] = tie[i];
        t.max_cand = max_cand;
        t.draw = (draw == 3) ? 1 : draw;
        for (int k = 0; k < K; ++k) t.P[K + k] = p[k];
        for (int nd = K - 1; nd >= 1; --nd) t.P[nd] = t.P[2 * nd] + t.P[2 * nd + 1];
        /* Wang 2020: a two-bin tree (glints gamma, rest 1 - gamma) at every sample */
        double wang_buf[64 * 2], wang_err[64 * 2];
        int K_tree = K;
        if (draw == 3) {
            K_tree = 2;
            t.K = 2;
            t.P[2] = gamma;
            t.P[3] = 1.0 - gamma;
            t.P[1] = 1.0;
        }

        double Mk[OR_MAXK];
        for (int k = 0; k < K; ++k) Mk[k] = 0.0;
        int cl4[4], ta[4], to[4];
        double tw[4];
        if (grid) {
            int fl_flag = footprint_cell(g, area, l0, fl, cl4, ta, to, tw);
            if (grid_flags) grid_flags[q] = fl_flag;
        }
        for (int lv = 0; lv < (grid ? 4 : 2); ++lv) {
            int l;
            double lw;
            int64_t vx[3], vy[3];
            double b[3];
            uint32_t key2;
            if (grid) { /* the uv lattice stretched by 2^a along the orientation o pi/8 */
                l = cl4[lv];
                lw = tw[lv];
                int an = ta[lv], o = to[lv];
                float up = ocs[o] * g[8] + osn[o] * g[9];
                float vp = ocs[o] * g[9] - osn[o] * g[8];
                lattice_vertices(ldexpf(up, -(l + an)), ldexpf(vp, -(l - an)), vx, vy, b);
                key2 = (((uint32_t)l) & 0x3FFu) | ((uint32_t)an << 10) | ((uint32_t)o << 12) | 0x8000u;
            } else {
                l = l0 + lv;
                lw = lv ? fl : 1.0 - fl;
                grid_vertices(g[8], g[9], l, vx, vy, b);
                key2 = ((uint32_t)l) & 0xFFFFu;
            }
            for (int c = 0; c < 3; ++c) {
                int v = lv * 3 + c;
                double w = lw * b[c];
                wv[q * nv + v] = w;
                vert[(q * nv + v) * 3 + 0] = vx[c];
                vert[(q * nv + v) * 3 + 1] = vy[c];
                vert[(q * nv + v) * 3 + 2] = grid ? (int64_t)key2 : l;
                t.key0 = (uint32_t)vx[c];
                t.key1 = (uint32_t)vy[c];
                t.key2 = key2;
                double N[2 * OR_MAXK], dN[2 * OR_MAXK];
                for (int i = 0; i < 2 * OR_MAXK; ++i) N[i] = dN[i] = 0.0;
                if (integer_mode) {
                    uint32_t in[4] = {t.key0, t.key1, t.key2 | (1u << 16), seed}, h[4];
                    or_pcg4d(in, h);
                    float xi0 = (float)or_xi(h[0]);
                    float fN = floorf(NP);
                    float frac = NP - fN;
                    N[1] = (double)fN + (xi0 < frac ? 1.0 : 0.0);
                } else {
                    N[1] = (double)NP;
                }
                nroot[q * nv + v] = N[1];
                double *co = cand + ((size_t)q * nv + v) * max_cand * K;
                double *ce = cand_err + ((size_t)q * nv + v) * max_cand * K;
                t.out = (K_tree == K) ? co : wang_buf;
                t.out_err = (K_tree == K) ? ce : wang_err;
                t.max_cand = (K_tree == K) ? max_cand : (max_cand < 64 ? max_cand : 64);
                t.n_out = 0;
                t.overflow = 0;
                tree_rec(&t, 1, N, dN);
                if (K_tree != K) /* two-bin outcomes into the first two of K bins */
                    for (int i = 0; i < t.n_out; ++i)
                        for (int k = 0; k < K; ++k) {
                            co[i * K + k] = k < 2 ? wang_buf[i * 2 + k] : 0.0;
                            ce[i * K + k] = k < 2 ? wang_err[i * 2 + k] : 0.0;
                        }
                ncand[q * nv + v] = t.overflow ? -1 : t.n_out;
                for (int k = 0; k < K; ++k) Mk[k] += w * co[k]; /* first = nominal outcome */
            }
        }
        flags[q] = t.flagged;
        double num = 0.0, den = 0.0;
        for (int k = 1; k < K; ++k) {
            num += L[k] * Mk[k];
            den += L[k] * p[k];
        }
        den *= (double)NP;
        if (draw == 3) {
            num = Mk[0];
            den = (double)NP * gamma;
        }
        if (den > 0.0)
            for (int c = 0; c < 3; ++c) rgb[3 * q + c] = Lo[c] * num / den;
    }
    return nbg;
}

/* Radiance of one pixel for a chosen valid count vector per grid sample
 * (Eq. iblglints:fin): L^_o = L_o sum_k L_k M_k / (N_P sum_k L_k p_k),
 * M_k = sum_i w_i n_k(i). counts: 6 x K. */
void or_radiance(const double *lo3, const double *pk, double np, const double *L, int K, const double *wv,
                 const double *counts, double *rgb, int draw, double gamma, int nv)
{
    double num = 0.0, den = 0.0;
    for (int k = 1; k < K; ++k) {
        double M = 0.0;
        for (int v = 0; v < nv; ++v) M += wv[v] * counts[v * K + k];
        num += L[k] * M;
        den += L[k] * pk[k];
    }
    den *= np;
    if (draw == 3) { /* Wang 2020: L_o M_1 / (N_P gamma) */
        num = 0.0;
        for (int v = 0; v < nv; ++v) num += wv[v] * counts[v * K];
        den = np * gamma;
    }
    for (int c = 0; c < 3; ++c) rgb[c] = den > 0.0 ? lo3[c] * num / den : 0.0;
}

/* One hierarchical multinomial draw with explicit uniforms, for statistical
 * tests of the tree: K bins with probabilities p, N trials at the root, key
 * and seed as in or_shade, draw as in or_shade's tree (0 dual-gated, 1 Eq.
 * gated, 2 Eq. oldgated); counts: K leaf counts (nominal outcome). */
void or_multinomial(const double *p, int K, double N, uint32_t key0, uint32_t key1, uint32_t key2, uint32_t seed,
                    int integer_mode, double *counts, int draw)
{
    tree_ctx t;
    memset(&t, 0, sizeof(t));
    t.draw = draw;
    double buf[OR_MAXK], ebuf[OR_MAXK];
    t.K = K;
    t.integer_mode = integer_mode;
    t.key0 = key0; t.key1 = key1; t.key2 = key2; t.seed = seed;
    t.max_cand = 1;
    t.out = buf;
    t.out_err = ebuf;
    for (int k = 0; k < K; ++k) t.P[K + k] = p[k];
    for (int nd = K - 1; nd >= 1; --nd) t.P[nd] = t.P[2 * nd] + t.P[2 * nd + 1];
    double Nv[2 * OR_MAXK], dN[2 * OR_MAXK];
    for (int i = 0; i < 2 * OR_MAXK; ++i) Nv[i] = dN[i] = 0.0;
    Nv[1] = N;
    tree_rec(&t, 1, Nv, dN);
    for (int k = 0; k < K; ++k) counts[k] = buf[k];
}

/* Threads of the per-pixel and per-texel loops (OpenMP; 1 when the oracle
 * was built without it).  The loops' iterations are independent, so results
 * do not depend on the thread count. */
void or_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
