// Per-pixel glint shading shared by the shading, serving and variant kernels
// (Sec. 4 Eq. iblglints:fin; Sec. 3.3 Eq. anisogrid; Sec. 5 Alg. 1, the
// single-gated forms Eq. gated / Eq. oldgated, and the hierarchical
// multinomial).  See glint_shade.cu for the per-pixel steps.
#pragma once
#include "glint_internal.cuh"
#include "glint_probs.cuh"
#include "glint_quantile.cuh"

namespace {

using namespace glint;

constexpr int kShadeNT = 128;

// |du/dx dv/dy - du/dy dv/dx| with one FMA correction (Kahan), every
// operation correctly rounded and never contracted.
__device__ __forceinline__ float footprint_area(float dudx, float dvdx, float dudy, float dvdy) {
    const float w = __fmul_rn(dudy, dvdx);
    const float e = __fmaf_rn(-dudy, dvdx, w);
    const float f = __fmaf_rn(dudx, dvdy, -w);
    return fabsf(__fadd_rn(f, e));
}

// Low 32 bits of the two's-complement integer held by an integral float.  For
// |f| >= 2^31 the value is mant 2^e with e >= 8; shifting the 24-bit mantissa
// gives the low word without a 64-bit conversion (which would use the FP64 pipe).
__device__ __forceinline__ uint32_t low32_of_integral(float f) {
    if (fabsf(f) < 2147483648.f) return (uint32_t)__float2int_rz(f);
    const uint32_t b = __float_as_uint(f);
    const int e = (int)((b >> 23) & 0xffu) - 150;
    const uint32_t mant = (b & 0x7fffffu) | 0x800000u;
    const uint32_t v = (e >= 32) ? 0u : (mant << e);
    return (b >> 31) ? (0u - v) : v;
}

// Hardware 2^x (MUFU.EX2, ftz): relative error below 2^-22 (PTX ISA, ex2.approx);
// the gate probabilities it produces are compared with uniforms >= 2^-24, so
// flushing subnormal results to 0 changes no decision.
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Hardware square root (sqrt.approx, relative error ~2^-23) for the Gaussian's
// standard deviation.
__device__ __forceinline__ float fast_sqrt(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct NodeParams {
    float p, q, lp, lq;  // node probability, complement, log2 p, log2 of (1 - c p)^(1/c)
};

// Dual-gated Gaussian (Alg. 1) for an integer number of trials N; returns n
// (nbar = N - n), 0 when N = 0.  Regions of xi1 (same as the printed masks):
// [0, P_{n=N}) -> N;  [P_{n=N}, P_{n=N} + P_{n=1}) -> 1;
// 1 - xi1 <= P_{nbar=N} + P_{nbar=1} -> 0;  otherwise the clamped, rounded
// Gaussian when N > 1, else 0.  For N >= 2 the single-trial terms vanish, so
// P_{n=N} = p^N and P_{nbar=N} = (1 - c p)^(N/c); for N = 1 the draw is one
// Bernoulli trial with probability p.  Evaluated without branches (the
// Gaussian is computed for every lane and the gates select), so that a warp
// whose lanes take different regions does not run the paths one after
// another.  The Gaussian N(mu, sigma^2), mu = 1 + (N - 2) p, is rounded half
// up as floor(sigma z + (mu + 1/2)).
__device__ __forceinline__ uint32_t draw_integer(uint32_t N, const NodeParams &np, uint32_t h1, uint32_t h2) {
    const float xi1 = hash_uniform(h1);
    const float xi1c = hash_uniform_complement(h1);
    const float Nf = __uint2float_rn(N);
    const float m = fmaxf(Nf - 2.f, 0.f);  // N - 2 trials left to the Gaussian (0 below N = 2)
    const float N2 = m + 2.f;
    const bool many = N >= 2u;
    const float Pall = many ? fast_exp2(N2 * np.lp) : 0.f;
    const float T1 = many ? Pall : ((N == 1u) ? np.p : 0.f);
    const float Sneg = fast_exp2(N2 * np.lq);  // decides only for N >= 2
    const float muh = fmaf(m, np.p, 1.5f);
    const float sigma = fast_sqrt(m * np.p * np.q);
    const float z = normal_quantile(hash_uniform(h2));
    const float G = fminf(fmaxf(floorf(fmaf(sigma, z, muh)), 1.f), kMaxCount);
    uint32_t r = min((uint32_t)G, N - 1u);
    r = (xi1c <= Sneg || !many) ? 0u : r;
    r = (xi1 < T1) ? 1u : r;
    return (xi1 < Pall) ? N : r;
}

// Dual-gated Gaussian (Alg. 1) with real-valued N and counts.
__device__ __forceinline__ void draw_real(float N, const NodeParams &np, uint32_t h1, uint32_t h2, float &n,
                                          float &nbar) {
    const float xi1 = hash_uniform(h1);
    const float xi1c = hash_uniform_complement(h1);
    const float N2 = fmaxf(2.f, N);
    const float a = fminf(fmaxf(N - 1.f, 0.f), 1.f);
    const float b = fmaxf(0.f, 1.f - fabsf(1.f - N));
    const float Pall = a * fast_exp2(N2 * np.lp);
    const float Pallneg = a * fast_exp2(N2 * np.lq);
    const float Pone = b * np.p, Poneneg = b * np.q;
    const bool B_all = xi1 < Pall;
    const bool B_allone = xi1 < Pall + Pone;
    const bool B_allneg = xi1c <= Pallneg;
    const bool B_alloneneg = xi1c <= Pallneg + Poneneg;
    const bool B_G = (N > 1.f) && !B_allone && !B_alloneneg;
    float G = 0.f;
    if (B_G) {
        const float mu = 1.f + (N2 - 2.f) * np.p;
        const float sigma = fast_sqrt(fmaxf((N2 - 2.f) * np.p * np.q, 0.f));
        const float z = normal_quantile(hash_uniform(h2));
        G = fminf(fmaxf(fmaf(sigma, z, mu), 1.f), N2 - 1.f);
    }
    n = (B_all ? N2 - 1.f : 0.f) + (B_allone ? 1.f : 0.f) + G;
    nbar = (B_allneg ? N2 - 1.f : 0.f) + (B_alloneneg ? 1.f : 0.f) + (B_G ? N2 - G : 0.f);
}


// log2(1 - x) for x in [0, 1/2] with a small relative error for every x
// (1 - x itself would lose the low bits of small x): with s = x / (2 - x) in
// [0, 1/3], ln(1 - x) = -2 atanh(s) = -2 (s + s^3/3 + s^5/5 + ...); the series
// to s^13 leaves a relative error below 3e-8, the hardware reciprocal in s
// about 2.4e-7.
__device__ __forceinline__ float log2_one_minus(float x) {
    constexpr float kTwoLog2e = 2.88539008177792681472f;
    const float s = __fdividef(x, 2.f - x);
    const float u = s * s;
    float t = 1.f / 13.f;
    t = fmaf(t, u, 1.f / 11.f);
    t = fmaf(t, u, 1.f / 9.f);
    t = fmaf(t, u, 1.f / 7.f);
    t = fmaf(t, u, 1.f / 5.f);
    t = fmaf(t, u, 1.f / 3.f);
    t = fmaf(t, u, 1.f);
    return -kTwoLog2e * (s * t);
}

// Node parameters of a binary split with probabilities p (left) and q = 1 - p
// (right): log2 p and log2 of the small-p biased complement, each logarithm
// taken of whichever of p, q is the smaller (1 - x near 1 is not accurate):
// log2 of the smaller one by the hardware lg2 (absolute error ~2^-22 on a
// value of magnitude >= 1), log2 of the larger one by log2_one_minus of the
// smaller.
// Both logarithms are evaluated once, of the smaller probability, and
// assigned by a select, so lanes on either side of 1/2 take the same path.
__device__ __forceinline__ NodeParams node_params(float pn, float qn) {
    NodeParams nd;
    nd.p = pn;
    nd.q = qn;
    const bool left_small = pn <= 0.5f;
    const float small = left_small ? pn : qn;
    const float l_small = __log2f(small), l_large = log2_one_minus(small);
    const float l2p = left_small ? l_small : l_large;
    const float l2q = left_small ? l_large : l_small;
    nd.lp = l2p;
    nd.lq = (pn >= kEps) ? l2q : (pn * (1.f / kEps)) * kLog2OneMinusEps;
    return nd;
}

// Single-gated Gaussian for an integer number of trials N >= 1 (Sec. 5,
// Eq. gated; with OLD, Eq. oldgated's floor instead of rounding): the gate
// opens (at least one positive trial) with probability 1 - (1 - c p)^(N/c),
// decided on the complement uniform as 1 - xi1 > (1 - c p)^(N/c); an open gate
// gives the Gaussian with one known positive trial, clamped to [1, N].
__device__ __forceinline__ uint32_t draw_single_integer(uint32_t N, const NodeParams &np, uint32_t h1, uint32_t h2,
                                                        bool old) {
    const float xi1c = hash_uniform_complement(h1);
    const float Nf = __uint2float_rn(N);
    const float Pnone = fast_exp2(Nf * np.lq);
    if (!(xi1c > Pnone)) return 0u;
    if (N == 1u) return 1u;
    const float mu = 1.f + (Nf - 1.f) * np.p;
    const float sigma = fast_sqrt((Nf - 1.f) * np.p * np.q);
    const float z = normal_quantile(hash_uniform(h2));
    const float g = fmaf(sigma, z, mu);
    float G = old ? floorf(g) : floorf(g + 0.5f);
    G = fminf(fmaxf(G, 1.f), Nf);
    return min((uint32_t)G, N);
}

// Single-gated Gaussian with real-valued N and counts (Eq. gated: gate
// min(N p, 1 - (1 - c p)^(N/c)), Gaussian clamped to [1, max(N, 1)]; with OLD,
// Eq. oldgated: gate 1 - (1 - c p)^(N/c) and the floor); nbar = max(N - n, 0).
__device__ __forceinline__ void draw_single_real(float N, const NodeParams &np, uint32_t h1, uint32_t h2, bool old,
                                                 float &n, float &nbar) {
    const float xi1 = hash_uniform(h1);
    const float xi1c = hash_uniform_complement(h1);
    const float Pnone = fast_exp2(N * np.lq);
    const bool open = (xi1c > Pnone) && (old || xi1 < N * np.p);
    n = 0.f;
    if (open) {
        const float mu = 1.f + (N - 1.f) * np.p;
        const float sigma = fast_sqrt(fmaxf((N - 1.f) * np.p * np.q, 0.f));
        const float z = normal_quantile(hash_uniform(h2));
        const float g = fminf(fmaxf(fmaf(sigma, z, mu), 1.f), fmaxf(N, 1.f));
        n = old ? floorf(g) : g;
    }
    nbar = fmaxf(N - n, 0.f);
}

// Orientations of the anisotropic grid: phi_o = o pi / 8, o = 0 .. 7, as FP32
// values of cos and sin (cos(pi/8), sin(pi/8), sqrt(2)/2 rounded to nearest).
__device__ __constant__ float kOrientCos[8] = {1.f, 0x1.d906bcp-1f, 0x1.6a09e6p-1f, 0x1.87de2ap-2f,
                                               0.f, -0x1.87de2ap-2f, -0x1.6a09e6p-1f, -0x1.d906bcp-1f};
__device__ __constant__ float kOrientSin[8] = {0.f, 0x1.87de2ap-2f, 0x1.6a09e6p-1f, 0x1.d906bcp-1f,
                                               1.f, 0x1.d906bcp-1f, 0x1.6a09e6p-1f, 0x1.87de2ap-2f};

// The anisotropic grid's footprint cell (Sec. 3.3, after the anisotropic
// grids the paper builds on): the footprint ellipse of the uv Jacobian has
// eigenvalues lam1 >= lam2 of J J^T; its coordinates are the level
// L = l0 + fl = log2 sqrt|P| (as the isotropic grid), the anisotropy
// A = log2(sqrt(lam1/lam2)) / 2 = (log2 lam1 - log2 |P|) / 2 clamped to [0, 2]
// (a lattice stretched by 2^a along the major axis and shrunk by 2^a across
// it), and the orientation O = theta / (pi/8) in [0, 8), theta = atan2(2b,
// a - c) / 2 the major axis' angle, periodic.  N_P is spread over the four
// vertices of the cell's Freudenthal tetrahedron: fractions sorted in
// decreasing order (ties: L, then A, then O) give the path of unit steps and
// the weights 1 - f1, f1 - f2, f2 - f3, f3.  Vertices with a = 0 use o = 0
// (an unstretched lattice has no orientation).
__device__ __forceinline__ void footprint_cell(float4 g3, float area, int l0, float fl, int *tl, int *ta, int *to,
                                               float *tw) {
    const float ea = g3.x * g3.x + g3.z * g3.z, ec = g3.y * g3.y + g3.w * g3.w;
    const float eb = g3.x * g3.y + g3.z * g3.w;
    const float hd = 0.5f * (ea - ec);
    const float lam1 = 0.5f * (ea + ec) + sqrtf(hd * hd + eb * eb);
    float A = 0.5f * (log2f(lam1) - log2f(area));
    A = fminf(fmaxf(A, 0.f), 2.f);
    float O = atan2f(eb, hd) * 1.27323954473516268615f;  // 4 / pi
    if (O < 0.f) O += 8.f;
    if (O >= 8.f) O -= 8.f;
    const int a0 = (A >= 2.f) ? 2 : (int)floorf(A);
    const float fa = A - (float)a0;
    const int o0 = min((int)floorf(O), 7);
    const float fo = O - (float)o0;
    // order of the unit steps: by decreasing fraction, ties in the order L, A, O
    const float f[3] = {fl, fa, fo};
    int ord[3] = {0, 1, 2};
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2 - i; ++j)
            if (f[ord[j + 1]] > f[ord[j]]) { const int t = ord[j]; ord[j] = ord[j + 1]; ord[j + 1] = t; }
    int cl = l0, ca = a0, co = o0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        if (v > 0) {
            const int ax = ord[v - 1];
            if (ax == 0) ++cl; else if (ax == 1) ++ca; else co = (co + 1) & 7;
        }
        tl[v] = cl;
        ta[v] = ca;
        to[v] = (ca == 0) ? 0 : co;
        const float hi = (v == 0) ? 1.f : f[ord[v - 1]];
        const float lo = (v == 3) ? 0.f : f[ord[v]];
        tw[v] = hi - lo;
    }
}

template <int K, bool INTEGER, bool DEBUG, int DRAW, int GRID>
__device__ __forceinline__ void shade_draws(const ShadeArgs &a, long q, const float4 &g0, const float4 &g2,
                                            const float4 &g3, float Lor, float Log, float Lob, const float *p);

// Steps 1-5 for pixel q of the frame described by a.  DRAW selects the binomial
// approximation at the tree nodes: dual-gated (the paper's), single-gated
// (Eq. gated), the older single-gated form (Eq. oldgated), or the Wang 2020
// comparison (a single-gated glint count with the environment-independent
// probability gamma, radiance L_o M / (N_P gamma); Sec. 7).
template <int K, bool INTEGER, bool DEBUG, int EV, int DRAW = kDrawDual, int GRID = 0>
__device__ __forceinline__ void shade_pixel(const ShadeArgs &a, long q) {
    constexpr int NS = GRID ? 12 : 6;  // grid samples per pixel
    const float4 g0 = ldg4(a.view_n0 + q);
    const float4 g1 = ldg4(a.normal_f0 + q);
    const float4 g2 = ldg4(a.uv_alpha + q);
    const float4 g3 = ldg4(a.duv + q);

    if (!(g0.w > 0.f)) {  // background
        a.out[q] = make_float4(0.f, 0.f, 0.f, 1.f);
        if (DEBUG) {
            if (a.dbg.np) a.dbg.np[q] = 0.f;
            if (a.dbg.p) for (int k = 0; k < K; ++k) a.dbg.p[q * K + k] = 0.f;
            if (a.dbg.lo) for (int c = 0; c < 3; ++c) a.dbg.lo[q * 3 + c] = 0.f;
            for (int v = 0; v < NS; ++v) {
                if (a.dbg.w) a.dbg.w[q * NS + v] = 0.f;
                if (a.dbg.nroot) a.dbg.nroot[q * NS + v] = 0.f;
                if (a.dbg.vert) for (int c = 0; c < 3; ++c) a.dbg.vert[(q * NS + v) * 3 + c] = 0;
                if (a.dbg.counts) for (int k = 0; k < K; ++k) a.dbg.counts[(q * NS + v) * K + k] = 0.f;
            }
        }
        return;
    }

    // ---- 1. smooth radiance and reflection probabilities
    float Lor, Log, Lob;
    float p[K];
    smooth_and_probs<K, EV>(a, q, g0, g1, g2, Lor, Log, Lob, p);
    shade_draws<K, INTEGER, DEBUG, DRAW, GRID>(a, q, g0, g2, g3, Lor, Log, Lob, p);
}

// Steps 2-5 for foreground pixel q given its smooth radiance (Lor, Log, Lob)
// and reflection probabilities p.
template <int K, bool INTEGER, bool DEBUG, int DRAW, int GRID>
__device__ __forceinline__ void shade_draws(const ShadeArgs &a, long q, const float4 &g0, const float4 &g2,
                                            const float4 &g3, float Lor, float Log, float Lob, const float *p) {
    constexpr int NS = GRID ? 12 : 6;  // grid samples per pixel

    // ---- 2. footprint, microfacet count, grid level
    const float area = footprint_area(g3.x, g3.y, g3.z, g3.w);
    const float NP = fminf(__fmul_rn(g0.w, area), kMaxCount);
    float den = 0.f;
#pragma unroll
    for (int k = 1; k < K; ++k) den = fmaf(__ldg(a.levels + k), p[k], den);
    den *= NP;

    if (DEBUG) {
        if (a.dbg.np) a.dbg.np[q] = NP;
        if (a.dbg.p) for (int k = 0; k < K; ++k) a.dbg.p[q * K + k] = p[k];
        if (a.dbg.lo) { a.dbg.lo[q * 3] = Lor; a.dbg.lo[q * 3 + 1] = Log; a.dbg.lo[q * 3 + 2] = Lob; }
    }
    if (!(area > 0.f) || !(NP > 0.f)) {
        a.out[q] = make_float4(0.f, 0.f, 0.f, 1.f);
        if (DEBUG) {
            for (int v = 0; v < NS; ++v) {
                if (a.dbg.w) a.dbg.w[q * NS + v] = 0.f;
                if (a.dbg.nroot) a.dbg.nroot[q * NS + v] = 0.f;
                if (a.dbg.vert) for (int c = 0; c < 3; ++c) a.dbg.vert[(q * NS + v) * 3 + c] = 0;
                if (a.dbg.counts) for (int k = 0; k < K; ++k) a.dbg.counts[(q * NS + v) * K + k] = 0.f;
            }
        }
        return;
    }
    int e2;
    const float mant = frexpf(area, &e2);  // area = mant 2^e2, mant in [1/2, 1)
    const int ep = e2 - 1;
    int l0 = (ep >= 0) ? ep / 2 : -((-ep + 1) / 2);
    float fl = 0.5f * ((float)(ep - 2 * l0) + log2f(2.f * mant));
    if (l0 < -24) { l0 = -24; fl = 0.f; }
    if (l0 > 23) { l0 = 23; fl = 1.f; }

    // ---- 3. node parameters of the balanced binary tree (heap order)
    float P[2 * K];
#pragma unroll
    for (int k = 0; k < K; ++k) P[K + k] = p[k];
#pragma unroll
    for (int n = K - 1; n >= 1; --n) P[n] = P[2 * n] + P[2 * n + 1];
    NodeParams nd[K];
    if (DRAW == kDrawWang) {
        nd[1] = node_params(a.gamma, 1.f - a.gamma);
    } else {
#pragma unroll
        for (int n = 1; n < K; ++n) {
            const float tot = P[n];
            const float inv = __fdividef(1.f, tot);  // hardware reciprocal, within 2 ulp
            const bool some = tot > 0.f;              // an empty subtree gets p = 0, q = 1
            nd[n] = node_params(some ? P[2 * n] * inv : 0.f, some ? P[2 * n + 1] * inv : 1.f);
        }
    }

    // ---- 4. six grid samples x (K-1) draws
    float M[K];
#pragma unroll
    for (int k = 0; k < K; ++k) M[k] = 0.f;
    const float F2 = 0x1.76cf5ep-2f;  // (sqrt(3) - 1) / 2
    const float fN = floorf(NP);
    const float fracN = NP - fN;
    // anisotropic grid: the footprint's cell in (level, anisotropy, orientation)
    int tv_l[4], tv_a[4], tv_o[4];
    float tv_w[4];
    if (GRID) footprint_cell(g3, area, l0, fl, tv_l, tv_a, tv_o, tv_w);
#pragma unroll 1
    for (int lv = 0; lv < (GRID ? 4 : 2); ++lv) {
        int l;
        float lw, x, y;
        uint32_t key2;
        if (GRID) {  // the uv lattice stretched along the vertex's orientation
            l = tv_l[lv];
            lw = tv_w[lv];
            const int an = tv_a[lv], o = tv_o[lv];
            const float cs = kOrientCos[o], sn = kOrientSin[o];
            const float up = __fadd_rn(__fmul_rn(cs, g2.x), __fmul_rn(sn, g2.y));
            const float vp = __fsub_rn(__fmul_rn(cs, g2.y), __fmul_rn(sn, g2.x));
            x = ldexpf(up, -(l + an));
            y = ldexpf(vp, -(l - an));
            key2 = (((uint32_t)l) & 0x3FFu) | ((uint32_t)an << 10) | ((uint32_t)o << 12) | 0x8000u;
        } else {
            l = l0 + lv;
            lw = lv ? fl : 1.f - fl;
            x = ldexpf(g2.x, -l);
            y = ldexpf(g2.y, -l);
            key2 = ((uint32_t)l) & 0xFFFFu;
        }
        const float sk = __fmul_rn(__fadd_rn(x, y), F2);
        const float xs = __fadd_rn(x, sk), ys = __fadd_rn(y, sk);
        const float fi = floorf(xs), fj = floorf(ys);
        const float fx = __fsub_rn(xs, fi), fy = __fsub_rn(ys, fj);
        const uint32_t ii = low32_of_integral(fi), jj = low32_of_integral(fj);
        const bool tri = fx > fy;
        const float bmax = tri ? fx : fy, bmin = tri ? fy : fx;
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            const uint32_t vx = ii + ((c == 2 || (c == 1 && tri)) ? 1u : 0u);
            const uint32_t vy = jj + ((c == 2 || (c == 1 && !tri)) ? 1u : 0u);
            const float bc = (c == 0) ? 1.f - bmax : (c == 1) ? bmax - bmin : bmin;
            const float w = lw * bc;
            // the vertex's uniforms: hash call 1 gives the root's dither (word 0)
            // and node 1's pair (words 1, 2); siblings 2m, 2m+1 share call m + 1
            // (words 0, 1 and 2, 3), made once either of them has trials
            uint4 h = pcg4d(make_uint4(vx, vy, key2 | (1u << 16), a.seed));
            float cnt[K];
            float nroot;
            if (INTEGER) {
                uint32_t N[2 * K];
                N[1] = (uint32_t)fN + ((hash_uniform(h.x) < fracN) ? 1u : 0u);
                if (DRAW == kDrawWang) {
#pragma unroll
                    for (int n = 2; n < 2 * K; ++n) N[n] = 0u;
                    if (N[1] > 0u) {
                        N[K] = draw_single_integer(N[1], nd[1], h.y, h.z, false);
                        N[K + 1] = N[1] - N[K];
                    }
                } else {
#pragma unroll
                    for (int n = 1; n < K; ++n) {
                        uint32_t nl = 0u, nr = 0u;
                        if (n >= 2 && !(n & 1) && (N[n] | N[n + 1]))
                            h = pcg4d(make_uint4(vx, vy, key2 | ((uint32_t)(1 + n / 2) << 16), a.seed));
                        const uint32_t u1 = (n == 1) ? h.y : (n & 1) ? h.z : h.x;
                        const uint32_t u2 = (n == 1) ? h.z : (n & 1) ? h.w : h.y;
                        if (DRAW == kDrawDual) {
                            // no branch: an empty node draws 0, and the
                            // independent draws of sibling nodes interleave
                            nl = draw_integer(N[n], nd[n], u1, u2);
                            nr = N[n] - nl;
                        } else if (N[n] > 0u) {
                            nl = draw_single_integer(N[n], nd[n], u1, u2, DRAW == kDrawSingleOld);
                            nr = N[n] - nl;
                        }
                        N[2 * n] = nl;
                        N[2 * n + 1] = nr;
                    }
                }
                nroot = __uint2float_rn(N[1]);
#pragma unroll
                for (int k = 0; k < K; ++k) cnt[k] = __uint2float_rn(N[K + k]);
            } else {
                float N[2 * K];
                N[1] = NP;
                if (DRAW == kDrawWang) {
#pragma unroll
                    for (int n = 2; n < 2 * K; ++n) N[n] = 0.f;
                    draw_single_real(N[1], nd[1], h.y, h.z, false, N[K], N[K + 1]);
                } else {
#pragma unroll
                    for (int n = 1; n < K; ++n) {
                        float nl = 0.f, nr = 0.f;
                        if (n >= 2 && !(n & 1) && (N[n] > 0.f || N[n + 1] > 0.f))
                            h = pcg4d(make_uint4(vx, vy, key2 | ((uint32_t)(1 + n / 2) << 16), a.seed));
                        const uint32_t u1 = (n == 1) ? h.y : (n & 1) ? h.z : h.x;
                        const uint32_t u2 = (n == 1) ? h.z : (n & 1) ? h.w : h.y;
                        if (N[n] > 0.f) {
                            if (DRAW == kDrawDual) draw_real(N[n], nd[n], u1, u2, nl, nr);
                            else draw_single_real(N[n], nd[n], u1, u2, DRAW == kDrawSingleOld, nl, nr);
                        }
                        N[2 * n] = nl;
                        N[2 * n + 1] = nr;
                    }
                }
                nroot = NP;
#pragma unroll
                for (int k = 0; k < K; ++k) cnt[k] = N[K + k];
            }
#pragma unroll
            for (int k = 0; k < K; ++k) M[k] = fmaf(w, cnt[k], M[k]);
            if (DEBUG) {
                const int v = lv * 3 + c;
                if (a.dbg.w) a.dbg.w[q * NS + v] = w;
                if (a.dbg.nroot) a.dbg.nroot[q * NS + v] = nroot;
                if (a.dbg.vert) {
                    a.dbg.vert[(q * NS + v) * 3 + 0] = (int32_t)vx;
                    a.dbg.vert[(q * NS + v) * 3 + 1] = (int32_t)vy;
                    a.dbg.vert[(q * NS + v) * 3 + 2] = GRID ? (int32_t)key2 : l;
                }
                if (a.dbg.counts) for (int k = 0; k < K; ++k) a.dbg.counts[(q * NS + v) * K + k] = cnt[k];
            }
        }
    }

    // ---- 5. radiance
    float num = 0.f;
    if (DRAW == kDrawWang) {  // L_o M / (N_P gamma), M the glint count (bin 1)
        num = M[0];
        den = NP * a.gamma;
    } else {
#pragma unroll
        for (int k = 1; k < K; ++k) num = fmaf(__ldg(a.levels + k), M[k], num);
    }
    float4 o = make_float4(0.f, 0.f, 0.f, 1.f);
    if (den > 0.f) {
        const float ratio = num / den;
        o.x = Lor * ratio;
        o.y = Log * ratio;
        o.z = Lob * ratio;
    }
    a.out[q] = o;
}


}  // namespace
