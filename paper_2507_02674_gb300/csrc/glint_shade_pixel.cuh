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

// Dual-gated Gaussian (Alg. 1) for an integer number of trials N >= 1;
// returns n (nbar = N - n).  Regions of xi1 (same as the printed masks):
// [0, P_{n=N}) -> N;  [P_{n=N}, P_{n=N} + P_{n=1}) -> 1;
// 1 - xi1 <= P_{nbar=N} + P_{nbar=1} -> 0;  otherwise the clamped, rounded
// Gaussian when N > 1, else 0.
__device__ __forceinline__ uint32_t draw_integer(uint32_t N, const NodeParams &np, uint32_t h1, uint32_t h2) {
    const float xi1 = hash_uniform(h1);
    const float xi1c = hash_uniform_complement(h1);
    const float Nf = __uint2float_rn(N);
    const float N2 = fmaxf(2.f, Nf);
    const float a = (N >= 2u) ? 1.f : 0.f;
    const float b = (N == 1u) ? 1.f : 0.f;
    const float Pall = a * fast_exp2(N2 * np.lp);
    const float T1 = Pall + b * np.p;
    const float Sneg = a * fast_exp2(N2 * np.lq) + b * np.q;
    if (xi1 < Pall) return N;
    if (xi1 < T1) return 1u;
    if (xi1c <= Sneg || N < 2u) return 0u;
    const float mu = 1.f + (N2 - 2.f) * np.p;
    const float sigma = fast_sqrt((N2 - 2.f) * np.p * np.q);
    const float z = normal_quantile(hash_uniform(h2));
    float G = floorf(fmaf(sigma, z, mu) + 0.5f);
    G = fminf(fmaxf(G, 1.f), kMaxCount);
    return min((uint32_t)G, N - 1u);
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


// Node parameters of a binary split with probabilities p (left) and q = 1 - p
// (right): log2 p and log2 of the small-p biased complement, each logarithm
// taken of whichever of p, q is the smaller (1 - x near 1 is not accurate).
__device__ __forceinline__ NodeParams node_params(float pn, float qn) {
    constexpr float kLog2e = 1.44269504088896340736f;
    NodeParams nd;
    nd.p = pn;
    nd.q = qn;
    float l2p, l2q;
    if (pn <= 0.5f) {
        l2p = log2f(pn);
        l2q = log1pf(-pn) * kLog2e;
    } else {
        l2p = log1pf(-qn) * kLog2e;
        l2q = log2f(qn);
    }
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

// Steps 1-5 for pixel q of the frame described by a.  DRAW selects the binomial
// approximation at the tree nodes: dual-gated (the paper's), single-gated
// (Eq. gated), the older single-gated form (Eq. oldgated), or the Wang 2020
// comparison (a single-gated glint count with the environment-independent
// probability gamma, radiance L_o M / (N_P gamma); Sec. 7).
template <int K, bool INTEGER, bool DEBUG, int EV, int DRAW = kDrawDual>
__device__ __forceinline__ void shade_pixel(const ShadeArgs &a, long q) {
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
            for (int v = 0; v < 6; ++v) {
                if (a.dbg.w) a.dbg.w[q * 6 + v] = 0.f;
                if (a.dbg.nroot) a.dbg.nroot[q * 6 + v] = 0.f;
                if (a.dbg.vert) for (int c = 0; c < 3; ++c) a.dbg.vert[(q * 6 + v) * 3 + c] = 0;
                if (a.dbg.counts) for (int k = 0; k < K; ++k) a.dbg.counts[(q * 6 + v) * K + k] = 0.f;
            }
        }
        return;
    }

    // ---- 1. smooth radiance and reflection probabilities
    float Lor, Log, Lob;
    float p[K];
    smooth_and_probs<K, EV>(a, q, g0, g1, g2, Lor, Log, Lob, p);

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
            for (int v = 0; v < 6; ++v) {
                if (a.dbg.w) a.dbg.w[q * 6 + v] = 0.f;
                if (a.dbg.nroot) a.dbg.nroot[q * 6 + v] = 0.f;
                if (a.dbg.vert) for (int c = 0; c < 3; ++c) a.dbg.vert[(q * 6 + v) * 3 + c] = 0;
                if (a.dbg.counts) for (int k = 0; k < K; ++k) a.dbg.counts[(q * 6 + v) * K + k] = 0.f;
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
            float pn = 0.f, qn = 1.f;
            if (tot > 0.f) {
                const float inv = 1.f / tot;
                pn = P[2 * n] * inv;
                qn = P[2 * n + 1] * inv;
            }
            nd[n] = node_params(pn, qn);
        }
    }

    // ---- 4. six grid samples x (K-1) draws
    float M[K];
#pragma unroll
    for (int k = 0; k < K; ++k) M[k] = 0.f;
    const float F2 = 0x1.76cf5ep-2f;  // (sqrt(3) - 1) / 2
    const float fN = floorf(NP);
    const float fracN = NP - fN;
#pragma unroll 1
    for (int lv = 0; lv < 2; ++lv) {
        const int l = l0 + lv;
        const float lw = lv ? fl : 1.f - fl;
        const float x = ldexpf(g2.x, -l), y = ldexpf(g2.y, -l);
        const float sk = __fmul_rn(__fadd_rn(x, y), F2);
        const float xs = __fadd_rn(x, sk), ys = __fadd_rn(y, sk);
        const float fi = floorf(xs), fj = floorf(ys);
        const float fx = __fsub_rn(xs, fi), fy = __fsub_rn(ys, fj);
        const uint32_t ii = low32_of_integral(fi), jj = low32_of_integral(fj);
        const bool tri = fx > fy;
        const float bmax = tri ? fx : fy, bmin = tri ? fy : fx;
        const uint32_t key2 = ((uint32_t)l) & 0xFFFFu;
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            const uint32_t vx = ii + ((c == 2 || (c == 1 && tri)) ? 1u : 0u);
            const uint32_t vy = jj + ((c == 2 || (c == 1 && !tri)) ? 1u : 0u);
            const float bc = (c == 0) ? 1.f - bmax : (c == 1) ? bmax - bmin : bmin;
            const float w = lw * bc;
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
                        if (N[n] > 0u) {
                            if (n > 1) h = pcg4d(make_uint4(vx, vy, key2 | ((uint32_t)n << 16), a.seed));
                            nl = (DRAW == kDrawDual) ? draw_integer(N[n], nd[n], h.y, h.z)
                                                     : draw_single_integer(N[n], nd[n], h.y, h.z, DRAW == kDrawSingleOld);
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
                        if (N[n] > 0.f) {
                            if (n > 1) h = pcg4d(make_uint4(vx, vy, key2 | ((uint32_t)n << 16), a.seed));
                            if (DRAW == kDrawDual) draw_real(N[n], nd[n], h.y, h.z, nl, nr);
                            else draw_single_real(N[n], nd[n], h.y, h.z, DRAW == kDrawSingleOld, nl, nr);
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
                if (a.dbg.w) a.dbg.w[q * 6 + v] = w;
                if (a.dbg.nroot) a.dbg.nroot[q * 6 + v] = nroot;
                if (a.dbg.vert) {
                    a.dbg.vert[(q * 6 + v) * 3 + 0] = (int32_t)vx;
                    a.dbg.vert[(q * 6 + v) * 3 + 1] = (int32_t)vy;
                    a.dbg.vert[(q * 6 + v) * 3 + 2] = l;
                }
                if (a.dbg.counts) for (int k = 0; k < K; ++k) a.dbg.counts[(q * 6 + v) * K + k] = cnt[k];
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
