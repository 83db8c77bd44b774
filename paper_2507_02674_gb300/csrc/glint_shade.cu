// Per-pixel glint shading (Sec. 4 Eq. iblglints:fin; Sec. 3.3 Eq. anisogrid;
// Sec. 5 Alg. 1 and the hierarchical multinomial).
//
// One thread per pixel.  G-buffer reads are four coalesced float4 loads per
// pixel (64 B), the output one float4 store (16 B).  The filtered maps (~2 MB)
// and the 64 x 64 table stay resident in L2/L1 across the frame.  Per pixel:
//   1. smooth radiance L_o = prefRGB (F0 A + B) and p_k = V W_k, p_1 = U + V W_1
//      from 8 bilinear taps of the two filtered levels bracketing the pixel's
//      roughness and 4 table taps (E1);
//   2. footprint |P| and N_P in correctly rounded FP32 (same operation order
//      as any IEEE implementation), grid level and triangle vertices likewise;
//   3. per node of the balanced binary tree over the K bins: node probability
//      p, its complement q (both from the subtree masses), log2 p and the log2
//      of the small-p biased complement, each logarithm taken of whichever of
//      p, q is below 1/2 -- computed once per pixel, reused by all six samples;
//   4. six samples x (K-1) dual-gated draws: a pcg4d hash of (vertex, level,
//      node, seed) gives the uniforms, two hardware exp2 give the gate
//      probabilities, and the normal quantile is evaluated only when the
//      Gaussian branch is taken;
// 64 registers per thread (8 blocks of 128 threads per SM) measured fastest.
//   5. L^_o = L_o sum_k L_k M_k / (N_P sum_k L_k p_k).
#include "glint_internal.cuh"
#include "glint_probs.cuh"
#include "glint_quantile.cuh"

using namespace glint;

namespace {

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

// p_k only, one thread per pixel (background 0).
template <int K, int EV>
__global__ void __launch_bounds__(kShadeNT) k_probs(ShadeArgs a) {
    const long q = (long)blockIdx.x * kShadeNT + threadIdx.x;
    if (q >= a.npix) return;
    const float4 g0 = ldg4(a.view_n0 + q);
    float p[K];
    if (g0.w > 0.f) {
        float lr, lg, lb;
        smooth_and_probs<K, EV>(a, q, g0, ldg4(a.normal_f0 + q), ldg4(a.uv_alpha + q), lr, lg, lb, p);
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) p[k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) a.p_out[q * K + k] = p[k];
}

// Steps 1-5 for pixel q of the frame described by a.
template <int K, bool INTEGER, bool DEBUG, int EV>
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
#pragma unroll
    for (int n = 1; n < K; ++n) {
        const float tot = P[n];
        float pn = 0.f, qn = 1.f;
        if (tot > 0.f) {
            const float inv = 1.f / tot;
            pn = P[2 * n] * inv;
            qn = P[2 * n + 1] * inv;
        }
        nd[n].p = pn;
        nd[n].q = qn;
        // log2 p and log2 q from whichever of p, q is the smaller (both are
        // accurate relative to themselves; 1 - x near 1 is not)
        constexpr float kLog2e = 1.44269504088896340736f;
        float l2p, l2q;
        if (pn <= 0.5f) {
            l2p = log2f(pn);
            l2q = log1pf(-pn) * kLog2e;
        } else {
            l2p = log1pf(-qn) * kLog2e;
            l2q = log2f(qn);
        }
        nd[n].lp = l2p;
        nd[n].lq = (pn >= kEps) ? l2q : (pn * (1.f / kEps)) * kLog2OneMinusEps;
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
#pragma unroll
                for (int n = 1; n < K; ++n) {
                    uint32_t nl = 0u, nr = 0u;
                    if (N[n] > 0u) {
                        if (n > 1) h = pcg4d(make_uint4(vx, vy, key2 | ((uint32_t)n << 16), a.seed));
                        nl = draw_integer(N[n], nd[n], h.y, h.z);
                        nr = N[n] - nl;
                    }
                    N[2 * n] = nl;
                    N[2 * n + 1] = nr;
                }
                nroot = __uint2float_rn(N[1]);
#pragma unroll
                for (int k = 0; k < K; ++k) cnt[k] = __uint2float_rn(N[K + k]);
            } else {
                float N[2 * K];
                N[1] = NP;
#pragma unroll
                for (int n = 1; n < K; ++n) {
                    float nl = 0.f, nr = 0.f;
                    if (N[n] > 0.f) {
                        if (n > 1) h = pcg4d(make_uint4(vx, vy, key2 | ((uint32_t)n << 16), a.seed));
                        draw_real(N[n], nd[n], h.y, h.z, nl, nr);
                    }
                    N[2 * n] = nl;
                    N[2 * n + 1] = nr;
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
#pragma unroll
    for (int k = 1; k < K; ++k) num = fmaf(__ldg(a.levels + k), M[k], num);
    float4 o = make_float4(0.f, 0.f, 0.f, 1.f);
    if (den > 0.f) {
        const float ratio = num / den;
        o.x = Lor * ratio;
        o.y = Log * ratio;
        o.z = Lob * ratio;
    }
    a.out[q] = o;
}

template <int K, bool INTEGER, bool DEBUG, int EV>
__global__ void __launch_bounds__(kShadeNT, 8) k_shade(ShadeArgs a) {
    const long q = (long)blockIdx.x * kShadeNT + threadIdx.x;
    if (q >= a.npix) return;
    shade_pixel<K, INTEGER, DEBUG, EV>(a, q);
}

// Serving: one launch over a work list of (frame, pixel range) items of many
// frames (resolutions, maps and seeds may differ; K is shared).  Block b
// takes items b, b + G, ...; the frame's arguments are staged in shared memory.
template <int K, int EV>
__global__ void __launch_bounds__(kShadeNT, 8) k_serve(const ShadeArgs *__restrict__ frames,
                                                       const ServeItem *__restrict__ items, int nitems) {
    __shared__ ShadeArgs sa;
#pragma unroll 1
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const ServeItem item = items[it];
        __syncthreads();  // the previous item's readers are done
        if (threadIdx.x == 0) sa = frames[item.frame];
        __syncthreads();
#pragma unroll 1
        for (int off = threadIdx.x; off < item.count; off += kShadeNT)
            shade_pixel<K, true, false, EV>(sa, item.first + off);
    }
}

__global__ void k_quantile(const float *__restrict__ p, float *__restrict__ z, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = normal_quantile(p[i]);
}

template <int K, int EV>
void launch_ke(const ShadeArgs &args, bool integer, bool debug, cudaStream_t s) {
    const unsigned grid = (unsigned)((args.npix + kShadeNT - 1) / kShadeNT);
    if (integer) {
        if (debug) k_shade<K, true, true, EV><<<grid, kShadeNT, 0, s>>>(args);
        else k_shade<K, true, false, EV><<<grid, kShadeNT, 0, s>>>(args);
    } else {
        if (debug) k_shade<K, false, true, EV><<<grid, kShadeNT, 0, s>>>(args);
        else k_shade<K, false, false, EV><<<grid, kShadeNT, 0, s>>>(args);
    }
}

template <int K>
cudaError_t launch_k(const ShadeArgs &args, bool integer, bool debug, int ev, cudaStream_t s) {
    if (ev == EV_E2) launch_ke<K, EV_E2>(args, integer, debug, s);
    else if (ev == EV_GIVEN) launch_ke<K, EV_GIVEN>(args, integer, debug, s);
    else launch_ke<K, EV_E1>(args, integer, debug, s);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_probs(const ShadeArgs &args, int ev, cudaStream_t s) {
    const unsigned grid = (unsigned)((args.npix + kShadeNT - 1) / kShadeNT);
    if (ev == EV_E2) k_probs<K, EV_E2><<<grid, kShadeNT, 0, s>>>(args);
    else k_probs<K, EV_E1><<<grid, kShadeNT, 0, s>>>(args);
    return cudaGetLastError();
}

}  // namespace

cudaError_t glint_launch_quantile(const float *p, float *z, long n, cudaStream_t s) {
    if (n > 0) k_quantile<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, z, n);
    return cudaGetLastError();
}

cudaError_t glint_launch_shade(const glint_ctx *ctx, const glint_env *env, const glint_gbuffer *g,
                               const glint_params *p, const float *pk_in, float *out, const glint_debug *dbg,
                               cudaStream_t s, int *launches) {
    ShadeArgs a = make_args(ctx, env, g, p);
    a.out = reinterpret_cast<float4 *>(out);
    a.dbg = dbg ? *dbg : glint_debug{};
    a.pk_in = pk_in;
    const int ev = pk_in ? EV_GIVEN : (p->evaluator == GLINT_EVAL_E2 ? EV_E2 : EV_E1);
    const bool debug = dbg != nullptr;
    const bool integer = p->count_mode == GLINT_COUNT_INTEGER;
    if (launches) *launches = 0;
    if (a.npix == 0) return cudaSuccess;
    cudaError_t e;
    switch (env->d.K) {
    case 2: e = launch_k<2>(a, integer, debug, ev, s); break;
    case 4: e = launch_k<4>(a, integer, debug, ev, s); break;
    case 8: e = launch_k<8>(a, integer, debug, ev, s); break;
    case 16: e = launch_k<16>(a, integer, debug, ev, s); break;
    default: return cudaErrorInvalidValue;
    }
    if (launches) *launches = 1;
    return e;
}

cudaError_t glint_launch_probs(const glint_ctx *ctx, const glint_env *env, const glint_gbuffer *g,
                               const glint_params *p, float *p_out, cudaStream_t s) {
    ShadeArgs a = make_args(ctx, env, g, p);
    a.p_out = p_out;
    const int ev = p->evaluator == GLINT_EVAL_E2 ? EV_E2 : EV_E1;
    if (a.npix == 0) return cudaSuccess;
    switch (env->d.K) {
    case 2: return launch_probs<2>(a, ev, s);
    case 4: return launch_probs<4>(a, ev, s);
    case 8: return launch_probs<8>(a, ev, s);
    case 16: return launch_probs<16>(a, ev, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t glint_launch_serve(int K, bool given, const ShadeArgs *frames, const ServeItem *items, int nitems, int grid,
                               cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    switch (K) {
    case 2: given ? k_serve<2, EV_GIVEN><<<grid, kShadeNT, 0, s>>>(frames, items, nitems)
                  : k_serve<2, EV_E1><<<grid, kShadeNT, 0, s>>>(frames, items, nitems); break;
    case 4: given ? k_serve<4, EV_GIVEN><<<grid, kShadeNT, 0, s>>>(frames, items, nitems)
                  : k_serve<4, EV_E1><<<grid, kShadeNT, 0, s>>>(frames, items, nitems); break;
    case 8: given ? k_serve<8, EV_GIVEN><<<grid, kShadeNT, 0, s>>>(frames, items, nitems)
                  : k_serve<8, EV_E1><<<grid, kShadeNT, 0, s>>>(frames, items, nitems); break;
    case 16: given ? k_serve<16, EV_GIVEN><<<grid, kShadeNT, 0, s>>>(frames, items, nitems)
                   : k_serve<16, EV_E1><<<grid, kShadeNT, 0, s>>>(frames, items, nitems); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
