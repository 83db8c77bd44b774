// BF16 MLP surrogate of the per-component reflection probabilities p_k
// (the NDF mass of Eq. probhk that the E2 quadrature computes), trained and
// evaluated on the tensor cores with FP32 accumulation.
//
// Network: 64 inputs (glint_probs.cuh: E1's p_k, the filtered weights W_k at
// five taps across the anisotropic lobe, mu_o, sqrt a_x, sqrt a_y) -> 64 ->
// 64 -> K, ReLU, and p = softmax(logits + log max(p^E1, 1e-6)): the network
// learns a correction of E1 towards the anisotropic integral.  Parameters
// (FP32 master copy, `glint_mlp_param_count` floats):
//   W1 [64 in][64 out], b1[64], W2 [64][64], b2[64], W3 [64][16] (columns >= K
//   unused), b3[16].
// The tensor-core copies are BF16 in both layouts: W^T [out][in] for the
// forward pass (B fragments read (k, k+1) pairs contiguously) and W [in][out]
// for the backward pass.
//
// Tensor cores: warp-level mma.sync.m16n8k16 (BF16 in, FP32 accumulate).  A
// layer for a 16-row tile is 4 k-steps x (out/8) n-tiles; the FP32
// accumulator fragments of two adjacent n-tiles are exactly the A fragment of
// the next layer's k-step, so activations stay in registers between layers
// (ReLU and BF16 rounding applied on the way).  The inference and forward
// kernels are persistent: each block stages the weights in shared memory once
// and loops over 128-row tiles.
#include <cuda_bf16.h>

#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <string>
#include <vector>

#include "glint_internal.cuh"
#include "glint_probs.cuh"
#include "glint_shade_pixel.cuh"

using namespace glint;

namespace {

constexpr int kIn = 64;
constexpr int kHid = 64;
constexpr int kOutPad = 16;
constexpr int kP = kIn * kHid + kHid + kHid * kHid + kHid + kHid * kOutPad + kOutPad;  // 9360
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kIn * kHid, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kOutPad;
constexpr int kNT = 128;  // threads (samples) per block
constexpr int kLpStride = 17;  // floats per log-prior row in shared memory (odd: no bank conflicts)

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ uint32_t pair16(const __nv_bfloat16 *lo, const __nv_bfloat16 *hi) {
    const uint32_t a = *reinterpret_cast<const uint16_t *>(lo);
    const uint32_t b = *reinterpret_cast<const uint16_t *>(hi);
    return a | (b << 16);
}

// Every [rows][64] BF16 tile in shared memory (inputs, activations,
// backpropagated signals and the 64-wide weight matrices) is stored with its
// eight 16-byte chunks per row permuted by chunk ^ (row & 7): the fragment
// loads of mma.sync (8 consecutive rows x 4 words, or 8 rows apart in the
// transposed gradient reads) then hit 32 distinct banks.
__device__ __forceinline__ int word_at(int r, int w) {
    return r * 32 + ((((w >> 2) ^ (r & 7)) << 2) | (w & 3));
}
__device__ __forceinline__ const __nv_bfloat16 *el(const __nv_bfloat16 *m, int r, int c) {
    return m + 2 * word_at(r, c >> 1) + (c & 1);
}
__device__ __forceinline__ uint32_t wd(const __nv_bfloat16 *m, int r, int w) {
    return reinterpret_cast<const uint32_t *>(m)[word_at(r, w)];
}

// Copy a row-major [ROWS][64] BF16 matrix from global memory into the
// swizzled layout, 16 bytes a thread at a time, for blocks of NT threads: all
// of a thread's loads are issued before its stores, so their latencies overlap
// instead of adding up.
template <int ROWS, int NT>
__device__ __forceinline__ void copy_swz(__nv_bfloat16 *dst, const __nv_bfloat16 *src) {
    constexpr int kChunks = ROWS * 8, kPer = (kChunks + NT - 1) / NT;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    uint4 v[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int i = j * NT + (int)threadIdx.x;
        if (i < kChunks) v[j] = __ldg(s4 + i);
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int i = j * NT + (int)threadIdx.x;
        if (i < kChunks) d4[(i >> 3) * 8 + ((i & 7) ^ ((i >> 3) & 7))] = v[j];
    }
}

struct SmemW {
    __nv_bfloat16 w1t[kHid * kIn], w2t[kHid * kHid], w3t[kOutPad * kHid];  // [out][in]
    float b1[kHid], b2[kHid], b3[kOutPad];
};
struct SmemWB {
    __nv_bfloat16 w2[kHid * kHid], w3[kHid * kOutPad];  // [in][out] (backward)
};

template <int NT>
__device__ void load_weights(SmemW &s, const __nv_bfloat16 *wt, const float *params) {
    copy_swz<kHid, NT>(s.w1t, wt);
    copy_swz<kHid, NT>(s.w2t, wt + kHid * kIn);
    copy_swz<kOutPad, NT>(s.w3t, wt + kHid * kIn + kHid * kHid);
    const int i = threadIdx.x;
    if (i < kHid) {
        s.b1[i] = __ldg(params + kOffB1 + i);
        s.b2[i] = __ldg(params + kOffB2 + i);
    } else if (i < kHid + kOutPad) {
        s.b3[i - kHid] = __ldg(params + kOffB3 + i - kHid);
    }
}

// One layer for a warp's 16-row tile: c[j] = bias + A (16 x 64) W^T[j-th 8 columns].
template <int NT>
__device__ __forceinline__ void layer_fwd(const uint32_t a[4][4], const __nv_bfloat16 *wt, const float *bias,
                                          float c[NT][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        c[j][0] = c[j][2] = bias[j * 8 + 2 * t];
        c[j][1] = c[j][3] = bias[j * 8 + 2 * t + 1];
    }
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            mma16816(c[j], a[ks], wd(wt, j * 8 + g, ks * 8 + t), wd(wt, j * 8 + g, ks * 8 + t + 4));
        }
    }
}

// ReLU, BF16 rounding, and the accumulators of n-tiles (2ks, 2ks+1) as the A
// fragment of k-step ks.
__device__ __forceinline__ void relu_to_a(const float c[8][4], uint32_t a[4][4]) {
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        a[ks][0] = pack_bf16(fmaxf(c[2 * ks][0], 0.f), fmaxf(c[2 * ks][1], 0.f));
        a[ks][1] = pack_bf16(fmaxf(c[2 * ks][2], 0.f), fmaxf(c[2 * ks][3], 0.f));
        a[ks][2] = pack_bf16(fmaxf(c[2 * ks + 1][0], 0.f), fmaxf(c[2 * ks + 1][1], 0.f));
        a[ks][3] = pack_bf16(fmaxf(c[2 * ks + 1][2], 0.f), fmaxf(c[2 * ks + 1][3], 0.f));
    }
}

// A fragments of a 16-row tile of a row-major [rows][64] BF16 matrix in smem.
__device__ __forceinline__ void load_a(const __nv_bfloat16 *m, int row0, uint32_t a[4][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        a[ks][0] = wd(m, row0 + g, ks * 8 + t);
        a[ks][1] = wd(m, row0 + g + 8, ks * 8 + t);
        a[ks][2] = wd(m, row0 + g, ks * 8 + t + 4);
        a[ks][3] = wd(m, row0 + g + 8, ks * 8 + t + 4);
    }
}

// Store the (ReLU'd, BF16) accumulators of a 16-row tile to smem [rows][64].
__device__ __forceinline__ void store_c_bf16(__nv_bfloat16 *m, int row0, const float c[8][4], bool relu) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float v0 = c[j][0], v1 = c[j][1], v2 = c[j][2], v3 = c[j][3];
        if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); v2 = fmaxf(v2, 0.f); v3 = fmaxf(v3, 0.f); }
        uint32_t *w = reinterpret_cast<uint32_t *>(m);
        w[word_at(row0 + g, j * 4 + t)] = pack_bf16(v0, v1);
        w[word_at(row0 + g + 8, j * 4 + t)] = pack_bf16(v2, v3);
    }
}

// Softmax over the K logits plus log-prior (lp: smem [rows][16]) of each row
// of a 16-row tile (cols >= K ignored); the 8 (or 16) logits of a row live in
// the 4 lanes of its quad.
template <int NT>
__device__ __forceinline__ void softmax_rows(float c[NT][4], int K, const float *lp, int row0) {
    const int t = threadIdx.x & 3, g = (threadIdx.x & 31) >> 2;
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // rows g and g + 8
        const float *lr = lp + (row0 + g + 8 * h) * kLpStride;
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int e = 0; e < 2; ++e)
                if (j * 8 + 2 * t + e < K) c[j][2 * h + e] += lr[j * 8 + 2 * t + e];
        float mx = -INFINITY;
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int e = 0; e < 2; ++e)
                if (j * 8 + 2 * t + e < K) mx = fmaxf(mx, c[j][2 * h + e]);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
        float sum = 0.f;
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const bool ok = j * 8 + 2 * t + e < K;
                const float v = ok ? expf(c[j][2 * h + e] - mx) : 0.f;
                c[j][2 * h + e] = v;
                sum += v;
            }
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        sum += __shfl_xor_sync(0xffffffffu, sum, 2);
        const float inv = 1.f / sum;
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            c[j][2 * h] *= inv;
            c[j][2 * h + 1] *= inv;
        }
    }
}

// ------------------------------------------------------------------ inference
// Shared memory of the inference kernels: weights, one 128-row input tile
// (swizzled) and its log-priors.
struct SmemInfer {
    SmemW w;
    __align__(16) __nv_bfloat16 xs[kNT * 64];
    float lp[kNT * kLpStride];
    int fg[kNT];
};

// Sink of mlp_features into row r of the staged tile: each pair of inputs is
// rounded to BF16 and stored at its swizzled word as soon as it is computed.
template <int K>
struct SmemRowSink {
    SmemInfer &sm;
    int r;
    __device__ __forceinline__ void group(int i, const float *v) {
        uint32_t *w32 = reinterpret_cast<uint32_t *>(sm.xs);
#pragma unroll
        for (int j = 0; j < K / 2; ++j) w32[word_at(r, i / 2 + j)] = pack_bf16(v[2 * j], v[2 * j + 1]);
    }
    __device__ __forceinline__ void log_prior(const float *l) {
#pragma unroll
        for (int k = 0; k < kOutPad; ++k) sm.lp[r * kLpStride + k] = k < K ? l[k] : 0.f;
    }
    __device__ __forceinline__ void tail(int i, const float *v) {
        uint32_t *w32 = reinterpret_cast<uint32_t *>(sm.xs);
        w32[word_at(r, i / 2)] = pack_bf16(v[0], v[1]);
        w32[word_at(r, i / 2 + 1)] = pack_bf16(v[2], 0.f);
#pragma unroll
        for (int w = 3 * K + 2; w < 32; ++w) w32[word_at(r, w)] = 0u;
    }
    // a background row or one past the end: zero inputs and log-priors
    __device__ __forceinline__ void zero() {
        uint4 *x4 = reinterpret_cast<uint4 *>(sm.xs);
#pragma unroll
        for (int q = 0; q < 8; ++q) x4[r * 8 + q] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int k = 0; k < kOutPad; ++k) sm.lp[r * kLpStride + k] = 0.f;
    }
};

// Network on the staged tile: rows [0, 128) of xs/lp; p of live rows to
// p_out[(base + r) K + k] (0 where fg[r] == 0).
template <int NT>
__device__ __forceinline__ void net_tile(const SmemInfer &sm, long base, long n, int K, float *__restrict__ p_out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        const int row0 = warp * 32 + mt * 16;
        uint32_t a[4][4];
        float c[8][4];
        load_a(sm.xs, row0, a);
        layer_fwd<8>(a, sm.w.w1t, sm.w.b1, c);
        relu_to_a(c, a);
        layer_fwd<8>(a, sm.w.w2t, sm.w.b2, c);
        relu_to_a(c, a);
        float o[NT][4];
        layer_fwd<NT>(a, sm.w.w3t, sm.w.b3, o);
        softmax_rows<NT>(o, K, sm.lp, row0);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = row0 + g + 8 * h;
            const long i = base + r;
            if (i >= n) continue;
            const bool fg = sm.fg[r] != 0;
#pragma unroll
            for (int j = 0; j < NT; ++j)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int col = j * 8 + 2 * t + e;
                    if (col < K) p_out[i * K + col] = fg ? o[j][2 * h + e] : 0.f;
                }
        }
    }
}

// p of given inputs: x (n x 64 BF16, row-major), lp (n x K).  Persistent.
template <int NT>
__global__ void __launch_bounds__(kNT) k_mlp_forward(const uint4 *__restrict__ x, const float *__restrict__ lp, long n,
                                                     int K, const __nv_bfloat16 *__restrict__ wt,
                                                     const float *__restrict__ params, float *__restrict__ p_out) {
    __shared__ SmemInfer sm;
    load_weights<kNT>(sm.w, wt, params);
    const long ntiles = (n + kNT - 1) / kNT;
#pragma unroll 1
    for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long base = tile * kNT;
        __syncthreads();  // the previous tile's readers are done
        uint4 *x4 = reinterpret_cast<uint4 *>(sm.xs);
        // 128 rows x 8 uint4: consecutive threads read consecutive 16-byte pieces
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int idx = it * kNT + threadIdx.x;
            const int r = idx >> 3, q = idx & 7;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (base + r < n) v = __ldg(x + (base + r) * 8 + q);
            x4[r * 8 + (q ^ (r & 7))] = v;
        }
        for (int idx = threadIdx.x; idx < kNT * kOutPad; idx += kNT) {
            const int r = idx / kOutPad, k = idx % kOutPad;
            sm.lp[r * kLpStride + k] = (base + r < n && k < K) ? __ldg(lp + (base + r) * K + k) : 0.f;
        }
        sm.fg[threadIdx.x] = 1;
        __syncthreads();
        net_tile<NT>(sm, base, n, K, p_out);
    }
}

// Features and network fused: p of every pixel of a G-buffer (background 0).
template <int K>
__global__ void __launch_bounds__(kNT, 4) k_mlp_infer(ShadeArgs a, const __nv_bfloat16 *__restrict__ wt,
                                                   const float *__restrict__ params, float *__restrict__ p_out) {
    __shared__ SmemInfer sm;
    load_weights<kNT>(sm.w, wt, params);
    const long ntiles = (a.npix + kNT - 1) / kNT;
#pragma unroll 1
    for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long base = tile * kNT;
        const long q = base + threadIdx.x;
        __syncthreads();  // the previous tile's readers are done
        SmemRowSink<K> sink{sm, (int)threadIdx.x};
        bool fg = false;
        if (q < a.npix) {
            const float4 g0 = ldg4(a.view_n0 + q);
            fg = g0.w > 0.f;
            if (fg) {
                const float4 g1 = ldg4(a.normal_f0 + q), g2 = ldg4(a.uv_alpha + q);
                float pe[K];
                e1_probs<K>(a, g0, g1, g2, pe);
                mlp_features<K>(a, q, g0, g1, g2, pe, sink);
            }
        }
        if (!fg) sink.zero();
        sm.fg[threadIdx.x] = fg ? 1 : 0;
        __syncthreads();
        net_tile<(K > 8 ? 2 : 1)>(sm, base, a.npix, K, p_out);
    }
}

// ------------------------------------------------------------------ shading
// The surrogate fused into the shading: a block of kFusedNT pixels computes
// their inputs (mlp_features, as k_mlp_infer), the network on the tile (warp w
// on rows [32 w, 32 w + 32)), and the glint draws (shade_draws) with the
// network's p_k from shared memory -- no per-pixel p_k leaves the chip.  The
// smooth radiance comes from the colour channels at E1's taps, in the same
// pass as E1's p_k (one reflection direction, level pair and table fetch).  Two blocks of 256 threads per SM: 69 KB of
// shared memory each (weights, the input tile, log-priors then p_k in place),
// leaving ~90 KB of L1 for the texel gathers of the inputs, and up to 128
// registers a thread (no spills; three blocks at 80 registers spilled and
// took 3% longer).
constexpr int kFusedNT = 256;

struct SmemFused {
    SmemW w;
    __align__(16) __nv_bfloat16 xs[kFusedNT * 64];
    float lp[kFusedNT * kLpStride];  // log-priors, then p_k in place
    int fg[kFusedNT];
};

// Sink of mlp_features into row r of the fused kernel's tile (as SmemRowSink).
template <int K>
struct FusedRowSink {
    SmemFused &sm;
    int r;
    __device__ __forceinline__ void group(int i, const float *v) {
        uint32_t *w32 = reinterpret_cast<uint32_t *>(sm.xs);
        if constexpr (K == 8) {  // groups start at multiples of 8 inputs: one whole 16-byte chunk
            *reinterpret_cast<uint4 *>(w32 + word_at(r, i / 2)) =
                make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                           pack_bf16(v[6], v[7]));
        } else {
#pragma unroll
            for (int j = 0; j < K / 2; ++j) w32[word_at(r, i / 2 + j)] = pack_bf16(v[2 * j], v[2 * j + 1]);
        }
    }
    __device__ __forceinline__ void log_prior(const float *l) {
#pragma unroll
        for (int k = 0; k < kOutPad; ++k) sm.lp[r * kLpStride + k] = k < K ? l[k] : 0.f;
    }
    __device__ __forceinline__ void tail(int i, const float *v) {
        uint32_t *w32 = reinterpret_cast<uint32_t *>(sm.xs);
        w32[word_at(r, i / 2)] = pack_bf16(v[0], v[1]);
        w32[word_at(r, i / 2 + 1)] = pack_bf16(v[2], 0.f);
#pragma unroll
        for (int w = 3 * K + 2; w < 32; ++w) w32[word_at(r, w)] = 0u;
    }
    __device__ __forceinline__ void zero() {
        uint4 *x4 = reinterpret_cast<uint4 *>(sm.xs);
#pragma unroll
        for (int q = 0; q < 8; ++q) x4[r * 8 + q] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int k = 0; k < kOutPad; ++k) sm.lp[r * kLpStride + k] = 0.f;
    }
};

// One tile of the fused kernel: pixel q of frame `a` (valid: q is one of the
// tile's pixels) with the block's kFusedNT threads; the weights are in sm.w.
// Every thread of the block calls it (it synchronises twice).
template <int K, bool INTEGER, bool DEBUG>
__device__ __forceinline__ void fused_tile(const ShadeArgs &a, SmemFused &sm, long q, bool valid) {
    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f);
    bool fg = false;
    if (valid) {
        g0 = ldg4(a.view_n0 + q);
        fg = g0.w > 0.f;
    }
    FusedRowSink<K> sink{sm, (int)threadIdx.x};
    float L[3] = {0.f, 0.f, 0.f};  // the smooth radiance, from E1's taps
    if (fg) {
        const float4 g1 = ldg4(a.normal_f0 + q), g2 = ldg4(a.uv_alpha + q);
        float pe[K];
        e1_probs<K, true>(a, g0, g1, g2, pe, L);
        mlp_features<K>(a, q, g0, g1, g2, pe, sink);
    } else {
        sink.zero();
    }
    sm.fg[threadIdx.x] = fg ? 1 : 0;
    __syncthreads();
    {
        constexpr int NT = K > 8 ? 2 : 1;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll 1
        for (int mt = 0; mt < 2; ++mt) {
            const int row0 = warp * 32 + mt * 16;
            uint32_t af[4][4];
            float c[8][4];
            load_a(sm.xs, row0, af);
            layer_fwd<8>(af, sm.w.w1t, sm.w.b1, c);
            relu_to_a(c, af);
            layer_fwd<8>(af, sm.w.w2t, sm.w.b2, c);
            relu_to_a(c, af);
            float o[NT][4];
            layer_fwd<NT>(af, sm.w.w3t, sm.w.b3, o);
            softmax_rows<NT>(o, K, sm.lp, row0);  // reads each lane's own log-priors
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float *pr = sm.lp + (row0 + g + 8 * h) * kLpStride;
#pragma unroll
                for (int j = 0; j < NT; ++j)
#pragma unroll
                    for (int e = 0; e < 2; ++e)
                        if (j * 8 + 2 * t + e < K) pr[j * 8 + 2 * t + e] = o[j][2 * h + e];
            }
        }
    }
    __syncthreads();
    if (!valid) return;
    if (!fg) {
        shade_pixel<K, INTEGER, DEBUG, EV_NONE>(a, q);  // background: black, debug outputs 0
        return;
    }
    const float4 g2 = ldg4(a.uv_alpha + q), g3 = ldg4(a.duv + q);
    float p[K];
#pragma unroll
    for (int k = 0; k < K; ++k) p[k] = sm.lp[threadIdx.x * kLpStride + k];
    shade_draws<K, INTEGER, DEBUG, kDrawDual, 0>(a, q, g0, g2, g3, L[0], L[1], L[2], p);
}

template <int K, bool INTEGER, bool DEBUG>
__global__ void __launch_bounds__(kFusedNT, 2) k_shade_mlp(ShadeArgs a, const __nv_bfloat16 *__restrict__ wt,
                                                          const float *__restrict__ params) {
    extern __shared__ __align__(16) unsigned char fused_smem[];
    SmemFused &sm = *reinterpret_cast<SmemFused *>(fused_smem);
    load_weights<kFusedNT>(sm.w, wt, params);
    const long q = (long)blockIdx.x * kFusedNT + threadIdx.x;
    fused_tile<K, INTEGER, DEBUG>(a, sm, q, q < a.npix);
}

// Serving with the fused surrogate: one launch over a work list of (frame,
// pixel range) items of frames on the surrogate path.  Block b takes items
// b, b + G, ...; the frame's arguments are staged in shared memory and the
// weights reloaded when the item's network differs from the block's last;
// each item runs in tiles of kFusedNT pixels.  A pixel comes out as
// k_shade_mlp computes it.
struct SmemServeFused {
    SmemFused f;
    ShadeArgs sa;
};

template <int K>
__global__ void __launch_bounds__(kFusedNT, 2) k_serve_mlp(const ShadeArgs *__restrict__ frames,
                                                          const ServeItem *__restrict__ items, int nitems) {
    extern __shared__ __align__(16) unsigned char fused_smem[];
    SmemServeFused &sm = *reinterpret_cast<SmemServeFused *>(fused_smem);
    const void *held = nullptr;
#pragma unroll 1
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const ServeItem item = items[it];
        __syncthreads();  // the previous item's readers of sa, the weights and the tile are done
        if (threadIdx.x == 0) sm.sa = frames[item.frame];
        __syncthreads();
        if (sm.sa.mlp_wt != held) {  // uniform over the block
            held = sm.sa.mlp_wt;
            load_weights<kFusedNT>(sm.f.w, reinterpret_cast<const __nv_bfloat16 *>(sm.sa.mlp_wt), sm.sa.mlp_params);
        }
        const long end = item.first + item.count;
#pragma unroll 1
        for (long base = item.first; base < end; base += kFusedNT) {
            __syncthreads();  // the previous tile's readers of xs and lp are done
            const long q = base + threadIdx.x;
            fused_tile<K, true, false>(sm.sa, sm.f, q, q < end);
        }
    }
}

// Inputs of every pixel: x (n x 64 BF16, background rows 0), lp (n x K).
template <int K>
__global__ void __launch_bounds__(kNT) k_mlp_features(ShadeArgs a, uint4 *__restrict__ x, float *__restrict__ lp) {
    const long q = (long)blockIdx.x * kNT + threadIdx.x;
    if (q >= a.npix) return;
    float f[kMlpIn], l[K];
    const float4 g0 = ldg4(a.view_n0 + q);
    const bool fg = g0.w > 0.f;
    if (fg) {
        ArraySink<K> sink{f, l};
        const float4 g1 = ldg4(a.normal_f0 + q), g2 = ldg4(a.uv_alpha + q);
        float pe[K];
        e1_probs<K>(a, g0, g1, g2, pe);
        mlp_features<K>(a, q, g0, g1, g2, pe, sink);
    } else {
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) f[i] = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) l[k] = 0.f;
    }
#pragma unroll
    for (int v = 0; v < 8; ++v)
        x[q * 8 + v] = make_uint4(pack_bf16(f[8 * v], f[8 * v + 1]), pack_bf16(f[8 * v + 2], f[8 * v + 3]),
                                  pack_bf16(f[8 * v + 4], f[8 * v + 5]), pack_bf16(f[8 * v + 6], f[8 * v + 7]));
#pragma unroll
    for (int k = 0; k < K; ++k) lp[q * K + k] = l[k];
}

// ------------------------------------------------------------------ training
// Forward and backward over chunks of kChunk samples.  Block b handles chunks
// b, b + G, b + 2G, ... (G = gridDim.x) of the batch and accumulates its
// gradient (each sample's loss weighted by 1/batch) in partial[b][kP], always
// in the same order, so the result does not depend on scheduling; its summed
// squared error sum_k (p_k - y_k)^2 goes to loss[b].  A chunk of 32 samples gives a batch of 8192
// 256 blocks, so every SM has work; the 16-row tiles of the chunk go to the
// warps in turn.
constexpr int kChunk = 32;
static_assert(kChunk * 8 % 128 == 0, "whole 16-byte pieces of inputs per thread");

// Fragments of the transposed operands of the weight-gradient products
// (ldmatrix .trans from row-major [samples][cols] tiles): the 16 x 16 A
// fragment of act^T (rows = columns m0.., k = samples k0..) from a swizzled
// [rows][64] BF16 tile, and the 16 x 8 B fragments of two adjacent n-tiles
// (n0.., n0 + 8..) of a [rows][ld] tile (ld = 64 swizzled or 16 plain).
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t r[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ uint32_t row_chunk_addr(const __nv_bfloat16 *m, int ld, int row, int chunk) {
    const int c = ld == 64 ? (chunk ^ (row & 7)) : chunk;  // 16-byte chunk within the row
    return smem_u32(m + row * ld + c * 8);
}
__device__ __forceinline__ void frag_at(const __nv_bfloat16 *act, int k0, int m0, uint32_t a[4]) {
    const int L = threadIdx.x & 31;
    ldsm_x4_trans(a, row_chunk_addr(act, 64, k0 + (L & 7) + ((L >> 4) << 3), (m0 >> 3) + ((L >> 3) & 1)));
}
__device__ __forceinline__ void frag_b2(const __nv_bfloat16 *dz, int ld, int k0, int n0, uint32_t b[4]) {
    // matrices: (k0.., n0), (k0 + 8.., n0), (k0.., n0 + 8), (k0 + 8.., n0 + 8)
    const int L = threadIdx.x & 31;
    ldsm_x4_trans(b, row_chunk_addr(dz, ld, k0 + (L & 7) + (((L >> 3) & 1) << 3), (n0 >> 3) + (L >> 4)));
}

// Programmatic dependent launch between the training kernels: a kernel's
// blocks may become resident while the previous kernel of the stream still
// runs; griddepcontrol.wait (first, before any global read or write) holds
// them until that kernel has completed and its writes are visible, and
// launch_dependents lets the next kernel's blocks be scheduled.  Without the
// launch attribute both are no-ops.
__device__ __forceinline__ void pdl_wait_then_release() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <int NT>
__global__ void __launch_bounds__(kNT) k_mlp_grad(const uint4 *__restrict__ xg, const float *__restrict__ lpg,
                                                  const float *__restrict__ targets, long n_total, long first,
                                                  long batch, int K, const __nv_bfloat16 *__restrict__ wt,
                                                  const __nv_bfloat16 *__restrict__ wb,
                                                  const float *__restrict__ params, float *__restrict__ partial,
                                                  float *__restrict__ loss) {
    constexpr int CH = kChunk, MT = CH / 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemW &sw = *reinterpret_cast<SmemW *>(smem_raw);
    SmemWB &sb = *reinterpret_cast<SmemWB *>(smem_raw + sizeof(SmemW));
    __nv_bfloat16 *xs = reinterpret_cast<__nv_bfloat16 *>(smem_raw + sizeof(SmemW) + sizeof(SmemWB));
    __nv_bfloat16 *h1 = xs + CH * 64;
    __nv_bfloat16 *h2 = h1 + CH * 64;     // H2, later dZ1
    __nv_bfloat16 *dz = h2 + CH * 64;     // dZ2
    __nv_bfloat16 *dz3 = dz + CH * 64;    // [CH][16]
    float *red = reinterpret_cast<float *>(dz3 + CH * 16);  // kNT floats
    float *lps = red + kNT;                                  // [CH][kLpStride] log-priors
    float *ys = lps + CH * kLpStride;                        // [CH][16] targets

    // stage chunk c's inputs, log-priors and targets in shared memory
    auto stage = [&](long c) {
        const long base = first + c * CH;  // samples [base, base + CH) of the data set, wrapping
        const long nb = first + batch;
        uint4 *xs4 = reinterpret_cast<uint4 *>(xs);
        constexpr int kXPer = CH * 8 / kNT;  // 16-byte pieces of the chunk's inputs per thread
        uint4 xv[kXPer];
#pragma unroll
        for (int it = 0; it < kXPer; ++it) {
            const int idx = it * kNT + threadIdx.x, r = idx >> 3, q = idx & 7;
            const long i = base + r;
            xv[it] = (i < nb) ? __ldg(xg + (i % n_total) * 8 + q) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int it = 0; it < kXPer; ++it) {
            const int idx = it * kNT + threadIdx.x, r = idx >> 3, q = idx & 7;
            xs4[r * 8 + (q ^ (r & 7))] = xv[it];
        }
#pragma unroll
        for (int it = 0; it < (CH * kOutPad + kNT - 1) / kNT; ++it) {
            const int idx = it * kNT + threadIdx.x;
            const int r = idx / kOutPad, k = idx % kOutPad;
            const long i = base + r;
            const bool ok = idx < CH * kOutPad && i < nb && k < K;
            const long src = (i % n_total) * K + k;
            const float lv = ok ? __ldg(lpg + src) : 0.f, yv = ok ? __ldg(targets + src) : 0.f;
            if (idx < CH * kOutPad) {
                lps[r * kLpStride + k] = lv;
                ys[r * 16 + k] = yv;
            }
        }
    };
    // The training data are read-only for every kernel of the library, so the
    // first chunk is staged before the wait on the previous kernel (in a
    // training run, the previous step's Adam update); a launch whose
    // predecessor may write them does not use programmatic dependent launch.
    const long nchunks = (batch + CH - 1) / CH;
    if ((long)blockIdx.x < nchunks) stage(blockIdx.x);
    pdl_wait_then_release();
    load_weights<kNT>(sw, wt, params);
    copy_swz<kHid, kNT>(sb.w2, wb);
    {  // W3 [in][out] unswizzled: 64 rows of 16 BF16, 2 chunks of 16 bytes each
        const uint4 *s4 = reinterpret_cast<const uint4 *>(wb + kHid * kHid);
        reinterpret_cast<uint4 *>(sb.w3)[threadIdx.x] = __ldg(s4 + threadIdx.x);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float invB = 1.f / (float)batch;
    float *part = partial + (size_t)blockIdx.x * kP;
    float lsum = 0.f;

    // dst (+)= A^T dZ over the chunk's samples: M = inputs (warp w owns rows
    // [16 w, 16 w + 16)), N = outputs (ntiles of 8), K = samples
    auto grad_w = [&](const __nv_bfloat16 *act, const __nv_bfloat16 *dzm, int ldz, float *dst, int ldo, bool acc,
                      auto ntiles_c) {
        constexpr int NJ = decltype(ntiles_c)::value;
        const int m0 = warp * 16;
        float c[NJ][4];
#pragma unroll
        for (int j = 0; j < NJ; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < MT; ++ks) {
            uint32_t a[4];
            frag_at(act, ks * 16, m0, a);
#pragma unroll
            for (int j = 0; j < NJ; j += 2) {
                uint32_t b[4];
                frag_b2(dzm, ldz, ks * 16, j * 8, b);
                mma16816(c[j], a, b[0], b[1]);
                mma16816(c[j + 1], a, b[2], b[3]);
            }
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int col = j * 8 + 2 * t;
            float *d0 = dst + (m0 + g) * ldo + col, *d1 = dst + (m0 + g + 8) * ldo + col;
            float v0 = c[j][0], v1 = c[j][1], v2 = c[j][2], v3 = c[j][3];
            if (acc) { v0 += d0[0]; v1 += d0[1]; v2 += d1[0]; v3 += d1[1]; }
            d0[0] = v0; d0[1] = v1; d1[0] = v2; d1[1] = v3;
        }
    };
    // column sums of a [CH][ld] BF16 matrix into dst (+)= : thread t sums
    // column t % ncol over rows of parity t / ncol (ncol * 2 <= kNT threads),
    // the two halves added in shared memory in a fixed order
    auto col_sums = [&](const __nv_bfloat16 *m, int ld, int ncol, float *dst, bool acc) {
        const int col = threadIdx.x % ncol, half = threadIdx.x / ncol;
        float s = 0.f;
        if (half < 2) {
#pragma unroll
            for (int r = half; r < CH; r += 2) s += __bfloat162float(ld == 64 ? *el(m, r, col) : m[r * ld + col]);
        }
        if (half == 1) red[col] = s;
        __syncthreads();
        if (half == 0) {
            s += red[col];
            dst[col] = acc ? dst[col] + s : s;
        }
        __syncthreads();
    };

#pragma unroll 1
    for (long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const bool acc = chunk != (long)blockIdx.x;
        const long base = first + chunk * CH;  // samples [base, base + CH) of the data set, wrapping
        const long nb = first + batch;
        if (acc) stage(chunk);  // the block's first chunk was staged before the dependency wait
        __syncthreads();
        // forward, and dZ3 = 2 p (d - p.d) / batch with d = p - y
#pragma unroll 1
        for (int mt = warp; mt < MT; mt += kNT / 32) {
            const int row0 = mt * 16;
            uint32_t a[4][4];
            float c[8][4];
            load_a(xs, row0, a);
            layer_fwd<8>(a, sw.w1t, sw.b1, c);
            store_c_bf16(h1, row0, c, true);
            relu_to_a(c, a);
            layer_fwd<8>(a, sw.w2t, sw.b2, c);
            store_c_bf16(h2, row0, c, true);
            relu_to_a(c, a);
            float o[NT][4];
            layer_fwd<NT>(a, sw.w3t, sw.b3, o);
            softmax_rows<NT>(o, K, lps, row0);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                // squared error of p: with d = p - y and s = sum_k p_k d_k (the
                // row's four lanes), dL/dz_k = 2 p_k (d_k - s) / B
                const int r = row0 + g + 8 * h;
                const long i = base + r;
                const bool live = i < nb;
                float dv[2][2], sdot = 0.f;
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int col = j * 8 + 2 * t + e;
                        dv[j][e] = 0.f;
                        if (live && col < K) {
                            const float pv = o[j < NT ? j : 0][2 * h + e];
                            dv[j][e] = pv - ys[r * 16 + col];
                            sdot = fmaf(pv, dv[j][e], sdot);
                            lsum = fmaf(dv[j][e], dv[j][e], lsum);
                        }
                    }
                sdot += __shfl_xor_sync(0xffffffffu, sdot, 1);
                sdot += __shfl_xor_sync(0xffffffffu, sdot, 2);
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int col = j * 8 + 2 * t + e;
                        float d = 0.f;
                        if (live && col < K) {
                            const float pv = o[j < NT ? j : 0][2 * h + e];
                            d = 2.f * pv * (dv[j][e] - sdot) * invB;
                        }
                        dz3[r * 16 + col] = __float2bfloat16_rn(d);
                    }
            }
        }
        __syncthreads();
        // dZ2 = (dZ3 W3^T) * 1[H2 > 0]; W3 [in][out] gives (k, k+1) pairs
#pragma unroll 1
        for (int mt = warp; mt < MT; mt += kNT / 32) {
            const int row0 = mt * 16;
            uint32_t a[4];
            {
                const __nv_bfloat16 *r0 = dz3 + (row0 + g) * 16 + 2 * t;
                const __nv_bfloat16 *r1 = dz3 + (row0 + g + 8) * 16 + 2 * t;
                a[0] = ld32(r0); a[1] = ld32(r1); a[2] = ld32(r0 + 8); a[3] = ld32(r1 + 8);
            }
            float c[8][4];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
                const __nv_bfloat16 *row = sb.w3 + (j * 8 + g) * kOutPad + 2 * t;
                mma16816(c[j], a, ld32(row), ld32(row + 8));
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = j * 8 + 2 * t;
                if (!(__bfloat162float(*el(h2, row0 + g, col)) > 0.f)) c[j][0] = 0.f;
                if (!(__bfloat162float(*el(h2, row0 + g, col + 1)) > 0.f)) c[j][1] = 0.f;
                if (!(__bfloat162float(*el(h2, row0 + g + 8, col)) > 0.f)) c[j][2] = 0.f;
                if (!(__bfloat162float(*el(h2, row0 + g + 8, col + 1)) > 0.f)) c[j][3] = 0.f;
            }
            store_c_bf16(dz, row0, c, false);
        }
        __syncthreads();
        grad_w(h2, dz3, 16, part + kOffW3, kOutPad, acc, std::integral_constant<int, 2>{});
        grad_w(h1, dz, 64, part + kOffW2, kHid, acc, std::integral_constant<int, 8>{});
        col_sums(dz3, 16, kOutPad, part + kOffB3, acc);
        col_sums(dz, 64, kHid, part + kOffB2, acc);
        // dZ1 = (dZ2 W2^T) * 1[H1 > 0], written over H2
#pragma unroll 1
        for (int mt = warp; mt < MT; mt += kNT / 32) {
            const int row0 = mt * 16;
            uint32_t a[4][4];
            load_a(dz, row0, a);
            float c[8][4];
#pragma unroll
            for (int j = 0; j < 8; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    mma16816(c[j], a[ks], wd(sb.w2, j * 8 + g, ks * 8 + t), wd(sb.w2, j * 8 + g, ks * 8 + t + 4));
                }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = j * 8 + 2 * t;
                if (!(__bfloat162float(*el(h1, row0 + g, col)) > 0.f)) c[j][0] = 0.f;
                if (!(__bfloat162float(*el(h1, row0 + g, col + 1)) > 0.f)) c[j][1] = 0.f;
                if (!(__bfloat162float(*el(h1, row0 + g + 8, col)) > 0.f)) c[j][2] = 0.f;
                if (!(__bfloat162float(*el(h1, row0 + g + 8, col + 1)) > 0.f)) c[j][3] = 0.f;
            }
            store_c_bf16(h2, row0, c, false);
        }
        __syncthreads();
        grad_w(xs, h2, 64, part + kOffW1, kHid, acc, std::integral_constant<int, 8>{});
        col_sums(h2, 64, kHid, part + kOffB1, acc);  // ends with a barrier: xs, h1, h2, dz free
    }
    // the block's summed squared error: warp sums, then the four in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) red[warp] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) loss[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
}

// The BF16 copies (forward W^T [out][in], backward W [in][out]) of FP32
// parameter i (biases have none).
__device__ __forceinline__ void refresh_one(int i, float w, __nv_bfloat16 *__restrict__ wt,
                                            __nv_bfloat16 *__restrict__ wb) {
    const __nv_bfloat16 b = __float2bfloat16_rn(w);
    if (i >= kOffW1 && i < kOffB1) {
        const int k = i - kOffW1, in = k / kHid, out = k % kHid;
        wt[out * kIn + in] = b;
    } else if (i >= kOffW2 && i < kOffB2) {
        const int k = i - kOffW2, in = k / kHid, out = k % kHid;
        wt[kHid * kIn + out * kHid + in] = b;
        wb[k] = b;
    } else if (i >= kOffW3 && i < kOffB3) {
        const int k = i - kOffW3, in = k / kOutPad, out = k % kOutPad;
        wt[kHid * kIn + kHid * kHid + out * kHid + in] = b;
        wb[kHid * kHid + k] = b;
    }
}

// Sum the per-block gradients into grad in a fixed order (deterministic):
// a block of 256 threads takes 32 consecutive parameters; warp w sums the
// partials of blocks w, w + 8, w + 16, ... in that order, and the eight warp
// sums are added in warp order.  Then (if lr > 0) one Adam step on the FP32
// master copy and, when wt is not NULL, its BF16 copies.
constexpr int kRedParams = 32, kRedWarps = 8;
__global__ void __launch_bounds__(kRedParams * kRedWarps) k_mlp_reduce_adam(
    const float *__restrict__ partial, int nblk, float *__restrict__ grad, float *__restrict__ params,
    float *__restrict__ m, float *__restrict__ v, int K, float lr, float beta1, float beta2, float eps, float bc1,
    float bc2, __nv_bfloat16 *__restrict__ wt, __nv_bfloat16 *__restrict__ wb) {
    __shared__ float part_sum[kRedWarps][kRedParams];
    pdl_wait_then_release();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * kRedParams + lane;
    float gs = 0.f;
    if (i < kP) {
        // partials in batches of 8 loads in flight, summed in block order
        int b = warp;
        for (; b + 7 * kRedWarps < nblk; b += 8 * kRedWarps) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = partial[(size_t)(b + u * kRedWarps) * kP + i];
#pragma unroll
            for (int u = 0; u < 8; ++u) gs += v[u];
        }
        for (; b < nblk; b += kRedWarps) gs += partial[(size_t)b * kP + i];
    }
    part_sum[warp][lane] = gs;
    __syncthreads();
    if (warp != 0 || i >= kP) return;
    // output columns >= K carry no parameters: no gradient, no update
    const bool unused = (i >= kOffW3 && i < kOffB3 && (i - kOffW3) % kOutPad >= K) || (i >= kOffB3 && i - kOffB3 >= K);
    if (unused) {
        grad[i] = 0.f;
        return;
    }
    float g = 0.f;
#pragma unroll
    for (int w = 0; w < kRedWarps; ++w) g += part_sum[w][lane];
    grad[i] = g;
    if (!(lr > 0.f)) return;
    const float mi = beta1 * m[i] + (1.f - beta1) * g;
    const float vi = beta2 * v[i] + (1.f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float w = params[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    params[i] = w;
    if (wt) refresh_one(i, w, wt, wb);
}

// BF16 copies of the weights in both layouts from the FP32 master copy.
__global__ void k_mlp_refresh(const float *__restrict__ params, __nv_bfloat16 *__restrict__ wt,
                              __nv_bfloat16 *__restrict__ wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kIn * kHid) {  // W1: [in][out] -> wt [out][in]
        const int in = i / kHid, out = i % kHid;
        wt[out * kIn + in] = __float2bfloat16_rn(params[kOffW1 + i]);
    } else if (i < kIn * kHid + kHid * kHid) {
        const int k = i - kIn * kHid, in = k / kHid, out = k % kHid;
        const __nv_bfloat16 w = __float2bfloat16_rn(params[kOffW2 + k]);
        wt[kHid * kIn + out * kHid + in] = w;
        wb[k] = w;
    } else if (i < kIn * kHid + kHid * kHid + kHid * kOutPad) {
        const int k = i - kIn * kHid - kHid * kHid, in = k / kOutPad, out = k % kOutPad;
        const __nv_bfloat16 w = __float2bfloat16_rn(params[kOffW3 + k]);
        wt[kHid * kIn + kHid * kHid + out * kHid + in] = w;
        wb[kHid * kHid + k] = w;
    }
}

// He-uniform initial weights from pcg4d(layer, index, seed, 0), zero biases.
__global__ void k_mlp_init(float *__restrict__ params, uint32_t seed, int K) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kP) return;
    int layer = -1, fan_in = 1, idx = i;
    if (i < kOffB1) { layer = 1; fan_in = kIn; }
    else if (i >= kOffW2 && i < kOffB2) { layer = 2; fan_in = kHid; idx = i - kOffW2; }
    else if (i >= kOffW3 && i < kOffB3) { layer = 3; fan_in = kHid; idx = i - kOffW3; }
    float w = 0.f;
    if (layer > 0) {
        const uint4 h = pcg4d(make_uint4((uint32_t)layer, (uint32_t)idx, seed, 0u));
        const float u = hash_uniform(h.x) * 2.f - 1.f;
        const float lim = sqrtf(6.f / (float)fan_in) * (layer == 1 ? 2.f : 1.f);
        w = u * lim;
        if (layer == 3 && (idx % kOutPad) >= K) w = 0.f;
    }
    params[i] = w;
}

}  // namespace

struct glint_mlp {
    glint_ctx *ctx = nullptr;
    int device = 0;      // ctx->device
    int K = 8;
    long max_batch = 0;
    int max_grid = 0;    // resident training blocks (rows of `partial`)
    int infer_grid = 0;  // resident blocks of the persistent inference kernels
    float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *partial = nullptr, *loss = nullptr;
    __nv_bfloat16 *wt = nullptr, *wb = nullptr;
    long step = 0;
    int last_launches = 0;
};

namespace {

constexpr int kNW = kIn * kHid + kHid * kHid + kHid * kOutPad;  // weights (no biases)

size_t grad_smem() {
    return sizeof(SmemW) + sizeof(SmemWB) + sizeof(__nv_bfloat16) * (4 * kChunk * 64 + kChunk * 16) +
           sizeof(float) * (kNT + kChunk * kLpStride + kChunk * 16);
}

void mlp_free(glint_mlp *g) {
    cudaFree(g->params); cudaFree(g->grad); cudaFree(g->m); cudaFree(g->v);
    cudaFree(g->partial); cudaFree(g->loss); cudaFree(g->wt); cudaFree(g->wb);
}

bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

template <int K>
void launch_features(const ShadeArgs &a, uint4 *x, float *lp, cudaStream_t s) {
    k_mlp_features<K><<<(unsigned)((a.npix + kNT - 1) / kNT), kNT, 0, s>>>(a, x, lp);
}

}  // namespace

cudaError_t glint_launch_mlp_infer(const glint_ctx *ctx, const glint_env *env, const glint_mlp *g,
                                   const glint_gbuffer *smp, float *p_out, cudaStream_t s) {
    glint_params prm{};
    ShadeArgs a = make_args(ctx, env, smp, &prm);
    if (a.npix == 0) return cudaSuccess;
    const long ntiles = (a.npix + kNT - 1) / kNT;
    const unsigned grid = (unsigned)std::min<long>(ntiles, g->infer_grid);
    switch (g->K) {
    case 2: k_mlp_infer<2><<<grid, kNT, 0, s>>>(a, g->wt, g->params, p_out); break;
    case 4: k_mlp_infer<4><<<grid, kNT, 0, s>>>(a, g->wt, g->params, p_out); break;
    case 8: k_mlp_infer<8><<<grid, kNT, 0, s>>>(a, g->wt, g->params, p_out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

namespace {
template <int K, bool INTEGER, bool DEBUG>
cudaError_t launch_shade_mlp(const ShadeArgs &a, const glint_mlp *m, cudaStream_t s) {
    const size_t smem = sizeof(SmemFused);
    cudaError_t e = cudaFuncSetAttribute(k_shade_mlp<K, INTEGER, DEBUG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((a.npix + kFusedNT - 1) / kFusedNT);
    k_shade_mlp<K, INTEGER, DEBUG><<<grid, kFusedNT, smem, s>>>(a, m->wt, m->params);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_shade_mlp_k(const ShadeArgs &a, const glint_mlp *m, bool integer, bool debug, cudaStream_t s) {
    if (integer) return debug ? launch_shade_mlp<K, true, true>(a, m, s) : launch_shade_mlp<K, true, false>(a, m, s);
    return debug ? launch_shade_mlp<K, false, true>(a, m, s) : launch_shade_mlp<K, false, false>(a, m, s);
}
}  // namespace

cudaError_t glint_launch_shade_mlp(const glint_ctx *ctx, const glint_env *env, const glint_gbuffer *g,
                                   const glint_params *p, float *out, const glint_debug *dbg, cudaStream_t s) {
    ShadeArgs a = make_args(ctx, env, g, p);
    a.out = reinterpret_cast<float4 *>(out);
    a.dbg = dbg ? *dbg : glint_debug{};
    if (a.npix == 0) return cudaSuccess;
    const bool integer = p->count_mode == GLINT_COUNT_INTEGER, debug = dbg != nullptr;
    switch (p->mlp->K) {
    case 2: return launch_shade_mlp_k<2>(a, p->mlp, integer, debug, s);
    case 4: return launch_shade_mlp_k<4>(a, p->mlp, integer, debug, s);
    case 8: return launch_shade_mlp_k<8>(a, p->mlp, integer, debug, s);
    default: return cudaErrorInvalidValue;
    }
}

namespace {
template <int K>
cudaError_t launch_serve_mlp_k(int num_sms, const ShadeArgs *frames, const ServeItem *items, int nitems,
                               cudaStream_t s) {
    static int per_sm = 0;  // resident blocks per SM
    const size_t smem = sizeof(SmemServeFused);
    if (!per_sm) {
        cudaError_t e = cudaFuncSetAttribute(k_serve_mlp<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve_mlp<K>, kFusedNT, smem);
        if (e != cudaSuccess) return e;
        per_sm = std::max(per_sm, 1);
    }
    const int grid = std::min(nitems, per_sm * num_sms);
    k_serve_mlp<K><<<grid, kFusedNT, smem, s>>>(frames, items, nitems);
    return cudaGetLastError();
}
}  // namespace

cudaError_t glint_launch_serve_mlp(int K, int num_sms, const ShadeArgs *frames, const ServeItem *items, int nitems,
                                   cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    switch (K) {
    case 2: return launch_serve_mlp_k<2>(num_sms, frames, items, nitems, s);
    case 4: return launch_serve_mlp_k<4>(num_sms, frames, items, nitems, s);
    case 8: return launch_serve_mlp_k<8>(num_sms, frames, items, nitems, s);
    default: return cudaErrorInvalidValue;
    }
}

void glint_mlp_weights(const glint_mlp *g, const void **wt, const float **params) {
    *wt = g->wt;
    *params = g->params;
}

int glint_mlp_k(const glint_mlp *g) { return g ? g->K : 0; }
int glint_mlp_device(const glint_mlp *g) { return g ? g->device : -1; }

namespace {
// A launch whose blocks may start while the stream's previous kernel runs
// (pdl: the kernel waits on it with pdl_wait_then_release), or an ordinary one.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                       cudaStream_t s, Args... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace

extern "C" {

int glint_mlp_param_count(void) { return kP; }

glint_status glint_mlp_create(glint_ctx *ctx, int K, long max_batch, uint32_t seed, glint_mlp **out) {
    set_error("%s", "");
    if (!ctx || !out) { set_error("glint_mlp_create: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    *out = nullptr;
    if (K != 2 && K != 4 && K != 8) {
        set_error("glint_mlp_create: K = %d; the surrogate's 64 inputs hold 6K + 3 features, so K is 2, 4 or 8", K);
        return K == 16 ? GLINT_ERR_UNSUPPORTED : GLINT_ERR_INVALID_ARG;
    }
    if (max_batch < 1 || max_batch > (1L << 30)) {
        set_error("glint_mlp_create: max_batch %ld outside [1, 2^30]", max_batch);
        return GLINT_ERR_INVALID_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) { set_error("glint_mlp_create: cannot select device"); return GLINT_ERR_CUDA; }
    glint_mlp *g = new glint_mlp();
    g->ctx = ctx;
    g->device = ctx->device;
    g->K = K;
    g->max_batch = max_batch;
    glint_status st = GLINT_OK;
    const size_t smem = grad_smem();
    st = cuda_status(cudaFuncSetAttribute(k_mlp_grad<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                     "glint_mlp_create: smem");
    int per_sm = 0, per_sm_inf = 0, per_sm_fwd = 0;
    if (st == GLINT_OK)
        st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_grad<1>, kNT, smem),
                         "glint_mlp_create: occupancy");
    if (st == GLINT_OK) {
        cudaError_t e = K == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_inf, k_mlp_infer<2>, kNT, 0)
                      : K == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_inf, k_mlp_infer<4>, kNT, 0)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_inf, k_mlp_infer<8>, kNT, 0);
        st = cuda_status(e, "glint_mlp_create: occupancy");
    }
    if (st == GLINT_OK)
        st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_fwd, k_mlp_forward<1>, kNT, 0),
                         "glint_mlp_create: occupancy");
    if (st == GLINT_OK && (per_sm < 1 || per_sm_inf < 1 || per_sm_fwd < 1)) {
        set_error("glint_mlp_create: a surrogate kernel does not fit an SM");
        st = GLINT_ERR_UNSUPPORTED;
    }
    const long nchunks_max = (max_batch + kChunk - 1) / kChunk;
    g->max_grid = (int)std::min<long>((long)per_sm * ctx->num_sms, nchunks_max);
    g->infer_grid = std::max(1, std::min(per_sm_inf, per_sm_fwd) * ctx->num_sms);
    auto alloc = [&](void **p, size_t bytes) {
        if (st == GLINT_OK) st = cuda_status(cudaMalloc(p, bytes), "glint_mlp_create");
    };
    alloc((void **)&g->params, sizeof(float) * kP);
    alloc((void **)&g->grad, sizeof(float) * kP);
    alloc((void **)&g->m, sizeof(float) * kP);
    alloc((void **)&g->v, sizeof(float) * kP);
    alloc((void **)&g->partial, sizeof(float) * kP * (size_t)std::max(g->max_grid, 1));
    alloc((void **)&g->loss, sizeof(float) * (size_t)std::max(g->max_grid, 1));
    alloc((void **)&g->wt, sizeof(__nv_bfloat16) * kNW);
    alloc((void **)&g->wb, sizeof(__nv_bfloat16) * (kHid * kHid + kHid * kOutPad));
    if (st == GLINT_OK) st = cuda_status(cudaMemset(g->m, 0, sizeof(float) * kP), "glint_mlp_create");
    if (st == GLINT_OK) st = cuda_status(cudaMemset(g->v, 0, sizeof(float) * kP), "glint_mlp_create");
    if (st == GLINT_OK) st = cuda_status(cudaMemset(g->grad, 0, sizeof(float) * kP), "glint_mlp_create");
    if (st == GLINT_OK) {
        k_mlp_init<<<(kP + 255) / 256, 256>>>(g->params, seed, K);
        k_mlp_refresh<<<(kNW + 255) / 256, 256>>>(g->params, g->wt, g->wb);
        st = cuda_status(cudaDeviceSynchronize(), "glint_mlp_create: init");
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (st != GLINT_OK) { mlp_free(g); delete g; return st; }
    *out = g;
    return GLINT_OK;
}

void glint_mlp_destroy(glint_mlp *g) {
    if (!g) return;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != g->device && cudaSetDevice(g->device) != cudaSuccess) cudaGetLastError();
    mlp_free(g);
    if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
    delete g;
}

glint_status glint_mlp_set_params(glint_mlp *g, const float *host, long n) {
    set_error("%s", "");
    if (!g || !host || n != kP) { set_error("glint_mlp_set_params: need %d floats", kP); return GLINT_ERR_INVALID_ARG; }
    glint_status st = cuda_status(cudaMemcpy(g->params, host, sizeof(float) * kP, cudaMemcpyHostToDevice),
                                  "glint_mlp_set_params");
    if (st != GLINT_OK) return st;
    k_mlp_refresh<<<(kNW + 255) / 256, 256>>>(g->params, g->wt, g->wb);
    return cuda_status(cudaDeviceSynchronize(), "glint_mlp_set_params");
}

glint_status glint_mlp_export(const glint_mlp *g, int item, float *host, long n) {
    set_error("%s", "");
    if (!g || !host) { set_error("glint_mlp_export: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    const float *src = item == GLINT_MLP_PARAMS ? g->params : item == GLINT_MLP_GRAD ? g->grad
                     : item == GLINT_MLP_ADAM_M ? g->m : item == GLINT_MLP_ADAM_V ? g->v : nullptr;
    if (!src || n != kP) { set_error("glint_mlp_export: item %d, need %d floats", item, kP); return GLINT_ERR_INVALID_ARG; }
    return cuda_status(cudaMemcpy(host, src, sizeof(float) * kP, cudaMemcpyDeviceToHost), "glint_mlp_export");
}

glint_status glint_mlp_import_state(glint_mlp *g, const float *params, const float *m, const float *v, long n,
                                    long step) {
    set_error("%s", "");
    if (!g || !params || !m || !v || n != kP || step < 0) {
        set_error("glint_mlp_import_state: need %d floats of each and step >= 0", kP);
        return GLINT_ERR_INVALID_ARG;
    }
    glint_status st = cuda_status(cudaMemcpy(g->m, m, sizeof(float) * kP, cudaMemcpyHostToDevice), "glint_mlp_import_state");
    if (st == GLINT_OK) st = cuda_status(cudaMemcpy(g->v, v, sizeof(float) * kP, cudaMemcpyHostToDevice), "glint_mlp_import_state");
    if (st != GLINT_OK) return st;
    g->step = step;
    return glint_mlp_set_params(g, params, kP);
}

long glint_mlp_step(const glint_mlp *g) { return g ? g->step : -1; }

glint_status glint_mlp_features(glint_ctx *ctx, const glint_env *env, const glint_gbuffer *gb, uint16_t *x_out,
                                float *lp_out, void *stream) {
    set_error("%s", "");
    if (!ctx || !env || !gb) { set_error("glint_mlp_features: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    if (env->ctx != ctx) { set_error("glint_mlp_features: environment belongs to another context"); return GLINT_ERR_INVALID_ARG; }
    if (env->d.K != 2 && env->d.K != 4 && env->d.K != 8) {
        set_error("glint_mlp_features: environment K = %d (the surrogate takes K = 2, 4 or 8)", env->d.K);
        return GLINT_ERR_UNSUPPORTED;
    }
    if (gb->width < 0 || gb->height < 0 || (long)gb->width * gb->height > (1L << 31)) {
        set_error("glint_mlp_features: width %d x height %d out of range", gb->width, gb->height);
        return GLINT_ERR_INVALID_ARG;
    }
    const long n = (long)gb->width * gb->height;
    if (n == 0) return GLINT_OK;
    if (!gb->view_n0 || !gb->normal_f0 || !gb->uv_alpha || !gb->tangent || !x_out || !lp_out) {
        set_error("glint_mlp_features: the view, normal, uv/alpha and tangent planes and both outputs are required");
        return GLINT_ERR_INVALID_ARG;
    }
    if (!aligned(gb->view_n0, 16) || !aligned(gb->normal_f0, 16) || !aligned(gb->uv_alpha, 16) ||
        !aligned(gb->tangent, 16) || !aligned(x_out, 16) || !aligned(lp_out, 4)) {
        set_error("glint_mlp_features: planes and x_out must be 16-byte aligned, lp_out 4-byte aligned");
        return GLINT_ERR_INVALID_ARG;
    }
    glint_params prm{};
    const ShadeArgs a = make_args(ctx, env, gb, &prm);
    cudaStream_t s = (cudaStream_t)stream;
    uint4 *x = reinterpret_cast<uint4 *>(x_out);
    switch (env->d.K) {
    case 2: launch_features<2>(a, x, lp_out, s); break;
    case 4: launch_features<4>(a, x, lp_out, s); break;
    default: launch_features<8>(a, x, lp_out, s); break;
    }
    ctx->last_launches = 1;
    return cuda_status(cudaGetLastError(), "glint_mlp_features");
}

glint_status glint_mlp_forward(const glint_mlp *g, const uint16_t *x, const float *lp, long n, float *p_out,
                               void *stream) {
    set_error("%s", "");
    if (!g || n < 0) { set_error("glint_mlp_forward: NULL network or n < 0"); return GLINT_ERR_INVALID_ARG; }
    if (n == 0) return GLINT_OK;
    if (!x || !lp || !p_out || !aligned(x, 16) || !aligned(lp, 4) || !aligned(p_out, 4)) {
        set_error("glint_mlp_forward: x (16-byte aligned), lp and p_out are required");
        return GLINT_ERR_INVALID_ARG;
    }
    const long ntiles = (n + kNT - 1) / kNT;
    const unsigned grid = (unsigned)std::min<long>(ntiles, g->infer_grid);
    k_mlp_forward<1><<<grid, kNT, 0, (cudaStream_t)stream>>>(reinterpret_cast<const uint4 *>(x), lp, n, g->K, g->wt,
                                                             g->params, p_out);
    const_cast<glint_mlp *>(g)->last_launches = 1;
    return cuda_status(cudaGetLastError(), "glint_mlp_forward");
}

namespace {
// One optimisation step (two launches): the per-block gradients, then their
// sum in block order with the Adam update of the FP32 parameters and of their
// BF16 copies.  *grid_out receives the number of gradient blocks.  after_step:
// the stream's previous kernel is this network's Adam update (the gradient
// kernel may then start during it; it never writes the training data).
cudaError_t enqueue_step(glint_mlp *g, const uint16_t *x, const float *lp, const float *targets, long n_total,
                         long first, long batch, float lr, cudaStream_t s, bool after_step,
                         int *grid_out = nullptr) {
    const long nchunks = (batch + kChunk - 1) / kChunk;
    const int grid = (int)std::min<long>(nchunks, g->max_grid);
    if (grid_out) *grid_out = grid;
    cudaError_t e = launch_pdl(after_step, k_mlp_grad<1>, grid, kNT, grad_smem(), s,
                               reinterpret_cast<const uint4 *>(x), lp, targets, n_total, first % n_total, batch, g->K,
                               (const __nv_bfloat16 *)g->wt, (const __nv_bfloat16 *)g->wb, (const float *)g->params,
                               g->partial, g->loss);
    const long t = lr > 0.f ? g->step + 1 : std::max(g->step, 1L);
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)t));
    const float bc2 = (float)(1.0 - std::pow(0.999, (double)t));
    if (e != cudaSuccess) return e;
    e = launch_pdl(true, k_mlp_reduce_adam, (kP + kRedParams - 1) / kRedParams, kRedParams * kRedWarps, 0, s,
                   (const float *)g->partial, grid, g->grad, g->params, g->m, g->v, g->K, lr, 0.9f, 0.999f, 1e-8f,
                   bc1, bc2, g->wt, g->wb);
    if (e == cudaSuccess && lr > 0.f) g->step = t;
    return e;
}
}  // namespace

glint_status glint_mlp_train(glint_mlp *g, const uint16_t *x, const float *lp, const float *targets, long n_total,
                             long first, long batch, long steps, float lr_max, float lr_min, void *stream) {
    set_error("%s", "");
    if (!g || !x || !lp || !targets) { set_error("glint_mlp_train: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    if (batch < 1 || batch > g->max_batch || n_total < 1 || first < 0 || steps < 0 || !(lr_max > 0.f) ||
        !(lr_max < 1.f) || !(lr_min > 0.f) || !(lr_min <= lr_max)) {
        set_error("glint_mlp_train: batch %ld outside [1, %ld], empty data, first or steps < 0, or not "
                  "0 < lr_min <= lr_max < 1", batch, g->max_batch);
        return GLINT_ERR_INVALID_ARG;
    }
    if (!aligned(x, 16) || !aligned(lp, 4) || !aligned(targets, 4)) {
        set_error("glint_mlp_train: x must be 16-byte aligned, lp and targets 4-byte aligned");
        return GLINT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    long i = 0;
    for (; i < steps && e == cudaSuccess; ++i) {
        const double cosine = 0.5 * (1.0 + std::cos(3.14159265358979323846 * (double)i / (double)steps));
        const float lr = (float)std::max((double)lr_max * cosine, (double)lr_min);
        e = enqueue_step(g, x, lp, targets, n_total, (first + i * batch) % n_total, batch, lr, s, i > 0);
    }
    g->last_launches = (int)std::min<long>(2 * i, 1L << 30);
    if (e != cudaSuccess) return cuda_status(e, "glint_mlp_train");
    return cuda_status(cudaGetLastError(), "glint_mlp_train");
}

glint_status glint_mlp_train_step(glint_mlp *g, const uint16_t *x, const float *lp, const float *targets,
                                  long n_total, long first, long batch, float lr, float *loss_out, void *stream) {
    set_error("%s", "");
    if (!g || !x || !lp || !targets) { set_error("glint_mlp_train_step: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    if (batch < 1 || batch > g->max_batch || n_total < 1 || first < 0 || !(lr >= 0.f) || !(lr < 1.f)) {
        set_error("glint_mlp_train_step: batch %ld outside [1, %ld], empty data, first < 0 or lr %g outside [0, 1)",
                  batch, g->max_batch, (double)lr);
        return GLINT_ERR_INVALID_ARG;
    }
    if (!aligned(x, 16) || !aligned(lp, 4) || !aligned(targets, 4)) {
        set_error("glint_mlp_train_step: x must be 16-byte aligned, lp and targets 4-byte aligned");
        return GLINT_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int grid = 0;
    const cudaError_t e = enqueue_step(g, x, lp, targets, n_total, first, batch, lr, s, false, &grid);
    g->last_launches = 2;
    glint_status st = cuda_status(e != cudaSuccess ? e : cudaGetLastError(), "glint_mlp_train_step");
    if (st != GLINT_OK || !loss_out) return st;
    std::vector<float> l(grid);
    st = cuda_status(cudaMemcpyAsync(l.data(), g->loss, sizeof(float) * grid, cudaMemcpyDeviceToHost, s),
                     "glint_mlp_train_step: loss");
    if (st == GLINT_OK) st = cuda_status(cudaStreamSynchronize(s), "glint_mlp_train_step: loss");
    double acc = 0.0;
    for (float v : l) acc += v;
    *loss_out = (float)(acc / (double)batch);
    return st;
}

glint_status glint_mlp_infer(const glint_mlp *g, glint_ctx *ctx, const glint_env *env, const glint_gbuffer *gb,
                             float *p_out, void *stream) {
    set_error("%s", "");
    if (!g || !ctx || !env || !gb) { set_error("glint_mlp_infer: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    if (env->ctx != ctx || g->ctx != ctx) { set_error("glint_mlp_infer: network, environment and context differ"); return GLINT_ERR_INVALID_ARG; }
    if (env->d.K != g->K) { set_error("glint_mlp_infer: network K %d, environment K %d", g->K, env->d.K); return GLINT_ERR_INVALID_ARG; }
    if (gb->width < 0 || gb->height < 0 || (long)gb->width * gb->height > (1L << 31)) {
        set_error("glint_mlp_infer: width %d x height %d out of range", gb->width, gb->height);
        return GLINT_ERR_INVALID_ARG;
    }
    const long n = (long)gb->width * gb->height;
    if (n == 0) return GLINT_OK;
    if (!gb->view_n0 || !gb->normal_f0 || !gb->uv_alpha || !gb->tangent || !p_out) {
        set_error("glint_mlp_infer: the view, normal, uv/alpha and tangent planes and p_out are required");
        return GLINT_ERR_INVALID_ARG;
    }
    if (!aligned(gb->view_n0, 16) || !aligned(gb->normal_f0, 16) || !aligned(gb->uv_alpha, 16) ||
        !aligned(gb->tangent, 16) || !aligned(p_out, 4)) {
        set_error("glint_mlp_infer: planes must be 16-byte aligned, p_out 4-byte aligned");
        return GLINT_ERR_INVALID_ARG;
    }
    glint_status st = cuda_status(glint_launch_mlp_infer(ctx, env, g, gb, p_out, (cudaStream_t)stream),
                                  "glint_mlp_infer");
    const_cast<glint_mlp *>(g)->last_launches = 1;
    return st;
}

int glint_mlp_get_k(const glint_mlp *g) { return g ? g->K : 0; }
int glint_mlp_last_launches(const glint_mlp *g) { return g ? g->last_launches : 0; }

static bool little_endian() {
    const uint32_t one = 1;
    unsigned char b;
    memcpy(&b, &one, 1);
    return b == 1;
}

glint_status glint_mlp_save(const glint_mlp *g, const char *path) {
    set_error("%s", "");
    if (!g || !path) { set_error("glint_mlp_save: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    if (!little_endian()) { set_error("glint_mlp_save: big-endian host"); return GLINT_ERR_UNSUPPORTED; }
    std::vector<float> buf(3 * (size_t)kP);
    glint_status st = glint_mlp_export(g, GLINT_MLP_PARAMS, buf.data(), kP);
    if (st == GLINT_OK) st = glint_mlp_export(g, GLINT_MLP_ADAM_M, buf.data() + kP, kP);
    if (st == GLINT_OK) st = glint_mlp_export(g, GLINT_MLP_ADAM_V, buf.data() + 2 * kP, kP);
    if (st != GLINT_OK) return st;
    FILE *f = fopen(path, "wb");
    if (!f) { set_error("glint_mlp_save: cannot open %s", path); return GLINT_ERR_INVALID_ARG; }
    char head[256];
    const int n = snprintf(head, sizeof(head),
                           "{\"format\": \"glint_mlp\", \"version\": 1, \"K\": %d, \"params\": %d, \"step\": %ld, "
                           "\"arrays\": [\"params\", \"adam_m\", \"adam_v\"], \"dtype\": \"float32-le\"}\n",
                           g->K, kP, g->step);
    const bool ok = fwrite(head, 1, (size_t)n, f) == (size_t)n && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    if (fclose(f) != 0 || !ok) { set_error("glint_mlp_save: write to %s failed", path); return GLINT_ERR_INVALID_ARG; }
    return GLINT_OK;
}

glint_status glint_mlp_load(glint_ctx *ctx, const char *path, long max_batch, glint_mlp **out) {
    set_error("%s", "");
    if (!ctx || !path || !out) { set_error("glint_mlp_load: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!little_endian()) { set_error("glint_mlp_load: big-endian host"); return GLINT_ERR_UNSUPPORTED; }
    FILE *f = fopen(path, "rb");
    if (!f) { set_error("glint_mlp_load: cannot open %s", path); return GLINT_ERR_INVALID_ARG; }
    char head[512] = {0};
    if (!fgets(head, sizeof(head), f)) { fclose(f); set_error("glint_mlp_load: empty file"); return GLINT_ERR_INVALID_ARG; }
    int K = 0, np = 0, ver = 0;
    long step = -1;
    const char *pk = strstr(head, "\"K\":"), *pp = strstr(head, "\"params\":"), *ps = strstr(head, "\"step\":"),
               *pv = strstr(head, "\"version\":");
    if (!strstr(head, "\"format\": \"glint_mlp\"") || !pk || !pp || !ps || !pv || sscanf(pk + 4, "%d", &K) != 1 ||
        sscanf(pp + 9, "%d", &np) != 1 || sscanf(ps + 7, "%ld", &step) != 1 || sscanf(pv + 10, "%d", &ver) != 1 ||
        ver != 1 || np != kP || step < 0) {
        fclose(f);
        set_error("glint_mlp_load: %s is not a version-1 glint_mlp file with %d parameters", path, kP);
        return GLINT_ERR_INVALID_ARG;
    }
    std::vector<float> buf(3 * (size_t)kP);
    const bool ok = fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    if (!ok) { set_error("glint_mlp_load: %s is truncated", path); return GLINT_ERR_INVALID_ARG; }
    glint_mlp *g = nullptr;
    glint_status st = glint_mlp_create(ctx, K, max_batch, 0u, &g);
    if (st != GLINT_OK) return st;
    st = glint_mlp_import_state(g, buf.data(), buf.data() + kP, buf.data() + 2 * kP, kP, step);
    if (st != GLINT_OK) { glint_mlp_destroy(g); return st; }
    *out = g;
    return GLINT_OK;
}

glint_status glint_mlp_generate(glint_ctx *ctx, const glint_env *env, const glint_gbuffer *gbuf, int e2_samples,
                                uint16_t *x_out, float *lp_out, float *targets_out, void *stream) {
    glint_status st = glint_mlp_features(ctx, env, gbuf, x_out, lp_out, stream);
    if (st != GLINT_OK) return st;
    glint_params p{};
    p.evaluator = GLINT_EVAL_E2;
    p.e2_samples = e2_samples;
    st = glint_reflect_probs(ctx, env, gbuf, &p, targets_out, stream);
    ctx->last_launches = 2;
    return st;
}

}  // extern "C"
