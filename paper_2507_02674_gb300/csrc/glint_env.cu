// Per-environment preprocessing: radiance levels, fuzzy weights, pyramid and
// filtered maps (Sec. 4 "Discrete Radiance Levels", "Fuzzy Indicator
// Functions", Eq. wkdefpractice, "Integrated NDF" Eq. rtiblndf; Sec. 3.4
// Eq. rtibl).
//
// Data layout in HBM.  Pyramid: per level, the texels' colour (R, G, B, 0),
// one float4 each, then their weights w_1..w_K, Cpad/4 - 1 float4 each
// (Cpad = 4 ceil((3+K)/4); 32 bytes at K = 8, read with one 256-bit load);
// levels concatenated.  Filtered maps: R levels of W_r/2 x W_r texels, each
// texel the record (R, G, B, w_1..w_K, 0 padding) of Cpad floats (or an fp32
// colour and K codes for a compressed format), levels concatenated; beside
// them a weights-only copy (Cpad/4 - 1 float4 a texel, the weights as stored).
// Brightness min/max go through a small per-block scratch array and a
// finished-block counter.
#include <stdio.h>

#include "glint_internal.cuh"

using namespace glint;

namespace {

constexpr int kNT = 256;

__device__ __forceinline__ float4 load_texel(const void *texels, int fmt, long i) {
    if (fmt == GLINT_FMT_RGBA16F) {
        const uint2 raw = __ldg(reinterpret_cast<const uint2 *>(texels) + i);
        const __half2 rg = *reinterpret_cast<const __half2 *>(&raw.x);
        const __half2 ba = *reinterpret_cast<const __half2 *>(&raw.y);
        const float2 f0 = __half22float2(rg), f1 = __half22float2(ba);
        return make_float4(f0.x, f0.y, f1.x, f1.y);
    }
    return __ldg(reinterpret_cast<const float4 *>(texels) + i);
}

// Rec. 709 luminance of scaled radiance, clamped at 0.
__device__ __forceinline__ float brightness(float4 t, float scale) {
    float y = 0.2126f * (t.x * scale) + 0.7152f * (t.y * scale) + 0.0722f * (t.z * scale);
    return fmaxf(y, 0.f);
}

// Step 2 from the per-block (min, max) pairs: lo = max(min Y, ell),
// hi = max(max Y, lo); L_1 = 0, L_k = lo (hi/lo)^((k-1)/(K-1)) =
// exp(lerp(ln lo, ln hi, (k-1)/(K-1))).  Run by one block.
__device__ void levels_from_partials(const float2 *partial, int nblk, int K, float ell, float *levels) {
    float lo = INFINITY, hi = -INFINITY;
    for (int i = threadIdx.x; i < nblk; i += kNT) {
        const float2 v = __ldcg(partial + i);  // written by other blocks: read from L2
        lo = fminf(lo, v.x);
        hi = fmaxf(hi, v.y);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __shared__ float2 red[kNT / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_float2(lo, hi);
    __syncthreads();
    if (threadIdx.x == 0) {
        float mn = red[0].x, mx = red[0].y;
        for (int w = 1; w < kNT / 32; ++w) {
            mn = fminf(mn, red[w].x);
            mx = fmaxf(mx, red[w].y);
        }
        lo = fmaxf(mn, ell);
        hi = fmaxf(mx, lo);
        const float l2 = log2f(hi / lo);
        levels[0] = 0.f;
        for (int k = 2; k <= K; ++k) {
            const float a = (float)(k - 1) / (float)(K - 1);
            levels[k - 1] = lo * exp2f(a * l2);
        }
        levels[K] = lo;
        levels[K + 1] = hi;
    }
}

// Steps 1 and 2: per-block min / max of the brightness into the scratch
// array; the last block to finish (counted in *done, which it resets) turns
// the pairs into the levels.
__global__ void __launch_bounds__(kNT) k_minmax(const void *__restrict__ texels, int fmt, long n, float scale,
                                                  float2 *__restrict__ partial, unsigned *__restrict__ done, int K,
                                                  float ell, float *__restrict__ levels) {
    float lo = INFINITY, hi = -INFINITY;
    for (long i = (long)blockIdx.x * kNT + threadIdx.x; i < n; i += (long)gridDim.x * kNT) {
        const float y = brightness(load_texel(texels, fmt, i), scale);
        lo = fminf(lo, y);
        hi = fmaxf(hi, y);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __shared__ float2 red[kNT / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_float2(lo, hi);
    __syncthreads();
    if (threadIdx.x < 32) {
        float2 v = threadIdx.x < kNT / 32 ? red[threadIdx.x] : make_float2(INFINITY, -INFINITY);
        for (int o = 16; o > 0; o >>= 1) {
            v.x = fminf(v.x, __shfl_xor_sync(0xffffffffu, v.x, o));
            v.y = fmaxf(v.y, __shfl_xor_sync(0xffffffffu, v.y, o));
        }
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();  // this block's pair is visible before it is counted
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    levels_from_partials(partial, gridDim.x, K, ell, levels);
    if (threadIdx.x == 0) *done = 0u;
}

// Channel vector of one texel in the pyramid's slot order (R, G, B, 0,
// w_1 .. w_K, 0 padding; Cpad floats): the fuzzy weights of the two levels
// bracketing its brightness (Eq. wkdefpractice).
__device__ __forceinline__ void texel_channels(float4 t, float scale, int K, const float *L, int Cpad, bool log_w,
                                               float *v) {
    const float R = t.x * scale, G = t.y * scale, B = t.z * scale;
    const float Y = fmaxf(0.2126f * R + 0.7152f * G + 0.0722f * B, 0.f);
    // bracket: largest j in [0, K-2] with L[j] <= Y; Y >= L[K-1] -> w_K = 1
    int j = 0;
    for (int k = 1; k < K - 1; ++k)
        if (L[k] <= Y) j = k;
    const bool top = Y >= L[K - 1];
    // log space (optional, Sec. 7): between L_j > 0 and L_{j+1}; linear below L_2 (L_1 = 0)
    const float tt = (log_w && j > 0) ? (logf(Y) - logf(L[j])) / (logf(L[j + 1]) - logf(L[j]))
                                      : (Y - L[j]) / (L[j + 1] - L[j]);
    v[0] = R; v[1] = G; v[2] = B; v[3] = 0.f;
    for (int c = 4; c < Cpad; ++c) {
        const int k = c - 4;
        float val = 0.f;
        if (k < K) {
            if (top) val = (k == K - 1) ? 1.f : 0.f;
            else if (k == j) val = 1.f - tt;
            else if (k == j + 1) val = tt;
        }
        v[c] = val;
    }
}

// Slot c of texel i of a pyramid level (float4 units of the split storage):
// slot 0 is the colour (R, G, B, 0) at rgb4 + i, slots 1 .. C4-1 the weights
// at w4 + i (C4 - 1) + c - 1.
template <int C4>
__device__ __forceinline__ size_t pyr_slot(size_t rgb4, size_t w4, size_t i, int c) {
    return c == 0 ? rgb4 + i : w4 + i * (C4 - 1) + (c - 1);
}

// Steps 3 and 4: pyramid.  Each block takes a T x T tile of pyramid level m
// (T <= 32, a power of two), writes it (for m = 0 computing the channels of the
// texels first) and reduces it through log2 T further levels in shared memory,
// writing each.  A texel of level l+1 is the solid-angle weighted mean of its
// 2 x 2 children; the weight of a row spanning [theta0, theta1] is
// cos theta0 - cos theta1 = 2 sin(mid) sin(half), written as a product to stay
// accurate near the poles.  With tail_to > m + nlev the last block to finish
// (counted in *done, which it resets) builds levels m + nlev + 1 .. tail_to
// from level m + nlev, which every block has written by then.
template <bool FROM_TEXELS, int C4>
__global__ void __launch_bounds__(kNT) k_pyramid(const void *__restrict__ texels, int fmt, float scale, int K,
                                                   const float *__restrict__ levels, float4 *__restrict__ pyr,
                                                   const size_t *__restrict__ rgb4, const size_t *__restrict__ w4,
                                                   int m, int Ws, int Hs, int T, int nlev, int log_w, int tail_to,
                                                   unsigned *__restrict__ done) {
    constexpr int Cpad = 4 * C4;
    extern __shared__ float4 smem4[];
    float4 *bufA = smem4;                        // T*T texels of C4 float4
    float4 *bufB = smem4 + (size_t)T * T * C4;   // (T/2)^2 texels
    __shared__ float L[GLINT_MAX_K];
    __shared__ float4 rw[16];  // per row of the level being built: w0, w1, 1 / (2 (w0 + w1))
    if (FROM_TEXELS) {
        if (threadIdx.x < K) L[threadIdx.x] = levels[threadIdx.x];
        __syncthreads();
    }
    // T is a power of two (2^nlev): tile coordinates by shifts and masks
    const int tiles_x = Ws >> nlev;
    const int tx0 = ((int)blockIdx.x & (tiles_x - 1)) << nlev, ty0 = ((int)blockIdx.x / tiles_x) << nlev;
    for (int i = threadIdx.x; i < T * T; i += kNT) {
        const int lx = i & (T - 1), ly = i >> nlev;
        const size_t gi = (size_t)(ty0 + ly) * Ws + (tx0 + lx);
        float4 *v = bufA + (size_t)i * C4;
        if (FROM_TEXELS) {
            float tmp[3 + GLINT_MAX_K + 1];
            texel_channels(load_texel(texels, fmt, (long)gi), scale, K, L, Cpad, log_w != 0, tmp);
#pragma unroll
            for (int c = 0; c < C4; ++c) {
                v[c] = make_float4(tmp[4 * c], tmp[4 * c + 1], tmp[4 * c + 2], tmp[4 * c + 3]);
                pyr[pyr_slot<C4>(rgb4[0], w4[0], gi, c)] = v[c];
            }
        } else {
#pragma unroll
            for (int c = 0; c < C4; ++c) v[c] = __ldcg(pyr + pyr_slot<C4>(rgb4[m], w4[m], gi, c));
        }
    }
    __syncthreads();
    int cur = T;
    for (int l = 1; l <= nlev; ++l) {
        const int nxt = cur / 2, lg = nlev - l;  // nxt = 2^lg
        const int Hp = Hs >> (l - 1), Wd = Ws >> l;  // parent height, level width
        const float half = 0.5f * kPi / (float)Hp;
        const int X0 = tx0 >> l, Y0 = ty0 >> l;
        if (threadIdx.x < nxt) {
            const int Y = Y0 + threadIdx.x;
            const float w0 = sinf((2.f * Y + 0.5f) * (kPi / (float)Hp)) * sinf(half);
            const float w1 = sinf((2.f * Y + 1.5f) * (kPi / (float)Hp)) * sinf(half);
            rw[threadIdx.x] = make_float4(w0, w1, 1.f / (2.f * (w0 + w1)), 0.f);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nxt * nxt * C4; i += kNT) {
            const int c = i % C4, t = i / C4;  // C4 is a constant: no division
            const int x = t & (nxt - 1), y = t >> lg;
            const float4 wr = rw[y];
            const float w0 = wr.x, w1 = wr.y, inv = wr.z;
            const float4 a0 = bufA[((2 * y) * cur + 2 * x) * C4 + c];
            const float4 a1 = bufA[((2 * y) * cur + 2 * x + 1) * C4 + c];
            const float4 b0 = bufA[((2 * y + 1) * cur + 2 * x) * C4 + c];
            const float4 b1 = bufA[((2 * y + 1) * cur + 2 * x + 1) * C4 + c];
            float4 r;
            r.x = (w0 * (a0.x + a1.x) + w1 * (b0.x + b1.x)) * inv;
            r.y = (w0 * (a0.y + a1.y) + w1 * (b0.y + b1.y)) * inv;
            r.z = (w0 * (a0.z + a1.z) + w1 * (b0.z + b1.z)) * inv;
            r.w = (w0 * (a0.w + a1.w) + w1 * (b0.w + b1.w)) * inv;
            bufB[t * C4 + c] = r;
            pyr[pyr_slot<C4>(rgb4[m + l], w4[m + l], (size_t)(Y0 + y) * Wd + X0 + x, c)] = r;
        }
        __syncthreads();  // (also: every store of the level issued before the block is counted as done)
        float4 *tmp = bufA;
        bufA = bufB;
        bufB = tmp;
        cur = nxt;
    }
    if (tail_to <= m + nlev) return;
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();  // this block's levels are visible before it is counted
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    int Wc = Ws >> nlev, Hc = Hs >> nlev;  // level m + nlev, the parent of the first tail level
    for (int l = m + nlev + 1; l <= tail_to; ++l) {
        const int Wd = Wc / 2, Hd = Hc / 2;
        const float half = 0.5f * kPi / (float)Hc;
        for (int i = threadIdx.x; i < Wd * Hd * C4; i += kNT) {
            const int c = i % C4, t = i / C4;
            const int x = t % Wd, Y = t / Wd;
            const float w0 = sinf((2.f * Y + 0.5f) * (kPi / (float)Hc)) * sinf(half);
            const float w1 = sinf((2.f * Y + 1.5f) * (kPi / (float)Hc)) * sinf(half);
            const size_t r4 = rgb4[l - 1], ww4 = w4[l - 1];
            const float4 a0 = __ldcg(pyr + pyr_slot<C4>(r4, ww4, (size_t)(2 * Y) * Wc + 2 * x, c));
            const float4 a1 = __ldcg(pyr + pyr_slot<C4>(r4, ww4, (size_t)(2 * Y) * Wc + 2 * x + 1, c));
            const float4 b0 = __ldcg(pyr + pyr_slot<C4>(r4, ww4, (size_t)(2 * Y + 1) * Wc + 2 * x, c));
            const float4 b1 = __ldcg(pyr + pyr_slot<C4>(r4, ww4, (size_t)(2 * Y + 1) * Wc + 2 * x + 1, c));
            const float inv = 1.f / (2.f * (w0 + w1));
            float4 r;
            r.x = (w0 * (a0.x + a1.x) + w1 * (b0.x + b1.x)) * inv;
            r.y = (w0 * (a0.y + a1.y) + w1 * (b0.y + b1.y)) * inv;
            r.z = (w0 * (a0.z + a1.z) + w1 * (b0.z + b1.z)) * inv;
            r.w = (w0 * (a0.w + a1.w) + w1 * (b0.w + b1.w)) * inv;
            pyr[pyr_slot<C4>(rgb4[l], w4[l], (size_t)Y * Wd + x, c)] = r;
        }
        __syncthreads();  // level l complete before it is read
        Wc = Wd;
        Hc = Hd;
    }
    if (threadIdx.x == 0) *done = 0u;
}

// Upper pyramid levels whose base holds at most this many texels are built
// by the last block of the launch that writes the base.
constexpr long kPyrTailTexels = 2048;

// Step 5a: filter sample table (Hammersley points mapped through the GGX
// distribution of microfacet normals weighted by cos theta_h):
// u1 = (j+1/2)/S, u2 = radical inverse of j, cos^2 th = (1-u1)/(1+(a^2-1)u1),
// reflected direction weights (sin 2th cos ph, sin 2th sin ph, cos 2th) in the
// frame (e1, e2, r), valid iff cos 2th > 0 (a prefix of j), and the pyramid
// level lod = 0.5 log2(Omega_s / Omega_0) - 1/2 with Omega_s = 4/(S D(h))
// (the bias of filtered importance sampling that keeps the filtered maps
// closest to the exact convolution on maps with bright suns).
__global__ void k_filter_table(int R, int S, float s_min, float s_max, int W, int H, int M, float4 *table,
                               int *nvalid) {
    const int r = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const float sr = (R > 1) ? s_min + (s_max - s_min) * (float)r / (float)(R - 1) : s_min;
    const float alpha = sr * sr, a2 = alpha * alpha;
    // cos^2 = (1-u)/(1-u+a^2 u), sin^2 = a^2 u/(1-u+a^2 u), cos 2th = (1-u-a^2 u)/(1-u+a^2 u):
    // each a ratio of sums of non-negative terms (no cancellation in FP32).
    if (j == 0) {
        int nv = 0;
        for (int k = 0; k < S; ++k) {
            const float u1 = ((float)k + 0.5f) / (float)S;
            if ((1.f - u1) - a2 * u1 > 0.f) ++nv;
        }
        nvalid[r] = nv;
    }
    if (j >= S) return;
    const float u1 = ((float)j + 0.5f) / (float)S;
    const float u2 = (float)__brev((unsigned)j) * 0x1p-32f;
    const float den = (1.f - u1) + a2 * u1;
    const float c2 = (1.f - u1) / den;
    const float s2 = a2 * u1 / den;
    const float cos2t = ((1.f - u1) - a2 * u1) / den;
    float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
    if (cos2t > 0.f) {
        const float sin2t = 2.f * sqrtf(c2 * s2);
        float sp, cp;
        sincosf(kTwoPi * u2, &sp, &cp);
        const float d = s2 + a2 * c2;  // = c2 (a^2 - 1) + 1
        const float D = a2 / (kPi * d * d);
        const float omega_s = 4.f / ((float)S * D);
        const float omega0 = 4.f * kPi / ((float)W * (float)H);
        float lod = 0.5f * log2f(omega_s / omega0) - 0.5f;
        lod = fminf(fmaxf(lod, 0.f), (float)(M - 1));
        e = make_float4(sin2t * cp, sin2t * sp, cos2t, lod);
    }
    table[(size_t)r * S + j] = e;
}

// Step 5b: filtered maps.  Level r is a W_r x W_r/2 equirect grid; the
// levels are concatenated and the grid of blocks runs over all of them (block
// ranges per level in FilterLevels).  kFilterSplit adjacent threads per output
// texel share its samples; their sums are combined with shuffles.  Result: the
// mean over the level's valid samples of the trilinear pyramid look-up at
// w_i = a e1 + b e2 + c r, where r is the texel direction, e1 = d r / d theta,
// e2 = d r / d phi / sin theta.
struct FilterLevels {
    int nlev;
    int width[33];
    int blk[33];          // first block of level r; blk[nlev] = total blocks
    long long off[33];    // first texel of level r
};

constexpr int kFilterSplit = 2;  // threads per output texel (samples strided over them)

template <int C4>
__global__ void __launch_bounds__(128) k_filter(const float4 *__restrict__ pyr, const size_t *__restrict__ rgb4,
                                                  const size_t *__restrict__ w4,
                                                  int W, int H, int M, const float4 *__restrict__ table,
                                                  const int *__restrict__ nvalid, int S, const FilterLevels fl,
                                                  float4 *__restrict__ out, float4 *__restrict__ outw, int wfmt,
                                                  int rec4, int K) {
    extern __shared__ float4 tab[];
    int r = 0;
    while (r + 1 < fl.nlev && (int)blockIdx.x >= fl.blk[r + 1]) ++r;
    const int Wo = fl.width[r], Ho = Wo / 2;
    const int nv = nvalid[r];
    for (int k = threadIdx.x; k < nv; k += blockDim.x) tab[k] = table[(size_t)r * S + k];
    __syncthreads();
    const int g = threadIdx.x % kFilterSplit;
    const int t = ((int)blockIdx.x - fl.blk[r]) * (blockDim.x / kFilterSplit) + threadIdx.x / kFilterSplit;
    const bool active = t < Wo * Ho;
    const int tt = active ? t : 0;
    const int x = tt % Wo, y = tt / Wo;
    const float th = kPi * ((float)y + 0.5f) / (float)Ho;
    const float ph = kTwoPi * ((float)x + 0.5f) / (float)Wo;
    float st, ct, sp, cp;
    sincosf(th, &st, &ct);
    sincosf(ph, &sp, &cp);
    const float rx = st * cp, ry = ct, rz = st * sp;
    const float e1x = ct * cp, e1y = -st, e1z = ct * sp;
    const float e2x = -sp, e2z = cp;
    // colour and weights accumulated apart (the pyramid's split storage);
    // every channel goes through the same multiply-adds as in the record layout
    constexpr int KW4 = C4 - 1;
    float4 accr = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 accw[KW4];
#pragma unroll
    for (int c = 0; c < KW4; ++c) accw[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = g; k < nv; k += kFilterSplit) {
        const float4 smp = tab[k];
        const float dx = smp.x * e1x + smp.y * e2x + smp.z * rx;
        const float dy = smp.x * e1y + smp.z * ry;
        const float dz = smp.x * e1z + smp.y * e2z + smp.z * rz;
        const float lod = smp.w;
        const int m0 = (int)floorf(lod);
        const float f = lod - (float)m0;
        const int m1 = min(m0 + 1, M - 1);
        const float th_i = acosf(fminf(fmaxf(dy, -1.f), 1.f));
        float ph_i = atan2f(dz, dx);
        if (ph_i < 0.f) ph_i += kTwoPi;
#pragma unroll
        for (int lv = 0; lv < 2; ++lv) {
            const int m = lv ? m1 : m0;
            const float wl = lv ? f : 1.f - f;
            const int Wm = W >> m, Hm = H >> m;
            const float xx = ph_i * (kInvTwoPi * (float)Wm) - 0.5f;
            const float yy = th_i * (kInvPi * (float)Hm) - 0.5f;
            const Taps tp = equirect_taps(xx, yy, Wm, Hm);
            const float4 *prgb = pyr + rgb4[m], *pw = pyr + w4[m];
            const int idx[4] = {tp.i00, tp.i01, tp.i10, tp.i11};
            float4 tr[4], tw[4][KW4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                tr[j] = __ldg(prgb + idx[j]);
                if constexpr (KW4 == 2) {
                    ldg8(pw + (size_t)idx[j] * 2, tw[j][0], tw[j][1]);  // 32-byte aligned (even level offsets)
                } else {
#pragma unroll
                    for (int c = 0; c < KW4; ++c) tw[j][c] = __ldg(pw + (size_t)idx[j] * KW4 + c);
                }
            }
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            v = fma4(tp.w00, tr[0], v);
            v = fma4(tp.w01, tr[1], v);
            v = fma4(tp.w10, tr[2], v);
            v = fma4(tp.w11, tr[3], v);
            accr = fma4(wl, v, accr);
#pragma unroll
            for (int c = 0; c < KW4; ++c) {
                float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
                u = fma4(tp.w00, tw[0][c], u);
                u = fma4(tp.w01, tw[1][c], u);
                u = fma4(tp.w10, tw[2][c], u);
                u = fma4(tp.w11, tw[3][c], u);
                accw[c] = fma4(wl, u, accw[c]);
            }
        }
    }
    // sum the partial means of the kFilterSplit adjacent lanes of a texel
#pragma unroll
    for (int o = 1; o < kFilterSplit; o <<= 1) {
        accr.x += __shfl_xor_sync(0xffffffffu, accr.x, o);
        accr.y += __shfl_xor_sync(0xffffffffu, accr.y, o);
        accr.z += __shfl_xor_sync(0xffffffffu, accr.z, o);
#pragma unroll
        for (int c = 0; c < KW4; ++c) {
            accw[c].x += __shfl_xor_sync(0xffffffffu, accw[c].x, o);
            accw[c].y += __shfl_xor_sync(0xffffffffu, accw[c].y, o);
            accw[c].z += __shfl_xor_sync(0xffffffffu, accw[c].z, o);
            accw[c].w += __shfl_xor_sync(0xffffffffu, accw[c].w, o);
        }
    }
    // back to the record layout (R, G, B, W_1 .. W_K, zero padding)
    float4 acc[C4];
    {
        float ch[4 * C4];
        ch[0] = accr.x; ch[1] = accr.y; ch[2] = accr.z;
#pragma unroll
        for (int c = 0; c < KW4; ++c) {
            ch[3 + 4 * c] = accw[c].x; ch[4 + 4 * c] = accw[c].y; ch[5 + 4 * c] = accw[c].z; ch[6 + 4 * c] = accw[c].w;
        }
        ch[4 * C4 - 1] = 0.f;
#pragma unroll
        for (int c = 0; c < C4; ++c) acc[c] = make_float4(ch[4 * c], ch[4 * c + 1], ch[4 * c + 2], ch[4 * c + 3]);
    }
    if (!active || g != 0) return;
    const float inv = nv > 0 ? 1.f / (float)nv : 0.f;
    const int kw4 = (K + 3) / 4;
    float4 *ow = outw + ((size_t)fl.off[r] + t) * kw4;
    if (wfmt == GLINT_WFMT_F32) {
        float4 *o = out + ((size_t)fl.off[r] + t) * C4;
        float ch[C4 * 4 + 4];
#pragma unroll
        for (int c = 0; c < C4; ++c) {
            o[c] = make_float4(acc[c].x * inv, acc[c].y * inv, acc[c].z * inv, acc[c].w * inv);
            ch[4 * c] = acc[c].x * inv; ch[4 * c + 1] = acc[c].y * inv;
            ch[4 * c + 2] = acc[c].z * inv; ch[4 * c + 3] = acc[c].w * inv;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) ch[C4 * 4 + i] = 0.f;
#pragma unroll
        for (int c = 0; c < C4; ++c)  // weights w_k are channels 3 + k; zero past K
            if (c < kw4)
                ow[c] = make_float4(4 * c < K ? ch[3 + 4 * c] : 0.f, 4 * c + 1 < K ? ch[4 + 4 * c] : 0.f,
                                    4 * c + 2 < K ? ch[5 + 4 * c] : 0.f, 4 * c + 3 < K ? ch[6 + 4 * c] : 0.f);
        return;
    }
    // compressed record: (R, G, B, 0) float32, then K weight codes
    float ch[C4 * 4];
#pragma unroll
    for (int c = 0; c < C4; ++c) {
        ch[4 * c] = acc[c].x * inv; ch[4 * c + 1] = acc[c].y * inv;
        ch[4 * c + 2] = acc[c].z * inv; ch[4 * c + 3] = acc[c].w * inv;
    }
    float4 *o = out + ((size_t)fl.off[r] + t) * rec4;
    o[0] = make_float4(ch[0], ch[1], ch[2], 0.f);
    uint32_t words[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    float dec[C4 * 4];  // the weights as the stored codes decode
#pragma unroll
    for (int k = 0; k < C4 * 4; ++k) dec[k] = 0.f;
#pragma unroll
    for (int k = 0; k < C4 * 4 - 3; ++k) {
        if (k >= K) break;
        const float wv = fminf(fmaxf(ch[3 + k], 0.f), 1.f);
        if (wfmt == GLINT_WFMT_UNORM8) {
            const uint32_t c8 = __float2uint_rn(wv * 255.f) & 0xffu;
            words[k / 4] |= c8 << (8 * (k % 4));
            dec[k] = (float)c8 * (1.f / 255.f);
        } else {
            const uint32_t c16 = (wfmt == GLINT_WFMT_F16) ? (uint32_t)__half_as_ushort(__float2half_rn(ch[3 + k]))
                                                         : (__float2uint_rn(wv * 65535.f) & 0xffffu);
            words[k / 2] |= c16 << (16 * (k % 2));
            dec[k] = (wfmt == GLINT_WFMT_F16) ? __half2float(__ushort_as_half((unsigned short)c16))
                                              : (float)c16 * (1.f / 65535.f);
        }
    }
#pragma unroll
    for (int c = 0; c < C4; ++c)
        if (c < kw4) ow[c] = make_float4(dec[4 * c], dec[4 * c + 1], dec[4 * c + 2], dec[4 * c + 3]);
    uint4 *q = reinterpret_cast<uint4 *>(o + 1);
    for (int i = 0; i < rec4 - 1; ++i) q[i] = make_uint4(words[4 * i], words[4 * i + 1], words[4 * i + 2], words[4 * i + 3]);
}

}  // namespace

template <int C4>
cudaError_t launch_pyramid(bool first, unsigned blocks, size_t smem, cudaStream_t s, const void *texels,
                           const glint_env_desc &d, float scale, glint_env *env, int m, int Ws, int Hs, int T, int nlev,
                           int tail_to) {
    if (first) {
        cudaFuncSetAttribute(k_pyramid<true, C4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_pyramid<true, C4><<<blocks, kNT, smem, s>>>(texels, d.format, scale, d.K, env->levels,
                                                       reinterpret_cast<float4 *>(env->pyr), env->pyr_rgb4_dev,
                                                       env->pyr_w4_dev, 0, Ws, Hs, T, nlev, d.weight_space, tail_to,
                                                       env->done + 1);
    } else {
        cudaFuncSetAttribute(k_pyramid<false, C4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_pyramid<false, C4><<<blocks, kNT, smem, s>>>(nullptr, d.format, scale, d.K, env->levels,
                                                        reinterpret_cast<float4 *>(env->pyr), env->pyr_rgb4_dev,
                                                        env->pyr_w4_dev, m, Ws, Hs, T, nlev, 0, tail_to,
                                                        env->done + 1);
    }
    return cudaGetLastError();
}

// Pyramid level offsets (float4 units) are in a small device array that
// glint_env_create fills.
cudaError_t glint_launch_env(glint_env *env, const void *texels, cudaStream_t s, int *launches) {
    const glint_env_desc &d = env->d;
    const long n = (long)d.width * d.height;
    const float scale = ldexpf(1.f, d.scale_log2);
    const int C4 = env->Cpad / 4;
    (void)n;
    int nl = 0;
    k_minmax<<<env->nblk_minmax, kNT, 0, s>>>(texels, d.format, n, scale, env->partial, env->done, d.K, d.ell,
                                                env->levels);
    ++nl;
    {
        // level 0 and the next log2 T levels from the texels (T = 32), then
        // tiles of 32 while the base is large, and the last levels by the last
        // block of the launch that writes their base (1024 x 512 map: one
        // launch, levels 0-5 by tiles and 6-9 by the last block; 16 x 16
        // tiles left a 64 x 32 base whose five serial levels cost more)
        int m = 0, Ws = d.width, Hs = d.height;
        bool first = true;
        while (first || m < env->M - 1) {
            const int T = Hs < 32 ? Hs : 32;
            int nlev = 0;
            while ((1 << nlev) < T) ++nlev;
            const bool tail = m + nlev < env->M - 1 && (long)(Ws >> nlev) * (Hs >> nlev) <= kPyrTailTexels;
            const int tail_to = tail ? env->M - 1 : -1;
            const size_t smem = sizeof(float) * env->Cpad * ((size_t)T * T + (size_t)(T / 2) * (T / 2));
            const unsigned blocks = (unsigned)((Ws / T) * (Hs / T));
            cudaError_t e = cudaSuccess;
            switch (C4) {
            case 2: e = launch_pyramid<2>(first, blocks, smem, s, texels, d, scale, env, m, Ws, Hs, T, nlev, tail_to); break;
            case 3: e = launch_pyramid<3>(first, blocks, smem, s, texels, d, scale, env, m, Ws, Hs, T, nlev, tail_to); break;
            case 5: e = launch_pyramid<5>(first, blocks, smem, s, texels, d, scale, env, m, Ws, Hs, T, nlev, tail_to); break;
            default: return cudaErrorInvalidValue;
            }
            if (e != cudaSuccess) return e;
            ++nl;
            first = false;
            m += nlev;
            Ws >>= nlev;
            Hs >>= nlev;
            if (tail || nlev == 0) break;
        }
    }
    {
        FilterLevels fl{};
        fl.nlev = d.levels;
        int blk = 0;
        for (int r = 0; r < d.levels; ++r) {
            fl.width[r] = env->fw[r];
            fl.off[r] = env->foff[r];
            fl.blk[r] = blk;
            const int per_block = 128 / kFilterSplit;
            blk += (int)((env->fw[r] * (env->fw[r] / 2) + per_block - 1) / per_block);
        }
        fl.blk[d.levels] = blk;
        const size_t smem = sizeof(float4) * (size_t)d.samples;
        const float4 *pyr4 = reinterpret_cast<const float4 *>(env->pyr);
        float4 *out4 = reinterpret_cast<float4 *>(env->filt);
        switch (C4) {
        case 2:
            k_filter<2><<<blk, 128, smem, s>>>(pyr4, env->pyr_rgb4_dev, env->pyr_w4_dev, d.width, d.height, env->M, env->table, env->nvalid,
                                               d.samples, fl, out4, env->filtw, d.weight_format, env->frec4, d.K);
            break;
        case 3:
            k_filter<3><<<blk, 128, smem, s>>>(pyr4, env->pyr_rgb4_dev, env->pyr_w4_dev, d.width, d.height, env->M, env->table, env->nvalid,
                                               d.samples, fl, out4, env->filtw, d.weight_format, env->frec4, d.K);
            break;
        case 5:
            k_filter<5><<<blk, 128, smem, s>>>(pyr4, env->pyr_rgb4_dev, env->pyr_w4_dev, d.width, d.height, env->M, env->table, env->nvalid,
                                               d.samples, fl, out4, env->filtw, d.weight_format, env->frec4, d.K);
            break;
        default:
            return cudaErrorInvalidValue;
        }
        ++nl;
    }
    if (launches) *launches = nl;
    return cudaGetLastError();
}

// The filter sample table depends only on the description (levels, samples,
// roughness range, map size); glint_env_create builds it once.
cudaError_t glint_launch_filter_table(glint_env *env, cudaStream_t s) {
    const glint_env_desc &d = env->d;
    dim3 grid((d.samples + 127) / 128, d.levels);
    k_filter_table<<<grid, 128, 0, s>>>(d.levels, d.samples, d.s_min, d.s_max, d.width, d.height, env->M, env->table,
                                        env->nvalid);
    return cudaGetLastError();
}
