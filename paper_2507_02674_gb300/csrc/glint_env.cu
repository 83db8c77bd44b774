// Per-environment preprocessing: radiance levels, fuzzy weights, pyramid and
// filtered maps (Sec. 4 "Discrete Radiance Levels", "Fuzzy Indicator
// Functions", Eq. wkdefpractice, "Integrated NDF" Eq. rtiblndf; Sec. 3.4
// Eq. rtibl).
//
// Data layout in HBM: every per-texel channel vector (R, G, B, w_1..w_K) is
// stored contiguously and padded to Cpad = 4 ceil((3+K)/4) floats, so one texel
// is Cpad/4 aligned float4 loads (3 for K = 8).  The pyramid levels are
// concatenated; the filtered maps are R levels of Ho x Wo texels of the same
// layout.  Brightness min/max go through a small per-block scratch array.
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

// Step 1: per-block min / max of the brightness into the scratch array.
__global__ void __launch_bounds__(kNT) k_minmax(const void *__restrict__ texels, int fmt, long n, float scale,
                                                  float2 *__restrict__ partial) {
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
}

// Step 2: lo = max(min Y, ell), hi = max(max Y, lo);
// L_1 = 0, L_k = lo (hi/lo)^((k-1)/(K-1)) = exp(lerp(ln lo, ln hi, (k-1)/(K-1))).
__global__ void __launch_bounds__(kNT) k_levels(const float2 *__restrict__ partial, int nblk, int K, float ell,
                                                  float *__restrict__ levels) {
    float lo = INFINITY, hi = -INFINITY;
    for (int i = threadIdx.x; i < nblk; i += kNT) {
        lo = fminf(lo, partial[i].x);
        hi = fmaxf(hi, partial[i].y);
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

// Step 3: channels (R, G, B, w_1 .. w_K) of every texel (pyramid level 0).
__global__ void __launch_bounds__(kNT) k_weights(const void *__restrict__ texels, int fmt, long n, float scale,
                                                   int K, int Cpad, const float *__restrict__ levels,
                                                   float *__restrict__ ch0) {
    __shared__ float L[GLINT_MAX_K];
    if (threadIdx.x < K) L[threadIdx.x] = levels[threadIdx.x];
    __syncthreads();
    const long i = (long)blockIdx.x * kNT + threadIdx.x;
    if (i >= n) return;
    const float4 t = load_texel(texels, fmt, i);
    const float R = t.x * scale, G = t.y * scale, B = t.z * scale;
    const float Y = fmaxf(0.2126f * R + 0.7152f * G + 0.0722f * B, 0.f);
    float4 *dst = reinterpret_cast<float4 *>(ch0 + (size_t)i * Cpad);
    // bracket: largest j in [0, K-2] with L[j] <= Y; Y >= L[K-1] -> w_K = 1
    int j = 0;
    for (int k = 1; k < K - 1; ++k)
        if (L[k] <= Y) j = k;
    const bool top = Y >= L[K - 1];
    const float tt = (Y - L[j]) / (L[j + 1] - L[j]);
    // write channel vector in float4 chunks
    for (int c4 = 0; c4 < Cpad / 4; ++c4) {
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = c4 * 4 + e;
            float val = 0.f;
            if (c == 0) val = R;
            else if (c == 1) val = G;
            else if (c == 2) val = B;
            else if (c < 3 + K) {
                const int k = c - 3;
                if (top) val = (k == K - 1) ? 1.f : 0.f;
                else if (k == j) val = 1.f - tt;
                else if (k == j + 1) val = tt;
            }
            v[e] = val;
        }
        dst[c4] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// Step 4: one pyramid level from the previous one; the weight of a texel row
// spanning [theta0, theta1] is cos theta0 - cos theta1 = 2 sin(mid) sin(half),
// written as a product to stay accurate near the poles.  One thread per
// (destination texel, float4 chunk).
__global__ void __launch_bounds__(kNT) k_mip(const float4 *__restrict__ src, int Ws, int Hs, int C4,
                                               float4 *__restrict__ dst) {
    const int Wd = Ws >> 1, Hd = Hs >> 1;
    const long total = (long)Wd * Hd * C4;
    const long id = (long)blockIdx.x * kNT + threadIdx.x;
    if (id >= total) return;
    const int c = (int)(id % C4);
    const long t = id / C4;
    const int x = (int)(t % Wd), y = (int)(t / Wd);
    const float half = 0.5f * kPi / (float)Hs;
    const float w0 = sinf((2.f * y + 0.5f) * (kPi / (float)Hs)) * sinf(half);
    const float w1 = sinf((2.f * y + 1.5f) * (kPi / (float)Hs)) * sinf(half);
    const float4 a0 = src[((long)(2 * y) * Ws + 2 * x) * C4 + c];
    const float4 a1 = src[((long)(2 * y) * Ws + 2 * x + 1) * C4 + c];
    const float4 b0 = src[((long)(2 * y + 1) * Ws + 2 * x) * C4 + c];
    const float4 b1 = src[((long)(2 * y + 1) * Ws + 2 * x + 1) * C4 + c];
    const float inv = 1.f / (2.f * (w0 + w1));
    float4 r;
    r.x = (w0 * (a0.x + a1.x) + w1 * (b0.x + b1.x)) * inv;
    r.y = (w0 * (a0.y + a1.y) + w1 * (b0.y + b1.y)) * inv;
    r.z = (w0 * (a0.z + a1.z) + w1 * (b0.z + b1.z)) * inv;
    r.w = (w0 * (a0.w + a1.w) + w1 * (b0.w + b1.w)) * inv;
    dst[id] = r;
}

// Step 5a: filter sample table (Hammersley points mapped through the GGX
// distribution of microfacet normals weighted by cos theta_h):
// u1 = (j+1/2)/S, u2 = radical inverse of j, cos^2 th = (1-u1)/(1+(a^2-1)u1),
// reflected direction weights (sin 2th cos ph, sin 2th sin ph, cos 2th) in the
// frame (e1, e2, r), valid iff cos 2th > 0 (a prefix of j), and the pyramid
// level lod = 0.5 log2(Omega_s / Omega_0) + 1 with Omega_s = 4/(S D(h)).
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
        float lod = 0.5f * log2f(omega_s / omega0) + 1.f;
        lod = fminf(fmaxf(lod, 0.f), (float)(M - 1));
        e = make_float4(sin2t * cp, sin2t * sp, cos2t, lod);
    }
    table[(size_t)r * S + j] = e;
}

// Step 5b: filtered maps.  One thread per output texel (r, y, x) of an
// Wo x Ho equirect grid; mean over the level's valid samples of the trilinear
// pyramid look-up at w_i = a e1 + b e2 + c r, where r is the texel direction,
// e1 = d r / d theta, e2 = d r / d phi / sin theta.
template <int C4>
__global__ void __launch_bounds__(128) k_filter(const float4 *__restrict__ pyr, const size_t *__restrict__ off4,
                                                  int W, int H, int M, const float4 *__restrict__ table,
                                                  const int *__restrict__ nvalid, int S, int Wo, int Ho,
                                                  float4 *__restrict__ out) {
    extern __shared__ float4 tab[];
    const int r = blockIdx.y;
    const int nv = nvalid[r];
    for (int k = threadIdx.x; k < nv; k += blockDim.x) tab[k] = table[(size_t)r * S + k];
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Wo * Ho) return;
    const int x = t % Wo, y = t / Wo;
    const float th = kPi * ((float)y + 0.5f) / (float)Ho;
    const float ph = kTwoPi * ((float)x + 0.5f) / (float)Wo;
    float st, ct, sp, cp;
    sincosf(th, &st, &ct);
    sincosf(ph, &sp, &cp);
    const float rx = st * cp, ry = ct, rz = st * sp;
    const float e1x = ct * cp, e1y = -st, e1z = ct * sp;
    const float e2x = -sp, e2z = cp;
    float4 acc[C4];
#pragma unroll
    for (int c = 0; c < C4; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < nv; ++k) {
        const float4 s = tab[k];
        const float dx = s.x * e1x + s.y * e2x + s.z * rx;
        const float dy = s.x * e1y + s.z * ry;
        const float dz = s.x * e1z + s.y * e2z + s.z * rz;
        const float lod = s.w;
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
            const float4 *base = pyr + off4[m];
#pragma unroll
            for (int c = 0; c < C4; ++c) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                v = fma4(tp.w00, __ldg(base + (size_t)tp.i00 * C4 + c), v);
                v = fma4(tp.w01, __ldg(base + (size_t)tp.i01 * C4 + c), v);
                v = fma4(tp.w10, __ldg(base + (size_t)tp.i10 * C4 + c), v);
                v = fma4(tp.w11, __ldg(base + (size_t)tp.i11 * C4 + c), v);
                acc[c] = fma4(wl, v, acc[c]);
            }
        }
    }
    const float inv = nv > 0 ? 1.f / (float)nv : 0.f;
    float4 *o = out + ((size_t)r * Wo * Ho + t) * C4;
#pragma unroll
    for (int c = 0; c < C4; ++c)
        o[c] = make_float4(acc[c].x * inv, acc[c].y * inv, acc[c].z * inv, acc[c].w * inv);
}

}  // namespace

// Pyramid level offsets (float4 units) are in a small device array that
// glint_env_create fills.
cudaError_t glint_launch_env(glint_env *env, const void *texels, cudaStream_t s, int *launches) {
    const glint_env_desc &d = env->d;
    const long n = (long)d.width * d.height;
    const float scale = ldexpf(1.f, d.scale_log2);
    const int C4 = env->Cpad / 4;
    int nl = 0;
    k_minmax<<<env->nblk_minmax, kNT, 0, s>>>(texels, d.format, n, scale, env->partial);
    ++nl;
    k_levels<<<1, kNT, 0, s>>>(env->partial, env->nblk_minmax, d.K, d.ell, env->levels);
    ++nl;
    k_weights<<<(unsigned)((n + kNT - 1) / kNT), kNT, 0, s>>>(texels, d.format, n, scale, d.K, env->Cpad,
                                                               env->levels, env->pyr);
    ++nl;
    for (int m = 1; m < env->M; ++m) {
        const int Ws = d.width >> (m - 1), Hs = d.height >> (m - 1);
        const long total = (long)(Ws / 2) * (Hs / 2) * C4;
        k_mip<<<(unsigned)((total + kNT - 1) / kNT), kNT, 0, s>>>(
            reinterpret_cast<const float4 *>(env->pyr + env->pyr_off[m - 1]), Ws, Hs, C4,
            reinterpret_cast<float4 *>(env->pyr + env->pyr_off[m]));
        ++nl;
    }
    {
        dim3 grid((d.samples + 127) / 128, d.levels);
        k_filter_table<<<grid, 128, 0, s>>>(d.levels, d.samples, d.s_min, d.s_max, d.width, d.height, env->M,
                                            env->table, env->nvalid);
        ++nl;
    }
    {
        const int texels_out = d.out_width * env->Ho;
        dim3 grid((texels_out + 127) / 128, d.levels);
        const size_t smem = sizeof(float4) * (size_t)d.samples;
        const float4 *pyr4 = reinterpret_cast<const float4 *>(env->pyr);
        const size_t *off4 = env->pyr_off4_dev;
        float4 *out4 = reinterpret_cast<float4 *>(env->filt);
        switch (C4) {
        case 2:
            k_filter<2><<<grid, 128, smem, s>>>(pyr4, off4, d.width, d.height, env->M, env->table, env->nvalid,
                                                d.samples, d.out_width, env->Ho, out4);
            break;
        case 3:
            k_filter<3><<<grid, 128, smem, s>>>(pyr4, off4, d.width, d.height, env->M, env->table, env->nvalid,
                                                d.samples, d.out_width, env->Ho, out4);
            break;
        case 5:
            k_filter<5><<<grid, 128, smem, s>>>(pyr4, off4, d.width, d.height, env->M, env->table, env->nvalid,
                                                d.samples, d.out_width, env->Ho, out4);
            break;
        default:
            return cudaErrorInvalidValue;
        }
        ++nl;
    }
    if (launches) *launches = nl;
    return cudaGetLastError();
}
