// Reflection probabilities p_k of a pixel (Eq. probhk): E1 from the filtered
// maps and tables (Eq. rtiblndf), E2 by quadrature of the anisotropic NDF, or
// given; shared by the shading kernel and the surrogate's feature kernels.
#pragma once
#include "glint_internal.cuh"

namespace glint {

struct ShadeArgs {
    const float4 *view_n0, *normal_f0, *uv_alpha, *duv, *tangent;
    float4 *out;
    long npix;
    const float4 *lut;
    int lut_n;
    const float4 *filt;
    const float4 *filtw;  // the filtered weights alone: ceil(K/4) float4 per texel
    const int2 *flev;  // (width, first texel) of each filtered level
    int wfmt;          // glint_weight_format of the filtered maps' weights
    int frec4;         // 16-byte units per texel record of a compressed format
    int R;
    float s_min, s_max;
    float s_scale;     // (R - 1) / (s_max - s_min): filtered level per unit of sqrt(alpha)
    const float *levels;
    uint32_t seed;
    glint_debug dbg;
    // E2: weights pyramid
    const float4 *pyr;
    const size_t *pyr_w4;  // float4 offset of each pyramid level's weights (C4 - 1 float4 per texel)
    int envW, envH, envM, e2S;
    const float *pk_in;  // EV_GIVEN: p_k per pixel (npix x K)
    float *p_out;        // k_probs: p_k per pixel (npix x K)
    int draw;                 // kDraw*
    float gamma;              // kDrawWang: the environment-independent reflection probability
    const void *mlp_wt;       // serving: the frame's surrogate (BF16 weight copies)
    const float *mlp_params;  //          and its FP32 parameters (biases)
};

// One work item of the serving kernels: pixels [first, first + count) of
// frame `frame` (an index into the tick's frame table).
struct ServeItem {
    int frame;
    int count;
    long first;
};

// Binomial approximation at the tree nodes (glint_draw).
constexpr int kDrawDual = 0, kDrawSingle = 1, kDrawSingleOld = 2, kDrawWang = 3;

// Source of the reflection probabilities p_k (EV_NONE: smooth radiance only,
// p left to the caller; EV_E1A: E1 with multi-tap look-ups along an
// anisotropic lobe).
constexpr int EV_E1 = 0, EV_E2 = 1, EV_GIVEN = 2, EV_NONE = 3, EV_E1A = 4;

// E2: reflection probabilities of an anisotropic GGX footprint by quadrature
// (Eq. probhk).  Points of the projected-area slope distribution in
// (s, u2), u1 = 1 - s^2, r = sqrt(1 - s^2)/s, slope = (a_x r cos phi,
// a_y r sin phi), h' = (-slope, 1) in (t, b = n x t, n); bounded weight
// 2 sqrt(s^2 + rho^2 (1 - s^2)); valid iff 2 w_o.h' > mu_o |h'|^2
// (n . w_i > 0); w_k read bilinearly at pyramid level m, the coarsest whose
// texel pi/H_m is at most 4 min(a_x, a_y)/S (an exact FP32 comparison).
template <int K, int C4>
__device__ __forceinline__ void e2_probabilities(const ShadeArgs &a, long q, float4 g0, float4 g1, float4 g2,
                                                 float mu_o, float *p) {
    const float4 tg = ldg4(a.tangent + q);
    const float tn = tg.x * g1.x + tg.y * g1.y + tg.z * g1.z;
    float tx = tg.x - tn * g1.x, ty = tg.y - tn * g1.y, tz = tg.z - tn * g1.z;
    const float tinv = 1.f / sqrtf(tx * tx + ty * ty + tz * tz);
    tx *= tinv; ty *= tinv; tz *= tinv;
    const float bx = g1.y * tz - g1.z * ty, by = g1.z * tx - g1.x * tz, bz = g1.x * ty - g1.y * tx;
    const float ot = g0.x * tx + g0.y * ty + g0.z * tz;
    const float ob = g0.x * bx + g0.y * by + g0.z * bz;
    const int S = a.e2S;
    const float lx = fminf(g2.z, g2.w) * (4.0f / (float)S);
    int m = 0;
    for (int k = 0; k < a.envM; ++k)
        if ((float)(a.envH >> k) * lx >= kPi) m = k;
    const int Wm = a.envW >> m, Hm = a.envH >> m;
    constexpr int KW4 = C4 - 1;
    const float4 *levw = a.pyr + a.pyr_w4[m];  // the level's weights W_1 .. W_K
    const float ax2 = g2.z * g2.z, ay2 = g2.w * g2.w;
    float sum_all = 0.f, sum_inv = 0.f;
    float acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.f;
#pragma unroll 1
    for (int ia = 0; ia < S; ++ia) {
        const float sv = ((float)ia + 0.5f) / (float)S;
        const float r = sqrtf(1.f - sv * sv) / sv;
#pragma unroll 1
        for (int ic = 0; ic < S; ++ic) {
            float sp, cp;
            sincospif(2.f * ((float)ic + 0.5f) / (float)S, &sp, &cp);
            const float sx = g2.z * r * cp, sy = g2.w * r * sp;
            const float rho2 = ax2 * cp * cp + ay2 * sp * sp;
            const float wgt = 2.f * sqrtf(sv * sv + rho2 * (1.f - sv * sv));
            const float hl2 = 1.f + sx * sx + sy * sy;
            const float oh = -sx * ot - sy * ob + mu_o;
            sum_all += wgt;
            if (!(2.f * oh - mu_o * hl2 > 0.f)) {
                sum_inv += wgt;
                continue;
            }
            const float il = rsqrtf(hl2);
            const float hx = (-sx * tx - sy * bx + g1.x) * il;
            const float hy = (-sx * ty - sy * by + g1.y) * il;
            const float hz = (-sx * tz - sy * bz + g1.z) * il;
            const float c2 = 2.f * oh * il;
            const float dx = c2 * hx - g0.x, dy = c2 * hy - g0.y, dz = c2 * hz - g0.z;
            float ex, ey;
            dir_to_texel(dx, dy, dz, Wm, Hm, ex, ey);
            const Taps tp = equirect_taps(ex, ey, Wm, Hm);
            float w[KW4 * 4];
            const int idx[4] = {tp.i00, tp.i01, tp.i10, tp.i11};
            float4 tw[4][KW4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if constexpr (KW4 == 2) {
                    ldg8(levw + (size_t)idx[j] * 2, tw[j][0], tw[j][1]);  // 32-byte aligned (even level offsets)
                } else {
#pragma unroll
                    for (int c = 0; c < KW4; ++c) tw[j][c] = __ldg(levw + (size_t)idx[j] * KW4 + c);
                }
            }
#pragma unroll
            for (int c = 0; c < KW4; ++c) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                v = fma4(tp.w00, tw[0][c], v);
                v = fma4(tp.w01, tw[1][c], v);
                v = fma4(tp.w10, tw[2][c], v);
                v = fma4(tp.w11, tw[3][c], v);
                w[4 * c] = v.x; w[4 * c + 1] = v.y; w[4 * c + 2] = v.z; w[4 * c + 3] = v.w;
            }
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] = fmaf(wgt, w[k], acc[k]);
        }
    }
    const float inv = 1.f / sum_all;
    p[0] = (sum_inv + acc[0]) * inv;
#pragma unroll
    for (int k = 1; k < K; ++k) p[k] = acc[k] * inv;
}

__device__ __forceinline__ float4 lut_fetch(const float4 *lut, int n, float mu, float s) {
    float x = fminf(fmaxf(mu * (float)n - 0.5f, 0.f), (float)(n - 1));
    float y = fminf(fmaxf(s * (float)n - 0.5f, 0.f), (float)(n - 1));
    const float fx0 = floorf(x), fy0 = floorf(y);
    const int x0 = (int)fx0, y0 = (int)fy0;
    const int x1 = min(x0 + 1, n - 1), y1 = min(y0 + 1, n - 1);
    const float fx = x - fx0, fy = y - fy0;
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    r = fma4((1.f - fy) * (1.f - fx), __ldg(lut + y0 * n + x0), r);
    r = fma4((1.f - fy) * fx, __ldg(lut + y0 * n + x1), r);
    r = fma4(fy * (1.f - fx), __ldg(lut + y1 * n + x0), r);
    r = fma4(fy * fx, __ldg(lut + y1 * n + x1), r);
    return r;
}


// Channels (R, G, B, W_1 .. W_K) of the filtered maps at direction (th, ph),
// bilinear in the levels r0 and r1 blended by ft, into ch[0 .. 3+K) (RGB only
// unless NEED_W).  FP32 maps hold C4 float4 per texel; compressed ones a
// record of frec4 x 16 bytes: (R, G, B, -) as float4, then the K weights as
// FP16, UNORM16 or UNORM8 codes.
__device__ __forceinline__ float decode_w(uint32_t word, int j, int wfmt) {
    if (wfmt == GLINT_WFMT_UNORM8) return (float)((word >> (8 * j)) & 0xffu) * (1.f / 255.f);
    const uint32_t h = (word >> (16 * j)) & 0xffffu;
    if (wfmt == GLINT_WFMT_F16) return __half2float(__ushort_as_half((unsigned short)h));
    return (float)h * (1.f / 65535.f);
}

template <int K, int C4, bool NEED_W>
__device__ __forceinline__ void filtered_channels(const ShadeArgs &a, float th, float ph, int r0, int r1, float ft,
                                                  float *ch) {
    if (a.wfmt == GLINT_WFMT_F32) {
        float4 cc[C4];
#pragma unroll
        for (int c = 0; c < C4; ++c) cc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int lv = 0; lv < 2; ++lv) {
            const int2 lev = __ldg(a.flev + (lv ? r1 : r0));
            const int Wr = lev.x, Hr = lev.x / 2;
            const Taps tp = equirect_taps(ph * (kInvTwoPi * (float)Wr) - 0.5f, th * (kInvPi * (float)Hr) - 0.5f, Wr, Hr);
            const float4 *base = a.filt + (size_t)lev.y * C4;
            const float wl = lv ? ft : 1.f - ft;
            constexpr int CN = NEED_W ? C4 : 1;
#pragma unroll
            for (int c = 0; c < CN; ++c) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                v = fma4(tp.w00, __ldg(base + (size_t)tp.i00 * C4 + c), v);
                v = fma4(tp.w01, __ldg(base + (size_t)tp.i01 * C4 + c), v);
                v = fma4(tp.w10, __ldg(base + (size_t)tp.i10 * C4 + c), v);
                v = fma4(tp.w11, __ldg(base + (size_t)tp.i11 * C4 + c), v);
                cc[c] = fma4(wl, v, cc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < C4; ++c) {
            ch[4 * c] = cc[c].x; ch[4 * c + 1] = cc[c].y; ch[4 * c + 2] = cc[c].z; ch[4 * c + 3] = cc[c].w;
        }
        return;
    }
    // compressed weights
    const int rec = a.frec4, wfmt = a.wfmt;
    const int per_word = (wfmt == GLINT_WFMT_UNORM8) ? 4 : 2;
    float4 rgb = make_float4(0.f, 0.f, 0.f, 0.f);
    float w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = 0.f;
#pragma unroll
    for (int lv = 0; lv < 2; ++lv) {
        const int2 lev = __ldg(a.flev + (lv ? r1 : r0));
        const int Wr = lev.x, Hr = lev.x / 2;
        const Taps tp = equirect_taps(ph * (kInvTwoPi * (float)Wr) - 0.5f, th * (kInvPi * (float)Hr) - 0.5f, Wr, Hr);
        const float4 *base = a.filt + (size_t)lev.y * rec;
        const float wl = lv ? ft : 1.f - ft;
        const int idx[4] = {tp.i00, tp.i01, tp.i10, tp.i11};
        const float tw[4] = {tp.w00, tp.w01, tp.w10, tp.w11};
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int t = 0; t < 4; ++t) v = fma4(tw[t], __ldg(base + (size_t)idx[t] * rec), v);
        rgb = fma4(wl, v, rgb);
        if (NEED_W) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint32_t *codes = reinterpret_cast<const uint32_t *>(base + (size_t)idx[t] * rec + 1);
                const float f = wl * tw[t];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const uint32_t word = __ldg(codes + k / per_word);  // same word: loaded once after CSE
                    w[k] = fmaf(f, decode_w(word, k % per_word, wfmt), w[k]);
                }
            }
        }
    }
    ch[0] = rgb.x; ch[1] = rgb.y; ch[2] = rgb.z;
#pragma unroll
    for (int k = 0; k < K; ++k) ch[3 + k] = w[k];
}

template <int K>
__device__ __forceinline__ void e1a_weights(const ShadeArgs &a, long q, float4 g0, float4 g1, float4 g2, float mu,
                                            float rx, float ry, float rz, float *W);

// Step 1: smooth radiance (L_o) and the reflection probabilities p_k.
template <int K, int EV>
__device__ __forceinline__ void smooth_and_probs(const ShadeArgs &a, long q, float4 g0, float4 g1, float4 g2,
                                                 float &Lor, float &Log, float &Lob, float *p) {
    constexpr int C4 = (3 + K + 3) / 4;
    const float mu_o = g1.x * g0.x + g1.y * g0.y + g1.z * g0.z;
    const float rx = 2.f * mu_o * g1.x - g0.x;
    const float ry = 2.f * mu_o * g1.y - g0.y;
    const float rz = 2.f * mu_o * g1.z - g0.z;
    const float mu_c = fminf(fmaxf(mu_o, 1e-4f), 1.f);
    const float s = sqrtf(sqrtf(g2.z * g2.w));
    const float4 tab = lut_fetch(a.lut, a.lut_n, mu_c, s);  // V, U, A, B
    float tl = (s - a.s_min) * a.s_scale;
    tl = fminf(fmaxf(tl, 0.f), (float)(a.R - 1));
    const int r0 = (int)floorf(tl);
    const int r1 = min(r0 + 1, a.R - 1);
    const float ft = tl - (float)r0;
    // direction of w_r on the unit sphere, then texel coordinates per level
    const float th_r = acosf(fminf(fmaxf(ry, -1.f), 1.f));
    float ph_r = atan2f(rz, rx);
    if (ph_r < 0.f) ph_r += kTwoPi;
    float ch[C4 * 4];
    // E2 and given p_k need the colour channels only
    filtered_channels<K, C4, EV == EV_E1>(a, th_r, ph_r, r0, r1, ft, ch);
    const float Eb = g1.w * tab.z + tab.w;
    Lor = ch[0] * Eb;
    Log = ch[1] * Eb;
    Lob = ch[2] * Eb;
    if (EV == EV_E2) {
        e2_probabilities<K, C4>(a, q, g0, g1, g2, mu_o, p);
    } else if (EV == EV_GIVEN) {
#pragma unroll
        for (int k = 0; k < K; ++k) p[k] = __ldg(a.pk_in + q * K + k);
    } else if (EV == EV_NONE) {
    } else if (EV == EV_E1A) {
        float W[K];
        e1a_weights<K>(a, q, g0, g1, g2, mu_o, rx, ry, rz, W);
        p[0] = tab.y + tab.x * W[0];
#pragma unroll
        for (int k = 1; k < K; ++k) p[k] = tab.x * W[k];
    } else {
        p[0] = tab.y + tab.x * ch[3];
#pragma unroll
        for (int k = 1; k < K; ++k) p[k] = tab.x * ch[3 + k];
    }
}


inline ShadeArgs make_args(const glint_ctx *ctx, const glint_env *env, const glint_gbuffer *g, const glint_params *p) {
    ShadeArgs a{};
    a.view_n0 = reinterpret_cast<const float4 *>(g->view_n0);
    a.tangent = reinterpret_cast<const float4 *>(g->tangent);
    a.normal_f0 = reinterpret_cast<const float4 *>(g->normal_f0);
    a.uv_alpha = reinterpret_cast<const float4 *>(g->uv_alpha);
    a.duv = reinterpret_cast<const float4 *>(g->duv);
    a.npix = (long)g->width * g->height;
    a.lut = ctx->lut;
    a.lut_n = ctx->lut_n;
    a.filt = reinterpret_cast<const float4 *>(env->filt);
    a.filtw = env->filtw;
    a.wfmt = env->d.weight_format;
    a.frec4 = env->frec4;
    a.R = env->d.levels;
    a.flev = env->flev;
    a.s_min = env->d.s_min;
    a.s_max = env->d.s_max;
    a.s_scale = (a.R > 1) ? (float)(a.R - 1) / (a.s_max - a.s_min) : 0.f;
    a.levels = env->levels;
    a.seed = p->seed;
    a.pyr = reinterpret_cast<const float4 *>(env->pyr);
    a.pyr_w4 = env->pyr_w4_dev;
    a.envW = env->d.width;
    a.envH = env->d.height;
    a.envM = env->M;
    a.e2S = p->e2_samples > 0 ? p->e2_samples : 16;
    a.draw = p->draw;
    a.gamma = p->gamma;
    return a;
}


}  // namespace glint

namespace glint {

// ---------------------------------------------------------------------------
// Inputs of the p_k surrogate (no counterpart in the paper): per pixel
//   [ p_k of E1 (K) | W_k at 5 taps (5K) | mu_o, sqrt a_x, sqrt a_y | 0 ... ]
// (64 values) and the prior log max(p_k^E1, 1e-6) added to the output logits.
// W_k is read from the filtered maps at roughness parameter s = sqrt(min(a_x,
// a_y)) in the directions w_r (centre) and normalize(w_r +- a_x J_t),
// normalize(w_r +- a_y J_b), where J_t = 2 (-(w_o.t) n - mu_o t) is the
// derivative of the mirror direction with respect to the slope along the
// tangent t (made orthogonal to n) and J_b likewise along b = n x t: the
// lobe's extent along its two axes, including the stretch at grazing views.
constexpr int kMlpIn = 64;
constexpr int kMlpTaps = 5;
constexpr float kPriorFloor = 1e-6f;

// The filtered weights W_1 .. W_K alone at direction (th, ph), bilinear in
// the levels r0 and r1 blended by ft, from the weights-only copy of the
// filtered maps (ceil(K/4) float4 per texel instead of the full record).
// Each weight goes through the same multiply-adds, in the same order, as in
// filtered_channels with FP32 weights, so the values are the same.
template <int K>
__device__ __forceinline__ void filtered_w(const ShadeArgs &a, float th, float ph, int r0, int r1, float ft,
                                           float *W) {
    constexpr int KW4 = (K + 3) / 4;
    float4 cc[KW4];
#pragma unroll
    for (int c = 0; c < KW4; ++c) cc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int lv = 0; lv < 2; ++lv) {
        const int2 lev = __ldg(a.flev + (lv ? r1 : r0));
        const int Wr = lev.x, Hr = lev.x / 2;
        const Taps tp = equirect_taps(ph * (kInvTwoPi * (float)Wr) - 0.5f, th * (kInvPi * (float)Hr) - 0.5f, Wr, Hr);
        const float4 *base = a.filtw + (size_t)lev.y * KW4;
        const float wl = lv ? ft : 1.f - ft;
        if constexpr (KW4 == 2) {
            // 32-byte texels in a cudaMalloc'd buffer: every texel is 32-byte aligned
            float4 t[4][2];
            ldg8(base + (size_t)tp.i00 * 2, t[0][0], t[0][1]);
            ldg8(base + (size_t)tp.i01 * 2, t[1][0], t[1][1]);
            ldg8(base + (size_t)tp.i10 * 2, t[2][0], t[2][1]);
            ldg8(base + (size_t)tp.i11 * 2, t[3][0], t[3][1]);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                v = fma4(tp.w00, t[0][c], v);
                v = fma4(tp.w01, t[1][c], v);
                v = fma4(tp.w10, t[2][c], v);
                v = fma4(tp.w11, t[3][c], v);
                cc[c] = fma4(wl, v, cc[c]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < KW4; ++c) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                v = fma4(tp.w00, __ldg(base + (size_t)tp.i00 * KW4 + c), v);
                v = fma4(tp.w01, __ldg(base + (size_t)tp.i01 * KW4 + c), v);
                v = fma4(tp.w10, __ldg(base + (size_t)tp.i10 * KW4 + c), v);
                v = fma4(tp.w11, __ldg(base + (size_t)tp.i11 * KW4 + c), v);
                cc[c] = fma4(wl, v, cc[c]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float4 v = cc[k / 4];
        W[k] = (k % 4 == 0) ? v.x : (k % 4 == 1) ? v.y : (k % 4 == 2) ? v.z : v.w;
    }
}

// W_1 .. W_K of the filtered maps at unit direction d and roughness parameter
// s (the two levels bracketing s, bilinear in each, as E1 does for w_r).
template <int K>
__device__ __forceinline__ void filtered_weights_only(const ShadeArgs &a, float dx, float dy, float dz, float s,
                                                      float *W) {
    float tl = (s - a.s_min) * a.s_scale;
    tl = fminf(fmaxf(tl, 0.f), (float)(a.R - 1));
    const int r0 = (int)floorf(tl);
    const int r1 = min(r0 + 1, a.R - 1);
    const float ft = tl - (float)r0;
    const float th = acosf(fminf(fmaxf(dy, -1.f), 1.f));
    float ph = atan2f(dz, dx);
    if (ph < 0.f) ph += kTwoPi;
    filtered_w<K>(a, th, ph, r0, r1, ft, W);
}

// Filtered weights of the anisotropic E1 (multi-tap look-ups): the lobe of
// reflected directions as an ellipse with axes J_t a_x, J_b a_y, J_t = 2 (-(w_o.t)
// n - mu_o t) and J_b likewise the derivatives of the mirror direction with
// respect to the slope (t made orthogonal to n, b = n x t); the filtered
// weights read at roughness a_l = min(|J_t| a_x, |J_b| a_y) / 2 at the five
// Gauss-Hermite nodes x_j along the longer axis u, d_j = normalize(w_r +
// x_j sigma u), sigma^2 = 0.4 (L_max^2 - L_min^2), weighted by the rule's w_j.
template <int K>
__device__ __forceinline__ void e1a_weights(const ShadeArgs &a, long q, float4 g0, float4 g1, float4 g2, float mu,
                                            float rx, float ry, float rz, float *W) {
    const float4 tg = ldg4(a.tangent + q);
    const float tn = tg.x * g1.x + tg.y * g1.y + tg.z * g1.z;
    float tx = tg.x - tn * g1.x, ty = tg.y - tn * g1.y, tz = tg.z - tn * g1.z;
    const float tinv = 1.f / sqrtf(tx * tx + ty * ty + tz * tz);
    tx *= tinv; ty *= tinv; tz *= tinv;
    const float bx = g1.y * tz - g1.z * ty, by = g1.z * tx - g1.x * tz, bz = g1.x * ty - g1.y * tx;
    const float ot = g0.x * tx + g0.y * ty + g0.z * tz;
    const float ob = g0.x * bx + g0.y * by + g0.z * bz;
    const float jtx = -2.f * (ot * g1.x + mu * tx), jty = -2.f * (ot * g1.y + mu * ty), jtz = -2.f * (ot * g1.z + mu * tz);
    const float jbx = -2.f * (ob * g1.x + mu * bx), jby = -2.f * (ob * g1.y + mu * by), jbz = -2.f * (ob * g1.z + mu * bz);
    const float nt = sqrtf(jtx * jtx + jty * jty + jtz * jtz), nb = sqrtf(jbx * jbx + jby * jby + jbz * jbz);
    const float Lt = nt * g2.z, Lb = nb * g2.w;
    const bool along_t = Lt >= Lb;
    const float Lmin = fminf(Lt, Lb), Lmax = fmaxf(Lt, Lb);
    const float ux = along_t ? jtx / nt : jbx / nb, uy = along_t ? jty / nt : jby / nb,
                uz = along_t ? jtz / nt : jbz / nb;
    const float s = sqrtf(fminf(fmaxf(0.5f * Lmin, 1e-4f), 1.f));
    const float sigma = sqrtf(0.4f * (Lmax * Lmax - Lmin * Lmin));
    constexpr float kX[5] = {0.f, -1.3556261799742659f, 1.3556261799742659f, -2.8569700138728056f,
                             2.8569700138728056f};
    constexpr float kW[5] = {0.53333333333333333f, 0.22207592200561265f, 0.22207592200561265f,
                             0.011257411327720690f, 0.011257411327720690f};
#pragma unroll
    for (int k = 0; k < K; ++k) W[k] = 0.f;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const float o = kX[j] * sigma;
        const float dx = rx + o * ux, dy = ry + o * uy, dz = rz + o * uz;
        const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
        float w[K];
        filtered_weights_only<K>(a, dx * il, dy * il, dz * il, s, w);
#pragma unroll
        for (int k = 0; k < K; ++k) W[k] = fmaf(kW[j], w[k], W[k]);
    }
}

// E1's p_k (step 1 of smooth_and_probs without the colour channels), from
// the weights-only copy: p_1 = U + V W_1, p_k = V W_k.  With COLOUR, also the
// smooth radiance L = E_b c of smooth_and_probs from the colour channels at the
// same taps (one reflection direction, level pair and table fetch for both):
// the same values as smooth_and_probs computes.
template <int K, bool COLOUR = false>
__device__ __forceinline__ void e1_probs(const ShadeArgs &a, float4 g0, float4 g1, float4 g2, float *p,
                                         float *L = nullptr) {
    const float mu_o = g1.x * g0.x + g1.y * g0.y + g1.z * g0.z;
    const float rx = 2.f * mu_o * g1.x - g0.x;
    const float ry = 2.f * mu_o * g1.y - g0.y;
    const float rz = 2.f * mu_o * g1.z - g0.z;
    const float mu_c = fminf(fmaxf(mu_o, 1e-4f), 1.f);
    const float s = sqrtf(sqrtf(g2.z * g2.w));
    const float4 tab = lut_fetch(a.lut, a.lut_n, mu_c, s);  // V, U, A, B
    float tl = (s - a.s_min) * a.s_scale;
    tl = fminf(fmaxf(tl, 0.f), (float)(a.R - 1));
    const int r0 = (int)floorf(tl);
    const int r1 = min(r0 + 1, a.R - 1);
    const float ft = tl - (float)r0;
    const float th_r = acosf(fminf(fmaxf(ry, -1.f), 1.f));
    float ph_r = atan2f(rz, rx);
    if (ph_r < 0.f) ph_r += kTwoPi;
    float W[K];
    filtered_w<K>(a, th_r, ph_r, r0, r1, ft, W);
    p[0] = tab.y + tab.x * W[0];
#pragma unroll
    for (int k = 1; k < K; ++k) p[k] = tab.x * W[k];
    if constexpr (COLOUR) {
        constexpr int C4 = (3 + K + 3) / 4;
        float ch[C4 * 4];
        filtered_channels<K, C4, false>(a, th_r, ph_r, r0, r1, ft, ch);
        const float Eb = g1.w * tab.z + tab.w;
        L[0] = ch[0] * Eb;
        L[1] = ch[1] * Eb;
        L[2] = ch[2] * Eb;
    }
}

// The surrogate's inputs of foreground pixel q with E1's p_k pe (e1_probs),
// handed to `sink` as they are computed (so that no caller has to hold all 64
// at once): sink.group(i, v) receives inputs i .. i+K (E1's p_k at 0, tap t's
// weights at K + t K), sink.log_prior(lp) the K log-priors, and sink.tail(i,
// s) the scalars mu, sqrt a_x, sqrt a_y at 6K .. 6K+3, after which the inputs
// up to 64 are 0.
template <int K, class Sink>
__device__ __forceinline__ void mlp_features(const ShadeArgs &a, long q, float4 g0, float4 g1, float4 g2,
                                             const float *pe, Sink &sink) {
    sink.group(0, pe);
    float lp[K];
#pragma unroll
    for (int k = 0; k < K; ++k) lp[k] = logf(fmaxf(pe[k], kPriorFloor));
    sink.log_prior(lp);
    const float4 tg = ldg4(a.tangent + q);
    const float tn = tg.x * g1.x + tg.y * g1.y + tg.z * g1.z;
    float tx = tg.x - tn * g1.x, ty = tg.y - tn * g1.y, tz = tg.z - tn * g1.z;
    const float tinv = 1.f / sqrtf(tx * tx + ty * ty + tz * tz);
    tx *= tinv; ty *= tinv; tz *= tinv;
    const float bx = g1.y * tz - g1.z * ty, by = g1.z * tx - g1.x * tz, bz = g1.x * ty - g1.y * tx;
    const float mu = g1.x * g0.x + g1.y * g0.y + g1.z * g0.z;
    const float ot = g0.x * tx + g0.y * ty + g0.z * tz;
    const float ob = g0.x * bx + g0.y * by + g0.z * bz;
    const float rx = 2.f * mu * g1.x - g0.x, ry = 2.f * mu * g1.y - g0.y, rz = 2.f * mu * g1.z - g0.z;
    const float jtx = -2.f * (ot * g1.x + mu * tx), jty = -2.f * (ot * g1.y + mu * ty), jtz = -2.f * (ot * g1.z + mu * tz);
    const float jbx = -2.f * (ob * g1.x + mu * bx), jby = -2.f * (ob * g1.y + mu * by), jbz = -2.f * (ob * g1.z + mu * bz);
    const float s = sqrtf(fminf(g2.z, g2.w));
#pragma unroll
    for (int tap = 0; tap < kMlpTaps; ++tap) {
        float dx = rx, dy = ry, dz = rz;
        if (tap > 0) {
            const float sg = (tap & 1) ? 1.f : -1.f;
            const float e = sg * ((tap <= 2) ? g2.z : g2.w);
            dx += e * ((tap <= 2) ? jtx : jbx);
            dy += e * ((tap <= 2) ? jty : jby);
            dz += e * ((tap <= 2) ? jtz : jbz);
        }
        const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
        float w[K];
        filtered_weights_only<K>(a, dx * il, dy * il, dz * il, s, w);
        sink.group(K + tap * K, w);
    }
    const float sc[3] = {mu, sqrtf(g2.z), sqrtf(g2.w)};
    sink.tail(6 * K, sc);
}

// Sink into plain arrays: x[0 .. 64) and lp[0 .. K).
template <int K>
struct ArraySink {
    float *x, *lp;
    __device__ __forceinline__ void group(int i, const float *v) {
#pragma unroll
        for (int k = 0; k < K; ++k) x[i + k] = v[k];
    }
    __device__ __forceinline__ void log_prior(const float *l) {
#pragma unroll
        for (int k = 0; k < K; ++k) lp[k] = l[k];
    }
    __device__ __forceinline__ void tail(int i, const float *v) {
        x[i] = v[0];
        x[i + 1] = v[1];
        x[i + 2] = v[2];
#pragma unroll
        for (int j = 6 * K + 3; j < kMlpIn; ++j) x[j] = 0.f;
    }
};

}  // namespace glint
