// Internal declarations of the CUDA library (not part of the C ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "glint.h"

namespace glint {

// Resident blocks per SM of the shading kernels (k_shade, k_serve,
// k_shade_var; 128 threads each), their launch bound and the serving grid's
// unit.  Six blocks give 80 registers a thread: the per-node draw code
// spills at 64 registers (eight blocks), and a wider budget leaves too few
// warps to fill the issue slots (1080p frame, K = 8: 0.378 ms at 8 blocks,
// 0.342 ms at 6, 0.354 ms at 5, 0.403 ms at 4).
constexpr int kShadeMinBlocks = 6;
// K = 16 (15 draws a pixel, 16-entry arrays) spills 232 bytes at 80
// registers; four blocks (128 registers) cut that to 40 and the 3840 x 2160
// grazing frame from 1.393 to 1.320 ms (five blocks: 1.398 ms).
constexpr int shade_min_blocks(int K) { return K >= 16 ? 4 : kShadeMinBlocks; }

constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kInvTwoPi = 0.159154943091895335769f;
constexpr float kInvPi = 0.318309886183790671538f;
// Bias constant of the small-p fix of Sec. 5, eps = 10^-3.54, and log2(1 - eps).
constexpr float kEps = 2.88403156446293e-4f;
constexpr float kLog2OneMinusEps = -4.161378019489348e-4f;
// Largest FP32 value below 2^32: N_P saturates here so counts fit in uint32.
constexpr float kMaxCount = 4294967040.0f;

void set_error(const char *fmt, ...);
glint_status cuda_status(cudaError_t e, const char *what);

}  // namespace glint

struct glint_ctx {
    int device = 0;
    int num_sms = 0;
    int lut_n = 64;
    int lut_q = 128;
    float4 *lut = nullptr;  // lut_n * lut_n nodes: (V, U, A, B)
    int last_launches = 0;
};

struct glint_env {
    glint_ctx *ctx = nullptr;
    int device = 0;            // ctx->device, kept for destruction after the context
    glint_env_desc d{};
    int C = 0;      // 3 + K channels
    int Cpad = 0;   // channels padded to a multiple of 4
    int M = 0;      // pyramid levels
    int nblk_minmax = 0;
    float *levels = nullptr;   // K levels, then lo, hi
    float2 *partial = nullptr; // scratch: per-block (min, max) of the brightness
    unsigned *done = nullptr;  // scratch: two counters of finished blocks (min/max, pyramid), 0 between updates
    float *pyr = nullptr;      // pyramid, all levels, Cpad floats per texel
    // Pyramid level m, in float4 units of `pyr`: its n_m texels' colour (R, G, B, 0)
    // at pyr_rgb4[m], then their weights W_1 .. W_K (Cpad/4 - 1 float4 per texel,
    // zero past K) at pyr_w4[m] = pyr_rgb4[m] + n_m.  n_m is even, so at K = 8
    // every texel's 32 bytes of weights are 32-byte aligned.
    size_t pyr_rgb4[24] = {};
    size_t pyr_w4[24] = {};
    size_t *pyr_rgb4_dev = nullptr;  // the same offsets on the device
    size_t *pyr_w4_dev = nullptr;
    float4 *table = nullptr;   // R x S filter samples (built once at creation)
    int *nvalid = nullptr;     // R valid sample counts
    float *filt = nullptr;     // filtered levels, concatenated: Cpad floats per texel (F32 weights) or
                               // records of frec4 x 16 bytes (compressed weights)
    int frec4 = 0;             // 16-byte units per texel record of a compressed weight format
    float4 *filtw = nullptr;   // the filtered weights alone, ceil(K/4) float4 per filtered texel (as decoded
                               // from the stored format): the surrogate's input look-ups read only these
    int fw[33] = {};           // width of filtered level r (height fw/2)
    long long foff[33] = {};   // first texel of level r in filt; foff[R] = total
    int2 *flev = nullptr;      // device copy of (width, first texel) per level
    int last_launches = 0;
};

namespace glint {

// ---------------------------------------------------------------- device helpers

// pcg4d hash (Jarzynski & Olano, "Hash Functions for GPU Rendering", JCGT 2020).
__device__ __forceinline__ uint4 pcg4d(uint4 v) {
    v.x = v.x * 1664525u + 1013904223u;
    v.y = v.y * 1664525u + 1013904223u;
    v.z = v.z * 1664525u + 1013904223u;
    v.w = v.w * 1664525u + 1013904223u;
    v.x += v.y * v.w; v.y += v.z * v.x; v.z += v.x * v.y; v.w += v.y * v.z;
    v.x ^= v.x >> 16; v.y ^= v.y >> 16; v.z ^= v.z >> 16; v.w ^= v.w >> 16;
    v.x += v.y * v.w; v.y += v.z * v.x; v.z += v.x * v.y; v.w += v.y * v.z;
    return v;
}

// Uniform in (0,1) from the top 23 bits m of a hash word, (2m+1) 2^-24: exact
// in FP32, never 0 or 1, and 1 - xi is exact.  Built without an integer
// conversion: the float with exponent 0 and mantissa m is 1 + m 2^-23, and
// subtracting 1 - 2^-24 leaves (2m+1) 2^-24, which has at most 24 significant
// bits and so is the exact difference (checked for every m).
__device__ __forceinline__ float hash_uniform(uint32_t h) {
    return __fsub_rn(__uint_as_float((h >> 9) | 0x3F800000u), 0x1.fffffep-1f);
}
__device__ __forceinline__ float hash_uniform_complement(uint32_t h) {
    return __fsub_rn(1.f, hash_uniform(h));
}

// Equirect texel coordinates of a direction (texel centres at integers).
__device__ __forceinline__ void dir_to_texel(float dx, float dy, float dz, int W, int H, float &x, float &y) {
    float th = acosf(fminf(fmaxf(dy, -1.f), 1.f));
    float ph = atan2f(dz, dx);
    if (ph < 0.f) ph += kTwoPi;
    x = ph * (kInvTwoPi * (float)W) - 0.5f;
    y = th * (kInvPi * (float)H) - 0.5f;
}

// Bilinear taps of an equirect level: wrap in phi, clamp in theta.  Every
// level's width is a power of two, so the wrap is a mask (two's complement
// also wraps x0 = -1 to W - 1).
struct Taps {
    int i00, i01, i10, i11;
    float w00, w01, w10, w11;
};
__device__ __forceinline__ Taps equirect_taps(float x, float y, int W, int H) {
    float fx0 = floorf(x), fy0 = floorf(y);
    float fx = x - fx0, fy = y - fy0;
    int x0 = (int)fx0, y0 = (int)fy0;
    const int xa = x0 & (W - 1);
    const int xb = (xa + 1) & (W - 1);
    int ya = min(max(y0, 0), H - 1);
    int yb = min(max(y0 + 1, 0), H - 1);
    Taps t;
    t.i00 = ya * W + xa; t.i01 = ya * W + xb; t.i10 = yb * W + xa; t.i11 = yb * W + xb;
    t.w00 = (1.f - fy) * (1.f - fx); t.w01 = (1.f - fy) * fx;
    t.w10 = fy * (1.f - fx); t.w11 = fy * fx;
    return t;
}

__device__ __forceinline__ float4 ldg4(const float4 *p) { return __ldg(p); }
// Two float4 at a 32-byte aligned address in one 256-bit read-only load
// (ld.global.nc.v8, sm_100 and later).
__device__ __forceinline__ void ldg8(const float4 *p, float4 &lo, float4 &hi) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
        : "l"(p));
}

__device__ __forceinline__ float4 fma4(float w, float4 a, float4 acc) {
    acc.x = fmaf(w, a.x, acc.x); acc.y = fmaf(w, a.y, acc.y);
    acc.z = fmaf(w, a.z, acc.z); acc.w = fmaf(w, a.w, acc.w);
    return acc;
}

}  // namespace glint

// Launchers implemented in the .cu files (return cudaGetLastError()).
cudaError_t glint_launch_lut(float4 *lut, int n, int q, cudaStream_t s);
cudaError_t glint_launch_env(glint_env *env, const void *texels, cudaStream_t s, int *launches);
cudaError_t glint_launch_filter_table(glint_env *env, cudaStream_t s);
cudaError_t glint_launch_quantile(const float *p, float *z, long n, cudaStream_t s);
// The MLP surrogate (glint_mlp.cu): p_k of every pixel of `g` into p (npix x K).
cudaError_t glint_launch_mlp_infer(const glint_ctx *ctx, const glint_env *env, const glint_mlp *m,
                                   const glint_gbuffer *g, float *p, cudaStream_t s);
int glint_mlp_k(const glint_mlp *m);
int glint_mlp_device(const glint_mlp *m);
// Device address of `bytes` bytes of host memory at `p` when all of them lie
// in one page-locked allocation the current device can address, else NULL.
const void *glint_host_device_view(const void *p, size_t bytes);
// Serving launches: the shading kernel (glint_shade.cu) and the shading with
// the surrogate fused in (glint_mlp.cu) over a work list; frames/items are device-addressable arrays
// (the server passes page-locked host tables).
namespace glint { struct ShadeArgs; struct ServeItem; }
cudaError_t glint_launch_serve(int K, const glint::ShadeArgs *frames, const glint::ServeItem *items, int nitems,
                               int grid, cudaStream_t s);
cudaError_t glint_launch_serve_mlp(int K, int num_sms, const glint::ShadeArgs *frames, const glint::ServeItem *items,
                                   int nitems, cudaStream_t s);
void glint_mlp_weights(const glint_mlp *m, const void **wt, const float **params);
// Shading with a comparison draw (glint_variants.cu).
cudaError_t glint_launch_shade_variant(const glint::ShadeArgs &a, int K, bool integer, int draw, int grid,
                                       cudaStream_t s);
// Shading with the surrogate fused in (inputs, network and draws in one
// kernel; p_k stays on chip).
cudaError_t glint_launch_shade_mlp(const glint_ctx *ctx, const glint_env *env, const glint_gbuffer *g,
                                   const glint_params *p, float *out, const glint_debug *dbg, cudaStream_t s);
// p_k only (E1 or E2), background pixels 0.
cudaError_t glint_launch_probs(const glint_ctx *ctx, const glint_env *env, const glint_gbuffer *g,
                               const glint_params *p, float *p_out, cudaStream_t s);
// pk_in: p_k per pixel (npix x K) to use instead of E1/E2, or NULL.
cudaError_t glint_launch_shade(const glint_ctx *ctx, const glint_env *env, const glint_gbuffer *g,
                               const glint_params *p, const float *pk_in, float *out, const glint_debug *dbg,
                               cudaStream_t s, int *launches);
