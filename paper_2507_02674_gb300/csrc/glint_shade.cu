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
//   4. six samples x (K-1) dual-gated draws: pcg4d hashes of (vertex, level,
//      call, seed) give the uniforms (one call for the root's dither and node
//      1, one per pair of sibling nodes), two hardware exp2 give the gate
//      probabilities, and the Gaussian (normal quantile) is computed for every
//      node, the gates selecting among the outcomes without branches;
//   5. L^_o = L_o sum_k L_k M_k / (N_P sum_k L_k p_k).
// 80 registers per thread (6 blocks of 128 threads per SM) measured fastest.
#include "glint_shade_pixel.cuh"

using namespace glint;

namespace {

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

template <int K, bool INTEGER, bool DEBUG, int EV>
__global__ void __launch_bounds__(kShadeNT, shade_min_blocks(K)) k_shade(ShadeArgs a) {
    const long q = (long)blockIdx.x * kShadeNT + threadIdx.x;
    if (q >= a.npix) return;
    shade_pixel<K, INTEGER, DEBUG, EV>(a, q);
}

// Serving: one launch over a work list of (frame, pixel range) items of many
// frames (resolutions, maps and seeds may differ; K is shared).  Block b
// takes items b, b + G, ...; the frame's arguments are staged in shared memory.
template <int K>
__global__ void __launch_bounds__(kShadeNT, shade_min_blocks(K)) k_serve(const ShadeArgs *__restrict__ frames,
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
            shade_pixel<K, true, false, EV_E1>(sa, item.first + off);
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
    else if (ev == EV_E1A) launch_ke<K, EV_E1A>(args, integer, debug, s);
    else launch_ke<K, EV_E1>(args, integer, debug, s);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_probs(const ShadeArgs &args, int ev, cudaStream_t s) {
    const unsigned grid = (unsigned)((args.npix + kShadeNT - 1) / kShadeNT);
    if (ev == EV_E2) k_probs<K, EV_E2><<<grid, kShadeNT, 0, s>>>(args);
    else if (ev == EV_E1A) k_probs<K, EV_E1A><<<grid, kShadeNT, 0, s>>>(args);
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
    if (p->draw != GLINT_DRAW_DUAL || p->grid != GLINT_GRID_ISOTROPIC) {  // comparison draws, anisotropic grid
        if (launches) *launches = a.npix ? 1 : 0;
        return glint_launch_shade_variant(a, env->d.K, p->count_mode == GLINT_COUNT_INTEGER, p->draw, p->grid, s);
    }
    const int ev = pk_in ? EV_GIVEN : (p->evaluator == GLINT_EVAL_E2 ? EV_E2
                                       : p->evaluator == GLINT_EVAL_E1_ANISO ? EV_E1A : EV_E1);
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
    const int ev = p->evaluator == GLINT_EVAL_E2 ? EV_E2 : p->evaluator == GLINT_EVAL_E1_ANISO ? EV_E1A : EV_E1;
    if (a.npix == 0) return cudaSuccess;
    switch (env->d.K) {
    case 2: return launch_probs<2>(a, ev, s);
    case 4: return launch_probs<4>(a, ev, s);
    case 8: return launch_probs<8>(a, ev, s);
    case 16: return launch_probs<16>(a, ev, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t glint_launch_serve(int K, const ShadeArgs *frames, const ServeItem *items, int nitems, int grid,
                               cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    switch (K) {
    case 2: k_serve<2><<<grid, kShadeNT, 0, s>>>(frames, items, nitems); break;
    case 4: k_serve<4><<<grid, kShadeNT, 0, s>>>(frames, items, nitems); break;
    case 8: k_serve<8><<<grid, kShadeNT, 0, s>>>(frames, items, nitems); break;
    case 16: k_serve<16><<<grid, kShadeNT, 0, s>>>(frames, items, nitems); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
