// Shading with the comparison draws of Sec. 5 and Sec. 7 (single-gated
// Gaussians, Eq. gated; the older form, Eq. oldgated; Wang 2020's
// environment-independent glints) and with the anisotropic grid (footprint
// level, anisotropy and orientation, Sec. 3.3), all with the E1 probabilities
// and the per-pixel intermediates available.  A translation unit of its own so
// that the build compiles it in parallel with the main shading kernels.
#include "glint_shade_pixel.cuh"

namespace {

template <int K, bool INTEGER, int DRAW, int GRID>
__global__ void __launch_bounds__(kShadeNT, shade_min_blocks(K)) k_shade_var(ShadeArgs a) {
    const long q = (long)blockIdx.x * kShadeNT + threadIdx.x;
    if (q >= a.npix) return;
    shade_pixel<K, INTEGER, true, EV_E1, DRAW, GRID>(a, q);
}

template <int K, int DRAW, int GRID>
void launch_kd(const ShadeArgs &a, bool integer, cudaStream_t s) {
    const unsigned grid = (unsigned)((a.npix + kShadeNT - 1) / kShadeNT);
    if (integer) k_shade_var<K, true, DRAW, GRID><<<grid, kShadeNT, 0, s>>>(a);
    else k_shade_var<K, false, DRAW, GRID><<<grid, kShadeNT, 0, s>>>(a);
}

template <int K>
void launch_k(const ShadeArgs &a, bool integer, int draw, int grid, cudaStream_t s) {
    if (grid) launch_kd<K, kDrawDual, 1>(a, integer, s);
    else if (draw == kDrawSingle) launch_kd<K, kDrawSingle, 0>(a, integer, s);
    else if (draw == kDrawSingleOld) launch_kd<K, kDrawSingleOld, 0>(a, integer, s);
    else launch_kd<K, kDrawWang, 0>(a, integer, s);
}

}  // namespace

cudaError_t glint_launch_shade_variant(const ShadeArgs &a, int K, bool integer, int draw, int grid, cudaStream_t s) {
    if (a.npix == 0) return cudaSuccess;
    switch (K) {
    case 2: launch_k<2>(a, integer, draw, grid, s); break;
    case 4: launch_k<4>(a, integer, draw, grid, s); break;
    case 8: launch_k<8>(a, integer, draw, grid, s); break;
    case 16: launch_k<16>(a, integer, draw, grid, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
