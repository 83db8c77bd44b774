// glint_env_levels_noalloc: the radiance levels of an environment map computed
// without allocating any memory.
//
// Some callers cannot call cudaMalloc: frame loops that must never stall on an
// allocation (cudaMalloc and cudaFree may synchronise the device), and host
// applications such as engines and plug-in hosts that own every device
// allocation through their own allocator.  For them the per-block (min, max)
// partial results of the brightness reduction live in the fixed array below,
// which every GPU that loads this library holds until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Nothing in it needs to start at zero: each block overwrites its
// own slot before the levels kernel of the same call reads it.  Calls whose
// work overlaps on the GPU (e.g. on two streams at once) race on the array.
#include "glint_internal.cuh"

using namespace glint;

namespace {

constexpr int kNT = 256;
constexpr int kMaxBlocks = GLINT_NOALLOC_MAX_BLOCKS;

// Scratch: one (min, max) pair per reduction block, kMaxBlocks * 8 bytes.
static __device__ __align__(256) float2 g_noalloc_partial[kMaxBlocks];

__device__ __forceinline__ float4 load_texel_na(const void *texels, int fmt, long i) {
    if (fmt == GLINT_FMT_RGBA16F) {
        const uint2 raw = __ldg(reinterpret_cast<const uint2 *>(texels) + i);
        const float2 f0 = __half22float2(*reinterpret_cast<const __half2 *>(&raw.x));
        const float2 f1 = __half22float2(*reinterpret_cast<const __half2 *>(&raw.y));
        return make_float4(f0.x, f0.y, f1.x, f1.y);
    }
    return __ldg(reinterpret_cast<const float4 *>(texels) + i);
}

__global__ void __launch_bounds__(kNT) k_minmax_na(const void *__restrict__ texels, int fmt, long n, float scale,
                                                     float2 *__restrict__ partial) {
    float lo = INFINITY, hi = -INFINITY;
    for (long i = (long)blockIdx.x * kNT + threadIdx.x; i < n; i += (long)gridDim.x * kNT) {
        const float4 t = load_texel_na(texels, fmt, i);
        const float y = fmaxf(0.2126f * (t.x * scale) + 0.7152f * (t.y * scale) + 0.0722f * (t.z * scale), 0.f);
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
    if (threadIdx.x == 0) {
        float2 v = red[0];
        for (int w = 1; w < kNT / 32; ++w) {
            v.x = fminf(v.x, red[w].x);
            v.y = fmaxf(v.y, red[w].y);
        }
        partial[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(kNT) k_levels_na(const float2 *__restrict__ partial, int nblk, int K, float ell,
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
        for (int k = 2; k <= K; ++k) levels[k - 1] = lo * exp2f((float)(k - 1) / (float)(K - 1) * l2);
        levels[K] = lo;
        levels[K + 1] = hi;
    }
}

// Device address of the scratch array in the current context.  In host code
// g_noalloc_partial names a host-side stand-in, not device memory, so the
// address is asked of the runtime on every call: a cached address would go
// stale when the module is loaded again (after cudaDeviceReset, or in another
// context that a plug-in host makes current), and the query allocates nothing.
glint_status scratch_address(float2 **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess) return cuda_status(e, "glint_env_levels_noalloc: cudaGetSymbolAddress");
    *out = reinterpret_cast<float2 *>(p);
    return GLINT_OK;
}

}  // namespace

extern "C" glint_status glint_env_levels_noalloc(int device, const void *texels, int width, int height, int format,
                                                 int scale_log2, int K, float ell, float *levels_out, void *stream) {
    set_error("%s", "");
    if (!texels || !levels_out) {
        set_error("glint_env_levels_noalloc: NULL texels or output");
        return GLINT_ERR_INVALID_ARG;
    }
    const bool pow2 = height > 0 && (height & (height - 1)) == 0;
    if (!pow2 || height < 2 || width != 2 * height) {
        set_error("glint_env_levels_noalloc: need width = 2 height, height a power of two (got %d x %d)", width,
                  height);
        return GLINT_ERR_INVALID_ARG;
    }
    if (height > GLINT_NOALLOC_MAX_HEIGHT) {
        set_error("glint_env_levels_noalloc: height %d exceeds the maximum %d of the fixed scratch array", height,
                  GLINT_NOALLOC_MAX_HEIGHT);
        return GLINT_ERR_INVALID_ARG;
    }
    if (format != GLINT_FMT_RGBA32F && format != GLINT_FMT_RGBA16F) {
        set_error("glint_env_levels_noalloc: unknown format %d", format);
        return GLINT_ERR_INVALID_ARG;
    }
    if (K != 2 && K != 4 && K != 8 && K != 16) {
        set_error("glint_env_levels_noalloc: K = %d, must be 2, 4, 8 or 16", K);
        return GLINT_ERR_INVALID_ARG;
    }
    if (!(ell > 0.f) || scale_log2 < -64 || scale_log2 > 64) {
        set_error("glint_env_levels_noalloc: ell must be > 0 and |scale_log2| <= 64");
        return GLINT_ERR_INVALID_ARG;
    }
    const size_t align = (format == GLINT_FMT_RGBA32F) ? 16u : 8u;
    if (((uintptr_t)texels % align) != 0 || ((uintptr_t)levels_out & 3u) != 0) {
        set_error("glint_env_levels_noalloc: misaligned texels or output");
        return GLINT_ERR_INVALID_ARG;
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != device) {
        glint_status st = cuda_status(cudaSetDevice(device), "glint_env_levels_noalloc: cudaSetDevice");
        if (st != GLINT_OK) return st;
    }
    float2 *partial = nullptr;
    glint_status st = scratch_address(&partial);
    if (st == GLINT_OK) {
        const long n = (long)width * height;
        const int nblk = (int)((n + kNT - 1) / kNT < kMaxBlocks ? (n + kNT - 1) / kNT : kMaxBlocks);
        const float scale = ldexpf(1.f, scale_log2);
        cudaStream_t s = (cudaStream_t)stream;
        k_minmax_na<<<nblk, kNT, 0, s>>>(texels, format, n, scale, partial);
        k_levels_na<<<1, kNT, 0, s>>>(partial, nblk, K, ell, levels_out);
        st = cuda_status(cudaGetLastError(), "glint_env_levels_noalloc: launch");
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return st;
}
