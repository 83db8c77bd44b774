// Host side of the C ABI declared in include/glint.h: argument checks, device
// allocation, error reporting and launch accounting.  All computation is in
// the kernels of glint_lut.cu, glint_env.cu and glint_shade.cu.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "glint_internal.cuh"

namespace glint {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

glint_status cuda_status(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return GLINT_OK;
    set_error("%s: CUDA error %d (%s)", what, (int)e, cudaGetErrorString(e));
    return (e == cudaErrorMemoryAllocation) ? GLINT_ERR_OOM : GLINT_ERR_CUDA;
}

// Makes `dev` current for the lifetime of the guard and restores the caller's
// device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
        if (!ok) cudaGetLastError();  // a failed switch must not poison later calls' status
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// IEEE 754 binary16 -> float (host).
static float half_to_float(uint16_t h) {
    const uint32_t sign = (uint32_t)(h >> 15) << 31;
    const int e = (h >> 10) & 0x1f;
    const uint32_t m = h & 0x3ffu;
    float v;
    if (e == 0) v = ldexpf((float)m, -24);                       // zero and subnormals
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexpf((float)(m | 0x400u), e - 25);
    uint32_t b;
    memcpy(&b, &v, 4);
    b |= sign;
    memcpy(&v, &b, 4);
    return v;
}
static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace glint

using namespace glint;

// Device address of `bytes` bytes of host memory at `p` when all of them lie
// in one page-locked allocation the current device can address, else NULL.
const void *glint_host_device_view(const void *p, size_t bytes) {
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    const char *last = static_cast<const char *>(p) + bytes - 1;
    if (cudaPointerGetAttributes(&b, last) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    if (b.type != cudaMemoryTypeHost ||
        static_cast<const char *>(b.devicePointer) != static_cast<const char *>(a.devicePointer) + (bytes - 1))
        return nullptr;
    return a.devicePointer;
}

extern "C" {

int glint_abi_version(void) { return GLINT_ABI_VERSION; }

const char *glint_last_error(void) { return g_err; }

glint_status glint_ctx_create(int device, int lut_n, int lut_q, glint_ctx **out) {
    g_err[0] = 0;
    if (!out) { set_error("glint_ctx_create: out is NULL"); return GLINT_ERR_INVALID_ARG; }
    *out = nullptr;
    if (lut_n == 0) lut_n = 64;
    if (lut_q == 0) lut_q = 128;
    if (lut_n < 2 || lut_n > 256 || lut_q < 8 || lut_q > 1024) {
        set_error("glint_ctx_create: lut_n %d must be in [2,256], lut_q %d in [8,1024]", lut_n, lut_q);
        return GLINT_ERR_INVALID_ARG;
    }
    int ndev = 0;
    glint_status st = cuda_status(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (st != GLINT_OK) return st;
    if (device < 0 || device >= ndev) {
        set_error("glint_ctx_create: device %d out of range (%d devices)", device, ndev);
        return GLINT_ERR_INVALID_ARG;
    }
    DeviceGuard guard(device);
    if (!guard.ok) { set_error("glint_ctx_create: cannot select device %d", device); return GLINT_ERR_CUDA; }
    glint_ctx *c = new glint_ctx();
    c->device = device;
    c->lut_n = lut_n;
    c->lut_q = lut_q;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    st = cuda_status(cudaMalloc(&c->lut, sizeof(float4) * (size_t)lut_n * lut_n), "glint_ctx_create: table");
    if (st == GLINT_OK) st = cuda_status(glint_launch_lut(c->lut, lut_n, lut_q, 0), "glint_ctx_create: table kernel");
    if (st == GLINT_OK) st = cuda_status(cudaStreamSynchronize(0), "glint_ctx_create: table kernel");
    if (st != GLINT_OK) {
        cudaFree(c->lut);
        delete c;
        return st;
    }
    c->last_launches = 1;
    *out = c;
    return GLINT_OK;
}

void glint_ctx_destroy(glint_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard guard(ctx->device);
    cudaFree(ctx->lut);
    delete ctx;
}

glint_status glint_lut_export(const glint_ctx *ctx, float *host_dst, size_t bytes) {
    g_err[0] = 0;
    if (!ctx || !host_dst) { set_error("glint_lut_export: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    const size_t need = sizeof(float4) * (size_t)ctx->lut_n * ctx->lut_n;
    if (bytes < need) { set_error("glint_lut_export: need %zu bytes, got %zu", need, bytes); return GLINT_ERR_INVALID_ARG; }
    DeviceGuard guard(ctx->device);
    return cuda_status(cudaMemcpy(host_dst, ctx->lut, need, cudaMemcpyDeviceToHost), "glint_lut_export");
}

static void env_free(glint_env *e) {
    cudaFree(e->flev);
    cudaFree(e->levels);
    cudaFree(e->partial);
    cudaFree(e->done);
    cudaFree(e->pyr);
    cudaFree(e->pyr_rgb4_dev);
    cudaFree(e->pyr_w4_dev);
    cudaFree(e->table);
    cudaFree(e->nvalid);
    cudaFree(e->filt);
    cudaFree(e->filtw);
}

glint_status glint_env_create(glint_ctx *ctx, const glint_env_desc *d, glint_env **out) {
    g_err[0] = 0;
    if (!ctx || !d || !out) { set_error("glint_env_create: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!is_pow2(d->height) || d->height < 2 || d->height > 8192 || d->width != 2 * d->height) {
        set_error("glint_env_create: need width = 2 height, height a power of two in [2, 8192] (got %d x %d)",
                  d->width, d->height);
        return GLINT_ERR_INVALID_ARG;
    }
    if (d->format != GLINT_FMT_RGBA32F && d->format != GLINT_FMT_RGBA16F) {
        set_error("glint_env_create: unknown format %d", d->format);
        return GLINT_ERR_INVALID_ARG;
    }
    if (d->K != 2 && d->K != 4 && d->K != 8 && d->K != 16) {
        set_error("glint_env_create: K = %d, must be 2, 4, 8 or 16", d->K);
        return GLINT_ERR_INVALID_ARG;
    }
    if (!(d->ell > 0.f) || d->scale_log2 < -64 || d->scale_log2 > 64) {
        set_error("glint_env_create: ell must be > 0 and |scale_log2| <= 64");
        return GLINT_ERR_INVALID_ARG;
    }
    if (d->weight_format < GLINT_WFMT_F32 || d->weight_format > GLINT_WFMT_UNORM8) {
        set_error("glint_env_create: unknown weight format %d", d->weight_format);
        return GLINT_ERR_INVALID_ARG;
    }
    if (d->weight_space != GLINT_WEIGHTS_LINEAR && d->weight_space != GLINT_WEIGHTS_LOG) {
        set_error("glint_env_create: unknown weight space %d", d->weight_space);
        return GLINT_ERR_INVALID_ARG;
    }
    if (d->levels < 1 || d->levels > 32 || d->samples < 1 || d->samples > 2048 || !is_pow2(d->out_width) ||
        d->out_width < 4 || d->out_width > 4096) {
        set_error("glint_env_create: levels in [1,32], samples in [1,2048], out_width a power of two in [4,4096]");
        return GLINT_ERR_INVALID_ARG;
    }
    if (!(d->s_min > 0.f) || !(d->s_max >= d->s_min) || !(d->s_max <= 1.f) || (d->levels > 1 && !(d->s_max > d->s_min))) {
        set_error("glint_env_create: need 0 < s_min < s_max <= 1 (s_min = s_max only with one level)");
        return GLINT_ERR_INVALID_ARG;
    }
    DeviceGuard guard(ctx->device);
    glint_env *e = new glint_env();
    e->ctx = ctx;
    e->device = ctx->device;
    e->d = *d;
    e->C = 3 + d->K;
    e->Cpad = (e->C + 3) / 4 * 4;
    // Filtered level r: the power of two nearest (in log2) to 2 pi / alpha_r
    // texels around the equator (texels of about alpha_r radians, the mip
    // chain of real-time IBL), clamped to [min(8, out_width), out_width].
    {
        const int lo = d->out_width < 8 ? d->out_width : 8;
        long long off = 0;
        for (int r = 0; r < d->levels; ++r) {
            const double sr = (d->levels > 1) ? (double)d->s_min + ((double)d->s_max - (double)d->s_min) * r /
                                                                       (d->levels - 1)
                                              : (double)d->s_min;
            const double alpha = sr * sr;
            const double ex = floor(log2(2.0 * 3.14159265358979323846 / alpha) + 0.5);
            double w = ex > 30.0 ? 1073741824.0 : pow(2.0, ex);
            if (w > d->out_width) w = d->out_width;
            if (w < lo) w = lo;
            e->fw[r] = (int)w;
            e->foff[r] = off;
            off += (long long)e->fw[r] * (e->fw[r] / 2);
        }
        e->foff[d->levels] = off;
    }
    int M = 1;
    while ((d->height >> (M - 1)) > 1) ++M;
    e->M = M;
    size_t off4 = 0;  // float4 units
    for (int m = 0; m < M; ++m) {
        const size_t nm = (size_t)(d->width >> m) * (d->height >> m);
        e->pyr_rgb4[m] = off4;
        e->pyr_w4[m] = off4 + nm;
        off4 += nm * (size_t)(e->Cpad / 4);
    }
    const long n = (long)d->width * d->height;
    e->nblk_minmax = (int)std::min<long>((n + 255) / 256, (long)std::max(ctx->num_sms, 1) * 8);
    glint_status st = GLINT_OK;
    auto alloc = [&](void **p, size_t bytes, const char *what) {
        if (st == GLINT_OK) st = cuda_status(cudaMalloc(p, bytes), what);
    };
    alloc((void **)&e->levels, sizeof(float) * (d->K + 2), "glint_env_create: levels");
    alloc((void **)&e->partial, sizeof(float2) * e->nblk_minmax, "glint_env_create: scratch");
    alloc((void **)&e->done, sizeof(unsigned) * 2, "glint_env_create: scratch");
    if (st == GLINT_OK) st = cuda_status(cudaMemset(e->done, 0, sizeof(unsigned) * 2), "glint_env_create: scratch");
    alloc((void **)&e->pyr, sizeof(float4) * off4, "glint_env_create: pyramid");
    alloc((void **)&e->pyr_rgb4_dev, sizeof(size_t) * M, "glint_env_create: pyramid offsets");
    alloc((void **)&e->pyr_w4_dev, sizeof(size_t) * M, "glint_env_create: pyramid offsets");
    alloc((void **)&e->table, sizeof(float4) * (size_t)d->levels * d->samples, "glint_env_create: filter table");
    alloc((void **)&e->nvalid, sizeof(int) * d->levels, "glint_env_create: filter table");
    if (d->weight_format != GLINT_WFMT_F32) {
        const int bytes_w = d->K * (d->weight_format == GLINT_WFMT_UNORM8 ? 1 : 2);
        e->frec4 = 1 + (bytes_w + 15) / 16;
    }
    const size_t frec_bytes = d->weight_format == GLINT_WFMT_F32 ? sizeof(float) * e->Cpad : 16u * (size_t)e->frec4;
    alloc((void **)&e->filt, frec_bytes * (size_t)e->foff[d->levels], "glint_env_create: filtered maps");
    alloc((void **)&e->filtw, sizeof(float4) * ((d->K + 3) / 4) * (size_t)e->foff[d->levels],
          "glint_env_create: filtered weights");
    alloc((void **)&e->flev, sizeof(int2) * d->levels, "glint_env_create: filtered level table");
    if (st == GLINT_OK)
        st = cuda_status(cudaMemcpy(e->pyr_rgb4_dev, e->pyr_rgb4, sizeof(size_t) * M, cudaMemcpyHostToDevice),
                         "glint_env_create: pyramid offsets");
    if (st == GLINT_OK)
        st = cuda_status(cudaMemcpy(e->pyr_w4_dev, e->pyr_w4, sizeof(size_t) * M, cudaMemcpyHostToDevice),
                         "glint_env_create: pyramid offsets");
    if (st == GLINT_OK) {
        std::vector<int2> lev(d->levels);
        for (int r = 0; r < d->levels; ++r) lev[r] = make_int2(e->fw[r], (int)e->foff[r]);
        st = cuda_status(cudaMemcpy(e->flev, lev.data(), sizeof(int2) * d->levels, cudaMemcpyHostToDevice),
                         "glint_env_create: filtered level table");
    }
    if (st == GLINT_OK) st = cuda_status(glint_launch_filter_table(e, 0), "glint_env_create: filter table");
    if (st == GLINT_OK) st = cuda_status(cudaStreamSynchronize(0), "glint_env_create: filter table");
    if (st != GLINT_OK) {
        env_free(e);
        delete e;
        return st;
    }
    *out = e;
    return GLINT_OK;
}

glint_status glint_env_update(glint_env *env, const void *texels, void *stream) {
    g_err[0] = 0;
    if (!env || !texels) { set_error("glint_env_update: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    if (!aligned16(texels) && env->d.format == GLINT_FMT_RGBA32F) {
        set_error("glint_env_update: RGBA32F texels must be 16-byte aligned");
        return GLINT_ERR_INVALID_ARG;
    }
    if (((uintptr_t)texels & 7u) != 0) {
        set_error("glint_env_update: texels must be 8-byte aligned");
        return GLINT_ERR_INVALID_ARG;
    }
    DeviceGuard guard(env->ctx->device);
    int nl = 0;
    glint_status st = cuda_status(glint_launch_env(env, texels, (cudaStream_t)stream, &nl), "glint_env_update");
    env->last_launches = nl;
    return st;
}

glint_status glint_env_levels(const glint_env *env, float *host_L, int K) {
    g_err[0] = 0;
    if (!env || !host_L || K != env->d.K) {
        set_error("glint_env_levels: NULL argument or K mismatch");
        return GLINT_ERR_INVALID_ARG;
    }
    DeviceGuard guard(env->ctx->device);
    return cuda_status(cudaMemcpy(host_L, env->levels, sizeof(float) * K, cudaMemcpyDeviceToHost), "glint_env_levels");
}

glint_status glint_env_export(const glint_env *env, int item, int index, void *host_dst, size_t bytes) {
    g_err[0] = 0;
    if (!env || !host_dst) { set_error("glint_env_export: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    DeviceGuard guard(env->ctx->device);
    const glint_env_desc &d = env->d;
    auto copy = [&](const void *src, size_t n) -> glint_status {
        if (bytes < n) { set_error("glint_env_export: need %zu bytes, got %zu", n, bytes); return GLINT_ERR_INVALID_ARG; }
        return cuda_status(cudaMemcpy(host_dst, src, n, cudaMemcpyDeviceToHost), "glint_env_export");
    };
    auto copy_unpadded = [&](const float *src, size_t texels) -> glint_status {
        const size_t n = texels * env->C * sizeof(float);
        if (bytes < n) { set_error("glint_env_export: need %zu bytes, got %zu", n, bytes); return GLINT_ERR_INVALID_ARG; }
        std::vector<float> tmp(texels * env->Cpad);
        glint_status st = cuda_status(cudaMemcpy(tmp.data(), src, tmp.size() * sizeof(float), cudaMemcpyDeviceToHost),
                                      "glint_env_export");
        if (st != GLINT_OK) return st;
        float *dst = (float *)host_dst;
        for (size_t t = 0; t < texels; ++t)
            memcpy(dst + t * env->C, tmp.data() + t * env->Cpad, sizeof(float) * env->C);
        return GLINT_OK;
    };
    switch (item) {
    case GLINT_ENV_LOHI: return copy(env->levels + d.K, 2 * sizeof(float));
    case GLINT_ENV_LEVELS: return copy(env->levels, d.K * sizeof(float));
    case GLINT_ENV_PYRAMID:
        if (index < 0 || index >= env->M) { set_error("glint_env_export: pyramid level %d out of range", index); return GLINT_ERR_INVALID_ARG; }
    {
        // colour and weights of the level, interleaved into 3 + K floats per texel
        const size_t texels = (size_t)(d.width >> index) * (d.height >> index);
        const size_t n = texels * env->C * sizeof(float);
        if (bytes < n) { set_error("glint_env_export: need %zu bytes, got %zu", n, bytes); return GLINT_ERR_INVALID_ARG; }
        const int kw4 = env->Cpad / 4 - 1;
        std::vector<float> tmp(texels * env->Cpad);
        const float4 *p4 = reinterpret_cast<const float4 *>(env->pyr);
        glint_status st = cuda_status(cudaMemcpy(tmp.data(), p4 + env->pyr_rgb4[index], tmp.size() * sizeof(float),
                                                 cudaMemcpyDeviceToHost), "glint_env_export");
        if (st != GLINT_OK) return st;
        const float *rgb = tmp.data(), *w = tmp.data() + 4 * texels;
        float *dst = (float *)host_dst;
        for (size_t t = 0; t < texels; ++t) {
            memcpy(dst + t * env->C, rgb + 4 * t, sizeof(float) * 3);
            memcpy(dst + t * env->C + 3, w + (size_t)4 * kw4 * t, sizeof(float) * d.K);
        }
        return GLINT_OK;
    }
    case GLINT_ENV_FILTERED: {
        const size_t texels = (size_t)env->foff[d.levels];
        if (d.weight_format == GLINT_WFMT_F32) return copy_unpadded(env->filt, texels);
        // compressed records: decode to the float layout (3 + K floats per texel)
        const size_t n = texels * env->C * sizeof(float);
        if (bytes < n) { set_error("glint_env_export: need %zu bytes, got %zu", n, bytes); return GLINT_ERR_INVALID_ARG; }
        const size_t rb = 16u * (size_t)env->frec4;
        std::vector<unsigned char> raw(texels * rb);
        glint_status st = cuda_status(cudaMemcpy(raw.data(), env->filt, raw.size(), cudaMemcpyDeviceToHost),
                                      "glint_env_export");
        if (st != GLINT_OK) return st;
        float *dst = (float *)host_dst;
        for (size_t t = 0; t < texels; ++t) {
            const unsigned char *r = raw.data() + t * rb;
            memcpy(dst + t * env->C, r, 3 * sizeof(float));
            for (int k = 0; k < d.K; ++k) {
                float v;
                if (d.weight_format == GLINT_WFMT_UNORM8) {
                    v = (float)r[16 + k] * (1.f / 255.f);
                } else {
                    uint16_t c;
                    memcpy(&c, r + 16 + 2 * k, 2);
                    v = d.weight_format == GLINT_WFMT_F16 ? half_to_float(c) : (float)c * (1.f / 65535.f);
                }
                dst[t * env->C + 3 + k] = v;
            }
        }
        return GLINT_OK;
    }
    case GLINT_ENV_FILTERED_WIDTHS: {
        const size_t n = sizeof(int) * d.levels;
        if (bytes < n) { set_error("glint_env_export: need %zu bytes, got %zu", n, bytes); return GLINT_ERR_INVALID_ARG; }
        memcpy(host_dst, env->fw, n);
        return GLINT_OK;
    }
    case GLINT_ENV_TABLE: {
        const size_t nt = sizeof(float4) * (size_t)d.levels * d.samples;
        const size_t n = nt + sizeof(int) * d.levels;
        if (bytes < n) { set_error("glint_env_export: need %zu bytes, got %zu", n, bytes); return GLINT_ERR_INVALID_ARG; }
        glint_status st = cuda_status(cudaMemcpy(host_dst, env->table, nt, cudaMemcpyDeviceToHost), "glint_env_export");
        if (st != GLINT_OK) return st;
        return cuda_status(cudaMemcpy((char *)host_dst + nt, env->nvalid, sizeof(int) * d.levels, cudaMemcpyDeviceToHost),
                           "glint_env_export");
    }
    default:
        set_error("glint_env_export: unknown item %d", item);
        return GLINT_ERR_INVALID_ARG;
    }
}

void glint_env_destroy(glint_env *env) {
    if (!env) return;
    DeviceGuard guard(env->device);  // the context may already be gone
    env_free(env);
    delete env;
}

// Checks shared by glint_shade and glint_reflect_probs.
static glint_status check_shade_args(const char *who, glint_ctx *ctx, const glint_env *env, const glint_gbuffer *g,
                                     const glint_params *p, const void *out) {
    if (!ctx || !env || !g || !p) { set_error("%s: NULL argument", who); return GLINT_ERR_INVALID_ARG; }
    if (env->ctx != ctx) { set_error("%s: environment belongs to another context", who); return GLINT_ERR_INVALID_ARG; }
    if (g->width < 0 || g->height < 0 || (long)g->width * g->height > (1L << 31)) {
        set_error("%s: width %d x height %d out of range", who, g->width, g->height);
        return GLINT_ERR_INVALID_ARG;
    }
    if (p->count_mode != GLINT_COUNT_INTEGER && p->count_mode != GLINT_COUNT_REAL) {
        set_error("%s: unknown count mode %d", who, p->count_mode);
        return GLINT_ERR_INVALID_ARG;
    }
    if (p->evaluator != GLINT_EVAL_E1 && p->evaluator != GLINT_EVAL_E2 && p->evaluator != GLINT_EVAL_MLP &&
        p->evaluator != GLINT_EVAL_GIVEN && p->evaluator != GLINT_EVAL_E1_ANISO) {
        set_error("%s: unknown evaluator %d", who, p->evaluator);
        return GLINT_ERR_INVALID_ARG;
    }
    if (p->evaluator == GLINT_EVAL_E2 && (p->e2_samples < 0 || p->e2_samples > 256)) {
        set_error("%s: e2_samples %d outside [0, 256]", who, p->e2_samples);
        return GLINT_ERR_INVALID_ARG;
    }
    if (p->draw < GLINT_DRAW_DUAL || p->draw > GLINT_DRAW_WANG2020) {
        set_error("%s: unknown draw %d", who, p->draw);
        return GLINT_ERR_INVALID_ARG;
    }
    if (p->draw != GLINT_DRAW_DUAL && p->evaluator != GLINT_EVAL_E1) {
        set_error("%s: the comparison draws run with the E1 evaluator", who);
        return GLINT_ERR_UNSUPPORTED;
    }
    if (p->grid != GLINT_GRID_ISOTROPIC && p->grid != GLINT_GRID_ANISOTROPIC) {
        set_error("%s: unknown grid %d", who, p->grid);
        return GLINT_ERR_INVALID_ARG;
    }
    if (p->grid == GLINT_GRID_ANISOTROPIC && (p->draw != GLINT_DRAW_DUAL || p->evaluator != GLINT_EVAL_E1)) {
        set_error("%s: the anisotropic grid runs with the E1 evaluator and dual-gated draws", who);
        return GLINT_ERR_UNSUPPORTED;
    }
    if (p->draw == GLINT_DRAW_WANG2020 && !(p->gamma > 0.f && p->gamma <= 1.f)) {
        set_error("%s: gamma %g outside (0, 1]", who, (double)p->gamma);
        return GLINT_ERR_INVALID_ARG;
    }
    if (p->evaluator == GLINT_EVAL_MLP) {
        if (!p->mlp) { set_error("%s: the MLP evaluator needs params->mlp", who); return GLINT_ERR_INVALID_ARG; }
        if (glint_mlp_k(p->mlp) != env->d.K) {
            set_error("%s: network K %d differs from the environment's %d", who, glint_mlp_k(p->mlp), env->d.K);
            return GLINT_ERR_INVALID_ARG;
        }
        if (glint_mlp_device(p->mlp) != ctx->device) {
            set_error("%s: network lives on another device", who);
            return GLINT_ERR_INVALID_ARG;
        }
    }
    const long npix = (long)g->width * g->height;
    if (npix > 0) {
        if (!g->view_n0 || !g->normal_f0 || !g->uv_alpha || !out) {
            set_error("%s: NULL G-buffer plane or output", who);
            return GLINT_ERR_INVALID_ARG;
        }
        if (!aligned16(g->view_n0) || !aligned16(g->normal_f0) || !aligned16(g->uv_alpha) || !aligned16(g->duv) ||
            !aligned16(g->tangent)) {
            set_error("%s: G-buffer planes must be 16-byte aligned", who);
            return GLINT_ERR_INVALID_ARG;
        }
        if ((p->evaluator == GLINT_EVAL_E2 || p->evaluator == GLINT_EVAL_MLP ||
             p->evaluator == GLINT_EVAL_E1_ANISO) && !g->tangent) {
            set_error("%s: the E2, MLP and anisotropic E1 evaluators need the tangent plane", who);
            return GLINT_ERR_INVALID_ARG;
        }
    }
    return GLINT_OK;
}

glint_status glint_shade(glint_ctx *ctx, const glint_env *env, const glint_gbuffer *g, const glint_params *p,
                         float *out_rgba, const glint_debug *dbg, void *stream) {
    g_err[0] = 0;
    glint_status st = check_shade_args("glint_shade", ctx, env, g, p, out_rgba);
    if (st != GLINT_OK) return st;
    const long npix = (long)g->width * g->height;
    if (npix > 0) {
        if (!g->duv) { set_error("glint_shade: NULL duv plane"); return GLINT_ERR_INVALID_ARG; }
        if (!aligned16(out_rgba)) { set_error("glint_shade: output must be 16-byte aligned"); return GLINT_ERR_INVALID_ARG; }
        if (p->evaluator == GLINT_EVAL_GIVEN && (!p->p_scratch || ((uintptr_t)p->p_scratch & 3u))) {
            set_error("glint_shade: the GIVEN evaluator needs params->p_scratch (width*height*K floats)");
            return GLINT_ERR_INVALID_ARG;
        }
    }
    DeviceGuard guard(ctx->device);
    if (p->evaluator == GLINT_EVAL_MLP) {  // inputs, network and draws in one kernel
        st = cuda_status(glint_launch_shade_mlp(ctx, env, g, p, out_rgba, dbg, (cudaStream_t)stream),
                         "glint_shade: MLP");
        ctx->last_launches = npix > 0 ? 1 : 0;
        return st;
    }
    int nl = 0;
    const float *pk_in = p->evaluator == GLINT_EVAL_GIVEN ? p->p_scratch : nullptr;
    st = cuda_status(glint_launch_shade(ctx, env, g, p, pk_in, out_rgba, dbg, (cudaStream_t)stream, &nl),
                     "glint_shade");
    ctx->last_launches = nl;
    return st;
}

// ---------------------------------------------------------------------------
// Shading a frame held in host memory: bands of whole rows, uploaded on the
// pipe's upload stream, shaded on the caller's stream, downloaded on the
// pipe's download stream.  Slot s of the staging is reused by every band
// b = s (mod slots); four events per slot order the reuse:
//   uploaded[s]   the band's planes are on the device      (upload -> shade)
//   shaded[s]     the shading has read the planes           (shade -> next upload)
//   downloaded[s] the output has left the slot              (download -> next shade)
// ---------------------------------------------------------------------------
struct glint_hostpipe {
    static constexpr int kMaxSlots = 16;
    glint_ctx *ctx = nullptr;
    int device = 0;
    long band = 0;                 // pixels per slot
    int slots = 0;
    char *mem = nullptr;           // slots x 6 planes x band float4
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t entry = nullptr;
    cudaEvent_t uploaded[kMaxSlots] = {}, shaded[kMaxSlots] = {}, downloaded[kMaxSlots] = {};
    int last_launches = 0;
    int last_in_place = 0;
    float4 *plane(int slot, int i) const {  // i = 0..4 inputs, 5 output
        return reinterpret_cast<float4 *>(mem) + ((size_t)slot * 6 + i) * (size_t)band;
    }
};

static void hostpipe_free(glint_hostpipe *hp) {
    if (hp->up) cudaStreamSynchronize(hp->up);
    if (hp->down) cudaStreamSynchronize(hp->down);
    for (int s = 0; s < glint_hostpipe::kMaxSlots; ++s) {
        if (hp->uploaded[s]) cudaEventDestroy(hp->uploaded[s]);
        if (hp->shaded[s]) cudaEventDestroy(hp->shaded[s]);
        if (hp->downloaded[s]) cudaEventDestroy(hp->downloaded[s]);
    }
    if (hp->entry) cudaEventDestroy(hp->entry);
    if (hp->up) cudaStreamDestroy(hp->up);
    if (hp->down) cudaStreamDestroy(hp->down);
    cudaFree(hp->mem);
    delete hp;
}

glint_status glint_hostpipe_create(glint_ctx *ctx, long band_pixels, int slots, glint_hostpipe **out) {
    g_err[0] = 0;
    if (!ctx || !out) { set_error("glint_hostpipe_create: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    *out = nullptr;
    if (band_pixels < 1 || band_pixels > (1L << 28) || slots < 2 || slots > glint_hostpipe::kMaxSlots) {
        set_error("glint_hostpipe_create: band_pixels %ld must be in [1, 2^28], slots %d in [2, %d]", band_pixels, slots,
                  glint_hostpipe::kMaxSlots);
        return GLINT_ERR_INVALID_ARG;
    }
    DeviceGuard guard(ctx->device);
    if (!guard.ok) { set_error("glint_hostpipe_create: cannot select device %d", ctx->device); return GLINT_ERR_CUDA; }
    glint_hostpipe *hp = new glint_hostpipe();
    hp->ctx = ctx;
    hp->device = ctx->device;
    hp->band = band_pixels;
    hp->slots = slots;
    glint_status st = cuda_status(cudaMalloc(&hp->mem, sizeof(float4) * 6 * (size_t)slots * (size_t)band_pixels),
                                  "glint_hostpipe_create: staging");
    if (st == GLINT_OK) st = cuda_status(cudaStreamCreateWithFlags(&hp->up, cudaStreamNonBlocking), "glint_hostpipe_create");
    if (st == GLINT_OK) st = cuda_status(cudaStreamCreateWithFlags(&hp->down, cudaStreamNonBlocking), "glint_hostpipe_create");
    if (st == GLINT_OK) st = cuda_status(cudaEventCreateWithFlags(&hp->entry, cudaEventDisableTiming), "glint_hostpipe_create");
    for (int s = 0; s < slots && st == GLINT_OK; ++s) {
        st = cuda_status(cudaEventCreateWithFlags(&hp->uploaded[s], cudaEventDisableTiming), "glint_hostpipe_create");
        if (st == GLINT_OK) st = cuda_status(cudaEventCreateWithFlags(&hp->shaded[s], cudaEventDisableTiming), "glint_hostpipe_create");
        if (st == GLINT_OK) st = cuda_status(cudaEventCreateWithFlags(&hp->downloaded[s], cudaEventDisableTiming), "glint_hostpipe_create");
    }
    if (st != GLINT_OK) {
        hostpipe_free(hp);
        return st;
    }
    *out = hp;
    return GLINT_OK;
}

void glint_hostpipe_destroy(glint_hostpipe *pipe) {
    if (!pipe) return;
    DeviceGuard guard(pipe->device);
    hostpipe_free(pipe);
}

int glint_hostpipe_last_launches(const glint_hostpipe *pipe) { return pipe ? pipe->last_launches : 0; }
int glint_hostpipe_last_in_place(const glint_hostpipe *pipe) { return pipe ? pipe->last_in_place : 0; }


glint_status glint_shade_host(glint_hostpipe *pipe, const glint_env *env, const glint_gbuffer *hg,
                              const glint_params *p, float *out_host, int rows_per_band, unsigned flags,
                              void *stream) {
    g_err[0] = 0;
    if (!pipe) { set_error("glint_shade_host: NULL pipe"); return GLINT_ERR_INVALID_ARG; }
    if (flags & ~(GLINT_HOST_INPUTS_READY | GLINT_HOST_STAGED)) {
        set_error("glint_shade_host: unknown flags 0x%x", flags);
        return GLINT_ERR_INVALID_ARG;
    }
    glint_status st = check_shade_args("glint_shade_host", pipe->ctx, env, hg, p, out_host);
    if (st != GLINT_OK) return st;
    pipe->last_launches = 0;
    pipe->last_in_place = 0;
    const int W = hg->width, H = hg->height;
    if ((long)W * H == 0) return GLINT_OK;
    if (!hg->view_n0 || !hg->normal_f0 || !hg->uv_alpha || !hg->duv) {
        set_error("glint_shade_host: NULL G-buffer plane");
        return GLINT_ERR_INVALID_ARG;
    }
    const bool with_tangent = hg->tangent != nullptr;
    DeviceGuard guard(pipe->device);
    if (!guard.ok) { set_error("glint_shade_host: cannot select device %d", pipe->device); return GLINT_ERR_CUDA; }
    if (!(flags & GLINT_HOST_STAGED)) {
        // in place: every buffer in page-locked memory this device addresses
        const size_t plane_bytes = sizeof(float4) * (size_t)W * H;
        const float *src[5] = {hg->view_n0, hg->normal_f0, hg->uv_alpha, hg->duv, hg->tangent};
        const void *dv[6] = {};
        bool in_place = true;
        for (int i = 0; i < 5 && in_place; ++i) {
            if (i == 4 && !with_tangent) break;
            dv[i] = glint_host_device_view(src[i], plane_bytes);
            in_place = dv[i] != nullptr;
        }
        if (in_place) {
            dv[5] = glint_host_device_view(out_host, plane_bytes);
            in_place = dv[5] != nullptr;
        }
        if (in_place) {
            glint_gbuffer g = {static_cast<const float *>(dv[0]), static_cast<const float *>(dv[1]),
                               static_cast<const float *>(dv[2]), static_cast<const float *>(dv[3]), W, H,
                               with_tangent ? static_cast<const float *>(dv[4]) : nullptr};
            st = glint_shade(pipe->ctx, env, &g, p, static_cast<float *>(const_cast<void *>(dv[5])), nullptr, stream);
            pipe->last_launches = pipe->ctx->last_launches;
            pipe->last_in_place = 1;
            return st;
        }
    }
    if ((long)W > pipe->band) {
        set_error("glint_shade_host: a row of %d pixels does not fit a band of %ld", W, pipe->band);
        return GLINT_ERR_INVALID_ARG;
    }
    const long cap_rows = pipe->band / W;
    long rpb = rows_per_band;
    if (rpb < 0 || rpb > cap_rows) {
        set_error("glint_shade_host: rows_per_band %d outside [0, %ld] for width %d and bands of %ld pixels",
                  rows_per_band, cap_rows, W, pipe->band);
        return GLINT_ERR_INVALID_ARG;
    }
    if (rpb == 0) rpb = std::min(cap_rows, std::max(1L, ((long)H + 7) / 8));
    const int K = env->d.K;
    cudaStream_t cs = (cudaStream_t)stream;
    if (!(flags & GLINT_HOST_INPUTS_READY)) {  // uploads after the stream's earlier work
        st = cuda_status(cudaEventRecord(pipe->entry, cs), "glint_shade_host: entry");
        if (st == GLINT_OK) st = cuda_status(cudaStreamWaitEvent(pipe->up, pipe->entry, 0), "glint_shade_host: entry");
    }
    const long nb = ((long)H + rpb - 1) / rpb;
    const float *src[5] = {hg->view_n0, hg->normal_f0, hg->uv_alpha, hg->duv, hg->tangent};
    int launches = 0;
    for (long b = 0; b < nb && st == GLINT_OK; ++b) {
        const int s = (int)(b % pipe->slots);
        const long r0 = b * rpb;
        const int rows = (int)std::min(rpb, (long)H - r0);
        const size_t off = (size_t)r0 * W, n = (size_t)rows * W;
        // upload once the shading of the slot's previous band has read it
        st = cuda_status(cudaStreamWaitEvent(pipe->up, pipe->shaded[s], 0), "glint_shade_host: upload");
        for (int i = 0; i < 5 && st == GLINT_OK; ++i) {
            if (i == 4 && !with_tangent) break;
            st = cuda_status(cudaMemcpyAsync(pipe->plane(s, i), src[i] + 4 * off, sizeof(float4) * n,
                                             cudaMemcpyDefault, pipe->up), "glint_shade_host: upload");
        }
        if (st == GLINT_OK) st = cuda_status(cudaEventRecord(pipe->uploaded[s], pipe->up), "glint_shade_host: upload");
        // shade once the planes are there and the slot's previous output has left
        if (st == GLINT_OK) st = cuda_status(cudaStreamWaitEvent(cs, pipe->uploaded[s], 0), "glint_shade_host: shade");
        if (st == GLINT_OK) st = cuda_status(cudaStreamWaitEvent(cs, pipe->downloaded[s], 0), "glint_shade_host: shade");
        if (st != GLINT_OK) break;
        glint_gbuffer g = {reinterpret_cast<const float *>(pipe->plane(s, 0)),
                           reinterpret_cast<const float *>(pipe->plane(s, 1)),
                           reinterpret_cast<const float *>(pipe->plane(s, 2)),
                           reinterpret_cast<const float *>(pipe->plane(s, 3)), W, rows,
                           with_tangent ? reinterpret_cast<const float *>(pipe->plane(s, 4)) : nullptr};
        glint_params pb = *p;
        if (pb.p_scratch) pb.p_scratch = p->p_scratch + off * (size_t)K;
        float *outb = reinterpret_cast<float *>(pipe->plane(s, 5));
        st = glint_shade(pipe->ctx, env, &g, &pb, outb, nullptr, stream);
        if (st != GLINT_OK) break;
        launches += pipe->ctx->last_launches;
        st = cuda_status(cudaEventRecord(pipe->shaded[s], cs), "glint_shade_host: shade");
        // download once shaded
        if (st == GLINT_OK) st = cuda_status(cudaStreamWaitEvent(pipe->down, pipe->shaded[s], 0), "glint_shade_host: download");
        if (st == GLINT_OK)
            st = cuda_status(cudaMemcpyAsync(out_host + 4 * off, outb, sizeof(float4) * n, cudaMemcpyDefault,
                                             pipe->down), "glint_shade_host: download");
        if (st == GLINT_OK) st = cuda_status(cudaEventRecord(pipe->downloaded[s], pipe->down), "glint_shade_host: download");
    }
    // the caller's stream completes after the last download (the download stream is in order)
    if (st == GLINT_OK)
        st = cuda_status(cudaStreamWaitEvent(cs, pipe->downloaded[(int)((nb - 1) % pipe->slots)], 0),
                         "glint_shade_host: completion");
    pipe->last_launches = launches;
    return st;
}

glint_status glint_reflect_probs(glint_ctx *ctx, const glint_env *env, const glint_gbuffer *g,
                                 const glint_params *p, float *p_out, void *stream) {
    g_err[0] = 0;
    glint_status st = check_shade_args("glint_reflect_probs", ctx, env, g, p, p_out);
    if (st != GLINT_OK) return st;
    if (((uintptr_t)p_out & 3u)) { set_error("glint_reflect_probs: p_out misaligned"); return GLINT_ERR_INVALID_ARG; }
    if (p->evaluator == GLINT_EVAL_GIVEN) {
        set_error("glint_reflect_probs: the GIVEN evaluator has nothing to compute");
        return GLINT_ERR_INVALID_ARG;
    }
    DeviceGuard guard(ctx->device);
    if (p->evaluator == GLINT_EVAL_MLP)
        st = cuda_status(glint_launch_mlp_infer(ctx, env, p->mlp, g, p_out, (cudaStream_t)stream), "glint_reflect_probs");
    else
        st = cuda_status(glint_launch_probs(ctx, env, g, p, p_out, (cudaStream_t)stream), "glint_reflect_probs");
    ctx->last_launches = (long)g->width * g->height > 0 ? 1 : 0;
    return st;
}

glint_status glint_normal_quantile(const float *p, float *z, long n, void *stream) {
    g_err[0] = 0;
    if (n < 0 || (n > 0 && (!p || !z))) {
        set_error("glint_normal_quantile: NULL argument or negative count");
        return GLINT_ERR_INVALID_ARG;
    }
    return cuda_status(glint_launch_quantile(p, z, n, (cudaStream_t)stream), "glint_normal_quantile");
}

int glint_env_last_launches(const glint_env *env) { return env ? env->last_launches : 0; }
int glint_ctx_last_launches(const glint_ctx *ctx) { return ctx ? ctx->last_launches : 0; }

}  // extern "C"
