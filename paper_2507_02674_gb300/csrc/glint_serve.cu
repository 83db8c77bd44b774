// Serving: continuous batching of glint-shaded frames (no counterpart in the
// paper).  Host runtime: FIFO admission by device memory (first-fit arena over
// one allocation).  A frame whose buffers are all page-locked is shaded in
// place: the kernels read its G-buffer from, and write its result to, host
// memory over the CPU-GPU link, so no frame waits on another's copies; other
// frames are copied in on two upload streams (3840 x 2160-class frames apart
// from the rest) and out on a third.  Each tick plans (frame, pixel range)
// items over the admitted frames whose inputs are on hand (a tile of each,
// then the frames with the fewest pixels left first) and makes one persistent
// shading launch over them (plus the surrogate's fused inference first for
// frames on that path); the tick's tables stay in page-locked memory that the
// kernels read directly.
#include <algorithm>
#include <chrono>
#include <deque>
#include <iterator>
#include <map>
#include <vector>

#include "glint_internal.cuh"
#include "glint_probs.cuh"

using namespace glint;

// ------------------------------------------------------------------ arena
struct glint_arena {
    size_t bytes = 0, align = 256, used = 0;
    std::map<size_t, size_t> free_;  // offset -> size, disjoint, coalesced
    std::map<size_t, size_t> live;   // offset -> size
};

extern "C" {

glint_arena *glint_arena_create(size_t bytes, size_t align) {
    if (align == 0 || (align & (align - 1)) != 0) return nullptr;
    glint_arena *a = new glint_arena();
    a->align = align;
    a->bytes = bytes / align * align;
    if (a->bytes) a->free_[0] = a->bytes;
    return a;
}

void glint_arena_destroy(glint_arena *a) { delete a; }

long long glint_arena_alloc(glint_arena *a, size_t bytes) {
    if (!a || bytes == 0) return -1;
    const size_t need = (bytes + a->align - 1) / a->align * a->align;
    for (auto it = a->free_.begin(); it != a->free_.end(); ++it) {
        if (it->second < need) continue;
        const size_t off = it->first, rest = it->second - need;
        a->free_.erase(it);
        if (rest) a->free_[off + need] = rest;
        a->live[off] = need;
        a->used += need;
        return (long long)off;
    }
    return -1;
}

int glint_arena_free(glint_arena *a, long long offset) {
    if (!a || offset < 0) return -1;
    auto it = a->live.find((size_t)offset);
    if (it == a->live.end()) return -1;
    size_t off = it->first, size = it->second;
    a->live.erase(it);
    a->used -= size;
    auto next = a->free_.lower_bound(off);
    if (next != a->free_.end() && off + size == next->first) {  // merge with the following range
        size += next->second;
        next = a->free_.erase(next);
    }
    if (next != a->free_.begin()) {  // merge with the preceding range
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            prev->second += size;
            return 0;
        }
    }
    a->free_[off] = size;
    return 0;
}

size_t glint_arena_used(const glint_arena *a) { return a ? a->used : 0; }

size_t glint_arena_largest_free(const glint_arena *a) {
    size_t m = 0;
    if (a)
        for (const auto &f : a->free_) m = std::max(m, f.second);
    return m;
}

int glint_plan_tick(long *next, const long *npix, int nframes, long tick_pixels, int tile_pixels, int *item_frame,
                    long *item_first, int *item_count, int max_items) {
    if (!next || !npix || nframes <= 0 || tile_pixels <= 0 || max_items <= 0) return 0;
    int n = 0;
    long planned = 0;
    auto take = [&](int f) {
        const long c = std::min<long>(tile_pixels - next[f] % tile_pixels, npix[f] - next[f]);
        item_frame[n] = f;
        item_first[n] = next[f];
        item_count[n] = (int)c;
        ++n;
        next[f] += c;
        planned += c;
    };
    // every unfinished frame progresses by one tile, so frames admitted later
    // are not starved by large ones ahead of them ...
    for (int f = 0; f < nframes && n < max_items; ++f)
        if (next[f] < npix[f]) take(f);
    // ... then the rest of the budget goes to the frames with the fewest
    // pixels left (admission order among equals): a small frame behind a 4K
    // one finishes in this tick instead of waiting for the 4K frame's ticks
    std::vector<int> order;
    for (int f = 0; f < nframes; ++f)
        if (next[f] < npix[f]) order.push_back(f);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return npix[a] - next[a] < npix[b] - next[b]; });
    for (size_t i = 0; i < order.size() && n < max_items && planned < tick_pixels; ++i) {
        const int f = order[i];
        while (next[f] < npix[f] && n < max_items && planned < tick_pixels) take(f);
    }
    return n;
}

}  // extern "C"

// ------------------------------------------------------------------ server
namespace {

constexpr int kPiece = 1024;  // pixels per staged work item

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Frame {
    long id = 0;
    long env_version = 0;      // version of its map the frame is shaded with
    glint_frame_request req{};
    long npix = 0;
    long next = 0;             // pixels enqueued for shading so far
    long long arena_off = -1;
    float *dev = nullptr;      // base of the frame's device block
    glint_gbuffer gb{};        // device planes
    float *out = nullptr;      // device output
    cudaEvent_t uploaded = nullptr, downloaded = nullptr;
    bool in_place = false;     // shaded where it lies: gb and out address the caller's page-locked buffers
    bool ready = false;        // `uploaded` has completed (or in place): the frame can be planned
    bool copying_back = false; // `downloaded` is recorded (after the copy back, or the last tick if in place)
    double submit_s = 0, admit_s = 0;
};

struct EnvEntry {  // a resident map
    glint_env *env = nullptr;
    const glint_mlp *mlp = nullptr;
    long applied = 0;          // updates applied so far
    long requested = 0;        // updates requested so far
    const void *texels = nullptr;  // the latest requested update's texels (device)
};

// One tick's frame table and work list, in page-locked host memory that the
// kernels read directly (v_* are the device addresses): a table copy would
// queue on the copy engine behind frame uploads.
struct Slot {
    ShadeArgs *h_frames = nullptr, *v_frames = nullptr;
    ServeItem *h_items = nullptr, *v_items = nullptr;
    cudaEvent_t done = nullptr;
    bool used = false;
};

}  // namespace

struct glint_server {
    glint_ctx *ctx = nullptr;
    int device = 0;  // ctx->device, kept for destruction after the context
    int K = 8;
    glint_server_desc d{};
    int max_items = 0;   // planned items per tick at most
    int max_staged = 0;  // staged items per tick at most (planned items after cutting surrogate ones)
    std::chrono::steady_clock::time_point t0;
    char *pool = nullptr;
    glint_arena *arena = nullptr;
    cudaStream_t copy = nullptr;  // uploads of frames above kLargeFrame pixels
    cudaStream_t copy_small = nullptr;  // uploads of the others (never queued behind a large frame's)
    cudaStream_t back = nullptr;  // copies back (never queued behind uploads)
    std::vector<EnvEntry> envs;
    std::deque<Frame> queue;
    std::vector<Frame> active;  // admission order
    std::vector<glint_frame_done> finished;
    std::vector<Slot> slots;
    long tick_no = 0;
    long next_id = 1;
    glint_server_stats st{};
};

namespace {

// Device bytes of a frame: its planes and output, none if shaded in place.
size_t frame_bytes(const glint_frame_request &r, bool in_place) {
    const size_t n = (size_t)r.width * (size_t)r.height;
    const size_t planes = (r.evaluator == GLINT_EVAL_MLP) ? 5 : 4;
    return in_place ? 0 : (planes + 1) * ((n * 16 + 255) / 256 * 256);
}

void free_frame_events(Frame &f) {
    if (f.uploaded) cudaEventDestroy(f.uploaded);
    if (f.downloaded) cudaEventDestroy(f.downloaded);
    f.uploaded = f.downloaded = nullptr;
}

// Moves frames whose copy back has completed to `finished` and frees them.
void retire(glint_server *s) {
    for (size_t i = 0; i < s->active.size();) {
        Frame &f = s->active[i];
        cudaError_t q = f.copying_back ? cudaEventQuery(f.downloaded) : cudaErrorNotReady;
        // "not ready" is a state, not an error: drop it from the last-error slot only
        if (q == cudaErrorNotReady && cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
        if (q == cudaSuccess) {
            s->finished.push_back(glint_frame_done{f.id, f.submit_s, f.admit_s, now_s(s->t0)});
            if (f.arena_off >= 0) glint_arena_free(s->arena, f.arena_off);
            free_frame_events(f);
            s->active.erase(s->active.begin() + (long)i);
            s->st.active -= 1;
        } else {
            ++i;
        }
    }
}

// Frames above this many pixels (3840 x 2160 in the serving mix) upload on
// their own stream, so that a small frame admitted behind one does not wait
// for its ~530 MB upload.
constexpr long kLargeFrame = 1920L * 1080L;
cudaStream_t upload_stream(glint_server *s, const Frame &f) { return f.npix > kLargeFrame ? s->copy : s->copy_small; }

glint_status admit(glint_server *s) {
    while (!s->queue.empty() && (int)s->active.size() < s->d.max_frames) {
        Frame &q = s->queue.front();
        if (s->envs[q.req.env].applied < q.env_version) break;  // FIFO: waits for its map's update
        const size_t bytes = frame_bytes(q.req, q.in_place);
        long long off = -1;
        if (bytes > 0) {
            off = glint_arena_alloc(s->arena, bytes);
            if (off < 0) break;  // FIFO: the head waits until memory frees up
        }
        Frame f = q;
        s->queue.pop_front();
        f.arena_off = off;
        char *p = off >= 0 ? s->pool + off : nullptr;
        glint_status st = GLINT_OK;
        if (f.in_place) {
            f.ready = true;
        } else {
            const size_t plane = ((size_t)f.npix * 16 + 255) / 256 * 256;
            const float *src[5] = {f.req.view_n0, f.req.normal_f0, f.req.uv_alpha, f.req.duv, f.req.tangent};
            float *dst[5] = {};
            const int nplanes = (f.req.evaluator == GLINT_EVAL_MLP) ? 5 : 4;
            for (int i = 0; i < nplanes; ++i) {
                dst[i] = reinterpret_cast<float *>(p);
                p += plane;
                if (st == GLINT_OK)
                    st = cuda_status(cudaMemcpyAsync(dst[i], src[i], (size_t)f.npix * 16, cudaMemcpyHostToDevice,
                                                     upload_stream(s, f)),
                                     "glint_server_tick: upload");
            }
            f.out = reinterpret_cast<float *>(p);
            f.gb = glint_gbuffer{dst[0], dst[1], dst[2], dst[3], f.req.width, f.req.height, dst[4]};
            if (st == GLINT_OK)
                st = cuda_status(cudaEventCreateWithFlags(&f.uploaded, cudaEventDisableTiming), "glint_server_tick");
            if (st == GLINT_OK) st = cuda_status(cudaEventRecord(f.uploaded, upload_stream(s, f)), "glint_server_tick");
        }
        if (st == GLINT_OK) st = cuda_status(cudaEventCreateWithFlags(&f.downloaded, cudaEventDisableTiming), "glint_server_tick");
        if (st != GLINT_OK) {
            if (off >= 0) glint_arena_free(s->arena, off);
            free_frame_events(f);
            return st;
        }
        f.admit_s = now_s(s->t0);
        s->active.push_back(f);
        s->st.queued -= 1;
        s->st.active += 1;
        s->st.used_bytes = glint_arena_used(s->arena);
        s->st.peak_bytes = std::max(s->st.peak_bytes, s->st.used_bytes);
    }
    return GLINT_OK;
}

// Applies each map's latest requested update once no admitted frame still
// needs the previous version (queued frames of the previous version are
// admitted and finished first, in FIFO order).  The update runs on the compute
// stream, so later ticks see the new map.
glint_status apply_updates(glint_server *s, cudaStream_t cs) {
    for (size_t e = 0; e < s->envs.size(); ++e) {
        EnvEntry &en = s->envs[e];
        if (en.applied == en.requested) continue;
        bool busy = false;
        for (const Frame &f : s->active)
            if (f.req.env == (int)e && f.env_version < en.requested) busy = true;
        for (const Frame &f : s->queue)
            if (f.req.env == (int)e && f.env_version < en.requested) busy = true;
        if (busy) continue;
        int nl = 0;
        glint_status st = cuda_status(glint_launch_env(en.env, en.texels, cs, &nl), "glint_server_tick: map update");
        if (st != GLINT_OK) return st;
        en.env->last_launches = nl;
        en.applied = en.requested;
        s->st.launches += nl;
    }
    return GLINT_OK;
}

}  // namespace

extern "C" {

glint_status glint_server_update_env(glint_server *s, int env_id, const void *texels) {
    set_error("%s", "");
    if (!s || !texels) { set_error("glint_server_update_env: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    if (env_id < 0 || env_id >= (int)s->envs.size()) {
        set_error("glint_server_update_env: unknown env %d", env_id);
        return GLINT_ERR_INVALID_ARG;
    }
    EnvEntry &en = s->envs[env_id];
    en.texels = texels;
    en.requested += 1;
    return GLINT_OK;
}

glint_status glint_server_create(glint_ctx *ctx, int K, const glint_server_desc *desc, glint_server **out) {
    set_error("%s", "");
    if (!ctx || !desc || !out) { set_error("glint_server_create: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    *out = nullptr;
    if (K != 2 && K != 4 && K != 8 && K != 16) { set_error("glint_server_create: K = %d", K); return GLINT_ERR_INVALID_ARG; }
    glint_server_desc d = *desc;
    if (d.tick_pixels == 0) d.tick_pixels = 2097152;
    if (d.tile_pixels == 0) d.tile_pixels = 16384;
    if (d.max_frames == 0) d.max_frames = 64;
    if (d.max_inflight_ticks == 0) d.max_inflight_ticks = 2;
    if (d.memory_budget < (1u << 20) || d.tick_pixels < 128 || d.tile_pixels < 128 || d.tile_pixels % 128 ||
        d.max_frames < 1 || d.max_frames > 4096 || d.max_inflight_ticks < 1 || d.max_inflight_ticks > 16 ||
        (d.upload != 0 && d.upload != 1)) {
        set_error("glint_server_create: memory_budget >= 1 MiB, tick_pixels >= 128, tile_pixels a multiple of 128, "
                  "max_frames in [1, 4096], max_inflight_ticks in [1, 16], upload 0 or 1");
        return GLINT_ERR_INVALID_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) { set_error("glint_server_create: cannot select device"); return GLINT_ERR_CUDA; }
    glint_server *s = new glint_server();
    s->ctx = ctx;
    s->device = ctx->device;
    s->K = K;
    s->d = d;
    s->t0 = std::chrono::steady_clock::now();
    // a tick touches each admitted frame's ranges: at most tick_pixels / tile + one partial item per frame
    s->max_items = (int)std::min<long>(d.tick_pixels / d.tile_pixels + 2L * d.max_frames, 1L << 20);
    // a planned item spans at most tile_pixels pixels: cut into kPiece-pixel pieces it gives at most
    // tile_pixels / kPiece + 1 of them
    s->max_staged = s->max_items * (d.tile_pixels / kPiece + 2);
    glint_status st = cuda_status(cudaMalloc(&s->pool, d.memory_budget), "glint_server_create: pool");
    if (st == GLINT_OK) {
        s->arena = glint_arena_create(d.memory_budget, 256);
        if (!s->arena) st = GLINT_ERR_OOM;
    }
    if (st == GLINT_OK) st = cuda_status(cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking), "glint_server_create");
    if (st == GLINT_OK)
        st = cuda_status(cudaStreamCreateWithFlags(&s->copy_small, cudaStreamNonBlocking), "glint_server_create");
    if (st == GLINT_OK) st = cuda_status(cudaStreamCreateWithFlags(&s->back, cudaStreamNonBlocking), "glint_server_create");
    s->slots.resize(d.max_inflight_ticks + 1);
    for (auto &sl : s->slots) {
        if (st != GLINT_OK) break;
        st = cuda_status(cudaMallocHost(&sl.h_frames, sizeof(ShadeArgs) * d.max_frames), "glint_server_create");
        if (st == GLINT_OK) st = cuda_status(cudaMallocHost(&sl.h_items, sizeof(ServeItem) * s->max_staged), "glint_server_create");
        if (st == GLINT_OK)
            st = cuda_status(cudaHostGetDevicePointer(reinterpret_cast<void **>(&sl.v_frames), sl.h_frames, 0),
                             "glint_server_create");
        if (st == GLINT_OK)
            st = cuda_status(cudaHostGetDevicePointer(reinterpret_cast<void **>(&sl.v_items), sl.h_items, 0),
                             "glint_server_create");
        if (st == GLINT_OK) st = cuda_status(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming), "glint_server_create");
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (st != GLINT_OK) {
        glint_server_destroy(s);
        return st;
    }
    *out = s;
    return GLINT_OK;
}

void glint_server_destroy(glint_server *s) {
    if (!s) return;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != s->device && cudaSetDevice(s->device) != cudaSuccess) cudaGetLastError();
    cudaDeviceSynchronize();
    for (auto &f : s->active) free_frame_events(f);
    for (auto &sl : s->slots) {
        cudaFreeHost(sl.h_frames);
        cudaFreeHost(sl.h_items);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    if (s->copy) cudaStreamDestroy(s->copy);
    if (s->copy_small) cudaStreamDestroy(s->copy_small);
    if (s->back) cudaStreamDestroy(s->back);
    cudaFree(s->pool);
    glint_arena_destroy(s->arena);
    if (prev >= 0) cudaSetDevice(prev);
    delete s;
}

glint_status glint_server_add_env(glint_server *s, const glint_env *env, const glint_mlp *mlp, int *env_id) {
    set_error("%s", "");
    if (!s || !env || !env_id) { set_error("glint_server_add_env: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    if (env->ctx != s->ctx || env->d.K != s->K) {
        set_error("glint_server_add_env: environment of another context or K %d (server K %d)", env->d.K, s->K);
        return GLINT_ERR_INVALID_ARG;
    }
    if (mlp && (glint_mlp_k(mlp) != s->K || glint_mlp_device(mlp) != s->ctx->device)) {
        set_error("glint_server_add_env: network K or device differs");
        return GLINT_ERR_INVALID_ARG;
    }
    EnvEntry e;
    e.env = const_cast<glint_env *>(env);
    e.mlp = mlp;
    s->envs.push_back(e);
    *env_id = (int)s->envs.size() - 1;
    return GLINT_OK;
}

glint_status glint_server_submit(glint_server *s, const glint_frame_request *r, long *id) {
    set_error("%s", "");
    if (!s || !r || !id) { set_error("glint_server_submit: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    if (r->env < 0 || r->env >= (int)s->envs.size()) { set_error("glint_server_submit: unknown env %d", r->env); return GLINT_ERR_INVALID_ARG; }
    if (r->width < 1 || r->height < 1 || (long)r->width * r->height > (1L << 31)) {
        set_error("glint_server_submit: width %d x height %d", r->width, r->height);
        return GLINT_ERR_INVALID_ARG;
    }
    if (r->evaluator != GLINT_EVAL_E1 && r->evaluator != GLINT_EVAL_MLP) {
        set_error("glint_server_submit: evaluator %d (E1 or MLP)", r->evaluator);
        return GLINT_ERR_INVALID_ARG;
    }
    if (r->evaluator == GLINT_EVAL_MLP && (!s->envs[r->env].mlp || !r->tangent)) {
        set_error("glint_server_submit: the surrogate path needs the environment's network and a tangent plane");
        return GLINT_ERR_INVALID_ARG;
    }
    if (!r->view_n0 || !r->normal_f0 || !r->uv_alpha || !r->duv || !r->out_rgba) {
        set_error("glint_server_submit: NULL plane or output");
        return GLINT_ERR_INVALID_ARG;
    }
    Frame f;
    f.req = *r;
    f.npix = (long)r->width * r->height;
    if (!s->d.upload) {
        // in place when every buffer is page-locked host memory the device addresses
        int prev = -1;
        cudaGetDevice(&prev);
        if (prev != s->device) cudaSetDevice(s->device);
        const size_t pb = (size_t)f.npix * 16;
        const float *src[5] = {r->view_n0, r->normal_f0, r->uv_alpha, r->duv, r->tangent};
        const int nplanes = (r->evaluator == GLINT_EVAL_MLP) ? 5 : 4;
        const void *dv[5] = {};
        bool ok = true;
        for (int i = 0; i < nplanes && ok; ++i) ok = (dv[i] = glint_host_device_view(src[i], pb)) != nullptr;
        const void *dout = ok ? glint_host_device_view(r->out_rgba, pb) : nullptr;
        if (dout) {
            f.in_place = true;
            f.gb = glint_gbuffer{static_cast<const float *>(dv[0]), static_cast<const float *>(dv[1]),
                                 static_cast<const float *>(dv[2]), static_cast<const float *>(dv[3]), r->width,
                                 r->height, static_cast<const float *>(dv[4])};
            f.out = static_cast<float *>(const_cast<void *>(dout));
        }
        if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
    }
    const size_t bytes = frame_bytes(*r, f.in_place);
    if (bytes > s->arena->bytes) {
        set_error("glint_server_submit: the frame needs %zu bytes, more than the budget %zu", bytes, s->d.memory_budget);
        return GLINT_ERR_INVALID_ARG;
    }
    f.id = s->next_id++;
    f.env_version = s->envs[r->env].requested;
    f.submit_s = now_s(s->t0);
    s->queue.push_back(f);
    s->st.queued += 1;
    *id = f.id;
    return GLINT_OK;
}

glint_status glint_server_tick(glint_server *s, void *stream, int *launched) {
    set_error("%s", "");
    if (launched) *launched = 0;
    if (!s) { set_error("glint_server_tick: NULL server"); return GLINT_ERR_INVALID_ARG; }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->ctx->device) cudaSetDevice(s->ctx->device);
    cudaStream_t cs = (cudaStream_t)stream;
    retire(s);
    glint_status st = apply_updates(s, cs);
    if (st == GLINT_OK) st = admit(s);
    // frames with pixels left whose upload has completed, in admission order:
    // the compute stream never waits on an upload, so a frame still being
    // copied in holds up no other frame's shading
    std::vector<int> idx;
    for (int i = 0; i < (int)s->active.size(); ++i) {
        Frame &f = s->active[i];
        if (f.next >= f.npix) continue;
        if (!f.ready) {
            const cudaError_t q = cudaEventQuery(f.uploaded);
            if (q == cudaErrorNotReady) {
                if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();  // a state, not an error
                continue;
            }
            if (q != cudaSuccess) { st = cuda_status(q, "glint_server_tick: upload"); break; }
            f.ready = true;
        }
        idx.push_back(i);
    }
    int nl = 0;
    if (st == GLINT_OK && !idx.empty()) {
        Slot &sl = s->slots[s->tick_no % s->slots.size()];
        if (sl.used) st = cuda_status(cudaEventSynchronize(sl.done), "glint_server_tick: wait");
        // plan: surrogate-path frames first (their items precede the plain ones)
        std::vector<int> order;
        for (int i : idx) if (s->active[i].req.evaluator == GLINT_EVAL_MLP) order.push_back(i);
        const int n_mlp_frames = (int)order.size();
        for (int i : idx) if (s->active[i].req.evaluator != GLINT_EVAL_MLP) order.push_back(i);
        std::vector<long> next(order.size()), npix(order.size());
        for (size_t j = 0; j < order.size(); ++j) {
            next[j] = s->active[order[j]].next;
            npix[j] = s->active[order[j]].npix;
        }
        std::vector<int> pf(s->max_items), pc(s->max_items);
        std::vector<long> pfirst(s->max_items);
        const int nit = glint_plan_tick(next.data(), npix.data(), (int)order.size(), s->d.tick_pixels,
                                        s->d.tile_pixels, pf.data(), pfirst.data(), pc.data(), s->max_items);
        // items of surrogate-path frames first (stable), grouped by network
        std::vector<int> perm(nit);
        for (int k = 0; k < nit; ++k) perm[k] = k;
        std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) {
            const bool mx = pf[x] < n_mlp_frames, my = pf[y] < n_mlp_frames;
            if (mx != my) return mx;
            if (!mx) return false;
            return s->envs[s->active[order[pf[x]]].req.env].mlp < s->envs[s->active[order[pf[y]]].req.env].mlp;
        });
        // items are cut into pieces of kPiece pixels, so that a tick of a few
        // frames still spreads over every SM
        std::vector<int> it_f, it_c;
        std::vector<long> it_first;
        for (int k = 0; k < nit; ++k) {
            const int j = pf[perm[k]];
            long first = pfirst[perm[k]];
            const long end = first + pc[perm[k]];
            while (first < end) {
                const long c = std::min<long>(kPiece - first % kPiece, end - first);
                it_f.push_back(j);
                it_first.push_back(first);
                it_c.push_back((int)c);
                first += c;
            }
        }
        const int nit_all = (int)it_f.size();
        if (nit_all > s->max_staged) {  // cannot happen with the bound above; refuse rather than overflow
            set_error("glint_server_tick: %d staged items exceed the capacity %d", nit_all, s->max_staged);
            st = GLINT_ERR_UNSUPPORTED;
        }
        // frame table of this tick (frames that received items) and the work list
        std::vector<int> table_of(order.size(), -1);
        int nframes = 0, n_mlp_items = 0;
        for (int k = 0; k < nit_all && st == GLINT_OK; ++k) {
            const int j = it_f[k];
            if (table_of[j] < 0) {
                Frame &f = s->active[order[j]];
                glint_params prm{};
                prm.seed = f.req.seed;
                const glint_env *env = s->envs[f.req.env].env;
                ShadeArgs a = make_args(s->ctx, env, &f.gb, &prm);
                a.out = reinterpret_cast<float4 *>(f.out);
                if (f.req.evaluator == GLINT_EVAL_MLP)
                    glint_mlp_weights(s->envs[f.req.env].mlp, &a.mlp_wt, &a.mlp_params);
                table_of[j] = nframes;
                sl.h_frames[nframes++] = a;

            }
            sl.h_items[k] = ServeItem{table_of[j], it_c[k], it_first[k]};
            if (j < n_mlp_frames) ++n_mlp_items;
        }
        // surrogate path: one launch of the shading with the network fused in
        // over its frames' items (grouped by network), then the plain items
        if (st == GLINT_OK && n_mlp_items > 0) {
            st = cuda_status(glint_launch_serve_mlp(s->K, s->ctx->num_sms, sl.v_frames, sl.v_items, n_mlp_items, cs),
                             "glint_server_tick: shade (surrogate)");
            ++nl;
        }
        if (st == GLINT_OK && nit_all > n_mlp_items) {
            const int grid = std::min(nit_all - n_mlp_items, s->ctx->num_sms * glint::shade_min_blocks(s->K));
            st = cuda_status(glint_launch_serve(s->K, sl.v_frames, sl.v_items + n_mlp_items, nit_all - n_mlp_items,
                                                grid, cs), "glint_server_tick: shade");
            ++nl;
        }
        if (st == GLINT_OK) st = cuda_status(cudaEventRecord(sl.done, cs), "glint_server_tick");
        sl.used = true;
        // progress, and copies back of frames this tick completes
        for (size_t j = 0; j < order.size() && st == GLINT_OK; ++j) {
            Frame &f = s->active[order[j]];
            f.next = next[j];
            if (f.next == f.npix && !f.copying_back) {
                if (f.in_place) {  // this tick's kernels write the result into the caller's buffer
                    st = cuda_status(cudaEventRecord(f.downloaded, cs), "glint_server_tick");
                } else {
                    st = cuda_status(cudaStreamWaitEvent(s->back, sl.done, 0), "glint_server_tick");
                    if (st == GLINT_OK)
                        st = cuda_status(cudaMemcpyAsync(f.req.out_rgba, f.out, (size_t)f.npix * 16,
                                                         cudaMemcpyDeviceToHost, s->back),
                                         "glint_server_tick: download");
                    if (st == GLINT_OK) st = cuda_status(cudaEventRecord(f.downloaded, s->back), "glint_server_tick");
                }
                f.copying_back = true;
            }
        }
        s->tick_no += 1;
        s->st.ticks += 1;
        s->st.launches += nl;
        s->st.items += nit_all;
    }
    if (launched) *launched = nl;
    if (prev >= 0 && prev != s->ctx->device) cudaSetDevice(prev);
    return st;
}

glint_status glint_server_poll(glint_server *s, glint_frame_done *done, int max_done, int *n_done) {
    set_error("%s", "");
    if (!s || !n_done || (max_done > 0 && !done)) { set_error("glint_server_poll: NULL argument"); return GLINT_ERR_INVALID_ARG; }
    retire(s);
    const int n = std::min<int>(max_done, (int)s->finished.size());
    for (int i = 0; i < n; ++i) done[i] = s->finished[i];
    s->finished.erase(s->finished.begin(), s->finished.begin() + n);
    s->st.done += n;
    *n_done = n;
    s->st.used_bytes = glint_arena_used(s->arena);
    return GLINT_OK;
}

glint_status glint_server_stats_get(const glint_server *s, glint_server_stats *out) {
    if (!s || !out) return GLINT_ERR_INVALID_ARG;
    *out = s->st;
    return GLINT_OK;
}

}  // extern "C"
