/*
 * glint.h -- C ABI of the GB300 (sm_103a) library for real-time image-based
 * lighting of glints (Kneiphof & Klein, "Real-Time Image-based Lighting of
 * Glints", EGSR 2025, arXiv 2507.02674).
 *
 * The library computes, per pixel of a G-buffer, the outgoing radiance of a
 * glittery microfacet surface lit by an environment map (Sec. 4,
 * Eq. iblglints:fin), and the per-environment data it needs: K radiance levels,
 * fuzzy weights and their filtered maps (Sec. 4 "Discrete Radiance Levels",
 * "Fuzzy Indicator Functions", "Integrated NDF").
 *
 * Conventions for every call
 *  - Pointers documented as "device" must point to device memory of the
 *    context's GPU; "host" pointers to ordinary host memory.  The library never
 *    frees caller memory; caller buffers must stay alive until the work enqueued
 *    on `stream` has completed.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls that only enqueue work return before it finishes.
 *  - Every call returns a glint_status.  On failure the call has no effect on
 *    its outputs' ownership, and glint_last_error() returns a message for the
 *    calling thread.  No call aborts the process or throws across the ABI.
 *  - Handles are opaque; they are created and destroyed only by the library.
 *    A handle may be used from one host thread at a time.
 *
 * Memory layouts
 *  - Environment map: equirectangular, `width` x `height` texels, width =
 *    2 height, height a power of two; row y spans polar angle
 *    theta in [pi y/H, pi (y+1)/H] around +y, column x spans
 *    phi in [2 pi x/W, 2 pi (x+1)/W]; direction
 *    (sin th cos ph, cos th, sin th sin ph).  Texels are RGBA, row-major,
 *    float32 (16 bytes) or float16 (8 bytes); radiance = stored value *
 *    2^scale_log2; alpha is ignored.  Values must be finite and >= 0.
 *  - G-buffer: four planes of `width*height` float4, row-major, each 16-byte
 *    aligned (see glint_gbuffer).
 *  - Output: `width*height` float4 (R, G, B, 1), row-major, 16-byte aligned.
 */
#ifndef GLINT_H
#define GLINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GLINT_ABI_VERSION 8
#define GLINT_MAX_K 16

typedef enum glint_status {
    GLINT_OK = 0,
    GLINT_ERR_INVALID_ARG = 1, /* a size, pointer or enum is out of range */
    GLINT_ERR_OOM = 2,         /* device allocation failed */
    GLINT_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the code) */
    GLINT_ERR_NOT_READY = 4,   /* the request cannot be admitted now */
    GLINT_ERR_TIMEOUT = 5,     /* a bounded wait gave up */
    GLINT_ERR_UNSUPPORTED = 6  /* a valid configuration this build does not handle */
} glint_status;

typedef enum glint_format {
    GLINT_FMT_RGBA32F = 0,
    GLINT_FMT_RGBA16F = 1
} glint_format;

typedef enum glint_evaluator {
    GLINT_EVAL_E1 = 0, /* p_k from the filtered maps and tables (Eq. rtiblndf), isotropic sqrt(a_x a_y) */
    GLINT_EVAL_E2 = 1, /* p_k by per-pixel quadrature of the anisotropic NDF (Eq. probhk) */
    GLINT_EVAL_MLP = 2, /* p_k from a trained glint_mlp surrogate of E2 (no counterpart in the paper) */
    GLINT_EVAL_GIVEN = 3, /* p_k supplied by the caller in params->p_scratch (width*height*K floats) */
    GLINT_EVAL_E1_ANISO = 4 /* E1 with multi-tap look-ups along the anisotropic lobe (the multiple filtered
                               look-ups the paper's related work and limitations point to for anisotropy):
                               the lobe of reflected directions as an ellipse with axes J_t a_x, J_b a_y
                               (J the derivatives of the mirror direction with respect to the slope), the
                               filtered maps read at the minor axis' roughness at five Gauss-Hermite nodes
                               along the major axis; needs the tangent plane */
} glint_evaluator;

typedef enum glint_count_mode {
    GLINT_COUNT_INTEGER = 0, /* uint32 counts: N_P dithered at each tree root, Gaussian rounded */
    GLINT_COUNT_REAL = 1     /* real-valued counts, Alg. 1 as printed */
} glint_count_mode;

typedef struct glint_ctx glint_ctx;
typedef struct glint_env glint_env;
typedef struct glint_mlp glint_mlp;

/* ABI version of the loaded library (GLINT_ABI_VERSION). */
int glint_abi_version(void);

/* Message describing the last failed call on the calling thread ("" if none).
 * The pointer stays valid until the next library call on this thread. */
const char *glint_last_error(void);

/* Context on CUDA device `device`.  Builds the microfacet tables on the GPU:
 * for lut_n x lut_n texel-centre nodes over (mu_o, sqrt alpha), the visible
 * reflecting microfacet area over the total microfacet area V = E_D / D_H and
 * its complement U (Sec. 4 Eq. rtiblndf; Sec. 3.2), and the split-sum albedo
 * terms A, B with Schlick F and height-correlated Smith G2 (Sec. 3.4
 * Eq. rtibl), each by a lut_q x lut_q midpoint quadrature.
 * lut_n in [2, 256] (default 64), lut_q in [8, 1024] (default 128); 0 selects
 * the default.  Blocks until the tables are built.  *out is owned by the
 * caller and released with glint_ctx_destroy. */
glint_status glint_ctx_create(int device, int lut_n, int lut_q, glint_ctx **out);

/* Releases the context (NULL is ignored).  All environments made from it must
 * be destroyed first. */
void glint_ctx_destroy(glint_ctx *ctx);

/* Copies the tables to host memory: lut_n * lut_n * 4 floats, row j (sqrt
 * alpha = (j+1/2)/lut_n), column i (mu_o = (i+1/2)/lut_n), channels
 * (V, U, A, B).  `bytes` must be at least that size.  Synchronous. */
glint_status glint_lut_export(const glint_ctx *ctx, float *host_dst, size_t bytes);

/* Description of an environment and of its filtered data. */
typedef struct glint_env_desc {
    int width;        /* texels, = 2 * height */
    int height;       /* power of two, 2 .. 8192 */
    int format;       /* glint_format */
    int scale_log2;   /* radiance = stored * 2^scale_log2, |scale_log2| <= 64 */
    int K;            /* radiance levels: 2, 4, 8 or 16 (Sec. 4, K in {4, 8} in the paper) */
    float ell;        /* lower clip of the minimum brightness (Sec. 4), > 0 */
    int levels;       /* R filtered roughness levels, 1 .. 32 */
    int samples;      /* S filter samples per output texel, 1 .. 2048 */
    int out_width;    /* width of the widest filtered level (power of two, 4 .. 4096); level r is
                         the power of two nearest 2 pi / alpha_r, clamped to
                         [min(8, out_width), out_width], height = width / 2 */
    float s_min;      /* sqrt(alpha) of filtered level 0, > 0 */
    float s_max;      /* sqrt(alpha) of filtered level R-1, >= s_min */
    int weight_space; /* glint_weight_space: interpolation of the fuzzy weights between the two
                         levels bracketing a texel's brightness (Sec. 7 "Linear vs Logarithmic
                         Radiance"; the paper uses linear) */
    int weight_format; /* glint_weight_format: storage of the filtered maps' weights W_k (Sec. 7
                          "Texture Precision") */
} glint_env_desc;

typedef enum glint_weight_format {
    GLINT_WFMT_F32 = 0,     /* float32 channels, (3+K) padded to a multiple of 4 per texel */
    GLINT_WFMT_F16 = 1,     /* per texel: (R, G, B) float32 + K float16 weights (round to nearest even) */
    GLINT_WFMT_UNORM16 = 2, /* ... + K 16-bit codes round(65535 W) */
    GLINT_WFMT_UNORM8 = 3   /* ... + K 8-bit codes round(255 W): the precision the paper finds too low */
} glint_weight_format;

typedef enum glint_weight_space {
    GLINT_WEIGHTS_LINEAR = 0, /* w = (Y - L_j) / (L_{j+1} - L_j) (Eq. wkdefpractice) */
    GLINT_WEIGHTS_LOG = 1     /* w = (ln Y - ln L_j) / (ln L_{j+1} - ln L_j); linear below L_2 (L_1 = 0) */
} glint_weight_space;

/* Allocates an environment's device buffers (levels, weights pyramid,
 * filtered maps, scratch) for the given description and builds the filter's
 * sample table (it depends only on the description); blocks until done.  The
 * map itself is processed by glint_env_update.  *out is released with
 * glint_env_destroy. */
glint_status glint_env_create(glint_ctx *ctx, const glint_env_desc *desc, glint_env **out);

/* Recomputes all per-environment data from `texels` (device; width * height
 * RGBA texels in desc.format) on `stream`, allocating nothing:
 *   1. brightness Y = Rec. 709 luminance, lo = max(min Y, ell), hi = max Y
 *      (Sec. 4 "Discrete Radiance Levels");
 *   2. levels L_1 = 0, L_k = exp(lerp(ln lo, ln hi, (k-1)/(K-1)));
 *   3. per texel the fuzzy weights of the two bracketing levels
 *      (Eq. wkdefpractice), giving channels (R, G, B, w_1 .. w_K);
 *   4. a solid-angle weighted 2x2 pyramid of those channels;
 *   5. for each of R roughness levels the map filtered with the kernel
 *      p_{L_i} ~ D(h) under n = v = r (Sec. 3.4 Eq. rtibl, Sec. 4
 *      Eq. rtiblndf) by filtered importance sampling with S Hammersley samples.
 * The texels must not change until the stream has passed this work.  Two
 * updates of one environment must not overlap on the GPU (they share its
 * buffers and its finished-block counters); order them on one stream, or
 * give each frame in flight its own environment. */
glint_status glint_env_update(glint_env *env, const void *texels, void *stream);

/* Copies the K radiance levels to host memory (K floats).  Synchronous. */
glint_status glint_env_levels(const glint_env *env, float *host_L, int K);

/* What glint_env_export copies. */
typedef enum glint_env_item {
    GLINT_ENV_LOHI = 0,      /* 2 floats: lo, hi */
    GLINT_ENV_LEVELS = 1,    /* K floats */
    GLINT_ENV_PYRAMID = 2,   /* pyramid level `index`: (H>>index) x (W>>index) x C floats */
    GLINT_ENV_FILTERED = 3,  /* all filtered levels concatenated: level r is W_r/2 x W_r x C floats */
    GLINT_ENV_TABLE = 4,     /* filter sample table: R x S x 4 floats, then R int32 valid counts */
    GLINT_ENV_FILTERED_WIDTHS = 5 /* R int32: W_r of each filtered level */
} glint_env_item;

/* Copies one item to host memory; C = 3 + K channels per texel, padded to a
 * multiple of 4 in device memory and unpadded in the copy.  `bytes` must be at
 * least the item's size.  Synchronous. */
glint_status glint_env_export(const glint_env *env, int item, int index, void *host_dst, size_t bytes);

/* Releases an environment (NULL is ignored). */
void glint_env_destroy(glint_env *env);

/* G-buffer: four device planes of width*height float4, 16-byte aligned.
 *   view_n0:   w_o.xyz (unit vector from the surface to the viewer), N_0
 *              (microfacets per unit uv area; <= 0 marks a background pixel,
 *              shaded black)
 *   normal_f0: n.xyz (unit shading normal), F0 (Schlick)
 *   uv_alpha:  u, v, alpha_x, alpha_y (GGX roughness)
 *   duv:       du/dx, dv/dx, du/dy, dv/dy (screen-space uv derivatives)
 *   tangent:   t.xyz (direction of alpha_x), unused w; may be NULL for E1,
 *              required for E2 */
typedef struct glint_gbuffer {
    const float *view_n0;
    const float *normal_f0;
    const float *uv_alpha;
    const float *duv;
    int width;
    int height;
    const float *tangent;
} glint_gbuffer;

typedef struct glint_params {
    uint32_t seed;   /* user seed of the grid-vertex hashes */
    int count_mode;  /* glint_count_mode */
    int evaluator;   /* glint_evaluator */
    int e2_samples;  /* E2: S x S quadrature points, S in [1, 256] (0 = 16) */
    const glint_mlp *mlp; /* GLINT_EVAL_MLP: the network; its K must equal the environment's */
    float *p_scratch;     /* GLINT_EVAL_GIVEN: device, width*height*K floats (4-byte aligned), the
                             p_k to shade with (read only).  Caller-owned.  Not used by
                             GLINT_EVAL_MLP (the network's p_k never leave the chip) */
    int draw;             /* glint_draw: binomial approximation at the tree nodes (0 = the paper's) */
    float gamma;          /* GLINT_DRAW_WANG2020: reflection probability of a microfacet, (0, 1] */
    int grid;             /* glint_grid: the grid N_P is spread over (0 = two levels x uv triangle) */
} glint_params;

typedef enum glint_grid {
    GLINT_GRID_ISOTROPIC = 0,  /* 2 footprint levels x 3 uv-triangle vertices = 6 samples (Sec. 3.3) */
    GLINT_GRID_ANISOTROPIC = 1 /* the footprint's tetrahedral cell in (level, anisotropy, orientation)
                                  x 3 vertices of a uv lattice stretched along the footprint:
                                  12 samples; debug arrays hold 12 samples per pixel (E1, dual) */
} glint_grid;

typedef enum glint_draw {
    GLINT_DRAW_DUAL = 0,       /* dual-gated Gaussians (Alg. 1), the paper's method */
    GLINT_DRAW_SINGLE = 1,     /* single-gated Gaussians generalised to real N (Eq. gated); comparison */
    GLINT_DRAW_SINGLE_OLD = 2, /* the earlier single-gated form with a floor (Eq. oldgated); comparison */
    GLINT_DRAW_WANG2020 = 3    /* Wang et al. 2020 on the same grid (Sec. 7): one single-gated count per
                                  sample with probability gamma, independent of the map;
                                  L^_o = L_o M / (N_P gamma); counts: bin 1 the glints, bin 2 the rest */
} glint_draw;

/* Optional per-pixel intermediate results (device; each pointer may be NULL).
 *   p:      npix x K   reflection probabilities p_k (Eq. probhk)
 *   np:     npix       microfacet count N_P of the footprint
 *   vert:   npix x 6 x 3 int32: low 32 bits of grid vertex x, y, and level (anisotropic grid:
 *           npix x 12 x 3, the third entry the packed (level, anisotropy, orientation) key;
 *           w, nroot and counts likewise hold 12 samples per pixel)
 *   w:      npix x 6   grid sample weights w_i (Eq. anisogrid)
 *   nroot:  npix x 6   trials at each sample's tree root (float)
 *   counts: npix x 6 x K per-sample bin counts n_k(i) (float; integers in
 *           integer mode)
 *   lo:     npix x 3   smooth radiance L_o (Eq. rtibl) */
typedef struct glint_debug {
    float *p;
    float *np;
    int32_t *vert;
    float *w;
    float *nroot;
    float *counts;
    float *lo;
} glint_debug;

/* Glint shading of every pixel of `gbuf` (Sec. 4 Eq. iblglints:fin):
 *   L^_o = L_o * sum_k L_k M_k / (N_P * sum_k L_k p_k)
 * with L_o the smooth split-sum radiance, p_k = V W_k (k >= 2) and
 * p_1 = U + V W_1 from the filtered maps and tables (E1), or, with
 * GLINT_EVAL_E2, p_k = int D(h) 1[n.w_i > 0] w_k(w_i) dh / int D(h) dh of the
 * anisotropic footprint by an S x S quadrature of the GGX slope distribution
 * reading the weights pyramid (masked mass in p_1), or, with GLINT_EVAL_MLP,
 * p_k from params->mlp evaluated inside the shading kernel (one launch: each
 * block of 256 pixels computes the network's inputs, runs the network on the
 * tensor cores and draws with its p_k from shared memory), or, with
 * GLINT_EVAL_GIVEN, the p_k in params->p_scratch,
 * N_P = N_0 |det duv|, and
 * M_k = sum_i w_i n_k(i) over six triangle-grid samples (Sec. 3.3
 * Eq. anisogrid), each a hierarchical multinomial of dual-gated Gaussian
 * binomials (Alg. 1, Sec. 5) seeded by a hash of its grid vertex.
 * out_rgba: device, width*height float4.  dbg may be NULL.  Enqueued on
 * `stream`; env must have been updated on the same stream (or synchronised). */
glint_status glint_shade(glint_ctx *ctx, const glint_env *env, const glint_gbuffer *gbuf,
                         const glint_params *params, float *out_rgba, const glint_debug *dbg, void *stream);

/* ---- shading a frame held in host memory ----
 * The same per-pixel shading as glint_shade (Sec. 4 Eq. iblglints:fin; each
 * pixel depends only on its own G-buffer texel, the environment and the seed,
 * so results equal glint_shade's bit for bit), for a caller whose G-buffer
 * and output live in host memory.  Two ways, chosen per call:
 *  - in place: when every buffer lies in page-locked host memory the device
 *    can address (cudaHostAlloc / cudaMallocHost, or cudaHostRegister), the
 *    shading kernels read the planes and write the output there directly
 *    over the host link, in one pass: the transfer overlaps the arithmetic
 *    inside the kernel, with no staging and no copies;
 *  - staged (pageable buffers, or GLINT_HOST_STAGED): the frame is cut into
 *    bands of whole rows, and band b's planes are copied host -> device on
 *    the pipe's upload stream, shaded on `stream`, and its output copied
 *    device -> host on the pipe's download stream, so that the copies of one
 *    band overlap the shading of the others.  A glint_hostpipe owns the device staging for `slots` bands (2 to 16)
 * of up to band_pixels pixels each (five 16-byte input planes and one 16-byte
 * output plane per pixel, allocated once at creation on ctx's device), the two
 * copy streams and the events that order them.  Uploads run at most `slots`
 * bands ahead of the shading: as many slots as a frame has bands let the
 * upload link run without waiting for the shading. */
typedef struct glint_hostpipe glint_hostpipe;

glint_status glint_hostpipe_create(glint_ctx *ctx, long band_pixels, int slots, glint_hostpipe **out);
/* Waits for the pipe's copies, then frees it.  NULL is ignored. */
void glint_hostpipe_destroy(glint_hostpipe *pipe);

/* host_gbuf: HOST pointers to the width*height float4 planes (tangent only for
 * E2 and the MLP evaluator; it is uploaded whenever non-NULL); out_rgba_host:
 * HOST, width*height float4.  Pinned host memory (cudaHostAlloc or
 * cudaHostRegister) lets the copies overlap; pageable memory gives the same
 * results with copies that block the calling thread (device buffers work too:
 * the staged copies take their direction from the addresses).  params as glint_shade
 * (params->p_scratch stays a DEVICE buffer of width*height*K floats for the
 * GIVEN evaluator; band b uses its rows of it).  rows_per_band (staged
 * frames only; a frame shaded in place ignores it): 0 picks about an eighth of
 * the frame, capped by the pipe's band_pixels; a band of more pixels than
 * band_pixels, or a row wider than it, is GLINT_ERR_INVALID_ARG.  The uploads start after the work enqueued on
 * `stream` before the call, unless flags holds GLINT_HOST_INPUTS_READY: the
 * host planes are final when the call is made, and the uploads start at once,
 * alongside that work (an environment update enqueued just before, say); the
 * shading of each band still follows it on `stream` (in place, the kernels
 * read the planes in stream order and the flag changes nothing).  The call
 * returns once
 * everything is enqueued and `stream` then waits for the last download, so
 * out_rgba_host is complete when `stream` is.  The host buffers must stay
 * valid and unchanged until then.  Calls on one pipe are ordered through its
 * staging: a call's uploads wait until the previous call's shading has read
 * the slots they overwrite; one host thread at a time may call with a given
 * pipe.  Unknown flag bits are GLINT_ERR_INVALID_ARG. */
#define GLINT_HOST_INPUTS_READY 1u
#define GLINT_HOST_STAGED 2u /* stage through the pipe even when the buffers could be used in place */
glint_status glint_shade_host(glint_hostpipe *pipe, const glint_env *env, const glint_gbuffer *host_gbuf,
                              const glint_params *params, float *out_rgba_host, int rows_per_band,
                              unsigned flags, void *stream);
/* Kernel launches of the last glint_shade_host call on `pipe` (every band). */
int glint_hostpipe_last_launches(const glint_hostpipe *pipe);
/* 1 if the last glint_shade_host call on `pipe` shaded in place, 0 if staged. */
int glint_hostpipe_last_in_place(const glint_hostpipe *pipe);

/* Reflection probabilities p_k (Eq. probhk) of every pixel of `gbuf` under
 * params->evaluator (E1, E2 or MLP; GIVEN is rejected; seed and count mode
 * are ignored), the
 * quantity glint_shade feeds to the counts.  p_out: device, width*height*K
 * floats, pixel-major; background pixels (N_0 <= 0) get 0.  Used to generate
 * the surrogate's training targets (E2) and to measure its error.  Enqueued on
 * `stream`. */
glint_status glint_reflect_probs(glint_ctx *ctx, const glint_env *env, const glint_gbuffer *gbuf,
                                 const glint_params *params, float *p_out, void *stream);

/* ---------------------------------------------------------------------------
 * Learned surrogate of the per-component NDF mass (no counterpart in the
 * paper).  A BF16 MLP with FP32 accumulation corrects E1's p_k towards the
 * anisotropic integral that E2 computes, for K in {2, 4, 8}:
 *   x = ( p_k^E1 (K) | W_k at five taps (5K) | mu_o, sqrt a_x, sqrt a_y | 0 )
 *       (64 values); W_k is read from the filtered maps at roughness
 *       parameter s = sqrt(min(a_x, a_y)) in the directions w_r and
 *       normalize(w_r + a_x J_t), normalize(w_r - a_x J_t),
 *       normalize(w_r + a_y J_b), normalize(w_r - a_y J_b), in that order,
 *       where J_t = 2 (-(w_o.t) n - mu_o t) (t the tangent made orthogonal to
 *       n) and J_b likewise for b = n x t;
 *   lp = log max(p_k^E1, 1e-6);
 *   h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2),
 *   p = softmax((h2 W3 + b3)[0..K) + lp)
 * with x, W, h1 and h2 rounded to BF16 and every sum accumulated in FP32.
 * Parameters (FP32 master copy, glint_mlp_param_count() floats, in order):
 *   W1 [64 in][64 out], b1 [64], W2 [64][64], b2 [64], W3 [64][16], b3 [16]
 * (columns >= K of W3 and b3 are unused and stay fixed).  Training minimises
 * the mean squared error sum_k (p_k - y_k)^2 against target distributions y
 * (e.g. E2's p_k from glint_reflect_probs; the quantity the surrogate's error
 * is judged by) with Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8, FP32).  The gradient of a batch is accumulated per resident block
 * in a fixed order and summed over blocks in block order, so a step is
 * deterministic.  Inputs x are stored as BF16 bit patterns (uint16), 64 per
 * sample, row-major; lp as K floats per sample.
 * ------------------------------------------------------------------------- */

typedef enum glint_mlp_item {
    GLINT_MLP_PARAMS = 0, /* FP32 master parameters */
    GLINT_MLP_GRAD = 1,   /* gradient of the last glint_mlp_train_step */
    GLINT_MLP_ADAM_M = 2, /* Adam first moment */
    GLINT_MLP_ADAM_V = 3  /* Adam second moment */
} glint_mlp_item;

/* Number of FP32 parameters (9360). */
int glint_mlp_param_count(void);

/* A network for K in {2, 4, 8} components (K = 16 gives GLINT_ERR_UNSUPPORTED)
 * on ctx's device, trainable with batches of up to max_batch samples
 * (1 .. 2^30).  Weights He-uniform from a pcg4d hash of (layer, index, seed),
 * biases 0, Adam moments 0, step 0. */
glint_status glint_mlp_create(glint_ctx *ctx, int K, long max_batch, uint32_t seed, glint_mlp **out);
void glint_mlp_destroy(glint_mlp *mlp);

/* Copies glint_mlp_param_count() host floats into the master parameters and
 * refreshes the BF16 copies (synchronous). */
glint_status glint_mlp_set_params(glint_mlp *mlp, const float *host, long n);

/* Copies one glint_mlp_item (n = glint_mlp_param_count() floats) to host
 * memory (synchronous). */
glint_status glint_mlp_export(const glint_mlp *mlp, int item, float *host, long n);

/* Restores parameters, Adam moments and the step counter (checkpoint resume;
 * training continues bit-identically).  Synchronous. */
glint_status glint_mlp_import_state(glint_mlp *mlp, const float *params, const float *adam_m, const float *adam_v,
                                    long n, long step);

/* Adam steps taken so far. */
long glint_mlp_step(const glint_mlp *mlp);

/* The surrogate's inputs of every pixel of `gbuf` (view_n0, normal_f0,
 * uv_alpha and tangent planes) under environment `env` (K in {2, 4, 8}):
 * x_out (device, width*height*64 uint16 BF16 patterns, 16-byte aligned) and
 * lp_out (device, width*height*K floats); background rows are 0.  Enqueued on
 * `stream`. */
glint_status glint_mlp_features(glint_ctx *ctx, const glint_env *env, const glint_gbuffer *gbuf, uint16_t *x_out,
                                float *lp_out, void *stream);

/* p_out (device, n*K floats) = the network applied to given inputs x (device,
 * n*64 BF16 patterns, 16-byte aligned) and lp (device, n*K floats).  Enqueued
 * on `stream`. */
glint_status glint_mlp_forward(const glint_mlp *mlp, const uint16_t *x, const float *lp, long n, float *p_out,
                               void *stream);

/* One optimisation step on samples first, first+1, ..., first+batch-1 (indices
 * modulo n_total) of the inputs x, lp (as glint_mlp_forward) against
 * `targets` (device, n_total*K floats, each row a distribution).  lr = 0 only
 * computes the gradient (GLINT_MLP_GRAD); 0 < lr < 1 also takes an Adam step.
 * If loss_out is not NULL the batch's mean squared error is written there
 * (host) and the call waits for the stream.  Enqueued on `stream`. */
glint_status glint_mlp_train_step(glint_mlp *mlp, const uint16_t *x, const float *lp, const float *targets,
                                  long n_total, long first, long batch, float lr, float *loss_out, void *stream);

/* `steps` Adam steps, enqueued without returning to the caller in between:
 * step i trains on samples first + i*batch, ... (indices modulo n_total) with
 * learning rate max(lr_max * (1 + cos(pi i / steps)) / 2, lr_min) (a cosine
 * schedule), exactly as the same sequence of glint_mlp_train_step calls would
 * (same kernels, same order: the results are equal bit for bit).  No counterpart in the
 * paper (the surrogate is this library's).  0 < lr_min <= lr_max < 1; x, lp,
 * targets as glint_mlp_train_step.  Enqueued on `stream`; two launches per
 * step. */
glint_status glint_mlp_train(glint_mlp *mlp, const uint16_t *x, const float *lp, const float *targets, long n_total,
                             long first, long batch, long steps, float lr_max, float lr_min, void *stream);

/* p_out (device, width*height*K floats) = the network's p_k of every pixel of
 * `gbuf` under `env` (inputs computed on the fly, one persistent launch);
 * background pixels get 0.  The network's K must equal the environment's.
 * Enqueued on `stream`. */
glint_status glint_mlp_infer(const glint_mlp *mlp, glint_ctx *ctx, const glint_env *env, const glint_gbuffer *gbuf,
                             float *p_out, void *stream);

int glint_mlp_get_k(const glint_mlp *mlp);
int glint_mlp_last_launches(const glint_mlp *mlp);

/* Checkpoint: writes one line of JSON header ({"format": "glint_mlp",
 * "version": 1, "K", "params", "step", "arrays": ["params", "adam_m",
 * "adam_v"], "dtype": "float32-le"}) and then the three arrays as
 * little-endian float32 to `path` (synchronous). */
glint_status glint_mlp_save(const glint_mlp *mlp, const char *path);
/* A network restored from a glint_mlp_save file (parameters, Adam moments and
 * step: training continues bit-identically), trainable with batches of up to
 * max_batch samples. */
glint_status glint_mlp_load(glint_ctx *ctx, const char *path, long max_batch, glint_mlp **out);

/* Training samples of every pixel of `gbuf` under `env`: the inputs and
 * log-priors of glint_mlp_features and, as targets, E2's p_k with an
 * e2_samples x e2_samples quadrature (glint_reflect_probs).  targets_out:
 * device, width*height*K floats.  Enqueued on `stream`. */
glint_status glint_mlp_generate(glint_ctx *ctx, const glint_env *env, const glint_gbuffer *gbuf, int e2_samples,
                                uint16_t *x_out, float *lp_out, float *targets_out, void *stream);

/* ---------------------------------------------------------------------------
 * Serving (no counterpart in the paper): a continuous-batching request loop.
 * Frames of any resolution, each with one of the resident environments (and
 * its surrogate), are submitted from host memory; a tick admits queued frames
 * while their device buffers fit the memory budget (FIFO).  A frame whose
 * buffers all lie in page-locked memory the device addresses is shaded in
 * place (the kernels read its G-buffer and write its result over the CPU-GPU
 * link; it holds no device memory), unless the server was created with
 * upload = 1; other frames are copied to the device on copy streams.  A tick
 * shades a tile of every admitted frame whose inputs are on hand and then up
 * to tick_pixels pixels, frames with the fewest pixels left first, in one
 * persistent launch over a work list of (frame, pixel range) items (and one
 * more, of the shading with the network fused in, for frames on the surrogate
 * path).  Finished frames are copied back (unless shaded in place)
 * and released; glint_server_poll reports them.  A frame's pixels are computed
 * exactly as glint_shade's kernel computes them, whatever else shares its
 * ticks and wherever its buffers lie.  One host thread drives a server.
 * ------------------------------------------------------------------------- */
typedef struct glint_server glint_server;

typedef struct glint_server_desc {
    size_t memory_budget;   /* device bytes for admitted frames' buffers (one allocation at creation) */
    long tick_pixels;       /* pixels shaded per tick at most (0 = 2097152: ~0.3 ms of shading in device memory,
                               ~0.7 ms in place; smaller ticks let small frames finish sooner) */
    int tile_pixels;        /* pixels per planned item, a multiple of 128 (0 = 16384); items are
                               launched in pieces of 1024 pixels */
    int max_frames;         /* admitted frames at most (0 = 64) */
    int max_inflight_ticks; /* ticks enqueued on the GPU at most; a tick waits for older ones (0 = 2) */
    int upload;             /* 1: copy every frame into the budget's device memory; 0: shade frames in
                               page-locked host memory in place (no device memory) */
} glint_server_desc;

/* A frame.  Planes are HOST memory in glint_gbuffer's layout (page-locked
 * memory is shaded in place, or lets the copies overlap with shading); tangent
 * is required on the surrogate path.  out_rgba: HOST, width*height float4.  The caller keeps all
 * of them alive until glint_server_poll has reported the frame. */
typedef struct glint_frame_request {
    int env;          /* index from glint_server_add_env */
    int width;
    int height;
    uint32_t seed;
    int evaluator;    /* GLINT_EVAL_E1 or GLINT_EVAL_MLP */
    const float *view_n0;
    const float *normal_f0;
    const float *uv_alpha;
    const float *duv;
    const float *tangent;
    float *out_rgba;
} glint_frame_request;

/* A finished frame: its id and host-clock times (seconds since the server's
 * creation) of submission, admission and completion (its result in out_rgba). */
typedef struct glint_frame_done {
    long id;
    double submit_s;
    double admit_s;
    double done_s;
} glint_frame_done;

typedef struct glint_server_stats {
    long queued;          /* submitted, not admitted */
    long active;          /* admitted, not reported */
    long done;            /* reported by glint_server_poll */
    size_t used_bytes;    /* device bytes held by admitted frames */
    size_t peak_bytes;
    long ticks;           /* ticks that launched work */
    long launches;        /* kernel launches of those ticks */
    long items;           /* work items of those ticks */
} glint_server_stats;

/* A server for environments with K components on ctx's device. */
glint_status glint_server_create(glint_ctx *ctx, int K, const glint_server_desc *desc, glint_server **out);
/* Waits for the server's work and frees it. */
void glint_server_destroy(glint_server *server);
/* Makes `env` (updated, same context and K) resident for requests; `mlp` (may
 * be NULL) is its surrogate for GLINT_EVAL_MLP.  *env_id receives the index. */
glint_status glint_server_add_env(glint_server *server, const glint_env *env, const glint_mlp *mlp, int *env_id);
/* Requests an update of resident map `env_id` from `texels` (device, the
 * map's size and format; the caller keeps them unchanged until the update
 * has run): frames submitted before the call are shaded with the map as it
 * was, frames submitted after it with the updated map.  A tick runs the
 * update (glint_env_update's launches, on the tick's stream) once no admitted
 * or queued frame needs the previous version; until then the newer frames
 * wait in the queue.  Several requests before it runs collapse into the
 * latest. */
glint_status glint_server_update_env(glint_server *server, int env_id, const void *texels);
/* Queues a frame and returns its id; GLINT_ERR_INVALID_ARG if the request is
 * malformed or its buffers could never fit the memory budget. */
glint_status glint_server_submit(glint_server *server, const glint_frame_request *req, long *id);
/* Admits, enqueues one tick of work on `stream` and the copies of finished
 * frames; *launched (may be NULL) receives the kernel launches. */
glint_status glint_server_tick(glint_server *server, void *stream, int *launched);
/* Up to max_done finished frames (copied back), in completion order. */
glint_status glint_server_poll(glint_server *server, glint_frame_done *done, int max_done, int *n_done);
glint_status glint_server_stats_get(const glint_server *server, glint_server_stats *stats);

/* Device-memory admission bookkeeping used by the server (host only, no
 * device memory): first-fit over [0, bytes) with `align`-byte granularity and
 * coalescing of freed neighbours. */
typedef struct glint_arena glint_arena;
glint_arena *glint_arena_create(size_t bytes, size_t align);
void glint_arena_destroy(glint_arena *arena);
/* Offset of a new block of `bytes`, or -1 if no free range holds it. */
long long glint_arena_alloc(glint_arena *arena, size_t bytes);
/* 0, or -1 if `offset` is not an allocated block. */
int glint_arena_free(glint_arena *arena, long long offset);
size_t glint_arena_used(const glint_arena *arena);
size_t glint_arena_largest_free(const glint_arena *arena);

/* The tick planner (host only): frames in admission order with next[f] of
 * npix[f] pixels planned so far.  Items are ranges of at most tile_pixels
 * pixels ending at multiples of tile_pixels (or the frame's end): first one
 * item for every unfinished frame, so that every admitted frame progresses in
 * every tick, then items for the frames with the fewest pixels left (frame
 * order among equals) until tick_pixels are planned; at most max_items in all.  Writes the items, advances next[] and returns the item
 * count. */
int glint_plan_tick(long *next, const long *npix, int nframes, long tick_pixels, int tile_pixels, int *item_frame,
                    long *item_first, int *item_count, int max_items);

/* Standard normal quantile z = Phi^-1(p) as the shading kernel evaluates it for
 * the Gaussian part of the dual-gated draw (Alg. 1): for n device floats p in
 * (0, 1), device output z.  Relative error below 2.3e-7 on the uniforms the
 * kernel draws, p = (2m + 1) 2^-24 (FP32).  Enqueued on `stream`. */
glint_status glint_normal_quantile(const float *p, float *z, long n, void *stream);

/* Fixed scratch of glint_env_levels_noalloc: one (min, max) float pair per
 * reduction block, GLINT_NOALLOC_MAX_BLOCKS pairs (8 KB per device). */
#define GLINT_NOALLOC_MAX_BLOCKS 1024
#define GLINT_NOALLOC_MAX_HEIGHT 8192

/* Radiance levels of an environment map (steps 1 and 2 of glint_env_update:
 * brightness min and max, lo, hi and L_1 .. L_K) computed without allocating
 * any memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- frame loops that must never stall on
 * an allocation (cudaMalloc/cudaFree may synchronise the device) and host
 * applications such as engines and plug-in hosts that own every device
 * allocation through their own allocator.
 *
 * texels: device, width x height RGBA texels in `format` (width = 2 height,
 * height a power of two, at most GLINT_NOALLOC_MAX_HEIGHT; larger maps are
 * rejected with GLINT_ERR_INVALID_ARG).  levels_out: device, K + 2 floats
 * written as L_1 .. L_K, lo, hi (the layout glint_env_levels and
 * GLINT_ENV_LOHI report).  Work is enqueued on `stream` of device `device`.
 * The block partials of the reduction go to a fixed array inside the library
 * that every GPU loading it holds until the process exits.  Every call looks
 * up that array's address in the calling thread's current context for
 * `device` (a host query that allocates nothing), so the call stays correct
 * after cudaDeviceReset or when a host makes its own context current; the
 * first call on a device may load the library's module there, so make it
 * before any stream capture.  All calls in a context share the array and it
 * keeps the last call's contents; calls whose work overlaps on the GPU race on
 * it, so issue them on one stream or order them. */
glint_status glint_env_levels_noalloc(int device, const void *texels, int width, int height, int format,
                                      int scale_log2, int K, float ell, float *levels_out, void *stream);

/* Number of kernel launches the most recent glint_env_update / glint_shade on
 * this environment / context enqueued (for launch accounting). */
int glint_env_last_launches(const glint_env *env);
int glint_ctx_last_launches(const glint_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* GLINT_H */
