"""Thin ctypes binding of the C ABI in ``include/glint.h``.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libglint.so``.  PyTorch provides device memory and streams.  If
the library is missing, importing this module raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libglint.so")

GLINT_OK = 0
FMT_RGBA32F, FMT_RGBA16F = 0, 1
COUNT_INTEGER, COUNT_REAL = 0, 1
EVAL_E1, EVAL_E2, EVAL_MLP, EVAL_GIVEN, EVAL_E1_ANISO = 0, 1, 2, 3, 4
MLP_PARAMS, MLP_GRAD, MLP_ADAM_M, MLP_ADAM_V = 0, 1, 2, 3
ABI_VERSION = 8
HOST_INPUTS_READY = 1
HOST_STAGED = 2
GRID_ISOTROPIC, GRID_ANISOTROPIC = 0, 1
WFMT_F32, WFMT_F16, WFMT_UNORM16, WFMT_UNORM8 = 0, 1, 2, 3
DRAW_DUAL, DRAW_SINGLE, DRAW_SINGLE_OLD, DRAW_WANG2020 = 0, 1, 2, 3
WEIGHTS_LINEAR, WEIGHTS_LOG = 0, 1
ENV_LOHI, ENV_LEVELS, ENV_PYRAMID, ENV_FILTERED, ENV_TABLE, ENV_FILTERED_WIDTHS = 0, 1, 2, 3, 4, 5
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NOT_READY", 5: "TIMEOUT", 6: "UNSUPPORTED"}


class GlintError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"glint status {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class EnvDesc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("format", ctypes.c_int),
                ("scale_log2", ctypes.c_int), ("K", ctypes.c_int), ("ell", ctypes.c_float),
                ("levels", ctypes.c_int), ("samples", ctypes.c_int), ("out_width", ctypes.c_int),
                ("s_min", ctypes.c_float), ("s_max", ctypes.c_float), ("weight_space", ctypes.c_int),
                ("weight_format", ctypes.c_int)]


class GBufferDesc(ctypes.Structure):
    _fields_ = [("view_n0", ctypes.c_void_p), ("normal_f0", ctypes.c_void_p), ("uv_alpha", ctypes.c_void_p),
                ("duv", ctypes.c_void_p), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("tangent", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint32), ("count_mode", ctypes.c_int), ("evaluator", ctypes.c_int),
                ("e2_samples", ctypes.c_int), ("mlp", ctypes.c_void_p), ("p_scratch", ctypes.c_void_p),
                ("draw", ctypes.c_int), ("gamma", ctypes.c_float), ("grid", ctypes.c_int)]


class Debug(ctypes.Structure):
    _fields_ = [("p", ctypes.c_void_p), ("np", ctypes.c_void_p), ("vert", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("nroot", ctypes.c_void_p), ("counts", ctypes.c_void_p), ("lo", ctypes.c_void_p)]


class ServerDesc(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_size_t), ("tick_pixels", ctypes.c_long), ("tile_pixels", ctypes.c_int),
                ("max_frames", ctypes.c_int), ("max_inflight_ticks", ctypes.c_int), ("upload", ctypes.c_int)]


class FrameRequest(ctypes.Structure):
    _fields_ = [("env", ctypes.c_int), ("width", ctypes.c_int), ("height", ctypes.c_int), ("seed", ctypes.c_uint32),
                ("evaluator", ctypes.c_int), ("view_n0", ctypes.c_void_p), ("normal_f0", ctypes.c_void_p),
                ("uv_alpha", ctypes.c_void_p), ("duv", ctypes.c_void_p), ("tangent", ctypes.c_void_p),
                ("out_rgba", ctypes.c_void_p)]


class FrameDone(ctypes.Structure):
    _fields_ = [("id", ctypes.c_long), ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_long), ("active", ctypes.c_long), ("done", ctypes.c_long),
                ("used_bytes", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t), ("ticks", ctypes.c_long),
                ("launches", ctypes.c_long), ("items", ctypes.c_long)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2507_02674_gb300.build.build() "
                          "(the CUDA library is the only implementation)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    lib.glint_abi_version.restype = I
    lib.glint_last_error.restype = ctypes.c_char_p
    lib.glint_ctx_create.argtypes = [I, I, I, ctypes.POINTER(P)]
    lib.glint_ctx_destroy.argtypes = [P]
    lib.glint_ctx_destroy.restype = None
    lib.glint_lut_export.argtypes = [P, P, S]
    lib.glint_env_create.argtypes = [P, ctypes.POINTER(EnvDesc), ctypes.POINTER(P)]
    lib.glint_env_update.argtypes = [P, P, P]
    lib.glint_env_levels.argtypes = [P, P, I]
    lib.glint_env_export.argtypes = [P, I, I, P, S]
    lib.glint_env_destroy.argtypes = [P]
    lib.glint_env_destroy.restype = None
    lib.glint_shade.argtypes = [P, P, ctypes.POINTER(GBufferDesc), ctypes.POINTER(Params), P,
                                ctypes.POINTER(Debug), P]
    lib.glint_normal_quantile.argtypes = [P, P, ctypes.c_long, P]
    lib.glint_reflect_probs.argtypes = [P, P, ctypes.POINTER(GBufferDesc), ctypes.POINTER(Params), P, P]
    lib.glint_hostpipe_create.argtypes = [P, ctypes.c_long, I, ctypes.POINTER(P)]
    lib.glint_hostpipe_destroy.argtypes = [P]
    lib.glint_hostpipe_destroy.restype = None
    lib.glint_hostpipe_last_launches.argtypes = [P]
    lib.glint_hostpipe_last_launches.restype = I
    lib.glint_hostpipe_last_in_place.argtypes = [P]
    lib.glint_hostpipe_last_in_place.restype = I
    lib.glint_shade_host.argtypes = [P, P, ctypes.POINTER(GBufferDesc), ctypes.POINTER(Params), P, I,
                                     ctypes.c_uint, P]
    L, F = ctypes.c_long, ctypes.c_float
    lib.glint_mlp_param_count.restype = I
    lib.glint_mlp_create.argtypes = [P, I, L, ctypes.c_uint32, ctypes.POINTER(P)]
    lib.glint_mlp_destroy.argtypes = [P]
    lib.glint_mlp_destroy.restype = None
    lib.glint_mlp_set_params.argtypes = [P, P, L]
    lib.glint_mlp_export.argtypes = [P, I, P, L]
    lib.glint_mlp_import_state.argtypes = [P, P, P, P, L, L]
    lib.glint_mlp_step.argtypes = [P]
    lib.glint_mlp_step.restype = L
    lib.glint_mlp_features.argtypes = [P, P, ctypes.POINTER(GBufferDesc), P, P, P]
    lib.glint_mlp_forward.argtypes = [P, P, P, L, P, P]
    lib.glint_mlp_train_step.argtypes = [P, P, P, P, L, L, L, F, ctypes.POINTER(F), P]
    lib.glint_mlp_train.argtypes = [P, P, P, P, L, L, L, L, F, F, P]
    lib.glint_mlp_infer.argtypes = [P, P, P, ctypes.POINTER(GBufferDesc), P, P]
    lib.glint_mlp_save.argtypes = [P, ctypes.c_char_p]
    lib.glint_mlp_load.argtypes = [P, ctypes.c_char_p, L, ctypes.POINTER(P)]
    lib.glint_mlp_generate.argtypes = [P, P, ctypes.POINTER(GBufferDesc), I, P, P, P, P]
    lib.glint_mlp_get_k.argtypes = [P]
    lib.glint_mlp_get_k.restype = I
    lib.glint_mlp_last_launches.argtypes = [P]
    lib.glint_mlp_last_launches.restype = I
    Z, LL = ctypes.c_size_t, ctypes.c_longlong
    lib.glint_arena_create.argtypes = [Z, Z]
    lib.glint_arena_create.restype = P
    lib.glint_arena_destroy.argtypes = [P]
    lib.glint_arena_destroy.restype = None
    lib.glint_arena_alloc.argtypes = [P, Z]
    lib.glint_arena_alloc.restype = LL
    lib.glint_arena_free.argtypes = [P, LL]
    lib.glint_arena_used.argtypes = [P]
    lib.glint_arena_used.restype = Z
    lib.glint_arena_largest_free.argtypes = [P]
    lib.glint_arena_largest_free.restype = Z
    lib.glint_plan_tick.argtypes = [P, P, I, L, I, P, P, P, I]
    lib.glint_server_create.argtypes = [P, I, ctypes.POINTER(ServerDesc), ctypes.POINTER(P)]
    lib.glint_server_destroy.argtypes = [P]
    lib.glint_server_destroy.restype = None
    lib.glint_server_add_env.argtypes = [P, P, P, ctypes.POINTER(I)]
    lib.glint_server_submit.argtypes = [P, ctypes.POINTER(FrameRequest), ctypes.POINTER(L)]
    lib.glint_server_update_env.argtypes = [P, I, P]
    lib.glint_server_tick.argtypes = [P, P, ctypes.POINTER(I)]
    lib.glint_server_poll.argtypes = [P, P, I, ctypes.POINTER(I)]
    lib.glint_server_stats_get.argtypes = [P, ctypes.POINTER(ServerStats)]
    lib.glint_env_last_launches.argtypes = [P]
    lib.glint_env_last_launches.restype = I
    lib.glint_ctx_last_launches.argtypes = [P]
    lib.glint_ctx_last_launches.restype = I
    if lib.glint_abi_version() != ABI_VERSION:
        raise ImportError(f"{LIB_PATH} has ABI {lib.glint_abi_version()}, the binding expects {ABI_VERSION}")
    return lib


lib = _load()


def _check(status: int):
    if status != GLINT_OK:
        raise GlintError(status, lib.glint_last_error().decode())


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t) -> int | None:
    return None if t is None else t.data_ptr()


class Context:
    """glint_ctx: a device and its microfacet tables."""

    def __init__(self, device: int = 0, lut_n: int = 64, lut_q: int = 128):
        h = ctypes.c_void_p()
        _check(lib.glint_ctx_create(device, lut_n, lut_q, ctypes.byref(h)))
        self.handle = h
        self.device = device
        self.lut_n = lut_n

    def lut(self) -> np.ndarray:
        out = np.zeros((self.lut_n, self.lut_n, 4), np.float32)
        _check(lib.glint_lut_export(self.handle, out.ctypes.data, out.nbytes))
        return out

    def last_launches(self) -> int:
        return lib.glint_ctx_last_launches(self.handle)

    def close(self):
        if self.handle:
            lib.glint_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class EnvConfig:
    K: int = 8
    ell: float = 1e-4
    levels: int = 8
    samples: int = 64
    out_width: int = 256
    s_min: float = 0.02 ** 0.5
    s_max: float = 0.5 ** 0.5
    weight_space: int = 0  # WEIGHTS_LINEAR (the paper's) or WEIGHTS_LOG
    weight_format: int = 0  # WFMT_F32, WFMT_F16, WFMT_UNORM16 or WFMT_UNORM8 (filtered weights' storage)


class Env:
    """glint_env: device buffers of one environment's levels, pyramid and filtered maps."""

    def __init__(self, ctx: Context, width: int, height: int, fmt: int, scale_log2: int, cfg: EnvConfig):
        self.ctx = ctx
        self.cfg = cfg
        self.desc = EnvDesc(width, height, fmt, scale_log2, cfg.K, cfg.ell, cfg.levels, cfg.samples, cfg.out_width,
                            cfg.s_min, cfg.s_max, cfg.weight_space, cfg.weight_format)
        h = ctypes.c_void_p()
        _check(lib.glint_env_create(ctx.handle, ctypes.byref(self.desc), ctypes.byref(h)))
        self.handle = h
        self.C = 3 + cfg.K
        self.M = 1
        while (height >> (self.M - 1)) > 1:
            self.M += 1

    def update(self, texels, stream=None):
        """Recompute levels, weights, pyramid and filtered maps from device texels."""
        _check(lib.glint_env_update(self.handle, texels.data_ptr(), _stream_handle(stream)))

    def levels(self) -> np.ndarray:
        out = np.zeros(self.cfg.K, np.float32)
        _check(lib.glint_env_levels(self.handle, out.ctypes.data, self.cfg.K))
        return out

    def export(self, item: int, index: int = 0) -> np.ndarray:
        d = self.desc
        if item == ENV_LOHI:
            out = np.zeros(2, np.float32)
        elif item == ENV_LEVELS:
            out = np.zeros(d.K, np.float32)
        elif item == ENV_PYRAMID:
            out = np.zeros((d.height >> index, d.width >> index, self.C), np.float32)
        elif item == ENV_FILTERED_WIDTHS:
            out = np.zeros(d.levels, np.int32)
        elif item == ENV_FILTERED:
            widths = self.export(ENV_FILTERED_WIDTHS)
            total = int(sum(int(w) * (int(w) // 2) for w in widths))
            flat = np.zeros((total, self.C), np.float32)
            _check(lib.glint_env_export(self.handle, item, index, flat.ctypes.data, flat.nbytes))
            return widths, flat
        elif item == ENV_TABLE:
            raw = np.zeros(d.levels * d.samples * 4 + d.levels, np.float32)
            _check(lib.glint_env_export(self.handle, item, index, raw.ctypes.data, raw.nbytes))
            table = raw[:d.levels * d.samples * 4].reshape(d.levels, d.samples, 4).copy()
            nvalid = raw[d.levels * d.samples * 4:].view(np.int32).copy()
            return table, nvalid
        else:
            raise ValueError(item)
        _check(lib.glint_env_export(self.handle, item, index, out.ctypes.data, out.nbytes))
        return out

    def last_launches(self) -> int:
        return lib.glint_env_last_launches(self.handle)

    def close(self):
        if self.handle:
            lib.glint_env_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _gbuffer(planes, width: int, height: int, tangent=None) -> GBufferDesc:
    duv = planes[3] if len(planes) > 3 else None
    return GBufferDesc(_dptr(planes[0]), _dptr(planes[1]), _dptr(planes[2]), _dptr(duv), width, height,
                       _dptr(tangent))


def _params(seed=0, count_mode=COUNT_INTEGER, evaluator=EVAL_E1, e2_samples=16, mlp=None, p_scratch=None,
            draw=DRAW_DUAL, gamma=0.0, grid=GRID_ISOTROPIC):
    return Params(seed & 0xFFFFFFFF, count_mode, evaluator, e2_samples,
                  mlp.handle.value if mlp is not None else None, _dptr(p_scratch), draw, gamma, grid)


def shade(ctx: Context, env: Env, planes, width: int, height: int, out, seed: int = 0,
          count_mode: int = COUNT_INTEGER, debug: dict | None = None, stream=None, tangent=None,
          evaluator: int = EVAL_E1, e2_samples: int = 16, mlp=None, p_scratch=None, draw: int = DRAW_DUAL,
          gamma: float = 0.0, grid: int = GRID_ISOTROPIC):
    """glint_shade over a G-buffer given as four device tensors of (npix, 4) float32
    (plus an optional (npix, 4) tangent tensor, needed by E2 and the MLP)."""
    g = _gbuffer(planes, width, height, tangent)
    p = _params(seed, count_mode, evaluator, e2_samples, mlp, p_scratch, draw, gamma, grid)
    dbg = None
    if debug is not None:
        dbg = Debug(*(_dptr(debug.get(k)) for k in ("p", "np", "vert", "w", "nroot", "counts", "lo")))
    _check(lib.glint_shade(ctx.handle, env.handle, ctypes.byref(g), ctypes.byref(p), _dptr(out),
                           ctypes.byref(dbg) if dbg is not None else None, _stream_handle(stream)))


class HostPipe:
    """glint_hostpipe: device staging, copy streams and events for shading
    frames held in host memory (glint_shade_host), in bands of whole rows."""

    def __init__(self, ctx: Context, band_pixels: int, slots: int = 2):
        h = ctypes.c_void_p()
        _check(lib.glint_hostpipe_create(ctx.handle, band_pixels, slots, ctypes.byref(h)))
        self.handle = h
        self.ctx = ctx

    def shade(self, env: "Env", planes, width: int, height: int, out, seed: int = 0,
              count_mode: int = COUNT_INTEGER, stream=None, tangent=None, evaluator: int = EVAL_E1,
              e2_samples: int = 16, mlp=None, p_scratch=None, draw: int = DRAW_DUAL, gamma: float = 0.0,
              grid: int = GRID_ISOTROPIC, rows_per_band: int = 0, inputs_ready: bool = False,
              staged: bool = False):
        """glint_shade_host: planes (and tangent) are HOST tensors of (npix, 4)
        float32, pinned for overlapped copies; out a HOST (npix, 4) float32
        tensor, complete once `stream` is; p_scratch stays on the device.
        Pinned buffers are shaded in place (the kernels read and write host
        memory directly) unless staged; others go through the pipe's bands.
        inputs_ready: the host planes are final now, so staged uploads need
        not wait for the work already enqueued on `stream`."""
        g = _gbuffer(planes, width, height, tangent)
        p = _params(seed, count_mode, evaluator, e2_samples, mlp, p_scratch, draw, gamma, grid)
        _check(lib.glint_shade_host(self.handle, env.handle, ctypes.byref(g), ctypes.byref(p), _dptr(out),
                                    rows_per_band,
                                    (HOST_INPUTS_READY if inputs_ready else 0) | (HOST_STAGED if staged else 0),
                                    _stream_handle(stream)))

    def last_launches(self) -> int:
        return lib.glint_hostpipe_last_launches(self.handle)

    def last_in_place(self) -> bool:
        return bool(lib.glint_hostpipe_last_in_place(self.handle))

    def close(self):
        if self.handle:
            lib.glint_hostpipe_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reflect_probs(ctx: Context, env: Env, planes, width: int, height: int, out, evaluator: int = EVAL_E1,
                  e2_samples: int = 16, tangent=None, mlp=None, stream=None):
    """glint_reflect_probs: p_k of every pixel into `out` (device, (npix, K) float32)."""
    g = _gbuffer(planes, width, height, tangent)
    p = _params(0, COUNT_INTEGER, evaluator, e2_samples, mlp, None)
    _check(lib.glint_reflect_probs(ctx.handle, env.handle, ctypes.byref(g), ctypes.byref(p), _dptr(out),
                                   _stream_handle(stream)))


class Mlp:
    """glint_mlp: the BF16 surrogate of p_k, its FP32 master weights and Adam state."""

    def __init__(self, ctx: Context, K: int, max_batch: int, seed: int = 0):
        h = ctypes.c_void_p()
        _check(lib.glint_mlp_create(ctx.handle, K, max_batch, seed & 0xFFFFFFFF, ctypes.byref(h)))
        self.handle = h
        self.ctx = ctx
        self.K = K
        self.max_batch = max_batch
        self.n_params = lib.glint_mlp_param_count()

    def set_params(self, params: np.ndarray):
        a = np.ascontiguousarray(params, np.float32)
        _check(lib.glint_mlp_set_params(self.handle, a.ctypes.data, a.size))

    def export(self, item: int = MLP_PARAMS) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        _check(lib.glint_mlp_export(self.handle, item, out.ctypes.data, out.size))
        return out

    def import_state(self, params, adam_m, adam_v, step: int):
        arrs = [np.ascontiguousarray(a, np.float32) for a in (params, adam_m, adam_v)]
        _check(lib.glint_mlp_import_state(self.handle, arrs[0].ctypes.data, arrs[1].ctypes.data,
                                          arrs[2].ctypes.data, self.n_params, step))

    @property
    def step(self) -> int:
        return lib.glint_mlp_step(self.handle)

    def features(self, env: "Env", planes, width: int, height: int, tangent, x=None, lp=None, stream=None):
        """glint_mlp_features: inputs (npix, 64) int16 BF16 patterns and
        log-priors (npix, K) float32 of every pixel, on the device."""
        return mlp_features(self.ctx, env, planes, width, height, tangent, x, lp, stream)

    def forward(self, x, lp, out=None, stream=None):
        """glint_mlp_forward on given inputs x ((n, 64) BF16 patterns) and lp ((n, K))."""
        import torch
        n = x.shape[0]
        if out is None:
            out = torch.empty(n, self.K, device=x.device)
        _check(lib.glint_mlp_forward(self.handle, _dptr(x), _dptr(lp), n, _dptr(out), _stream_handle(stream)))
        return out

    def train_step(self, x, lp, targets, first: int, batch: int, lr: float, want_loss: bool = False, stream=None):
        """glint_mlp_train_step on samples first .. first+batch-1 (wrapping) of x, lp, targets."""
        loss = ctypes.c_float(0.0)
        _check(lib.glint_mlp_train_step(self.handle, _dptr(x), _dptr(lp), _dptr(targets), x.shape[0], first, batch,
                                        lr, ctypes.byref(loss) if want_loss else None, _stream_handle(stream)))
        return float(loss.value) if want_loss else None

    def train(self, x, lp, targets, first: int, batch: int, steps: int, lr_max: float, lr_min: float, stream=None):
        """glint_mlp_train: `steps` Adam steps on consecutive batches with a cosine learning-rate schedule."""
        _check(lib.glint_mlp_train(self.handle, _dptr(x), _dptr(lp), _dptr(targets), x.shape[0], first, batch, steps,
                                   lr_max, lr_min, _stream_handle(stream)))

    def infer(self, env: "Env", planes, width: int, height: int, tangent, out, stream=None):
        """glint_mlp_infer: p_k of every pixel (inputs computed on the fly)."""
        g = _gbuffer(planes, width, height, tangent)
        _check(lib.glint_mlp_infer(self.handle, self.ctx.handle, env.handle, ctypes.byref(g), _dptr(out),
                                   _stream_handle(stream)))
        return out

    def save(self, path: str):
        """glint_mlp_save: parameters, Adam moments and step (JSON header + float32 LE)."""
        _check(lib.glint_mlp_save(self.handle, os.fsencode(path)))

    @classmethod
    def load(cls, ctx: Context, path: str, max_batch: int):
        """glint_mlp_load: a network restored from a checkpoint file."""
        h = ctypes.c_void_p()
        _check(lib.glint_mlp_load(ctx.handle, os.fsencode(path), max_batch, ctypes.byref(h)))
        self = cls.__new__(cls)
        self.handle, self.ctx, self.max_batch = h, ctx, max_batch
        self.K = lib.glint_mlp_get_k(h)
        self.n_params = lib.glint_mlp_param_count()
        return self

    def last_launches(self) -> int:
        return lib.glint_mlp_last_launches(self.handle)

    def close(self):
        if self.handle:
            lib.glint_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_features(ctx: Context, env: Env, planes, width: int, height: int, tangent, x=None, lp=None, stream=None):
    """glint_mlp_features: the surrogate's inputs of every pixel under `env`:
    x (npix, 64) int16 tensor of BF16 bit patterns, lp (npix, K) float32."""
    import torch
    n = width * height
    dev = planes[0].device
    if x is None:
        x = torch.empty(n, 64, dtype=torch.int16, device=dev)
    if lp is None:
        lp = torch.empty(n, env.cfg.K, device=dev)
    g = _gbuffer(planes, width, height, tangent)
    _check(lib.glint_mlp_features(ctx.handle, env.handle, ctypes.byref(g), _dptr(x), _dptr(lp),
                                  _stream_handle(stream)))
    return x, lp


class Arena:
    """glint_arena: host bookkeeping of device-memory admission (first fit, coalescing)."""

    def __init__(self, nbytes: int, align: int = 256):
        self.handle = lib.glint_arena_create(nbytes, align)
        if not self.handle:
            raise GlintError(1, "glint_arena_create: align must be a power of two")

    def alloc(self, nbytes: int) -> int:
        return lib.glint_arena_alloc(self.handle, nbytes)

    def free(self, offset: int) -> int:
        return lib.glint_arena_free(self.handle, offset)

    @property
    def used(self) -> int:
        return lib.glint_arena_used(self.handle)

    @property
    def largest_free(self) -> int:
        return lib.glint_arena_largest_free(self.handle)

    def close(self):
        if self.handle:
            lib.glint_arena_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_tick(next_px, npix, tick_pixels: int, tile_pixels: int, max_items: int = 1 << 16):
    """glint_plan_tick: (items as (frame, first, count) rows, advanced next)."""
    nxt = np.ascontiguousarray(next_px, np.int64).copy()
    npx = np.ascontiguousarray(npix, np.int64)
    f = np.zeros(max_items, np.int32)
    first = np.zeros(max_items, np.int64)
    cnt = np.zeros(max_items, np.int32)
    n = lib.glint_plan_tick(nxt.ctypes.data, npx.ctypes.data, len(npx), tick_pixels, tile_pixels, f.ctypes.data,
                            first.ctypes.data, cnt.ctypes.data, max_items)
    return np.stack([f[:n].astype(np.int64), first[:n], cnt[:n].astype(np.int64)], 1), nxt


class Server:
    """glint_server: continuous batching of frames submitted from host memory."""

    def __init__(self, ctx: Context, K: int, memory_budget: int, tick_pixels: int = 0, tile_pixels: int = 0,
                 max_frames: int = 0, max_inflight_ticks: int = 0, upload: bool = False):
        self.ctx = ctx
        self.desc = ServerDesc(memory_budget, tick_pixels, tile_pixels, max_frames, max_inflight_ticks, int(upload))
        h = ctypes.c_void_p()
        _check(lib.glint_server_create(ctx.handle, K, ctypes.byref(self.desc), ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def add_env(self, env: Env, mlp=None) -> int:
        i = ctypes.c_int()
        _check(lib.glint_server_add_env(self.handle, env.handle, mlp.handle if mlp is not None else None,
                                        ctypes.byref(i)))
        return i.value

    def update_env(self, env_id: int, texels):
        """glint_server_update_env: later frames of this map use `texels` (device)."""
        _check(lib.glint_server_update_env(self.handle, env_id, _dptr(texels)))
        self._keep[("env", env_id, id(texels))] = texels

    def submit(self, env_id: int, planes, width: int, height: int, out, seed: int = 0,
               evaluator: int = EVAL_E1, tangent=None) -> int:
        """planes, tangent, out: host tensors, kept alive until polled (all pinned: shaded in place unless
        the server uploads; else copied in and out)."""
        r = FrameRequest(env_id, width, height, seed & 0xFFFFFFFF, evaluator, _dptr(planes[0]), _dptr(planes[1]),
                         _dptr(planes[2]), _dptr(planes[3]), _dptr(tangent), _dptr(out))
        fid = ctypes.c_long()
        _check(lib.glint_server_submit(self.handle, ctypes.byref(r), ctypes.byref(fid)))
        self._keep[fid.value] = (planes, tangent, out)
        return fid.value

    def tick(self, stream=None) -> int:
        n = ctypes.c_int()
        _check(lib.glint_server_tick(self.handle, _stream_handle(stream), ctypes.byref(n)))
        return n.value

    def poll(self, max_done: int = 256):
        arr = (FrameDone * max_done)()
        n = ctypes.c_int()
        _check(lib.glint_server_poll(self.handle, arr, max_done, ctypes.byref(n)))
        out = []
        for i in range(n.value):
            d = arr[i]
            self._keep.pop(d.id, None)
            out.append((d.id, d.submit_s, d.admit_s, d.done_s))
        return out

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib.glint_server_stats_get(self.handle, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self.handle:
            lib.glint_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_generate(ctx: Context, env: Env, planes, width: int, height: int, tangent, e2_samples: int = 32,
                 stream=None):
    """glint_mlp_generate: training inputs, log-priors and E2 targets of every pixel."""
    import torch
    n = width * height
    dev = planes[0].device
    x = torch.empty(n, 64, dtype=torch.int16, device=dev)
    lp = torch.empty(n, env.cfg.K, device=dev)
    y = torch.empty(n, env.cfg.K, device=dev)
    g = _gbuffer(planes, width, height, tangent)
    _check(lib.glint_mlp_generate(ctx.handle, env.handle, ctypes.byref(g), e2_samples, _dptr(x), _dptr(lp), _dptr(y),
                                  _stream_handle(stream)))
    return x, lp, y


def normal_quantile(p, out=None, stream=None):
    """Phi^-1 of a device float32 tensor, as the shading kernel computes it."""
    import torch
    if out is None:
        out = torch.empty_like(p)
    _check(lib.glint_normal_quantile(p.data_ptr(), out.data_ptr(), p.numel(), _stream_handle(stream)))
    return out


def debug_buffers(npix: int, K: int, device="cuda", samples: int = 6):
    """Device tensors for every optional intermediate output of glint_shade
    (samples: 6 for the isotropic grid, 12 for the anisotropic one)."""
    import torch
    return {"p": torch.zeros(npix, K, device=device), "np": torch.zeros(npix, device=device),
            "vert": torch.zeros(npix, samples, 3, dtype=torch.int32, device=device),
            "w": torch.zeros(npix, samples, device=device), "nroot": torch.zeros(npix, samples, device=device),
            "counts": torch.zeros(npix, samples, K, device=device), "lo": torch.zeros(npix, 3, device=device)}
