"""Plain FP64 CPU oracle for per-pixel glint shading under an environment map.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this
package.  The product library never imports, links or runs it, and the two
share no code.

The arithmetic lives in ``glint_oracle.c`` (each function cites the passage of
Kneiphof & Klein, "Real-Time Image-based Lighting of Glints", EGSR 2025, that
it follows).  This module compiles that file with gcc and wraps it with
ctypes; it only converts arrays.

Parity status of each function: every function is pinned by tests under
``tests/test_oracle_*.py`` against closed forms, the paper's printed outcome
table (Fig. "gatingdiagram"), brute force or independent library routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glint_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# Tie model of the FP32 kernel (see or_shade in glint_oracle.c):
# relative error of subtree probability masses, of the FP32 normal quantile,
# of an FP32 exp2/log2 chain, an absolute floor of every threshold, and an
# absolute error of subtree masses.
# The absolute mass error, 2^-23, for every evaluator: a fuzzy weight 1 - t of
# a texel whose brightness lies just below a radiance level (Sec. 4, Eq.
# wkdefpractice) is a small difference of FP32 values, so its rounding, up to
# ~2^-24 of the bracket, is an absolute error; the pyramid, the prefilter and
# the E2 quadrature average texels (weights summing to one) and p_k = V W_k
# with V <= 1, so no mass carries more than 2^-24 of it, plus its own
# roundings: bound 2^-23.  (Measured on a GB300: 1.95e-11 on p_k = 5.6e-8 over
# every pixel of the 1080p frame for E1; E2, whose FP32 texel coordinates also
# move mass between neighbouring texels, 5e-10 at K = 8 and 3.7e-8 beyond the
# relative bound at K = 16, where the sixteen levels sit closer.)
TIE_DEFAULT = (2.0 ** -14, 2.0 ** -20, 2.0 ** -21, 2.0 ** -23, 2.0 ** -23)
# The E2 quadrature reads single pyramid texels per point at FP32 texel
# coordinates (up to ~1.2e-4 texel of error, w_k changing by at most 1 per
# texel), so a mass carried by a few points moves by ~1e-4 of itself
# (measured on a GB300: 8.9e-5): relative bound 2^-12.
TIE_E2 = (2.0 ** -12, 2.0 ** -20, 2.0 ** -21, 2.0 ** -23, 2.0 ** -23)
NV = 6


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2, no FP
    contraction; OpenMP over pixels and texels where gcc has it)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                "-o", _LIB, _SRC, "-lm"]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.run(base, check=True)
    return _LIB


def set_threads(n: int) -> None:
    """Threads of the oracle's pixel and texel loops (0: every core)."""
    _load().or_set_threads(int(n))


def threads() -> int:
    return _load().or_max_threads()


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        D = ctypes.c_double
        I = ctypes.c_int
        L = ctypes.c_long
        P = ctypes.c_void_p
        U = ctypes.c_uint32
        lib.or_pcg4d.argtypes = [P, P]
        lib.or_xi.argtypes = [U]
        lib.or_xi.restype = D
        lib.or_node_stream.argtypes = [ctypes.c_int, P, P]
        lib.or_node_stream.restype = None
        lib.or_node_uniforms.argtypes = [U, U, U, U, ctypes.c_int, P]
        lib.or_node_uniforms.restype = None
        lib.or_ndtri.argtypes = [D]
        lib.or_ndtri.restype = D
        lib.or_eps.restype = D
        lib.or_dualgated_thresholds.argtypes = [D, D, P, P, P]
        lib.or_dualgated.argtypes = [D, D, D, D, I, P, P]
        lib.or_singlegated_old.argtypes = [D, D, D, D]
        lib.or_singlegated_old.restype = D
        lib.or_singlegated.argtypes = [D, D, D, D]
        lib.or_singlegated.restype = D
        lib.or_ggx_d.argtypes = [D, D]
        lib.or_ggx_d.restype = D
        lib.or_lut.argtypes = [I, I, P]
        lib.or_lut_point.argtypes = [D, D, I, P]
        lib.or_projected_area.argtypes = [D, I]
        lib.or_projected_area.restype = D
        lib.or_dualgated_many.argtypes = [D, D, P, P, L, I, P, P]
        lib.or_total_area.argtypes = [D, I]
        lib.or_total_area.restype = D
        lib.or_env_decompose.argtypes = [P, I, I, D, I, D, P, P, P, I]
        lib.or_mip_count.argtypes = [I]
        lib.or_mip_count.restype = I
        lib.or_env_mips.argtypes = [P, I, I, I, P]
        lib.or_prefilter_table.argtypes = [I, I, D, D, I, I, P, P]
        lib.or_filtered_widths.argtypes = [I, D, D, I, P]
        lib.or_prefilter.argtypes = [P, I, I, I, P, P, I, I, P, P, L, P]
        lib.or_prefilter_exact.argtypes = [P, I, I, I, D, P, L, P]
        lib.or_shade.argtypes = [P, L, P, I, P, I, D, D, P, I, P, I, U, I, P, I,
                                 P, P, P, P, P, P, P, P, P, P, P, I, P, I, P, I, I, P, P, I, D, I, P]
        lib.or_e2_pk.argtypes = [P, P, P, ctypes.c_float, ctypes.c_float, I, P, I, I, I, I, P]
        lib.or_e2_pk.restype = I
        lib.or_mlp_features.argtypes = [P, P, L, P, I, P, I, D, D, P, I, I, P, P, P]
        lib.or_mlp_features.restype = None
        lib.or_shade.restype = L
        lib.or_radiance.argtypes = [P, P, D, P, I, P, P, P, I, D, I]
        lib.or_multinomial.argtypes = [P, I, D, U, U, U, U, I, P, I]
        lib.or_set_threads.argtypes = [I]
        lib.or_set_threads.restype = None
        lib.or_max_threads.restype = I
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- primitives
def pcg4d(v) -> np.ndarray:
    lib = _load()
    a = np.ascontiguousarray(np.asarray(v, dtype=np.uint32).reshape(4))
    out = np.zeros(4, np.uint32)
    lib.or_pcg4d(_ptr(a), _ptr(out))
    return out


def xi(h: int) -> float:
    return _load().or_xi(int(h) & 0xFFFFFFFF)


def node_stream(node: int) -> tuple:
    """(hash call index, first output word) of tree node `node`'s two uniforms."""
    c, w = ctypes.c_int(), ctypes.c_int()
    _load().or_node_stream(int(node), ctypes.byref(c), ctypes.byref(w))
    return c.value, w.value


def node_uniforms(key, seed: int, node: int) -> np.ndarray:
    """xi1, xi2 of tree node `node` at the grid vertex keyed (x, y, level key)."""
    out = np.zeros(2)
    _load().or_node_uniforms(int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF, int(key[2]) & 0xFFFFFFFF,
                             int(seed) & 0xFFFFFFFF, int(node), _ptr(out))
    return out


def ndtri(p: float) -> float:
    return _load().or_ndtri(float(p))


def eps() -> float:
    return _load().or_eps()


def dualgated_thresholds(N: float, p: float):
    lib = _load()
    T = np.zeros(4)
    mu = ctypes.c_double()
    sg = ctypes.c_double()
    lib.or_dualgated_thresholds(float(N), float(p), _ptr(T), ctypes.byref(mu), ctypes.byref(sg))
    return T, mu.value, sg.value


def dualgated(N: float, p: float, xi1: float, xi2: float, integer_mode: bool = False):
    lib = _load()
    n = ctypes.c_double()
    nb = ctypes.c_double()
    lib.or_dualgated(float(N), float(p), float(xi1), float(xi2), int(integer_mode), ctypes.byref(n),
                     ctypes.byref(nb))
    return n.value, nb.value


def singlegated_old(N, p, xi1, xi2) -> float:
    return _load().or_singlegated_old(float(N), float(p), float(xi1), float(xi2))


def singlegated(N, p, xi1, xi2) -> float:
    return _load().or_singlegated(float(N), float(p), float(xi1), float(xi2))


def ggx_d(cos_h: float, alpha: float) -> float:
    return _load().or_ggx_d(float(cos_h), float(alpha))


def lut(n: int = 64, Q: int = 128) -> np.ndarray:
    """(n, n, 4) table over (sqrt alpha rows, mu_o columns): V, U, A, B."""
    out = np.zeros((n, n, 4))
    _load().or_lut(n, Q, _ptr(out))
    return out


def lut_point(mu: float, alpha: float, Q: int = 128) -> np.ndarray:
    """(V, U, A, B) at one (mu_o, alpha) by the table's quadrature."""
    out = np.zeros(4)
    _load().or_lut_point(float(mu), float(alpha), int(Q), _ptr(out))
    return out


def projected_area(alpha: float, Q: int = 128) -> float:
    return _load().or_projected_area(float(alpha), int(Q))


def dualgated_many(N: float, p: float, xi1, xi2, integer_mode: bool = False):
    lib = _load()
    xi1 = np.ascontiguousarray(xi1, dtype=np.float64)
    xi2 = np.ascontiguousarray(np.broadcast_to(xi2, xi1.shape), dtype=np.float64)
    n = np.zeros(xi1.shape)
    nb = np.zeros(xi1.shape)
    lib.or_dualgated_many(float(N), float(p), _ptr(xi1), _ptr(xi2), xi1.size, int(integer_mode), _ptr(n), _ptr(nb))
    return n, nb


def total_area(alpha: float, Q: int = 128) -> float:
    return _load().or_total_area(float(alpha), int(Q))


# ---------------------------------------------------------------- environment
@dataclass
class EnvOracle:
    levels: np.ndarray      # (K,)
    lohi: np.ndarray        # (2,)
    ch0: np.ndarray         # (H, W, 3+K)
    mips: list              # list of (H>>m, W>>m, 3+K)
    mips_flat: np.ndarray


def env_decompose(rgba: np.ndarray, scale: float, K: int, ell: float, log_space: bool = False):
    lib = _load()
    rgba = np.ascontiguousarray(rgba, dtype=np.float32)
    H, W = rgba.shape[:2]
    L = np.zeros(K)
    lohi = np.zeros(2)
    ch0 = np.zeros((H, W, 3 + K))
    lib.or_env_decompose(_ptr(rgba), W, H, float(scale), K, float(ell), _ptr(L), _ptr(lohi), _ptr(ch0),
                         int(log_space))
    return L, lohi, ch0


def mip_count(H: int) -> int:
    return _load().or_mip_count(int(H))


def env_mips(ch0: np.ndarray):
    lib = _load()
    H, W, C = ch0.shape
    M = mip_count(H)
    total = sum((W >> m) * (H >> m) * C for m in range(M))
    flat = np.zeros(total)
    lib.or_env_mips(_ptr(np.ascontiguousarray(ch0)), W, H, C, _ptr(flat))
    levels, off = [], 0
    for m in range(M):
        n = (W >> m) * (H >> m) * C
        levels.append(flat[off:off + n].reshape(H >> m, W >> m, C))
        off += n
    return flat, levels


def env_full(rgba: np.ndarray, scale: float, K: int, ell: float, log_space: bool = False) -> EnvOracle:
    L, lohi, ch0 = env_decompose(rgba, scale, K, ell, log_space)
    flat, levels = env_mips(ch0)
    return EnvOracle(L, lohi, ch0, levels, flat)


def prefilter_table(R: int, S: int, s_min: float, s_max: float, W: int, H: int):
    table = np.zeros((R, S, 4))
    nvalid = np.zeros(R, np.int32)
    _load().or_prefilter_table(R, S, float(s_min), float(s_max), W, H, _ptr(table), _ptr(nvalid))
    return table, nvalid


@dataclass
class Filtered:
    widths: np.ndarray      # (R,) level widths (height = width / 2)
    flat: np.ndarray        # (total texels, C), levels concatenated
    levels: list            # per level (W_r / 2, W_r, C) views of flat
    s_min: float
    s_max: float


def filtered_widths(R: int, s_min: float, s_max: float, Wmax: int) -> np.ndarray:
    w = np.zeros(R, np.int32)
    _load().or_filtered_widths(R, float(s_min), float(s_max), int(Wmax), _ptr(w))
    return w


WFMT_F32, WFMT_F16, WFMT_UNORM16, WFMT_UNORM8 = 0, 1, 2, 3


def quantize_weights(flat: np.ndarray, wfmt: int) -> np.ndarray:
    """The filtered maps' weight channels (columns 3..) as the stored format
    gives them back (Sec. 7 "Texture Precision"): float16 rounded to nearest
    even, or unorm codes round(W (2^b - 1)) of the weight clamped to [0, 1]
    (ties to even), divided back.  RGB is kept."""
    out = np.array(flat, dtype=np.float64, copy=True)
    w = out[:, 3:]
    if wfmt == WFMT_F16:
        out[:, 3:] = w.astype(np.float16).astype(np.float64)
    elif wfmt in (WFMT_UNORM16, WFMT_UNORM8):
        m = 65535.0 if wfmt == WFMT_UNORM16 else 255.0
        out[:, 3:] = np.rint(np.clip(w, 0.0, 1.0) * m) / m
    elif wfmt != WFMT_F32:
        raise ValueError(wfmt)
    return out


def prefilter(env: EnvOracle, R: int, S: int, s_min: float, s_max: float, Wmax: int, idx=None, wfmt: int = 0):
    """Filtered environment as a Filtered (all levels), or only the listed flat
    texel indices of the concatenation as an (n, C) array; weights stored in
    format wfmt (quantize_weights)."""
    lib = _load()
    H, W, C = env.ch0.shape
    table, nvalid = prefilter_table(R, S, s_min, s_max, W, H)
    widths = filtered_widths(R, s_min, s_max, Wmax)
    total = int(sum(int(w) * (int(w) // 2) for w in widths))
    if idx is None:
        flat = np.zeros((total, C))
        lib.or_prefilter(_ptr(env.mips_flat), W, H, C, _ptr(table), _ptr(nvalid), R, S, _ptr(widths), None, 0,
                         _ptr(flat))
        flat = quantize_weights(flat, wfmt)
        levels, off = [], 0
        for w in widths:
            n = int(w) * (int(w) // 2)
            levels.append(flat[off:off + n].reshape(int(w) // 2, int(w), C))
            off += n
        return Filtered(widths, flat, levels, s_min, s_max)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros((len(idx), C))
    lib.or_prefilter(_ptr(env.mips_flat), W, H, C, _ptr(table), _ptr(nvalid), R, S, _ptr(widths), _ptr(idx),
                     len(idx), _ptr(out))
    return quantize_weights(out, wfmt)


def prefilter_with(env: EnvOracle, table: np.ndarray, nvalid: np.ndarray, widths) -> list:
    """or_prefilter with a given sample table and level widths (tests plant
    mistakes in either); returns the levels as (W_r / 2, W_r, C) arrays."""
    lib = _load()
    H, W, C = env.ch0.shape
    R, S = table.shape[0], table.shape[1]
    widths = np.ascontiguousarray(widths, dtype=np.int32)
    nvalid = np.ascontiguousarray(nvalid, dtype=np.int32)
    total = int(sum(int(w) * (int(w) // 2) for w in widths))
    flat = np.zeros((total, C))
    lib.or_prefilter(_ptr(env.mips_flat), W, H, C, _ptr(np.ascontiguousarray(table, dtype=np.float64)),
                     _ptr(nvalid), R, S, _ptr(widths), None, 0, _ptr(flat))
    levels, off = [], 0
    for w in widths:
        n = int(w) * (int(w) // 2)
        levels.append(flat[off:off + n].reshape(int(w) // 2, int(w), C))
        off += n
    return levels


def prefilter_exact(ch0: np.ndarray, alpha: float, dirs: np.ndarray) -> np.ndarray:
    lib = _load()
    H, W, C = ch0.shape
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((len(dirs), C))
    lib.or_prefilter_exact(_ptr(np.ascontiguousarray(ch0)), W, H, C, float(alpha), _ptr(dirs), len(dirs), _ptr(out))
    return out


# ---------------------------------------------------------------- shading
@dataclass
class ShadeOracle:
    rgb: np.ndarray       # (n, 3) nominal outcome
    lo: np.ndarray        # (n, 3) smooth radiance L_o
    pk: np.ndarray        # (n, K)
    np_: np.ndarray       # (n,) float32 N_P
    vert: np.ndarray      # (n, 6, 3) int64 vertex x, y, level
    wv: np.ndarray        # (n, 6) sample weights
    nroot: np.ndarray     # (n, 6) trials at each tree root
    ncand: np.ndarray     # (n, 6) number of valid count vectors (-1: overflow)
    cand: np.ndarray      # (n, 6, max_cand, K)
    cand_err: np.ndarray  # (n, 6, max_cand, K)
    flags: np.ndarray     # (n,) decisions too close to call
    levels: np.ndarray    # (K,)
    e2_flags: np.ndarray  # (n,) E2 points on the validity boundary (0 for E1)
    draw: int = 0         # binomial approximation (0 dual-gated, 1 Eq. gated, 2 Eq. oldgated, 3 Wang 2020)
    gamma: float = 0.0    # Wang 2020 reflection probability
    grid: int = 0         # 0 isotropic (6 samples per pixel), 1 anisotropic (12)
    grid_flags: np.ndarray = None  # (n,) anisotropic cell decisions too close to call


def gbuffer_rows(planes) -> np.ndarray:
    """Stack the four (n, 4) G-buffer planes into the oracle's (n, 16) rows."""
    return np.ascontiguousarray(np.concatenate([np.asarray(p, np.float32).reshape(-1, 4) for p in planes], axis=1))


def shade(gb16: np.ndarray, pref: Filtered, s_min: float, s_max: float, lut_tab: np.ndarray, levels: np.ndarray,
          seed: int, integer_mode: bool = True, tie=TIE_DEFAULT, max_cand: int = 8, evaluator: int = 0,
          tangents=None, e2_S: int = 16, env: "EnvOracle | None" = None, pk_in=None, draw: int = 0,
          gamma: float = 0.0, grid: int = 0) -> ShadeOracle:
    """Per-pixel shading (or_shade).  evaluator 0 = E1, 1 = E2 (needs tangents
    and env), 2 = the p_k given in pk_in (npix x K), 3 = anisotropic E1 by
    multi-tap filtered look-ups (needs tangents)."""
    lib = _load()
    gb16 = np.ascontiguousarray(gb16, dtype=np.float32).reshape(-1, 16)
    n = gb16.shape[0]
    R = len(pref.widths)
    C = pref.flat.shape[1]
    widths = np.ascontiguousarray(pref.widths, dtype=np.int32)
    K = len(levels)
    flat = np.ascontiguousarray(pref.flat, dtype=np.float64)
    lut_tab = np.ascontiguousarray(lut_tab, dtype=np.float64)
    nlut = lut_tab.shape[0]
    levels = np.ascontiguousarray(levels, dtype=np.float64)
    tie_a = np.asarray(tie, dtype=np.float64)
    nv = 12 if grid else NV
    o = ShadeOracle(rgb=np.zeros((n, 3)), lo=np.zeros((n, 3)), pk=np.zeros((n, K)), np_=np.zeros(n, np.float32),
                    vert=np.zeros((n, nv, 3), np.int64), wv=np.zeros((n, nv)), nroot=np.zeros((n, nv)),
                    ncand=np.zeros((n, nv), np.int32), cand=np.zeros((n, nv, max_cand, K)),
                    cand_err=np.zeros((n, nv, max_cand, K)), flags=np.zeros(n, np.int32), levels=levels,
                    e2_flags=np.zeros(n, np.int32), draw=int(draw), gamma=float(gamma), grid=int(grid),
                    grid_flags=np.zeros(n, np.int32))
    if evaluator == 1:
        tangents = np.ascontiguousarray(tangents, dtype=np.float32).reshape(-1, 4)
        mips = env.mips_flat
        H, W = env.ch0.shape[:2]
    elif evaluator == 3:
        tangents = np.ascontiguousarray(tangents, dtype=np.float32).reshape(-1, 4)
        mips, W, H = None, 0, 0
    else:
        tangents, mips, W, H = None, None, 0, 0
    if evaluator == 2:
        pk_in = np.ascontiguousarray(np.asarray(pk_in, np.float64).reshape(n, K))
    else:
        pk_in = None
    lib.or_shade(_ptr(gb16), n, _ptr(flat), R, _ptr(widths), C, float(s_min), float(s_max), _ptr(lut_tab), nlut,
                 _ptr(levels), K, ctypes.c_uint32(seed & 0xFFFFFFFF), int(integer_mode), _ptr(tie_a), max_cand,
                 _ptr(o.rgb), _ptr(o.lo), _ptr(o.pk), _ptr(o.np_), _ptr(o.vert), _ptr(o.wv), _ptr(o.nroot),
                 _ptr(o.ncand), _ptr(o.cand), _ptr(o.cand_err), _ptr(o.flags), int(evaluator),
                 None if tangents is None else _ptr(tangents), int(e2_S), None if mips is None else _ptr(mips), W, H,
                 _ptr(o.e2_flags), None if pk_in is None else _ptr(pk_in), int(draw), float(gamma), int(grid),
                 _ptr(o.grid_flags))
    return o


def mlp_features(gb16: np.ndarray, tangents: np.ndarray, pref: Filtered, s_min: float, s_max: float,
                 lut_tab: np.ndarray, K: int, want_dirs: bool = False):
    """Inputs x (npix, 64) and log-priors lp (npix, K) of the p_k surrogate
    (or_mlp_features), and with want_dirs the five tap directions (npix, 5, 3)."""
    lib = _load()
    gb16 = np.ascontiguousarray(gb16, dtype=np.float32).reshape(-1, 16)
    n = gb16.shape[0]
    tangents = np.ascontiguousarray(tangents, dtype=np.float32).reshape(-1, 4)
    flat = np.ascontiguousarray(pref.flat, dtype=np.float64)
    widths = np.ascontiguousarray(pref.widths, dtype=np.int32)
    lut_tab = np.ascontiguousarray(lut_tab, dtype=np.float64)
    x = np.zeros((n, 64))
    lp = np.zeros((n, K))
    dirs = np.zeros((n, 5, 3)) if want_dirs else None
    lib.or_mlp_features(_ptr(gb16), _ptr(tangents), n, _ptr(flat), len(pref.widths), _ptr(widths), flat.shape[1],
                        float(s_min), float(s_max), _ptr(lut_tab), lut_tab.shape[0], K, _ptr(x), _ptr(lp),
                        None if dirs is None else _ptr(dirs))
    return (x, lp, dirs) if want_dirs else (x, lp)


def e2_pk(wo, n, t, ax: float, ay: float, S: int, env: EnvOracle, K: int):
    """E2 reflection probabilities of one pixel and its count of boundary points."""
    lib = _load()
    H, W, C = env.ch0.shape
    pk = np.zeros(K)
    f = lib.or_e2_pk(_ptr(np.ascontiguousarray(wo, np.float64)), _ptr(np.ascontiguousarray(n, np.float64)),
                     _ptr(np.ascontiguousarray(t, np.float64)), float(ax), float(ay), int(S), _ptr(env.mips_flat),
                     W, H, C, K, _ptr(pk))
    return pk, f


def radiance(o: ShadeOracle, q: int, counts: np.ndarray) -> np.ndarray:
    """Radiance of pixel q for a chosen (6, K) count array drawn from its candidate lists."""
    lib = _load()
    K = o.pk.shape[1]
    out = np.zeros(3)
    lo3 = np.ascontiguousarray(o.lo[q])
    pk = np.ascontiguousarray(o.pk[q])
    wv = np.ascontiguousarray(o.wv[q])
    nv = o.wv.shape[1]
    c = np.ascontiguousarray(counts, dtype=np.float64).reshape(nv, K)
    lib.or_radiance(_ptr(lo3), _ptr(pk), float(o.np_[q]), _ptr(o.levels), K, _ptr(wv), _ptr(c), _ptr(out),
                    int(o.draw), float(o.gamma), nv)
    return out


def multinomial(p, N: float, key=(0, 0, 0), seed: int = 0, integer_mode: bool = True, draw: int = 0) -> np.ndarray:
    lib = _load()
    p = np.ascontiguousarray(p, dtype=np.float64)
    K = len(p)
    out = np.zeros(K)
    lib.or_multinomial(_ptr(p), K, float(N), ctypes.c_uint32(key[0] & 0xFFFFFFFF), ctypes.c_uint32(key[1] & 0xFFFFFFFF),
                       ctypes.c_uint32(key[2] & 0xFFFFFFFF), ctypes.c_uint32(seed & 0xFFFFFFFF), int(integer_mode),
                       _ptr(out), int(draw))
    return out
