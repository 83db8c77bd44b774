"""Method parameters shared by the oracle tests and the GPU parity tests, and a
helper that runs the oracle's full pipeline (decompose, pyramid, filter,
tables, shade).  Test infrastructure."""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class MethodParams:
    K: int = 4                     # radiance levels (power of two)
    R: int = 8                     # filtered levels, sqrt(alpha) evenly in [s_min, s_max]
    S: int = 64                    # filter samples per output texel
    Wo: int = 64                   # widest filtered level (level r: ~2 pi / alpha_r texels, at most Wo)
    ell: float = 1e-4              # clip of the minimum radiance
    s_min: float = math.sqrt(0.02)
    s_max: float = math.sqrt(0.5)
    nlut: int = 64                 # table resolution
    Q: int = 128                   # table quadrature points per axis
    seed: int = 0
    integer_mode: bool = True
    log_weights: bool = False      # fuzzy weights interpolated in log space (Sec. 7)
    wfmt: int = 0                  # storage of the filtered weights (0 float32, 1 float16, 2 unorm16, 3 unorm8)

    def with_(self, **kw) -> "MethodParams":
        return replace(self, **kw)


_LUT_CACHE = {}


def oracle_lut(orc, mp: MethodParams) -> np.ndarray:
    key = (mp.nlut, mp.Q)
    if key not in _LUT_CACHE:
        _LUT_CACHE[key] = orc.lut(mp.nlut, mp.Q)
    return _LUT_CACHE[key]


def oracle_env(orc, env, mp: MethodParams):
    e = orc.env_full(env.rgba32(), env.scale, mp.K, mp.ell, mp.log_weights)
    pref = orc.prefilter(e, mp.R, mp.S, mp.s_min, mp.s_max, mp.Wo, wfmt=mp.wfmt)
    return e, pref


def oracle_shade(orc, rows16: np.ndarray, env, mp: MethodParams, tie=None, max_cand: int = 64, env_pref=None,
                 evaluator: int = 0, tangents=None, e2_S: int = 16, pk_in=None, draw: int = 0, gamma: float = 0.0,
                 grid: int = 0):
    e, pref = env_pref if env_pref is not None else oracle_env(orc, env, mp)
    lut = oracle_lut(orc, mp)
    return orc.shade(rows16, pref, mp.s_min, mp.s_max, lut, e.levels, mp.seed, mp.integer_mode,
                     tie=orc.TIE_E2 if (tie is None and evaluator == 1) else (orc.TIE_DEFAULT if tie is None
                                                                                      else tie),
                     max_cand=max_cand, evaluator=evaluator,
                     tangents=tangents, e2_S=e2_S, env=e, pk_in=pk_in, draw=draw, gamma=gamma, grid=grid)
