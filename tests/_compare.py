"""Element-by-element comparison of the CUDA shading outputs with the oracle.

Integer and index outputs are compared exactly: N_P (FP32 bits), grid vertices
(low 32 bits and level), the dithered trials of every tree root, and the bin
counts, which must be one of the oracle's valid count vectors for that tree (the
oracle lists every outcome that an FP32 evaluation of a near-tie decision can
give).  Floating-point outputs are compared with stated tolerances; radiance is
compared with the oracle's radiance for the count vectors the kernel produced.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

RAD_RTOL = 1e-4        # relative tolerance on radiance
RAD_ATOL_FRAC = 1e-6   # absolute floor, as a fraction of the largest smooth radiance
P_RTOL = 2.0 ** -14    # relative tolerance on p_k: the oracle's tie-model bound e_P
P_ATOL = 2.0 ** -23    # absolute floor on p_k: the tie model's absolute mass error
LO_RTOL = 1e-4
W_ATOL = 2e-6


@dataclass
class ShadeReport:
    npix: int = 0
    trees: int = 0
    trees_multi: int = 0          # trees whose oracle set had more than one valid outcome
    trees_unresolved: int = 0     # oracle enumeration overflowed (invariants only)
    radiance_skipped: int = 0     # pixels with an overflowed tree: radiance not compared
    nonunique: int = 0            # pixels whose p_k is not unique in FP32 (invariants only)
    nondefault: int = 0           # trees where the kernel took a non-nominal valid outcome
    max_p_rel: float = 0.0
    max_p_abs: float = 0.0
    max_lo_rel: float = 0.0
    max_rad_rel: float = 0.0
    failures: list = field(default_factory=list)

    def ok(self) -> bool:
        return not self.failures

    def summary(self) -> str:
        return (f"pixels={self.npix} trees={self.trees} multi={self.trees_multi} unresolved={self.trees_unresolved} "
                f"max|dp|={self.max_p_abs:.2e} "
                f"nondefault={self.nondefault} rad_skipped={self.radiance_skipped} nonunique={self.nonunique} max|dp/p|={self.max_p_rel:.2e} max|dLo/Lo|={self.max_lo_rel:.2e} "
                f"max|dL/L|={self.max_rad_rel:.2e} failures={len(self.failures)}")


def _rel(a, b, floor):
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def compare_shade(orc, o, gpu: dict, rgb_gpu: np.ndarray, integer_mode: bool = True, max_fail: int = 20,
                  nonunique=None, p_atol: float = P_ATOL, p_rtol: float = P_RTOL,
                  rad_rtol: float = RAD_RTOL) -> ShadeReport:
    """o: oracle.ShadeOracle for n pixels; gpu: numpy copies of the debug outputs
    for the same pixels (keys p, np, vert, w, nroot, counts, lo); rgb_gpu (n, 3).
    nonunique: optional mask of pixels whose p_k an FP32 evaluation may not
    reproduce (e.g. an E2 quadrature point on the validity boundary); for those
    only the invariants (N_P, grid, root trials, count conservation) are
    checked.  p_atol: absolute error allowed on p_k on top of P_RTOL (the tie
    model's absolute mass error).  rad_rtol: relative radiance tolerance (wider
    when the two sides' p_k may legitimately differ, e.g. by one stored code of
    a compressed weight)."""
    rep = ShadeReport(npix=len(o.np_))
    nu = np.zeros(len(o.np_), bool) if nonunique is None else np.asarray(nonunique, bool)
    rep.nonunique = int(nu.sum())
    K = o.pk.shape[1]

    def fail(msg):
        if len(rep.failures) < max_fail:
            rep.failures.append(msg)
        else:
            rep.failures.append("...")

    # N_P: the same FP32 operations on both sides
    bad = np.nonzero(o.np_.view(np.uint32) != gpu["np"].astype(np.float32).view(np.uint32))[0]
    for q in bad[:5]:
        fail(f"N_P pixel {q}: oracle {o.np_[q]!r} gpu {gpu['np'][q]!r}")
    fg_all = o.np_ > 0
    fg = fg_all & ~nu
    scale_lo = max(float(np.max(np.abs(o.lo))), 1e-30)

    # p_k and smooth radiance
    pr = _rel(gpu["p"][fg].astype(np.float64), o.pk[fg], 1e-30)
    pr = np.where(o.pk[fg] < 1e-30, np.abs(gpu["p"][fg]), pr)
    rep.max_p_rel = float(pr.max()) if pr.size else 0.0
    pa = np.abs(gpu["p"][fg].astype(np.float64) - o.pk[fg])
    rep.max_p_abs = float(pa.max()) if pa.size else 0.0
    over = pa > p_rtol * o.pk[fg] + p_atol
    if np.any(over):
        q, k = np.argwhere(over)[0]
        fail(f"p_k beyond the tie model: pixel {np.nonzero(fg)[0][q]} k={k} p={o.pk[fg][q, k]:.3e} "
             f"|dp|={pa[q, k]:.3e}")
    lr = _rel(gpu["lo"][fg].astype(np.float64), o.lo[fg], RAD_ATOL_FRAC * scale_lo)
    rep.max_lo_rel = float(lr.max()) if lr.size else 0.0
    if rep.max_lo_rel > LO_RTOL:
        fail(f"L_o rel error {rep.max_lo_rel:.3e}")

    # grid samples (on the anisotropic grid a nonunique pixel's cell itself may differ)
    vchk = fg_all & ~nu if getattr(o, "grid", 0) else fg_all
    vo = o.vert.copy()
    vo[..., :2] = vo[..., :2] & 0xFFFFFFFF
    vg = gpu["vert"].astype(np.int64)
    vg[..., :2] = vg[..., :2] & 0xFFFFFFFF
    badv = np.nonzero(np.any(vo[vchk] != vg[vchk], axis=(1, 2)))[0]
    for q in badv[:5]:
        fail(f"grid vertices pixel {np.nonzero(vchk)[0][q]}: oracle {vo[vchk][q].tolist()} "
             f"gpu {vg[vchk][q].tolist()}")
    wd = np.abs(gpu["w"][vchk] - o.wv[vchk])
    if wd.size and wd.max() > W_ATOL:
        fail(f"grid weights differ by {wd.max():.3e}")
    if integer_mode:
        badn = np.nonzero(np.any(gpu["nroot"][vchk] != o.nroot[vchk], axis=1))[0]
        for q in badn[:5]:
            fail(f"root trials pixel {np.nonzero(vchk)[0][q]}: oracle {o.nroot[vchk][q]} "
                 f"gpu {gpu['nroot'][vchk][q]}")
        # debug counts are float32: above 2^24 each carries a rounding of N 2^-24
        cs = gpu["counts"].astype(np.float64).sum(-1)
        nr = gpu["nroot"].astype(np.float64)
        badc = np.nonzero(np.any(np.abs(cs[fg_all] - nr[fg_all]) > (o.pk.shape[1] + 1) * nr[fg_all] * 2.0 ** -24,
                                 axis=1))[0]
        for q in badc[:5]:
            fail(f"counts do not sum to the root trials at pixel {np.nonzero(fg_all)[0][q]}")

    # counts: membership in the oracle's valid set; radiance for the chosen vectors
    cg = gpu["counts"].astype(np.float64)
    for q in np.nonzero(fg)[0]:
        nv = o.wv.shape[1]
        chosen = np.zeros((nv, K))
        nondefault = False
        unresolved = False
        for v in range(nv):
            rep.trees += 1
            nc = o.ncand[q, v]
            cvec = cg[q, v]
            if nc < 0:
                rep.trees_unresolved += 1
                if integer_mode and (cvec.sum() != o.nroot[q, v] or np.any(cvec < 0)):
                    fail(f"pixel {q} sample {v}: counts {cvec} do not sum to {o.nroot[q, v]}")
                unresolved = True
                continue
            if nc > 1:
                rep.trees_multi += 1
            cands = o.cand[q, v, :nc]
            # exact candidates carry tolerance 0; subtrees whose Gaussian rounding
            # cannot be called carry the oracle's propagated count tolerance
            tol = o.cand_err[q, v, :nc]
            if not integer_mode:
                tol = tol + 2e-5 * np.abs(cands) + 1e-5
            hit = np.nonzero(np.all(np.abs(cands - cvec[None, :]) <= tol, axis=1))[0]
            if hit.size == 0:
                d = cvec - cands[0]
                fail(f"pixel {q} sample {v}: N={o.nroot[q, v]:.0f} gpu-oracle={d.tolist()} "
                     f"tol={tol[0].tolist()} ncand={nc}")
                chosen[v] = cands[0]
                continue
            if np.any(tol[hit[0]] > 0):
                # an interval candidate (counts known to the oracle only within
                # its tie-model tolerance): the radiance is evaluated at the
                # counts the kernel produced, which were just checked against it
                chosen[v] = cvec
                nondefault = True
            else:
                chosen[v] = cands[hit[0]]
            if hit[0] != 0:
                rep.nondefault += 1
                nondefault = True
        if unresolved:  # the oracle did not list every valid outcome of this pixel
            rep.radiance_skipped += 1
            continue
        ref = orc.radiance(o, q, chosen) if nondefault else o.rgb[q]
        err = np.abs(rgb_gpu[q] - ref)
        bound = rad_rtol * np.abs(ref) + RAD_ATOL_FRAC * scale_lo
        rel = float(np.max(err / np.maximum(np.abs(ref), RAD_ATOL_FRAC * scale_lo)))
        rep.max_rad_rel = max(rep.max_rad_rel, rel)
        if np.any(err > bound):
            fail(f"radiance pixel {q}: gpu {rgb_gpu[q].tolist()} oracle {ref.tolist()} rel {rel:.3e}")
    bg = ~fg_all
    if np.any(rgb_gpu[bg] != 0):
        fail("background / empty-footprint pixels are not black")
    return rep
