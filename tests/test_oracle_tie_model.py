"""The oracle's tie model against a perturbed evaluation of the same frame
(CPU only).  The tie model claims that an evaluation whose subtree masses,
quantiles and gate thresholds are off by FP32-sized errors draws counts inside
the candidate set it enumerates.  Here the errors are made on purpose: the
map's texels are scaled by independent relative amounts of up to 2^-22 (a few
FP32 units, so every mass moves by far less than the model's e_P = 2^-14) and
the frame is shaded again with the tie model off.  Every count vector of the
perturbed run must lie in the unperturbed run's candidate set, its p_k within
the model's bound, and the draws that did move show that the perturbation
reached the decisions."""
import numpy as np

from paper_2507_02674_gb300 import synth
from tests._compare import compare_shade
from tests._pipeline import MethodParams, oracle_env, oracle_shade

ZERO_TIE = (0.0, 0.0, 0.0, 0.0, 0.0)


def _as_gpu(o):
    """The perturbed run's outputs in the layout compare_shade takes for the
    kernel's debug outputs (its FP64 count vector as the counts)."""
    return {"p": o.pk, "np": o.np_, "vert": o.vert.astype(np.int32), "w": o.wv, "nroot": o.nroot,
            "counts": o.cand[:, :, 0, :], "lo": o.lo}


def test_perturbed_evaluation_stays_in_the_candidate_sets(orc):
    mp = MethodParams(K=8, Wo=64, seed=5)
    env = synth.env_hdr(seed=3, W=128, H=64)
    gb = synth.gbuffer_random(4000, seed=17, width=4000)
    rows = gb.rows16()
    ref = oracle_shade(orc, rows, env, mp, tie=orc.TIE_DEFAULT, max_cand=64)
    rng = np.random.default_rng(9)
    rgba = env.rgba32().astype(np.float64)
    rgba[..., :3] *= 1.0 + rng.uniform(-2.0 ** -22, 2.0 ** -22, size=rgba[..., :3].shape)
    e = orc.env_full(rgba.astype(np.float32), env.scale, mp.K, mp.ell)
    pref = orc.prefilter(e, mp.R, mp.S, mp.s_min, mp.s_max, mp.Wo)
    pert = oracle_shade(orc, rows, env, mp, tie=ZERO_TIE, max_cand=2, env_pref=(e, pref))
    rep = compare_shade(orc, ref, _as_gpu(pert), pert.rgb)
    print(rep.summary())
    assert rep.ok(), rep.failures[:5]
    # the perturbation reached the draws: some count vectors differ from the
    # unperturbed run's FP64 outcome (and were accepted as tie candidates)
    moved = np.any(pert.cand[:, :, 0, :] != ref.cand[:, :, 0, :], axis=2) & (ref.ncand > 0)
    print(f"draw vectors moved by the perturbation: {int(moved.sum())} of {moved.size}")
    assert moved.sum() >= 1 and rep.trees_multi > 0
    # teeth: without the tie model the same moved draws are not accepted
    bare = oracle_shade(orc, rows, env, mp, tie=ZERO_TIE, max_cand=64)
    rep0 = compare_shade(orc, bare, _as_gpu(pert), pert.rgb)
    print(rep0.failures[:3])
    assert not rep0.ok()
    assert all("sample" in f for f in rep0.failures if f != "...")
