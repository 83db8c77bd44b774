"""The element-by-element comparison used by the GPU parity tests, checked on
the CPU: the oracle's own outputs, laid out as the kernel's debug buffers, pass
it; each planted mistake (a radiance off by 1e-3, one trial moved between two
bins of a tree whose outcome is unique, a wrong grid vertex, a wrong N_P bit)
fails it; counts moved inside an interval candidate's tolerance pass when the
radiance is the one those counts give, and fail when it is not."""
import numpy as np
import pytest

from paper_2507_02674_gb300 import synth
from tests._compare import compare_shade
from tests._pipeline import MethodParams, oracle_shade


@pytest.fixture(scope="module")
def case(orc):
    mp = MethodParams(K=4, Wo=64, seed=5)
    env = synth.env_tiny(0)
    gb = synth.gbuffer_random(300, seed=17)
    o = oracle_shade(orc, gb.rows16(), env, mp)
    assert np.all(o.ncand > 0)
    return o


def _as_kernel(o):
    gpu = {"p": o.pk.astype(np.float32), "np": o.np_.copy(), "vert": o.vert.copy(),
           "w": o.wv.astype(np.float32), "nroot": o.nroot.astype(np.float32),
           "counts": o.cand[:, :, 0, :].astype(np.float32), "lo": o.lo.astype(np.float32)}
    return gpu, o.rgb.copy()


def test_oracle_outputs_pass(orc, case):
    gpu, rgb = _as_kernel(case)
    rep = compare_shade(orc, case, gpu, rgb)
    assert rep.ok(), rep.failures
    assert rep.trees == 6 * int(np.sum(case.np_ > 0))


def test_radiance_off_fails(orc, case):
    gpu, rgb = _as_kernel(case)
    q = int(np.argmax(np.abs(case.rgb).sum(1)))
    rgb[q] *= 1.001
    assert not compare_shade(orc, case, gpu, rgb).ok()


def test_moved_trial_fails(orc, case):
    gpu, rgb = _as_kernel(case)
    # a tree with one exact outcome and at least one trial in bin 0
    sel = np.argwhere((case.ncand == 1) & np.all(case.cand_err[:, :, 0, :] == 0, axis=-1)
                      & (case.cand[:, :, 0, 0] >= 1))
    q, v = sel[0]
    gpu["counts"][q, v, 0] -= 1
    gpu["counts"][q, v, 1] += 1
    assert not compare_shade(orc, case, gpu, rgb).ok()


def test_wrong_vertex_fails(orc, case):
    gpu, rgb = _as_kernel(case)
    q = int(np.nonzero(case.np_ > 0)[0][0])
    gpu["vert"][q, 2, 0] += 1
    assert not compare_shade(orc, case, gpu, rgb).ok()


def test_wrong_np_bit_fails(orc, case):
    gpu, rgb = _as_kernel(case)
    q = int(np.nonzero(case.np_ > 0)[0][0])
    gpu["np"][q] = np.nextafter(gpu["np"][q], np.float32(np.inf))
    assert not compare_shade(orc, case, gpu, rgb).ok()


def test_interval_candidate_radiance_at_kernel_counts(orc, case):
    gpu, rgb = _as_kernel(case)
    # a tree whose outcome the oracle knows only within a tolerance: move
    # d <= tolerance trials between two bins (the sum is kept)
    err = case.cand_err[:, :, 0, :]
    cnt = case.cand[:, :, 0, :]
    d = np.floor(np.minimum(err[..., 0], err[..., 1]))
    sel = np.argwhere((d >= 1) & (cnt[..., 0] >= d))
    if sel.size == 0:
        pytest.skip("no interval candidate with a tolerance of one trial in this case")
    q, v = sel[0]
    gpu["counts"][q, v, 0] -= d[q, v]
    gpu["counts"][q, v, 1] += d[q, v]
    moved = gpu["counts"][q].astype(np.float64)
    rgb_moved = orc.radiance(case, q, moved)
    rgb[q] = rgb_moved
    assert compare_shade(orc, case, gpu, rgb).ok()
    if np.max(np.abs(rgb_moved - case.rgb[q]) / np.abs(case.rgb[q])) > 2e-4:
        rgb[q] = case.rgb[q]  # the candidate's radiance no longer matches the moved counts
        assert not compare_shade(orc, case, gpu, rgb).ok()
