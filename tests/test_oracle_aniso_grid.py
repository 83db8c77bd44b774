"""Pins of the oracle's anisotropic grid (the footprint's level, anisotropy and
orientation cell, our reading of the anisotropic grids of Sec. 3.3): weights form a partition of
unity; a round footprint reduces to the isotropic grid's two levels and
lattices; an elongated, rotated footprint lands in the cell its axes and angle
predict; counts conserve N; the estimator averages to the smooth radiance.
CPU only."""
import numpy as np
import pytest

from paper_2507_02674_gb300 import synth
from tests._pipeline import MethodParams, oracle_env, oracle_lut


@pytest.fixture(scope="module")
def frame(orc):
    mp = MethodParams(K=4, Wo=64)
    env = synth.env_tiny(0)
    e, pref = oracle_env(orc, env, mp)
    return mp, e, pref, oracle_lut(orc, mp)


def _shade(orc, frame, rows, grid, seed=0, max_cand=1):
    mp, e, pref, lut = frame
    return orc.shade(rows, pref, mp.s_min, mp.s_max, lut, e.levels, seed, True, tie=[0, 0, 0, 0, 0],
                     max_cand=max_cand, grid=grid)


def _rows(n, rng, jac):
    gb = synth.gbuffer_random(n, seed=int(rng.integers(1 << 30)))
    rows = gb.rows16()
    rows[:, 3] = 1e4
    rows[:, 12:16] = jac
    return rows


def _keys(o):
    k = o.vert[..., 2]
    return k & 0x3FF, (k >> 10) & 3, (k >> 12) & 7


def test_partition_of_unity_and_rare_flags(orc, frame):
    rng = np.random.default_rng(1)
    gb = synth.gbuffer_random(2000, seed=3)
    o = _shade(orc, frame, gb.rows16(), 1)
    fg = o.np_ > 0
    assert o.wv.shape[1] == 12
    np.testing.assert_allclose(o.wv[fg].sum(1), 1.0, atol=1e-12)
    assert np.all(o.wv[fg] >= -1e-15)
    assert np.all(o.vert[fg][..., 2] & 0x8000)
    assert o.grid_flags[fg].mean() < 0.02


def test_round_footprint_reduces_to_the_isotropic_grid(orc, frame):
    rng = np.random.default_rng(2)
    s = 10.0 ** rng.uniform(-3, -1, size=(300, 1))
    rows = _rows(300, rng, np.c_[s, 0 * s, 0 * s, s])
    iso = _shade(orc, frame, rows, 0)
    ani = _shade(orc, frame, rows, 1)
    lvl, an, ori = _keys(ani)
    live = ani.wv > 1e-6  # the path also steps A, with weight f_A ~ 0 (area is FP32)
    assert np.all(an[live] == 0) and np.all(ori[live] == 0)
    assert np.all(ani.grid_flags == 1)  # a round footprint has no well-defined orientation
    for q in range(300):
        l0 = iso.vert[q, 0, 2]
        for lv in (0, 1):
            sel = ((lvl[q] & 0x3FF) == ((l0 + lv) & 0x3FF)) & live[q]
            # the cell's weight at each level is the isotropic grid's level weight
            assert ani.wv[q, sel].sum() == pytest.approx(iso.wv[q, 3 * lv:3 * lv + 3].sum(), abs=1e-6)
            # and its lattice vertices are the isotropic ones of that level
            iso_v = {tuple(v) for v in iso.vert[q, 3 * lv:3 * lv + 3, :2].tolist()}
            ani_v = {tuple(v) for v in ani.vert[q, sel, :2].tolist()}
            assert ani_v <= iso_v


@pytest.mark.parametrize("k", [0, 2, 5, 7])
def test_elongated_rotated_footprint_lands_in_its_cell(orc, frame, k):
    """Axes s 2^1.3 and s / 2^1.3 (anisotropy A = 1.3) rotated by
    (k + 0.6) pi/8 (O = k + 0.6): the cell spans a in {1, 2} with weight 0.3
    at a = 2, and o in {k, k+1} with weight 0.4 at o = k."""
    rng = np.random.default_rng(k)
    phi = (k + 0.6) * np.pi / 8
    R = np.array([[np.cos(phi), -np.sin(phi)], [np.sin(phi), np.cos(phi)]])
    s = 1e-2
    J = R @ np.diag([s * 2 ** 1.3, s / 2 ** 1.3])  # columns: d(uv)/dx, d(uv)/dy
    jac = np.array([J[0, 0], J[1, 0], J[0, 1], J[1, 1]])
    rows = _rows(50, rng, jac)
    o = _shade(orc, frame, rows, 1)
    assert np.all(o.grid_flags == 0)
    lvl, an, ori = _keys(o)
    for q in range(50):
        w = o.wv[q]
        live = w > 1e-9
        assert set(an[q][live].tolist()) <= {1, 2}
        assert set(ori[q][live].tolist()) <= {k, (k + 1) % 8}
        assert w[an[q] == 2].sum() == pytest.approx(0.3, abs=1e-6)
        assert w[ori[q] == k].sum() == pytest.approx(0.4, abs=1e-6)


def test_counts_conserved_and_estimator_converges(orc, frame):
    rng = np.random.default_rng(4)
    gb = synth.gbuffer_random(40, seed=9, n_lo=1e3, n_hi=1e4)
    rows = gb.rows16()
    t = rng.uniform(0, np.pi, size=40)
    sx, sy = 10.0 ** rng.uniform(-2, -1, size=40), 10.0 ** rng.uniform(-3, -2, size=40)
    rows[:, 12] = np.cos(t) * sx
    rows[:, 13] = np.sin(t) * sx
    rows[:, 14] = -np.sin(t) * sy
    rows[:, 15] = np.cos(t) * sy
    rows[:, 3] = 2e4 / (sx * sy)  # N_P = 2e4
    acc = None
    S = 150
    for seed in range(S):
        o = _shade(orc, frame, rows, 1, seed=seed)
        c = o.cand[:, :, 0, :]
        np.testing.assert_array_equal(c.sum(-1), o.nroot)
        acc = o.rgb if acc is None else acc + o.rgb
    fg = (o.np_ > 0) & (o.lo.sum(1) > 0)
    rel = np.abs(acc[fg] / S - o.lo[fg]).sum(1) / o.lo[fg].sum(1)
    assert np.median(rel) < 0.02, np.median(rel)
