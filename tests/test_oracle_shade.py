"""Pins of the oracle's per-pixel shading: footprint and grid (Sec. 3.2, Sec. 3.3
Eq. anisogrid), the hierarchical multinomial (Sec. 5), and the glint radiance
(Sec. 4 Eq. iblglints:fin) against invariants, limits and brute force.  CPU only."""
import math

import numpy as np
import pytest

from paper_2507_02674_gb300 import synth
from tests._pipeline import MethodParams, oracle_env, oracle_shade

ZERO_TIE = (0.0, 0.0, 0.0, 0.0)


@pytest.fixture(scope="module")
def sphere_case(orc):
    mp = MethodParams(K=4, Wo=64)
    env = synth.env_tiny(0)
    gb = synth.gbuffer_sphere()
    ep = oracle_env(orc, env, mp)
    o = oracle_shade(orc, gb.rows16(), env, mp, env_pref=ep)
    return mp, env, gb, ep, o


def test_footprint_count(sphere_case):
    """N_P = N_0 |P| with |P| the absolute determinant of the uv Jacobian
    (Sec. 3.2), FP32 within 2 ulp of the FP64 value."""
    mp, env, gb, ep, o = sphere_case
    r = gb.rows16().astype(np.float64)
    fg = r[:, 3] > 0
    det = np.abs(r[:, 12] * r[:, 15] - r[:, 14] * r[:, 13])
    want = r[:, 3] * det
    assert np.all(o.np_[~fg] == 0)
    assert np.allclose(o.np_[fg], want[fg], rtol=2.5e-7)
    assert np.all(o.rgb[~fg] == 0)


def test_grid_samples(sphere_case):
    """Six samples: three triangle vertices at levels l0 and l0 + 1 with
    l0 = floor(log2 sqrt|P|); weights are barycentric times level weights and
    sum to one (Eq. anisogrid); the two other corners of a triangle are the
    (1,0)/(0,1) and (1,1) neighbours of its first corner."""
    mp, env, gb, ep, o = sphere_case
    r = gb.rows16().astype(np.float64)
    fg = o.np_ > 0
    area = np.abs(r[:, 12] * r[:, 15] - r[:, 14] * r[:, 13])
    L = 0.5 * np.log2(np.where(fg, area, 1.0))
    l0 = o.vert[:, 0, 2]
    frac = L - np.floor(L)
    safe = fg & (frac > 1e-6) & (frac < 1 - 1e-6)
    assert np.all(l0[safe] == np.floor(L[safe]))
    assert np.all(o.vert[fg, 3, 2] == l0[fg] + 1)
    assert np.allclose(o.wv[fg].sum(1), 1.0, atol=1e-12)
    assert np.all(o.wv[fg] >= -1e-12)
    for lv in (0, 3):
        v0, v1, v2 = o.vert[fg, lv, :2], o.vert[fg, lv + 1, :2], o.vert[fg, lv + 2, :2]
        assert np.all(v2 - v0 == 1)
        d = v1 - v0
        assert np.all(((d[:, 0] == 1) & (d[:, 1] == 0)) | ((d[:, 0] == 0) & (d[:, 1] == 1)))
    # level weights 1 - f and f
    f_lvl = o.wv[fg, 3:].sum(1)
    assert np.allclose(f_lvl, frac[fg], atol=1e-6)


def _vertex_weights(o, q):
    d = {}
    for v in range(6):
        key = tuple(int(x) for x in o.vert[q, v])
        d[key] = d.get(key, 0.0) + o.wv[q, v]
    return d


def test_grid_weights_continuous(orc):
    """Moving the shading point by a tiny uv offset changes the vertex weights by
    a tiny amount, even across triangle and cell edges (Sec. 3.3: outcomes are
    interpolated linearly over the triangle grid)."""
    mp = MethodParams(K=2, Wo=16)
    env = synth.env_constant(1.0)
    rng = np.random.default_rng(3)
    n = 400
    gb = synth.gbuffer_random(n, seed=5)
    rows = gb.rows16()
    rows[:, 12:16] = [0.01, 0.0, 0.0, 0.01]        # |P| = 1e-4, cells of size 2^-7..2^-6
    rows[:, 8:10] = rng.uniform(-3, 3, size=(n, 2))
    rows2 = rows.copy()
    rows2[:, 8] += np.float32(3e-5)
    ep = oracle_env(orc, env, mp)
    o1 = oracle_shade(orc, rows, env, mp, env_pref=ep, tie=ZERO_TIE)
    o2 = oracle_shade(orc, rows2, env, mp, env_pref=ep, tie=ZERO_TIE)
    changed = 0
    for q in range(n):
        a, b = _vertex_weights(o1, q), _vertex_weights(o2, q)
        keys = set(a) | set(b)
        dist = sum(abs(a.get(k, 0.0) - b.get(k, 0.0)) for k in keys)
        changed += set(a) != set(b)
        assert dist < 0.05, (q, dist)
    assert changed > 0  # some points crossed an edge


def test_count_conservation_and_dither(sphere_case):
    """Each sample's counts sum to its trials (the bins of one multinomial, Sec. 4),
    and the dithered trials are floor(N_P) or floor(N_P) + 1 with mean N_P."""
    mp, env, gb, ep, o = sphere_case
    fg = o.np_ > 0
    nom = o.cand[:, :, 0, :]
    assert np.array_equal(nom.sum(-1)[fg], o.nroot[fg])
    ok = o.ncand > 0
    for q, v in zip(*np.nonzero(ok)):
        for c in range(o.ncand[q, v]):
            assert o.cand[q, v, c].sum() == o.nroot[q, v]
    fl = np.floor(o.np_[fg].astype(np.float64))[:, None]
    d = o.nroot[fg] - fl
    assert np.all((d == 0) | (d == 1))
    resid = (o.nroot[fg] - o.np_[fg, None].astype(np.float64)).mean()
    assert abs(resid) < 4 * 0.5 / math.sqrt(d.size)
    assert np.all(o.cand[fg] >= 0)


def test_candidates_reduce_to_nominal_without_tie_model(orc, sphere_case):
    mp, env, gb, ep, o = sphere_case
    o0 = oracle_shade(orc, gb.rows16(), env, mp, env_pref=ep, tie=ZERO_TIE)
    fg = o0.np_ > 0
    assert np.all(o0.ncand[fg] == 1)
    assert np.array_equal(o0.cand[:, :, 0], o.cand[:, :, 0])
    assert np.array_equal(o0.rgb, o.rgb)
    assert (o.ncand > 1).mean() < 0.05


def test_k2_tree_is_one_binomial(orc):
    """With K = 2 the hierarchy is a single call of Alg. 1 on p_1 / (p_1 + p_2)."""
    for N in (0.0, 1.0, 2.0, 3.0, 17.0, 1000.0):
        for p in ((0.3, 0.7), (0.999, 0.001), (1e-6, 1.0)):
            for key in ((1, 2, 3), (99, 7, 5)):
                c = orc.multinomial(p, N, key, seed=11)
                h = orc.pcg4d([key[0], key[1], key[2] | (1 << 16), 11])
                n, nb = orc.dualgated(N, p[0] / (p[0] + p[1]), orc.xi(h[1]), orc.xi(h[2]), True)
                assert (c[0], c[1]) == (n, nb)


@pytest.mark.parametrize("K,N", [(4, 50.0), (8, 1000.0), (16, 20000.0)])
def test_multinomial_marginal_means(orc, K, N):
    """Hierarchical sampling of dual-gated binomials approximates the multinomial
    (Sec. 5): the marginal means over many seeds are N p_k within 5 standard
    errors plus the approximation's own bias.  Alg. 1 centres the Gaussian part on
    1 + (N-2) p instead of the binomial's N p, a shift of (1 - 2p) per draw when
    neither gate fires, so each tree level can move a bin by up to one count."""
    rng = np.random.default_rng(K)
    p = rng.dirichlet(np.ones(K) * 0.7)
    draws = np.array([orc.multinomial(p, N, (i, 3 * i + 1, 2), seed=77) for i in range(3000)])
    assert np.all(draws.sum(1) == N)
    m = draws.mean(0)
    se = np.sqrt(N * p * (1 - p) / len(draws)) + 1e-9
    assert np.all(np.abs(m - N * p) < 5 * se + math.log2(K)), (m, N * p)


def test_white_furnace_identity_and_convergence(orc):
    """Constant environment (Sec. 6 'White Furnace'): all radiance sits in level K,
    so L^_o = L_o M_K / (N_P p_K) exactly, and the mean over seeds of L^_o converges
    to the smooth L_o (the glint model's expectation is the smooth model)."""
    mp = MethodParams(K=4, Wo=16)
    env = synth.env_constant(1.0)
    gb = synth.gbuffer_sphere(16, 16, N0=2e3)
    rows = gb.rows16()
    ep = oracle_env(orc, env, mp)
    acc = None
    nseed = 300
    for s in range(nseed):
        o = oracle_shade(orc, rows, env, mp.with_(seed=s), env_pref=ep, tie=ZERO_TIE)
        fg = o.np_ > 0
        MK = (o.wv[:, :, None] * o.cand[:, :, 0, :]).sum(1)[:, -1]
        with np.errstate(invalid="ignore", divide="ignore"):
            want = o.lo * (MK / (o.np_ * o.pk[:, -1]))[:, None]
        assert np.allclose(o.rgb[fg], want[fg], rtol=1e-12)
        acc = o.rgb if acc is None else acc + o.rgb
        assert np.allclose(o.pk[fg, 1:3], 0.0) and np.allclose(o.pk[fg].sum(1), 1.0, atol=1e-12)
    mean = acc / nseed
    fg = o.np_ > 0
    # per-pixel standard error of M_K / (N_P p_K) is about sqrt((1-p)/(N p) / nseed)
    rel = np.abs(mean[fg, 0] / o.lo[fg, 0] - 1)
    bound = 6 * np.sqrt((1 - o.pk[fg, -1]) / (o.np_[fg] * o.pk[fg, -1]) / nseed) + 0.01
    assert np.mean(rel < bound) > 0.97


def test_large_n_converges_to_smooth(orc):
    """N -> infinity: M_k / N_P -> p_k and L^_o -> L_o (the discrete NDF converges
    to the smooth one, Sec. 3.2)."""
    mp = MethodParams(K=8, Wo=32)
    env = synth.env_tiny(2)
    gb = synth.gbuffer_sphere(24, 24, N0=5e8)
    o = oracle_shade(orc, gb.rows16(), env, mp, tie=ZERO_TIE)
    fg = o.np_ > 0
    M = (o.wv[:, :, None] * o.cand[:, :, 0, :]).sum(1)
    frac = M[fg] / o.np_[fg, None]
    assert np.allclose(frac, o.pk[fg], atol=1e-3)
    rel = np.abs(o.rgb[fg] - o.lo[fg]) / o.lo[fg]
    assert np.median(rel) < 1e-3 and np.max(rel) < 0.05


def test_count_saturation(orc):
    """N_P saturates at the largest FP32 value below 2^32 (uint32 counts)."""
    mp = MethodParams(K=4, Wo=16)
    env = synth.env_tiny(0)
    rows = synth.gbuffer_random(4, seed=2).rows16()
    rows[:, 3] = 1e15
    rows[:, 12:16] = [1.0, 0.0, 0.0, 1.0]
    o = oracle_shade(orc, rows, env, mp, tie=ZERO_TIE)
    assert np.all(o.np_ == np.float32(4294967040.0))
    assert np.all(o.nroot == 4294967040.0)


def test_background_and_empty_footprint(orc):
    mp = MethodParams(K=4, Wo=16)
    env = synth.env_tiny(0)
    gb = synth.gbuffer_random(8, seed=1)
    rows = gb.rows16()
    rows[0, 3] = 0.0            # background
    rows[1, 12:16] = 0.0        # zero footprint
    rows[2, 3] = 1e-30          # N_P underflows to 0
    o = oracle_shade(orc, rows, env, mp)
    assert np.all(o.rgb[:3] == 0) and np.all(o.np_[:2] == 0) and np.all(o.nroot[2] == 0)
    assert np.all(o.rgb[3:] >= 0)
