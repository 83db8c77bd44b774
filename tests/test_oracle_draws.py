"""Pins of the oracle's comparison draws (Sec. 5 single-gated Gaussians,
Eq. gated and Eq. oldgated; Sec. 7 Wang 2020): a tree node reproduces the
single-gated formula at the node's own hashed uniforms; counts are conserved;
the gate opens with the probability of at least one positive trial; the
older form is the floor of the newer one; Wang's estimator averages to the
smooth radiance.  CPU only."""
import numpy as np
import pytest

from paper_2507_02674_gb300 import synth
from tests._pipeline import MethodParams, oracle_env, oracle_lut


def _node_uniforms(orc, key, seed):
    h = orc.pcg4d([key[0], key[1], key[2] | (1 << 16), seed])
    return orc.xi(int(h[1])), orc.xi(int(h[2]))


@pytest.mark.parametrize("N", [0.4, 1.0, 2.5, 7.0, 40.0, 1e4])
def test_real_single_node_is_eq_gated(orc, N):
    """K = 2, real counts: the node's n equals Eq. gated at its uniforms (for
    p >= eps, where the biased and the plain no-hit probability coincide)."""
    rng = np.random.default_rng(int(N * 10))
    for i in range(300):
        p = float(rng.uniform(0.01, 0.99))
        key = (int(rng.integers(0, 2 ** 31)), int(rng.integers(0, 2 ** 31)), int(rng.integers(0, 64)))
        xi1, xi2 = _node_uniforms(orc, key, i)
        n, nb = orc.multinomial([p, 1 - p], N, key, i, integer_mode=False, draw=1)
        want = orc.singlegated(N, p, xi1, xi2)
        assert n == pytest.approx(want, rel=1e-12, abs=1e-12)
        assert nb == pytest.approx(max(N - n, 0.0), abs=1e-12)
        n_old, nb_old = orc.multinomial([p, 1 - p], N, key, i, integer_mode=False, draw=2)
        if N >= 1.0:  # Eq. oldgated as printed (its clamp [1, N] is empty below N = 1)
            assert n_old == orc.singlegated_old(N, p, xi1, xi2)
        else:  # reading: clamp to [1, max(N, 1)], then the floor
            assert n_old in (0.0, 1.0)
        assert nb_old == pytest.approx(max(N - n_old, 0.0), abs=1e-12)


@pytest.mark.parametrize("draw", [1, 2])
def test_integer_single_counts_conserved_and_gate_rate(orc, draw):
    """Integer counts: every tree conserves its trials; the fraction of nodes
    with n >= 1 matches 1 - (1 - p)^N (99.9% binomial confidence)."""
    rng = np.random.default_rng(draw)
    for K in (2, 4, 8):
        for _ in range(50):
            p = rng.dirichlet(np.ones(K))
            N = int(rng.integers(1, 1000))
            c = orc.multinomial(p, N, (int(rng.integers(2 ** 31)), 3, 1), int(rng.integers(2 ** 31)), True, draw)
            assert c.sum() == N and np.all(c >= 0) and np.all(c == np.round(c))
    for N, p in ((1, 0.3), (3, 0.2), (20, 0.01), (500, 0.002)):
        trials = 4000
        hits = sum(orc.multinomial([p, 1 - p], N, (s, 7, 2), 11, True, draw)[0] >= 1 for s in range(trials))
        want = 1 - (1 - p) ** N
        tol = 3.3 * np.sqrt(want * (1 - want) / trials) + 1e-9
        assert abs(hits / trials - want) <= tol, (N, p, hits / trials, want)


def test_old_form_is_floor_of_the_rounded_form(orc):
    """Integer counts with the gate open: Eq. oldgated floors the Gaussian the
    newer form rounds, so n_old <= n_new <= n_old + 1."""
    rng = np.random.default_rng(3)
    for s in range(2000):
        N = int(rng.integers(2, 5000))
        p = float(rng.uniform(0.05, 0.95))
        a = orc.multinomial([p, 1 - p], N, (s, 1, 0), 5, True, 1)[0]
        b = orc.multinomial([p, 1 - p], N, (s, 1, 0), 5, True, 2)[0]
        assert (a == 0) == (b == 0)
        assert b <= a <= b + 1


def test_wang2020_estimator_converges_to_smooth_radiance(orc):
    """Sec. 7 Wang 2020 on the same grid: counts are single-gated with the map-
    independent gamma, bins (glints, rest) conserve N, and L_o M / (N_P gamma)
    averages to L_o over seeds."""
    mp = MethodParams(K=4, Wo=64)
    env = synth.env_tiny(0)
    e, pref = oracle_env(orc, env, mp)
    lut = oracle_lut(orc, mp)
    gb = synth.gbuffer_random(60, seed=8, n_lo=1e3, n_hi=1e4)
    rows = gb.rows16()
    s = np.sqrt(2e4 / rows[:, 3])  # footprints holding N_P = 2e4 microfacets
    rows[:, 12:16] = np.stack([s, 0 * s, 0 * s, s], 1)
    gamma = 0.05
    acc = None
    S = 200
    for seed in range(S):
        o = orc.shade(rows, pref, mp.s_min, mp.s_max, lut, e.levels, seed, True, tie=[0, 0, 0, 0, 0],
                      max_cand=1, draw=3, gamma=gamma)
        c = o.cand[:, :, 0, :]
        fg = o.np_ > 0
        assert np.all(c[fg][:, :, 2:] == 0)
        np.testing.assert_array_equal(c[fg][:, :, 0] + c[fg][:, :, 1], o.nroot[fg])
        acc = o.rgb if acc is None else acc + o.rgb
    fg = o.np_ > 0
    mean = acc[fg] / S
    # relative standard error of the mean of S estimates ~ 1 / sqrt(S N_P gamma) = 0.5%
    rel = np.abs(mean - o.lo[fg]).sum(1) / o.lo[fg].sum(1)
    assert np.median(rel) < 0.01 and np.max(rel) < 0.03, (np.median(rel), np.max(rel))
