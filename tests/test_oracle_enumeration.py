"""Counts of the glint estimator on tiny footprints against explicit
microfacets (Sec. 3.2 "Discrete Normal Distribution", Eq. discrete_ndf and
Eq. probh_def; Sec. 5 Alg. 1 and the hierarchical multinomial).

The microfacet model of Sec. 3.2 is enumerated here with code of its own: a
footprint holds N_P microfacets whose normals are drawn i.i.d. with density
D(h) / D_H over the hemisphere (the unprojected microfacet area); each one
mirrors w_o about its normal, a reflection below the surface or a normal
facing away from w_o counts for the dummy component (bin 1), and a valid
reflection w_i joins component k with probability w_k(w_i), the fuzzy weight
of Sec. 4 read bilinearly from the map.  Three claims are checked.

1. The frequencies of the components over many microfacets equal the
   probabilities p_k that E2 integrates (Eq. probh_def without the n = v = r
   approximation), to the statistical error of the enumeration.
2. The oracle's per-vertex counts follow the exact distribution of the
   balanced tree of dual-gated draws: a dynamic program written here from
   Alg. 1's outcome probabilities -- n = N with probability p^N, n = 0 with
   the biased (1 - c p)^(N/c) where it does not overlap the first gate, and
   otherwise the Gaussian N(1 + (N-2) p, (N-2) p q) rounded half up and
   clamped to [1, N-1] -- propagates the pmf of the trials down the tree.  The
   oracle's means and variances over thousands of hashed vertices match it.
3. Against the enumerated microfacets (the model Alg. 1 approximates) the
   counts' means agree within one count and their variances
   within a factor of two (Alg. 1 centres its Gaussian on 1 + (N-2) p instead
   of N p; Sec. 5 "Dual Gating").  Grid interpolation of the six samples
   divides the estimator's variance by sum_i w_i^2 (Sec. 3.3).
"""
import math

import numpy as np
import pytest
from scipy.special import ndtr

from paper_2507_02674_gb300 import synth
from tests._pipeline import MethodParams, oracle_env, oracle_shade

K = 4
ALPHA = 0.15
EPS = 10.0 ** -3.54


def _frame():
    nrm = np.array([0.2, 0.9, 0.1])
    nrm /= np.linalg.norm(nrm)
    tg = np.cross(nrm, [0.0, 0.0, 1.0])
    tg /= np.linalg.norm(tg)
    wo = np.array([0.5, 0.7, 0.4])
    wo /= np.linalg.norm(wo)
    return wo, nrm, tg, np.cross(nrm, tg)


def _bilinear(w0, d):
    H, W = w0.shape[:2]
    th = np.arccos(np.clip(d[:, 1], -1.0, 1.0))
    ph = np.arctan2(d[:, 2], d[:, 0]) % (2.0 * np.pi)
    x, y = ph / (2.0 * np.pi) * W - 0.5, th / np.pi * H - 0.5
    x0, y0 = np.floor(x), np.floor(y)
    fx, fy = x - x0, y - y0
    xa = x0.astype(int) % W
    xb = (xa + 1) % W
    ya, yb = np.clip(y0.astype(int), 0, H - 1), np.clip(y0.astype(int) + 1, 0, H - 1)
    return (((1 - fy) * (1 - fx))[:, None] * w0[ya, xa] + ((1 - fy) * fx)[:, None] * w0[ya, xb]
            + (fy * (1 - fx))[:, None] * w0[yb, xa] + (fy * fx)[:, None] * w0[yb, xb])


def enumerate_microfacets(w0, N, trials, rng):
    """(trials, K) component counts of N explicit microfacets per trial."""
    wo, nrm, tg, bt = _frame()
    # theta of the normal with density D(theta) sin(theta) (area measure):
    # numerical CDF on a fine grid, inverted by interpolation
    th = np.linspace(0.0, np.pi / 2, 400001)
    c = np.cos(th)
    t2 = np.tan(np.minimum(th, np.pi / 2 - 1e-9)) ** 2
    dens = np.where(c > 1e-9, ALPHA ** 2 / (np.pi * c ** 4 * (ALPHA ** 2 + t2) ** 2), 0.0) * np.sin(th)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(th))])
    cdf /= cdf[-1]
    n = N * trials
    t = np.interp(rng.random(n), cdf, th)
    ph = 2.0 * np.pi * rng.random(n)
    h = (np.sin(t) * np.cos(ph))[:, None] * tg + (np.sin(t) * np.sin(ph))[:, None] * bt + np.cos(t)[:, None] * nrm
    oh = h @ wo
    wi = 2.0 * oh[:, None] * h - wo
    valid = (oh > 0.0) & (wi @ nrm > 0.0)
    k = (rng.random(n)[:, None] >= np.cumsum(_bilinear(w0, wi), 1)).sum(1)
    k = np.where(valid, np.minimum(k, K - 1), 0)
    counts = np.zeros((trials, K))
    np.add.at(counts, (np.repeat(np.arange(trials), N), k), 1.0)
    return counts


def node_pmf(Nmax, p):
    """T[N, n]: probability that a dual-gated node with N trials and node
    probability p gives n to its left child (integer counts, Alg. 1)."""
    T = np.zeros((Nmax + 1, Nmax + 1))
    T[0, 0] = 1.0
    if Nmax >= 1:
        T[1, 1], T[1, 0] = p, 1.0 - p
    q = 1.0 - p
    cb = max(1.0, EPS / p) if p > 0 else math.inf
    for N in range(2, Nmax + 1):
        t_all = p ** N
        t_none = 1.0 if p == 0 else max(0.0, 1.0 - cb * p) ** (N / cb)
        P0 = 1.0 - max(t_all, 1.0 - t_none)
        PG = max(0.0, 1.0 - t_none - t_all)
        T[N, N] += t_all
        T[N, 0] += P0
        mu, var = 1.0 + (N - 2) * p, (N - 2) * p * q
        g = np.arange(1, N)
        if var <= 0.0:
            G = min(max(math.floor(mu + 0.5), 1), N - 1)
            T[N, G] += PG
            continue
        sd = math.sqrt(var)
        upper = np.where(g == N - 1, 1.0, ndtr((g + 0.5 - mu) / sd))
        lower = np.where(g == 1, 0.0, ndtr((g - 0.5 - mu) / sd))
        T[N, 1:N] += PG * (upper - lower)
    return T


def tree_leaf_moments(pk, N):
    """Mean and variance of each bin's count for one vertex with N trials."""
    Kb = len(pk)
    P = np.zeros(2 * Kb)
    P[Kb:] = pk
    for n in range(Kb - 1, 0, -1):
        P[n] = P[2 * n] + P[2 * n + 1]
    pmf = {1: np.eye(N + 1)[N]}
    for n in range(1, Kb):
        p = P[2 * n] / P[n] if P[n] > 0 else 0.0
        T = node_pmf(N, p)
        left = pmf[n] @ T
        right = np.zeros(N + 1)
        for M in range(N + 1):
            right[:M + 1] += pmf[n][M] * T[M, M::-1][:M + 1]
        pmf[2 * n], pmf[2 * n + 1] = left, right
    j = np.arange(N + 1)
    mean = np.array([pmf[Kb + k] @ j for k in range(Kb)])
    var = np.array([pmf[Kb + k] @ (j * j) for k in range(Kb)]) - mean ** 2
    return mean, var


@pytest.fixture(scope="module")
def setup(orc):
    mp = MethodParams(K=K, Wo=64)
    env = synth.env_tiny(0)
    e, pref = oracle_env(orc, env, mp)
    wo, nrm, tg, _ = _frame()
    pk, _ = orc.e2_pk(wo, nrm, tg, ALPHA, ALPHA, 256, e, K)
    return mp, env, e, pref, pk


def test_e2_probabilities_equal_microfacet_frequencies(setup):
    mp, env, e, pref, pk = setup
    rng = np.random.default_rng(0)
    counts = enumerate_microfacets(e.ch0[..., 3:], 300, 10000, rng)  # 3e6 microfacets
    f = counts.sum(0) / counts.sum()
    se = np.sqrt(pk * (1.0 - pk) / counts.sum())
    assert np.all(np.abs(f - pk) < 5.0 * se + 1e-5), (f, pk)


def _oracle_counts(orc, setup, N, copies):
    mp, env, e, pref, pk = setup
    wo, nrm, tg, _ = _frame()
    rows = np.zeros((copies, 16), np.float32)
    rows[:, 0:3], rows[:, 3] = wo, N
    rows[:, 4:7], rows[:, 7] = nrm, 0.9
    rows[:, 8:10] = np.random.default_rng(N).uniform(-2e3, 2e3, (copies, 2))  # independent lattice vertices
    rows[:, 10] = rows[:, 11] = ALPHA
    rows[:, 12] = rows[:, 15] = 1.0  # |P| = 1: N_P = N exactly, grid level 0
    o = oracle_shade(orc, rows, env, mp, env_pref=(e, pref), tie=(0.0, 0.0, 0.0, 0.0, 0.0), max_cand=2,
                     evaluator=2, pk_in=np.tile(pk, (copies, 1)))
    assert np.all(o.nroot == N)
    return o


@pytest.mark.parametrize("N", [3, 30, 300])
def test_counts_follow_the_exact_tree_distribution(orc, setup, N):
    pk = setup[4]
    o = _oracle_counts(orc, setup, N, 2000)
    cnt = o.cand[:, :, 0, :].reshape(-1, K)  # 12000 vertices
    assert np.all(cnt.sum(1) == N)
    mean, var = tree_leaf_moments(pk, N)
    n = len(cnt)
    assert np.all(np.abs(cnt.mean(0) - mean) < 5.0 * np.sqrt(var / n) + 1e-9), (cnt.mean(0), mean)
    # variance of a sample variance ~ 2 var^2 / n for near-normal counts, more
    # for the skewed small ones: 25% relative plus an absolute floor
    assert np.all(np.abs(cnt.var(0) - var) < 0.25 * var + 5.0 / n), (cnt.var(0), var)


@pytest.mark.parametrize("N", [3, 30, 300])
def test_counts_against_enumerated_microfacets(orc, setup, N):
    mp, env, e, pref, pk = setup
    o = _oracle_counts(orc, setup, N, 2000)
    cnt = o.cand[:, :, 0, :].reshape(-1, K)
    en = enumerate_microfacets(e.ch0[..., 3:], N, 12000, np.random.default_rng(N + 1))
    # means: within one count (Alg. 1's shifted Gaussian) plus
    # the statistical error of both samples
    se = np.sqrt(cnt.var(0) / len(cnt) + en.var(0) / len(en))
    assert np.all(np.abs(cnt.mean(0) - en.mean(0)) < 1.0 + 5.0 * se), (cnt.mean(0), en.mean(0))
    # variances within a factor of two where a bin holds a count on average
    big = en.var(0) > 0.05
    ratio = cnt.var(0)[big] / en.var(0)[big]
    assert np.all((ratio > 0.5) & (ratio < 2.0)), ratio
    # the estimator: six independent vertices weighted by w_i (sum 1)
    M = (o.wv[:, :, None] * o.cand[:, :, 0, :]).sum(1)
    sw2 = (o.wv ** 2).sum(1)
    assert np.allclose(o.wv.sum(1), 1.0)
    want = (sw2[:, None] * cnt.reshape(-1, 6, K).var(0).mean(0)[None, :]).mean(0)
    assert np.all(np.abs(M.var(0) - want) < 0.25 * want + 1e-3), (M.var(0), want)
