"""Pins of the oracle's binomial approximations (Sec. 5, Alg. 1, Fig. gatingdiagram,
Eq. oldgated / Eq. gated, App. B, Fig. smallp) against what the paper prints and
against closed forms.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy import special, stats

GOLD = os.path.join(os.path.dirname(__file__), "golden", "gating_diagram.json")
NGRID = 1 << 15
XI = (np.arange(NGRID) + 0.5) / NGRID


def _row_ns(label):
    return {"0": [0.0], "(0,1)": [0.3, 0.8], "1": [1.0], "(1,2)": [1.25, 1.7], "2": [2.0],
            ">2": [3.0, 5.5, 20.0]}[label]


@pytest.mark.parametrize("p", [0.1, 0.5, 0.9])
def test_gating_diagram_outcome_table(orc, p):
    """Outcome frequencies of Alg. 1 over xi1 equal the probabilities printed in
    Fig. gatingdiagram, for every row of the figure."""
    rows = json.load(open(GOLD))["rows"]
    for row in rows:
        for N in _row_ns(row["N"]):
            lam = N - math.floor(N)
            env = {"p1": p, "p2": 1 - p, "lam": lam, "N": N}
            modes = [False, True] if float(N).is_integer() else [False]
            for integer_mode in modes:
                n, nb = orc.dualgated_many(N, p, XI, 0.37, integer_mode)
                for sn, snb, prob in row["outcomes"]:
                    want = eval(prob, {}, env)
                    if sn == "G":
                        got = np.mean((n >= 1) & (nb >= 1) & np.isclose(n + nb, N))
                    else:
                        a = eval(sn, {}, env)
                        b = eval(snb, {}, env)
                        got = np.mean(np.isclose(n, a) & np.isclose(nb, b))
                    assert abs(got - want) <= 2.0 / NGRID + 1e-12, (row["N"], N, p, sn, snb, got, want)


def test_gating_outcomes_exhaust_unit_interval(orc):
    """Every xi1 lands in exactly one printed outcome (the boxes tile [0,1])."""
    for N in (0.0, 0.4, 1.0, 1.5, 2.0, 7.0):
        for p in (0.05, 0.5, 0.95):
            n, nb = orc.dualgated_many(N, p, XI, 0.61, False)
            assert np.all(n >= 0) and np.all(nb >= 0)
            if N <= 2:
                assert set(np.unique(np.round(n + nb, 9))) <= {0.0, 1.0, 2.0}


@pytest.mark.parametrize("N", [3.0, 7.5, 40.0, 1000.0])
@pytest.mark.parametrize("p", [0.2, 0.5, 0.73])
def test_dual_gating_symmetry(orc, N, p):
    """Dual gating treats positive and negative samples alike (Sec. 5 'Dual Gating'):
    b(N, p; xi1, xi2) = swap(b(N, 1-p; 1-xi1, 1-xi2)) away from threshold ties."""
    xi1 = XI[::7]
    for xi2 in (0.11, 0.5 + 2 ** -20, 0.93):
        for integer_mode in ([False, True] if N.is_integer() else [False]):
            n, nb = orc.dualgated_many(N, p, xi1, xi2, integer_mode)
            m, mb = orc.dualgated_many(N, 1 - p, 1 - xi1, 1 - xi2, integer_mode)
            T, _, _ = orc.dualgated_thresholds(N, p)
            far = np.min(np.abs(xi1[:, None] - T[None, :]), axis=1) > 1e-9
            assert np.allclose(n[far], mb[far], atol=1e-9)
            assert np.allclose(nb[far], m[far], atol=1e-9)


def _clamped_normal_mean(mu, sigma, a, b):
    al, be = (a - mu) / sigma, (b - mu) / sigma
    Pa, Pb = stats.norm.cdf(al), stats.norm.cdf(be)
    return a * Pa + b * (1 - Pb) + mu * (Pb - Pa) + sigma * (stats.norm.pdf(al) - stats.norm.pdf(be))


@pytest.mark.parametrize("N,p", [(3.0, 0.3), (10.0, 0.5), (57.3, 0.12), (400.0, 0.8)])
def test_mean_equals_closed_form(orc, N, p):
    """E[n] of Alg. 1 (real counts, N > 2) = N p^N + (1 - p^N - q^N) E[clamp(mu + sigma Z, 1, N-1)],
    the expectation of the figure's three outcomes with the clamped normal in closed form."""
    g1 = (np.arange(2048) + 0.5) / 2048
    g2 = (np.arange(512) + 0.5) / 512
    tot = 0.0
    for x2 in g2:
        n, _ = orc.dualgated_many(N, p, g1, x2, False)
        tot += n.mean()
    got = tot / len(g2)
    mu, sig = 1 + (N - 2) * p, math.sqrt((N - 2) * p * (1 - p))
    want = N * p ** N + (1 - p ** N - (1 - p) ** N) * _clamped_normal_mean(mu, sig, 1.0, N - 1)
    assert abs(got - want) <= 2e-3 * max(1.0, sig), (got, want)


@pytest.mark.parametrize("N,p", [(1000.0, 0.3), (5000.0, 0.01)])
def test_large_n_matches_binomial_moments(orc, N, p):
    """For large N the dual-gated, single-gated and binomial laws agree (Sec. 6
    'Dual-Gated Gaussians'): mean N p and variance N p (1-p) within 2%."""
    g = (np.arange(256) + 0.5) / 256
    vals = []
    for x2 in g:
        n, _ = orc.dualgated_many(N, p, g, x2, False)
        vals.append(n)
    v = np.concatenate(vals)
    assert abs(v.mean() - N * p) <= 0.02 * N * p
    assert abs(v.var() - N * p * (1 - p)) <= 0.05 * N * p * (1 - p)


def test_generalised_single_gate_probability_app_b(orc):
    """App. B: the gate probability min(N p, P_{n>=1}) equals N p for N < 1 and
    1 - (1-p)^N for N > 1; Eq. gated fires with exactly that probability."""
    for N in (0.05, 0.5, 0.99, 1.0, 1.5, 4.0, 30.0):
        for p in (0.01, 0.3, 0.8):
            fired = np.mean([orc.singlegated(N, p, x, 0.5) > 0 for x in XI[::64]])
            want = N * p if N < 1 else 1 - (1 - p) ** N
            assert abs(fired - want) <= 2.0 / len(XI[::64])
            # the positive outcome is clamped to [1, max(N, 1)]
            vals = [orc.singlegated(N, p, x, y) for x in (1e-6,) for y in (0.01, 0.5, 0.99)]
            assert all(1.0 <= v <= max(N, 1.0) + 1e-12 for v in vals)


def test_old_single_gate_is_integer_and_gated(orc):
    """Eq. oldgated: floor of the gated, clamped Gaussian; zero with probability (1-p)^N."""
    N, p = 12.0, 0.2
    vals = np.array([orc.singlegated_old(N, p, x, 0.3) for x in XI[::32]])
    assert np.all(vals == np.floor(vals))
    assert abs(np.mean(vals == 0) - (1 - p) ** N) <= 2.0 / len(vals)


def test_small_p_fp32_failure_and_bias(orc):
    """Fig. smallp / Sec. 5 'Numeric Gating Issues': a naive FP32 (1-p)^N is wrong
    for p < 10^-7.525 and N > 1/p, while the biased FP32 form (1 - c p)^(N/c),
    c = max(1, eps/p), eps = 10^-3.54, stays within ~1e-4 of the truth on
    (N, p) in [1, 1e16] x [1e-16, 1]; the oracle's FP64 thresholds stay within
    the truncation bound eps/(2e) of (1-p)^N."""
    eps = orc.eps()
    assert abs(eps - 10 ** -3.54) < 1e-18
    lp = np.linspace(-16, 0, 97)
    lN = np.linspace(0, 16, 97)
    P, NN = np.meshgrid(10.0 ** lp, 10.0 ** lN, indexing="ij")
    with np.errstate(divide="ignore"):  # p = 1: log(0) = -inf gives (1 - p)^N = 0
        truth = np.exp(NN * np.log1p(-P))
    naive = np.power(np.float32(1) - P.astype(np.float32), NN.astype(np.float32)).astype(np.float64)
    bad = (P < 10 ** -7.525) & (NN > 10.0 / P)
    assert bad.any() and np.all(np.abs(naive - truth)[bad] > 0.5)
    c = np.maximum(1.0, eps / P).astype(np.float32)
    biased = np.power(np.float32(1) - c * P.astype(np.float32), NN.astype(np.float32) / c).astype(np.float64)
    assert np.max(np.abs(biased - truth)) < 2e-4
    # oracle thresholds (FP64): T[2] = 1 - P_{nbar=N} for N >= 2
    worst = 0.0
    for p in 10.0 ** lp[::4]:
        for N in 10.0 ** lN[::4]:
            if N < 2:
                continue
            T, _, _ = orc.dualgated_thresholds(N, p)
            exact = 0.0 if p >= 1.0 else math.exp(N * math.log1p(-p))
            worst = max(worst, abs((1 - T[2]) - exact))
    assert worst <= eps / (2 * math.e) * 1.05


def test_ndtri_matches_scipy(orc):
    xs = np.concatenate([(np.arange(1, 4096) / 4096), [2 ** -24, 1 - 2 ** -24, 1e-10, 0.5 + 1e-9]])
    for x in xs:
        assert abs(orc.ndtri(x) - special.ndtri(x)) <= 1e-12 * max(1.0, abs(special.ndtri(x)))


def test_uniforms_exact_in_fp32(orc):
    rng = np.random.default_rng(0)
    for h in list(rng.integers(0, 2 ** 32, 2000)) + [0, 2 ** 32 - 1, 511, 512]:
        x = orc.xi(int(h))
        assert 0.0 < x < 1.0
        assert float(np.float32(x)) == x and float(np.float32(1.0 - x)) == 1.0 - x


def test_pcg4d_statistics(orc):
    """The hash is a reading (the paper names none): check its lanes are uniform
    and mutually uncorrelated, and that an input bit flips about half the output."""
    n = 1 << 14
    out = np.array([orc.pcg4d([i & 255, i >> 8, 3 | (1 << 16), 12345]) for i in range(n)], dtype=np.uint64)
    u = ((out >> 9) * 2 + 1) / 2.0 ** 24
    for lane in range(4):
        hist, _ = np.histogram(u[:, lane], bins=32, range=(0, 1))
        chi2 = np.sum((hist - n / 32) ** 2 / (n / 32))
        assert chi2 < stats.chi2.ppf(0.9999, 31)
    c = np.corrcoef(u.T)
    assert np.max(np.abs(c - np.eye(4))) < 0.05
    flips = []
    for i in range(256):
        a = orc.pcg4d([i, 7, 9, 11])
        b = orc.pcg4d([i ^ 1, 7, 9, 11])
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert 48 <= np.mean(flips) <= 80


@pytest.mark.parametrize("K", [2, 4, 8, 16])
def test_node_uniforms_use_each_hash_word_once(orc, K):
    """Reading of the per-vertex seed (the paper stores one random seed per grid
    vertex and names no per-node stream): node 1 takes words 1, 2 of hash call 1
    beside the root's dither (word 0), siblings 2m and 2m+1 share call m + 1
    (words 0, 1 and 2, 3).  Within one tree no (call, word) serves two uniforms,
    so every draw's xi1 and xi2 are distinct, independent hash words; a K = 8
    tree needs 4 calls."""
    used = {(1, 0)}  # the root's dither
    calls = set()
    for n in range(1, K):
        call, word = orc.node_stream(n)
        assert word in (0, 1, 2) and word + 1 <= 3
        for w in (word, word + 1):
            assert (call, w) not in used, (n, call, w)
            used.add((call, w))
        calls.add(call)
        if n >= 2:
            assert call == 1 + n // 2 and word == (2 if n & 1 else 0)
    assert len(used) == 2 * (K - 1) + 1
    assert sorted(calls) == list(range(1, K // 2 + 1))  # K/2 calls per tree (4 at K = 8)
    # the helper reads those words of that call
    key, seed = (12, -7, 5 | 0x8000), 99
    for n in range(1, K):
        call, word = orc.node_stream(n)
        h = orc.pcg4d([key[0] & 0xFFFFFFFF, key[1] & 0xFFFFFFFF, key[2] | (call << 16), seed])
        xi = orc.node_uniforms(key, seed, n)
        assert xi[0] == orc.xi(int(h[word])) and xi[1] == orc.xi(int(h[word + 1]))


def test_sibling_uniforms_are_uncorrelated(orc):
    """The two siblings that share a hash call draw from disjoint words: over
    many vertices their xi1 are uniform and uncorrelated, as are each node's xi1
    and xi2."""
    n = 4096
    rng = np.random.default_rng(5)
    keys = rng.integers(-5000, 5000, size=(n, 2))
    u = np.array([[*orc.node_uniforms((int(a), int(b), 7), 3, 2), *orc.node_uniforms((int(a), int(b), 7), 3, 3)]
                  for a, b in keys])
    c = np.corrcoef(u.T)
    assert np.max(np.abs(c - np.eye(4))) < 0.06
    for j in range(4):
        hist, _ = np.histogram(u[:, j], bins=16, range=(0, 1))
        assert np.sum((hist - n / 16) ** 2 / (n / 16)) < stats.chi2.ppf(0.9999, 15)
