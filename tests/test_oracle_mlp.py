"""Pins of the FP64 reference of the p_k surrogate (oracle/mlp.py and the
oracle's or_mlp_features) to facts outside themselves: PyTorch's bfloat16
conversion, central finite differences of the loss, closed forms of the
squared error at uniform and prior outputs and of the first Adam step, the
derivative of the mirror direction, and the tap features under constant and
two-tone maps.  CPU only."""
import numpy as np
import pytest
import torch

from oracle import mlp
from paper_2507_02674_gb300 import synth
from tests._pipeline import MethodParams, oracle_env, oracle_lut


def _data(n=24, K=8, seed=5, normalised=True):
    """Inputs shaped like the surrogate's (probabilities, then three scalars),
    log-priors and target distributions."""
    rng = np.random.default_rng(seed)
    X = np.zeros((n, 64))
    X[:, :6 * K] = rng.uniform(0, 1, size=(n, 6 * K))
    X[:, 6 * K:6 * K + 3] = rng.uniform(0.1, 1, size=(n, 3))
    lp = np.log(np.maximum(synth.distributions(n, K, seed=seed + 2).astype(np.float64), 1e-6))
    Y = synth.distributions(n, K, seed=seed + 1).astype(np.float64)
    Y /= Y.sum(axis=1, keepdims=True)
    if not normalised:
        Y = Y * rng.uniform(0.5, 2.0, size=(n, 1))
    return X, lp, Y


def test_bf16_matches_torch_conversion():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.uniform(-30, 30, size=5000),
                        # exact ties between two bfloat16 values
                        (1.0 + (2 * np.arange(1, 200) + 1) * 2.0 ** -8) * 2.0 ** rng.integers(-20, 20, size=199)])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)


def test_bf16_ties_to_even_and_rounding_delta():
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert mlp.bf16(-(1.0 + 2.0 ** -7)) == -(1.0 + 2.0 ** -7)
    # no boundary within reach: identical roundings; a boundary: one spacing
    assert mlp.rounding_delta(1.0 + 2.0 ** -10, 2.0 ** -12) == 0.0
    assert mlp.rounding_delta(1.0 + 2.0 ** -8, 2.0 ** -20) == pytest.approx(2.0 ** -7 + 2.0 ** -20)


@pytest.mark.parametrize("K", [2, 4, 8])
@pytest.mark.parametrize("normalised", [True, False])
def test_gradient_matches_finite_differences(K, normalised):
    X, lp, Y = _data(16, K, seed=7 + K, normalised=normalised)
    prm = synth.mlp_params(seed=3 + K, K=K).astype(np.float64)
    g, mag, L = mlp.gradient(prm, X, Y, K, lp, exact=True)
    assert L == pytest.approx(mlp.loss(prm, X, Y, K, lp, exact=True), rel=1e-14)
    rng = np.random.default_rng(K)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SIZES])
    idx = []
    for li in range(6):
        lo, hi = offs[li], offs[li + 1]
        cand = np.arange(lo, hi)
        if li == 0:
            cand = cand[(cand - lo) // 64 < 6 * K + 3]  # rows of used inputs
        if li in (4, 5):
            cand = cand[((cand - lo) % 16 if li == 4 else (cand - lo)) < K]
        idx.extend(rng.choice(cand, size=min(12, cand.size), replace=False))
    h = 1e-6
    for i in idx:
        pp, pm = prm.copy(), prm.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss(pp, X, Y, K, lp, exact=True) - mlp.loss(pm, X, Y, K, lp, exact=True)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])
    # unused output columns get no gradient
    W3 = g[offs[4]:offs[5]].reshape(64, 16)
    assert np.all(W3[:, K:] == 0) and np.all(g[offs[5] + K:] == 0)
    assert np.all(mag >= np.abs(g) - 1e-15)


def test_zero_output_layer_gives_the_prior():
    """With W3 = 0 and b3 = 0 the logits are the log-prior: p = normalised
    prior; without a prior p is uniform and the squared error of a target
    distribution y is sum_k y_k^2 - 1/K.  Targets equal to the prior are the
    loss's minimum: loss 0 and a zero gradient everywhere."""
    K = 8
    X, lp, Y = _data(32, K)
    d = mlp.unpack(synth.mlp_params(K=K).astype(np.float64))
    d["W3"][:] = 0.0
    d["b3"][:] = 0.0
    prm = mlp.pack(d)
    Yn = Y / Y.sum(1, keepdims=True)
    assert mlp.loss(prm, X, Yn, K) == pytest.approx(np.mean(np.sum(Yn ** 2, 1)) - 1.0 / K, rel=1e-12)
    prior = np.exp(lp) / np.exp(lp).sum(1, keepdims=True)
    np.testing.assert_allclose(mlp.forward(prm, X, K, lp, exact=True)["p"], prior, rtol=1e-12)
    g, _, L = mlp.gradient(prm, X, prior, K, lp, exact=True)
    assert L == pytest.approx(0.0, abs=1e-28)
    assert np.abs(g).max() < 1e-15
    # away from the minimum the output bias moves p towards y: -g . (y - p) > 0
    g, _, _ = mlp.gradient(prm, X, Yn, K, lp, exact=True)
    assert -np.dot(g[-16:][:K], np.mean(Yn - prior, axis=0)) > 0


def test_first_adam_step_is_lr_sign():
    rng = np.random.default_rng(2)
    w = rng.normal(size=mlp.N_PARAMS)
    g = rng.normal(size=mlp.N_PARAMS) * 1e-2
    z = np.zeros(mlp.N_PARAMS)
    w1, m1, v1 = mlp.adam(w, g, z, z, 1, 1e-3)
    np.testing.assert_allclose(w1 - w, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)


def test_mirror_mode_stays_near_exact():
    """BF16 rounding (relative 2^-9 per value, through three layers) is a small
    perturbation of the exact gradient; a misplaced rounding of a whole
    operand (e.g. of the logits) or a wrong mask would not be."""
    K = 8
    X, lp, Y = _data(64, K)
    prm = synth.mlp_params(K=K)
    g, _, L = mlp.gradient(prm, X, Y, K, lp)
    ge, _, Le = mlp.gradient(prm, X, Y, K, lp, exact=True)
    assert np.linalg.norm(g - ge) < 0.1 * np.linalg.norm(ge)
    assert abs(L - Le) < 1e-2 * Le


# ------------------------------------------------------------------ inputs
def _frame(orc, env, K):
    mp = MethodParams(K=K, Wo=64)
    e, pref = oracle_env(orc, env, mp)
    return mp, e, pref, oracle_lut(orc, mp)


def _pixel_rows(wo, n, t, ax, ay, N0=1e4):
    rows = np.zeros((len(wo), 16), np.float32)
    rows[:, 0:3], rows[:, 3] = wo, N0
    rows[:, 4:7], rows[:, 7] = n, 0.04
    rows[:, 10], rows[:, 11] = ax, ay
    rows[:, 12:16] = [1e-3, 0, 0, 1e-3]
    tan = np.zeros((len(wo), 4), np.float32)
    tan[:, :3] = t
    return rows, tan


def test_tap_directions_follow_the_mirror_derivative(orc):
    """For a tiny slope the taps are the mirror directions of the tilted
    normals n -+ a t and n -+ a b (to first order), at grazing views too."""
    mp, e, pref, lut = _frame(orc, synth.env_constant(), 2)
    rng = np.random.default_rng(1)
    m = 50
    n = rng.normal(size=(m, 3)); n /= np.linalg.norm(n, axis=1, keepdims=True)
    wo = rng.normal(size=(m, 3)); wo /= np.linalg.norm(wo, axis=1, keepdims=True)
    wo = np.where((np.sum(wo * n, 1) < 0)[:, None], -wo, wo)
    t = rng.normal(size=(m, 3)); t -= np.sum(t * n, 1)[:, None] * n; t /= np.linalg.norm(t, axis=1, keepdims=True)
    a = 1e-4
    rows, tan = _pixel_rows(wo, n, t, a, a)
    _, _, dirs = orc.mlp_features(rows, tan, pref, mp.s_min, mp.s_max, lut, 2, want_dirs=True)
    w64, n64 = rows[:, 0:3].astype(np.float64), rows[:, 4:7].astype(np.float64)
    t64 = tan[:, :3].astype(np.float64)
    t64 -= np.sum(t64 * n64, 1)[:, None] * n64
    t64 /= np.linalg.norm(t64, axis=1, keepdims=True)
    b64 = np.cross(n64, t64)

    def mirror(h):
        h = h / np.linalg.norm(h, axis=1, keepdims=True)
        return 2 * np.sum(w64 * h, 1)[:, None] * h - w64

    want = [mirror(n64), mirror(n64 - a * t64), mirror(n64 + a * t64), mirror(n64 - a * b64), mirror(n64 + a * b64)]
    for tap in range(5):
        np.testing.assert_allclose(dirs[:, tap], want[tap], atol=5e-7)


def test_taps_under_constant_and_two_tone_maps(orc):
    """A constant map puts every tap's weight in the brightest component; a map
    bright above the horizon and dark below tells the taps that lean up from
    those that lean down (signs of J_t and J_b)."""
    K = 2
    mp, e, pref, lut = _frame(orc, synth.env_constant(3.0), K)
    rows, tan = _pixel_rows(np.array([[0, 0, 1.0]]), np.array([[0, 0, 1.0]]), np.array([[0, 1.0, 0]]), 0.3, 0.03)
    x, lp = orc.mlp_features(rows, tan, pref, mp.s_min, mp.s_max, lut, K)
    np.testing.assert_allclose(x[0, K:6 * K].reshape(5, K), [[0, 1]] * 5, atol=1e-12)
    np.testing.assert_allclose(x[0, 6 * K:6 * K + 3], [1.0, np.sqrt(np.float32(0.3)), np.sqrt(np.float32(0.03))],
                               rtol=1e-7)
    assert np.all(x[0, 6 * K + 3:] == 0)
    np.testing.assert_allclose(lp[0], np.log(np.maximum(x[0, :K], 1e-6)))

    env = synth.env_constant(1.0, W=128, H=64)
    env.texels[:32, :, :3] = 1000.0  # upper hemisphere (y > 0) bright
    mp, e, pref, lut = _frame(orc, env, K)
    # view along +z on a surface facing +z: w_r = +z (horizontal); t = +y (up)
    rows, tan = _pixel_rows(np.array([[0, 0, 1.0]] * 2), np.array([[0, 0, 1.0]] * 2),
                            np.array([[0, 1.0, 0], [1.0, 0, 0]]), np.array([0.4, 0.02]), np.array([0.02, 0.4]))
    x, _ = orc.mlp_features(rows, tan, pref, mp.s_min, mp.s_max, lut, K)
    bright = x[:, K + 1:6 * K:K]  # W_2 of taps 0..4
    # pixel 0: J_t = -2 t points down, so tap 1 (w_r + a_x J_t) is dark, tap 2 bright
    assert bright[0, 1] < 0.05 and bright[0, 2] > 0.95
    # pixel 1: t = +x, b = n x t = +y, J_b = -2 b: tap 3 dark, tap 4 bright
    assert bright[1, 3] < 0.05 and bright[1, 4] > 0.95


def test_tangent_flip_swaps_taps_and_e1_part_matches_shading(orc):
    K = 4
    env = synth.env_hdr(seed=3, W=128, H=64)
    mp, e, pref, lut = _frame(orc, env, K)
    gb = synth.gbuffer_random(200, seed=4)
    rows, tan = gb.rows16(), gb.tangents()
    x, lp = orc.mlp_features(rows, tan, pref, mp.s_min, mp.s_max, lut, K)
    tan2 = tan.copy()
    tan2[:, :3] *= -1
    x2, _ = orc.mlp_features(rows, tan2, pref, mp.s_min, mp.s_max, lut, K)
    taps, taps2 = x[:, K:6 * K].reshape(-1, 5, K), x2[:, K:6 * K].reshape(-1, 5, K)
    np.testing.assert_allclose(taps2[:, [0, 2, 1, 4, 3]], taps, atol=1e-12)
    o = orc.shade(rows, pref, mp.s_min, mp.s_max, lut, e.levels, 0)
    fg = rows[:, 3] > 0
    np.testing.assert_allclose(x[fg, :K], o.pk[fg], rtol=1e-13, atol=1e-15)
    assert np.all(x[~fg] == 0)
