"""Pins of the E2 evaluator (Eq. probhk for an anisotropic GGX footprint by
quadrature) against brute-force enumeration of microfacets, symmetry,
convergence and the closed form at normal incidence.  CPU only."""
import math

import numpy as np
import pytest

from paper_2507_02674_gb300 import synth


@pytest.fixture(scope="module")
def env8(orc):
    env = synth.env_hdr(seed=7, W=128, H=64, fp16=False, scale_log2=0)
    return orc.env_full(env.rgba32(), 1.0, 8, 1e-4)


def _frame(theta_o, phi_t=0.3):
    n = np.array([0.0, 1.0, 0.0])
    t = np.array([math.cos(phi_t), 0.0, math.sin(phi_t)])
    b = np.cross(n, t)
    wo = math.sin(theta_o) * (0.6 * t + 0.8 * b) + math.cos(theta_o) * n
    return wo / np.linalg.norm(wo), n, t, b


def _level(H, ax, ay, S, M):
    x = np.float32(min(ax, ay)) * np.float32(4.0 / S)
    m = 0
    for k in range(M):
        if np.float32(H >> k) * x >= np.float32(math.pi):
            m = k
    return m


def _bilinear(lev, d):
    """Independent equirect bilinear look-up (wrap in phi, clamp in theta)."""
    Hm, Wm, C = lev.shape
    th = np.arccos(np.clip(d[:, 1], -1, 1))
    ph = np.mod(np.arctan2(d[:, 2], d[:, 0]), 2 * np.pi)
    x = ph / (2 * np.pi) * Wm - 0.5
    y = th / np.pi * Hm - 0.5
    x0, y0 = np.floor(x), np.floor(y)
    fx, fy = (x - x0)[:, None], (y - y0)[:, None]
    xa = np.mod(x0.astype(int), Wm)
    xb = np.mod(x0.astype(int) + 1, Wm)
    ya = np.clip(y0.astype(int), 0, Hm - 1)
    yb = np.clip(y0.astype(int) + 1, 0, Hm - 1)
    return ((1 - fy) * ((1 - fx) * lev[ya, xa] + fx * lev[ya, xb]) + fy * ((1 - fx) * lev[yb, xa] + fx * lev[yb, xb]))


@pytest.mark.parametrize("theta_o,ax,ay", [(0.2, 0.1, 0.3), (1.0, 0.25, 0.05), (1.3, 0.3, 0.3)])
def test_e2_matches_microfacet_enumeration(orc, env8, theta_o, ax, ay):
    """Brute force (Sec. 3.2): microfacet normals drawn with density D/D_H
    (anisotropic GGX, rejection from uniform hemisphere directions); each
    reflects w_o; the mean of 1[valid] w_k(w_i) is p_k, the invalid share goes
    to bin 1.  E2 with S = 64 must agree within Monte Carlo error plus the
    quadrature's O(1/S) error where the validity boundary cuts its cells."""
    wo, n, t, b = _frame(theta_o)
    S = 64
    pk, _ = orc.e2_pk(wo, n, t, ax, ay, S, env8, 8)
    m = _level(64, ax, ay, S, len(env8.mips))
    rng = np.random.default_rng(5)
    Dmax = 1 / (math.pi * ax * ay)
    hs = []
    while sum(len(h) for h in hs) < 300000:
        z = rng.uniform(0, 1, 3_000_000)
        ph = rng.uniform(0, 2 * np.pi, z.size)
        r = np.sqrt(1 - z * z)
        hx, hy = r * np.cos(ph), r * np.sin(ph)
        e = (hx / ax) ** 2 + (hy / ay) ** 2 + z * z
        D = 1 / (math.pi * ax * ay * e * e)
        keep = rng.uniform(0, Dmax, z.size) < D
        hs.append(np.stack([hx[keep], hy[keep], z[keep]], -1))
    hl = np.concatenate(hs)
    h = hl[:, 0:1] * t + hl[:, 1:2] * b + hl[:, 2:3] * n
    oh = h @ wo
    wi = 2 * oh[:, None] * h - wo
    valid = (wi @ n) > 0
    w = np.zeros((len(h), 8))
    w[valid] = _bilinear(env8.mips[m], wi[valid])[:, 3:]
    mc = w.mean(0)
    mc[0] += np.mean(~valid)
    se = np.sqrt(np.maximum(mc * (1 - mc), 1e-12) / len(h))
    assert np.all(np.abs(pk - mc) < 5 * se + 1.0 / S), (pk, mc)
    assert pk.sum() == pytest.approx(1.0, abs=1e-12)


def test_e2_swap_axes_symmetry(orc, env8):
    """Swapping alpha_x and alpha_y while turning the tangent by 90 degrees is the
    same footprint; with S divisible by 4 the quadrature points map onto each
    other, so E2 agrees to rounding."""
    wo, n, t, b = _frame(0.9)
    p1, _ = orc.e2_pk(wo, n, t, 0.07, 0.21, 32, env8, 8)
    p2, _ = orc.e2_pk(wo, n, b, 0.21, 0.07, 32, env8, 8)
    assert np.allclose(p1, p2, atol=1e-12)


def test_e2_converges_in_samples(orc, env8):
    wo, n, t, b = _frame(0.7)
    p32, _ = orc.e2_pk(wo, n, t, 0.2, 0.3, 32, env8, 8)
    p128, _ = orc.e2_pk(wo, n, t, 0.2, 0.3, 128, env8, 8)
    # a coarser pyramid level is read at S = 32; the masses still agree closely
    assert np.max(np.abs(p32 - p128)) < 0.02


def test_e2_constant_map_and_normal_incidence(orc):
    """Constant map: all radiance in level K, so p_K is the visible reflecting
    fraction; at normal incidence with alpha_x = alpha_y it is V(1, alpha) in
    closed form (theta_h < 45 degrees), up to the quadrature's O(1/S) jump error
    (at normal incidence a whole row of points changes validity at once)."""
    env = synth.env_constant(1.0, 64, 32)
    e = orc.env_full(env.rgba32(), 1.0, 4, 1e-4)
    n = np.array([0.0, 1.0, 0.0])
    t = np.array([1.0, 0.0, 0.0])
    for alpha in (0.1, 0.3):
        pk, _ = orc.e2_pk(n, n, t, alpha, alpha, 256, e, 4)
        assert pk[1] == 0 and pk[2] == 0
        b = 1 - alpha * alpha

        def F(s):
            r = math.sqrt(alpha * alpha + b * s * s)
            return 0.5 * s * r + alpha * alpha / (2 * math.sqrt(b)) * math.log(math.sqrt(b) * s + r)
        DH = 1 + alpha * alpha / math.sqrt(b) * math.log((1 + math.sqrt(b)) / alpha)
        V = 2 * (F(1.0) - F(alpha / math.sqrt(1 + alpha * alpha))) / DH
        assert pk[3] == pytest.approx(V, abs=1.0 / 256)
