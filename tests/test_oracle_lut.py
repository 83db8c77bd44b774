"""Pins of the oracle's microfacet tables (Sec. 3.2 total microfacet area D_H,
Sec. 4 Eq. rtiblndf visible reflecting area E_D, Sec. 3.4 split-sum albedo)
against closed forms, an independent quadrature and brute-force enumeration
of microfacets.  CPU only."""
import math

import numpy as np
import pytest


def _total_area_closed(alpha):
    """D_H(alpha) = int D(h) dh for isotropic GGX, integrated by hand:
    1 + a^2 / sqrt(1 - a^2) * ln((1 + sqrt(1 - a^2)) / a)."""
    if alpha == 1.0:
        return 2.0
    b = math.sqrt(1.0 - alpha * alpha)
    return 1.0 + alpha * alpha / b * math.log((1.0 + b) / alpha)


def _antiderivative(s, a):
    b = 1.0 - a * a
    r = math.sqrt(a * a + b * s * s)
    if b == 0:
        return 0.5 * s * r + 0.0
    return 0.5 * s * r + a * a / (2 * math.sqrt(b)) * math.log(math.sqrt(b) * s + r)


@pytest.mark.parametrize("alpha", [0.02, 0.1, 0.15, 0.3, 0.5, 0.9, 1.0])
def test_total_area_closed_form(orc, alpha):
    """Sec. 3.2: D_H >= 1 with equality only in the limit of a flat surface;
    D_H(1) = 2 (D = 1/pi over the hemisphere)."""
    got = orc.total_area(alpha, 256)
    assert got == pytest.approx(_total_area_closed(alpha), rel=2e-6)
    assert got >= 1.0


@pytest.mark.parametrize("alpha", [0.02, 0.2, 0.7])
def test_projected_area_is_one(orc, alpha):
    """The projected microfacet area integrates to exactly 1 (Sec. 3.2)."""
    assert orc.projected_area(alpha, 128) == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("alpha", [0.02, 0.1, 0.3, 0.6])
def test_visible_fraction_normal_incidence(orc, alpha):
    """At w_o = n a microfacet reflects above the horizon iff theta_h < 45 deg,
    so E_D = 2 [F(1) - F(a / sqrt(1 + a^2))] with F the antiderivative of
    sqrt(a^2 + (1 - a^2) s^2); V = E_D / D_H."""
    s_star = alpha / math.sqrt(1 + alpha * alpha)
    ED = 2.0 * (_antiderivative(1.0, alpha) - _antiderivative(s_star, alpha))
    want = ED / _total_area_closed(alpha)
    Q = 128
    V, U, A, B = orc.lut_point(1.0, alpha, Q)
    # Q*Q-point midpoint rule in s across the indicator's jump at s*: at most
    # half a cell of density, plus the rule's smooth-part error
    jump = 2.0 * math.sqrt(alpha ** 2 + (1 - alpha ** 2) * s_star ** 2) / (2 * Q * Q) / _total_area_closed(alpha)
    assert V == pytest.approx(want, abs=jump + 1e-8)
    assert V + U == pytest.approx(1.0, abs=1e-11)


def test_table_limits(orc):
    """alpha -> 0 at normal incidence: every microfacet reflects (V -> 1) and the
    split-sum albedo with F0 = 1 tends to 1."""
    V, U, A, B = orc.lut_point(0.999, 1e-3, 256)
    assert V > 0.9999 and A + B == pytest.approx(1.0, abs=2e-3)
    t = orc.lut(16, 64)
    assert np.all((t[..., 0] >= 0) & (t[..., 0] <= 1))
    assert np.allclose(t[..., 0] + t[..., 1], 1.0, atol=1e-11)


def _ggx(cos_h, a):
    c2 = cos_h * cos_h
    d = c2 * (a * a - 1) + 1
    return np.where(cos_h > 0, a * a / (np.pi * d * d), 0.0)


def _lam(mu, a):
    t2 = (1 - mu * mu) / (mu * mu)
    return 0.5 * (-1 + np.sqrt(1 + a * a * t2))


@pytest.mark.parametrize("alpha", [0.25, 0.5])
@pytest.mark.parametrize("mu", [0.3, 0.7, 0.95])
def test_albedo_independent_quadrature(orc, alpha, mu):
    """E_rho with F = 1 (= A + B) against a plain quadrature over incoming
    directions of rho~ = G2 D / (4 n.v) (Sec. 3.1), in (theta_i, phi_i)."""
    nt, nph = 600, 1200
    th = (np.arange(nt) + 0.5) * (np.pi / 2) / nt
    ph = (np.arange(nph) + 0.5) * 2 * np.pi / nph
    T, P = np.meshgrid(th, ph, indexing="ij")
    wi = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1)
    wo = np.array([math.sqrt(1 - mu * mu), 0.0, mu])
    h = wi + wo
    h /= np.linalg.norm(h, axis=-1, keepdims=True)
    G2 = 1.0 / (1.0 + _lam(mu, alpha) + _lam(wi[..., 2], alpha))
    f = G2 * _ggx(h[..., 2], alpha) / (4 * mu)
    dA = np.sin(T) * (np.pi / 2 / nt) * (2 * np.pi / nph)
    want = np.sum(f * dA)
    V, U, A, B = orc.lut_point(mu, alpha, 256)
    assert A + B == pytest.approx(want, rel=2e-3)


@pytest.mark.parametrize("alpha,mu", [(0.2, 0.9), (0.5, 0.5), (0.5, 0.15)])
def test_visible_fraction_by_microfacet_enumeration(orc, alpha, mu):
    """Brute force (Sec. 3.2): draw microfacet normals with density D/D_H by
    rejection from uniform hemisphere directions, reflect w_o, and count the
    ones whose reflection leaves the surface: the fraction is V = E_D / D_H."""
    rng = np.random.default_rng(11)
    wo = np.array([math.sqrt(1 - mu * mu), 0.0, mu])
    Dmax = 1.0 / (math.pi * alpha * alpha)
    acc = []
    while sum(len(a) for a in acc) < 200000:
        z = rng.uniform(0, 1, 2_000_000)
        phi = rng.uniform(0, 2 * np.pi, z.size)
        r = np.sqrt(1 - z * z)
        keep = rng.uniform(0, Dmax, z.size) < _ggx(z, alpha)
        acc.append(np.stack([r * np.cos(phi), r * np.sin(phi), z], -1)[keep])
    h = np.concatenate(acc)
    vh = h @ wo
    wi_z = 2 * vh * h[:, 2] - mu
    frac = np.mean((vh > 0) & (wi_z > 0))
    V = orc.lut_point(mu, alpha, 512)[0]
    se = math.sqrt(frac * (1 - frac) / len(h))
    assert abs(V - frac) < 5 * se + 1e-3
