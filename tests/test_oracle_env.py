"""Pins of the oracle's environment decomposition (Sec. 4 'Discrete Radiance
Levels', 'Fuzzy Indicator Functions', Eq. wkdefpractice), its pyramid and its
filter (Sec. 3.4 Eq. rtibl, Sec. 4 Eq. rtiblndf).  CPU only."""
import math

import numpy as np
import pytest

from paper_2507_02674_gb300 import synth


def _lum(rgba, scale=1.0):
    x = rgba.astype(np.float64) * scale
    return np.maximum(0.2126 * x[..., 0] + 0.7152 * x[..., 1] + 0.0722 * x[..., 2], 0.0)


@pytest.mark.parametrize("K", [2, 4, 8, 16])
def test_levels_closed_form(orc, K):
    """L_1 = 0, L_K = max Y, L_2..L_K geometric between max(min Y, ell) and max Y."""
    env = synth.env_tiny(3)
    ell = 1e-4
    L, lohi, ch0 = orc.env_decompose(env.rgba32(), 1.0, K, ell)
    Y = _lum(env.texels)
    lo, hi = max(Y.min(), ell), Y.max()
    assert L[0] == 0.0
    assert lohi[0] == pytest.approx(lo, rel=1e-15) and lohi[1] == pytest.approx(hi, rel=1e-15)
    assert L[-1] == pytest.approx(hi, rel=1e-12)
    if K > 2:
        r = L[2:] / L[1:-1]
        assert np.allclose(r, (hi / lo) ** (1.0 / (K - 1)), rtol=1e-12)
    assert L[1] == pytest.approx(lo ** ((K - 2) / (K - 1)) * hi ** (1 / (K - 1)), rel=1e-12)


@pytest.mark.parametrize("K", [4, 8])
def test_weights_partition_and_reconstruct(orc, K):
    """Sum_k w_k = 1 and sum_k w_k L_k = Y for every texel below L_K; texels at or
    above L_K carry w_K = 1 (Sec. 4: w_k is the lerp factor between the two
    bracketing levels); at most two non-zero weights, adjacent."""
    env = synth.env_hdr(seed=5, W=128, H=64)
    L, lohi, ch0 = orc.env_decompose(env.rgba32(), env.scale, K, 1e-4)
    w = ch0[..., 3:]
    Y = _lum(env.rgba32(), env.scale)
    assert np.allclose(w.sum(-1), 1.0, atol=1e-14)
    assert np.all(w >= -1e-15)
    rec = (w * L).sum(-1)
    below = Y < L[-1]
    assert np.allclose(rec[below], Y[below], rtol=1e-12, atol=1e-300)
    assert np.all(w[~below][..., -1] == 1.0)
    nz = w > 0
    assert np.all(nz.sum(-1) <= 2)
    two = nz.sum(-1) == 2
    idx = np.argmax(nz, axis=-1)
    assert np.all(nz[two][np.arange(two.sum()), idx[two] + 1])
    assert np.allclose(ch0[..., :3], env.rgba32()[..., :3] * env.scale)


def test_weights_hand_case(orc):
    """Four texels worked by hand: Y = 0, 2, 8, 100 with ell = 2, K = 3 gives
    levels (0, sqrt(2*100), 100) = (0, 14.142..., 100)."""
    rgba = np.zeros((2, 4, 4), np.float32)
    for x, y in enumerate([0.0, 2.0, 8.0, 100.0]):
        rgba[0, x, :3] = y
        rgba[1, x, :3] = y
    L, lohi, ch0 = orc.env_decompose(rgba, 1.0, 3, 2.0)
    l2 = math.sqrt(200.0)
    assert np.allclose(L, [0.0, l2, 100.0], rtol=1e-13)
    w = ch0[0, :, 3:]
    assert np.allclose(w[0], [1, 0, 0])
    assert np.allclose(w[1], [1 - 2 / l2, 2 / l2, 0])
    assert np.allclose(w[2], [1 - 8 / l2, 8 / l2, 0])
    assert np.allclose(w[3], [0, 0, 1])


def test_constant_and_dark_env_degenerate(orc):
    """Constant map: every level above L_1 equals the constant, every texel w_K = 1.
    Black map: the clip ell sets both ends and every texel falls into bin 1."""
    env = synth.env_constant(3.5)
    L, lohi, ch0 = orc.env_decompose(env.rgba32(), 1.0, 4, 1e-4)
    assert np.allclose(L[1:], 3.5) and L[0] == 0
    assert np.all(ch0[..., 3 + 3] == 1.0)
    black = synth.env_constant(0.0)
    L, lohi, ch0 = orc.env_decompose(black.rgba32(), 1.0, 4, 1e-3)
    assert np.allclose(L[1:], 1e-3)
    assert np.all(ch0[..., 3] == 1.0)


def _texel_solid_angles(W, H):
    y = np.arange(H)
    band = np.cos(np.pi * y / H) - np.cos(np.pi * (y + 1) / H)
    return np.repeat(band[:, None], W, axis=1) * (2 * np.pi / W)


def test_pyramid_preserves_integrals(orc):
    """Each level is a solid-angle weighted mean of its children, so the integral
    of every channel over the sphere is the same on every level."""
    env = synth.env_hdr(seed=2, W=64, H=32)
    e = orc.env_full(env.rgba32(), env.scale, 4, 1e-4)
    ref = None
    for lev in e.mips:
        Hm, Wm, C = lev.shape
        integral = np.tensordot(_texel_solid_angles(Wm, Hm), lev, axes=([0, 1], [0, 1]))
        if ref is None:
            ref = integral
        assert np.allclose(integral, ref, rtol=1e-12)
    assert len(e.mips) == orc.mip_count(32) == 6 and e.mips[-1].shape[:2] == (1, 2)


def test_filter_constant_env(orc):
    """A constant environment filters to itself: RGB = constant, W_K = 1."""
    env = synth.env_constant(2.0)
    e = orc.env_full(env.rgba32(), 1.0, 4, 1e-4)
    pref = orc.prefilter(e, 4, 32, math.sqrt(0.02), math.sqrt(0.5), 16).flat
    assert np.allclose(pref[..., :3], 2.0, rtol=1e-13)
    assert np.allclose(pref[..., 3 + 3], 1.0, rtol=1e-13)
    assert np.allclose(pref[..., 3:6], 0.0, atol=1e-13)


def test_filter_partition_of_unity(orc):
    env = synth.env_tiny(0)
    e = orc.env_full(env.rgba32(), 1.0, 8, 1e-4)
    pref = orc.prefilter(e, 5, 64, math.sqrt(0.02), math.sqrt(0.5), 32).flat
    assert np.allclose(pref[..., 3:].sum(-1), 1.0, atol=1e-13)
    assert np.all(pref[..., 3:] >= 0)


def test_filter_narrow_lobe_is_identity(orc):
    """As alpha -> 0 every sample reflects into w_r and reads level 0, so the
    filtered map sampled at the texel centres of the source is the source."""
    env = synth.env_tiny(1)
    e = orc.env_full(env.rgba32(), 1.0, 4, 1e-4)
    pref = orc.prefilter(e, 1, 16, 1e-7, 1e-7, 64)
    assert np.allclose(pref.levels[0], e.ch0, rtol=1e-6, atol=1e-9)


def test_filtered_level_widths(orc):
    """Level r has about 2 pi / alpha_r texels around the equator (a power of two),
    clamped to the requested maximum: 256..16 for sqrt(alpha) in [sqrt .02, sqrt .5]."""
    w = orc.filtered_widths(8, math.sqrt(0.02), math.sqrt(0.5), 256)
    assert list(w) == [256, 128, 64, 32, 32, 16, 16, 16]
    for r, wr in enumerate(w):
        s = math.sqrt(0.02) + (math.sqrt(0.5) - math.sqrt(0.02)) * r / 7
        texel = 2 * math.pi / wr
        assert 2 ** -0.5 <= texel / s ** 2 <= 2 ** 0.5
    assert list(orc.filtered_widths(3, 0.9, 1.0, 4)) == [4, 4, 4]


def test_filter_sample_table(orc):
    """Hammersley table: reflected directions are unit vectors on the lobe side
    (cos 2 theta_h > 0); narrow lobes keep every sample, alpha = 0.5 keeps the
    fraction u < 0.8 (tan^2 theta_h < 1); lod grows as D(h) falls."""
    tab, nv = orc.prefilter_table(2, 64, math.sqrt(0.02), math.sqrt(0.5), 1024, 512)
    assert nv[0] == 64
    assert nv[1] == int(np.sum((np.arange(64) + 0.5) / 64 < 0.8))
    for r in range(2):
        t = tab[r, :nv[r]]
        assert np.allclose(np.linalg.norm(t[:, :3], axis=1), 1.0, atol=1e-14)
        assert np.all(t[:, 2] > 0)
        assert np.all(np.diff(t[:, 3]) >= -1e-12)


def test_filter_close_to_exact_convolution(orc):
    """Filtered importance sampling vs the plain texel-sum quadrature of the same
    kernel (Sec. 3.4): the difference is the sampling and mip error, bounded here
    on a smooth map."""
    env = synth.env_hdr(seed=9, W=128, H=64, n_suns=0, sigma=0.7, fp16=False, scale_log2=0)
    e = orc.env_full(env.rgba32(), 1.0, 4, 1e-4)
    s = math.sqrt(0.3)
    Wo, Ho = 16, 8
    pref = orc.prefilter(e, 1, 256, s, s, Wo)
    assert list(pref.widths) == [Wo]
    y, x = np.meshgrid(np.arange(Ho), np.arange(Wo), indexing="ij")
    th, ph = np.pi * (y + 0.5) / Ho, 2 * np.pi * (x + 0.5) / Wo
    dirs = np.stack([np.sin(th) * np.cos(ph), np.cos(th), np.sin(th) * np.sin(ph)], -1).reshape(-1, 3)
    ex = orc.prefilter_exact(e.ch0, 0.3, dirs).reshape(Ho, Wo, -1)
    lev = pref.levels[0]
    rel = np.abs(lev[..., :3] - ex[..., :3]) / ex[..., :3]
    assert np.median(rel) < 0.03 and np.max(rel) < 0.12
    assert np.max(np.abs(lev[..., 3:] - ex[..., 3:])) < 0.05


def test_log_space_weights(orc):
    """Sec. 7 "Linear vs Logarithmic Radiance": weights interpolated in log
    space reconstruct ln Y = sum_k w_k ln L_k exactly between L_2 and L_K, keep
    the partition of unity, fall back to linear below L_2 (L_1 = 0) and give
    w_K = 1 at the top; linear weights reconstruct Y instead."""
    rng = np.random.default_rng(5)
    H, W = 16, 32
    rgba = np.zeros((H, W, 4), np.float32)
    rgba[..., :3] = (10.0 ** rng.uniform(-3, 3, size=(H, W, 1))).astype(np.float32)
    rgba[..., 3] = 1
    K = 8
    L, lohi, ch_lin = orc.env_decompose(rgba, 1.0, K, 1e-4)
    L2, lohi2, ch_log = orc.env_decompose(rgba, 1.0, K, 1e-4, log_space=True)
    assert np.array_equal(L, L2) and np.array_equal(lohi, lohi2)
    Y = np.maximum(rgba[..., :3].astype(np.float64) @ [0.2126, 0.7152, 0.0722], 0)
    w_lin, w_log = ch_lin[..., 3:], ch_log[..., 3:]
    np.testing.assert_allclose(w_log.sum(-1), 1.0, atol=1e-12)
    np.testing.assert_allclose((w_lin * L).sum(-1), Y, rtol=1e-12)
    mid = (Y >= L[1]) & (Y < L[-1])
    lnL = np.log(np.maximum(L, 1e-300))
    recon = (w_log * np.where(L > 0, lnL, 0.0)).sum(-1)
    np.testing.assert_allclose(recon[mid], np.log(Y[mid]), rtol=0, atol=1e-12)
    low = Y < L[1]
    assert low.any() and mid.any()
    np.testing.assert_array_equal(w_log[low], w_lin[low])
    top = Y >= L[-1]
    assert np.all(w_log[top][:, -1] == 1.0)
    # ln is concave, so the log-space factor (ln Y - ln L_j)/(ln L_{j+1} - ln L_j)
    # is at least the linear one: log weights lean to the upper level
    j = np.argmax(w_lin[mid] > 0, axis=-1)
    assert np.all(w_log[mid][np.arange(j.size), j] <= w_lin[mid][np.arange(j.size), j] + 1e-12)


def test_weight_storage_formats_and_precision_study(orc):
    """Sec. 7 "Texture Precision": the filtered weights stored as float16,
    unorm16 or unorm8.  The quantisers follow their definitions (hand values),
    and the paper's finding holds: 16-bit storage changes p_k by ~1e-5 (RMSE)
    while 8-bit loses small weights outright and changes the glint image far
    more."""
    from tests._pipeline import MethodParams, oracle_shade
    flat = np.array([[1.0, 2.0, 3.0, 0.5, 1.0 / 3.0, 0.0, 1.0, 1e-3, -1e-9]])
    u16 = orc.quantize_weights(flat, orc.WFMT_UNORM16)[0]
    assert u16[3] == 32768 / 65535 and u16[4] == 21845 / 65535 and u16[5] == 0 and u16[6] == 1
    assert u16[7] == 66 / 65535 and u16[8] == 0 and list(u16[:3]) == [1.0, 2.0, 3.0]
    u8 = orc.quantize_weights(flat, orc.WFMT_UNORM8)[0]
    assert u8[3] == 128 / 255 and u8[4] == 85 / 255 and u8[7] == 0.0
    f16 = orc.quantize_weights(flat, orc.WFMT_F16)[0]
    assert f16[4] == 0.333251953125 and f16[3] == 0.5 and f16[7] == 0.0010004043579101562

    env = synth.env_hdr(seed=3, W=256, H=128)
    rows = synth.gbuffer_random(1500, seed=5).rows16()
    res = {}
    for wf in (0, 1, 2, 3):
        res[wf] = oracle_shade(orc, rows, env, MethodParams(K=8, Wo=128, wfmt=wf), tie=[0, 0, 0, 0, 0], max_cand=1)
    fg = res[0].np_ > 0
    p0 = res[0].pk[fg]

    def p_rmse(wf):
        return float(np.sqrt(np.mean((res[wf].pk[fg] - p0) ** 2)))

    def img(wf):
        d = np.abs(res[wf].rgb[fg] - res[0].rgb[fg]).sum(1) / np.maximum(res[0].rgb[fg].sum(1), 1e-12)
        return float(np.median(d))

    assert p_rmse(1) < 1e-4 and p_rmse(2) < 1e-4 and p_rmse(3) > 2e-4
    assert img(3) > 10 * max(img(1), img(2))
    small = (p0 > 1e-3) & (p0 < 1.5e-3)
    assert small.any() and np.all(res[3].pk[fg][small] != p0[small])


def _bilinear_dirs(lev, d):
    """Bilinear look-up of an equirect level (wrap in phi, clamp in theta) at
    unit directions d, as the shading look-ups read the filtered maps."""
    Hl, Wl = lev.shape[:2]
    th = np.arccos(np.clip(d[:, 1], -1.0, 1.0))
    ph = np.arctan2(d[:, 2], d[:, 0]) % (2.0 * np.pi)
    x, y = ph / (2.0 * np.pi) * Wl - 0.5, th / np.pi * Hl - 0.5
    x0, y0 = np.floor(x), np.floor(y)
    fx, fy = (x - x0)[:, None], (y - y0)[:, None]
    xa = x0.astype(int) % Wl
    xb = (xa + 1) % Wl
    ya, yb = np.clip(y0.astype(int), 0, Hl - 1), np.clip(y0.astype(int) + 1, 0, Hl - 1)
    return ((1 - fy) * ((1 - fx) * lev[ya, xa] + fx * lev[ya, xb])
            + fy * ((1 - fx) * lev[yb, xa] + fx * lev[yb, xb]))


# Bounds of the filter against the exact convolution on a map with two suns
# (radiance 1e3-1e4, 2-6 degrees wide) at 64 samples, measured on this map
# with lod bias -1/2 and set about 1.3x above it: (median and 90th percentile
# of the relative luminance error, 99th percentile of the largest absolute
# weight error), at 3000 random directions read through the level's bilinear
# look-up.
FILTER_BOUNDS = {0.05: (0.034, 0.22, 0.015), 0.15: (0.13, 0.32, 0.028), 0.4: (0.107, 0.32, 0.025)}


def _filter_errors(orc, e, alpha, d, ex, lod_shift=0.0, width_scale=1.0):
    s = math.sqrt(alpha)
    H, W = e.ch0.shape[:2]
    table, nvalid = orc.prefilter_table(1, 64, s, s, W, H)
    table[:, :nvalid[0], 3] = np.clip(table[:, :nvalid[0], 3] + lod_shift, 0, orc.mip_count(H) - 1)
    widths = (orc.filtered_widths(1, s, s, 256) * width_scale).astype(np.int32)
    got = _bilinear_dirs(orc.prefilter_with(e, table, nvalid, widths)[0], d)
    Y = lambda v: v[:, :3] @ np.array([0.2126, 0.7152, 0.0722])  # noqa: E731
    rel = np.abs(Y(got) - Y(ex)) / Y(ex)
    werr = np.abs(got[:, 3:] - ex[:, 3:]).max(1)
    return np.median(rel), np.percentile(rel, 90), np.percentile(werr, 99)


@pytest.fixture(scope="module")
def sun_map(orc):
    env = synth.env_hdr(seed=5, W=256, H=128, n_suns=2, sun_lo=1e3, sun_hi=1e4, fp16=False, scale_log2=0,
                        sigma=1.0)
    e = orc.env_full(env.rgba32(), env.scale, 4, 1e-4)
    rng = np.random.default_rng(3)
    d = rng.normal(size=(3000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    exact = {a: orc.prefilter_exact(e.ch0, a, d) for a in FILTER_BOUNDS}
    return e, d, exact


@pytest.mark.parametrize("alpha", sorted(FILTER_BOUNDS))
def test_filter_with_suns_against_exact_convolution(orc, sun_map, alpha):
    """Filtered importance sampling (Sec. 3.4 Eq. rtibl, Sec. 4 Eq. rtiblndf)
    against the plain texel-sum convolution of the same kernel, on a map with
    bright suns, at three roughness levels, through the bilinear look-up the
    shading uses: within the bounds above."""
    e, d, exact = sun_map
    err = _filter_errors(orc, e, alpha, d, exact[alpha])
    assert all(v <= b for v, b in zip(err, FILTER_BOUNDS[alpha])), (err, FILTER_BOUNDS[alpha])


@pytest.mark.parametrize("mistake", [{"lod_shift": 1.5}, {"lod_shift": 0.5}, {"lod_shift": -1.0},
                                     {"width_scale": 0.5}])
def test_filter_bounds_catch_a_wrong_lod_or_width(orc, sun_map, mistake):
    """The bounds have teeth: the published lod bias +1 (a shift of +1.5), a
    shift of 1/2 either way, or levels half as wide as the width rule gives,
    planted in the oracle's sample table or level widths, exceed a bound at one
    of the three roughness levels at least."""
    e, d, exact = sun_map
    over = [any(v > b for v, b in zip(_filter_errors(orc, e, a, d, exact[a], **mistake), FILTER_BOUNDS[a]))
            for a in sorted(FILTER_BOUNDS)]
    assert any(over), mistake
