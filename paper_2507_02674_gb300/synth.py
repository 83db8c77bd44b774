"""Seeded synthetic inputs: environment maps and G-buffers.

This module only makes input data (ray casting of simple scenes, random HDR
environment maps, random materials).  It holds none of the shading method's
arithmetic and is the one module that both the CUDA path's tests/benchmark and
the CPU oracle's tests draw their inputs from.

G-buffer layout (what the shading call reads): four planes of float4 per
pixel, row-major over the image,
  plane 0: w_o.xyz (unit vector from the surface towards the viewer), N_0
           (microfacets per unit uv area; <= 0 marks a background pixel)
  plane 1: n.xyz (unit shading normal), F0 (Schlick reflectance)
  plane 2: u, v, alpha_x, alpha_y
  plane 3: du/dx, dv/dx, du/dy, dv/dy (screen-space derivatives of uv)
  tangent (optional fifth plane): t.xyz, 0 -- the direction of alpha_x, used by
           the anisotropic quadrature evaluator
Environment maps are equirectangular W x H (W = 2H) RGBA images, texel (x, y)
centred on phi = 2 pi (x+1/2)/W, theta = pi (y+1/2)/H around the +y axis,
direction (sin th cos ph, cos th, sin th sin ph).  Radiance = stored value *
2^scale_log2.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class GBuffer:
    width: int
    height: int
    planes: list  # four float32 arrays (H, W, 4)
    desc: str = ""
    tangent: np.ndarray | None = None  # (H, W, 4) float32: t.xyz, 0

    @property
    def npix(self) -> int:
        return self.width * self.height

    def rows16(self) -> np.ndarray:
        """(npix, 16) float32 rows: the four planes side by side."""
        return np.ascontiguousarray(
            np.concatenate([p.reshape(-1, 4) for p in self.planes], axis=1).astype(np.float32))

    def nbytes(self) -> int:
        return sum(p.nbytes for p in self.planes)

    def tangents(self) -> np.ndarray:
        """(npix, 4) float32 tangent rows."""
        return np.ascontiguousarray(self.tangent.reshape(-1, 4).astype(np.float32))


@dataclass
class EnvMap:
    texels: np.ndarray  # (H, W, 4) float32 or float16
    scale_log2: int = 0
    desc: str = ""

    @property
    def width(self) -> int:
        return self.texels.shape[1]

    @property
    def height(self) -> int:
        return self.texels.shape[0]

    def rgba32(self) -> np.ndarray:
        """Stored texels as float32 (exact for float16 storage)."""
        return np.ascontiguousarray(self.texels.astype(np.float32))

    @property
    def scale(self) -> float:
        return float(2.0 ** self.scale_log2)


# ------------------------------------------------------------------ env maps
def _texel_dirs(W: int, H: int) -> np.ndarray:
    y, x = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    th = np.pi * (y + 0.5) / H
    ph = 2.0 * np.pi * (x + 0.5) / W
    return np.stack([np.sin(th) * np.cos(ph), np.cos(th), np.sin(th) * np.sin(ph)], axis=-1)


def _dir(theta: float, phi: float) -> np.ndarray:
    return np.array([np.sin(theta) * np.cos(phi), np.cos(theta), np.sin(theta) * np.sin(phi)])


def _add_sun(img: np.ndarray, dirs: np.ndarray, d: np.ndarray, radiance: float, radius: float, tint=(1.0, 1.0, 1.0)):
    cosg = np.clip(dirs @ d, -1.0, 1.0)
    g = np.arccos(cosg)
    prof = radiance * np.exp(-0.5 * (g / radius) ** 2)
    for c in range(3):
        img[..., c] += tint[c] * prof


def env_tiny(seed: int = 0, W: int = 64, H: int = 32) -> EnvMap:
    """64 x 32 fp32 map: iid log-normal(0, 1) grey texels plus two Gaussian
    suns of radiance 1e3 and angular radius 2 degrees, centred on texels."""
    rng = np.random.default_rng(seed)
    dirs = _texel_dirs(W, H)
    img = np.zeros((H, W, 4))
    grey = np.exp(rng.normal(0.0, 1.0, size=(H, W)))
    img[..., 0] = img[..., 1] = img[..., 2] = grey
    for (x, y) in ((W // 4, (10 * H) // 32), ((5 * W) // 8, (6 * H) // 32)):
        th = np.pi * (y + 0.5) / H
        ph = 2.0 * np.pi * (x + 0.5) / W
        _add_sun(img, dirs, _dir(th, ph), 1e3, np.radians(2.0))
    img[..., 3] = 1.0
    return EnvMap(img.astype(np.float32), 0, f"tiny {W}x{H} fp32 log-normal(0,1) + 2 suns 1e3")


def env_hdr(seed: int = 1, W: int = 1024, H: int = 512, sigma: float = 1.5, n_suns: int = 4,
            sun_lo: float = 1e3, sun_hi: float = 1e5, fp16: bool = True, scale_log2: int = 4) -> EnvMap:
    """HDR map shaped like an outdoor probe: a smooth log-normal field with
    standard deviation `sigma` in log radiance (random low-frequency modes
    plus a sky/ground gradient), and `n_suns` Gaussian suns of radiance
    log-uniform in [sun_lo, sun_hi] and radius uniform in [1, 3] degrees.
    Stored as RGBA16F divided by 2^scale_log2 so the suns stay below the fp16
    maximum."""
    rng = np.random.default_rng(seed)
    dirs = _texel_dirs(W, H)
    field = np.zeros((H, W))
    for _ in range(24):
        k = rng.normal(size=3)
        k *= rng.uniform(1.0, 6.0) / np.linalg.norm(k)
        field += np.cos(dirs @ k + rng.uniform(0, 2 * np.pi)) * rng.uniform(0.5, 1.0)
    field += 0.8 * dirs[..., 1]  # brighter sky than ground
    field = (field - field.mean()) / field.std()
    logL = sigma * field
    img = np.zeros((H, W, 4))
    tint = np.stack([np.ones((H, W)), 0.95 + 0.05 * dirs[..., 1], 0.9 + 0.1 * dirs[..., 1]], axis=-1)
    img[..., :3] = np.exp(logL)[..., None] * tint
    for _ in range(n_suns):
        th = np.arccos(rng.uniform(-0.2, 0.95))
        ph = rng.uniform(0, 2 * np.pi)
        rad = np.exp(rng.uniform(np.log(sun_lo), np.log(sun_hi)))
        _add_sun(img, dirs, _dir(th, ph), rad, np.radians(rng.uniform(1.0, 3.0)), tint=(1.0, 0.96, 0.88))
    img[..., 3] = 1.0
    img[..., :3] /= 2.0 ** scale_log2
    dt = np.float16 if fp16 else np.float32
    return EnvMap(img.astype(dt), scale_log2,
                  f"hdr {W}x{H} {'RGBA16F' if fp16 else 'RGBA32F'} log-normal sigma={sigma} + {n_suns} suns")


def env_constant(value: float = 1.0, W: int = 64, H: int = 32) -> EnvMap:
    img = np.zeros((H, W, 4), np.float32)
    img[..., :3] = value
    img[..., 3] = 1.0
    return EnvMap(img, 0, f"constant {value}")


# ------------------------------------------------------------------ G-buffers
def _sphere_uv(nrm: np.ndarray, uv_scale: float):
    th = np.arccos(np.clip(nrm[..., 1], -1.0, 1.0))
    ph = np.arctan2(nrm[..., 2], nrm[..., 0])
    return uv_scale * ph / (2 * np.pi), uv_scale * th / np.pi


def _sphere_duv(nrm: np.ndarray, dn: np.ndarray, uv_scale: float):
    """uv differential of the sphere parametrisation for a normal change dn."""
    st = np.sqrt(np.maximum(1.0 - nrm[..., 1] ** 2, 1e-12))
    dth = -dn[..., 1] / st
    rxz = np.maximum(nrm[..., 0] ** 2 + nrm[..., 2] ** 2, 1e-12)
    dph = (nrm[..., 0] * dn[..., 2] - nrm[..., 2] * dn[..., 0]) / rxz
    return uv_scale * dph / (2 * np.pi), uv_scale * dth / np.pi


def _tangent_plane_hit(p, n, o, d):
    """Intersection of rays o + t d with the tangent planes (p, n)."""
    t = np.sum(n * (p - o), axis=-1) / np.where(np.abs(np.sum(n * d, -1)) > 1e-12, np.sum(n * d, -1), 1e-12)
    return o + t[..., None] * d


def gbuffer_sphere(W: int = 64, H: int = 64, alpha: float = 0.15, N0: float = 1e4, uv_scale: float = 8.0,
                   F0: float = 0.9) -> GBuffer:
    """Unit sphere at the origin seen head-on by an orthographic camera looking
    down -z; the frame spans [-1, 1]^2.  Isotropic alpha, constant density."""
    xs = -1.0 + (np.arange(W) + 0.5) * (2.0 / W)
    ys = 1.0 - (np.arange(H) + 0.5) * (2.0 / H)
    X, Y = np.meshgrid(xs, ys)
    r2 = X ** 2 + Y ** 2
    hit = r2 < 1.0
    Z = np.sqrt(np.maximum(1.0 - r2, 0.0))
    p = np.stack([X, Y, Z], -1)
    n = p.copy()
    wo = np.broadcast_to(np.array([0.0, 0.0, 1.0]), p.shape)
    d = np.broadcast_to(np.array([0.0, 0.0, -1.0]), p.shape)
    o = p + 5.0 * wo
    u, v = _sphere_uv(n, uv_scale)
    dx = np.array([2.0 / W, 0.0, 0.0])
    dy = np.array([0.0, -2.0 / H, 0.0])
    px = _tangent_plane_hit(p, n, o + dx, d) - p
    py = _tangent_plane_hit(p, n, o + dy, d) - p
    dudx, dvdx = _sphere_duv(n, px, uv_scale)
    dudy, dvdy = _sphere_duv(n, py, uv_scale)
    planes = [np.zeros((H, W, 4), np.float32) for _ in range(4)]
    planes[0][..., :3] = wo
    planes[0][..., 3] = np.where(hit, N0, 0.0)
    planes[1][..., :3] = np.where(hit[..., None], n, np.array([0.0, 0.0, 1.0]))
    planes[1][..., 3] = F0
    planes[2][..., 0] = np.where(hit, u, 0.0)
    planes[2][..., 1] = np.where(hit, v, 0.0)
    planes[2][..., 2] = alpha
    planes[2][..., 3] = alpha
    planes[3][..., 0] = np.where(hit, dudx, 0.0)
    planes[3][..., 1] = np.where(hit, dvdx, 0.0)
    planes[3][..., 2] = np.where(hit, dudy, 0.0)
    planes[3][..., 3] = np.where(hit, dvdy, 0.0)
    tan = np.zeros((H, W, 4), np.float32)
    ph = np.arctan2(n[..., 2], n[..., 0])
    tan[..., 0] = -np.sin(ph)
    tan[..., 2] = np.cos(ph)
    return GBuffer(W, H, planes, f"sphere {W}x{H} ortho alpha={alpha} N0={N0:g} uv x{uv_scale:g}", tan)


def _random_materials(rng, shape, a_lo, a_hi, n_lo, n_hi):
    ax = rng.uniform(a_lo, a_hi, size=shape)
    ay = rng.uniform(a_lo, a_hi, size=shape)
    N0 = 10.0 ** rng.uniform(np.log10(n_lo), np.log10(n_hi), size=shape)
    F0 = rng.uniform(0.5, 1.0, size=shape)
    return ax, ay, N0, F0


def gbuffer_scene(W: int = 1920, H: int = 1080, seed: int = 1, n_spheres: int = 16, fov_deg: float = 60.0,
                  cam_height: float = 4.0, pitch_deg: float = 35.0, a_lo: float = 0.03, a_hi: float = 0.3,
                  n_lo: float = 1e3, n_hi: float = 1e8, plane_uv: float = 1.0, sphere_uv: float = 8.0) -> GBuffer:
    """Ground plane y = 0 plus `n_spheres` spheres (radius U[0.2, 1], resting
    on the plane, centres in [-6, 6]^2), seen by a perspective camera at height
    `cam_height` pitched down by `pitch_deg` (the whole frame hits geometry for
    pitch > fov/2).  Per-pixel iid alpha_x, alpha_y ~ U[a_lo, a_hi], N_0
    log-uniform in [n_lo, n_hi], F0 ~ U[0.5, 1].  uv = plane_uv (x, z) on the
    plane, sphere_uv (phi/2pi, theta/pi) on spheres; uv derivatives by ray
    differentials on the tangent plane."""
    rng = np.random.default_rng(seed)
    radii = rng.uniform(0.2, 1.0, n_spheres)
    centres = np.stack([rng.uniform(-6, 6, n_spheres), radii, rng.uniform(-6, 6, n_spheres)], -1)
    pitch = np.radians(pitch_deg)
    dist = cam_height / np.tan(pitch)
    cam = np.array([0.0, cam_height, 3.0 + dist])
    fwd = np.array([0.0, -np.sin(pitch), -np.cos(pitch)])
    right = np.array([1.0, 0.0, 0.0])
    up = np.cross(right, fwd)
    tan_half = np.tan(np.radians(fov_deg) / 2)
    aspect = W / H

    def ray_dirs(px, py):
        sx = (2.0 * (px + 0.5) / W - 1.0) * tan_half * aspect
        sy = (1.0 - 2.0 * (py + 0.5) / H) * tan_half
        d = fwd + sx[..., None] * right + sy[..., None] * up
        return d / np.linalg.norm(d, axis=-1, keepdims=True)

    PY, PX = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    d = ray_dirs(PX, PY)
    o = np.broadcast_to(cam, d.shape)
    # nearest hit: plane
    t_best = np.where(d[..., 1] < -1e-9, -cam[1] / np.minimum(d[..., 1], -1e-9), np.inf)
    obj = np.full((H, W), -1, np.int32)
    for s in range(n_spheres):
        oc = cam - centres[s]
        b = d @ oc
        c = oc @ oc - radii[s] ** 2
        disc = b * b - c
        ok = disc > 0
        t = -b - np.sqrt(np.where(ok, disc, 0.0))
        better = ok & (t > 1e-6) & (t < t_best)
        t_best = np.where(better, t, t_best)
        obj = np.where(better, s, obj)
    hit = np.isfinite(t_best)
    t_best = np.where(hit, t_best, 1.0)
    p = cam + t_best[..., None] * d
    n = np.zeros_like(p)
    n[..., 1] = 1.0
    on_sphere = obj >= 0
    cs = centres[np.maximum(obj, 0)]
    rs = radii[np.maximum(obj, 0)]
    ns = (p - cs) / rs[..., None]
    n = np.where(on_sphere[..., None], ns, n)
    wo = -d
    dxr = ray_dirs(PX + 1.0, PY)
    dyr = ray_dirs(PX, PY + 1.0)
    px = _tangent_plane_hit(p, n, o, dxr) - p
    py = _tangent_plane_hit(p, n, o, dyr) - p
    # uv and derivatives
    u = plane_uv * p[..., 0]
    v = plane_uv * p[..., 2]
    dudx, dvdx = plane_uv * px[..., 0], plane_uv * px[..., 2]
    dudy, dvdy = plane_uv * py[..., 0], plane_uv * py[..., 2]
    su, sv = _sphere_uv(ns, sphere_uv)
    sdudx, sdvdx = _sphere_duv(ns, px / rs[..., None], sphere_uv)
    sdudy, sdvdy = _sphere_duv(ns, py / rs[..., None], sphere_uv)
    u = np.where(on_sphere, su, u)
    v = np.where(on_sphere, sv, v)
    dudx = np.where(on_sphere, sdudx, dudx)
    dvdx = np.where(on_sphere, sdvdx, dvdx)
    dudy = np.where(on_sphere, sdudy, dudy)
    dvdy = np.where(on_sphere, sdvdy, dvdy)
    ax, ay, N0, F0 = _random_materials(rng, (H, W), a_lo, a_hi, n_lo, n_hi)
    planes = [np.zeros((H, W, 4), np.float32) for _ in range(4)]
    planes[0][..., :3] = wo
    planes[0][..., 3] = np.where(hit, N0, 0.0)
    planes[1][..., :3] = n
    planes[1][..., 3] = F0
    planes[2][..., 0] = u
    planes[2][..., 1] = v
    planes[2][..., 2] = ax
    planes[2][..., 3] = ay
    planes[3][..., 0] = dudx
    planes[3][..., 1] = dvdx
    planes[3][..., 2] = dudy
    planes[3][..., 3] = dvdy
    tan = np.zeros((H, W, 4), np.float32)
    sph = np.arctan2(ns[..., 2], ns[..., 0])
    tan[..., 0] = np.where(on_sphere, -np.sin(sph), 1.0)
    tan[..., 2] = np.where(on_sphere, np.cos(sph), 0.0)
    return GBuffer(W, H, planes,
                   f"scene {W}x{H} plane+{n_spheres} spheres pitch={pitch_deg} alpha~U[{a_lo},{a_hi}] "
                   f"N0~logU[{n_lo:g},{n_hi:g}]", tan)


def gbuffer_random(n: int, seed: int = 7, a_lo: float = 0.03, a_hi: float = 0.3, n_lo: float = 1e3,
                   n_hi: float = 1e8, width: int | None = None) -> GBuffer:
    """Unstructured pixels with the distributions of the 1080p scene: random
    unit normals and view directions in the normal's upper hemisphere, random
    uv in [-50, 50]^2 and log-uniform footprint derivatives."""
    rng = np.random.default_rng(seed)
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    wo = rng.normal(size=(n, 3))
    wo /= np.linalg.norm(wo, axis=1, keepdims=True)
    wo = np.where((np.sum(wo * nrm, 1) < 0)[:, None], wo - 2 * np.sum(wo * nrm, 1)[:, None] * nrm, wo)
    uv = rng.uniform(-50, 50, size=(n, 2))
    mag = 10.0 ** rng.uniform(-4, -1, size=(n, 4))
    sgn = rng.choice([-1.0, 1.0], size=(n, 4))
    ax, ay, N0, F0 = _random_materials(rng, (n,), a_lo, a_hi, n_lo, n_hi)
    W = width or n
    H = (n + W - 1) // W
    planes = [np.zeros((H * W, 4), np.float32) for _ in range(4)]
    planes[0][:n, :3] = wo
    planes[0][:n, 3] = N0
    planes[1][:n, :3] = nrm
    planes[1][:n, 3] = F0
    planes[2][:n, :2] = uv
    planes[2][:n, 2] = ax
    planes[2][:n, 3] = ay
    planes[3][:n] = mag * sgn
    planes = [p.reshape(H, W, 4) for p in planes]
    t = rng.normal(size=(n, 3))
    t -= np.sum(t * nrm, 1)[:, None] * nrm
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    tan = np.zeros((H * W, 4), np.float32)
    tan[:n, :3] = t
    tan[n:, 0] = 1.0
    return GBuffer(W, H, planes, f"random {n} px", tan.reshape(H, W, 4))


def mlp_params(seed: int = 11, K: int = 8, bias: float = 0.1) -> np.ndarray:
    """Float32 parameter vector of the p_k surrogate (layout W1 [64][64], b1,
    W2 [64][64], b2, W3 [64][16], b3) with He-normal weights, small random
    biases and zero unused output columns (>= K)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(size=(64, 64)) * np.sqrt(2.0 / 36.0)
    W1[36:] = 0.0
    W2 = rng.normal(size=(64, 64)) * np.sqrt(2.0 / 64.0)
    W3 = rng.normal(size=(64, 16)) * np.sqrt(2.0 / 64.0)
    W3[:, K:] = 0.0
    b1, b2, b3 = (rng.uniform(-bias, bias, size=n) for n in (64, 64, 16))
    b3[K:] = 0.0
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3]).astype(np.float32)


def distributions(n: int, K: int, seed: int = 12, sharp: float = 2.0) -> np.ndarray:
    """(n, K) float32 rows that are probability distributions (softmax of
    Gaussian logits scaled by `sharp`), with about a tenth of the entries 0."""
    rng = np.random.default_rng(seed)
    z = rng.normal(size=(n, K)) * sharp
    z[rng.uniform(size=(n, K)) < 0.1] = -np.inf
    z[:, 0] = np.where(np.all(np.isinf(z), axis=1), 0.0, z[:, 0])
    e = np.exp(z - z.max(axis=1, keepdims=True))
    return (e / e.sum(axis=1, keepdims=True)).astype(np.float32)
