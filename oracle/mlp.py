"""FP64 reference of the BF16 MLP surrogate of the reflection probabilities.

Test infrastructure: only the tests, the smoke check and the CPU baseline of
the benchmark use this module; the library never does.

The paper has no learned part: the network stands in for the per-component
NDF mass p_k of Eq. probhk (what the E2 quadrature computes), so its maths has
no printed reference.  This module is the plain definition of the network
(inputs from the oracle's or_mlp_features: E1's p_k, filtered weights at five
taps, mu_o, sqrt a_x, sqrt a_y; logits plus the log-prior log max(p^E1,
1e-6)), its loss (the squared error sum_k (p_k - y_k)^2 of the output
distribution, the quantity the surrogate's error is judged by), the loss
gradient by backpropagation and one Adam step, in float64 numpy.  It is
pinned, independently of itself, by central finite differences of the loss
(exact mode), by closed forms (uniform logits give p = 1/K; the first Adam
step moves every weight by lr sign(g)), and
by the BF16 rounding agreeing with PyTorch's conversion.

Two modes:
  exact=False (mirror): inputs, weights and the activations h1, h2 and the
      backpropagated dZ3, dZ2, dZ1 are rounded to BF16 at the points where
      the tensor-core kernels round them; every sum is exact (float64).
  exact=True: no rounding at all (for the finite-difference pins).

Parameter vector (float32/float64, 9360 values, in order):
  W1 [64 in][64 out], b1 [64], W2 [64][64], b2 [64], W3 [64][16], b3 [16];
columns >= K of W3 and b3 are unused.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT_PAD = 64, 64, 16
SIZES = [("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("W3", (N_HID, N_OUT_PAD)), ("b3", (N_OUT_PAD,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)
ADAM_BETA1, ADAM_BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via float32, as float64."""
    f = np.asarray(x, np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def bf16_ulp(v) -> np.ndarray:
    """Spacing of bfloat16 values at |v| (8 significant bits)."""
    _, e = np.frexp(np.maximum(np.abs(np.asarray(v, np.float64)), 2.0 ** -126))
    return np.ldexp(1.0, e - 8)


def rounding_delta(v, dv) -> np.ndarray:
    """Bound on |bf16(v') - bf16(v)| for any v' with |v' - v| <= dv: 0 when no
    rounding boundary (a midpoint between two bfloat16 values) lies within dv
    of v, else dv plus one spacing."""
    v = np.asarray(v, np.float64)
    dv = np.asarray(dv, np.float64)
    lo_b = bf16(v - dv)
    hi_b = bf16(v + dv)
    return np.where(lo_b == hi_b, 0.0, dv + bf16_ulp(np.abs(v) + dv))


def unpack(params) -> dict:
    p = np.asarray(params, np.float64)
    assert p.size == N_PARAMS
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SIZES])


def softmax(z: np.ndarray) -> np.ndarray:
    e = np.exp(z - z.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def forward(params, X, K: int, lp=None, exact: bool = False) -> dict:
    """Network outputs and the cached activations.  X: (n, 64) inputs; lp:
    (n, K) log-priors added to the logits (None: 0)."""
    rnd = (lambda a: a) if exact else bf16
    w = unpack(params)
    W1, W2, W3 = rnd(w["W1"]), rnd(w["W2"]), rnd(w["W3"][:, :K])
    x = rnd(X)
    z1 = x @ W1 + w["b1"]
    h1 = rnd(np.maximum(z1, 0.0))
    z2 = h1 @ W2 + w["b2"]
    h2 = rnd(np.maximum(z2, 0.0))
    z3 = h2 @ W3 + w["b3"][:K]
    if lp is not None:
        z3 = z3 + np.asarray(lp, np.float64)
    out = {"x": x, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "z3": z3, "p": softmax(z3),
           "W1": W1, "W2": W2, "W3": W3}
    return out


def loss(params, X, Y, K: int, lp=None, exact: bool = True) -> float:
    """Mean over the batch of the squared error sum_k (p_k - y_k)^2."""
    p = forward(params, X, K, lp, exact)["p"]
    Y = np.asarray(Y, np.float64)
    return float(np.sum((p - Y) ** 2) / X.shape[0])


def gradient(params, X, Y, K: int, lp=None, exact: bool = False) -> tuple[np.ndarray, np.ndarray, float]:
    """Gradient of `loss` by backpropagation, an elementwise magnitude bound
    on each gradient entry (the same sums taken over absolute values, with the
    backpropagated signals also bounded in absolute value), and the loss."""
    rnd = (lambda a: a) if exact else bf16
    f = forward(params, X, K, lp, exact)
    Y = np.asarray(Y, np.float64)
    B = X.shape[0]
    # d loss / d z3 through the softmax: with d = p - y and s = sum_k p_k d_k,
    # dL/dz_k = 2 p_k (d_k - s) / B
    dd = f["p"] - Y
    sd = np.sum(f["p"] * dd, axis=1, keepdims=True)
    e3 = 2.0 * f["p"] * (dd - sd) / B
    d3 = rnd(e3)
    m2 = (f["h2"] > 0).astype(np.float64)
    m1 = (f["h1"] > 0).astype(np.float64)
    e2 = (d3 @ f["W3"].T) * m2
    d2 = rnd(e2)
    e1 = (d2 @ f["W2"].T) * m1
    d1 = rnd(e1)
    g = {"W1": f["x"].T @ d1, "b1": d1.sum(0), "W2": f["h1"].T @ d2, "b2": d2.sum(0),
         "W3": np.zeros((N_HID, N_OUT_PAD)), "b3": np.zeros(N_OUT_PAD)}
    g["W3"][:, :K] = f["h2"].T @ d3
    g["b3"][:K] = d3.sum(0)
    a3 = np.abs(d3)
    a2 = (a3 @ np.abs(f["W3"]).T) * m2
    a1 = (a2 @ np.abs(f["W2"]).T) * m1
    mag = {"W1": np.abs(f["x"]).T @ a1, "b1": a1.sum(0), "W2": np.abs(f["h1"]).T @ a2, "b2": a2.sum(0),
           "W3": np.zeros((N_HID, N_OUT_PAD)), "b3": np.zeros(N_OUT_PAD)}
    mag["W3"][:, :K] = np.abs(f["h2"]).T @ a3
    mag["b3"][:K] = a3.sum(0)
    L = float(np.sum(dd ** 2) / B)
    return pack(g), pack(mag), L


# Error model of an FP32 evaluation of the mirror-mode network (the tensor-core
# kernels): products of BF16 values are exact in FP32, sums carry at most
# ACC_FWD (64-term dot products) or ACC_GRAD (sums over a batch and over
# blocks) times the sum of the absolute terms; softmax carries SOFTMAX_REL
# relative error and an FP32 log-prior LP_REL relative error.
ACC_FWD = 2.0 ** -20
ACC_GRAD = 2.0 ** -14
SOFTMAX_REL = 2.0 ** -20
LP_REL = 2.0 ** -21


def error_bounds(params, X, Y, K: int, lp=None, feat_err=None):
    """Elementwise bounds on how far an FP32 evaluation of the mirror-mode
    network may lie from this module's, propagated through every BF16
    rounding (zero where no rounding boundary or ReLU kink is within reach):
    returns (tol_p (n, K), tol_grad (N_PARAMS,)).  Y may be None (forward
    only).  feat_err: bound on the inputs' error before their rounding to
    BF16 (scalar or broadcastable; 0 when both sides are given the same
    BF16 inputs); the log-priors carry LP_REL relative error."""
    f = forward(params, X, K, lp, exact=False)
    w = unpack(params)
    aW1, aW2, aW3 = np.abs(f["W1"]), np.abs(f["W2"]), np.abs(f["W3"])
    x, h1, h2 = f["x"], f["h1"], f["h2"]
    X = np.asarray(X, np.float64)
    fe = 0.0 if feat_err is None else np.asarray(feat_err, np.float64)
    dx = rounding_delta(X, np.broadcast_to(fe, X.shape))
    dz1 = dx @ aW1 + ACC_FWD * (np.abs(x) @ aW1 + np.abs(w["b1"]))
    dh1 = rounding_delta(np.maximum(f["z1"], 0.0), dz1)
    dz2 = dh1 @ aW2 + ACC_FWD * (np.abs(h1) @ aW2 + np.abs(w["b2"]))
    dh2 = rounding_delta(np.maximum(f["z2"], 0.0), dz2)
    dz3 = dh2 @ aW3 + ACC_FWD * (np.abs(h2) @ aW3 + np.abs(w["b3"][:K]))
    if lp is not None:
        dz3 = dz3 + LP_REL * np.abs(np.asarray(lp, np.float64))
    p = f["p"]
    dp = p * np.expm1(2.0 * dz3.max(axis=1, keepdims=True)) + SOFTMAX_REL * p
    if Y is None:
        return dp, None
    Y = np.asarray(Y, np.float64)
    B = X.shape[0]
    dd = p - Y
    sd = np.sum(p * dd, axis=1, keepdims=True)
    e3 = 2.0 * p * (dd - sd) / B
    d3 = bf16(e3)
    # p off by at most dp moves d by dp and s by sum_j (dp_j |d_j| + (p_j + dp_j) dp_j);
    # the FP32 arithmetic of d, s and the product adds a few units of 2^-24
    dsd = np.sum(dp * np.abs(dd) + (p + dp) * dp, axis=1, keepdims=True)
    de3 = (2.0 / B) * (dp * np.abs(dd - sd) + (p + dp) * (dp + dsd)) \
        + 2.0 ** -21 * (2.0 / B) * p * (np.abs(dd) + np.sum(p * np.abs(dd), axis=1, keepdims=True) + np.abs(Y) + p)
    dd3 = rounding_delta(e3, de3)
    # a ReLU mask may differ where the pre-activation is within reach of 0
    u2 = np.abs(f["z2"]) <= dz2
    u1 = np.abs(f["z1"]) <= dz1
    m2 = (h2 > 0).astype(np.float64)
    m1 = (h1 > 0).astype(np.float64)
    s2 = np.abs(d3) @ aW3.T
    e2 = (d3 @ f["W3"].T) * m2
    de2 = (dd3 @ aW3.T + ACC_FWD * s2) * m2 + np.where(u2, s2 + dd3 @ aW3.T, 0.0)
    d2 = bf16(e2)
    dd2 = rounding_delta(e2, de2)
    s1 = np.abs(d2) @ aW2.T
    e1 = (d2 @ f["W2"].T) * m1
    de1 = (dd2 @ aW2.T + ACC_FWD * s1) * m1 + np.where(u1, s1 + dd2 @ aW2.T, 0.0)
    d1 = bf16(e1)
    dd1 = rounding_delta(e1, de1)

    def prod_err(a, da, d, dd):
        aa, ad = np.abs(a), np.abs(d)
        return da.T @ ad + aa.T @ dd + da.T @ dd + ACC_GRAD * (aa.T @ ad)

    g = {"W1": prod_err(x, dx, d1, dd1), "b1": dd1.sum(0) + ACC_GRAD * np.abs(d1).sum(0),
         "W2": prod_err(h1, dh1, d2, dd2), "b2": dd2.sum(0) + ACC_GRAD * np.abs(d2).sum(0),
         "W3": np.zeros((N_HID, N_OUT_PAD)), "b3": np.zeros(N_OUT_PAD)}
    g["W3"][:, :K] = prod_err(h2, dh2, d3, dd3)
    g["b3"][:K] = dd3.sum(0) + ACC_GRAD * np.abs(d3).sum(0)
    return dp, pack(g)


def adam(params, grad, m, v, step: int, lr: float):
    """One Adam step (Kingma & Ba 2015) taken as step number `step` (>= 1):
    m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
    w <- w - lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps)."""
    g = np.asarray(grad, np.float64)
    m = ADAM_BETA1 * np.asarray(m, np.float64) + (1 - ADAM_BETA1) * g
    v = ADAM_BETA2 * np.asarray(v, np.float64) + (1 - ADAM_BETA2) * g * g
    mh = m / (1 - ADAM_BETA1 ** step)
    vh = v / (1 - ADAM_BETA2 ** step)
    w = np.asarray(params, np.float64) - lr * mh / (np.sqrt(vh) + ADAM_EPS)
    return w, m, v
