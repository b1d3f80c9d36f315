"""Oracle of the learned warm start: a plain float64 NumPy statement of the
per-point MLP, its gradient and its Adam update.  Test infrastructure: only
the tests, the smoke check and the benchmark's CPU leg use it; the CUDA path
shares nothing with it.

The warm start is an addition to the paper's method (its SCF runs start from
superposed atomic data, Section 6): a network maps features of a mesh point
(distances to the two nearest nuclei and the atomic Slater orbitals) to a
relative correction y of the superposition start s, psi = s (1 + y).

Definitions (F = 8 features, H hidden units, tanh):
- features of a point x with nearest nuclei at distances r1 <= r2 and
  separation R of those two nuclei:
  [e^-r1, e^-r2, tanh r1, tanh r2, (r2 - r1)/R, tanh((r1 + r2)/R - 1),
   R - 1.5, e^-(r1 + r2 - R)], each rounded to bfloat16 (with a decay rate
  z per nucleus the first two are e^-(z1 r1) and e^-(z2 r2));
- parameters, in this order: W1 (H x F), b1 (H), W2 (H x H), b2 (H),
  W3 (H), b3 (1); the weights W1, W2, W3 enter the products rounded to
  bfloat16, the biases unrounded;
- forward: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 . h2 + b3;
- loss: L = sum_p wt_p (y_p - t_p)^2, its gradient by the chain rule, with
  the gradient of a rounded weight applied to its unrounded master value;
- Adam (Kingma and Ba, 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 8


def n_params(F: int = N_FEATURES, H: int = 32) -> int:
    return H * F + H + H * H + H + H + 1


def bf16_round(x):
    """Nearest bfloat16 value (8 significant bits, exponent range of
    float32), ties to even, rounded directly from float64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)  # x = m 2^e, 0.5 <= |m| < 1
    q = np.ldexp(1.0, np.maximum(e - 8, -133))  # spacing of bfloat16 values at x
    return np.where(x == 0.0, x, np.rint(x / q) * q)


def unpack(params, F: int = N_FEATURES, H: int = 32):
    p = np.asarray(params, dtype=np.float64)
    if p.size != n_params(F, H):
        raise ValueError("parameter count")
    o = 0
    out = []
    for shape in ((H, F), (H,), (H, H), (H,), (H,), (1,)):
        k = int(np.prod(shape))
        out.append(p[o:o + k].reshape(shape))
        o += k
    return out


def features(xyz, nuclei, ordered: bool = False, scale=None):
    """xyz (3, n), nuclei (m, 3) with m >= 2: the bfloat16-rounded features
    (n, 8) of the definition above.  ordered (m = 2 only): r1 and r2 are the
    distances to the first and the second nucleus of the list, unsorted.
    scale (m,): a decay rate z per nucleus; the first two features are then
    e^-(z1 r1) and e^-(z2 r2) with z1, z2 the rates of the nuclei at r1, r2."""
    xyz = np.asarray(xyz, dtype=np.float64)
    nuc = np.asarray(nuclei, dtype=np.float64).reshape(-1, 3)
    if nuc.shape[0] < 2 or (ordered and nuc.shape[0] != 2):
        raise ValueError("need two nuclei (exactly two in list order)")
    d = np.sqrt(((xyz.T[:, None, :] - nuc[None, :, :]) ** 2).sum(axis=2))  # (n, m)
    if ordered:
        i1 = np.zeros(d.shape[0], dtype=np.int64)
        i2 = np.ones(d.shape[0], dtype=np.int64)
    else:
        order = np.argsort(d, axis=1, kind="stable")
        i1, i2 = order[:, 0], order[:, 1]
    rows = np.arange(d.shape[0])
    r1, r2 = d[rows, i1], d[rows, i2]
    z = np.ones(nuc.shape[0]) if scale is None else np.asarray(scale, dtype=np.float64).ravel()
    if z.size != nuc.shape[0] or not np.all(np.isfinite(z) & (z > 0)):
        raise ValueError("one finite positive decay rate per nucleus")
    R = np.sqrt(((nuc[i1] - nuc[i2]) ** 2).sum(axis=1))
    f = np.stack([np.exp(-z[i1] * r1), np.exp(-z[i2] * r2), np.tanh(r1), np.tanh(r2), (r2 - r1) / R,
                  np.tanh((r1 + r2) / R - 1.0), R - 1.5, np.exp(-(r1 + r2 - R))], axis=1)
    return bf16_round(f)


def forward(params, x, H: int = 32, round_weights: bool = True):
    """x (n, F).  Returns y (n,) and the intermediates (h1, h2).
    round_weights=False evaluates the unrounded float64 network."""
    W1, b1, W2, b2, W3, b3 = unpack(params, x.shape[1], H)
    if round_weights:
        W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3 + b3[0], (h1, h2)


def loss_grad(params, x, t, wt, H: int = 32, round_weights: bool = True):
    """Loss L = sum_p wt_p (y_p - t_p)^2 and dL/dparams (packed like
    params)."""
    W1, b1, W2, b2, W3, b3 = unpack(params, x.shape[1], H)
    W2r, W3r = (bf16_round(W2), bf16_round(W3)) if round_weights else (W2, W3)
    y, (h1, h2) = forward(params, x, H, round_weights)
    r = y - t
    L = float(np.sum(wt * r * r))
    dy = 2.0 * wt * r                       # dL/dy
    dz2 = dy[:, None] * W3r[None, :] * (1.0 - h2 * h2)
    dz1 = (dz2 @ W2r) * (1.0 - h1 * h1)
    g = [dz1.T @ x, dz1.sum(0), dz2.T @ h1, dz2.sum(0), dy @ h2, np.array([dy.sum()])]
    return L, np.concatenate([a.ravel() for a in g])


# --------------------------------------------------------------------------
# The tensor-core form (H = 64): the inputs of the three per-point products
# and of the gradient sums over points are rounded to bfloat16, as the tensor
# cores take them; everything else as above.
#   forward:  h1 = tanh(x W1^T + b1), z2 = bf16(h1) W2^T + b2, h2 = tanh z2,
#             y = W3 . h2 + b3;
#   gradient: dy = 2 wt (y - t), dz2 = dy W3 (1 - h2^2),
#             dz1 = (bf16(dz2) W2) (1 - h1^2),
#             dW1 = bf16(dz1)^T x, db1 = sum bf16(dz1),
#             dW2 = bf16(dz2)^T bf16(h1), db2 = sum bf16(dz2),
#             dW3 = bf16(dy) bf16(h2), db3 = sum bf16(dy).
# (W1, W2, W3 rounded to bfloat16 and x bfloat16 as before.)
# --------------------------------------------------------------------------
def forward_tc(params, x, H: int = 64):
    W1, b1, W2, b2, W3, b3 = unpack(params, x.shape[1], H)
    W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    h1 = np.tanh(x @ W1.T + b1)
    h1b = bf16_round(h1)
    h2 = np.tanh(h1b @ W2.T + b2)
    return h2 @ W3 + b3[0], (h1, h1b, h2)


def loss_grad_tc(params, x, t, wt, H: int = 64):
    W1, b1, W2, b2, W3, b3 = unpack(params, x.shape[1], H)
    W2r, W3r = bf16_round(W2), bf16_round(W3)
    y, (h1, h1b, h2) = forward_tc(params, x, H)
    r = y - t
    L = float(np.sum(wt * r * r))
    dy = 2.0 * wt * r
    dz2b = bf16_round(dy[:, None] * W3r[None, :] * (1.0 - h2 * h2))
    dz1b = bf16_round((dz2b @ W2r) * (1.0 - h1 * h1))
    dyb, h2b = bf16_round(dy), bf16_round(h2)
    g = [dz1b.T @ x, dz1b.sum(0), dz2b.T @ h1b, dz2b.sum(0), dyb @ h2b, np.array([dyb.sum()])]
    return L, np.concatenate([a.ravel() for a in g])


def adam_step(params, m, v, g, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t >= 1; returns (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1**t)
    vh = v / (1.0 - beta2**t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def train(params, x, t, wt, steps: int, lr, H: int = 32, beta1=0.9, beta2=0.999, eps=1e-8, tc: bool = False):
    """Full-batch Adam; lr is a number or a function of the step (1-based);
    tc: the tensor-core form.  Returns (params, losses before each update)."""
    p = np.asarray(params, dtype=np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    losses = []
    for k in range(1, steps + 1):
        L, g = loss_grad_tc(p, x, t, wt, H) if tc else loss_grad(p, x, t, wt, H)
        losses.append(L)
        p, m, v = adam_step(p, m, v, g, k, lr(k) if callable(lr) else lr, beta1, beta2, eps)
    return p, np.array(losses)


def warm_start(params, x, s, w, H: int = 32, tc: bool = False):
    """psi = s (1 + y) normalised in the quadrature-weighted norm."""
    y, _ = forward_tc(params, x, H) if tc else forward(params, x, H)
    psi = s * (1.0 + y)
    return psi / np.sqrt(np.sum(psi * psi * w))
