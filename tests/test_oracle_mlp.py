"""Pins of the warm-start MLP oracle (oracle/mlp.py) against facts outside
its own code: torch's float32 -> bfloat16 cast and hand-worked ties for the
rounding; closed forms of the features at a nucleus and at the bond
midpoint; a hand-evaluated network whose hidden-to-hidden matrix is not
symmetric (a transposed operand changes its value); central finite
differences and torch.autograd for the gradient; the first Adam step's
closed form and convergence on a convex quadratic."""
import math

import numpy as np
import pytest

import oracle.mlp as M
from paper_2003_01833_gb300 import workloads as W

torch = pytest.importorskip("torch")


# ------------------------------------------------------------ bf16 rounding
def test_bf16_matches_torch_cast_of_float32_values():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-30, 30, size=5000),
                        rng.uniform(-1, 1, size=2000)]).astype(np.float32).astype(np.float64)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16_round(x), ref)


def test_bf16_ties_go_to_even_by_hand():
    u = 2.0 ** -7  # spacing of bfloat16 values in [1, 2)
    assert M.bf16_round(1.0 + 0.5 * u) == 1.0               # tie, 1.0 is even
    assert M.bf16_round(1.0 + 1.5 * u) == 1.0 + 2 * u       # tie, 1 + 2u is even
    assert M.bf16_round(1.0 + 0.5 * u + 2.0 ** -40) == 1.0 + u
    assert M.bf16_round(-(1.0 + 1.5 * u)) == -(1.0 + 2 * u)
    assert M.bf16_round(0.0) == 0.0
    sub = 2.0 ** -133  # smallest subnormal bfloat16
    assert M.bf16_round(1.5 * sub) == 2 * sub and M.bf16_round(0.5 * sub) == 0.0
    v = M.bf16_round(np.pi)
    assert M.bf16_round(v) == v and abs(v - np.pi) <= 2.0 ** -7


# ---------------------------------------------------------------- features
def test_features_closed_forms():
    R = 1.4
    nuc = np.array([[-R / 2, 0, 0], [R / 2, 0, 0]])
    pts = np.array([[-R / 2, 0, 0], [0, 0, 0], [R / 2, 0, 0]]).T
    f = M.features(pts, nuc)
    b = M.bf16_round
    at_nucleus = b([1.0, math.exp(-R), 0.0, math.tanh(R), 1.0, 0.0, R - 1.5, 1.0])
    midpoint = b([math.exp(-R / 2), math.exp(-R / 2), math.tanh(R / 2), math.tanh(R / 2), 0.0, 0.0, R - 1.5, 1.0])
    np.testing.assert_array_equal(f[0], at_nucleus)
    np.testing.assert_array_equal(f[2], at_nucleus)
    np.testing.assert_array_equal(f[1], midpoint)
    # a point on the bond axis beyond the right nucleus: r2 - r1 = R
    g = M.features(np.array([[R / 2 + 3.0, 0, 0]]).T, nuc)[0]
    assert g[4] == 1.0 and g[7] == b(math.exp(-(3.0 + R + 3.0 - R)))


def test_features_do_not_depend_on_nucleus_order():
    rng = np.random.default_rng(1)
    nuc = np.array([[-0.8, 0.1, 0], [0.9, 0, 0.2]])
    pts = rng.normal(size=(3, 500)) * 3
    np.testing.assert_array_equal(M.features(pts, nuc), M.features(pts, nuc[::-1]))
    f = M.features(pts, nuc)
    np.testing.assert_array_equal(M.bf16_round(f), f)
    assert np.all((f[:, 4] >= 0) & (f[:, 4] <= 1))


# ----------------------------------------------------------------- forward
def _tiny_params():
    """F = 8, H = 2; every weight exactly representable in bfloat16."""
    W1 = np.zeros((2, 8))
    W1[0, 0], W1[1, 0] = 0.5, -0.25
    b1 = np.array([0.0, 0.125])
    W2 = np.array([[0.0, 2.0], [0.5, 0.0]])
    b2 = np.zeros(2)
    W3 = np.array([1.0, -1.0])
    b3 = np.array([0.25])
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, b3])


def test_forward_hand_evaluated():
    x = np.zeros((1, 8))
    x[0, 0] = 1.0
    y, _ = M.forward(_tiny_params(), x, H=2)
    h1 = (math.tanh(0.5), math.tanh(-0.25 + 0.125))
    expect = math.tanh(2.0 * h1[1]) - math.tanh(0.5 * h1[0]) + 0.25
    assert abs(y[0] - expect) < 1e-15
    transposed = math.tanh(0.5 * h1[1]) - math.tanh(2.0 * h1[0]) + 0.25
    assert abs(expect - transposed) > 0.1


def test_forward_invariants():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(100, 8))
    p = W.mlp_init(3)
    p0 = np.zeros_like(p)
    p0[-1] = 0.375
    np.testing.assert_array_equal(M.forward(p0, x)[0], 0.375)  # a zero network is its output bias
    # with zero biases the network is odd
    y1, _ = M.forward(p, x)
    y2, _ = M.forward(p, -x)
    np.testing.assert_allclose(y1, -y2, atol=1e-15)
    # doubling W3 and b3 doubles y (powers of two commute with the rounding)
    q = p.copy()
    q[-33:] *= 2.0
    q[-1] = 0.5
    p1 = p.copy()
    p1[-1] = 0.25
    np.testing.assert_allclose(M.forward(q, x)[0], 2.0 * M.forward(p1, x)[0], rtol=1e-14, atol=1e-15)


# ---------------------------------------------------------------- gradient
def _problem(seed=4, n=40, H=5):
    rng = np.random.default_rng(seed)
    x = M.bf16_round(rng.uniform(-1, 1, size=(n, 8)))
    t = rng.normal(size=n) * 0.3
    wt = rng.uniform(0.1, 1.0, size=n) / n
    p = rng.normal(size=M.n_params(8, H)) * 0.7
    return p, x, t, wt, H


def test_gradient_against_central_differences():
    p, x, t, wt, H = _problem()
    _, g = M.loss_grad(p, x, t, wt, H, round_weights=False)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (M.loss_grad(p + e, x, t, wt, H, False)[0] - M.loss_grad(p - e, x, t, wt, H, False)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_gradient_against_autograd():
    p, x, t, wt, H = _problem(seed=5)
    L, g = M.loss_grad(p, x, t, wt, H, round_weights=False)
    pt = torch.tensor(p, requires_grad=True)
    o = 0
    parts = []
    for shape in ((H, 8), (H,), (H, H), (H,), (H,), (1,)):
        k = int(np.prod(shape))
        parts.append(pt[o:o + k].reshape(shape))
        o += k
    W1, b1, W2, b2, W3, b3 = parts
    xt = torch.tensor(x)
    y = torch.tanh(torch.tanh(xt @ W1.T + b1) @ W2.T + b2) @ W3 + b3
    Lt = (torch.tensor(wt) * (y - torch.tensor(t)) ** 2).sum()
    Lt.backward()
    assert abs(Lt.item() - L) < 1e-14
    np.testing.assert_allclose(g, pt.grad.numpy(), rtol=1e-12, atol=1e-15)


def test_rounded_gradient_is_the_straight_through_one():
    """With rounded weights the gradient is that of the float64 network at
    the rounded weights, applied to the unrounded master values."""
    p, x, t, wt, H = _problem(seed=6)
    W1, b1, W2, b2, W3, b3 = M.unpack(p, 8, H)
    pr = np.concatenate([M.bf16_round(W1).ravel(), b1, M.bf16_round(W2).ravel(), b2, M.bf16_round(W3), b3])
    La, ga = M.loss_grad(p, x, t, wt, H, round_weights=True)
    Lb, gb = M.loss_grad(pr, x, t, wt, H, round_weights=False)
    assert La == Lb
    np.testing.assert_array_equal(ga, gb)


# -------------------------------------------------------------------- Adam
def test_adam_first_step_closed_form():
    rng = np.random.default_rng(7)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    q, m, v = M.adam_step(p, np.zeros(50), np.zeros(50), g, 1, lr=0.01, eps=1e-8)
    np.testing.assert_allclose(q, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-13)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-13)


def test_adam_converges_on_a_convex_quadratic():
    a = np.array([1.0, 10.0, 0.1])
    c = np.array([0.3, -2.0, 5.0])
    p = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    for k in range(1, 5001):
        p, m, v = M.adam_step(p, m, v, 2 * a * (p - c), k, lr=0.05 * (1 - k / 5001) + 1e-4)
    np.testing.assert_allclose(p, c, atol=1e-3)


def test_training_fits_a_teacher_network():
    rng = np.random.default_rng(8)
    x = M.bf16_round(rng.uniform(-1, 1, size=(400, 8)))
    teacher = rng.normal(size=M.n_params(8, 8)) * 0.8
    t = M.forward(teacher, x, H=8)[0]
    wt = np.full(400, 1 / 400)
    p, losses = M.train(W.mlp_init(9, 8, 8), x, t, wt, 600, 1e-2, H=8)
    assert losses[-1] < 3e-2 * losses[0] and np.all(np.isfinite(p))


def test_zero_network_warm_start_is_the_superposition_start():
    rng = np.random.default_rng(10)
    s = rng.uniform(0.1, 1.0, size=300)
    w = rng.uniform(0.5, 1.5, size=300)
    x = rng.normal(size=(300, 8))
    psi = M.warm_start(np.zeros(M.n_params()), x, s, w)
    np.testing.assert_allclose(psi, s / np.sqrt(np.sum(s * s * w)), rtol=1e-14)
    assert abs(np.sum(psi * psi * w) - 1.0) < 1e-14
