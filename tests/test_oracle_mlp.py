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


# ------------------------------------------------- the tensor-core form (H = 64)
def _bf16_torch(a):
    """bfloat16 rounding by torch's own cast (float64 -> float32 is exact for
    these values' 8 significant bits only after rounding, so cast the float64
    value directly to bfloat16)."""
    return a.to(torch.bfloat16).to(torch.float64)


def test_tensor_core_form_against_autograd_with_straight_through_rounding():
    """forward_tc and loss_grad_tc against torch: the same network written
    with torch's bfloat16 cast at each rounding point, differentiated by
    autograd with the rounding passed straight through (x + (round(x) - x)
    detached)."""
    rng = np.random.default_rng(11)
    H, n = 64, 500
    p = rng.normal(size=M.n_params(8, H)) * 0.3
    x = M.bf16_round(rng.normal(size=(n, 8)))
    t = rng.normal(size=n) * 0.2
    wt = rng.uniform(0.5, 1.5, size=n)
    L, g = M.loss_grad_tc(p, x, t, wt, H)
    y, _ = M.forward_tc(p, x, H)
    pt = torch.tensor(p, requires_grad=True)
    o, parts = 0, []
    for shape in ((H, 8), (H,), (H, H), (H,), (H,), (1,)):
        k = int(np.prod(shape))
        parts.append(pt[o:o + k].reshape(shape))
        o += k
    W1, b1, W2, b2, W3, b3 = parts
    st = lambda a: a + (_bf16_torch(a) - a).detach()  # rounded value, identity gradient
    xt = torch.tensor(x)
    h1 = torch.tanh(xt @ st(W1).T + b1)
    h2 = torch.tanh(st(h1) @ st(W2).T + b2)
    yt = h2 @ st(W3) + b3
    np.testing.assert_allclose(yt.detach().numpy(), y, rtol=1e-13, atol=1e-15)
    # the backward pass with its own rounding points, written out by hand
    r = yt.detach() - torch.tensor(t)
    dy = 2 * torch.tensor(wt) * r
    W2r, W3r = _bf16_torch(W2.detach()), _bf16_torch(W3.detach())
    dz2b = _bf16_torch(dy[:, None] * W3r[None, :] * (1 - h2.detach() ** 2))
    dz1b = _bf16_torch((dz2b @ W2r) * (1 - h1.detach() ** 2))
    g_ref = torch.cat([(dz1b.T @ xt).ravel(), dz1b.sum(0), (dz2b.T @ _bf16_torch(h1.detach())).ravel(), dz2b.sum(0),
                       _bf16_torch(dy) @ _bf16_torch(h2.detach()), _bf16_torch(dy).sum()[None]])
    # torch's tanh and NumPy's can differ in the last bit, which now and then
    # moves a value across a bfloat16 rounding boundary: a rare entry
    # differs by about one bfloat16 unit of one term, every other agrees to
    # rounding (a misplaced rounding point would move most entries)
    gr = g_ref.numpy()
    d = np.abs(g - gr) / np.maximum(np.abs(gr), 1e-300)
    assert np.mean(d > 1e-10) < 5e-3 and d.max() < 1e-2, (np.mean(d > 1e-10), d.max())
    # and close to the exact gradient of the rounded-input network: the
    # rounding points change it by about 2^-8 relative
    Lt = (torch.tensor(wt) * (yt - torch.tensor(t)) ** 2).sum()
    Lt.backward()
    assert abs(Lt.item() - L) < 1e-12 * L
    rel = np.linalg.norm(g - pt.grad.numpy()) / np.linalg.norm(pt.grad.numpy())
    assert 1e-5 < rel < 2e-2, rel


def test_tensor_core_form_is_the_exact_form_when_rounding_is_exact():
    """With every activation and gradient value already a bfloat16 number
    the two forms coincide: a network with W1 = 0 (h1 = tanh(b1), chosen on
    bfloat16 values of tanh), W3 = 0 and b1, b2 set so that h1 is exact."""
    H, n = 64, 40
    rng = np.random.default_rng(3)
    p = np.zeros(M.n_params(8, H))
    W1, b1, W2, b2, W3, b3 = M.unpack(p, 8, H)
    h1_target = M.bf16_round(rng.uniform(-0.5, 0.5, size=H))
    b1[:] = np.arctanh(h1_target)
    W2[:] = M.bf16_round(rng.normal(size=(H, H)) * 0.1)
    b3[:] = 0.25
    x = M.bf16_round(rng.normal(size=(n, 8)))
    h1 = np.tanh(b1)
    assert np.max(np.abs(M.bf16_round(h1) - h1)) < 1e-15  # h1 is a bfloat16 number
    y_tc, _ = M.forward_tc(p, x, H)
    y_ex, _ = M.forward(p, x, H)
    np.testing.assert_allclose(y_tc, y_ex, rtol=0, atol=1e-15)


def test_ordered_features_follow_the_list_order():
    """List-order features of a heteronuclear pair: the same values as the
    sorted ones where the point is nearer the first nucleus, and r1, r2
    exchanged where it is nearer the second (so e^-r1 and e^-r2, tanh r1 and
    tanh r2 swap and (r2 - r1)/R changes sign); R and the symmetric features
    agree."""
    nuc = np.array([[-1.0, 0.0, 0.0], [1.2, 0.0, 0.0]])
    xyz = np.array([[-1.5, 0.3, 0.2], [2.0, -0.4, 0.1], [-1.0, 0.0, 0.0]]).T
    fo = M.features(xyz, nuc, ordered=True)
    fs = M.features(xyz, nuc)
    np.testing.assert_array_equal(fo[0], fs[0])            # nearer the first nucleus
    np.testing.assert_array_equal(fo[1, [1, 0, 3, 2]], fs[1, [0, 1, 2, 3]])
    assert fo[1, 4] == -fs[1, 4]
    np.testing.assert_array_equal(fo[1, 5:], fs[1, 5:])
    assert fo[2, 0] == 1.0 and fo[2, 2] == 0.0              # on the first nucleus: r1 = 0
    with pytest.raises(ValueError):
        M.features(xyz, np.zeros((3, 3)) + np.arange(3)[:, None], ordered=True)


def test_scaled_features_closed_forms():
    """Decay rates per nucleus: the first two features become e^-(z1 r1) and
    e^-(z2 r2) for the rates of the nuclei at r1 and r2, in closed form at
    the second nucleus and on the bond axis; rates of 1 give the plain
    features bit for bit; the other six features do not change."""
    R = 2.1
    nuc = np.array([[-R / 2, 0, 0], [R / 2, 0, 0]])
    z = np.array([5.7, 7.7])
    b = M.bf16_round
    pts = np.array([[R / 2, 0, 0], [-R / 2 - 0.3, 0, 0], [0.1, 0.4, -0.2]]).T
    f = M.features(pts, nuc, ordered=True, scale=z)
    assert f[0, 0] == b(math.exp(-z[0] * R)) and f[0, 1] == 1.0   # on the second nucleus: r2 = 0
    assert f[1, 0] == b(math.exp(-z[0] * 0.3)) and f[1, 1] == b(math.exp(-z[1] * (R + 0.3)))
    plain = M.features(pts, nuc, ordered=True)
    np.testing.assert_array_equal(f[:, 2:], plain[:, 2:])
    np.testing.assert_array_equal(M.features(pts, nuc, scale=[1.0, 1.0]), M.features(pts, nuc))
    # nearest-pair order: the rate follows the nucleus, not the slot
    s = M.features(pts, nuc, scale=z)
    assert s[0, 0] == 1.0 and s[0, 1] == b(math.exp(-z[0] * R))
    with pytest.raises(ValueError):
        M.features(pts, nuc, scale=[1.0, 0.0])
