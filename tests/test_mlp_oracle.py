"""Pins of the FP64 network oracle (CPU only): central finite differences, closed forms of
special cases, Adam's first step, and the bfloat16 format."""
import numpy as np

from oracle import mlp_oracle as M


def _params(rng, sizes, scale=1.0):
    n = M.layout(sizes)[1]
    return scale * rng.standard_normal(n)


def test_gradient_matches_central_differences():
    """Backward pass against (L(θ+h) - L(θ-h)) / 2h on every parameter of a small network
    (a dropped term, wrong sign or transposed product fails here)."""
    rng = np.random.default_rng(3)
    sizes = [4, 7, 6, 5]
    p = _params(rng, sizes, 0.5)
    x = rng.standard_normal((9, 4))
    t = rng.standard_normal((9, 5))
    _, g = M.loss_grad(p, sizes, x, t)
    h = 1e-6
    fd = np.zeros_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (M.loss_grad(p + e, sizes, x, t)[0] - M.loss_grad(p - e, sizes, x, t)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-6 * max(1.0, np.max(np.abs(g)))


def test_single_linear_layer_is_least_squares_gradient():
    """No hidden layer: y = x W^T + b and dL/dW = 2/n (y - t)^T x, dL/db = 2/n sum (y - t)."""
    rng = np.random.default_rng(4)
    sizes = [3, 2]
    p = _params(rng, sizes)
    x = rng.standard_normal((5, 3))
    t = rng.standard_normal((5, 2))
    W, b = p[:6].reshape(2, 3), p[6:]
    y = np.einsum("bi,oi->bo", x, W) + b
    loss, g = M.loss_grad(p, sizes, x, t)
    assert np.isclose(loss, np.mean((y - t) ** 2))
    r = 2 * (y - t) / y.size
    assert np.allclose(g[:6].reshape(2, 3), np.einsum("bo,bi->oi", r, x))
    assert np.allclose(g[6:], r.sum(0))


def test_hidden_tanh_layer_closed_form():
    """One tanh unit: y = v tanh(w x + c) + d; all four derivatives by hand."""
    sizes = [1, 1, 1]
    w, c, v, d = 0.7, -0.2, 1.3, 0.1
    p = np.array([w, c, v, d])
    x, t = np.array([[0.9]]), np.array([[0.4]])
    h = np.tanh(w * 0.9 + c)
    y = v * h + d
    loss, g = M.loss_grad(p, sizes, x, t)
    r = 2 * (y - 0.4)
    assert np.isclose(loss, (y - 0.4) ** 2)
    assert np.allclose(g, [r * v * (1 - h * h) * 0.9, r * v * (1 - h * h), r * h, r])


def test_adam_first_step_is_lr_times_sign():
    """From zero moments, bias correction makes the first step lr g / (|g| + eps)."""
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p, m, v = M.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-8)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_definition():
    """bfloat16 keeps 8 significant bits: exact values stay, ties go to the even neighbour,
    everything rounds to the nearer of its two neighbours."""
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -7)
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5, 1e-3, 65504.0], np.float32)
    r = M.bf16_round(vals)
    assert r[0] == one and r[1] == one                    # tie -> even (1.0)
    assert r[2] == np.float32(1.0 + 2 * ulp)              # tie between 1+ulp and 1+2ulp -> even (1+2ulp)
    assert r[3] == one and r[4] == np.float32(-2.5)
    rng = np.random.default_rng(5)
    a = rng.standard_normal(10000).astype(np.float32) * 10
    ra = M.bf16_round(a)
    assert np.all(ra.view(np.uint32) & 0xFFFF == 0)
    # the nearer neighbour: |a - r| <= half the bf16 spacing at a
    sp = 2.0 ** (np.floor(np.log2(np.abs(a))) - 7)
    assert np.all(np.abs(a.astype(np.float64) - ra) <= 0.5 * sp + 1e-30)


def test_only_weights_are_rounded_to_bf16():
    """The network keeps FP32 master parameters; its products see BF16 weights, while the biases
    enter the epilogue in FP32: weights_bf16 rounds exactly the weight slots of the flat layout."""
    sizes = [3, 5, 2]
    lay, n = M.layout(sizes)
    p = (1.0 + np.arange(n, dtype=np.float32) * np.float32(1e-3)).astype(np.float32)  # none exact in BF16
    q = M.weights_bf16(p, sizes)
    for (w, b, i, o) in lay:
        assert np.array_equal(q[b:b + o], p[b:b + o])
        W = q[w:w + i * o]
        assert np.all(W.view(np.uint32) & 0xFFFF == 0) and not np.array_equal(W, p[w:w + i * o])
        assert np.all(np.abs(W - p[w:w + i * o]) <= np.abs(p[w:w + i * o]) * 2.0 ** -8)
