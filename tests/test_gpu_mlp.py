"""GPU warm-start network vs the FP64 oracle (oracle/mlp_oracle.py).

The library multiplies BF16 weights and BF16 activations with FP32 accumulation; the oracle runs
in FP64 on the same BF16-rounded weights. Each BF16 rounding of an activation or a gradient is
relative 2^-9; through five products the relative L2 error stays below a few 1e-3 (tolerances
2e-2 outputs, 3e-2 gradients). Adam runs in FP32 on both sides' own inputs: 1e-5.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu

WARM = [5, 512, 512, 512, 512, 768]   # the warm-start network
RAGGED = [7, 100, 33, 70]             # sizes off every tile boundary


@pytest.fixture(scope="module")
def N():
    import __graft_entry__ as g
    g.build()
    from paper_1608_04601_gb300 import mlp
    return mlp


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("sizes,batch", [(WARM, 256), (WARM, 1), (RAGGED, 37), (RAGGED, 64)])
def test_forward_matches_oracle(N, sizes, batch):
    rng = np.random.default_rng(11)
    net = N.MLP(sizes, max_batch=max(batch, 64), seed=7)
    p = M.weights_bf16(net.get_params(), sizes)
    x = rng.standard_normal((batch, sizes[0])).astype(np.float32)
    y = net.forward(x).cpu().numpy()
    ref = M.forward(p, sizes, x)[-1]
    assert y.shape == ref.shape
    assert _rel(y, ref) < 2e-2
    net.close()


def test_initial_weights_are_glorot_uniform(N):
    net = N.MLP(WARM, max_batch=8, seed=3)
    p = net.get_params()
    for (w, b, i, o) in M.layout(WARM)[0]:
        a = np.sqrt(6.0 / (i + o))
        W = p[w:w + i * o]
        assert np.all(np.abs(W) <= a) and abs(np.mean(W)) < 0.05 * a
        assert abs(np.var(W) / (a * a / 3) - 1) < 0.05          # uniform variance a^2/3
        assert np.all(p[b:b + o] == 0)
    net.close()


@pytest.mark.parametrize("sizes,batch", [(WARM, 256), (RAGGED, 37), (WARM, 37), ([16, 64, 40, 24], 200)])
def test_gradients_match_oracle(N, sizes, batch):
    rng = np.random.default_rng(12)
    net = N.MLP(sizes, max_batch=batch, seed=9)
    p0 = net.get_params()
    p0[M.layout(sizes)[0][-1][1]:] += 0.1 * rng.standard_normal(sizes[-1]).astype(np.float32)  # non-zero biases
    net.set_params(p0)
    p = M.weights_bf16(p0, sizes)
    x = rng.standard_normal((batch, sizes[0])).astype(np.float32)
    t = rng.standard_normal((batch, sizes[-1])).astype(np.float32)
    loss = net.loss_grad(x, t)
    g = net.grads()
    ref_loss, ref_g = M.loss_grad(p, sizes, x, t)
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss
    for (w, b, i, o) in M.layout(sizes)[0]:
        assert _rel(g[w:w + i * o], ref_g[w:w + i * o]) < 3e-2
        assert _rel(g[b:b + o], ref_g[b:b + o]) < 3e-2
    net.close()


def test_adam_step_matches_oracle(N):
    """One update from the library's own gradients: the FP32 Adam kernel against the oracle's step."""
    rng = np.random.default_rng(13)
    sizes = RAGGED
    net = N.MLP(sizes, max_batch=64, seed=5)
    x = rng.standard_normal((64, sizes[0])).astype(np.float32)
    t = rng.standard_normal((64, sizes[-1])).astype(np.float32)
    m = np.zeros(net.n_params)
    v = np.zeros(net.n_params)
    p = net.get_params().astype(np.float64)
    for step in (1, 2, 3):
        net.loss_grad(x, t)
        g = net.grads().astype(np.float64)
        net.adam(1e-3)
        p, m, v = M.adam(p, g, m, v, step, 1e-3)
        assert np.max(np.abs(net.get_params() - p)) <= 1e-5 * max(1.0, np.max(np.abs(p)))
    net.close()


def test_training_fits_smooth_profiles(N):
    """Property: Adam on the tensor-core products drives the loss of a smooth target family
    (three profile shapes over 256 points, parametrised by 5 inputs) down by two orders."""
    import torch
    rng = np.random.default_rng(14)
    B = 256
    x = rng.uniform(-1, 1, (B, 5)).astype(np.float32)
    s = np.linspace(0, 1, 256)
    amp = 1 + 0.5 * x[:, :1]
    t = np.concatenate([amp * np.sin(np.pi * s) ** 2, (amp + 0.2 * x[:, 1:2]) * np.sin(np.pi * s),
                        0.5 + 0.3 * x[:, 2:3] * np.cos(2 * np.pi * s)], axis=1).astype(np.float32)
    net = N.MLP(WARM, max_batch=B, seed=2)
    xd, td = torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda")
    first = net.train_step(xd, td, 1e-3)
    for _ in range(300):
        last = net.train_step(xd, td, 1e-3, sync=False)
    last = net.loss_grad(xd, td)
    assert last < 1e-2 * first
    net.close()


def test_rejects_batches_beyond_capacity(N):
    net = N.MLP(RAGGED, max_batch=8, seed=1)
    with pytest.raises(RuntimeError):
        net.forward(np.zeros((9, RAGGED[0]), np.float32))
    net.close()
