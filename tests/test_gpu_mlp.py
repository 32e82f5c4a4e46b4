"""Controller network kernels against the FP64 oracle network (forward, gradient, Adam step)."""
import numpy as np
import pytest

from oracle import mlp as omlp
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _batch(B, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, 12)).astype(np.float32)
    mc = rng.integers(-1, 3, B).astype(np.int32)        # some -1: no label
    tl = rng.uniform(-6, -2, B).astype(np.float32)
    dc = rng.integers(0, 5, B).astype(np.int32)         # some 4: out of range, no label
    rt = rng.normal(size=B).astype(np.float32)
    return X, mc, tl, dc, rt


def _dev(*arrs):
    import torch
    return [torch.from_numpy(a).cuda() for a in arrs]


@pytest.mark.parametrize("B", [1, 127, 300])
def test_forward_matches_oracle(B):
    need_gpu()
    from paper_2105_07544_b300 import MLP
    p = MLP.init_params(3)
    p[-9:] = np.linspace(-0.5, 0.5, 9)                  # non-zero output biases
    X = _batch(B, B)[0]
    net = MLP(p)
    y_dev = net.forward(_dev(X)[0]).cpu().numpy()
    y_host = net.forward(X)
    net.close()
    y_ref, _ = omlp.forward(p.astype(np.float64), X.astype(np.float64))
    scale = np.abs(y_ref).max()
    assert np.abs(y_dev - y_ref).max() <= 1e-5 * scale
    np.testing.assert_array_equal(y_dev, y_host)


@pytest.mark.parametrize("B", [5, 300])
def test_gradient_matches_oracle_and_is_deterministic(B):
    need_gpu()
    from paper_2105_07544_b300 import MLP
    p = MLP.init_params(7)
    X, mc, tl, dc, rt = _batch(B, 100 + B)
    net = MLP(p)
    g1, l1 = net.gradient(*_dev(X, mc, tl, dc, rt))
    g2, l2 = net.gradient(*_dev(X, mc, tl, dc, rt))
    net.close()
    np.testing.assert_array_equal(g1, g2)
    lref, gref = omlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), mc, tl, dc, rt)
    np.testing.assert_allclose(l1, lref, rtol=1e-5, atol=1e-6)
    # per block of parameters: error relative to that block's largest entry
    off = 0
    for name, shape in omlp.SHAPES:
        k = int(np.prod(shape))
        ref = gref[off:off + k]
        assert np.abs(g1[off:off + k] - ref).max() <= 1e-4 * max(np.abs(ref).max(), 1e-6), name
        off += k


def test_adam_step_matches_oracle_update():
    need_gpu()
    from paper_2105_07544_b300 import MLP
    p = MLP.init_params(11).astype(np.float32)
    X, mc, tl, dc, rt = _batch(64, 5)
    net = MLP(p)
    lr = 1e-3
    net.train_step(*_dev(X, mc, tl, dc, rt), lr=lr)
    p1 = net.params()
    net.close()
    _, g = omlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), mc, tl, dc, rt)
    # first Adam step (bias-corrected): p - lr * g / (|g| + eps)
    expect = p - lr * g / (np.abs(g) + 1e-8)
    big = np.abs(g) > 1e-3 * np.abs(g).max()       # where the step is lr * sign(g) robustly
    np.testing.assert_allclose(p1[big], expect[big], rtol=0, atol=1e-6)


def test_training_reduces_loss():
    need_gpu()
    from paper_2105_07544_b300 import MLP
    rng = np.random.default_rng(0)
    X = rng.normal(size=(512, 12)).astype(np.float32)
    mc = (X[:, 0] > 0).astype(np.int32) + (X[:, 1] > 1).astype(np.int32)
    tl = (-4 + X[:, 2]).astype(np.float32)
    dc = np.clip((X[:, 3] + 2).astype(np.int32), 0, 3).astype(np.int32)
    rt = (0.3 * X[:, 4] - 0.2).astype(np.float32)
    net = MLP(MLP.init_params(0))
    args = _dev(X, mc, tl, dc, rt)
    first = net.train_step(*args, lr=3e-3).sum()
    for _ in range(400):
        last = net.train_step(*args, lr=3e-3).sum()
    net.close()
    assert last < 0.25 * first


def test_invalid_arguments():
    need_gpu()
    from paper_2105_07544_b300 import MLP, GmresError
    with pytest.raises(ValueError):
        MLP(np.zeros(10, np.float32))
    net = MLP(MLP.init_params(0))
    X, mc, tl, dc, rt = _batch(4, 0)
    with pytest.raises(GmresError):
        net.train_step(*_dev(X, mc, tl, dc, rt), lr=-1.0)
    net.close()
