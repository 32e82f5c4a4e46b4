"""Pins of the controller-network oracle (no GPU): the analytic gradient against central finite
differences in FP64, and closed-form special cases of the loss."""
import numpy as np

from oracle import mlp as om


def _batch(seed, B=16):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, om.NPARAMS)
    X = rng.normal(0, 1, (B, 12))
    mc = rng.integers(-1, 3, B)
    dc = rng.integers(-1, 4, B)
    tl = rng.uniform(-6, -2, B)
    rt = rng.normal(0, 0.3, B)
    return p, X, mc, tl, dc, rt


def test_gradient_matches_central_differences():
    p, X, mc, tl, dc, rt = _batch(0)
    _, g = om.loss_and_grad(p, X, mc, tl, dc, rt)
    rng = np.random.default_rng(1)
    idx = rng.choice(om.NPARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (om.loss_and_grad(pp, X, mc, tl, dc, rt)[0].sum() -
              om.loss_and_grad(pm, X, mc, tl, dc, rt)[0].sum()) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd))


def test_uniform_logits_give_log_class_count():
    """Zero last layer: every logit 0, so CE = log(#classes) and the regression outputs are 0."""
    p, X, mc, tl, dc, rt = _batch(2)
    w3 = om.unpack(p)
    off = om.NPARAMS - (9 * 64 + 9)
    p[off:] = 0.0
    mc[:] = 1
    dc[:] = 3
    losses, _ = om.loss_and_grad(p, X, mc, tl, dc, rt)
    assert np.isclose(losses[0], np.log(3)) and np.isclose(losses[2], np.log(4))
    assert np.isclose(losses[1], np.mean(tl ** 2)) and np.isclose(losses[3], np.mean(rt ** 2))


def test_missing_labels_drop_their_terms():
    p, X, mc, tl, dc, rt = _batch(3)
    mc[:] = -1
    dc[:] = -1
    losses, g = om.loss_and_grad(p, X, mc, tl, dc, rt)
    assert losses[0] == 0 and losses[2] == 0
    y, _ = om.forward(p, X)
    # the only gradient through the head rows 0..2 and 4..7 is zero
    gW3 = g[om.NPARAMS - (9 * 64 + 9): om.NPARAMS - 9].reshape(9, 64)
    assert np.all(gW3[[0, 1, 2, 4, 5, 6, 7]] == 0)
