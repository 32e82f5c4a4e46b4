"""The learned parameter controller end to end on the GPU: training with the library's kernels
on the packaged sweep data set, then held-out systems solved with its suggestions against the
default parameters, convergence decided by the oracle's FP64 residual."""
import os

import numpy as np
import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

DATA = os.path.join(os.path.dirname(__file__), "..", "paper_2105_07544_b300", "data",
                    "controller_train.npz")


@pytest.fixture(scope="module")
def trained():
    need_gpu()
    from paper_2105_07544_b300 import controller as C
    d = dict(np.load(DATA))
    return C.Controller.train(d["X"], *C.dataset_labels(d), steps=1500)


def test_training_is_deterministic_and_lowers_the_loss(trained):
    from paper_2105_07544_b300 import controller as C
    d = dict(np.load(DATA))
    again = C.Controller.train(d["X"], *C.dataset_labels(d), steps=1500)
    np.testing.assert_array_equal(again.params, trained.params)
    first, last = np.sum(trained.history[0][1]), np.sum(trained.history[-1][1])
    assert last < 0.5 * first


def test_held_out_systems_converge_faster_than_with_the_default(trained, tmp_path):
    import synth
    from oracle.gmres import spmv
    from paper_2105_07544_b300 import controller as C
    path = tmp_path / "c.bin"
    trained.save(path)
    ctrl = C.Controller.load(path)
    rows = C.evaluate(ctrl, range(C.HELDOUT0, C.HELDOUT0 + 8), 128, 256, log=lambda *a, **k: None)
    for r in rows:
        A, b, _ = synth.workload_controller(r["idx"], 128, 256)
        assert r["res_ctrl"] <= 1e-10 and r["res_default"] <= 1e-10
    ratios = np.array([r["t_ctrl"] / r["t_default"] for r in rows])
    assert np.median(ratios) < 1.0
    # the deciding check itself: recompute one solution's residual with the oracle's FP64 SpMV
    A, b, start = synth.workload_controller(rows[0]["idx"], 128, 256)
    _, _, x = C.run_config(A, b, rows[0]["m"], rows[0]["tol"], rows[0]["d"], start)
    x = x.cpu().numpy()
    assert np.linalg.norm(b - spmv(A, x)) / np.linalg.norm(b) <= 1e-10


def test_runtime_guard_reverts_to_the_default(trained, monkeypatch):
    import synth
    from paper_2105_07544_b300 import controller as C
    # a suggestion that cannot converge within its iteration cap triggers the guard
    monkeypatch.setattr(trained, "suggest", lambda f: (25, 1e-2, 0, False))
    A, b, start = synth.workload_controller(C.HELDOUT0, 128, 256)
    x, info = trained.solve(A, b, start, maxiter=25)
    assert info["fallback"] and (info["m"], info["tol"], info["d"]) == C.DEFAULT
    assert np.isfinite(info["time"])
    assert C.fp64_relres(A, b, x) <= 1e-10


CKPT = os.path.join(os.path.dirname(__file__), "..", "paper_2105_07544_b300", "data",
                    "controller.ckpt")
# the packaged checkpoint is trained on the small systems above and on systems of sides 500-2000
DATA_LARGE = os.path.join(os.path.dirname(DATA), "controller_train_large.npz")


def test_native_decisions_equal_the_python_drivers_on_the_training_features():
    """Same checkpoint, same features: the C ABI's decision (FP32 forward pass in the library's
    MLP kernels, the fallback rule) equals the Python driver's, on all 836 training systems'
    features (every branch of the rule is taken)."""
    need_gpu()
    import paper_2105_07544_b300 as g
    from paper_2105_07544_b300 import controller as C
    d = C.load_datasets([DATA, DATA_LARGE])
    py = C.Controller.load(CKPT)
    nat = g.NativeController(CKPT)
    choices = set()
    Y = py.predict(d["X"])
    for f, y in zip(d["X"], Y):
        s = nat.decide(f)
        np.testing.assert_allclose(s["outputs"], y, rtol=1e-5, atol=1e-5)
        m, tol, dd, fb = py.suggest(f)
        assert (s["m"], s["d"]) == (m, dd) and s["tol"] == pytest.approx(tol, rel=1e-12)
        assert fb == (s["choice"] != "network")
        choices.add(s["choice"])
    assert "network" in choices
    nat.close()


@pytest.mark.parametrize("idx", [3, 17])
def test_native_features_match_the_python_driver(idx):
    """The library's own features of a system equal the Python driver's (host SciPy matrix
    features, the library's Arnoldi and cycle): the first eleven to rounding; the twelfth is a
    wall time measured separately by each."""
    need_gpu()
    import torch
    import paper_2105_07544_b300 as g
    import synth
    from paper_2105_07544_b300 import controller as C
    A, b, _ = synth.workload_controller(idx, 128, 256)
    fp = C.features(A, b)
    s = g.Solver(A, m=60, poly_degree=10, poly_start=synth.poly_start_vector(A.n, 0))
    nat = g.NativeController(CKPT)
    fn = nat.features(s, torch.from_numpy(b).cuda())
    np.testing.assert_allclose(fn[:11], fp[:11], rtol=1e-12, atol=1e-14)
    assert -6 < fn[11] < 1
    sug = nat.suggest(s, b)                         # host right-hand side
    np.testing.assert_allclose(sug["features"][:11], fp[:11], rtol=1e-12, atol=1e-14)
    again = nat.decide(sug["features"])
    assert (again["m"], again["tol"], again["d"], again["choice"]) == \
        (sug["m"], sug["tol"], sug["d"], sug["choice"])
    s.close()
    nat.close()
