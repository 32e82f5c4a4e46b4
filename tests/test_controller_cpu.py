"""Host logic of the learned parameter controller: structural features, labels, the fallback
rule and the versioned checkpoint (no GPU)."""
import numpy as np
import pytest

import synth
from paper_2105_07544_b300 import controller as C


def test_matrix_features_of_the_laplacian_have_closed_forms():
    N = 20
    A = synth.laplace2d(N)
    f = C.matrix_features(A)
    assert f[0] == pytest.approx(np.log10(N * N))
    assert f[1] == pytest.approx((5 * N * N - 4 * N) / (N * N))       # mean nnz per row
    assert f[2] == 5
    assert f[3] == pytest.approx(1.0)          # interior rows: |4| / (4 x |-1|)
    assert f[4] == 0.0                          # symmetric
    assert f[5] == pytest.approx(-12.0)         # no convection
    assert f[6] == pytest.approx(0.0) and f[7] == pytest.approx(2.0)   # Gershgorin / diagonal


def test_matrix_features_see_convection():
    A = synth.convdiff2d(30, 0.3, peclet=300.0)
    f = C.matrix_features(A)
    assert f[4] > 0.05
    h = 1.0 / 31
    beta = h * 300.0
    diag = 4 + beta * (abs(np.cos(0.3)) + abs(np.sin(0.3)))
    # the largest |a_ij - a_ji| is beta x the larger wind component
    assert 10 ** f[5] == pytest.approx(beta * max(abs(np.cos(0.3)), abs(np.sin(0.3))) / diag,
                                       rel=1e-9)


def _result(times, default_time):
    configs = C.grid_configs()
    return C.SweepResult(configs, np.asarray(times, float), np.zeros(len(configs)), default_time)


def test_labels_pick_the_fastest_setting():
    T = np.full(61, np.inf)
    T[0] = 1.0
    k = C.grid_configs().index((100, 1e-3, 25))
    T[k] = 0.25
    mc, tl, dc, rt = C.labels(_result(T, 1.0))
    assert (mc, dc) == (2, 2)
    assert tl == pytest.approx(-3.0)
    assert rt == pytest.approx(np.log(0.25))


def test_labels_when_the_default_wins_or_nothing_converges():
    T = np.full(61, 2.0)
    T[0] = 1.0
    assert C.labels(_result(T, 1.0)) == (1, C.LOG_TOL_FULL, 0, 0.0)
    assert C.labels(_result(np.full(61, np.inf), np.inf))[:1] == (-1,)
    T = np.full(61, np.inf)
    T[5] = 0.1
    assert C.labels(_result(T, np.inf))[3] == C.RATIO_FLOOR


def test_suggest_falls_back_unless_a_gain_is_predicted(monkeypatch):
    c = C.Controller(params=np.zeros(5577, np.float32), mean=np.zeros(12), std=np.ones(12))
    y = np.zeros((1, 9))
    y[0, 2] = 5.0            # m = 100
    y[0, 3] = -3.5           # inner tol 10^-3.5
    y[0, 7] = 5.0            # d = 40
    y[0, 8] = np.log(0.99)   # not enough predicted gain
    monkeypatch.setattr(c, "predict", lambda X: y)
    assert c.suggest(np.zeros(12)) == C.DEFAULT + (True,)
    y[0, 8] = np.log(0.5)
    m, tol, d, fb = c.suggest(np.zeros(12))
    assert (m, d, fb) == (100, 40, False) and tol == pytest.approx(10 ** -3.5)
    y[0, 3] = 3.0            # out of range: clipped to the grid's ends
    assert c.suggest(np.zeros(12))[1] == pytest.approx(1e-2)


def test_checkpoint_round_trip_and_corruption(tmp_path):
    rng = np.random.default_rng(0)
    c = C.Controller(params=rng.normal(size=5577).astype(np.float32), mean=rng.normal(size=12),
                     std=rng.uniform(1, 2, 12))
    p = tmp_path / "c.bin"
    c.save(p)
    d = C.Controller.load(p)
    np.testing.assert_array_equal(d.params, c.params)
    np.testing.assert_array_equal(d.mean, c.mean)
    np.testing.assert_array_equal(d.std, c.std)
    raw = bytearray(p.read_bytes())
    raw[100] ^= 1
    p.write_bytes(bytes(raw))
    with pytest.raises(ValueError, match="CRC"):
        C.Controller.load(p)
    p.write_bytes(b"NOTACKPT" + bytes(raw[8:]))
    with pytest.raises(ValueError, match="not a controller"):
        C.Controller.load(p)


def test_checkpoint_version_is_checked(tmp_path, monkeypatch):
    c = C.Controller(params=np.zeros(5577, np.float32), mean=np.zeros(12), std=np.ones(12))
    monkeypatch.setattr(C, "VERSION", 99)
    c.save(tmp_path / "v.bin")
    monkeypatch.setattr(C, "VERSION", 1)
    with pytest.raises(ValueError, match="version"):
        C.Controller.load(tmp_path / "v.bin")


def test_dataset_labels_match_per_system_labels():
    rng = np.random.default_rng(3)
    T = rng.uniform(0.1, 1.0, (5, 61))
    T[2, 10:] = np.inf
    data = dict(T=T, configs=np.array(C.grid_configs(), dtype=np.float64))
    mc, tl, dc, rt = C.dataset_labels(data)
    for i in range(5):
        e = C.labels(_result(T[i], T[i, 0]))
        assert (mc[i], dc[i]) == (e[0], e[2])
        assert tl[i] == pytest.approx(e[1]) and rt[i] == pytest.approx(e[3], abs=1e-6)


def test_data_sets_combine_and_untimed_settings_never_label(tmp_path):
    """Two generated files (one from before the pruned grid, without a `tried` mask) combine
    system by system; a setting that was not run keeps time inf, so it is never a label."""
    cfg = np.array(C.grid_configs(), dtype=np.float64)
    rng = np.random.default_rng(5)
    T1 = rng.uniform(0.1, 1.0, (3, 61))
    np.savez(tmp_path / "a.npz", idx=np.arange(3), n=np.full(3, 100), X=rng.normal(size=(3, 12)),
             T=T1, IT=np.ones((3, 61), np.int64), configs=cfg)
    tried = np.array([True] + [c in set(C.PRUNED_GRID) for c in C.grid_configs()[1:]])
    assert tried.sum() == 31 and len(C.PRUNED_GRID) == 30
    T2 = np.where(tried, rng.uniform(0.5, 1.0, (2, 61)), np.inf)
    T2[:, 1] = np.inf                      # make an untried setting the "fastest" if it had run
    np.savez(tmp_path / "b.npz", idx=np.arange(20, 22), n=np.full(2, 400),
             X=rng.normal(size=(2, 12)), T=T2, IT=np.ones((2, 61), np.int64),
             tried=np.tile(tried, (2, 1)), configs=cfg)
    d = C.load_datasets([tmp_path / "a.npz", tmp_path / "b.npz"])
    assert d["X"].shape == (5, 12) and list(d["idx"]) == [0, 1, 2, 20, 21]
    assert d["tried"][:3].all() and (d["tried"][3:] == tried).all()
    mc, tl, dc, rt = C.dataset_labels(d)
    for i in (3, 4):
        k = int(np.argmin(d["T"][i]))
        assert tried[k]
        m, tol, deg = C.grid_configs()[k]
        assert (C.M_CLASSES[mc[i]], C.D_CLASSES[dc[i]]) == (m, deg)
    np.savez(tmp_path / "c.npz", **{**dict(np.load(tmp_path / "b.npz")), "configs": cfg[::-1]})
    with pytest.raises(ValueError, match="grids"):
        C.load_datasets([tmp_path / "a.npz", tmp_path / "c.npz"])


def test_evaluation_summary_counts_unconverged_references_apart():
    """A reference solve that did not converge (time inf) is counted, not divided by."""
    from paper_2105_07544_b300 import controller as c
    inf = float("inf")
    rows = [dict(t_ctrl=1.0, t_default=4.0, t_fixed=2.0, res_ctrl=1e-11, fallback=False, guard=False),
            dict(t_ctrl=2.0, t_default=inf, t_fixed=1.0, res_ctrl=1e-11, fallback=False, guard=False),
            dict(t_ctrl=3.0, t_default=6.0, t_fixed=inf, res_ctrl=2e-10, fallback=True, guard=False)]
    s = c.summarize(rows, (25, 1e-6, 25))
    assert s["systems"] == 3 and s["converged"] == 2 and s["fallbacks"] == 1
    vd = s["vs_default"]
    assert vd["systems"] == 2 and vd["reference_not_converged"] == 1
    assert vd["median"] == 0.375 and abs(vd["total"] - 0.4) < 1e-15
    assert abs(vd["geomean"] - (0.25 * 0.5) ** 0.5) < 1e-15
    vf = s["vs_fixed"]
    assert vf["systems"] == 2 and vf["median"] == 1.25 and vf["reference_not_converged"] == 1


def test_suggest_prefers_the_best_fixed_setting_unless_the_network_predicts_more(monkeypatch):
    c = C.Controller(params=np.zeros(5577, np.float32), mean=np.zeros(12), std=np.ones(12),
                     fixed=(25, 1e-6, 25), fixed_ratio=0.2)
    y = np.zeros((1, 9))
    y[0, 1] = 5.0            # m = 50
    y[0, 6] = 5.0            # d = 25
    y[0, 3] = -2.0
    monkeypatch.setattr(c, "predict", lambda X: y)
    y[0, 8] = np.log(0.99)                     # no gain at all: the default
    assert c.suggest(np.zeros(12)) == C.DEFAULT + (True,)
    y[0, 8] = np.log(0.25)                     # a gain, but not beyond the fixed setting's 0.2/0.95
    assert c.suggest(np.zeros(12)) == (25, 1e-6, 25, True)
    y[0, 8] = np.log(0.1)                      # clearly beyond it: the network's choice
    assert c.suggest(np.zeros(12)) == (50, 1e-2, 25, False)


def test_checkpoint_v2_carries_the_fixed_setting_and_v1_still_loads(tmp_path):
    import struct
    import zlib
    rng = np.random.default_rng(1)
    c = C.Controller(params=rng.normal(size=5577).astype(np.float32), mean=rng.normal(size=12),
                     std=rng.uniform(1, 2, 12), fixed=(25, 1e-6, 25), fixed_ratio=0.1387)
    c.save(tmp_path / "v2.bin")
    d = C.Controller.load(tmp_path / "v2.bin")
    assert d.fixed == (25, 1e-6, 25) and d.fixed_ratio == 0.1387
    body = struct.pack("<II", 1, 5577) + c.mean.astype("<f8").tobytes() + \
        c.std.astype("<f8").tobytes() + c.params.astype("<f4").tobytes()
    (tmp_path / "v1.bin").write_bytes(b"GMRESMLP" + body + struct.pack("<I", zlib.crc32(body)))
    e = C.Controller.load(tmp_path / "v1.bin")
    assert e.fixed is None and np.array_equal(e.params, c.params)


def test_native_checkpoint_reader_rejects_bad_files(tmp_path):
    """The C ABI's reader checks magic, size, version and CRC before touching the GPU."""
    import ctypes
    import paper_2105_07544_b300 as g
    lib = g.load()
    c = C.Controller(params=np.zeros(5577, np.float32), mean=np.zeros(12), std=np.ones(12),
                     fixed=(25, 1e-6, 25), fixed_ratio=0.2)
    p = tmp_path / "c.bin"
    c.save(p)
    raw = p.read_bytes()
    h = ctypes.c_void_p()
    cases = {"missing": None, "crc": bytearray(raw), "magic": b"NOTACKPT" + raw[8:],
             "short": raw[:-9], "long": raw + b"\0"}
    cases["crc"][300] ^= 4
    for name, data in cases.items():
        q = tmp_path / f"{name}.bin"
        if data is not None:
            q.write_bytes(bytes(data))
        assert lib.gmres_controller_load(str(q).encode(), ctypes.byref(h)) == -1, name
    # a valid file passes the checks; creating the network then needs the GPU
    rc = lib.gmres_controller_load(str(p).encode(), ctypes.byref(h))
    assert rc in (0, -3)
    if rc == 0:
        lib.gmres_controller_destroy(h)
