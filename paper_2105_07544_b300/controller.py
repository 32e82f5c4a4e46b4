"""Learned GMRES-IR parameter controller.

The paper chooses the restart length (Section V-E), the inner tolerance and the polynomial
degree (Section V-F) by hand.  This module proposes them per system with a small MLP whose
forward, backward and Adam steps run in the library's own CUDA kernels (``MLP``):

* ``features``: 12 cheap numbers per system -- size and sparsity, diagonal dominance,
  nonsymmetry, an upwind-strength estimate, Gershgorin bounds, the extreme Ritz values of a
  10-step FP64 Arnoldi run (the library's kernels) and the residual drop and wall time of one
  GMRES-IR cycle with the default parameters;
* ``sweep``: the solver itself times GMRES-IR over the grid m in {25, 50, 100} x inner tolerance
  in {1e-6, ..., 1e-2} x degree in {0, 10, 25, 40} (60 settings) plus the default on a system;
  the fastest setting that converges is the label.  Settings are cut off at a multiple of the
  default's time (they cannot be the fastest past that point);
* ``Controller``: the trained network with the feature standardisation, ``suggest`` (with a
  fallback to the defaults whenever the network does not predict a gain), ``solve`` (with a
  runtime guard: a stagnating run is redone with the defaults), and a versioned checkpoint with a
  CRC32.
"""
from __future__ import annotations

import struct
import time
import zlib
from dataclasses import dataclass, field

import numpy as np

from . import MLP, Solver, hessenberg_eigvals

M_CLASSES = (25, 50, 100)
D_CLASSES = (0, 10, 25, 40)
TOL_GRID = (1e-6, 1e-5, 1e-4, 1e-3, 1e-2)
DEFAULT = (50, 0.0, 0)                 # (m, inner tol, degree): full inner cycles, no polynomial
LOG_TOL_FULL = -6.0                    # regression target standing for "full cycles"
FALLBACK_RATIO = 0.95
CUTOFF = 2.0                           # sweep settings stop at CUTOFF x the default's time
GUARD_CYCLES = 10                      # runtime guard: cycles without progress before reverting
MAGIC = b"GMRESMLP"
VERSION = 2                            # 2 adds the best fixed setting of the training sweep


def _tol_target(tol: float) -> float:
    return LOG_TOL_FULL if tol <= 0 else float(np.log10(tol))


def _tol_from_output(y: float) -> float:
    return 10.0 ** float(np.clip(y, -6.0, -2.0))


def matrix_features(A) -> np.ndarray:
    """Host-side structural features of a CSR matrix (8 of the 12)."""
    n = A.n
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    cnt = np.diff(A.rowptr)
    diag = np.zeros(n)
    isd = A.colidx == rows
    diag[rows[isd]] = A.val[isd]
    off = np.zeros(n)
    np.add.at(off, rows[~isd], np.abs(A.val[~isd]))
    dscale = np.mean(np.abs(diag)) or 1.0
    dom = np.min(np.abs(diag) / np.maximum(off, 1e-300))
    # nonsymmetry and upwind strength from the transposed pattern (same pattern for stencils)
    import scipy.sparse as sp
    M = sp.csr_matrix((A.val, A.colidx, A.rowptr), shape=(n, n))
    D = M - M.T
    nonsym = sp.linalg.norm(D) / max(sp.linalg.norm(M), 1e-300)
    pe = np.max(np.abs(D.data)) / dscale if D.nnz else 0.0
    gmin = np.min(diag - off) / dscale
    gmax = np.max(diag + off) / dscale
    return np.array([np.log10(n), cnt.mean(), cnt.max(), dom, nonsym, np.log10(pe + 1e-12),
                     gmin, gmax], dtype=np.float64)


def _dscale(A) -> float:
    """Mean |a_ii| over the n rows (a missing diagonal entry counts as 0), or 1 if that is 0."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    diag = np.zeros(A.n)
    np.add.at(diag, rows[A.colidx == rows], A.val[A.colidx == rows])
    return float(np.mean(np.abs(diag))) or 1.0


def features(A, b, device="cuda") -> np.ndarray:
    """The 12 features of a system (GPU work: a 10-step FP64 Arnoldi run and one IR cycle).
    The library computes the same features natively: ``native_features``."""
    import torch
    f8 = matrix_features(A)
    s = Solver(A, m=DEFAULT[0])
    bd = torch.from_numpy(np.asarray(b, np.float64)).to(device)
    H, _, steps = s.arnoldi(bd, min(10, A.n - 1) if A.n > 1 else 1, "f64", want_basis=False)
    k = max(1, steps)
    ev = hessenberg_eigvals(H[:k, :k])
    dscale = _dscale(A)
    s.set_params(maxiter=DEFAULT[0])
    s.ir_solve(bd, tol=1e-10)                 # captures the cycle graph
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st = s.ir_solve(bd, tol=1e-10)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    h = st.history
    drop = h[1] / h[0] if len(h) > 1 and h[0] > 0 else 1.0
    s.close()
    return np.concatenate([f8, [np.max(np.abs(ev)) / dscale, np.min(np.abs(ev)) / dscale,
                                np.log10(max(drop, 1e-30)), np.log10(max(el, 1e-6))]])


@dataclass
class SweepResult:
    configs: list                 # (m, tol, d)
    times: np.ndarray             # seconds (inf when not converged)
    iters: np.ndarray
    default_time: float

    def best(self):
        i = int(np.argmin(self.times))
        return self.configs[i], self.times[i]


def run_config(A, b, m, tol, d, start, maxiter=20000, time_limit=0.0, device="cuda",
               solver=None, stagnation_cycles=0):
    """Time one GMRES-IR solve with the given parameters: (seconds or inf, iterations, x).

    One cycle runs first (it captures the cycle's CUDA graph); the timed solve starts from zero.
    A solve that does not converge (iteration cap, time limit, stagnation) times as inf.
    """
    import torch
    own = solver is None
    s = solver or Solver(A, m=max(M_CLASSES), poly_degree=d, poly_start=start)
    bd = torch.from_numpy(np.asarray(b, np.float64)).to(device)
    s.set_params(m=m, inner_tol=tol, maxiter=m, time_limit_s=0.0)
    s.ir_solve(bd, tol=1e-10)
    s.set_params(maxiter=maxiter, time_limit_s=float(time_limit),
                 stagnation_cycles=stagnation_cycles)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, st = s.ir_solve(bd, tol=1e-10)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    if own:
        s.close()
    return (el if st.converged else np.inf), st.iters, x


def grid_configs():
    """The default followed by the 60 grid settings, in the order of a sweep's time arrays."""
    return [DEFAULT] + [(m, t, d) for d in D_CLASSES for m in M_CLASSES for t in TOL_GRID]


def sweep(A, b, start, maxiter=20000, grid=None, best_factor=4.0) -> SweepResult:
    """Time the default and the grid settings on one system (all 60, or those in ``grid``).

    A setting is cut off (time inf) once it runs past min(CUTOFF x default, best_factor x best
    so far): it cannot be the fastest.  Polynomial degrees that usually win are tried first so
    the bound tightens early.  Settings outside ``grid`` are not run and keep time inf.
    """
    configs = grid_configs()
    times = np.full(len(configs), np.inf)
    iters = np.zeros(len(configs), dtype=np.int64)
    todo = set(configs[1:]) if grid is None else set(grid)
    degrees = sorted({0} | {d for (_, _, d) in todo})
    solvers = {d: Solver(A, m=max(M_CLASSES), poly_degree=d, poly_start=start) for d in degrees}
    try:
        t_def, iters[0], _ = run_config(A, b, *DEFAULT, start, maxiter, solver=solvers[0])
        times[0] = t_def
        best = t_def
        for d in (10, 25, 40, 0):
            for m in M_CLASSES:
                for tol in TOL_GRID:
                    if (m, tol, d) not in todo:
                        continue
                    limit = min(CUTOFF * t_def, best_factor * best) if np.isfinite(best) else 0.0
                    k = configs.index((m, tol, d))
                    times[k], iters[k], _ = run_config(A, b, m, tol, d, start, maxiter, limit,
                                                       solver=solvers[d])
                    best = min(best, times[k])
    finally:
        for s in solvers.values():
            s.close()
    return SweepResult(configs, times, iters, t_def)


# Settings timed on the systems of the workload's sizes (sides 500-2000): on the 418-system sweep
# at sides 128-512, no setting without the polynomial was ever the fastest, and m = 100 was the
# fastest on 2 systems (within 10 % of the fastest on 6); they are left out there (time inf) so
# that a sweep costs half as much.
PRUNED_GRID = tuple((m, t, d) for d in (10, 25, 40) for m in (25, 50) for t in TOL_GRID)

# A further reduction for the larger sweeps at sides 500-2000: every other inner tolerance.  On the
# 81 systems swept over PRUNED_GRID, the five tolerances of a degree-10, m = 25 setting were all
# within 10 % of the fastest on the same 36 systems, so neighbouring tolerances rarely decide.
REDUCED_GRID = tuple((m, t, d) for d in (10, 25, 40) for m in (25, 50) for t in (1e-5, 1e-3, 1e-2))


RATIO_FLOOR = -5.0        # log time-ratio label when only the default failed to converge


def labels(res: SweepResult):
    """(m class, log10 tol target, d class, log time ratio) of the fastest converged setting.

    A system on which nothing converged gets class labels -1 (no cross-entropy term) and ratio 0.
    """
    (m, tol, d), t = res.best()
    if not np.isfinite(t):
        return -1, LOG_TOL_FULL, -1, 0.0
    if not np.isfinite(res.default_time):
        ratio = RATIO_FLOOR
    else:
        ratio = max(RATIO_FLOOR, float(np.log(t / res.default_time)))
    return M_CLASSES.index(m), _tol_target(tol), D_CLASSES.index(d), ratio


@dataclass
class Controller:
    params: np.ndarray
    mean: np.ndarray
    std: np.ndarray
    history: list = field(default_factory=list)
    fixed: tuple | None = None          # best fixed (m, tol, d) of the training sweep
    fixed_ratio: float = 0.0            # its median time ratio against the default there

    # ---- training -------------------------------------------------------------------------
    @classmethod
    def train(cls, X, mc, tl, dc, rt, steps=1500, lr=3e-3, seed=0):
        import torch
        X = np.asarray(X, np.float64)
        mean = X.mean(0)
        std = X.std(0) + 1e-6
        Xs = torch.tensor((X - mean) / std, dtype=torch.float32, device="cuda")
        lab = [torch.tensor(np.asarray(v), dtype=t, device="cuda")
               for v, t in ((mc, torch.int32), (tl, torch.float32), (dc, torch.int32),
                            (rt, torch.float32))]
        net = MLP(MLP.init_params(seed))
        hist = []
        for i in range(steps):
            loss = net.train_step(Xs, *lab, lr=lr)
            if i % 100 == 0 or i == steps - 1:
                hist.append((i, loss.tolist()))
        c = cls(params=net.params(), mean=mean, std=std, history=hist)
        net.close()
        return c

    # ---- inference ------------------------------------------------------------------------
    def predict(self, X):
        import torch
        X = np.atleast_2d(np.asarray(X, np.float64))
        net = MLP(self.params)
        Y = net.forward(torch.tensor((X - self.mean) / self.std, dtype=torch.float32,
                                     device="cuda")).cpu().numpy()
        net.close()
        return Y

    def suggest(self, feats):
        """(m, inner tol, degree, used_fallback) for one system's features.

        The network predicts (output 8) the log of the best achievable time over the default's.
        No predicted gain (ratio >= 0.95): the default.  With a best fixed setting known: when the
        predicted gain is not beyond that setting's median gain on the training systems (ratio
        >= its ratio / 0.95), that setting.  Otherwise the network's choice."""
        y = self.predict(feats)[0]
        if y[8] >= np.log(FALLBACK_RATIO):
            return DEFAULT + (True,)
        if self.fixed is not None and self.fixed_ratio > 0 and \
                y[8] >= np.log(self.fixed_ratio / FALLBACK_RATIO):
            return tuple(self.fixed) + (True,)
        m = M_CLASSES[int(np.argmax(y[0:3]))]
        d = D_CLASSES[int(np.argmax(y[4:8]))]
        return m, _tol_from_output(y[3]), d, False

    def solve(self, A, b, start, maxiter=20000, guard_maxiter=200000):
        """Controller-chosen GMRES-IR solve with the runtime guard: a suggested run that stagnates
        (GUARD_CYCLES cycles without a 10 % residual drop) or reaches ``maxiter`` is redone with
        the default parameters and ``guard_maxiter``."""
        m, tol, d, fb = self.suggest(features(A, b))
        t, it, x = run_config(A, b, m, tol, d, start, maxiter, stagnation_cycles=GUARD_CYCLES)
        if not np.isfinite(t):
            m, tol, d = DEFAULT
            t, it, x = run_config(A, b, m, tol, d, start, guard_maxiter)
            fb = True
        return x, dict(m=m, tol=tol, d=d, fallback=fb, time=t, iters=it)

    # ---- checkpoint ------------------------------------------------------------------------
    def save(self, path):
        m, tol, d = self.fixed if self.fixed is not None else (0, 0.0, 0)
        body = struct.pack("<II", VERSION, self.params.size) + \
            np.asarray(self.mean, "<f8").tobytes() + np.asarray(self.std, "<f8").tobytes() + \
            np.asarray(self.params, "<f4").tobytes() + \
            struct.pack("<idid", int(m), float(tol), int(d), float(self.fixed_ratio))
        with open(path, "wb") as f:
            f.write(MAGIC + body + struct.pack("<I", zlib.crc32(body)))

    @classmethod
    def load(cls, path):
        raw = open(path, "rb").read()
        if raw[:8] != MAGIC:
            raise ValueError("not a controller checkpoint")
        body, crc = raw[8:-4], struct.unpack("<I", raw[-4:])[0]
        if zlib.crc32(body) != crc:
            raise ValueError("checkpoint CRC mismatch")
        ver, npar = struct.unpack("<II", body[:8])
        if ver not in (1, 2):
            raise ValueError(f"checkpoint version {ver} not supported")
        mean = np.frombuffer(body[8:8 + 96], "<f8").copy()
        std = np.frombuffer(body[104:104 + 96], "<f8").copy()
        params = np.frombuffer(body[200:200 + 4 * npar], "<f4").copy()
        fixed, ratio = None, 0.0
        if ver == 2:
            m, tol, d, ratio = struct.unpack("<idid", body[200 + 4 * npar:200 + 4 * npar + 24])
            if m > 0 and ratio > 0:
                fixed = (int(m), float(tol), int(d))
        return cls(params=params, mean=mean, std=std, fixed=fixed, fixed_ratio=float(ratio))


# ---- data set, training and evaluation driver ---------------------------------------------------
HELDOUT0 = 50_000          # held-out systems use indices HELDOUT0, HELDOUT0 + 1, ...


def generate(indices, side_lo, side_hi, budget_s=0.0, out=None, log=print, grid=None,
             best_factor=4.0):
    """Features and sweep times of the controller systems with the given indices.

    Returns a dict of arrays: idx, n, X (features), T (times of the default and the 60 settings;
    inf where a setting did not converge, was cut off or, with ``grid``, was not run), IT
    (iterations), tried (which settings ran), configs.  Stops early (keeping finished systems)
    once ``budget_s`` seconds have passed; with ``out`` the data set is rewritten after every
    system.
    """
    import synth
    t0 = time.perf_counter()
    rows = []
    data = None
    configs = grid_configs()
    tried = np.array([True] + [grid is None or c in set(grid) for c in configs[1:]])
    for i in indices:
        if budget_s and time.perf_counter() - t0 > budget_s:
            break
        ts = time.perf_counter()
        A, b, start = synth.workload_controller(i, side_lo, side_hi)
        f = features(A, b)
        r = sweep(A, b, start, grid=grid, best_factor=best_factor)
        (cfg, tb) = r.best()
        log(f"{A.name:28s} n={A.n:7d} default {r.default_time * 1e3:8.1f} ms  best {cfg} "
            f"{tb * 1e3:8.1f} ms  (system {time.perf_counter() - ts:5.1f} s)", flush=True)
        rows.append((i, A.n, f, r.times, r.iters))
        data = dict(idx=np.array([r[0] for r in rows]), n=np.array([r[1] for r in rows]),
                    X=np.array([r[2] for r in rows]), T=np.array([r[3] for r in rows]),
                    IT=np.array([r[4] for r in rows]),
                    tried=np.tile(tried, (len(rows), 1)),
                    configs=np.array(configs, dtype=np.float64),
                    side_lo=side_lo, side_hi=side_hi)
        if out:
            np.savez_compressed(out, **data)
    return data


def load_datasets(paths):
    """One data set from several generated files (same settings grid), systems concatenated."""
    parts = [dict(np.load(p)) for p in paths]
    out = dict(configs=parts[0]["configs"])
    for p in parts[1:]:
        if not np.array_equal(p["configs"], out["configs"]):
            raise ValueError("data sets with different settings grids")
    for k in ("idx", "n", "X", "T", "IT"):
        out[k] = np.concatenate([p[k] for p in parts])
    out["tried"] = np.concatenate([p["tried"] if "tried" in p else np.ones_like(p["T"], bool)
                                   for p in parts])
    return out


def dataset_labels(data):
    """Labels of every system of a generated data set (see ``labels``)."""
    configs = [tuple(c) for c in data["configs"]]
    configs = [(int(m), float(t), int(d)) for m, t, d in configs]
    out = []
    for T in data["T"]:
        res = SweepResult(configs, T, np.zeros(len(T)), T[0])
        out.append(labels(res))
    mc, tl, dc, rt = (np.array(v) for v in zip(*out))
    return mc.astype(np.int32), tl.astype(np.float32), dc.astype(np.int32), rt.astype(np.float32)


def best_fixed_setting(data):
    """The single grid setting with the smallest median time ratio against the default over a
    data set (a non-learned baseline for the controller)."""
    T = np.asarray(data["T"])
    ok = np.isfinite(T[:, 0])
    R = T[ok] / T[ok, :1]
    med = np.median(np.where(np.isfinite(R), R, 1e9), axis=0)
    k = int(np.argmin(med[1:])) + 1
    return grid_configs()[k], float(med[k])


def fp64_relres(A, b, x):
    """||b - A x|| / ||b|| in FP64 on the host (scipy), what decides convergence."""
    import scipy.sparse as sp
    M = sp.csr_matrix((A.val, A.colidx, A.rowptr), shape=(A.n, A.n))
    x = x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
    return float(np.linalg.norm(b - M @ x) / np.linalg.norm(b))


def evaluate(ctrl, indices, side_lo, side_hi, fixed=None, log=print, budget_s=0.0):
    """Held-out evaluation: per system the controller's solve (features, suggestion, runtime
    guard) against the default, and against one fixed setting if given.  Times exclude the
    polynomial build; the controller's features are timed apart (``t_feat``).  Stops early
    (keeping the finished systems) once ``budget_s`` seconds have passed."""
    import synth
    rows = []
    t00 = time.perf_counter()
    for i in indices:
        if budget_s and time.perf_counter() - t00 > budget_s:
            break
        A, b, start = synth.workload_controller(i, side_lo, side_hi)
        t0 = time.perf_counter()
        f = features(A, b)
        t_feat = time.perf_counter() - t0
        m, tol, d, fb = ctrl.suggest(f)
        t_c, it_c, x_c = run_config(A, b, m, tol, d, start, stagnation_cycles=GUARD_CYCLES)
        guard = not np.isfinite(t_c)
        if guard:
            t_c, it_c, x_c = run_config(A, b, *DEFAULT, start, 200000)
        t_d, it_d, x_d = run_config(A, b, *DEFAULT, start)
        row = dict(idx=int(i), n=int(A.n), m=m, tol=tol, d=d, fallback=bool(fb), guard=bool(guard),
                   t_ctrl=t_c, t_feat=t_feat, t_default=t_d, it_ctrl=int(it_c),
                   it_default=int(it_d), res_ctrl=fp64_relres(A, b, x_c),
                   res_default=fp64_relres(A, b, x_d))
        if fixed is not None:
            row["t_fixed"] = run_config(A, b, *fixed, start)[0]
        rows.append(row)
        log(f"{A.name:28s} ({m:3d},{tol:.0e},{d:2d}){' fb' if fb else ''}{' guard' if guard else ''}"
            f"  ctrl {t_c * 1e3:8.1f} ms  default {t_d * 1e3:8.1f} ms  ratio {t_c / t_d:6.3f}"
            f"  res {row['res_ctrl']:.1e}", flush=True)
    return rows


def feature_cost(ckpt, indices, side_lo, side_hi, log=print):
    """Seconds per system for the features through the C ABI (``gmres_controller_features``
    and ``gmres_controller_suggest`` on a handle of the system, after one warm call) and through
    the Python driver (``features``)."""
    import torch
    import synth
    from . import NativeController
    nat = NativeController(str(ckpt))
    rows = []
    try:
        for i in indices:
            A, b, _ = synth.workload_controller(i, side_lo, side_hi)
            s = Solver(A, m=DEFAULT[0])
            bd = torch.from_numpy(b).cuda()
            nat.features(s, bd)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            nat.features(s, bd)
            torch.cuda.synchronize()
            t_nat = time.perf_counter() - t0
            t0 = time.perf_counter()
            sg = nat.suggest(s, bd)
            torch.cuda.synchronize()
            t_sug = time.perf_counter() - t0
            t0 = time.perf_counter()
            features(A, b)
            t_py = time.perf_counter() - t0
            s.close()
            rows.append(dict(idx=int(i), n=int(A.n), native_features_s=t_nat,
                             native_suggest_s=t_sug, python_features_s=t_py,
                             choice=sg["choice"]))
            log(f"{A.name:28s} n={A.n:7d}  C ABI {t_nat * 1e3:7.1f} ms  suggest {t_sug * 1e3:7.1f} ms"
                f"  Python {t_py * 1e3:7.1f} ms", flush=True)
    finally:
        nat.close()
    return rows


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="learned GMRES-IR parameter controller")
    sub = ap.add_subparsers(dest="cmd", required=True)
    g = sub.add_parser("gen", help="sweep systems and save features and times (.npz)")
    g.add_argument("--first", type=int, default=0)
    g.add_argument("--count", type=int, default=100)
    g.add_argument("--side-lo", type=int, default=128)
    g.add_argument("--side-hi", type=int, default=512)
    g.add_argument("--budget", type=float, default=0.0, help="seconds; 0 = no limit")
    g.add_argument("--grid", choices=["full", "pruned", "reduced"], default="full",
                   help="time all 60 settings, the 30 of PRUNED_GRID or the 18 of REDUCED_GRID")
    g.add_argument("--best-factor", type=float, default=4.0,
                   help="cut a setting off past this multiple of the best time so far")
    g.add_argument("--out", required=True)
    t = sub.add_parser("train", help="train on a data set and save a checkpoint")
    t.add_argument("--data", required=True, nargs="+", help="one or more generated data sets")
    t.add_argument("--steps", type=int, default=3000)
    t.add_argument("--out", required=True)
    e = sub.add_parser("eval", help="held-out evaluation against the default (JSON)")
    e.add_argument("--ckpt", required=True)
    e.add_argument("--data", nargs="+",
                   help="training data set(s): also time their best fixed setting")
    e.add_argument("--first", type=int, default=HELDOUT0)
    e.add_argument("--count", type=int, default=40)
    e.add_argument("--side-lo", type=int, default=128)
    e.add_argument("--side-hi", type=int, default=512)
    e.add_argument("--budget", type=float, default=0.0, help="seconds; 0 = no limit")
    e.add_argument("--out", required=True)
    c = sub.add_parser("cost", help="time the features: C ABI and Python driver (JSON)")
    c.add_argument("--ckpt", required=True)
    c.add_argument("--first", type=int, default=HELDOUT0)
    c.add_argument("--count", type=int, default=12)
    c.add_argument("--side-lo", type=int, default=128)
    c.add_argument("--side-hi", type=int, default=512)
    c.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    if a.cmd == "cost":
        import json
        rows = feature_cost(a.ckpt, range(a.first, a.first + a.count), a.side_lo, a.side_hi)
        with open(a.out, "w") as f:
            json.dump(rows, f, indent=1)
        return
    if a.cmd == "gen":
        generate(range(a.first, a.first + a.count), a.side_lo, a.side_hi, a.budget, a.out,
                 grid={"full": None, "pruned": PRUNED_GRID, "reduced": REDUCED_GRID}[a.grid],
                 best_factor=a.best_factor)
    elif a.cmd == "train":
        d = load_datasets(a.data)
        c = Controller.train(d["X"], *dataset_labels(d), steps=a.steps)
        c.fixed, c.fixed_ratio = best_fixed_setting(d)
        c.save(a.out)
        print("losses (step, [CE m, tol MSE, CE d, ratio MSE]):", c.history[0], c.history[-1])
    else:
        import json
        ctrl = Controller.load(a.ckpt)
        fixed = best_fixed_setting(load_datasets(a.data))[0] if a.data else None
        rows = evaluate(ctrl, range(a.first, a.first + a.count), a.side_lo, a.side_hi, fixed,
                        budget_s=a.budget)
        print(json.dumps(summarize(rows, fixed)))
        with open(a.out, "w") as f:
            json.dump(dict(summary=summarize(rows, fixed), systems=rows), f, indent=1)


def summarize(rows, fixed=None):
    """Ratios of the controller's solve time to the default's (and the fixed setting's), over
    the systems where the reference solve converged; the others are counted separately."""
    def ratios(key):
        both = [x for x in rows if np.isfinite(x[key]) and np.isfinite(x["t_ctrl"])]
        r = np.array([x["t_ctrl"] / x[key] for x in both])
        if not len(r):
            return dict(systems=0)
        return dict(systems=len(both), median=float(np.median(r)),
                    geomean=float(np.exp(np.mean(np.log(r)))),
                    total=float(sum(x["t_ctrl"] for x in both) / sum(x[key] for x in both)),
                    reference_not_converged=int(sum(not np.isfinite(x[key]) for x in rows)))
    return dict(systems=len(rows),
                converged=int(sum(x["res_ctrl"] <= 1e-10 for x in rows)),
                fallbacks=int(sum(x["fallback"] for x in rows)),
                guards=int(sum(x["guard"] for x in rows)),
                vs_default=ratios("t_default"),
                fixed_setting=list(fixed) if fixed else None,
                vs_fixed=ratios("t_fixed") if fixed else None)


if __name__ == "__main__":
    main()
