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
MAGIC = b"GMRESMLP"
VERSION = 1


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


def features(A, b, device="cuda") -> np.ndarray:
    """The 12 features of a system (GPU work: a 10-step FP64 Arnoldi run and one IR cycle)."""
    import torch
    f8 = matrix_features(A)
    s = Solver(A, m=DEFAULT[0])
    bd = torch.from_numpy(np.asarray(b, np.float64)).to(device)
    H, _, steps = s.arnoldi(bd, min(10, A.n - 1) if A.n > 1 else 1, "f64", want_basis=False)
    k = max(1, steps)
    ev = hessenberg_eigvals(H[:k, :k])
    dscale = np.mean(np.abs(A.val[A.colidx == np.repeat(np.arange(A.n), np.diff(A.rowptr))])) or 1.0
    s.set_params(maxiter=DEFAULT[0])
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
               solver=None):
    """Time one GMRES-IR solve with the given parameters: (seconds or inf, iterations, x).

    One cycle runs first (it captures the cycle's CUDA graph); the timed solve starts from zero.
    """
    import torch
    own = solver is None
    s = solver or Solver(A, m=max(M_CLASSES), poly_degree=d, poly_start=start)
    bd = torch.from_numpy(np.asarray(b, np.float64)).to(device)
    s.set_params(m=m, inner_tol=tol, maxiter=m, time_limit_s=0.0)
    s.ir_solve(bd, tol=1e-10)
    s.set_params(maxiter=maxiter, time_limit_s=float(time_limit))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, st = s.ir_solve(bd, tol=1e-10)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    if own:
        s.close()
    return (el if st.converged else np.inf), st.iters, x


def sweep(A, b, start, maxiter=20000) -> SweepResult:
    """Time the default and all 60 grid settings on one system."""
    solvers = {d: Solver(A, m=max(M_CLASSES), poly_degree=d, poly_start=start) for d in D_CLASSES}
    try:
        t_def, it_def, _ = run_config(A, b, *DEFAULT, start, maxiter, solver=solvers[0])
        limit = CUTOFF * t_def if np.isfinite(t_def) else 0.0
        configs, times, iters = [DEFAULT], [t_def], [it_def]
        for d in D_CLASSES:
            for m in M_CLASSES:
                for tol in TOL_GRID:
                    t, it, _ = run_config(A, b, m, tol, d, start, maxiter, limit, solver=solvers[d])
                    configs.append((m, tol, d))
                    times.append(t)
                    iters.append(it)
    finally:
        for s in solvers.values():
            s.close()
    return SweepResult(configs, np.array(times), np.array(iters), t_def)


def labels(res: SweepResult):
    """(m class, log10 tol target, d class, log time ratio) of the fastest converged setting."""
    (m, tol, d), t = res.best()
    ratio = np.log(t / res.default_time) if np.isfinite(res.default_time) and np.isfinite(t) else 0.0
    return M_CLASSES.index(m), _tol_target(tol), D_CLASSES.index(d), float(ratio)


@dataclass
class Controller:
    params: np.ndarray
    mean: np.ndarray
    std: np.ndarray
    history: list = field(default_factory=list)

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
        """(m, inner tol, degree, used_fallback) for one system's features."""
        y = self.predict(feats)[0]
        if y[8] >= np.log(FALLBACK_RATIO):
            return DEFAULT + (True,)
        m = M_CLASSES[int(np.argmax(y[0:3]))]
        d = D_CLASSES[int(np.argmax(y[4:8]))]
        return m, _tol_from_output(y[3]), d, False

    def solve(self, A, b, start, maxiter=5000):
        """Controller-chosen GMRES-IR solve with the runtime guard (stagnation -> defaults)."""
        m, tol, d, fb = self.suggest(features(A, b))
        t, it, x = run_config(A, b, m, tol, d, start, maxiter)
        if not np.isfinite(t):
            m, tol, d = DEFAULT
            t, it, x = run_config(A, b, m, tol, d, start, maxiter)
            fb = True
        return x, dict(m=m, tol=tol, d=d, fallback=fb, time=t, iters=it)

    # ---- checkpoint ------------------------------------------------------------------------
    def save(self, path):
        body = struct.pack("<II", VERSION, self.params.size) + \
            np.asarray(self.mean, "<f8").tobytes() + np.asarray(self.std, "<f8").tobytes() + \
            np.asarray(self.params, "<f4").tobytes()
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
        if ver != VERSION:
            raise ValueError(f"checkpoint version {ver} not supported")
        mean = np.frombuffer(body[8:8 + 96], "<f8").copy()
        std = np.frombuffer(body[104:104 + 96], "<f8").copy()
        params = np.frombuffer(body[200:200 + 4 * npar], "<f4").copy()
        return cls(params=params, mean=mean, std=std)
