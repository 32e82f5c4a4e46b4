"""gmresb3: multiprecision restarted GMRES (GMRES-IR) for one NVIDIA B300.

Thin ctypes binding of the C ABI in ``include/gmresb3.h`` (library ``_lib/libgmresb3.so``).
Every step of a solve runs in the library's CUDA kernels; this module only marshals arguments.
PyTorch tensors may be passed as device buffers (their stream is used); NumPy arrays are host
buffers.  There is no CPU fallback: if the library cannot be loaded, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

__all__ = ["Solver", "load", "GmresError", "F64", "F32", "BF16", "status_string"]

F64, F32, BF16 = 0, 1, 2
F16 = 3
_PREC = {"f64": F64, "f32": F32, "bf16": BF16, "f16": F16}

OK = 0
NOT_CONVERGED, NAN, LOSS_OF_ACCURACY, STAGNATION, TIMEOUT = 1, 2, 3, 4, 5


class CsrC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("colidx", ctypes.c_void_p), ("val", ctypes.c_void_p), ("on_device", ctypes.c_int)]


class PrecC(ctypes.Structure):
    _fields_ = [("matrix", ctypes.c_int), ("inner", ctypes.c_int), ("basis", ctypes.c_int),
                ("precond", ctypes.c_int)]


class ParamsC(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("maxiter", ctypes.c_int64), ("time_limit_s", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("use_graphs", ctypes.c_int),
                ("profiling", ctypes.c_int), ("stagnation_cycles", ctypes.c_int),
                ("max_loss_of_accuracy", ctypes.c_int), ("orth", ctypes.c_int)]


class TuningC(ctypes.Structure):
    _fields_ = [("sweep_stage_kb", ctypes.c_int), ("sweep_ctas_per_sm", ctypes.c_int),
                ("spmv_ctas_per_sm", ctypes.c_int), ("spmv_lanes_per_row", ctypes.c_int),
                ("cluster_cycle", ctypes.c_int)]


class BatchTuningC(ctypes.Structure):
    _fields_ = [("chunk_tiles", ctypes.c_int), ("sweep_smem_kb", ctypes.c_int),
                ("sweep_max_stages", ctypes.c_int), ("reserved", ctypes.c_int)]


class StatsC(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("cycles", ctypes.c_int64),
                ("rel_res_explicit", ctypes.c_double), ("rel_res_implicit", ctypes.c_double),
                ("status", ctypes.c_int), ("loss_of_accuracy", ctypes.c_int64),
                ("breakdowns", ctypes.c_int64), ("res_history", ctypes.c_void_p),
                ("res_history_cap", ctypes.c_int64), ("res_history_len", ctypes.c_int64),
                ("t_kernel", ctypes.c_double * 8), ("kernel_launches", ctypes.c_int64),
                ("solve_seconds", ctypes.c_double)]


KERNEL_CLASSES = ["spmv", "cgs_pass2", "cgs_update", "precond", "residual", "solution",
                  "cgs_proj", "other"]

# every symbol include/gmresb3.h declares, with its ctypes signature
_SIGS = {
    "gmres_default_params": (None, [ctypes.POINTER(ParamsC)]),
    "gmres_create": (ctypes.c_int, [ctypes.POINTER(CsrC), ctypes.c_int, ctypes.c_int, PrecC,
                                    ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "gmres_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "gmres_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gmres_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ParamsC)]),
    "gmres_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(TuningC)]),
    "gmres_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(TuningC)]),
    "gmres_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.POINTER(TuningC), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]),
    "gmres_ir_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_double, ctypes.POINTER(StatsC)]),
    "gmres_solve_fp64": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_double, ctypes.POINTER(StatsC)]),
    "gmres_solve_fp32": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_double, ctypes.POINTER(StatsC)]),
    "gmres_fd_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_double, ctypes.c_int64, ctypes.POINTER(StatsC),
                                      ctypes.POINTER(ctypes.c_int64)]),
    "gmres_set_block_jacobi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "gmres_block_jacobi_perm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "gmres_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gmres_spmv": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "gmres_precond_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "gmres_poly_roots": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "gmres_arnoldi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_int)]),
    "gmres_hessenberg_eigvals": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]),
    "gmres_precond_apply_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                                   ctypes.c_void_p]),
    "gmres_test_expire_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
}

class SuggestionC(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("inner_tol", ctypes.c_double), ("poly_degree", ctypes.c_int),
                ("choice", ctypes.c_int), ("predicted_ratio", ctypes.c_double),
                ("outputs", ctypes.c_double * 9), ("features", ctypes.c_double * 12)]


_SIGS.update({
    "gmres_controller_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]),
    "gmres_controller_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "gmres_controller_features": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gmres_controller_decide": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.POINTER(SuggestionC)]),
    "gmres_controller_suggest": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.POINTER(SuggestionC)]),
})


class BatchStatsC(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("cycles", ctypes.c_int64),
                ("block_steps", ctypes.c_int64), ("converged_systems", ctypes.c_int64),
                ("breakdowns", ctypes.c_int64), ("max_rel_res", ctypes.c_double),
                ("per_system_rel", ctypes.c_void_p), ("per_system_cycles", ctypes.c_void_p),
                ("per_system_cap", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("solve_seconds", ctypes.c_double), ("t_kernel", ctypes.c_double * 4),
                ("class_launches", ctypes.c_int64 * 4)]


BATCH_KERNEL_CLASSES = ["spmm", "sweep", "small", "cycle"]


_SIGS.update({
    "gmres_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                          PrecC, ctypes.POINTER(ctypes.c_void_p)]),
    "gmres_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "gmres_batch_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gmres_batch_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "gmres_batch_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BatchTuningC)]),
    "gmres_batch_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BatchTuningC)]),
    "gmres_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                            ctypes.c_int, ctypes.POINTER(BatchTuningC),
                                            ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]),
    "gmres_batch_ir_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_double, ctypes.c_int,
                                            ctypes.POINTER(BatchStatsC)]),
})

_SIGS.update({
    "gmres_mlp_num_params": (ctypes.c_int, []),
    "gmres_mlp_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "gmres_mlp_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "gmres_mlp_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "gmres_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_void_p]),
    "gmres_mlp_gradient": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 5 +
                           [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "gmres_mlp_train_step": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 5 +
                             [ctypes.c_int, ctypes.c_float, ctypes.c_void_p]),
})

_lib = None


def load(rebuild: bool = True) -> ctypes.CDLL:
    """Load (building first if stale) the CUDA library.  Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if rebuild else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"gmresb3 CUDA library missing: {path}")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().gmres_status_string(int(code)).decode()


class GmresError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {status_string(code)} ({code})")
        self.code = code


def _check(code: int, what: str) -> int:
    if code < 0:
        raise GmresError(code, what)
    return code


def _ptr(a) -> int:
    """Address of a contiguous torch tensor or NumPy array."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be contiguous")
    return a.ctypes.data


def _is_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


@dataclass
class SolveStats:
    status: int
    iters: int
    cycles: int
    rel_res: float
    rel_res_implicit: float
    loss_of_accuracy: int
    breakdowns: int
    kernel_launches: int
    solve_seconds: float
    t_kernel: dict = field(default_factory=dict)
    history: list = field(default_factory=list)

    @property
    def converged(self) -> bool:
        return self.status == OK


class Solver:
    """A handle on one matrix: GMRES-IR (FP32 inner, FP32 or BF16 basis) and FP64 GMRES.

    ``A`` has attributes ``n, rowptr, colidx, val`` (NumPy int32/int32/float64, host) or is a
    tuple of torch CUDA tensors ``(rowptr, colidx, val)``.  ``fp64_precond`` is the precision in
    which ``solve_fp64`` applies the polynomial ("f64", or "f32": variant (a) of Section III-D);
    GMRES-IR always applies it in FP32.
    """

    def __init__(self, A, m: int = 50, poly_degree: int = 0, basis: str = "f32",
                 poly_start=None, fp64_precond: str = "f64"):
        lib = load()
        self._lib = lib
        self.h = ctypes.c_void_p()
        if isinstance(A, tuple):
            rowptr, colidx, val = A
            n = rowptr.numel() - 1
            csr = CsrC(n, colidx.numel(), _ptr(rowptr), _ptr(colidx), _ptr(val), 1)
            self._keep = (rowptr, colidx, val)
        else:
            rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int32)
            colidx = np.ascontiguousarray(A.colidx, dtype=np.int32)
            val = np.ascontiguousarray(A.val, dtype=np.float64)
            n = int(A.n)
            csr = CsrC(n, int(rowptr[-1]), _ptr(rowptr), _ptr(colidx), _ptr(val), 0)
            self._keep = (rowptr, colidx, val)
        self.n = n
        self.m = m
        prec = PrecC(F32, F32, _PREC[basis], _PREC[fp64_precond])
        ps = None
        if poly_start is not None:
            ps = np.ascontiguousarray(poly_start, dtype=np.float64) if not _is_cuda(poly_start) \
                else poly_start
        _check(lib.gmres_create(ctypes.byref(csr), m, poly_degree, prec,
                                _ptr(ps) if ps is not None else None, ctypes.byref(self.h)),
               "gmres_create")
        self.params = ParamsC()
        lib.gmres_default_params(ctypes.byref(self.params))

    # ---- lifecycle ----
    def close(self):
        if self.h and self.h.value:
            self._lib.gmres_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, **kw):
        for k, v in kw.items():
            if not hasattr(self.params, k):
                raise KeyError(k)
            setattr(self.params, k, v)
        _check(self._lib.gmres_set_params(self.h, ctypes.byref(self.params)), "gmres_set_params")

    # ---- launch shapes ----
    TUNING_FIELDS = ("sweep_stage_kb", "sweep_ctas_per_sm", "spmv_ctas_per_sm", "spmv_lanes_per_row")

    def set_tuning(self, **kw):
        """Set launch shapes (see ``gmres_tuning_t``); unspecified fields keep their value."""
        t = TuningC()
        _check(self._lib.gmres_get_tuning(self.h, ctypes.byref(t)), "gmres_get_tuning")
        for k, v in kw.items():
            if k not in self.TUNING_FIELDS and k != "cluster_cycle":
                raise KeyError(k)
            setattr(t, k, int(v))
        _check(self._lib.gmres_set_tuning(self.h, ctypes.byref(t)), "gmres_set_tuning")

    def get_tuning(self) -> dict:
        t = TuningC()
        _check(self._lib.gmres_get_tuning(self.h, ctypes.byref(t)), "gmres_get_tuning")
        return {k: getattr(t, k) for k in self.TUNING_FIELDS}

    def autotune(self, b, cycles: int = 2):
        """Time GMRES-IR cycles under a grid of launch shapes and keep the fastest on this
        handle.  Returns (shapes, seconds per iteration chosen, seconds per iteration default)."""
        t = TuningC()
        tb, td = ctypes.c_double(), ctypes.c_double()
        self._stream(b)
        _check(self._lib.gmres_autotune(self.h, ctypes.c_void_p(_ptr(b)), int(cycles),
                                        ctypes.byref(t), ctypes.byref(tb), ctypes.byref(td)),
               "gmres_autotune")
        return {k: getattr(t, k) for k in self.TUNING_FIELDS}, tb.value, td.value

    def _stream(self, *tensors):
        import torch
        if any(_is_cuda(t) for t in tensors):
            _check(self._lib.gmres_set_stream(self.h, ctypes.c_void_p(
                torch.cuda.current_stream().cuda_stream)), "gmres_set_stream")

    # ---- solves ----
    def _solve(self, fn, b, x, tol, history_cap):
        if x is None:
            if _is_cuda(b):
                import torch
                x = torch.zeros_like(b)
            else:
                x = np.zeros(self.n)
        self._stream(b, x)
        hist = np.zeros(max(1, history_cap))
        st = StatsC()
        st.res_history = hist.ctypes.data
        st.res_history_cap = history_cap
        rc = fn(self.h, ctypes.c_void_p(_ptr(b)), ctypes.c_void_p(_ptr(x)), float(tol),
                ctypes.byref(st))
        _check(rc, "solve")
        s = SolveStats(status=rc, iters=st.iters, cycles=st.cycles, rel_res=st.rel_res_explicit,
                       rel_res_implicit=st.rel_res_implicit, loss_of_accuracy=st.loss_of_accuracy,
                       breakdowns=st.breakdowns, kernel_launches=st.kernel_launches,
                       solve_seconds=st.solve_seconds,
                       t_kernel={k: st.t_kernel[i] for i, k in enumerate(KERNEL_CLASSES)},
                       history=list(hist[: min(st.res_history_len, history_cap)]))
        return x, s

    def ir_solve(self, b, x=None, tol: float = 1e-10, history_cap: int = 4096):
        """GMRES-IR: returns (x, SolveStats).  ``x`` (if given) is the initial guess, updated in place."""
        return self._solve(self._lib.gmres_ir_solve, b, x, tol, history_cap)

    def solve_fp64(self, b, x=None, tol: float = 1e-10, history_cap: int = 4096):
        """Plain FP64 GMRES(m): returns (x, SolveStats)."""
        return self._solve(self._lib.gmres_solve_fp64, b, x, tol, history_cap)

    def solve_fp32(self, b, x=None, tol: float = 1e-6, history_cap: int = 4096):
        """Single-precision GMRES(m) (FP32 throughout): returns (x, SolveStats)."""
        return self._solve(self._lib.gmres_solve_fp32, b, x, tol, history_cap)

    def fd_solve(self, b, switch_iters: int, x=None, tol: float = 1e-10, history_cap: int = 4096):
        """GMRES-FD (Section III-C): FP32 GMRES for switch_iters iterations, then FP64 GMRES.
        Returns (x, SolveStats, iterations of the FP32 phase)."""
        k = ctypes.c_int64()
        fn = lambda h, bb, xx, t, st: self._lib.gmres_fd_solve(h, bb, xx, t, int(switch_iters), st,
                                                               ctypes.byref(k))
        x, st = self._solve(fn, b, x, tol, history_cap)
        return x, st, k.value

    # ---- building blocks (device tensors) ----
    def spmv(self, x, prec: str = "f64"):
        import torch
        y = torch.empty_like(x)
        self._stream(x)
        _check(self._lib.gmres_spmv(self.h, _PREC[prec], ctypes.c_void_p(_ptr(x)),
                                    ctypes.c_void_p(_ptr(y))), "gmres_spmv")
        return y

    def precond_apply(self, v, prec: str = "f64"):
        import torch
        z = torch.empty_like(v)
        self._stream(v)
        _check(self._lib.gmres_precond_apply(self.h, _PREC[prec], ctypes.c_void_p(_ptr(v)),
                                             ctypes.c_void_p(_ptr(z))), "gmres_precond_apply")
        return z

    def set_block_jacobi(self, block_size: int, reorder: bool = True):
        """Right-precondition later solves with block Jacobi (block_size 1..64, 0 removes it),
        blocks taken from the reverse Cuthill-McKee order when ``reorder``."""
        _check(self._lib.gmres_set_block_jacobi(self.h, int(block_size), int(bool(reorder))),
               "gmres_set_block_jacobi")

    def block_jacobi_perm(self) -> np.ndarray:
        p = np.zeros(self.n, dtype=np.int32)
        _check(self._lib.gmres_block_jacobi_perm(self.h, p.ctypes.data, self.n),
               "gmres_block_jacobi_perm")
        return p

    def poly_roots(self) -> np.ndarray:
        cnt = ctypes.c_int()
        re = np.zeros(256)
        im = np.zeros(256)
        _check(self._lib.gmres_poly_roots(self.h, re.ctypes.data, im.ctypes.data, 256,
                                          ctypes.byref(cnt)), "gmres_poly_roots")
        return re[: cnt.value] + 1j * im[: cnt.value]

    def arnoldi(self, r0, k: int, inner: str = "f64", want_basis: bool = True):
        """k Arnoldi steps from r0 (CUDA float64 tensor): returns (H (k+1) x k, V n x (k+1), steps)."""
        import torch
        H = np.zeros((k, k + 1))          # column-major (k+1) x k
        V = torch.zeros((k + 1, self.n), dtype=torch.float64, device=r0.device) if want_basis \
            else None
        steps = ctypes.c_int()
        self._stream(r0)
        _check(self._lib.gmres_arnoldi(self.h, _PREC[inner], k, ctypes.c_void_p(_ptr(r0)),
                                       H.ctypes.data,
                                       ctypes.c_void_p(_ptr(V)) if V is not None else None,
                                       ctypes.byref(steps)), "gmres_arnoldi")
        return H.T.copy(), (V.T if V is not None else None), steps.value


def hessenberg_eigvals(H: np.ndarray) -> np.ndarray:
    """Eigenvalues of a square upper Hessenberg matrix by the library's host QR routine."""
    lib = load()
    k = H.shape[0]
    Hc = np.asfortranarray(H, dtype=np.float64)
    re = np.zeros(k)
    im = np.zeros(k)
    _check(lib.gmres_hessenberg_eigvals(k, Hc.ctypes.data, re.ctypes.data, im.ctypes.data),
           "gmres_hessenberg_eigvals")
    return re + 1j * im


@dataclass
class BatchStats:
    status: int
    cycles: int
    block_steps: int
    converged_systems: int
    breakdowns: int
    max_rel_res: float
    per_system_rel: np.ndarray
    per_system_cycles: np.ndarray
    kernel_launches: int
    solve_seconds: float
    t_kernel: dict = field(default_factory=dict)
    class_launches: dict = field(default_factory=dict)

    @property
    def converged(self) -> bool:
        return self.status == OK


class BatchSolver:
    """Many independent systems with 8 right-hand sides each, solved together by block GMRES-IR
    (FP32 inner, BF16 basis, FP64 residual and update) on one GPU.

    ``systems`` is a list of CSR matrices (attributes n, rowptr, colidx, val).  Right-hand sides
    and solutions are passed as one array of all systems one after another, system s an
    n_s x 8 column-major block (``pack``/``unpack`` convert from and to lists of n_s x 8 arrays).
    """

    NRHS = 8

    def __init__(self, systems, m: int = 16):
        lib = load()
        self._lib = lib
        self.h = ctypes.c_void_p()
        self.sizes = [int(A.n) for A in systems]
        self._keep = []
        arr = (CsrC * len(systems))()
        for i, A in enumerate(systems):
            rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
            ci = np.ascontiguousarray(A.colidx, dtype=np.int32)
            va = np.ascontiguousarray(A.val, dtype=np.float64)
            self._keep += [rp, ci, va]
            arr[i] = CsrC(int(A.n), int(rp[-1]), _ptr(rp), _ptr(ci), _ptr(va), 0)
        _check(lib.gmres_batch_create(len(systems), ctypes.cast(arr, ctypes.c_void_p), self.NRHS, m,
                                      PrecC(F32, F32, BF16, F32), ctypes.byref(self.h)),
               "gmres_batch_create")
        self._keep = []

    def close(self):
        if self.h and self.h.value:
            self._lib.gmres_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pack(self, blocks):
        """List of n_s x 8 arrays -> one flat array (system after system, column-major)."""
        return np.concatenate([np.asarray(Bs, dtype=np.float64).T.ravel() for Bs in blocks])

    def unpack(self, flat):
        out, off = [], 0
        flat = flat.cpu().numpy() if hasattr(flat, "cpu") else np.asarray(flat)
        for n in self.sizes:
            out.append(flat[off: off + n * self.NRHS].reshape(self.NRHS, n).T.copy())
            off += n * self.NRHS
        return out

    def ir_solve(self, B, X=None, tol: float = 1e-10, max_cycles: int = 1000):
        """B: flat array (host NumPy or CUDA tensor).  Returns (X, BatchStats)."""
        if X is None:
            if _is_cuda(B):
                import torch
                X = torch.zeros_like(B)
            else:
                X = np.zeros_like(B)
        if _is_cuda(B):
            import torch
            _check(self._lib.gmres_batch_set_stream(self.h, ctypes.c_void_p(
                torch.cuda.current_stream().cuda_stream)), "gmres_batch_set_stream")
        nsys = len(self.sizes)
        rel = np.zeros(nsys)
        cyc = np.zeros(nsys, dtype=np.int64)
        st = BatchStatsC()
        st.per_system_rel = rel.ctypes.data
        st.per_system_cycles = cyc.ctypes.data
        st.per_system_cap = nsys
        rc = self._lib.gmres_batch_ir_solve(self.h, ctypes.c_void_p(_ptr(B)), ctypes.c_void_p(_ptr(X)),
                                            float(tol), int(max_cycles), ctypes.byref(st))
        _check(rc, "gmres_batch_ir_solve")
        return X, BatchStats(status=rc, cycles=st.cycles, block_steps=st.block_steps,
                             converged_systems=st.converged_systems, breakdowns=st.breakdowns,
                             max_rel_res=st.max_rel_res, per_system_rel=rel,
                             per_system_cycles=cyc, kernel_launches=st.kernel_launches,
                             solve_seconds=st.solve_seconds,
                             t_kernel={k: st.t_kernel[i] for i, k in enumerate(BATCH_KERNEL_CLASSES)},
                             class_launches={k: st.class_launches[i]
                                             for i, k in enumerate(BATCH_KERNEL_CLASSES)})

    def set_profiling(self, on: bool):
        """Time kernel classes with CUDA events (direct launches, no graph) in later solves."""
        _check(self._lib.gmres_batch_set_profiling(self.h, int(bool(on))), "gmres_batch_set_profiling")

    # ---- launch shapes ----
    TUNING_FIELDS = ("chunk_tiles", "sweep_smem_kb", "sweep_max_stages")

    def set_tuning(self, **kw):
        """Set launch shapes (see ``gmres_batch_tuning_t``); unspecified fields keep their value."""
        t = BatchTuningC()
        _check(self._lib.gmres_batch_get_tuning(self.h, ctypes.byref(t)), "gmres_batch_get_tuning")
        for k, v in kw.items():
            if k not in self.TUNING_FIELDS:
                raise KeyError(k)
            setattr(t, k, int(v))
        _check(self._lib.gmres_batch_set_tuning(self.h, ctypes.byref(t)), "gmres_batch_set_tuning")

    def get_tuning(self) -> dict:
        t = BatchTuningC()
        _check(self._lib.gmres_batch_get_tuning(self.h, ctypes.byref(t)), "gmres_batch_get_tuning")
        return {k: getattr(t, k) for k in self.TUNING_FIELDS}

    def autotune(self, B, tol: float = 1e-10, max_cycles: int = 1000):
        """Solve from X = 0 under a grid of launch shapes and keep the fastest on this batch.
        Returns (shapes, solve seconds chosen, solve seconds default)."""
        t = BatchTuningC()
        tb, td = ctypes.c_double(), ctypes.c_double()
        if _is_cuda(B):
            import torch
            _check(self._lib.gmres_batch_set_stream(self.h, ctypes.c_void_p(
                torch.cuda.current_stream().cuda_stream)), "gmres_batch_set_stream")
        _check(self._lib.gmres_batch_autotune(self.h, ctypes.c_void_p(_ptr(B)), float(tol),
                                              int(max_cycles), ctypes.byref(t), ctypes.byref(tb),
                                              ctypes.byref(td)), "gmres_batch_autotune")
        return {k: getattr(t, k) for k in self.TUNING_FIELDS}, tb.value, td.value


class MLP:
    """The controller network (12 -> 64 -> 64 -> 9) with the library's forward, backward and Adam
    kernels.  Inputs and labels are CUDA tensors; parameters are a flat float32 array."""

    N_IN, N_OUT = 12, 9

    def __init__(self, params):
        lib = load()
        self._lib = lib
        self.nparams = lib.gmres_mlp_num_params()
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.nparams:
            raise ValueError(f"expected {self.nparams} parameters")
        self.h = ctypes.c_void_p()
        _check(lib.gmres_mlp_create(p.ctypes.data, ctypes.byref(self.h)), "gmres_mlp_create")

    @staticmethod
    def init_params(seed: int = 0):
        """Seeded He-uniform initial parameters (the library draws no random numbers)."""
        rng = np.random.default_rng(seed)
        def lin(o, i):
            bound = np.sqrt(6.0 / i)
            return rng.uniform(-bound, bound, (o, i)).astype(np.float32), np.zeros(o, np.float32)
        w1, b1 = lin(64, 12)
        w2, b2 = lin(64, 64)
        w3, b3 = lin(9, 64)
        w3 *= 0.1
        return np.concatenate([w1.ravel(), b1, w2.ravel(), b2, w3.ravel(), b3])

    def close(self):
        if self.h and self.h.value:
            self._lib.gmres_mlp_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.zeros(self.nparams, np.float32)
        _check(self._lib.gmres_mlp_get_params(self.h, out.ctypes.data), "gmres_mlp_get_params")
        return out

    def forward(self, X):
        """Y[B][9] = net(X[B][12]); X a CUDA float32 tensor (returns one) or a host array."""
        if not _is_cuda(X):
            Xh = np.ascontiguousarray(X, dtype=np.float32)
            Y = np.zeros((Xh.shape[0], self.N_OUT), np.float32)
            _check(self._lib.gmres_mlp_forward(self.h, Xh.ctypes.data, Xh.shape[0], Y.ctypes.data),
                   "gmres_mlp_forward")
            return Y
        import torch
        X = X.contiguous()
        Y = torch.empty((X.shape[0], self.N_OUT), dtype=torch.float32, device=X.device)
        torch.cuda.current_stream().synchronize()
        _check(self._lib.gmres_mlp_forward(self.h, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                           ctypes.c_void_p(Y.data_ptr())), "gmres_mlp_forward")
        return Y

    def gradient(self, X, mc, tl, dc, rt):
        import torch
        g = np.zeros(self.nparams, np.float32)
        loss = np.zeros(4, np.float32)
        lab = [t.contiguous() for t in (mc, tl, dc, rt)]
        torch.cuda.current_stream().synchronize()
        _check(self._lib.gmres_mlp_gradient(self.h, ctypes.c_void_p(X.contiguous().data_ptr()),
                                            *[ctypes.c_void_p(t.data_ptr()) for t in lab],
                                            X.shape[0], g.ctypes.data, loss.ctypes.data),
               "gmres_mlp_gradient")
        return g, loss

    def train_step(self, X, mc, tl, dc, rt, lr: float):
        import torch
        loss = np.zeros(4, np.float32)
        lab = [t.contiguous() for t in (mc, tl, dc, rt)]
        torch.cuda.current_stream().synchronize()
        _check(self._lib.gmres_mlp_train_step(self.h, ctypes.c_void_p(X.contiguous().data_ptr()),
                                              *[ctypes.c_void_p(t.data_ptr()) for t in lab],
                                              X.shape[0], float(lr), loss.ctypes.data),
               "gmres_mlp_train_step")
        return loss


class NativeController:
    """The C ABI's learned controller (gmres_controller_*): a checkpoint file, the 12 features of a
    solver's system computed by the library, and the network's decision."""

    CHOICES = ("network", "default", "fixed")

    def __init__(self, path: str):
        self._lib = load()
        self.h = ctypes.c_void_p()
        _check(self._lib.gmres_controller_load(os.fsencode(path), ctypes.byref(self.h)),
               "gmres_controller_load")

    def close(self):
        if self.h:
            self._lib.gmres_controller_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _as_dict(sg: SuggestionC) -> dict:
        return dict(m=sg.m, tol=sg.inner_tol, d=sg.poly_degree,
                    choice=NativeController.CHOICES[sg.choice],
                    predicted_ratio=sg.predicted_ratio, outputs=np.array(sg.outputs[:]),
                    features=np.array(sg.features[:]))

    def features(self, solver: "Solver", b) -> np.ndarray:
        f = np.zeros(12)
        solver._stream(b)
        _check(self._lib.gmres_controller_features(solver.h, ctypes.c_void_p(_ptr(b)),
                                                   f.ctypes.data), "gmres_controller_features")
        return f

    def decide(self, feats) -> dict:
        f = np.ascontiguousarray(feats, dtype=np.float64)
        sg = SuggestionC()
        _check(self._lib.gmres_controller_decide(self.h, f.ctypes.data, ctypes.byref(sg)),
               "gmres_controller_decide")
        return self._as_dict(sg)

    def suggest(self, solver: "Solver", b) -> dict:
        sg = SuggestionC()
        solver._stream(b)
        _check(self._lib.gmres_controller_suggest(self.h, solver.h, ctypes.c_void_p(_ptr(b)),
                                                  ctypes.byref(sg)), "gmres_controller_suggest")
        return self._as_dict(sg)
