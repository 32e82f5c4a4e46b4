"""Algorithmic (compulsory) HBM bytes of the solver's kernels.

These are the bytes a kernel must move at least once: every matrix entry and index, every
basis column it streams, each vector it reads or writes once.  Cache effects cannot inflate a
throughput computed from them.  Sizes: value s_A, basis s_V, work vector s_W bytes; int32
indices (Section V-D keeps 4-byte indices in every precision).
"""
from __future__ import annotations


def spmv_bytes(n: int, nnz: int, s_a: int, s_x: int, s_y: int) -> int:
    """CSR SpMV y = A x: values + column indices + row pointers + x once + y once."""
    return nnz * (s_a + 4) + (n + 1) * 4 + n * s_x + n * s_y


def spmv_proj_bytes(n: int, nnz: int, ncols: int, s_a: int, s_x: int, s_w: int, s_v: int) -> int:
    """Inner SpMV fused with the first projection at step j (ncols = j+1): the SpMV's bytes (w
    written once) plus V_j read once; w is not read back."""
    return spmv_bytes(n, nnz, s_a, s_x, s_w) + ncols * n * s_v


def pass2_bytes(n, ncols, s_v, s_w) -> int:
    """Second pass (update 1 fused with projection 2): V_j and w read once."""
    return ncols * n * s_v + n * s_w


def update_bytes(n, ncols, s_v, s_w) -> int:
    """Update 2: V_j and w read, v_{j+1} written."""
    return ncols * n * s_v + n * s_w + n * s_v


def cycle_bytes(n, nnz, m, s_a, s_v, s_w) -> dict:
    """Per-class algorithmic bytes of one m-step cycle without preconditioner (keys match the
    profiling classes of the library; "spmv" is the SpMV fused with the first projection)."""
    return {
        "spmv": sum(spmv_proj_bytes(n, nnz, j + 1, s_a, s_v, s_w, s_v) for j in range(m)),
        "cgs_pass2": sum(pass2_bytes(n, j + 1, s_v, s_w) for j in range(m)),
        "cgs_update": sum(update_bytes(n, j + 1, s_v, s_w) for j in range(m)),
    }


def dcgs2_cycle_bytes(n, nnz, m, s_a, s_v, s_w) -> dict:
    """Per-class algorithmic bytes of one m-step DCGS2 cycle without preconditioner.  Step j:
    the SpMV of the candidate U_j fused with the reduction (A, and the j+1 basis columns -- U_j
    among them -- read once; x written); the update (the j+1 columns and x read; column j
    rewritten for j > 0 and column j+1 written); after the cycle one reduction over the m+1
    columns ("cgs_proj")."""
    return {
        "spmv": sum(spmv_bytes(n, nnz, s_a, 0, s_w) + (j + 1) * n * s_v for j in range(m)),
        "cgs_update": sum((j + 1) * n * s_v + n * s_w + (2 if j else 1) * n * s_v
                          for j in range(m)),
        "cgs_proj": (m + 1) * n * s_v,
    }


def poly_step_bytes(n: int, nnz: int, s_a: int = 4, s: int = 4) -> int:
    """One fused polynomial step: SpMV of x, plus P read, Y read and written, Pn written."""
    return nnz * (s_a + 4) + (n + 1) * 4 + n * s + 4 * n * s


def spmv_model_speedup(w: float) -> float:
    """Section V-D cache model: FP64 without x reuse (20 w n bytes) over FP32 with perfect x
    reuse ((8 w + 4) n bytes)."""
    return 20.0 * w / (8.0 * w + 4.0)


def batch_sweep_bytes(n_padded: int, m: int, nrhs: int = 8) -> float:
    """Algorithmic bytes of the block-CGS2 sweeps of one block cycle of the batched solver (all
    systems active): at block step k each of the three sweeps reads the k+1 basis blocks (BF16)
    and the FP32 block W; the update sweep also writes the new block (BF16)."""
    total = 0.0
    for k in range(m):
        blocks = k + 1
        read = n_padded * nrhs * (2 * blocks + 4)
        total += 3 * read + n_padded * nrhs * 2
    return total
