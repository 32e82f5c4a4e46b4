"""Helpers shared by the GPU parity tests (no solver arithmetic here)."""
import numpy as np
import pytest
import torch

import synth


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def random_csr(n, seed, min_nnz=0, max_nnz=9, dense_rows=(), dense_len=0):
    """Random sparse matrix with varied row lengths (some empty), optional long rows, and a
    dominant diagonal on rows that have entries; sorted columns."""
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        k = dense_len if i in dense_rows else int(rng.integers(min_nnz, max_nnz + 1))
        cols = set(rng.choice(n, size=min(k, n), replace=False).tolist()) if k else set()
        rows.append(sorted(cols))
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    colidx = np.array([c for r in rows for c in r], dtype=np.int32)
    val = rng.uniform(-1, 1, len(colidx))
    return synth.CSR(n=n, rowptr=rowptr.astype(np.int32), colidx=colidx, val=val)
