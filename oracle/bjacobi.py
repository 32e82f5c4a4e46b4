"""CPU oracle of the block Jacobi preconditioner with reverse Cuthill-McKee ordering (Section
III-D lists block Jacobi as the paper's second preconditioner; Section V-G applies it after an
RCM reordering, with block sizes 1 and 42).  TEST INFRASTRUCTURE ONLY.

Reading (the paper does not define its RCM variant): the graph is the symmetric pattern of
A + A^T without the diagonal.  Components are ordered one after another; each starts at the
unvisited node of smallest degree (ties: smallest index) and is traversed breadth first, each
node appending its unvisited neighbours in increasing (degree, index) order (Cuthill-McKee);
the whole sequence is then reversed.  perm[new] = old.  Block b is the index set
I_b = perm[b k : (b+1) k] (the last block may be shorter), and M^{-1} v is z[I_b] = A[I_b, I_b]^{-1}
v[I_b] for every block: the block-diagonal part of P A P^T, applied without permuting anything.
"""
from __future__ import annotations

from collections import deque

import numpy as np

F64, F32 = np.float64, np.float32


def _sym_adjacency(A):
    n = A.n
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    cols = np.asarray(A.colidx)
    off = rows != cols
    r = np.concatenate([rows[off], cols[off]])
    c = np.concatenate([cols[off], rows[off]])
    key = np.unique(r.astype(np.int64) * n + c)
    r, c = key // n, key % n
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(ptr, r + 1, 1)
    return np.cumsum(ptr), c


def rcm(A) -> np.ndarray:
    """Reverse Cuthill-McKee permutation (perm[new] = old) by the rules in the module docstring."""
    n = A.n
    ptr, nbr = _sym_adjacency(A)
    deg = np.diff(ptr)
    visited = np.zeros(n, dtype=bool)
    order = []
    by_degree = np.lexsort((np.arange(n), deg))      # start candidates: (degree, index)
    pos = 0
    while len(order) < n:
        while visited[by_degree[pos]]:
            pos += 1
        s = int(by_degree[pos])
        visited[s] = True
        q = deque([s])
        while q:
            u = q.popleft()
            order.append(u)
            nb = nbr[ptr[u]:ptr[u + 1]]
            nb = nb[~visited[nb]]
            if nb.size:
                nb = nb[np.lexsort((nb, deg[nb]))]
                visited[nb] = True
                q.extend(int(v) for v in nb)
    return np.array(order[::-1], dtype=np.int64)


class BlockJacobi:
    """Inverses of the diagonal blocks of P A P^T (FP64), applied as z[I_b] = B_b^{-1} v[I_b]."""

    def __init__(self, A, k: int, reorder: bool = True):
        import scipy.sparse as sp
        self.k = int(k)
        self.n = A.n
        self.perm = rcm(A) if reorder else np.arange(A.n)
        M = sp.csr_matrix((A.val, A.colidx, A.rowptr), shape=(A.n, A.n))
        self.blocks = []
        for b0 in range(0, A.n, self.k):
            I = self.perm[b0:b0 + self.k]
            B = M[I][:, I].toarray()
            self.blocks.append((I, np.linalg.inv(B)))

    def apply(self, v, dtype=F64):
        """M^{-1} v in `dtype` (FP32: inverses and v rounded to FP32, products in FP32)."""
        v = np.asarray(v)
        z = np.zeros(self.n, dtype=dtype)
        for I, inv in self.blocks:
            z[I] = inv.astype(dtype) @ v[I].astype(dtype)
        return z


def bandwidth(A, perm=None) -> int:
    """max |i - j| over the nonzeros of P A P^T (perm[new] = old)."""
    n = A.n
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    cols = np.asarray(A.colidx)
    if perm is None:
        return int(np.max(np.abs(rows - cols)))
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    return int(np.max(np.abs(inv[rows] - inv[cols])))
