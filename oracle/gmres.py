"""CPU oracle for restarted GMRES(m), GMRES-IR and the GMRES-polynomial preconditioner.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference leg may import this module.  It shares no code with the CUDA library:
it is a plain, slow, obviously correct NumPy restatement of the method, step by step in the
paper's order and notation, against which the GPU results are checked.

Passages followed (Loe et al., "Experimental Evaluation of Multiprecision Strategies for GMRES on
GPUs"):

* Algorithm 1 (GMRES(m) with blocked classical Gram-Schmidt) and Section III-A: two CGS passes per
  iteration (CGS2), each a transposed GEMV ``h = V_j^T w`` followed by ``w = w - V_j h``.
* Section III-A: convergence is ``||b - A x||_2 / ||b||_2 <= tol``; restart discards the basis and
  continues from the new residual.
* Algorithm 2 and Section III-B (GMRES-IR): residual and update in double, one GMRES(m) cycle in
  single per refinement step, convergence checked only at restart.
* Section III-D: right preconditioning ``A M^{-1} (M x) = b`` with ``M^{-1} = p(A)``, a GMRES
  polynomial.
* Section V-F: the implicit (Givens) residual of FP64 GMRES is checked against the explicit one;
  a mismatch is a "loss of accuracy".

Readings where the paper is silent (each is listed in the design notes):

* Lucky breakdown: ``h_{j+1,j} <= 10 u ||A z_j||`` with ``u`` the unit roundoff of the working
  precision; the cycle then ends with j columns.
* Givens: ``r = hypot(a, b), c = a / r, s = b / r``.
* FP64 GMRES stops inside a cycle when the implicit residual reaches ``tol ||b||``; GMRES-IR runs
  full cycles of m steps (or to ``inner_tol * gamma`` when an inner tolerance is given).
* The polynomial is the GMRES polynomial of degree d: its residual polynomial
  ``pi(t) = 1 - t p(t)`` has the harmonic Ritz values of ``d+1`` FP64 Arnoldi steps as roots,
  applied in modified Leja order as a product.

Matrix-vector products use ``scipy.sparse`` (a library sparse matmul) on the CSR arrays as given;
dense projections use NumPy matmul.  Low precisions are emulated by NumPy ``float32`` arithmetic
and by round-to-nearest-even truncation to bfloat16.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

F64 = np.float64
F32 = np.float32


# ---------------------------------------------------------------------------------------------
# Basic operations
# ---------------------------------------------------------------------------------------------

def csr_matrix(A, dtype=F64) -> sp.csr_matrix:
    """SciPy view of a CSR matrix (values cast to ``dtype`` by round-to-nearest)."""
    return sp.csr_matrix((A.val.astype(dtype), A.colidx, A.rowptr), shape=(A.n, A.n))


def spmv(A, x, dtype=F64) -> np.ndarray:
    """y = A x; y_i = sum over the stored entries p of row i of val_p * x_{col_p}."""
    return csr_matrix(A, dtype) @ np.asarray(x, dtype=dtype)


def unit_roundoff(dtype) -> float:
    return float(np.finfo(dtype).eps) / 2.0


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even), returned as float32.

    bfloat16 keeps the top 16 bits of the float32 encoding; rounding adds half an ulp of the
    kept part plus the kept part's lowest bit (ties to even) before truncating.
    """
    x = np.ascontiguousarray(x, dtype=F32)
    bits = x.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    out = (rounded & 0xFFFFFFFF).astype(np.uint32).view(F32)
    nan = np.isnan(x)
    if nan.any():
        out = out.copy()
        out[nan] = np.nan
    return out


def round_f16_scaled(v: np.ndarray) -> np.ndarray:
    """Store a unit basis vector in FP16 (round to nearest even) scaled by sqrt(n), so its
    entries are of order one rather than 1/sqrt(n) (Section VI names half precision as a future
    third precision; the scaling is a reading: storing raw unit vectors would push many entries
    of large vectors into FP16's subnormal range).  Returned as float32 in the unscaled units."""
    v = np.asarray(v, dtype=F32)
    s = F32(np.sqrt(v.shape[0]))
    return ((v * s).astype(np.float16).astype(F32) / s).astype(F32)


def givens(a: float, b: float):
    """Rotation with c a + s b = r, -s a + c b = 0: r = hypot(a, b), c = a/r, s = b/r."""
    r = np.hypot(a, b)
    if r == 0.0:
        return 1.0, 0.0, 0.0
    return a / r, b / r, r


# ---------------------------------------------------------------------------------------------
# One GMRES(m) cycle (Algorithm 1 with the CGS2 of Section III-A)
# ---------------------------------------------------------------------------------------------

@dataclass
class Cycle:
    y: np.ndarray           # least-squares solution (length k)
    V: np.ndarray           # basis, n x (k+1) (or n x k after a breakdown)
    H: np.ndarray           # Hessenberg H-bar, (k+1) x k
    k: int                  # steps taken
    gamma: float            # ||r0||
    implicit: list = field(default_factory=list)   # |g_{j+1}| after every step j
    breakdown: bool = False
    Az_norms: list = field(default_factory=list)


def gmres_cycle(apply_op, r0, m, dtype=F64, basis_round=None, stop_abs=0.0, h_dtype=None):
    """Run at most m Arnoldi steps on ``apply_op`` (z -> A M^{-1} z) from r0.

    ``dtype`` is the working precision of vectors and dot products; ``h_dtype`` the precision of
    the Hessenberg matrix and the Givens rotations (defaults to ``dtype``).  ``basis_round`` (if
    given) maps a freshly normalised basis vector to its stored form (e.g. bfloat16 rounding).
    The cycle stops early when the implicit residual |g_{j+1}| <= stop_abs, or at a lucky
    breakdown.
    """
    h_dtype = h_dtype or dtype
    u = unit_roundoff(dtype)
    n = r0.shape[0]
    r0 = np.asarray(r0, dtype=dtype)
    gamma = np.sqrt(np.dot(r0, r0))
    V = np.zeros((n, m + 1), dtype=dtype)
    v1 = r0 / gamma
    V[:, 0] = basis_round(v1) if basis_round else v1
    H = np.zeros((m + 1, m), dtype=h_dtype)      # raw Hessenberg
    R = np.zeros((m + 1, m), dtype=h_dtype)      # rotated copy
    cs = np.zeros(m, dtype=h_dtype)
    sn = np.zeros(m, dtype=h_dtype)
    g = np.zeros(m + 1, dtype=h_dtype)
    g[0] = gamma
    cyc = Cycle(y=None, V=V, H=H, k=0, gamma=float(gamma))
    k = 0
    for j in range(m):
        w = np.asarray(apply_op(V[:, j]), dtype=dtype)          # w_j = A v_j (Algorithm 1)
        Az = np.sqrt(np.dot(w, w))
        cyc.Az_norms.append(float(Az))
        Vj = V[:, : j + 1]
        h1 = Vj.T @ w                                           # CGS pass 1: H = V_j^T w
        w = w - Vj @ h1                                         # CGS pass 1: w = w - V_j H
        h2 = Vj.T @ w                                           # CGS pass 2 (Section III-A)
        w = w - Vj @ h2                                         # CGS pass 2
        H[: j + 1, j] = (h1 + h2).astype(h_dtype)
        hn = np.sqrt(np.dot(w, w))                              # h_{j+1,j} = ||w||
        H[j + 1, j] = hn
        # Givens rotations on the new column
        R[: j + 2, j] = H[: j + 2, j]
        for i in range(j):
            t = cs[i] * R[i, j] + sn[i] * R[i + 1, j]
            R[i + 1, j] = -sn[i] * R[i, j] + cs[i] * R[i + 1, j]
            R[i, j] = t
        c, s, r = givens(R[j, j], R[j + 1, j])
        cs[j], sn[j] = c, s
        R[j, j] = r
        R[j + 1, j] = 0.0
        g[j + 1] = -s * g[j]
        g[j] = c * g[j]
        k = j + 1
        cyc.implicit.append(float(abs(g[j + 1])))
        if hn <= 10.0 * u * Az:                                 # lucky breakdown
            cyc.breakdown = True
            break
        v = w / hn                                              # v_{j+1} = w / h_{j+1,j}
        V[:, j + 1] = basis_round(v) if basis_round else v
        if abs(g[j + 1]) <= stop_abs:
            break
    # back substitution R y = g on the k x k triangle (the least-squares step of Algorithm 1)
    y = np.zeros(k, dtype=h_dtype)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - np.dot(R[i, i + 1 : k], y[i + 1 : k])) / R[i, i]
    cyc.y = y
    cyc.k = k
    cyc.V = V[:, : k + 1] if not cyc.breakdown else V[:, :k]
    cyc.H = H[: k + 1, :k]
    return cyc


def gmres_cycle_dcgs2(apply_op, r0, m, dtype=F64, basis_round=None, stop_abs=0.0):
    """GMRES(m) cycle with classical Gram-Schmidt whose second pass is delayed by one step
    (DCGS2: Bielich, Langou, Thomas, Swirydowicz, Yamazaki, Boman, "Low-synch Gram-Schmidt with
    delayed reorthogonalization for Krylov solvers", Parallel Computing 2022).  A DIFFERENT
    ALGORITHM from the CGS2 of Section III-A: it reaches the same Arnoldi factorisation in exact
    arithmetic, with one global reduction per step instead of three.  The paper notes that one
    kernel launch per operation is a limit of its implementation (Section IV); this variant cuts
    the number of passes over the basis.

    Step j (j >= 1) starts from Q = [v_0 .. v_{j-1}] (final) and the candidate u_j (one projection
    done, not normalised), with the provisional column p = H[0:j, j-1].  In order:
      x = op(u_j)
      one reduction: s = Q^T u_j, alpha = u_j^T u_j, z = Q^T x, beta = u_j^T x
      nu = sqrt(alpha - s^T s)                      (norm of u_j after its second projection)
      H[0:j, j-1] = p + s,  H[j, j-1] = nu          (column j-1 final: Givens, stop tests)
      v_j = (u_j - Q s) / nu
      t = Hbar_j s  (Hbar_j = H[0:j+1, 0:j]);  c = [z, (beta - s^T z) / nu]
      H[0:j+1, j] = (c - t) / nu                    (= [Q, v_j]^T op(v_j), by A Q = Q_{j+1} Hbar_j)
      u_{j+1} = (x - Q z - v_j c_j) / nu            (= (I - Q_{j+1} Q_{j+1}^T) x / nu)
    Step 0: x = op(v_0), H[0, 0] = v_0^T x, u_1 = x - v_0 H[0, 0].  After the last step the
    candidate u_m is reorthogonalised once more to make column m-1 final.  Lucky breakdown at
    column j-1: nu <= 10 u ||op(v_{j-1})|| with ||op(v_{j-1})||^2 = ||H[0:j, j-1]_provisional||^2
    + nu^2.  ``basis_round`` maps a stored vector (v_j and the candidates) to its stored form.
    Returns a Cycle whose V has the k final columns plus v_k (formed for checks only).
    """
    u = unit_roundoff(dtype)
    n = r0.shape[0]
    rnd = basis_round or (lambda v: v)
    r0 = np.asarray(r0, dtype=dtype)
    gamma = np.sqrt(np.dot(r0, r0))
    V = np.zeros((n, m + 1), dtype=dtype)
    V[:, 0] = rnd(r0 / gamma)
    H = np.zeros((m + 1, m), dtype=F64)
    R = np.zeros((m + 1, m), dtype=F64)
    cs = np.zeros(m)
    sn = np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = gamma
    cyc = Cycle(y=None, V=V, H=H, k=0, gamma=float(gamma))
    # step 0
    x = np.asarray(apply_op(V[:, 0]), dtype=dtype)
    h00 = np.dot(V[:, 0], x)
    H[0, 0] = h00
    prov2 = float(h00) ** 2                       # ||provisional column||^2
    cand = rnd(x - V[:, 0] * h00)
    k = 0
    for j in range(1, m + 1):
        Q = V[:, :j]
        last = j == m
        if not last:
            x = np.asarray(apply_op(cand), dtype=dtype)        # op(u_j), before its second pass
        s = Q.T @ cand                                         # the one reduction of step j
        alpha = np.dot(cand, cand)
        if not last:
            z = Q.T @ x
            beta = np.dot(cand, x)
        nu2 = float(alpha) - float(np.dot(s, s))
        nu = np.sqrt(max(nu2, 0.0))
        # column j-1 final: provisional coefficients plus the delayed second pass
        H[:j, j - 1] += s
        H[j, j - 1] = nu
        R[: j + 1, j - 1] = H[: j + 1, j - 1]
        for i in range(j - 1):
            tmp = cs[i] * R[i, j - 1] + sn[i] * R[i + 1, j - 1]
            R[i + 1, j - 1] = -sn[i] * R[i, j - 1] + cs[i] * R[i + 1, j - 1]
            R[i, j - 1] = tmp
        c_, s_, r_ = givens(R[j - 1, j - 1], R[j, j - 1])
        cs[j - 1], sn[j - 1] = c_, s_
        R[j - 1, j - 1] = r_
        R[j, j - 1] = 0.0
        g[j] = -s_ * g[j - 1]
        g[j - 1] = c_ * g[j - 1]
        cyc.implicit.append(float(abs(g[j])))
        cyc.Az_norms.append(float(np.sqrt(prov2 + nu * nu)))
        k = j
        vj = rnd((cand - Q @ s) / nu) if nu > 0 else np.zeros(n, dtype=dtype)
        V[:, j] = vj
        if not (nu > 10.0 * u * np.sqrt(prov2 + nu * nu)):     # lucky breakdown (or NaN)
            cyc.breakdown = True
            break
        if last or abs(g[j]) <= stop_abs:
            break
        t = H[: j + 1, :j] @ s.astype(F64)
        cvec = np.concatenate([z.astype(F64), [(float(beta) - float(np.dot(s, z))) / nu]])
        hnew = (cvec - t) / nu
        H[: j + 1, j] = hnew
        prov2 = float(np.dot(hnew, hnew))
        cand = rnd(((x - Q @ z) - V[:, j] * dtype(cvec[j])) / dtype(nu))
    y = np.zeros(k)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - np.dot(R[i, i + 1: k], y[i + 1: k])) / R[i, i]
    cyc.y = y.astype(dtype)
    cyc.k = k
    cyc.V = V[:, : k + 1]
    cyc.H = H[: k + 1, :k]
    return cyc


def arnoldi(A, v0, k, dtype=F64):
    """k steps of Arnoldi with CGS2 (no least-squares solve).  Returns (V, H, steps)."""
    cyc = gmres_cycle(lambda z: spmv(A, z, dtype), np.asarray(v0, dtype), k, dtype=dtype)
    return cyc.V, cyc.H, cyc.k


def lstsq_givens(H, gamma):
    """min_y || gamma e1 - H y || by Givens rotations (the least-squares step of Algorithm 1)."""
    kp1, k = H.shape
    R = np.array(H, dtype=F64)
    g = np.zeros(kp1)
    g[0] = gamma
    for j in range(k):
        c, s, r = givens(R[j, j], R[j + 1, j])
        # rotate rows j, j+1 of every column from j on, and g
        for col in range(j, k):
            t = c * R[j, col] + s * R[j + 1, col]
            R[j + 1, col] = -s * R[j, col] + c * R[j + 1, col]
            R[j, col] = t
        g[j], g[j + 1] = c * g[j], -s * g[j]
    y = np.zeros(k)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - np.dot(R[i, i + 1 : k], y[i + 1 : k])) / R[i, i]
    return y, abs(g[k])


# ---------------------------------------------------------------------------------------------
# GMRES polynomial preconditioner (Section III-D)
# ---------------------------------------------------------------------------------------------

def harmonic_ritz(H):
    """Harmonic Ritz values of a (k+1) x k Arnoldi Hessenberg: eig(H_k + h^2 H_k^{-T} e_k e_k^T)."""
    k = H.shape[1]
    Hk = np.array(H[:k, :k], dtype=F64)
    hk = float(H[k, k - 1]) if H.shape[0] > k else 0.0
    ek = np.zeros(k)
    ek[-1] = 1.0
    f = np.linalg.solve(Hk.T, ek)
    M = Hk.copy()
    M[:, -1] += hk * hk * f
    return np.linalg.eigvals(M)


def leja_order(theta):
    """Modified Leja ordering: largest modulus first, then maximise the product of distances to
    the values already chosen; a complex value is taken with positive imaginary part first and is
    followed at once by its conjugate."""
    vals = [complex(t) for t in theta]
    # pair up conjugates: keep one representative (Im >= 0) with a multiplicity flag
    reps = []
    used = [False] * len(vals)
    for i, t in enumerate(vals):
        if used[i]:
            continue
        used[i] = True
        if t.imag == 0.0:
            reps.append((complex(t.real, 0.0), False))
            continue
        # find the conjugate
        best, bd = -1, np.inf
        for jx, u in enumerate(vals):
            if not used[jx]:
                d = abs(u - t.conjugate())
                if d < bd:
                    best, bd = jx, d
        used[best] = True
        reps.append((complex(t.real, abs(t.imag)), True))
    out = []
    chosen = []
    remaining = list(range(len(reps)))
    while remaining:
        if not chosen:
            pick = max(remaining, key=lambda i: (abs(reps[i][0]), -i))
        else:
            def score(i):
                z = reps[i][0]
                return sum(np.log(max(abs(z - c), 1e-300)) for c in chosen)
            pick = max(remaining, key=lambda i: (score(i), -i))
        remaining.remove(pick)
        z, pair = reps[pick]
        out.append(z)
        chosen.append(z)
        if pair:
            out.append(z.conjugate())
            chosen.append(z.conjugate())
    return np.array(out)


@dataclass
class Poly:
    roots: np.ndarray   # complex, Leja ordered, length d+1 (conjugates adjacent, +Im first)

    @property
    def degree(self) -> int:
        return len(self.roots) - 1


def poly_build(A, d, v0):
    """GMRES polynomial of degree d from d+1 FP64 Arnoldi steps on start vector v0.

    If Arnoldi breaks down after k < d+1 steps the degree drops to k-1.  d = 0 means no
    preconditioner (returns None).
    """
    if d <= 0:
        return None
    V, H, k = arnoldi(A, v0, d + 1)
    if H.shape[0] == H.shape[1]:   # breakdown: square H, exact invariant subspace
        theta = np.linalg.eigvals(H)
    else:
        theta = harmonic_ritz(H)
    return Poly(roots=leja_order(theta))


def poly_apply(A, poly, v, dtype=F64):
    """z = p(A) v with p(t) = sum_{k=1}^{d+1} theta_k^{-1} pi_{k-1}(t), pi_k = prod_{i<=k}(1 - t/theta_i).

    A conjugate pair (a +- ib) is taken in real arithmetic:
    y += (2a/|theta|^2) prod - (1/|theta|^2) A prod,
    prod <- prod - (2a/|theta|^2) A prod + (1/|theta|^2) A A prod.
    """
    if poly is None:
        return np.asarray(v, dtype=dtype).copy()
    if hasattr(poly, "apply"):                 # another right preconditioner (block Jacobi)
        return poly.apply(v, dtype)
    th = poly.roots
    K = len(th)
    prod = np.asarray(v, dtype=dtype).copy()
    y = np.zeros_like(prod)
    i = 0
    while i < K:
        t = th[i]
        if t.imag == 0.0:
            a = dtype(1.0 / t.real)
            y = y + a * prod
            if i < K - 1:
                prod = prod - a * spmv(A, prod, dtype)
            i += 1
        else:
            m2 = t.real * t.real + t.imag * t.imag
            c1 = dtype(2.0 * t.real / m2)
            c2 = dtype(1.0 / m2)
            Ap = spmv(A, prod, dtype)
            y = y + c1 * prod - c2 * Ap
            if i + 2 < K:
                AAp = spmv(A, Ap, dtype)
                prod = prod - c1 * Ap + c2 * AAp
            i += 2
    return y


def poly_power_coeffs(poly):
    """Power-form coefficients c_0..c_d of p(t) = (1 - pi(t)) / t (for small-degree checks)."""
    pi = np.array([1.0 + 0j])   # coefficients, lowest degree first
    for t in poly.roots:
        pi = np.convolve(pi, np.array([1.0, -1.0 / t]))
    one_minus = -pi
    one_minus[0] += 1.0
    c = one_minus[1:]
    return np.real_if_close(c, tol=1e6).real


def poly_apply_power(A, coeffs, v):
    """z = sum_k c_k A^k v by Horner's rule (FP64)."""
    z = coeffs[-1] * np.asarray(v, F64)
    for c in coeffs[-2::-1]:
        z = spmv(A, z) + c * v
    return z


# ---------------------------------------------------------------------------------------------
# Solvers
# ---------------------------------------------------------------------------------------------

@dataclass
class Result:
    x: np.ndarray
    iters: int
    cycles: int
    rel_res: float                  # explicit ||b - A x|| / ||b|| (FP64)
    converged: bool
    history: list = field(default_factory=list)   # explicit relative residual at each restart
    implicit_history: list = field(default_factory=list)
    loss_of_accuracy: int = 0
    breakdowns: int = 0


def gmres(A, b, m, tol, x0=None, maxiter=200000, poly=None, dtype=F64, max_loa=50,
          poly_dtype=None, orth="cgs2"):
    """Restarted GMRES(m) in one precision, right-preconditioned by p(A) (Algorithm 1).

    Stops inside a cycle when the implicit residual reaches tol ||b||, forms x and checks the
    explicit residual.  If it does not meet tol, the event is counted as a loss of accuracy
    (Section V-F) and GMRES restarts from the explicit residual.

    ``poly_dtype`` (default: ``dtype``) is the precision in which p(A) is applied: FP32 inside an
    FP64 solve is variant (a) of Section III-D (the vector is rounded to FP32, the polynomial
    applied in FP32, the result widened back).  ``orth``: "cgs2" (Section III-A) or "dcgs2"
    (:func:`gmres_cycle_dcgs2`).
    """
    cycle = gmres_cycle if orth == "cgs2" else gmres_cycle_dcgs2
    pd = dtype if poly_dtype is None else poly_dtype
    b = np.asarray(b, dtype=dtype)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=dtype).copy()
    bnorm = float(np.sqrt(np.dot(b.astype(F64), b.astype(F64))))
    op = (lambda z: spmv(A, z, dtype)) if poly is None else \
         (lambda z: spmv(A, poly_apply(A, poly, z.astype(pd), pd).astype(dtype), dtype))
    res = Result(x=x, iters=0, cycles=0, rel_res=np.inf, converged=False)
    while True:
        r = b - spmv(A, x, dtype)
        rel = float(np.linalg.norm(r.astype(F64))) / bnorm
        res.history.append(rel)
        res.rel_res = rel
        if rel <= tol:
            res.converged = True
            break
        if res.iters >= maxiter or res.loss_of_accuracy > max_loa:
            break
        mm = min(m, maxiter - res.iters)
        cyc = cycle(op, r, mm, dtype=dtype, stop_abs=tol * bnorm)
        res.implicit_history.extend(cyc.implicit)
        z = cyc.V[:, : cyc.k] @ cyc.y.astype(dtype)
        if poly is not None:
            z = poly_apply(A, poly, z.astype(pd), pd).astype(dtype)
        x = x + z
        res.iters += cyc.k
        res.cycles += 1
        res.breakdowns += int(cyc.breakdown)
        if cyc.implicit and cyc.implicit[-1] <= tol * bnorm:
            r = b - spmv(A, x, dtype)
            if float(np.linalg.norm(r.astype(F64))) / bnorm > tol:
                res.loss_of_accuracy += 1
    res.x = x
    return res


def gmres_fd(A, b, m, tol, switch_iters, maxiter=200000):
    """GMRES-FD (Section III-C): single-precision GMRES(m) for ``switch_iters`` iterations (or
    until it meets tol), then FP64 GMRES(m) started from that iterate.  Returns (result of the
    FP64 phase with iterations, cycles and history summed over both phases, FP32 iterations)."""
    x0 = None
    it32, cyc32, hist32, loa32 = 0, 0, [], 0
    if switch_iters > 0:
        # the FP32 phase runs to the switch point; a loss of accuracy only restarts it
        r32 = gmres(A, b, m, tol, maxiter=min(switch_iters, maxiter), dtype=F32,
                    max_loa=1 << 30)
        x0 = r32.x.astype(F64)
        it32, cyc32, hist32, loa32 = r32.iters, r32.cycles, r32.history, r32.loss_of_accuracy
    r = gmres(A, b, m, tol, x0=x0, maxiter=maxiter - it32, dtype=F64)
    r.iters += it32
    r.cycles += cyc32
    r.loss_of_accuracy += loa32
    r.history = list(hist32) + list(r.history)
    return r, it32


def gmres_ir(A, b, m, tol, x0=None, maxiter=200000, poly=None, basis="f32", inner_tol=0.0,
             orth="cgs2"):
    """GMRES-IR (Algorithm 2): FP64 residual and update, one FP32 GMRES(m) cycle per step.

    ``basis`` selects the stored precision of the Krylov basis ("f32", "bf16" or "f16", the last
    scaled by ``round_f16_scaled``); dot products
    accumulate in FP32.  The FP32 matrix is the round-to-nearest copy of the FP64 values.  The
    inner cycle runs m steps unless it breaks down or ``inner_tol > 0`` and the inner implicit
    residual falls to ``inner_tol * gamma``.  ``orth`` = "cgs2" (Section III-A) or "dcgs2" (the
    delayed-reorthogonalisation variant, :func:`gmres_cycle_dcgs2`).
    """
    cycle = gmres_cycle if orth == "cgs2" else gmres_cycle_dcgs2
    b = np.asarray(b, dtype=F64)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=F64).copy()
    bnorm = float(np.linalg.norm(b))
    rnd = {"bf16": round_bf16, "f16": round_f16_scaled}.get(basis)
    op = (lambda z: spmv(A, z, F32)) if poly is None else \
         (lambda z: spmv(A, poly_apply(A, poly, z, F32), F32))
    res = Result(x=x, iters=0, cycles=0, rel_res=np.inf, converged=False)
    r = b - spmv(A, x)                                    # r_0 = b - A x_0 [double] (Algorithm 2)
    while True:
        rel = float(np.linalg.norm(r)) / bnorm
        res.history.append(rel)
        res.rel_res = rel
        if rel <= tol:
            res.converged = True
            break
        if res.iters >= maxiter:
            break
        r32 = r.astype(F32)
        gamma = float(np.linalg.norm(r32.astype(F64)))
        cyc = cycle(op, r32, m, dtype=F32, basis_round=rnd,
                    stop_abs=inner_tol * gamma)          # GMRES(m) on A u = r [single]
        res.implicit_history.extend(cyc.implicit)
        u = cyc.V[:, : cyc.k] @ cyc.y.astype(F32)
        if poly is not None:
            u = poly_apply(A, poly, u, F32)
        x = x + u.astype(F64)                             # x = x + u [double]
        r = b - spmv(A, x)                                # r = b - A x [double]
        res.iters += cyc.k
        res.cycles += 1
        res.breakdowns += int(cyc.breakdown)
    res.x = x
    return res
