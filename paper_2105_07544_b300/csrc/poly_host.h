// Host-side (FP64) construction of the GMRES polynomial preconditioner (Section III-D):
// eigenvalues of small Hessenberg matrices, harmonic Ritz values, modified Leja ordering, and
// the schedule of fused SpMV steps that applies p(A).
#pragma once

#include <complex>
#include <vector>

namespace gmresb3 {

// Eigenvalues of the k x k upper Hessenberg matrix H (column-major, leading dimension ldh) by
// the implicit double-shift (Francis) QR iteration with deflation.  Returns false if an
// eigenvalue fails to converge within 60 sweeps per eigenvalue.
bool hessenberg_eigvals(int k, const double* H, int ldh, std::vector<std::complex<double>>& ev);

// Harmonic Ritz values of an Arnoldi Hessenberg H-bar ((k+1) x k, column-major, ld ldh):
// eigenvalues of H_k + h_{k+1,k}^2 H_k^{-T} e_k e_k^T.  With breakdown (hk1 == 0) these are the
// eigenvalues of H_k.
bool harmonic_ritz(int k, const double* H, int ldh, std::vector<std::complex<double>>& theta);

// Modified Leja order: largest modulus first, then the value maximising the product of
// distances to those already chosen; complex values appear as (a + ib, a - ib), b > 0.
std::vector<std::complex<double>> leja_order(const std::vector<std::complex<double>>& theta);

// One fused SpMV step of p(A) v (see k_poly_step): source/destination buffer ids.
enum PolyBuf { PB_IN = 0, PB_B0 = 1, PB_B1 = 2, PB_B2 = 3, PB_NONE = 4 };
struct PolyStepDesc {
  int x, p, pn;                      // SpMV input, own-row operand P, destination of Pn
  double cp_p, cp_x, cp_t;           // Pn = cp_p P + cp_x x + cp_t (A x)
  double cy_y, cy_p, cy_x, cy_t, cy_n;  // Y = cy_y Y + cy_p P + cy_x x + cy_t (A x) + cy_n Pn
  int write_y, read_y;
};

// Steps applying p(A) = sum_{k=1}^{d+1} pi_{k-1}(A) / theta_k, pi_k = prod_{i<=k} (1 - A/theta_i),
// to PB_IN with the result in Y; d = theta.size() - 1 SpMVs.  Conjugate pairs use real
// arithmetic.
std::vector<PolyStepDesc> poly_schedule(const std::vector<std::complex<double>>& theta);

}  // namespace gmresb3
