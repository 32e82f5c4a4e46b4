// Host FP64 routines of the polynomial preconditioner build (Section III-D).
#include "poly_host.h"

#include <algorithm>
#include <cmath>
#include <limits>

namespace gmresb3 {

namespace {

// 2 x 2 block [a b; c d] eigenvalues, stable for the real case.
void eig2(double a, double b, double c, double d, std::complex<double>& e1,
          std::complex<double>& e2) {
  const double p = 0.5 * (a - d);
  const double bc = b * c;
  const double disc = p * p + bc;
  const double mid = 0.5 * (a + d);
  if (disc >= 0.0) {
    const double sq = std::sqrt(disc);
    // the larger-magnitude root first, the other from the product (avoids cancellation)
    const double r1 = mid + (p >= 0 ? sq : -sq);
    const double det = a * d - bc;
    const double r2 = (r1 != 0.0) ? det / r1 : mid - (p >= 0 ? sq : -sq);
    e1 = {r1, 0.0};
    e2 = {r2, 0.0};
  } else {
    const double im = std::sqrt(-disc);
    e1 = {mid, im};
    e2 = {mid, -im};
  }
}

}  // namespace

bool hessenberg_eigvals(int k, const double* Hin, int ldh, std::vector<std::complex<double>>& ev) {
  ev.assign(k, {0.0, 0.0});
  if (k <= 0) return true;
  // working copy, row-major a[i][j]
  std::vector<double> a((size_t)k * k);
  auto A = [&](int i, int j) -> double& { return a[(size_t)i * k + j]; };
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) A(i, j) = (i <= j + 1) ? Hin[(size_t)j * ldh + i] : 0.0;
  // Balancing (Parlett and Reinsch): a diagonal similarity by powers of two that evens out the
  // row and column norms.  It keeps the Hessenberg form, changes no eigenvalue and matters for the
  // harmonic Ritz matrix, whose last column can be orders of magnitude larger than the rest.
  for (bool changed = true; changed;) {
    changed = false;
    for (int i = 0; i < k; ++i) {
      double c = 0.0, r = 0.0;
      for (int j = 0; j < k; ++j)
        if (j != i) {
          c += std::fabs(A(j, i));
          r += std::fabs(A(i, j));
        }
      if (c == 0.0 || r == 0.0) continue;
      // f = power of two with c f^2 within a factor 2 of r (column scaled by f, row by 1/f)
      double f = 1.0, cf2 = c;
      while (cf2 < 0.5 * r) {
        cf2 *= 4.0;
        f *= 2.0;
      }
      while (cf2 >= 2.0 * r) {
        cf2 *= 0.25;
        f *= 0.5;
      }
      const double sum = c + r, cs = c, rs = r;
      if (f != 1.0 && cs * f + rs / f < 0.95 * sum) {
        changed = true;
        for (int j = 0; j < k; ++j) A(i, j) /= f;
        for (int j = 0; j < k; ++j) A(j, i) *= f;
      }
    }
  }
  const double eps = std::numeric_limits<double>::epsilon();
  double anorm = 0.0;
  for (int i = 0; i < k; ++i)
    for (int j = std::max(0, i - 1); j < k; ++j) anorm += std::fabs(A(i, j));
  int hi = k - 1;
  int its = 0, total = 0;
  while (hi >= 0) {
    // find the start lo of the unreduced block ending at hi
    int lo = hi;
    while (lo > 0) {
      double s = std::fabs(A(lo - 1, lo - 1)) + std::fabs(A(lo, lo));
      if (s == 0.0) s = anorm;
      if (std::fabs(A(lo, lo - 1)) <= eps * s) {
        A(lo, lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {  // 1 x 1 block
      ev[hi] = {A(hi, hi), 0.0};
      --hi;
      its = 0;
      continue;
    }
    if (lo == hi - 1) {  // 2 x 2 block
      eig2(A(hi - 1, hi - 1), A(hi - 1, hi), A(hi, hi - 1), A(hi, hi), ev[hi - 1], ev[hi]);
      hi -= 2;
      its = 0;
      continue;
    }
    if (its >= 120 || total > 120 * k) return false;
    ++its;
    ++total;
    // Shifts: the eigenvalues of the trailing 2 x 2 block (sum s, product t).  Every 10th sweep
    // an exceptional pair breaks cycles (the ad hoc shifts of the EISPACK/LAPACK QR codes): a
    // double shift near 0.75 w +/- 0.66i w around a diagonal entry, w the size of two
    // subdiagonal entries, taken alternately at the top and the bottom of the active block.
    double s, t;
    if (its % 10 == 0) {
      const bool top = (its / 10) % 2 == 1;
      const double w = top ? std::fabs(A(lo + 1, lo)) + std::fabs(A(lo + 2, lo + 1))
                           : std::fabs(A(hi, hi - 1)) + std::fabs(A(hi - 1, hi - 2));
      const double h11 = 0.75 * w + (top ? A(lo, lo) : A(hi, hi));
      s = 2.0 * h11;
      t = h11 * h11 + 0.4375 * w * w;
    } else {
      s = A(hi - 1, hi - 1) + A(hi, hi);
      t = A(hi - 1, hi - 1) * A(hi, hi) - A(hi - 1, hi) * A(hi, hi - 1);
    }
    // first column of (H - s1 I)(H - s2 I) restricted to the block
    double x = A(lo, lo) * A(lo, lo) + A(lo, lo + 1) * A(lo + 1, lo) - s * A(lo, lo) + t;
    double y = A(lo + 1, lo) * (A(lo, lo) + A(lo + 1, lo + 1) - s);
    double z = A(lo + 1, lo) * A(lo + 2, lo + 1);
    for (int q = lo; q <= hi - 2; ++q) {
      // Householder reflector P = I - 2 v v^T / (v^T v) mapping (x, y, z) onto e1
      const double alpha = std::copysign(std::sqrt(x * x + y * y + z * z), x);
      if (alpha == 0.0) {
        if (q + 3 <= hi) {
          x = A(q + 1, q);
          y = A(q + 2, q);
          z = A(q + 3, q);
        }
        continue;
      }
      const double v0 = x + alpha, v1 = y, v2 = z;
      const double vv = v0 * v0 + v1 * v1 + v2 * v2;
      const double beta = 2.0 / vv;
      const int cstart = std::max(lo, q - 1);
      // rows q..q+2, columns cstart..hi
      for (int j = cstart; j <= hi; ++j) {
        const double d = beta * (v0 * A(q, j) + v1 * A(q + 1, j) + v2 * A(q + 2, j));
        A(q, j) -= d * v0;
        A(q + 1, j) -= d * v1;
        A(q + 2, j) -= d * v2;
      }
      // columns q..q+2, rows lo..min(q+3, hi)
      const int rend = std::min(q + 3, hi);
      for (int i = lo; i <= rend; ++i) {
        const double d = beta * (v0 * A(i, q) + v1 * A(i, q + 1) + v2 * A(i, q + 2));
        A(i, q) -= d * v0;
        A(i, q + 1) -= d * v1;
        A(i, q + 2) -= d * v2;
      }
      if (q > lo) {
        A(q + 1, q - 1) = 0.0;
        A(q + 2, q - 1) = 0.0;
      }
      x = A(q + 1, q);
      y = A(q + 2, q);
      if (q + 3 <= hi) z = A(q + 3, q);
    }
    // final 2 x 2 Givens rotation on rows/columns hi-1, hi
    {
      const int q = hi - 1;
      const double r = std::hypot(x, y);
      if (r != 0.0) {
        const double c = x / r, sn = y / r;
        for (int j = std::max(lo, q - 1); j <= hi; ++j) {
          const double u = A(q, j), v = A(q + 1, j);
          A(q, j) = c * u + sn * v;
          A(q + 1, j) = -sn * u + c * v;
        }
        for (int i = lo; i <= hi; ++i) {
          const double u = A(i, q), v = A(i, q + 1);
          A(i, q) = c * u + sn * v;
          A(i, q + 1) = -sn * u + c * v;
        }
        if (q > lo) A(q + 1, q - 1) = 0.0;
      }
    }
  }
  return true;
}

bool harmonic_ritz(int k, const double* H, int ldh, std::vector<std::complex<double>>& theta) {
  // M = H_k + hk1^2 f e_k^T with H_k^T f = e_k (only the last column of H_k changes, so M stays
  // upper Hessenberg)
  std::vector<double> M((size_t)k * k);
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) M[(size_t)j * k + i] = H[(size_t)j * ldh + i];
  const double hk1 = (ldh > k) ? H[(size_t)(k - 1) * ldh + k] : 0.0;
  if (hk1 != 0.0) {
    // solve H_k^T f = e_k by Gaussian elimination with partial pivoting on a dense copy
    std::vector<double> T((size_t)k * k);   // T = H_k^T, row-major T[i][j] = H[j][i]
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) T[(size_t)i * k + j] = H[(size_t)i * ldh + j];
    std::vector<double> f(k, 0.0);
    f[k - 1] = 1.0;
    std::vector<int> perm(k);
    for (int c = 0; c < k; ++c) {
      int piv = c;
      for (int r = c + 1; r < k; ++r)
        if (std::fabs(T[(size_t)r * k + c]) > std::fabs(T[(size_t)piv * k + c])) piv = r;
      if (T[(size_t)piv * k + c] == 0.0) return false;
      if (piv != c) {
        for (int j = 0; j < k; ++j) std::swap(T[(size_t)c * k + j], T[(size_t)piv * k + j]);
        std::swap(f[c], f[piv]);
      }
      for (int r = c + 1; r < k; ++r) {
        const double l = T[(size_t)r * k + c] / T[(size_t)c * k + c];
        if (l == 0.0) continue;
        for (int j = c; j < k; ++j) T[(size_t)r * k + j] -= l * T[(size_t)c * k + j];
        f[r] -= l * f[c];
      }
    }
    for (int r = k - 1; r >= 0; --r) {
      double s = f[r];
      for (int j = r + 1; j < k; ++j) s -= T[(size_t)r * k + j] * f[j];
      f[r] = s / T[(size_t)r * k + r];
    }
    for (int i = 0; i < k; ++i) M[(size_t)(k - 1) * k + i] += hk1 * hk1 * f[i];
  }
  return hessenberg_eigvals(k, M.data(), k, theta);
}

std::vector<std::complex<double>> leja_order(const std::vector<std::complex<double>>& theta) {
  // one representative (imag >= 0) per conjugate pair
  struct Rep {
    std::complex<double> z;
    bool pair;
  };
  std::vector<Rep> reps;
  std::vector<bool> used(theta.size(), false);
  for (size_t i = 0; i < theta.size(); ++i) {
    if (used[i]) continue;
    used[i] = true;
    const auto t = theta[i];
    if (t.imag() == 0.0) {
      reps.push_back({{t.real(), 0.0}, false});
      continue;
    }
    size_t best = i;
    double bd = std::numeric_limits<double>::infinity();
    for (size_t j = 0; j < theta.size(); ++j) {
      if (used[j]) continue;
      const double d = std::abs(theta[j] - std::conj(t));
      if (d < bd) {
        bd = d;
        best = j;
      }
    }
    if (best != i) used[best] = true;
    reps.push_back({{t.real(), std::fabs(t.imag())}, true});
  }
  std::vector<std::complex<double>> out, chosen;
  std::vector<int> remaining(reps.size());
  for (size_t i = 0; i < reps.size(); ++i) remaining[i] = (int)i;
  while (!remaining.empty()) {
    size_t pick_pos = 0;
    if (chosen.empty()) {
      double best = -1.0;
      for (size_t q = 0; q < remaining.size(); ++q) {
        const double a = std::abs(reps[remaining[q]].z);
        if (a > best) {
          best = a;
          pick_pos = q;
        }
      }
    } else {
      double best = -std::numeric_limits<double>::infinity();
      for (size_t q = 0; q < remaining.size(); ++q) {
        const auto z = reps[remaining[q]].z;
        double sc = 0.0;
        for (const auto& c : chosen) sc += std::log(std::max(std::abs(z - c), 1e-300));
        if (sc > best) {
          best = sc;
          pick_pos = q;
        }
      }
    }
    const Rep r = reps[remaining[pick_pos]];
    remaining.erase(remaining.begin() + pick_pos);
    out.push_back(r.z);
    chosen.push_back(r.z);
    if (r.pair) {
      out.push_back(std::conj(r.z));
      chosen.push_back(std::conj(r.z));
    }
  }
  return out;
}

std::vector<PolyStepDesc> poly_schedule(const std::vector<std::complex<double>>& th) {
  std::vector<PolyStepDesc> steps;
  const int K = (int)th.size();
  if (K <= 1) return steps;
  int prod = PB_IN;
  bool yinit = false;
  int i = 0;
  auto blank = [] {
    PolyStepDesc d{};
    d.x = d.p = PB_IN;
    d.pn = PB_NONE;
    return d;
  };
  auto other = [](int a) { return a == PB_B0 ? PB_B1 : PB_B0; };
  while (i < K) {
    PolyStepDesc d = blank();
    d.x = prod;
    d.p = prod;
    d.write_y = 1;
    d.read_y = yinit ? 1 : 0;
    d.cy_y = yinit ? 1.0 : 0.0;
    if (th[i].imag() == 0.0) {
      const double a = 1.0 / th[i].real();
      if (i + 1 == K - 1 && th[i + 1].imag() == 0.0) {
        // last two real roots in one SpMV: Y += (a + a2) P - a a2 A P
        const double a2 = 1.0 / th[i + 1].real();
        d.cy_p = a + a2;
        d.cy_t = -a * a2;
        steps.push_back(d);
        i += 2;
      } else {
        // Y += a P; Pn = P - a A P
        const int dst = other(prod);
        d.pn = dst;
        d.cp_p = 1.0;
        d.cp_t = -a;
        d.cy_p = a;
        steps.push_back(d);
        prod = dst;
        i += 1;
      }
      yinit = true;
    } else {
      const double m2 = th[i].real() * th[i].real() + th[i].imag() * th[i].imag();
      const double c1 = 2.0 * th[i].real() / m2, c2 = 1.0 / m2;
      // step 1: T1 = A P; Y += c1 P - c2 T1
      d.cy_p = c1;
      d.cy_t = -c2;
      if (i + 2 == K) {
        steps.push_back(d);
        i += 2;
        yinit = true;
        continue;
      }
      d.pn = PB_B2;
      d.cp_t = 1.0;
      steps.push_back(d);
      yinit = true;
      // step 2: Pn = P - c1 T1 + c2 A T1 (in place unless P is the input)
      PolyStepDesc e = blank();
      e.x = PB_B2;
      e.p = prod;
      e.pn = (prod == PB_IN) ? PB_B0 : prod;
      e.cp_p = 1.0;
      e.cp_x = -c1;
      e.cp_t = c2;
      i += 2;
      if (i == K - 1 && th[i].imag() == 0.0) {
        // the last root is real: Y += Pn / theta_last, no further SpMV
        e.write_y = 1;
        e.read_y = 1;
        e.cy_y = 1.0;
        e.cy_n = 1.0 / th[i].real();
        i += 1;
      }
      steps.push_back(e);
      prod = e.pn;
    }
  }
  return steps;
}

}  // namespace gmresb3
