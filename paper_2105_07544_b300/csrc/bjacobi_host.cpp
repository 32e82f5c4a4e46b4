// Host routines of the block Jacobi preconditioner (RCM ordering and block inverses).
#include "bjacobi_host.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <deque>
#include <thread>

namespace gmresb3 {

std::vector<int32_t> rcm_order(int n, const int32_t* rowptr, const int32_t* col) {
  // symmetric adjacency without the diagonal, neighbours unique
  std::vector<std::vector<int32_t>> adj(n);
  for (int i = 0; i < n; ++i)
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int j = col[p];
      if (j == i) continue;
      adj[i].push_back(j);
      adj[j].push_back(i);
    }
  std::vector<int> deg(n);
  for (int i = 0; i < n; ++i) {
    auto& a = adj[i];
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
    deg[i] = (int)a.size();
  }
  auto before = [&](int a, int b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; };
  std::vector<int32_t> start(n);
  for (int i = 0; i < n; ++i) start[i] = i;
  std::sort(start.begin(), start.end(), before);
  std::vector<char> visited(n, 0);
  std::vector<int32_t> order;
  order.reserve(n);
  std::vector<int32_t> nb;
  size_t sp = 0;
  while ((int)order.size() < n) {
    while (visited[start[sp]]) ++sp;
    const int s = start[sp];
    visited[s] = 1;
    std::deque<int32_t> q{s};
    while (!q.empty()) {
      const int u = q.front();
      q.pop_front();
      order.push_back(u);
      nb.clear();
      for (int v : adj[u])
        if (!visited[v]) nb.push_back(v);
      std::sort(nb.begin(), nb.end(), before);
      for (int v : nb) {
        visited[v] = 1;
        q.push_back(v);
      }
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

namespace {

// Gauss-Jordan inverse of the kb x kb row-major matrix a (destroyed) into x (row-major).
bool invert(int kb, std::vector<double>& a, std::vector<double>& x) {
  x.assign((size_t)kb * kb, 0.0);
  for (int i = 0; i < kb; ++i) x[(size_t)i * kb + i] = 1.0;
  for (int c = 0; c < kb; ++c) {
    int piv = c;
    for (int r = c + 1; r < kb; ++r)
      if (std::fabs(a[(size_t)r * kb + c]) > std::fabs(a[(size_t)piv * kb + c])) piv = r;
    const double pv = a[(size_t)piv * kb + c];
    if (pv == 0.0 || !std::isfinite(pv)) return false;
    if (piv != c)
      for (int j = 0; j < kb; ++j) {
        std::swap(a[(size_t)piv * kb + j], a[(size_t)c * kb + j]);
        std::swap(x[(size_t)piv * kb + j], x[(size_t)c * kb + j]);
      }
    const double inv = 1.0 / pv;
    for (int j = 0; j < kb; ++j) {
      a[(size_t)c * kb + j] *= inv;
      x[(size_t)c * kb + j] *= inv;
    }
    for (int r = 0; r < kb; ++r) {
      if (r == c) continue;
      const double f = a[(size_t)r * kb + c];
      if (f == 0.0) continue;
      for (int j = 0; j < kb; ++j) {
        a[(size_t)r * kb + j] -= f * a[(size_t)c * kb + j];
        x[(size_t)r * kb + j] -= f * x[(size_t)c * kb + j];
      }
    }
  }
  return true;
}

}  // namespace

bool block_inverses(int n, const int32_t* rowptr, const int32_t* col, const double* val,
                    const std::vector<int32_t>& perm, int k, std::vector<double>& inv,
                    int threads) {
  const int nb = (n + k - 1) / k;
  inv.assign((size_t)nb * k * k, 0.0);
  std::vector<int32_t> blk(n), pos(n);
  for (int i = 0; i < n; ++i) {
    blk[perm[i]] = i / k;
    pos[perm[i]] = i % k;
  }
  std::atomic<int> next{0};
  std::atomic<bool> ok{true};
  auto work = [&] {
    std::vector<double> a, x;
    for (;;) {
      const int b = next.fetch_add(1);
      if (b >= nb || !ok.load()) return;
      const int kb = std::min(k, n - b * k);
      a.assign((size_t)kb * kb, 0.0);
      for (int r = 0; r < kb; ++r) {
        const int row = perm[(size_t)b * k + r];
        for (int p = rowptr[row]; p < rowptr[row + 1]; ++p) {
          const int c = col[p];
          if (blk[c] == b) a[(size_t)r * kb + pos[c]] += val[p];
        }
      }
      if (!invert(kb, a, x)) {
        ok.store(false);
        return;
      }
      double* out = inv.data() + (size_t)b * k * k;   // column-major [c][r]
      for (int c = 0; c < kb; ++c)
        for (int r = 0; r < kb; ++r) out[(size_t)c * k + r] = x[(size_t)r * kb + c];
    }
  };
  const int nt = std::max(1, std::min(threads, nb));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  return ok.load();
}

}  // namespace gmresb3
