// Host FP64 dense kernels for the setup phase (principal factorisations,
// coarse block factorisation).  Row-major storage throughout.
#pragma once
#include <algorithm>
#include <atomic>
#include <cmath>
#include <functional>
#include <thread>
#include <vector>

namespace fetidp {
namespace host {

// Run f(i) for i in [0, n) on up to hardware_concurrency threads.
inline void parallel_for(int n, const std::function<void(int)>& f) {
  int nt = (int)std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  nt = std::min(nt, n);
  if (nt <= 1) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  std::atomic_int next{0};
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&]() {
      for (;;) {
        const int i = next.fetch_add(1);
        if (i >= n) break;
        f(i);
      }
    });
  for (auto& x : th) x.join();
}

// C (m x n) = alpha * op(A) op(B) + beta * C;  op(A) is m x k.
inline void gemm(bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
                 const double* B, int ldb, double beta, double* C, int ldc) {
  std::vector<double> row(n);
  for (int i = 0; i < m; ++i) {
    std::fill(row.begin(), row.end(), 0.0);
    for (int p = 0; p < k; ++p) {
      const double a = ta ? A[(size_t)p * lda + i] : A[(size_t)i * lda + p];
      if (a == 0.0) continue;
      if (!tb) {
        const double* b = B + (size_t)p * ldb;
        for (int j = 0; j < n; ++j) row[j] += a * b[j];
      } else {
        for (int j = 0; j < n; ++j) row[j] += a * B[(size_t)j * ldb + p];
      }
    }
    double* c = C + (size_t)i * ldc;
    if (beta == 0.0)
      for (int j = 0; j < n; ++j) c[j] = alpha * row[j];
    else
      for (int j = 0; j < n; ++j) c[j] = alpha * row[j] + beta * c[j];
  }
}

// In-place lower Cholesky A = L L^T (upper part left untouched).  false if not SPD.
inline bool cholesky(int n, double* A, int lda) {
  for (int j = 0; j < n; ++j) {
    double* aj = A + (size_t)j * lda;
    double s = aj[j];
    for (int k = 0; k < j; ++k) s -= aj[k] * aj[k];
    if (!(s > 0.0) || !std::isfinite(s)) return false;
    const double ljj = std::sqrt(s);
    aj[j] = ljj;
    const double inv = 1.0 / ljj;
    for (int i = j + 1; i < n; ++i) {
      double* ai = A + (size_t)i * lda;
      double t = ai[j];
      for (int k = 0; k < j; ++k) t -= ai[k] * aj[k];
      ai[j] = t * inv;
    }
  }
  return true;
}

// Inverse of an SPD matrix through Cholesky: Ainv = L^{-T} L^{-1}.  false if not SPD.
inline bool spd_inverse(int n, const double* A, int lda, double* Ainv, int ldi) {
  std::vector<double> L((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) L[(size_t)i * n + j] = (j <= i) ? A[(size_t)i * lda + j] : 0.0;
  if (!cholesky(n, L.data(), n)) return false;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) L[(size_t)i * n + j] = 0.0;
  // W = L^{-1} (lower triangular), column by column
  std::vector<double> W((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    W[(size_t)j * n + j] = 1.0 / L[(size_t)j * n + j];
    for (int i = j + 1; i < n; ++i) {
      double s = 0.0;
      const double* li = L.data() + (size_t)i * n;
      for (int k = j; k < i; ++k) s -= li[k] * W[(size_t)k * n + j];
      W[(size_t)i * n + j] = s / li[i];
    }
  }
  // Ainv = W^T W (symmetric): Ainv[i][j] = sum_{k >= max(i,j)} W[k][i] W[k][j]
  for (int i = 0; i < n; ++i) {
    double* out = Ainv + (size_t)i * ldi;
    for (int j = 0; j < n; ++j) out[j] = 0.0;
  }
  for (int k = 0; k < n; ++k) {
    const double* wk = W.data() + (size_t)k * n;
    for (int i = 0; i <= k; ++i) {
      const double a = wk[i];
      if (a == 0.0) continue;
      double* out = Ainv + (size_t)i * ldi;
      for (int j = 0; j <= k; ++j) out[j] += a * wk[j];
    }
  }
  return true;
}

// Diagonal-pivoted Cholesky solve of the small SPD(-semi) system G c = h (row-major nk x nk):
// pivots chosen as the largest remaining Schur diagonal (lowest index on ties), stop when it
// is <= drop_rel * max diag(G); coefficients of dropped columns are 0.
inline void gram_solve(int nk, const double* G, const double* h, double drop_rel, double* c) {
  std::vector<double> S(G, G + (size_t)nk * nk);
  double dmax = 0.0;
  for (int i = 0; i < nk; ++i) dmax = std::max(dmax, G[(size_t)i * nk + i]);
  std::vector<int> piv;
  std::vector<char> used(nk, 0);
  while ((int)piv.size() < nk) {
    int jb = -1;
    double best = 0.0;
    for (int i = 0; i < nk; ++i)
      if (!used[i] && (jb < 0 || S[(size_t)i * nk + i] > best)) {
        best = S[(size_t)i * nk + i];
        jb = i;
      }
    if (!(best > drop_rel * dmax)) break;
    used[jb] = 1;
    piv.push_back(jb);
    const double inv = 1.0 / std::sqrt(best);
    std::vector<double> col(nk);
    for (int i = 0; i < nk; ++i) col[i] = S[(size_t)i * nk + jb] * inv;
    for (int i = 0; i < nk; ++i)
      for (int j = 0; j < nk; ++j) S[(size_t)i * nk + j] -= col[i] * col[j];
  }
  const int np = (int)piv.size();
  std::vector<double> Lm((size_t)np * np, 0.0), y(np);
  for (int a = 0; a < np; ++a)
    for (int b = 0; b <= a; ++b) {
      double s = G[(size_t)piv[a] * nk + piv[b]];
      for (int k = 0; k < b; ++k) s -= Lm[(size_t)a * np + k] * Lm[(size_t)b * np + k];
      Lm[(size_t)a * np + b] = (a == b) ? std::sqrt(s) : s / Lm[(size_t)b * np + b];
    }
  for (int a = 0; a < np; ++a) {
    double s = h[piv[a]];
    for (int k = 0; k < a; ++k) s -= Lm[(size_t)a * np + k] * y[k];
    y[a] = s / Lm[(size_t)a * np + a];
  }
  for (int i = 0; i < nk; ++i) c[i] = 0.0;
  for (int a = np - 1; a >= 0; --a) {
    double s = y[a];
    for (int k = a + 1; k < np; ++k) s -= Lm[(size_t)k * np + a] * c[piv[k]];
    c[piv[a]] = s / Lm[(size_t)a * np + a];
  }
}

}  // namespace host
}  // namespace fetidp
