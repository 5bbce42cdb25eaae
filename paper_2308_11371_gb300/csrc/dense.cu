// Dense batched FP64 kernels of the setup phase: the principal cells' stiffness blocks
// K_rr, K_rp, K_pp (Eq. 39) assembled from their Gauss-point C_hat, the principal inverses
// K_rr^{-1} and S_dd = F_dd^{-1} (Sec. 3.1.1) by the symmetric sweep operator, and the products
// U_rp = K_rr^{-1} K_rp.
//
// Sweep operator on a symmetric matrix, pivot k (a = A_kk > 0 while A is positive definite):
//   A_kk <- -1/a,   A_ik <- A_ik / a (i != k),   A_ij <- A_ij - A_ik A_kj / a (i, j != k).
// Sweeping every index gives -A^{-1}.  Only the upper triangle is updated; one launch per pivot
// updates all matrices of the batch.  The old pivot column (= row, by symmetry) and 1/a are read
// from a buffer that the previous launch filled with the next pivot's column, so no thread reads
// an entry another thread of the same launch writes.
#include <cmath>

#include "common.cuh"

namespace fetidp {
namespace {

inline int grid_for(long long work, int threads) {
  long long g = (work + threads - 1) / threads;
  if (g > 152LL * 64) g = 152LL * 64;
  return (int)(g < 1 ? 1 : g);
}

// Element matrices of the principal cells added into K_rr, K_rp, K_pp (local order), one colour
// of elements per launch: elements of a colour (same index parities) share no node, so no two
// threads of a launch touch the same entry and the sums run in a fixed order (deterministic).
// One thread per (principal, element, row (A, i)); elements of other colours return.
template <int D>
__global__ void assemble_principal_kernel(const double* __restrict__ snap, const int* __restrict__ sigma,
                                          long long nsnap, int nrb, int e, int nc, int n, int nr,
                                          const int* __restrict__ iperm, double wq, double inv_h,
                                          double* __restrict__ Krr, double* __restrict__ Krp,
                                          double* __restrict__ Kpp, int color) {
  constexpr int NA = 1 << D;
  constexpr int ND = NA * D;
  constexpr int NI = D * D;
  const int nel = e * e * (D == 3 ? e : 1);
  const int np = n - nr;
  const long long total = (long long)nrb * nel * ND;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t / ((long long)nel * ND));
    const int r = (int)(t - (long long)k * nel * ND);
    const int el = r / ND, row = r - el * ND;
    const int A = row / D, i = row - A * D;
    const int ex = el % e, ey = (el / e) % e, ez = el / (e * e);
    if ((ex & 1) + 2 * (ey & 1) + 4 * (ez & 1) != color) continue;
    const double* Cel = snap + (long long)sigma[k] * nsnap + (long long)el * NA * nc;
    double krow[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) krow[q] = 0.0;
    for (int gp = 0; gp < NA; ++gp) {
      double dN[NA][D];
#pragma unroll
      for (int B = 0; B < NA; ++B)
#pragma unroll
        for (int a = 0; a < D; ++a) {
          double v = inv_h;
#pragma unroll
          for (int kk = 0; kk < D; ++kk) {
            const int off = (B >> kk) & 1;
            const double tk = gauss_t((gp >> kk) & 1);
            v *= (kk == a) ? (off ? 1.0 : -1.0) : (off ? tk : 1.0 - tk);
          }
          dN[B][a] = v;
        }
      const double* C = Cel + gp * nc;
      double w[D][D];   // w[j][b] = sum_a dN_A[a] C[(i,a),(j,b)]
#pragma unroll
      for (int j = 0; j < D; ++j)
#pragma unroll
        for (int b = 0; b < D; ++b) {
          double s = 0.0;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            int I = i * D + a, J = j * D + b;
            if (I > J) { const int tmp = I; I = J; J = tmp; }
            s += dN[A][a] * C[I * NI - I * (I - 1) / 2 + (J - I)];
          }
          w[j][b] = s;
        }
#pragma unroll
      for (int B = 0; B < NA; ++B)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          double s = 0.0;
#pragma unroll
          for (int b = 0; b < D; ++b) s += w[j][b] * dN[B][b];
          krow[B * D + j] += wq * s;
        }
    }
    int nodes[NA];
#pragma unroll
    for (int B = 0; B < NA; ++B) {
      const int bx = B & 1, by = (B >> 1) & 1, bz = (B >> 2) & 1;
      nodes[B] = (ex + bx) + (e + 1) * ((ey + by) + (e + 1) * (D == 3 ? (ez + bz) : 0));
    }
    const int la = iperm[nodes[A] * D + i];
#pragma unroll
    for (int B = 0; B < NA; ++B)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int lb = iperm[nodes[B] * D + j];
        const double v = krow[B * D + j];
        if (la < nr) {
          if (lb < nr) Krr[((long long)k * nr + la) * nr + lb] += v;
          else Krp[((long long)k * nr + la) * np + (lb - nr)] += v;
        } else if (lb >= nr) {
          Kpp[((long long)k * np + (la - nr)) * np + (lb - nr)] += v;
        }
      }
  }
}

// Pivot column 0 and 1/A_00 of every matrix (start of the sweep).
__global__ void sweep_init_kernel(const double* __restrict__ A, long long stride, int n, int lda, int batch,
                                  double* __restrict__ col, int* __restrict__ status) {
  const long long total = (long long)batch * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / n), i = (int)(t - (long long)b * n);
    const double v = A[b * stride + i];   // row 0 = column 0
    col[(long long)b * (n + 1) + i] = v;
    if (i == 0) {
      if (!(v > 0.0)) atomicExch(status, 1);
      col[(long long)b * (n + 1) + n] = 1.0 / v;
    }
  }
}

// One sweep step on the upper triangles; each thread updates 4 consecutive entries of a row.
__global__ void sweep_step_kernel(double* __restrict__ A, long long stride, int n, int lda, int batch, int k,
                                  const double* __restrict__ cin, double* __restrict__ cout,
                                  int* __restrict__ status) {
  const int nq = (n + 3) / 4;
  const long long total = (long long)batch * n * nq;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / ((long long)n * nq));
    const int r = (int)(t - (long long)b * n * nq);
    const int i = r / nq, j0 = 4 * (r - (r / nq) * nq);
    if (j0 + 3 < i) continue;                       // wholly below the diagonal
    const double* ci = cin + (long long)b * (n + 1);
    const double inv = ci[n];
    const double cii = ci[i] * inv;
    double* Ar = A + b * stride + (long long)i * lda;
    double* co = cout + (long long)b * (n + 1);
    for (int j = j0; j < j0 + 4 && j < n; ++j) {
      if (j < i) continue;
      double v;
      if (i == k) v = (j == k) ? -inv : ci[j] * inv;
      else if (j == k) v = cii;
      else v = fma(-cii, ci[j], Ar[j]);
      Ar[j] = v;
      if (k + 1 < n) {
        if (j == k + 1) co[i] = v;                  // entries (i, k+1), i <= k+1
        if (i == k + 1) {                           // entries (k+1, j), j >= k+1
          co[j] = v;
          if (j == k + 1) {
            if (!(v > 0.0)) atomicExch(status, 1);
            co[n] = 1.0 / v;
          }
        }
      }
    }
  }
}

// -A (upper) -> A^{-1} in both triangles.
__global__ void sweep_finish_kernel(double* __restrict__ A, long long stride, int n, int lda, int batch) {
  const long long total = (long long)batch * n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / ((long long)n * n));
    const int r = (int)(t - (long long)b * n * n);
    const int i = r / n, j = r - (r / n) * n;
    if (j < i) continue;
    double* Ab = A + b * stride;
    const double v = -Ab[(long long)i * lda + j];
    Ab[(long long)i * lda + j] = v;
    Ab[(long long)j * lda + i] = v;
  }
}

// C_b = A_b B_b (A: M x K row-major lda, B: K x N row-major ldb), one thread per output entry.
__global__ void batched_gemm_nn_kernel(const double* __restrict__ A, long long sa, int lda,
                                       const double* __restrict__ B, long long sb, int ldb, double* __restrict__ C,
                                       long long sc, int ldc, int M, int N, int K, int batch) {
  const long long total = (long long)batch * M * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / ((long long)M * N));
    const int r = (int)(t - (long long)b * M * N);
    const int i = r / N, j = r - (r / N) * N;
    const double* Ar = A + b * sa + (long long)i * lda;
    const double* Bc = B + b * sb + j;
    double s = 0.0;
    for (int q = 0; q < K; ++q) s = fma(Ar[q], Bc[(long long)q * ldb], s);
    C[b * sc + (long long)i * ldc + j] = s;
  }
}

// Out_b = (In_b block rows [r0, r0+M), cols [c0, c0+N)), optionally transposed.
__global__ void batched_block_copy_kernel(const double* __restrict__ in, long long si, int ldi, int r0, int c0,
                                          double* __restrict__ out, long long so, int ldo, int M, int N,
                                          int batch, bool transpose) {
  const long long total = (long long)batch * M * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / ((long long)M * N));
    const int r = (int)(t - (long long)b * M * N);
    const int i = r / N, j = r - (r / N) * N;
    const double v = in[b * si + (long long)(r0 + i) * ldi + c0 + j];
    if (transpose) out[b * so + (long long)j * ldo + i] = v;
    else out[b * so + (long long)i * ldo + j] = v;
  }
}

// out[b] = sum_l A_b[r0 + l][r0 + l], l < m (one warp per matrix).
__global__ void batched_diag_sum_kernel(const double* __restrict__ A, long long stride, int lda, int r0, int m,
                                        int batch, double* __restrict__ out) {
  const int w = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (w >= batch) return;
  double s = 0.0;
  for (int l = lane; l < m; l += 32) s += A[w * stride + (long long)(r0 + l) * lda + r0 + l];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) out[w] = s;
}

// C_b = alpha op(A_b) op(B_b) + beta C_b, op = identity or transpose, row-major operands.
// 32 x 32 output tile per block, 2 x 2 per thread, K chunks of 16 staged in shared memory.
constexpr int BG_T = 32, BG_K = 16;
__global__ void __launch_bounds__(256) batched_gemm_kernel(bool ta, bool tb, int M, int N, int K, double alpha,
                                                           const double* __restrict__ A, long long sa, int lda,
                                                           const double* __restrict__ B, long long sb, int ldb,
                                                           double beta, double* __restrict__ C, long long sc, int ldc) {
  __shared__ double As[BG_K][BG_T + 1];
  __shared__ double Bs[BG_K][BG_T + 1];
  const int bz = blockIdx.z;
  const double* Ab = A + bz * sa;
  const double* Bb = B + bz * sb;
  double* Cb = C + bz * sc;
  const int m0 = blockIdx.y * BG_T, n0 = blockIdx.x * BG_T;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int k0 = 0; k0 < K; k0 += BG_K) {
    for (int t = threadIdx.x; t < BG_K * BG_T; t += 256) {
      // op(A)[m][k]: m = m0 + r, k = k0 + q
      {
        int r, q;
        if (ta) { q = t / BG_T; r = t - q * BG_T; }   // A[k][m]: m fastest
        else { r = t / BG_K; q = t - r * BG_K; }      // A[m][k]: k fastest
        const int gm = m0 + r, gk = k0 + q;
        double v = 0.0;
        if (gm < M && gk < K) v = ta ? Ab[(long long)gk * lda + gm] : Ab[(long long)gm * lda + gk];
        As[q][r] = v;
      }
      // op(B)[k][n]: n = n0 + r
      {
        int r, q;
        if (tb) { r = t / BG_K; q = t - r * BG_K; }   // B[n][k]: k fastest
        else { q = t / BG_T; r = t - q * BG_T; }      // B[k][n]: n fastest
        const int gn = n0 + r, gk = k0 + q;
        double v = 0.0;
        if (gn < N && gk < K) v = tb ? Bb[(long long)gn * ldb + gk] : Bb[(long long)gk * ldb + gn];
        Bs[q][r] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < BG_K; ++q) {
      const double a0 = As[q][ty], a1 = As[q][ty + 16];
      const double b0 = Bs[q][tx], b1 = Bs[q][tx + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < M && gn < N) {
        double* cp = Cb + (long long)gm * ldc + gn;
        *cp = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * (*cp));
      }
    }
}

// A_b <- (A_b + A_b^T) / 2.
__global__ void batched_symmetrize_kernel(double* __restrict__ A, long long stride, int n, int lda, int batch) {
  const long long total = (long long)batch * n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / ((long long)n * n));
    const int r = (int)(t - (long long)b * n * n);
    const int i = r / n, j = r - (r / n) * n;
    if (j <= i) continue;
    double* Ab = A + b * stride;
    const double v = 0.5 * (Ab[(long long)i * lda + j] + Ab[(long long)j * lda + i]);
    Ab[(long long)i * lda + j] = v;
    Ab[(long long)j * lda + i] = v;
  }
}

// P_kj = K_rp^(k)T U_rp^(j) for all principal pairs (n_p x n_p each, contraction over n_r), one
// thread per (k, j, r, q).
__global__ void principal_pairs_kernel(const double* __restrict__ Krp, const double* __restrict__ Urp, int nrb,
                                       int nr, int np, double* __restrict__ P) {
  const long long total = (long long)nrb * nrb * np * np;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t % np), r = (int)((t / np) % np);
    const long long kj = t / ((long long)np * np);
    const int j = (int)(kj % nrb), k = (int)(kj / nrb);
    const double* a = Krp + (long long)k * nr * np + r;
    const double* b = Urp + (long long)j * nr * np + q;
    double s = 0.0;
    for (int i = 0; i < nr; ++i) s = fma(a[(long long)i * np], b[(long long)i * np], s);
    P[t] = s;
  }
}

// Per-cell S_pp_ring (Eq. 43): sym( sum_k alpha_k K_pp^(k) - sum_{k,j} alpha_k pi_j P_kj ),
// P_kj = K_rp^(k)T U_rp^(j).  One thread per (cell, r <= q).
__global__ void spp_cells_kernel(const double* __restrict__ alpha, const double* __restrict__ pi,
                                 const double* __restrict__ Kpp, const double* __restrict__ P, int nrb, int np,
                                 long long ncell, double* __restrict__ out) {
  const int npp = np * np;
  const long long total = ncell * npp;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long s = t / npp;
    const int rq = (int)(t - s * npp), r = rq / np, q = rq - (rq / np) * np;
    if (q < r) continue;
    const double* a = alpha + s * nrb;
    const double* p = pi + s * nrb;
    double x_rq = 0.0, x_qr = 0.0;
    for (int k = 0; k < nrb; ++k) {
      const double ak = a[k];
      double w_rq = Kpp[(long long)k * npp + r * np + q], w_qr = Kpp[(long long)k * npp + q * np + r];
      const double* Pk = P + (long long)k * nrb * npp;
      for (int j = 0; j < nrb; ++j) {
        w_rq -= p[j] * Pk[(long long)j * npp + r * np + q];
        w_qr -= p[j] * Pk[(long long)j * npp + q * np + r];
      }
      x_rq += ak * w_rq;
      x_qr += ak * w_qr;
    }
    const double v = 0.5 * (x_rq + x_qr);
    out[s * npp + r * np + q] = v;
    out[s * npp + q * np + r] = v;
  }
}

// Slab blocks of S_PP from the per-cell S_pp_ring: diagonal blocks A_i (slab i) and couplings
// C_i = S(slab i, slab i + 1).  One colour of cells per launch (cells of a colour share no vertex:
// no two threads add into the same entry; fixed colour order, deterministic sums).  One thread per
// (cell, corner k1, corner k2); cells of other colours return.
__global__ void coarse_assemble_kernel(const double* __restrict__ Spp, long long ncell, int d, int nck, int np,
                                       int ncx, int ncy, int vdx, int vdy, const int* __restrict__ vslab,
                                       const int* __restrict__ vpos, int b, double* __restrict__ A,
                                       double* __restrict__ C, int color) {
  const long long total = ncell * nck * nck;
  const long long bb = (long long)b * b;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long s = t / (nck * nck);
    const int kk = (int)(t - s * nck * nck), k1 = kk / nck, k2 = kk - (kk / nck) * nck;
    const int cx = (int)(s % ncx), cy = (int)((s / ncx) % ncy), cz = (int)(s / ((long long)ncx * ncy));
    if ((cx & 1) + 2 * (cy & 1) + 4 * (cz & 1) != color) continue;
    const long long v1 = (cx + (k1 & 1)) + (long long)vdx * ((cy + ((k1 >> 1) & 1)) + (long long)vdy * (cz + (d == 3 ? ((k1 >> 2) & 1) : 0)));
    const long long v2 = (cx + (k2 & 1)) + (long long)vdx * ((cy + ((k2 >> 1) & 1)) + (long long)vdy * (cz + (d == 3 ? ((k2 >> 2) & 1) : 0)));
    const int s1 = vslab[v1], s2 = vslab[v2];
    if (s1 < 0 || s2 < 0) continue;                 // clamped vertex
    double* dst;
    if (s1 == s2) dst = A + s1 * bb;
    else if (s2 == s1 + 1) dst = C + s1 * bb;
    else continue;
    const double* S = Spp + s * (long long)np * np;
    for (int c1 = 0; c1 < d; ++c1)
      for (int c2 = 0; c2 < d; ++c2) {
        const int r = vpos[v1] * d + c1, q = vpos[v2] * d + c2;
        dst[(long long)r * b + q] += S[(k1 * d + c1) * np + k2 * d + c2];
      }
  }
}

// Y[cell][m] = sum_k A[m][k] X[cell][k] in double-float arithmetic on the FP32 pipe (GB300
// issues FP32 at ~60x its FP64 rate).  Each FP64 operand is split into hi + lo floats (48
// significant bits); a product is hi*hi, made exact by an FMA residual, plus the cross terms;
// the sum is kept as an unevaluated pair (s, c) with TwoSum on the leading part.  Relative error
// ~K * 2^-46 of the largest term, against K * 2^-53 for FP64.  64 x 64 output tile per block,
// 4 x 4 per thread, K chunks of 16.
constexpr int DF_T = 64, DF_K = 16;
__global__ void __launch_bounds__(256) df_gemm_kernel(const double* __restrict__ A, int lda, int M, int K,
                                                      const double* __restrict__ X, int x_cs, long long ncols,
                                                      double* __restrict__ Y, int y_cs) {
  __shared__ float Ah[DF_K][DF_T + 1], Al[DF_K][DF_T + 1];
  __shared__ float Xh[DF_K][DF_T + 1], Xl[DF_K][DF_T + 1];
  const long long col0 = (long long)blockIdx.x * DF_T;
  const int m0 = blockIdx.y * DF_T;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { sh[i][j] = 0.f; sl[i][j] = 0.f; }
  for (int k0 = 0; k0 < K; k0 += DF_K) {
    for (int t = threadIdx.x; t < DF_K * DF_T; t += 256) {
      const int r = t / DF_K, q = t - r * DF_K;   // q fastest: coalesced rows of A and X
      const int gm = m0 + r, gk = k0 + q;
      const double av = (gm < M && gk < K) ? A[(size_t)gm * lda + gk] : 0.0;
      const float ah = (float)av;
      Ah[q][r] = ah;
      Al[q][r] = (float)(av - (double)ah);
      const long long gc = col0 + r;
      const double xv = (gc < ncols && gk < K) ? X[gc * x_cs + gk] : 0.0;
      const float xh = (float)xv;
      Xh[q][r] = xh;
      Xl[q][r] = (float)(xv - (double)xh);
    }
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < DF_K; ++q) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { ah[i] = Ah[q][ty + 16 * i]; al[i] = Al[q][ty + 16 * i]; }
#pragma unroll
      for (int j = 0; j < 4; ++j) { bh[j] = Xh[q][tx + 16 * j]; bl[j] = Xl[q][tx + 16 * j]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float p = ah[i] * bh[j];
          const float e = fmaf(ah[i], bh[j], -p) + fmaf(ah[i], bl[j], al[i] * bh[j]);
          const float t = sh[i][j] + p;            // TwoSum(sh, p)
          const float bv = t - sh[i][j];
          const float err = (sh[i][j] - (t - bv)) + (p - bv);
          sh[i][j] = t;
          sl[i][j] += err + e;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const long long gc = col0 + tx + 16 * j;
    if (gc >= ncols) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + ty + 16 * i;
      if (gm < M) Y[gc * y_cs + gm] = (double)sh[i][j] + (double)sl[i][j];
    }
  }
}

}  // namespace

fetidp_status k_assemble_principal(Ctx& c, const int* sigma_dev, int nrb, double* Krr, double* Krp, double* Kpp) {
  const int np = c.n - c.nr;
  ProfScope ps(c, FETIDP_K_SETUP, 0.0, (double)nrb * c.nsnap * 8.0);
  FD_CUDA(cudaMemsetAsync(Krr, 0, sizeof(double) * (size_t)nrb * c.nr * c.nr, c.stream));
  FD_CUDA(cudaMemsetAsync(Krp, 0, sizeof(double) * (size_t)nrb * c.nr * np, c.stream));
  FD_CUDA(cudaMemsetAsync(Kpp, 0, sizeof(double) * (size_t)nrb * np * np, c.stream));
  const double h = 1.0 / c.e, wq = std::pow(0.5 * h, c.d);
  const int NA = 1 << c.d;
  const long long work = (long long)nrb * c.nelem * NA * c.d;
  for (int color = 0; color < NA; ++color) {
    if (c.d == 2)
      assemble_principal_kernel<2><<<grid_for(work, 128), 128, 0, c.stream>>>(
          c.snap, sigma_dev, c.nsnap, nrb, c.e, c.nc, c.n, c.nr, c.perm + c.n, wq, 1.0 / h, Krr, Krp, Kpp, color);
    else
      assemble_principal_kernel<3><<<grid_for(work, 128), 128, 0, c.stream>>>(
          c.snap, sigma_dev, c.nsnap, nrb, c.e, c.nc, c.n, c.nr, c.perm + c.n, wq, 1.0 / h, Krr, Krp, Kpp, color);
    FD_CHECK_LAUNCH();
  }
  return FETIDP_OK;
}

fetidp_status k_spd_inverse_batched(Ctx& c, double* A, long long stride, int n, int lda, int batch, double* work,
                                    int* status) {
  ProfScope ps(c, FETIDP_K_SETUP, 2.0 * batch * (double)n * n * n / 2.0, 16.0 * batch * (double)n * n * n / 2.0);
  double* cbuf[2] = {work, work + (size_t)batch * (n + 1)};
  sweep_init_kernel<<<grid_for((long long)batch * n, 256), 256, 0, c.stream>>>(A, stride, n, lda, batch, cbuf[0],
                                                                               status);
  FD_CHECK_LAUNCH();
  const long long steps_work = (long long)batch * n * ((n + 3) / 4);
  const int g = grid_for(steps_work, 256);
  for (int k = 0; k < n; ++k) {
    sweep_step_kernel<<<g, 256, 0, c.stream>>>(A, stride, n, lda, batch, k, cbuf[k & 1], cbuf[(k + 1) & 1], status);
    FD_CHECK_LAUNCH();
  }
  sweep_finish_kernel<<<grid_for((long long)batch * n * n, 256), 256, 0, c.stream>>>(A, stride, n, lda, batch);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_batched_gemm_nn(Ctx& c, const double* A, long long sa, int lda, const double* B, long long sb,
                                int ldb, double* C, long long sc, int ldc, int M, int N, int K, int batch) {
  ProfScope ps(c, FETIDP_K_SETUP, 2.0 * batch * (double)M * N * K, 8.0 * batch * ((double)M * K + (double)M * N));
  batched_gemm_nn_kernel<<<grid_for((long long)batch * M * N, 128), 128, 0, c.stream>>>(A, sa, lda, B, sb, ldb, C,
                                                                                        sc, ldc, M, N, K, batch);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_batched_block_copy(Ctx& c, const double* in, long long si, int ldi, int r0, int c0, double* out,
                                   long long so, int ldo, int M, int N, int batch, bool transpose) {
  batched_block_copy_kernel<<<grid_for((long long)batch * M * N, 256), 256, 0, c.stream>>>(
      in, si, ldi, r0, c0, out, so, ldo, M, N, batch, transpose);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_batched_diag_sum(Ctx& c, const double* A, long long stride, int lda, int r0, int m, int batch,
                                 double* out) {
  batched_diag_sum_kernel<<<(batch * 32 + 255) / 256, 256, 0, c.stream>>>(A, stride, lda, r0, m, batch, out);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_df_gemm(Ctx& c, const double* A, int lda, int M, int K, const double* X, int x_cs, long long ncols,
                        double* Y, int y_cs) {
  ProfScope ps(c, FETIDP_K_SETUP, 2.0 * M * (double)K * ncols, 8.0 * ((double)M * K + (double)ncols * (K + M)));
  const dim3 grid((unsigned)((ncols + DF_T - 1) / DF_T), (unsigned)((M + DF_T - 1) / DF_T));
  df_gemm_kernel<<<grid, 256, 0, c.stream>>>(A, lda, M, K, X, x_cs, ncols, Y, y_cs);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_batched_gemm(Ctx& c, bool ta, bool tb, int M, int N, int K, double alpha, const double* A,
                             long long sa, int lda, const double* B, long long sb, int ldb, double beta, double* C,
                             long long sc, int ldc, int batch) {
  if (batch <= 0) return FETIDP_OK;
  ProfScope ps(c, FETIDP_K_SETUP, 2.0 * batch * (double)M * N * K, 8.0 * batch * ((double)M * K + (double)K * N));
  const dim3 grid((unsigned)((N + BG_T - 1) / BG_T), (unsigned)((M + BG_T - 1) / BG_T), (unsigned)batch);
  batched_gemm_kernel<<<grid, 256, 0, c.stream>>>(ta, tb, M, N, K, alpha, A, sa, lda, B, sb, ldb, beta, C, sc, ldc);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_batched_symmetrize(Ctx& c, double* A, long long stride, int n, int lda, int batch) {
  if (batch <= 0) return FETIDP_OK;
  batched_symmetrize_kernel<<<grid_for((long long)batch * n * n, 256), 256, 0, c.stream>>>(A, stride, n, lda, batch);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_spp_cells(Ctx& c, const double* Kpp, const double* P, double* out) {
  const int np = c.np;
  spp_cells_kernel<<<grid_for(c.N * np * np, 256), 256, 0, c.stream>>>(c.alpha, c.pi, Kpp, P, c.nrb, np, c.N, out);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_coarse_assemble(Ctx& c, const LatticeSpan& ls, const double* Spp, const int* vslab, const int* vpos,
                                int b, double* A, double* C) {
  const int nck = 1 << c.d;
  const int vdx = ls.geo.nc[0] + 1, vdy = ls.geo.nc[1] + 1;
  for (int color = 0; color < nck; ++color) {
    coarse_assemble_kernel<<<grid_for(ls.ncell * nck * nck, 256), 256, 0, c.stream>>>(
        Spp, ls.ncell, c.d, nck, c.np, ls.geo.nc[0], ls.geo.nc[1], vdx, vdy, vslab, vpos, b, A, C, color);
    FD_CHECK_LAUNCH();
  }
  return FETIDP_OK;
}

fetidp_status k_principal_pairs(Ctx& c, const double* Krp, double* P) {
  const long long total = (long long)c.nrb * c.nrb * c.np * c.np;
  principal_pairs_kernel<<<grid_for(total, 128), 128, 0, c.stream>>>(Krp, c.Urp, c.nrb, c.nr, c.np, P);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

}  // namespace fetidp
