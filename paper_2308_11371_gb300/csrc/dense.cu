// Dense batched FP64 kernels of the setup phase: the principal cells' stiffness blocks
// K_rr, K_rp, K_pp (Eq. 39) assembled from their Gauss-point C_hat, the principal inverses
// K_rr^{-1} and S_dd = F_dd^{-1} (Sec. 3.1.1) by the symmetric sweep operator, and the products
// U_rp = K_rr^{-1} K_rp.
//
// Sweep operator on a symmetric matrix, pivot k (a = A_kk > 0 while A is positive definite):
//   A_kk <- -1/a,   A_ik <- A_ik / a (i != k),   A_ij <- A_ij - A_ik A_kj / a (i, j != k).
// Sweeping every index gives -A^{-1}.  Only the upper triangle is updated, a panel of 32 pivots
// at a time (the block form below), for all matrices of the batch per launch.
#include <climits>
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

// Blocked sweep: sweeping the pivots of a panel P = [k0, k0 + nb) one by one equals the block
// form (Goodnight's SWP on an index set)
//   A_PP <- -A_PP^{-1},   A_iP <- A_iP A_PP^{-1},   A_ij <- A_ij - A_iP A_PP^{-1} A_Pj   (i, j not in P),
// and sweeps of disjoint sets compose.  A_PP is the current (Schur complement) block, positive
// definite while A is.  Each panel is one launch of sweep_panel_kernel (A_PP^{-1} in shared memory
// and W = V A_PP^{-1} for the panel column V = A_:P) and one of sweep_update_kernel (the rank-nb
// update of the upper triangle, 64 x 64 tiles): 2 launches per 32 pivots instead of 32.
constexpr int kSwNb = 32;     // panel width
constexpr int kSwRows = 64;   // largest rows per panel-kernel block and update tile edge

// grid: (row blocks of `rows` <= 64) x batch; 256 threads.  The nb x nb sweep runs on the upper
// triangle (mirrored in shared memory) with one reciprocal per pivot: GB300 issues FP64 at
// 2 FMA/clk/SM, so every redundant FP64 operation of this sequential part is latency.
__global__ void __launch_bounds__(256) sweep_panel_kernel(const double* __restrict__ A, long long stride, int n,
                                                          int lda, int k0, int nb, int rows, int nrb_rows,
                                                          double* __restrict__ V, double* __restrict__ W,
                                                          double* __restrict__ Sinv, int* __restrict__ status) {
  __shared__ double S[kSwNb][kSwNb + 1];
  __shared__ double Vs[kSwRows][kSwNb + 1];
  __shared__ double sinv;
  const int rb = blockIdx.x % nrb_rows;
  const long long b = blockIdx.x / nrb_rows;
  const int tid = threadIdx.x;
  const double* Ab = A + b * stride;
  // the panel block, both triangles from the upper one
  for (int t = tid; t < nb * nb; t += blockDim.x) {
    const int r = t / nb, q = t - (t / nb) * nb;
    S[r][q] = r <= q ? Ab[(long long)(k0 + r) * lda + k0 + q] : Ab[(long long)(k0 + q) * lda + k0 + r];
  }
  // this thread's upper-triangle entries (r <= q), at most 3 of the 528
  constexpr int kMaxE = (kSwNb * (kSwNb + 1) / 2 + 255) / 256;
  int er[kMaxE], eq[kMaxE], ne = 0;
  for (int t = tid; t < nb * (nb + 1) / 2 && ne < kMaxE; t += blockDim.x) {
    int r = 0, u = t;
    while (u >= nb - r) { u -= nb - r; ++r; }
    er[ne] = r;
    eq[ne] = r + u;
    ++ne;
  }
  __syncthreads();
  // sweep of the nb x nb block: S <- -A_PP^{-1}
  bool bad = false;
  for (int p = 0; p < nb; ++p) {
    if (tid == 0) {
      const double a = S[p][p];
      bad |= !(a > 0.0);
      sinv = 1.0 / a;
    }
    __syncthreads();
    const double inv = sinv;
    double nv[kMaxE];
#pragma unroll
    for (int e = 0; e < kMaxE; ++e) {
      if (e >= ne) break;
      const int r = er[e], q = eq[e];
      double v;
      if (r == p && q == p) v = -inv;
      else if (r == p) v = S[p][q] * inv;
      else if (q == p) v = S[r][p] * inv;
      else v = fma(-S[r][p] * inv, S[p][q], S[r][q]);
      nv[e] = v;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kMaxE; ++e) {
      if (e >= ne) break;
      S[er[e]][eq[e]] = nv[e];
      S[eq[e]][er[e]] = nv[e];
    }
    __syncthreads();
  }
  if (bad && rb == 0) atomicExch(status, 1);
  // V rows of this block: V_i = A_iP (zero for i in P, unused there)
  const int i0 = rb * rows;
  if (i0 + rows <= k0) {   // rows above the panel: A[i][k0 + p], contiguous in p
    for (int t = tid; t < rows * nb; t += blockDim.x) {
      const int li = t / nb, p = t - (t / nb) * nb;
      Vs[li][p] = Ab[(long long)(i0 + li) * lda + k0 + p];
    }
  } else {                 // rows at or below the panel: A[k0 + p][i], contiguous in i
    for (int t = tid; t < rows * nb; t += blockDim.x) {
      const int li = t % rows, p = t / rows, i = i0 + li;
      double v = 0.0;
      if (i < n) {
        if (i < k0) v = Ab[(long long)i * lda + k0 + p];
        else if (i >= k0 + nb) v = Ab[(long long)(k0 + p) * lda + i];
      }
      Vs[li][p] = v;
    }
  }
  __syncthreads();
  // W_i = V_i A_PP^{-1} = -V_i S; written with V (layout [b][i][p], p fastest)
  double* Vb = V + b * (long long)n * kSwNb;
  double* Wb = W + b * (long long)n * kSwNb;
  for (int t = tid; t < rows * nb; t += blockDim.x) {
    const int li = t / nb, p = t - (t / nb) * nb, i = i0 + li;
    if (i >= n) continue;
    double w = 0.0;
    for (int q = 0; q < nb; ++q) w = fma(Vs[li][q], S[q][p], w);
    Vb[(long long)i * kSwNb + p] = Vs[li][p];
    Wb[(long long)i * kSwNb + p] = -w;
  }
  if (rb == 0)
    for (int t = tid; t < nb * nb; t += blockDim.x)
      Sinv[b * kSwNb * kSwNb + (t / nb) * kSwNb + t % nb] = -S[t / nb][t % nb];
}

// Rank-nb update of the upper triangle for panel P, one TS x TS tile (I <= J) per block, 256
// threads of (TS/16) x (TS/16) entries.  grid: upper tiles x batch.
template <int TS>
__global__ void __launch_bounds__(256) sweep_update_kernel(double* __restrict__ A, long long stride, int n, int lda,
                                                           int k0, int nb, int ntile,
                                                           const double* __restrict__ V,
                                                           const double* __restrict__ W,
                                                           const double* __restrict__ Sinv) {
  constexpr int E = TS / 16;
  __shared__ double Ws[kSwNb][TS];
  __shared__ double Vs[kSwNb][TS];
  const int nup = ntile * (ntile + 1) / 2;
  const long long b = blockIdx.x / nup;
  int t = blockIdx.x - (int)(b * nup), I = 0;
  while (t >= ntile - I) { t -= ntile - I; ++I; }
  const int J = I + t;
  const int tid = threadIdx.x;
  const double* Wb = W + b * (long long)n * kSwNb;
  const double* Vb = V + b * (long long)n * kSwNb;
  for (int e = tid; e < TS * kSwNb; e += blockDim.x) {
    const int l = e / kSwNb, p = e - (e / kSwNb) * kSwNb;
    const int i = I * TS + l, j = J * TS + l;
    Ws[p][l] = (i < n && p < nb) ? Wb[(long long)i * kSwNb + p] : 0.0;
    Vs[p][l] = (j < n && p < nb) ? Vb[(long long)j * kSwNb + p] : 0.0;
  }
  __syncthreads();
  const int ty = tid / 16, tx = tid - (tid / 16) * 16;
  double acc[E][E] = {};
  for (int p = 0; p < nb; ++p) {
    double w[E], v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) { w[r] = Ws[p][ty * E + r]; v[r] = Vs[p][tx * E + r]; }
#pragma unroll
    for (int r = 0; r < E; ++r)
#pragma unroll
      for (int q = 0; q < E; ++q) acc[r][q] = fma(w[r], v[q], acc[r][q]);
  }
  double* Ab = A + b * stride;
  const double* Sb = Sinv + b * kSwNb * kSwNb;
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = I * TS + ty * E + r;
    if (i >= n) continue;
    const bool pi = i >= k0 && i < k0 + nb;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int j = J * TS + tx * E + q;
      if (j >= n || j < i) continue;
      const bool pj = j >= k0 && j < k0 + nb;
      double* a = Ab + (long long)i * lda + j;
      if (!pi && !pj) *a -= acc[r][q];
      else if (!pi) *a = Wb[(long long)i * kSwNb + (j - k0)];
      else if (!pj) *a = Wb[(long long)j * kSwNb + (i - k0)];
      else *a = -Sb[(i - k0) * kSwNb + (j - k0)];
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
// issues FP32 at ~60x its FP64 rate).  Each FP64 operand is split once (df_split_kernel) into
// float planes hi = fl(v), lo = fl(v - hi) (48 significant bits), zero-padded to whole tiles.  A
// term is hi*hi, made exact by an FMA residual, plus the two cross products; the sum is kept as
// an unevaluated pair (s, c) with TwoSum on the leading part: 12 FP32 instructions per term.
// Relative error ~K * 2^-46 of the largest term, against K * 2^-53 for FP64.  64 x 64 output
// tile per block, 4 x 4 per thread, K chunks of 16 staged by cp.async in two buffers.
constexpr int DF_T = 64, DF_K = 16, DF_LD = 20;   // smem rows of 16 floats + 4 pad (16-byte aligned)

__global__ void df_split_kernel(const double* __restrict__ src, long long rows, int cols, long long src_ld,
                                long long rows_p, int ld_p, float* __restrict__ hi, float* __restrict__ lo) {
  const long long total = rows_p * ld_p;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / ld_p;
    const int q = (int)(t - r * ld_p);
    const double v = (r < rows && q < cols) ? src[r * src_ld + q] : 0.0;
    const float h = (float)v;
    hi[t] = h;
    lo[t] = (float)(v - (double)h);
  }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

__global__ void __launch_bounds__(256, 2) df_gemm_kernel(const float* __restrict__ Ah, const float* __restrict__ Al,
                                                      const float* __restrict__ Xh, const float* __restrict__ Xl,
                                                      int ldk, int nkc, int M, long long ncols,
                                                      double* __restrict__ Y, int y_cs) {
  __shared__ __align__(16) float sA[2][2][DF_T][DF_LD];   // [buffer][hi, lo][row m][k]
  __shared__ __align__(16) float sX[2][2][DF_T][DF_LD];   // [buffer][hi, lo][column][k]
  // row tiles fastest: the blocks resident together share their X (snapshot) tiles, which are
  // then read from DRAM about once, while the table planes stay in L2
  const long long m0 = (long long)blockIdx.x * DF_T;
  const long long col0 = (long long)blockIdx.y * DF_T;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // one chunk: 4 planes x 64 rows x 4 quads of 16 bytes = 1024 copies, 4 per thread
  auto load = [&](int buf, int kc) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u, plane = e >> 8, row = (e >> 2) & 63, quad = e & 3;
      const long long off = (long long)kc * DF_K + quad * 4;
      switch (plane) {
        case 0: cp_async16(&sA[buf][0][row][quad * 4], Ah + (m0 + row) * ldk + off); break;
        case 1: cp_async16(&sA[buf][1][row][quad * 4], Al + (m0 + row) * ldk + off); break;
        case 2: cp_async16(&sX[buf][0][row][quad * 4], Xh + (col0 + row) * ldk + off); break;
        default: cp_async16(&sX[buf][1][row][quad * 4], Xl + (col0 + row) * ldk + off); break;
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  float s[4][4], cl[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { s[i][j] = 0.f; cl[i][j] = 0.f; }
  load(0, 0);
  for (int kc = 0; kc < nkc; ++kc) {
    const int buf = kc & 1;
    if (kc + 1 < nkc) {
      load(buf ^ 1, kc + 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
#pragma unroll
    for (int q4 = 0; q4 < DF_K; q4 += 4) {
      float4 bh[4], bl[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        bh[j] = *reinterpret_cast<const float4*>(&sX[buf][0][tx + 16 * j][q4]);
        bl[j] = *reinterpret_cast<const float4*>(&sX[buf][1][tx + 16 * j][q4]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 ah4 = *reinterpret_cast<const float4*>(&sA[buf][0][ty + 16 * i][q4]);
        const float4 al4 = *reinterpret_cast<const float4*>(&sA[buf][1][ty + 16 * i][q4]);
        const float ah[4] = {ah4.x, ah4.y, ah4.z, ah4.w}, al[4] = {al4.x, al4.y, al4.z, al4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float xh[4] = {bh[j].x, bh[j].y, bh[j].z, bh[j].w}, xl[4] = {bl[j].x, bl[j].y, bl[j].z, bl[j].w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float p = ah[q] * xh[q];
            const float e = fmaf(ah[q], xh[q], -p);     // exact: p + e = ah * xh
            float c = fmaf(ah[q], xl[q], cl[i][j]);
            c = fmaf(al[q], xh[q], c);
            const float t = s[i][j] + p;                // TwoSum(s, p)
            const float bv = t - s[i][j];
            const float err = (s[i][j] - (t - bv)) + (p - bv);
            s[i][j] = t;
            cl[i][j] = c + (err + e);
          }
        }
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
      const long long gm = m0 + ty + 16 * i;
      if (gm < M) Y[gc * y_cs + gm] = (double)s[i][j] + (double)cl[i][j];
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

fetidp_status k_spd_inverse_batched(Ctx& c, double* A, long long stride, int n, int lda, int batch, int* status) {
  ProfScope ps(c, FETIDP_K_SWEEP, 2.0 * batch * (double)n * n * n / 2.0, 16.0 * batch * (double)n * n * n / 2.0);
  if (n <= 0 || batch <= 0) return FETIDP_OK;
  double* buf = nullptr;
  const size_t vw = (size_t)batch * n * kSwNb;
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&buf), sizeof(double) * (2 * vw + (size_t)batch * kSwNb * kSwNb)));
  double *V = buf, *W = buf + vw, *Sinv = buf + 2 * vw;
  // 64-row blocks and tiles while they fill the GPU, else 32 (small batches of the coarse levels)
  const int n64 = (n + 63) / 64;
  const bool wide = (long long)n64 * (n64 + 1) / 2 * batch >= 2 * 152;
  const int ts = wide ? 64 : 32;
  const int nrows = (n + ts - 1) / ts;
  const long long panel_blocks = (long long)nrows * batch;
  const long long update_blocks = (long long)nrows * (nrows + 1) / 2 * batch;
  fetidp_status st = FETIDP_OK;
  if (panel_blocks > INT_MAX || update_blocks > INT_MAX) st = FETIDP_EINVAL;
  for (int k0 = 0; k0 < n && st == FETIDP_OK; k0 += kSwNb) {
    const int nb = n - k0 < kSwNb ? n - k0 : kSwNb;
    sweep_panel_kernel<<<(int)panel_blocks, 256, 0, c.stream>>>(A, stride, n, lda, k0, nb, ts, nrows, V, W, Sinv,
                                                                status);
    count_launch();
    if (wide)
      sweep_update_kernel<64><<<(int)update_blocks, 256, 0, c.stream>>>(A, stride, n, lda, k0, nb, nrows, V, W, Sinv);
    else
      sweep_update_kernel<32><<<(int)update_blocks, 256, 0, c.stream>>>(A, stride, n, lda, k0, nb, nrows, V, W, Sinv);
    count_launch();
    if (cudaPeekAtLastError() != cudaSuccess) st = FETIDP_ECUDA;
  }
  if (st == FETIDP_OK) {
    sweep_finish_kernel<<<grid_for((long long)batch * n * n, 256), 256, 0, c.stream>>>(A, stride, n, lda, batch);
    count_launch();
    if (cudaPeekAtLastError() != cudaSuccess) st = FETIDP_ECUDA;
  }
  tmp_free(c, buf);
  if (st == FETIDP_ECUDA) set_error(std::string("kernel launch: ") + cudaGetErrorString(cudaGetLastError()));
  else if (st == FETIDP_EINVAL) set_error("SPD inverse batch too large for one launch");
  return st;
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

int df_pad_rows(long long rows) { return (int)((rows + DF_T - 1) / DF_T * DF_T); }
int df_pad_k(int K) { return (K + DF_K - 1) / DF_K * DF_K; }

// A given as padded planes [df_pad_rows(M)][df_pad_k(K)]; X split here.
fetidp_status k_df_gemm_planes(Ctx& c, const float* Ah, const float* Al, int M, int K, const double* X, int x_cs,
                               long long ncols, double* Y, int y_cs) {
  if (M <= 0 || ncols <= 0) return FETIDP_OK;
  const int Kp = df_pad_k(K);
  const long long Mp = df_pad_rows(M), Np = (ncols + DF_T - 1) / DF_T * DF_T;
  if (Np / DF_T > 65535) {
    set_error("trace contraction: too many cells for one launch");
    return FETIDP_EINVAL;
  }
  float* buf = nullptr;
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&buf), sizeof(float) * 2 * (size_t)Np * Kp));
  float *Xh = buf, *Xl = buf + (size_t)Np * Kp;
  fetidp_status st = FETIDP_OK;
  {
    ProfScope ps(c, FETIDP_K_SETUP, 0.0, 16.0 * (double)ncols * K);
    df_split_kernel<<<grid_for(Np * Kp, 256), 256, 0, c.stream>>>(X, ncols, K, x_cs, Np, Kp, Xh, Xl);
    count_launch();
  }
  {
    ProfScope ps(c, FETIDP_K_TRACES, 2.0 * M * (double)K * ncols, 8.0 * ((double)M * K + (double)ncols * (K + M)));
    const dim3 grid((unsigned)(Mp / DF_T), (unsigned)(Np / DF_T));
    df_gemm_kernel<<<grid, 256, 0, c.stream>>>(Ah, Al, Xh, Xl, Kp, Kp / DF_K, M, ncols, Y, y_cs);
    count_launch();
  }
  if (cudaPeekAtLastError() != cudaSuccess) {
    set_error(std::string("kernel launch: ") + cudaGetErrorString(cudaGetLastError()));
    st = FETIDP_ECUDA;
  }
  tmp_free(c, buf);
  return st;
}

fetidp_status k_df_gemm(Ctx& c, const double* A, int lda, int M, int K, const double* X, int x_cs, long long ncols,
                        double* Y, int y_cs) {
  if (M <= 0 || ncols <= 0) return FETIDP_OK;
  const int Kp = df_pad_k(K);
  const long long Mp = df_pad_rows(M);
  float* buf = nullptr;
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&buf), sizeof(float) * 2 * (size_t)Mp * Kp));
  {
    ProfScope ps(c, FETIDP_K_SETUP, 0.0, 16.0 * (double)M * K);
    df_split_kernel<<<grid_for(Mp * Kp, 256), 256, 0, c.stream>>>(A, M, K, lda, Mp, Kp, buf, buf + (size_t)Mp * Kp);
    count_launch();
  }
  const fetidp_status st = k_df_gemm_planes(c, buf, buf + (size_t)Mp * Kp, M, K, X, x_cs, ncols, Y, y_cs);
  tmp_free(c, buf);
  return st;
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
