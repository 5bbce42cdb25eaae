// Cell-level FP64 kernels of the hot path.
//
// * snapshots: C_hat (Eq. 52) at every Gauss point of every cell; these are
//   the snapshot vectors of the greedy (Sec. 4.2.2) and the per-Gauss-point
//   macro data that the matrix-free K_s reads.
// * apply_K: y = K_s u (Eq. 5a through Eq. 52), matrix-free Q1 element loop,
//   elements processed in 2^d colours so that no two threads of a colour
//   touch the same node (deterministic, no atomics).
// * cell_gemv: per-cell dense operators assembled from the ROM (Eq. 43).
// * grouped_gemm: Y = sum_k c_k (A_k X), one principal operator A_k serving
//   every cell's column (Remark 7; Eq. 46a with separate outputs).
// * gram_solve: Eq. 46b with diagonal-pivoted Cholesky.
// * grad: adjoint compliance gradient -w^T dK_s/dr_s u.
#include <algorithm>

#include "common.cuh"

namespace fetidp {

namespace {

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

__global__ void snapshot_kernel(Geo g, const double* __restrict__ r_cell, long long ncell,
                                int nelem, int ngp, int nc, double* __restrict__ snap) {
  const long long total = ncell * nelem * ngp;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long cell = t / (nelem * ngp);
    const int rem = (int)(t - cell * nelem * ngp);
    const int el = rem / ngp, gp = rem - el * ngp;
    const int cx = (int)(cell % g.nc[0]);
    const int cy = (int)((cell / g.nc[0]) % g.nc[1]);
    const int cz = (int)(cell / ((long long)g.nc[0] * g.nc[1]));
    const int ex = el % g.e, ey = (el / g.e) % g.e, ez = el / (g.e * g.e);
    double eta[3], xi[3], J[3][3];
    gauss_point(g, cx, cy, cz, ex, ey, ez, gp, eta, xi);
    macro_jacobian(g, xi, J);
    const double E = youngs(g, strut_distance(g, eta), r_cell[cell]);
    double out[45];
    chat_upper(g.dim, g.nu, J, E, out);
    double* dst = snap + cell * (long long)nelem * ngp * nc + (long long)rem * nc;
    for (int k = 0; k < nc; ++k) dst[k] = out[k];
  }
}

// Element contribution f_e = sum_gp w dN^T C_hat dN u_e for one element and one vector.
template <int D, typename T>
__device__ __forceinline__ void element_apply(const double* __restrict__ chat_el, int nc,
                                              T wq, T inv_h, const T* ue, T* fe) {
  constexpr int NA = 1 << D;
  constexpr int NI = D * D;
  for (int k = 0; k < NA * D; ++k) fe[k] = T(0);
  for (int gp = 0; gp < NA; ++gp) {
    T t[D];
    for (int k = 0; k < D; ++k) t[k] = (T)gauss_t((gp >> k) & 1);
    // dN_A / dxi_a
    T dN[NA][D];
    for (int A = 0; A < NA; ++A) {
      for (int a = 0; a < D; ++a) {
        T v = inv_h;
        for (int k = 0; k < D; ++k) {
          const int off = (A >> k) & 1;
          if (k == a) v *= off ? T(1) : T(-1);
          else v *= off ? t[k] : T(1) - t[k];
        }
        dN[A][a] = v;
      }
    }
    T G[NI];
    for (int I = 0; I < NI; ++I) G[I] = T(0);
    for (int A = 0; A < NA; ++A)
      for (int i = 0; i < D; ++i)
        for (int a = 0; a < D; ++a) G[i * D + a] += ue[A * D + i] * dN[A][a];
    T S[NI];
    for (int I = 0; I < NI; ++I) S[I] = T(0);
    const double* C = chat_el + gp * nc;
    int q = 0;
    for (int I = 0; I < NI; ++I) {
      for (int J = I; J < NI; ++J) {
        const T cij = (T)C[q++];
        S[I] += cij * G[J];
        if (J != I) S[J] += cij * G[I];
      }
    }
    for (int A = 0; A < NA; ++A)
      for (int i = 0; i < D; ++i) {
        T v = T(0);
        for (int a = 0; a < D; ++a) v += dN[A][a] * S[i * D + a];
        fe[A * D + i] += wq * v;
      }
  }
}

// One block per (rhs, cell) column; vectors of the column processed VB at a time.
// T = double (FP64 path) or float (the Eq. 46b products of the mixed path).
template <int D, typename T>
__global__ void apply_K_kernel(int e, long long ncell, int n, int len, const int* __restrict__ perm,
                               const int* __restrict__ iperm, bool idp, const T* __restrict__ u,
                               long long u_rs, int u_cs, T* __restrict__ y, long long y_rs,
                               int y_cs, int nvec, int VB, const double* __restrict__ chat, int nc,
                               T wq, T inv_h, long long u_ext, long long y_ext) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  constexpr int NA = 1 << D;
  const long long col = blockIdx.x;
  const int rhs = (int)(col / ncell);
  const long long cell = col - (long long)rhs * ncell;
  const T* uc = u + rhs * u_rs + cell * u_cs;
  T* yc = y + rhs * y_rs + cell * y_cs;
  const double* chat_cell = chat + cell * (long long)nc * NA * (e * e * (D == 3 ? e : 1));
  T* us = sm;
  T* ys = sm + (size_t)VB * n;
  const int ecount[3] = {e, e, D == 3 ? e : 1};
  for (int v0 = 0; v0 < nvec; v0 += VB) {
    const int vb = min(VB, nvec - v0);
    for (int t = threadIdx.x; t < vb * n; t += blockDim.x) {
      const int v = t / n, i = t - v * n;     // i natural index
      T val;
      if (idp) {
        const int li = iperm[i];
        val = (li < len && FD_INB(rhs * u_rs + cell * u_cs + (long long)(v0 + v) * len + li, u_ext, 201))
                  ? uc[(size_t)(v0 + v) * len + li]
                  : T(0);
      } else {
        val = FD_INB(rhs * u_rs + cell * u_cs + (long long)(v0 + v) * len + i, u_ext, 201)
                  ? uc[(size_t)(v0 + v) * len + i]
                  : T(0);
      }
      us[t] = val;
      ys[t] = T(0);
    }
    __syncthreads();
    for (int color = 0; color < NA; ++color) {
      int cnt[3], par[3];
      int nel = 1;
      for (int k = 0; k < 3; ++k) {
        par[k] = (k < D) ? ((color >> k) & 1) : 0;
        cnt[k] = (k < D) ? (ecount[k] - par[k] + 1) / 2 : 1;
        nel *= cnt[k];
      }
      for (int t = threadIdx.x; t < vb * nel; t += blockDim.x) {
        const int v = t / nel, q = t - v * nel;
        const int qx = q % cnt[0], qy = (q / cnt[0]) % cnt[1], qz = q / (cnt[0] * cnt[1]);
        const int ex = par[0] + 2 * qx, ey = par[1] + 2 * qy, ez = par[2] + 2 * qz;
        const int el = ex + e * (ey + e * ez);
        int nodes[NA];
        for (int A = 0; A < NA; ++A) {
          const int ax = A & 1, ay = (A >> 1) & 1, az = (A >> 2) & 1;
          nodes[A] = (ex + ax) + (e + 1) * ((ey + ay) + (e + 1) * (D == 3 ? (ez + az) : 0));
        }
        T ue[NA * D], fe[NA * D];
        const T* uv = us + (size_t)v * n;
        for (int A = 0; A < NA; ++A)
          for (int i = 0; i < D; ++i) ue[A * D + i] = uv[nodes[A] * D + i];
        element_apply<D, T>(chat_cell + (size_t)el * NA * nc, nc, wq, inv_h, ue, fe);
        T* yv = ys + (size_t)v * n;
        for (int A = 0; A < NA; ++A)
          for (int i = 0; i < D; ++i) yv[nodes[A] * D + i] += fe[A * D + i];
      }
      __syncthreads();
    }
    for (int t = threadIdx.x; t < vb * len; t += blockDim.x) {
      const int v = t / len, li = t - v * len;
      const int nat = idp ? perm[li] : li;
      if (FD_INB(rhs * y_rs + cell * y_cs + (long long)(v0 + v) * len + li, y_ext, 202))
        yc[(size_t)(v0 + v) * len + li] = ys[(size_t)v * n + nat];
    }
    __syncthreads();
  }
}

// Per-cell dense operators: y[rhs,cell] = alpha M_cell x[rhs,cell] + beta y, M_cell at
// mats + cell*mstride with row stride ld (sub-blocks of the per-cell ROM operators).
constexpr int kMaxRhsGemv = 8;
__global__ void cell_gemv_kernel(const double* __restrict__ mats, long long mstride, int ld,
                                 int mrows, int mcols, const double* __restrict__ x, long long x_rs,
                                 int x_cs, double* __restrict__ y, long long y_rs, int y_cs,
                                 double alpha, double beta, int nrhs) {
  extern __shared__ double xs[];   // [nrhs][mcols]
  const long long cell = blockIdx.x;
  for (int t = threadIdx.x; t < nrhs * mcols; t += blockDim.x) {
    const int r = t / mcols, q = t - r * mcols;
    xs[t] = x[r * x_rs + cell * x_cs + q];
  }
  __syncthreads();
  const double* M = mats + cell * mstride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int row = warp; row < mrows; row += nw) {
    for (int r0 = 0; r0 < nrhs; r0 += kMaxRhsGemv) {
      const int rb = min(kMaxRhsGemv, nrhs - r0);
      double acc[kMaxRhsGemv];
      for (int r = 0; r < kMaxRhsGemv; ++r) acc[r] = 0.0;
      for (int q = lane; q < mcols; q += 32) {
        const double mv = M[(size_t)row * ld + q];
        for (int r = 0; r < rb; ++r) acc[r] += mv * xs[(r0 + r) * mcols + q];
      }
      for (int r = 0; r < rb; ++r) {
        double s = acc[r];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
          double* dst = y + (r0 + r) * y_rs + cell * y_cs + row;
          *dst = (beta == 0.0) ? alpha * s : alpha * s + beta * (*dst);
        }
      }
    }
  }
}

// Grouped FP64 GEMM, 64x64 output tile per block, 4x4 per thread, K chunks of 16.
constexpr int GT = 64, GK = 16;
__global__ void __launch_bounds__(256) grouped_gemm_kernel(
    const double* __restrict__ A, long long a_stride_k, int lda, int M, int K, int nk,
    const double* __restrict__ X, long long x_rs, int x_cs, double* __restrict__ Y, long long y_rs,
    int y_cs, const double* __restrict__ coef, double alpha, double beta, long long ncell, int nrhs,
    bool separate, long long y_k_stride) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Xs[GK][GT + 1];
  const long long ncols = ncell * nrhs;
  const long long col0 = (long long)blockIdx.x * GT;
  const int m0 = blockIdx.y * GT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads
  double tot[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) tot[i][j] = 0.0;
  for (int k = 0; k < nk; ++k) {
    const double* Ak = A + k * a_stride_k;
    double acc[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int kk0 = 0; kk0 < K; kk0 += GK) {
      for (int t = threadIdx.x; t < GK * GT; t += 256) {
        const int r = t / GK, q = t - r * GK;     // A: row r, k q  (q fastest -> coalesced rows)
        const int gm = m0 + r, gk = kk0 + q;
        As[q][r] = (gm < M && gk < K) ? Ak[(size_t)gm * lda + gk] : 0.0;
        const long long gc = col0 + r;            // X: column r, k q
        double xv = 0.0;
        if (gc < ncols && gk < K) {
          const int rhs = (int)(gc / ncell);
          const long long cell = gc - (long long)rhs * ncell;
          xv = X[rhs * x_rs + cell * x_cs + gk];
        }
        Xs[q][r] = xv;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < GK; ++q) {
        double a[4], b[4];
        for (int i = 0; i < 4; ++i) a[i] = As[q][ty + 16 * i];
        for (int j = 0; j < 4; ++j) b[j] = Xs[q][tx + 16 * j];
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
      }
      __syncthreads();
    }
    if (separate) {
      for (int j = 0; j < 4; ++j) {
        const long long gc = col0 + tx + 16 * j;
        if (gc >= ncols) continue;
        const int rhs = (int)(gc / ncell);
        const long long cell = gc - (long long)rhs * ncell;
        double* yc = Y + k * y_k_stride + rhs * y_rs + cell * y_cs;
        for (int i = 0; i < 4; ++i) {
          const int gm = m0 + ty + 16 * i;
          if (gm < M) yc[gm] = alpha * acc[i][j];
        }
      }
    } else {
      for (int j = 0; j < 4; ++j) {
        const long long gc = col0 + tx + 16 * j;
        double cf = 1.0;
        if (coef != nullptr && gc < ncols) {
          const long long cell = gc % ncell;
          cf = coef[cell * nk + k];
        }
        for (int i = 0; i < 4; ++i) tot[i][j] += cf * acc[i][j];
      }
    }
  }
  if (!separate) {
    for (int j = 0; j < 4; ++j) {
      const long long gc = col0 + tx + 16 * j;
      if (gc >= ncols) continue;
      const int rhs = (int)(gc / ncell);
      const long long cell = gc - (long long)rhs * ncell;
      double* yc = Y + rhs * y_rs + cell * y_cs;
      for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm < M) yc[gm] = (beta == 0.0) ? alpha * tot[i][j] : alpha * tot[i][j] + beta * yc[gm];
      }
    }
  }
}

// Eq. 46b for one (rhs, cell) per warp: G = R^T (K R) and h = R^T v by lane-strided dot
// products with a shuffle reduction, then lane 0 runs the diagonal-pivoted Cholesky and the
// triangular solves on the warp's shared-memory scratch, and the warp forms x = R c.  Pivots
// below drop_rel * max diag(G) are dropped (coefficient 0).
// Scratch per warp (doubles): G, S, L (nrb x nrb each), h, y, c, pivot column (nrb each),
// nrb ints (pivot order), 2 scalars (current pivot, its Schur diagonal), then two staging
// tiles of R and K R (nrb x 32 values of the basis type each, counted in doubles).
constexpr int kMaxRb = 64;
constexpr int kGramChunk = 32;
__host__ __device__ inline int gram_warp_doubles(int nrb, int tb_bytes) {
  return 3 * nrb * nrb + 5 * nrb + 2 + (2 * nrb * kGramChunk * tb_bytes + 7) / 8;
}

template <typename TB>
__global__ void gram_warp_kernel(const TB* __restrict__ R, const TB* __restrict__ KR,
                                 const double* __restrict__ v, long long v_rs, int v_cs,
                                 double* __restrict__ x, long long x_rs, int x_cs, int nr, int nrb,
                                 long long ncell, int nrhs, double drop_rel) {
  extern __shared__ double gwsm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long col = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
  if (col >= ncell * nrhs) return;                  // the whole warp leaves together
  const int nb2 = nrb * nrb;
  double* G = gwsm + (size_t)wib * gram_warp_doubles(nrb, (int)sizeof(TB));
  double* S = G + nb2;
  double* Lm = S + nb2;
  double* hs = Lm + nb2;
  double* ys = hs + nrb;
  double* cs = ys + nrb;
  double* colv = cs + nrb;
  int* piv = reinterpret_cast<int*>(colv + nrb);    // nrb ints in the next nrb doubles
  double* sc = colv + 2 * nrb;                      // [0] pivot index, [1] its Schur diagonal
  TB* Rt = reinterpret_cast<TB*>(sc + 2);           // nrb x kGramChunk
  TB* Kt = Rt + nrb * kGramChunk;                   // nrb x kGramChunk
  const int rhs = (int)(col / ncell);
  const long long cell = col - (long long)rhs * ncell;
  const TB* Rc = R + col * (long long)nrb * nr;
  const TB* KRc = KR + col * (long long)nrb * nr;
  const double* vc = v + rhs * v_rs + cell * v_cs;
  // G (upper triangle, row-major pair index p) and h: each lane owns pairs p = lane + 32 t and
  // h[lane + 32 t]; chunks of 32 entries of every basis vector are staged in shared memory
  // (coalesced loads), products in the basis type, chunk sums accumulated in FP64.
  const int npair = nrb * (nrb + 1) / 2;
  for (int p = lane; p < npair; p += 32) {
    int i = 0, rem = p;
    while (rem >= nrb - i) { rem -= nrb - i; ++i; }
    G[i * nrb + i + rem] = 0.0;
  }
  for (int i = lane; i < nrb; i += 32) hs[i] = 0.0;
  for (int q0 = 0; q0 < nr; q0 += kGramChunk) {
    const int qn = min(kGramChunk, nr - q0);
    __syncwarp();
    for (int i = 0; i < nrb; ++i) {
      Rt[i * kGramChunk + lane] = lane < qn ? Rc[(size_t)i * nr + q0 + lane] : TB(0);
      Kt[i * kGramChunk + lane] = lane < qn ? KRc[(size_t)i * nr + q0 + lane] : TB(0);
    }
    const double vq = lane < qn ? vc[q0 + lane] : 0.0;
    __syncwarp();
    for (int p = lane; p < npair; p += 32) {
      int i = 0, rem = p;
      while (rem >= nrb - i) { rem -= nrb - i; ++i; }
      const int j = i + rem;
      TB acc = TB(0);
      for (int q = 0; q < kGramChunk; ++q) acc += Rt[i * kGramChunk + q] * Kt[j * kGramChunk + q];
      G[i * nrb + j] += (double)acc;
    }
    for (int i = 0; i < nrb; ++i) {          // h_i += sum_q R_iq v_q (warp reduction)
      double s = (double)Rt[i * kGramChunk + lane] * vq;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) hs[i] += s;
    }
  }
  __syncwarp();
  for (int p = lane; p < npair; p += 32) {    // mirror the upper triangle
    int i = 0, rem = p;
    while (rem >= nrb - i) { rem -= nrb - i; ++i; }
    G[(i + rem) * nrb + i] = G[i * nrb + i + rem];
  }
  __syncwarp();
  for (int t = lane; t < nb2; t += 32) S[t] = G[t];
  double dmax = 0.0;
  for (int i = 0; i < nrb; ++i) dmax = fmax(dmax, G[i * nrb + i]);
  unsigned long long used = 0ull;                   // identical in every lane
  int np = 0;
  __syncwarp();
  while (np < nrb) {
    if (lane == 0) {
      // largest remaining Schur diagonal, lowest index on ties
      int jb = -1;
      double best = 0.0;
      for (int i = 0; i < nrb; ++i) {
        if ((used >> i) & 1ull) continue;
        const double dv = S[i * nrb + i];
        if (jb < 0 || dv > best) { best = dv; jb = i; }
      }
      sc[0] = (double)jb;
      sc[1] = best;
    }
    __syncwarp();
    const int jb = (int)sc[0];
    const double best = sc[1];
    if (jb < 0 || jb >= nrb || !(best > drop_rel * dmax)) break;   // uniform across the warp
    used |= 1ull << jb;
    if (lane == 0) piv[np] = jb;
    ++np;
    const double inv = 1.0 / sqrt(best);
    for (int i = lane; i < nrb; i += 32) colv[i] = S[i * nrb + jb] * inv;
    __syncwarp();
    for (int i = lane; i < nrb; i += 32)             // each lane owns rows i
      for (int j = 0; j < nrb; ++j) S[i * nrb + j] -= colv[i] * colv[j];
    __syncwarp();
  }
  if (lane == 0) {
    // Cholesky of G restricted to the pivots (pivot order)
    for (int a = 0; a < np; ++a)
      for (int b = 0; b <= a; ++b) {
        double s = G[piv[a] * nrb + piv[b]];
        for (int k = 0; k < b; ++k) s -= Lm[a * nrb + k] * Lm[b * nrb + k];
        Lm[a * nrb + b] = (a == b) ? sqrt(s) : s / Lm[b * nrb + b];
      }
    for (int a = 0; a < np; ++a) {
      double s = hs[piv[a]];
      for (int k = 0; k < a; ++k) s -= Lm[a * nrb + k] * ys[k];
      ys[a] = s / Lm[a * nrb + a];
    }
    for (int i = 0; i < nrb; ++i) cs[i] = 0.0;
    for (int a = np - 1; a >= 0; --a) {
      double s = ys[a];
      for (int k = a + 1; k < np; ++k) s -= Lm[k * nrb + a] * cs[piv[k]];
      cs[piv[a]] = s / Lm[a * nrb + a];
    }
  }
  __syncwarp();
  double* xc = x + rhs * x_rs + cell * x_cs;
  for (int q = lane; q < nr; q += 32) {
    double s = 0.0;
    for (int i = 0; i < nrb; ++i) s += cs[i] * (double)Rc[(size_t)i * nr + q];
    xc[q] = s;
  }
}

// g[rhs][cell] = - sum_e sum_gp w G(w)^T dC_hat/dr G(u), one block per (rhs, cell).
template <int D>
__global__ void grad_kernel(Geo g, const double* __restrict__ r_cell, long long ncell, int n,
                            const double* __restrict__ u, const double* __restrict__ w,
                            double* __restrict__ out, double wq, double inv_h) {
  extern __shared__ double sm[];
  constexpr int NA = 1 << D;
  constexpr int NI = D * D;
  const long long col = blockIdx.x;
  const int rhs = (int)(col / ncell);
  const long long cell = col - (long long)rhs * ncell;
  const double* uc = u + col * n;
  const double* wc = w + col * n;
  double* us = sm;
  double* ws = sm + n;
  for (int t = threadIdx.x; t < n; t += blockDim.x) { us[t] = uc[t]; ws[t] = wc[t]; }
  __syncthreads();
  const int e = g.e;
  const int nel = e * e * (D == 3 ? e : 1);
  const int cx = (int)(cell % g.nc[0]);
  const int cy = (int)((cell / g.nc[0]) % g.nc[1]);
  const int cz = (int)(cell / ((long long)g.nc[0] * g.nc[1]));
  double acc = 0.0;
  for (int t = threadIdx.x; t < nel * NA; t += blockDim.x) {
    const int el = t / NA, gp = t - el * NA;
    const int ex = el % e, ey = (el / e) % e, ez = el / (e * e);
    double eta[3], xi[3], J[3][3];
    gauss_point(g, cx, cy, cz, ex, ey, ez, gp, eta, xi);
    macro_jacobian(g, xi, J);
    const double dE = youngs_dr(g, strut_distance(g, eta), r_cell[cell]);
    if (dE == 0.0) continue;
    double C[45];
    chat_upper(D, g.nu, J, dE, C);
    double tq[D];
    for (int k = 0; k < D; ++k) tq[k] = gauss_t((gp >> k) & 1);
    double Gu[NI], Gw[NI];
    for (int I = 0; I < NI; ++I) { Gu[I] = 0.0; Gw[I] = 0.0; }
    for (int A = 0; A < NA; ++A) {
      const int ax = A & 1, ay = (A >> 1) & 1, az = (A >> 2) & 1;
      const int node = (ex + ax) + (e + 1) * ((ey + ay) + (e + 1) * (D == 3 ? (ez + az) : 0));
      for (int a = 0; a < D; ++a) {
        double dn = inv_h;
        for (int k = 0; k < D; ++k) {
          const int off = (A >> k) & 1;
          if (k == a) dn *= off ? 1.0 : -1.0;
          else dn *= off ? tq[k] : 1.0 - tq[k];
        }
        for (int i = 0; i < D; ++i) {
          Gu[i * D + a] += us[node * D + i] * dn;
          Gw[i * D + a] += ws[node * D + i] * dn;
        }
      }
    }
    int q = 0;
    double s = 0.0;
    for (int I = 0; I < NI; ++I)
      for (int Jx = I; Jx < NI; ++Jx) {
        const double cij = C[q++];
        s += cij * Gw[I] * Gu[Jx];
        if (Jx != I) s += cij * Gw[Jx] * Gu[I];
      }
    acc += wq * s;
  }
  // block reduction in fixed order
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    out[col] = -s;
  }
}

}  // namespace

fetidp_status k_snapshots(Ctx& c) {
  ProfScope ps(c, FETIDP_K_SETUP, 0.0, (double)c.N * c.nsnap * 8.0);
  const long long total = c.N * c.nelem * c.ngp;
  int grid = ceil_div(total, 256);
  if (grid > 152 * 32) grid = 152 * 32;
  snapshot_kernel<<<grid, 256, 0, c.stream>>>(c.geo, c.r_dev, c.N, c.nelem, c.ngp, c.nc, c.snap);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

// u, y: column (rhs, cell) holds nvec vectors of length len (n, or n_r when r_only).
fetidp_status k_apply_K(Ctx& c, CCellVec u, CellVec y, int nvec, int nrhs, bool idp, bool r_only,
                        const double* chat, double /*unused*/) {
  const int len = r_only ? c.nr : c.n;
  const int VB = nvec < 8 ? nvec : 8;
  {
    const double D = c.d, NA = c.ngp;
    const double fma = NA * D * D * 2.0 + D * D * D * D;   // gradient + stress + scatter per gp
    const double cols = (double)c.N * nrhs;
    c.prof_pending_flops = 2.0 * fma * c.nelem * c.ngp * nvec * cols;
    c.prof_pending_bytes = cols * (c.nsnap * 8.0 + 2.0 * nvec * len * 8.0);
  }
  ProfScope ps(c, FETIDP_K_APPLY_K, c.prof_pending_flops, c.prof_pending_bytes);
  const size_t smem = 2 * (size_t)VB * c.n * sizeof(double);
  const double h = 1.0 / c.e;
  const double wq = pow(0.5 * h, c.d);
  const dim3 grid((unsigned)(c.N * nrhs));
  if (c.d == 2) {
    cudaFuncSetAttribute(apply_K_kernel<2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    apply_K_kernel<2, double><<<grid, 256, smem, c.stream>>>(
        c.e, c.N, c.n, len, c.perm, c.perm + c.n, idp, u.p, u.rs, u.cs, y.p, y.rs, y.cs, nvec, VB,
        chat, c.nc, wq, 1.0 / h, u.ext, y.ext);
  } else {
    cudaFuncSetAttribute(apply_K_kernel<3, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    apply_K_kernel<3, double><<<grid, 256, smem, c.stream>>>(
        c.e, c.N, c.n, len, c.perm, c.perm + c.n, idp, u.p, u.rs, u.cs, y.p, y.rs, y.cs, nvec, VB,
        chat, c.nc, wq, 1.0 / h, u.ext, y.ext);
  }
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

// FP32 variant (local ROM bases of the mixed path): u, y float with the same view strides.
fetidp_status k_apply_K_f32(Ctx& c, const float* u, long long u_rs, int u_cs, float* y, long long y_rs,
                            int y_cs, int nvec, int nrhs, bool idp, bool r_only, long long ext) {
  const int len = r_only ? c.nr : c.n;
  const int VB = nvec < 16 ? nvec : 16;
  {
    const double D = c.d, NA = c.ngp;
    const double fma = NA * D * D * 2.0 + D * D * D * D;
    const double cols = (double)c.N * nrhs;
    c.prof_pending_flops = 2.0 * fma * c.nelem * c.ngp * nvec * cols;
    c.prof_pending_bytes = cols * (c.nsnap * 8.0 + 2.0 * nvec * len * 4.0);
  }
  ProfScope ps(c, FETIDP_K_APPLY_K, c.prof_pending_flops, c.prof_pending_bytes);
  const size_t smem = 2 * (size_t)VB * c.n * sizeof(float);
  const float h = 1.0f / c.e;
  const float wq = (float)pow(0.5 / c.e, c.d);
  const dim3 grid((unsigned)(c.N * nrhs));
  if (c.d == 2) {
    cudaFuncSetAttribute(apply_K_kernel<2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    apply_K_kernel<2, float><<<grid, 256, smem, c.stream>>>(c.e, c.N, c.n, len, c.perm, c.perm + c.n, idp,
                                                            u, u_rs, u_cs, y, y_rs, y_cs, nvec, VB,
                                                            c.snap, c.nc, wq, 1.0f / h, ext, ext);
  } else {
    cudaFuncSetAttribute(apply_K_kernel<3, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    apply_K_kernel<3, float><<<grid, 256, smem, c.stream>>>(c.e, c.N, c.n, len, c.perm, c.perm + c.n, idp,
                                                            u, u_rs, u_cs, y, y_rs, y_cs, nvec, VB,
                                                            c.snap, c.nc, wq, 1.0f / h, ext, ext);
  }
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_cell_gemv_strided(Ctx& c, const double* mats, long long mstride, int ld, int mrows,
                                  int mcols, CCellVec x, CellVec y, double alpha, double beta,
                                  int nrhs) {
  ProfScope ps(c, FETIDP_K_CELL_GEMV, 2.0 * mrows * mcols * (double)c.N * nrhs,
               8.0 * c.N * ((double)mrows * mcols + (double)nrhs * (mrows + mcols)));
  const size_t smem = (size_t)nrhs * mcols * sizeof(double);
  cudaFuncSetAttribute(cell_gemv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cell_gemv_kernel<<<(unsigned)c.N, 256, smem, c.stream>>>(mats, mstride, ld, mrows, mcols, x.p,
                                                           x.rs, x.cs, y.p, y.rs, y.cs, alpha, beta,
                                                           nrhs);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_grouped_gemm(Ctx& c, const double* A, long long a_stride_k, int lda, int M, int K,
                             CCellVec X, CellVec Y, const double* coef, double alpha, double beta,
                             int nrhs, bool separate, long long y_k_stride) {
  return k_grouped_gemm_n(c, A, a_stride_k, lda, M, K, c.nrb, X, Y, coef, alpha, beta, c.N, nrhs,
                          separate, y_k_stride);
}

fetidp_status k_grouped_gemm_n(Ctx& c, const double* A, long long a_stride_k, int lda, int M,
                               int K, int nk, CCellVec X, CellVec Y, const double* coef,
                               double alpha, double beta, long long ncell, int nrhs, bool separate,
                               long long y_k_stride) {
  const long long ncols = ncell * nrhs;
  ProfScope ps(c, FETIDP_K_GROUPED_GEMM, 2.0 * M * K * nk * (double)ncols,
               8.0 * ((double)nk * M * K + (double)ncols * K + (double)ncols * M * (separate ? nk : 1)));
  dim3 grid((unsigned)ceil_div(ncols, GT), (unsigned)ceil_div(M, GT));
  grouped_gemm_kernel<<<grid, 256, 0, c.stream>>>(A, a_stride_k, lda, M, K, nk, X.p, X.rs, X.cs,
                                                  Y.p, Y.rs, Y.cs, coef, alpha, beta, ncell, nrhs,
                                                  separate, y_k_stride);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

template <typename TB>
static fetidp_status gram_solve_t(Ctx& c, const TB* R, const TB* KR, CCellVec v, CellVec x, int nrhs) {
  if (c.nrb > kMaxRb) {
    set_error("n_rb above 64 is not supported by the Gram solve");
    return FETIDP_EINVAL;
  }
  const long long cols = c.N * nrhs;
  ProfScope ps(c, FETIDP_K_GRAM, cols * 2.0 * c.nr * (c.nrb * (c.nrb + 1) / 2.0 + 2.0 * c.nrb),
               cols * (double)sizeof(TB) * (2.0 * c.nrb * c.nr) + cols * 16.0 * c.nr);
  const size_t per_warp = (size_t)gram_warp_doubles(c.nrb, (int)sizeof(TB)) * sizeof(double);
  int wpb = (int)std::min<size_t>(8, (200 * 1024) / per_warp);
  if (wpb < 1) wpb = 1;
  const size_t smem = per_warp * wpb;
  cudaFuncSetAttribute(gram_warp_kernel<TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  gram_warp_kernel<TB><<<(unsigned)ceil_div(cols, wpb), 32 * wpb, smem, c.stream>>>(
      R, KR, v.p, v.rs, v.cs, x.p, x.rs, x.cs, c.nr, c.nrb, c.N, nrhs, 1e-12);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_gram_solve(Ctx& c, const double* R, const double* KR, CCellVec v, CellVec x,
                           int nrhs) {
  return gram_solve_t<double>(c, R, KR, v, x, nrhs);
}

fetidp_status k_gram_solve_f32(Ctx& c, const float* R, const float* KR, CCellVec v, CellVec x,
                               int nrhs, long long r_ext) {
  (void)r_ext;
  return gram_solve_t<float>(c, R, KR, v, x, nrhs);
}

fetidp_status k_grad(Ctx& c, const double* u, const double* w, double* g) {
  const double h = 1.0 / c.e;
  const double wq = pow(0.5 * h, c.d);
  const size_t smem = 2 * (size_t)c.n * sizeof(double);
  const dim3 grid((unsigned)(c.N * c.m));
  if (c.d == 2) {
    grad_kernel<2><<<grid, 256, smem, c.stream>>>(c.geo, c.r_dev, c.N, c.n, u, w, g, wq, 1.0 / h);
  } else {
    grad_kernel<3><<<grid, 256, smem, c.stream>>>(c.geo, c.r_dev, c.N, c.n, u, w, g, wq, 1.0 / h);
  }
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

FD_DEFINE_CHECK(fd_check_cell)

}  // namespace fetidp
