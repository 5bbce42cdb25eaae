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

// Contribution of one Gauss point gp of one element: f = w dN^T C_hat(gp) dN u_e (Eq. 52).
template <int D, typename T>
__device__ __forceinline__ void gp_apply(const double* __restrict__ chat_gp, int gp, T wq, T inv_h, const T* ue,
                                         T* fe) {
  constexpr int NA = 1 << D;
  constexpr int NI = D * D;
  T t[D];
  for (int k = 0; k < D; ++k) t[k] = (T)gauss_t((gp >> k) & 1);
  T dN[NA][D];
  for (int A = 0; A < NA; ++A)
    for (int a = 0; a < D; ++a) {
      T v = inv_h;
      for (int k = 0; k < D; ++k) {
        const int off = (A >> k) & 1;
        if (k == a) v *= off ? T(1) : T(-1);
        else v *= off ? t[k] : T(1) - t[k];
      }
      dN[A][a] = v;
    }
  T G[NI];
  for (int I = 0; I < NI; ++I) G[I] = T(0);
  for (int A = 0; A < NA; ++A)
    for (int i = 0; i < D; ++i)
      for (int a = 0; a < D; ++a) G[i * D + a] += ue[A * D + i] * dN[A][a];
  T S[NI];
  for (int I = 0; I < NI; ++I) S[I] = T(0);
  int q = 0;
  for (int I = 0; I < NI; ++I)
    for (int J = I; J < NI; ++J) {
      const T cij = (T)chat_gp[q++];
      S[I] += cij * G[J];
      if (J != I) S[J] += cij * G[I];
    }
  for (int A = 0; A < NA; ++A)
    for (int i = 0; i < D; ++i) {
      T v = T(0);
      for (int a = 0; a < D; ++a) v += dN[A][a] * S[i * D + a];
      fe[A * D + i] = wq * v;
    }
}

// One block per (cell, rhs) column, the cell slowest (the RHS of a cell share its C_hat in L2);
// vectors of the column processed VB at a time.  Within a colour group (elements that share no
// node) one thread per (vector, element, Gauss point); the 2^D threads of an element are adjacent
// lanes and sum their contributions with a fixed butterfly before one of them adds the element
// into the column's shared accumulator.  T = double (FP64 path) or float.
template <int D, typename T>
__global__ void apply_K_kernel(int e, long long ncell, int n, int len, const int* __restrict__ perm,
                               const int* __restrict__ iperm, bool idp, const T* __restrict__ u,
                               long long u_rs, int u_cs, T* __restrict__ y, long long y_rs,
                               int y_cs, int nvec, int VB, const double* __restrict__ chat, int nc,
                               T wq, T inv_h, long long u_ext, long long y_ext) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  constexpr int NA = 1 << D;
  const int nrhs = (int)(gridDim.x / ncell);
  const long long cell = blockIdx.x / nrhs;
  const int rhs = (int)(blockIdx.x - cell * nrhs);
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
      // uniform trip count (total and blockDim are multiples of NA): every lane reaches the shuffles
      const int total = vb * nel * NA;
      for (int t0 = 0; t0 < total; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        const bool live = t < total;
        const int gp = t & (NA - 1);
        const int vq = live ? t / NA : 0;
        const int v = vq / nel, q = vq - v * nel;
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
          for (int i = 0; i < D; ++i) ue[A * D + i] = live ? uv[nodes[A] * D + i] : T(0);
        gp_apply<D, T>(chat_cell + ((size_t)el * NA + gp) * nc, gp, wq, inv_h, ue, fe);
#pragma unroll
        for (int k = 0; k < NA * D; ++k)
          for (int o = 1; o < NA; o <<= 1) fe[k] += __shfl_xor_sync(0xffffffffu, fe[k], o);
        if (live && gp == 0) {
          T* yv = ys + (size_t)v * n;
          for (int A = 0; A < NA; ++A)
            for (int i = 0; i < D; ++i) yv[nodes[A] * D + i] += fe[A * D + i];
        }
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

// Index of entry (I, J) of a symmetric d^2 x d^2 matrix kept as its upper triangle, row-major.
__device__ __forceinline__ int sym_index(int I, int J, int NI) {
  if (I > J) { const int t = I; I = J; J = t; }
  return I * NI - I * (I - 1) / 2 + (J - I);
}

// Element matrices K_e = sum_gp w B^T C_hat B of every element of every cell in FP32 (C_hat
// rounded to FP32 first), row-major ND x ND, for the Eq. 46b products of the mixed path.  They
// depend on the cell's C_hat only, so they are formed once per setup instead of in every local
// ROM solve.  One thread per (cell, element, row (A, i)).
constexpr int kMultiThreads = 512;
template <int D>
__global__ void element_matrices_f32_kernel(const double* __restrict__ chat, long long ncell, int e, int nc,
                                            float wq, float inv_h, float* __restrict__ Kall) {
  constexpr int NA = 1 << D;
  constexpr int ND = NA * D;
  constexpr int NI = D * D;
  const int nel = e * e * (D == 3 ? e : 1);
  const int cpe = NA * nc;
  const long long total = ncell * nel * ND;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(t % ND);
    const long long ce = t / ND;                    // cell * nel + el
    const int A = row / D, i = row - A * D;
    const double* Ce = chat + ce * cpe;
    float krow[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) krow[k] = 0.f;
    for (int gp = 0; gp < NA; ++gp) {
      float dn[NA * D];                             // shape-function gradients at this Gauss point
#pragma unroll
      for (int B = 0; B < NA; ++B)
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float v = inv_h;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const int off = (B >> k) & 1;
            const float tk = (float)gauss_t((gp >> k) & 1);
            if (k == a) v *= off ? 1.f : -1.f;
            else v *= off ? tk : 1.f - tk;
          }
          dn[B * D + a] = v;
        }
      float w[D][D];   // w[j][b] = sum_a dN_A[a] C[(i,a),(j,b)]
#pragma unroll
      for (int j = 0; j < D; ++j)
#pragma unroll
        for (int b = 0; b < D; ++b) {
          float sacc = 0.f;
#pragma unroll
          for (int a = 0; a < D; ++a)
            sacc += dn[A * D + a] * (float)Ce[gp * nc + sym_index(i * D + a, j * D + b, NI)];
          w[j][b] = sacc;
        }
#pragma unroll
      for (int B = 0; B < NA; ++B)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          float sacc = 0.f;
#pragma unroll
          for (int b = 0; b < D; ++b) sacc += w[j][b] * dn[B * D + b];
          krow[B * D + j] += wq * sacc;
        }
    }
    float* kr = Kall + t * ND;
#pragma unroll
    for (int k = 0; k < ND; k += 4)
      *reinterpret_cast<float4*>(kr + k) = make_float4(krow[k], krow[k + 1], krow[k + 2], krow[k + 3]);
  }
}

// Multi-vector K_s application in FP32 (the Eq. 46b products K_s R of the mixed path).  One
// block per (cell, rhs, chunk of VB vectors), the cell slowest: the blocks of one cell run side
// by side and read its element matrices from L2, not once per chunk from HBM.  For each colour group (elements that share no node) the precomputed
// element matrices of its elements are staged in shared memory (contiguous, coalesced) and
// applied to all vectors of the chunk, one thread per (element, vector).  Vectors are stored
// dof-major with a padded stride, so the threads of an element read consecutive words and every
// K_e entry is a broadcast.  Global vectors are read and written in local order through the
// staged permutation, so no load depends on another.
// padded K_e row stride (in floats): 4 mod 32 so that neighbouring elements hit different banks;
// rows stay 16-byte aligned
__host__ __device__ constexpr int multi_ke_stride(int D) { return (D == 2 ? 64 : 576) + 4; }
template <int D>
__global__ void __launch_bounds__(kMultiThreads, 2) apply_K_multi_kernel(
    int e, long long ncell, int n, int len, const int* __restrict__ perm, bool idp,
    const float* __restrict__ u, long long u_rs, int u_cs, float* __restrict__ y, long long y_rs, int y_cs,
    int nvec, int VB, int nchunk, int nrhs, const float* __restrict__ Kall, int nelc_max, long long u_ext,
    long long y_ext) {
  constexpr int NA = 1 << D;
  constexpr int ND = NA * D;
  constexpr int KES = multi_ke_stride(D);
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int VBp = VB + 1;
  float* us = reinterpret_cast<float*>(sm_raw);        // [n][VBp]
  float* ys = us + (size_t)n * VBp;                     // [n][VBp]
  float* Ke = ys + (size_t)n * VBp;                     // [nelc_max][KES], rows of ND
  Ke = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(Ke) + 15) & ~uintptr_t(15));
  int* perm_s = reinterpret_cast<int*>(Ke + (size_t)nelc_max * KES);   // [n] local -> natural
  const int chunk = (int)(blockIdx.x % nchunk);
  const long long rest = blockIdx.x / nchunk;
  const int rhs = (int)(rest % nrhs);
  const long long cell = rest / nrhs;
  const float* uc = u + rhs * u_rs + cell * u_cs;
  float* yc = y + rhs * y_rs + cell * y_cs;
  const int nel = e * e * (D == 3 ? e : 1);
  const float* Kcell = Kall + cell * (long long)nel * ND * ND;
  const int ecount[3] = {e, e, D == 3 ? e : 1};
  for (int li = threadIdx.x; li < n; li += blockDim.x) perm_s[li] = idp ? perm[li] : li;
  __syncthreads();
  {
    const int v0 = chunk * VB;
    const int vb = min(VB, nvec - v0);
#pragma unroll 4
    for (int t = threadIdx.x; t < vb * len; t += blockDim.x) {
      const int v = t / len, li = t - v * len;
      float val = 0.f;
      if (FD_INB(rhs * u_rs + cell * u_cs + (long long)(v0 + v) * len + li, u_ext, 203))
        val = uc[(size_t)(v0 + v) * len + li];
      us[(size_t)perm_s[li] * VBp + v] = val;
    }
    for (int t = threadIdx.x; t < vb * (n - len); t += blockDim.x) {   // dofs outside the vector
      const int v = t / (n - len), r = t - v * (n - len);
      us[(size_t)perm_s[len + r] * VBp + v] = 0.f;
    }
    for (int t = threadIdx.x; t < n * VBp; t += blockDim.x) ys[t] = 0.f;
    for (int color = 0; color < NA; ++color) {
      int cnt[3], par[3];
      int nelc = 1;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        par[k] = (k < D) ? ((color >> k) & 1) : 0;
        cnt[k] = (k < D) ? (ecount[k] - par[k] + 1) / 2 : 1;
        nelc *= cnt[k];
      }
      __syncthreads();   // previous colour's K_e no longer read
      // the colour's element matrices, 16-byte loads
      for (int t = threadIdx.x; t < nelc * ND * (ND / 4); t += blockDim.x) {
        const int q = t / (ND * ND / 4), r = t - q * (ND * ND / 4);
        const int qx = q % cnt[0], qy = (q / cnt[0]) % cnt[1], qz = q / (cnt[0] * cnt[1]);
        const int el = (par[0] + 2 * qx) + e * ((par[1] + 2 * qy) + e * (par[2] + 2 * qz));
        const int row = (4 * r) / ND, k = 4 * r - row * ND;
        *reinterpret_cast<float4*>(Ke + (size_t)q * KES + row * ND + k) =
            *reinterpret_cast<const float4*>(Kcell + ((size_t)el * ND + row) * ND + k);
      }
      __syncthreads();
      // apply to every vector of the chunk
      for (int t = threadIdx.x; t < nelc * vb; t += blockDim.x) {
        const int q = t / vb, v = t - q * vb;
        const int qx = q % cnt[0], qy = (q / cnt[0]) % cnt[1], qz = q / (cnt[0] * cnt[1]);
        const int ex = par[0] + 2 * qx, ey = par[1] + 2 * qy, ez = par[2] + 2 * qz;
        int dof0[NA];
#pragma unroll
        for (int B = 0; B < NA; ++B) {
          const int bx = B & 1, by = (B >> 1) & 1, bz = (B >> 2) & 1;
          dof0[B] = D * ((ex + bx) + (e + 1) * ((ey + by) + (e + 1) * (D == 3 ? (ez + bz) : 0)));
        }
        float ue[ND];
#pragma unroll
        for (int B = 0; B < NA; ++B)
#pragma unroll
          for (int j = 0; j < D; ++j) ue[B * D + j] = us[(size_t)(dof0[B] + j) * VBp + v];
        const float* kq = Ke + (size_t)q * KES;
#pragma unroll
        for (int A = 0; A < NA; ++A)
#pragma unroll
          for (int i = 0; i < D; ++i) {
            const float* kr = kq + (A * D + i) * ND;
            float sacc = 0.f;
#pragma unroll
            for (int k = 0; k < ND; k += 4) {
              const float4 k4 = *reinterpret_cast<const float4*>(kr + k);
              sacc += k4.x * ue[k] + k4.y * ue[k + 1] + k4.z * ue[k + 2] + k4.w * ue[k + 3];
            }
            ys[(size_t)(dof0[A] + i) * VBp + v] += sacc;
          }
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int t = threadIdx.x; t < vb * len; t += blockDim.x) {
      const int v = t / len, li = t - v * len;
      if (FD_INB(rhs * y_rs + cell * y_cs + (long long)(v0 + v) * len + li, y_ext, 204))
        yc[(size_t)(v0 + v) * len + li] = ys[(size_t)perm_s[li] * VBp + v];
    }
    __syncthreads();
  }
}

// ---- K_rr^(s) R for many vectors as a sparse product (Eq. 46b, mixed path)
// Every cell has the same sparsity pattern, so K_rr^(s) (remaining DOF, local (i, d) order) is
// stored in ELL form: one column table [slot][row] shared by all cells and FP32 values
// [cell][slot][row] (row fastest, so a warp's 32 rows read 128 contiguous bytes per slot).  The
// values are summed from the element matrices once per setup, in a fixed order.

// val[cell][slot][row] = sum over the entry's contributions of Ke[cell][el][a][b]
__global__ void krr_ell_assemble_kernel(const float* __restrict__ Ke, long long ke_cell, const int* __restrict__ cnt,
                                        const int* __restrict__ idx, int cmax, int nnz, int nr, long long ncell,
                                        float* __restrict__ val) {
  const long long per = (long long)nnz * nr;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncell * per;
       t += (long long)gridDim.x * blockDim.x) {
    const long long cell = t / per;
    const int e = (int)(t - cell * per);
    const float* kc = Ke + cell * ke_cell;
    float v = 0.f;
    for (int q = 0; q < cnt[e]; ++q) v += kc[idx[(long long)e * cmax + q]];
    val[t] = v;
  }
}

constexpr int kSpVB = 16;   // vectors per block
constexpr int kSpLd = 20;   // shared row stride (floats): 16 vectors + 4, conflict-free 16-byte reads
// One block per (cell, rhs, chunk of kSpVB vectors), cell slowest: the vectors of the chunk are
// staged transposed ([dof][vector]) in shared memory, each thread owns rows and accumulates the
// chunk's kSpVB products in registers (four 16-byte shared reads per 16 FMAs per slot).
__global__ void __launch_bounds__(256) krr_spmm_f32_kernel(const int* __restrict__ ecol, const float* __restrict__ eval,
                                                           int nnz, int nr, int nrhs, int nchunk,
                                                           const float* __restrict__ u, long long u_rs, int u_cs,
                                                           float* __restrict__ y, long long y_rs, int y_cs, int nvec,
                                                           long long ext) {
  extern __shared__ __align__(16) float uss[];   // [nr][kSpLd]
  const int chunk = (int)(blockIdx.x % nchunk);
  const long long rest = blockIdx.x / nchunk;
  const int rhs = (int)(rest % nrhs);
  const long long cell = rest / nrhs;
  const int v0 = chunk * kSpVB, vb = min(kSpVB, nvec - v0);
  const long long base = rhs * u_rs + cell * u_cs;
  for (int t = threadIdx.x; t < kSpVB * nr; t += blockDim.x) {
    const int v = t / nr, q = t - v * nr;
    float x = 0.f;
    if (v < vb && FD_INB(base + (long long)(v0 + v) * nr + q, ext, 205)) x = u[base + (long long)(v0 + v) * nr + q];
    uss[q * kSpLd + v] = x;
  }
  __syncthreads();
  const float* ev = eval + cell * (long long)nnz * nr;
  const long long ybase = rhs * y_rs + cell * y_cs;
  for (int r = threadIdx.x; r < nr; r += blockDim.x) {
    float acc[kSpVB];
#pragma unroll
    for (int v = 0; v < kSpVB; ++v) acc[v] = 0.f;
    // eight slots' (column, value) pairs are loaded before any of them is used
    for (int sl0 = 0; sl0 < nnz; sl0 += 8) {
      int cc[8];
      float aa[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int sl = sl0 + u;
        cc[u] = sl < nnz ? __ldg(ecol + (long long)sl * nr + r) : 0;
        aa[u] = sl < nnz ? __ldcs(ev + (long long)sl * nr + r) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4* xs = reinterpret_cast<const float4*>(uss + cc[u] * kSpLd);
        const float a = aa[u];
#pragma unroll
        for (int v4 = 0; v4 < kSpVB / 4; ++v4) {
          const float4 x = xs[v4];
          acc[4 * v4] = fmaf(a, x.x, acc[4 * v4]);
          acc[4 * v4 + 1] = fmaf(a, x.y, acc[4 * v4 + 1]);
          acc[4 * v4 + 2] = fmaf(a, x.z, acc[4 * v4 + 2]);
          acc[4 * v4 + 3] = fmaf(a, x.w, acc[4 * v4 + 3]);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < kSpVB; ++v)
      if (v < vb && FD_INB(ybase + (long long)(v0 + v) * nr + r, ext, 206)) y[ybase + (long long)(v0 + v) * nr + r] = acc[v];
  }
}

// The same product for the nodal pattern of K_rr (every node's D rows share their neighbour
// nodes): one thread per node, so each 16-byte shared read of a neighbour component's vectors feeds
// D rows, and the warp's lanes read consecutive nodes' neighbours (regular, conflict-free
// addresses).  The D slots of neighbour k (D * n_r values, shared by the cell's (rhs, chunk)
// blocks through L2) are staged in shared memory by cp.async one neighbour ahead.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
template <int D>
__global__ void __launch_bounds__(352, 2) krr_spmm_nodal_f32_kernel(
    const int* __restrict__ nbr, const float* __restrict__ eval, int nnz, int nr, int nrhs, int nchunk,
    const float* __restrict__ u, long long u_rs, int u_cs, float* __restrict__ y, long long y_rs, int y_cs, int nvec,
    long long ext) {
  extern __shared__ __align__(16) float uss[];   // [nr][kSpLd], then two slot buffers [D * nr]
  float* evs = uss + (size_t)nr * kSpLd;
  const int chunk = (int)(blockIdx.x % nchunk);
  const long long rest = blockIdx.x / nchunk;
  const int rhs = (int)(rest % nrhs);
  const long long cell = rest / nrhs;
  const int v0 = chunk * kSpVB, vb = min(kSpVB, nvec - v0);
  const long long base = rhs * u_rs + cell * u_cs;
  const int nnode = nr / D, nk = nnz / D, sl = D * nr;
  const float* ev = eval + cell * (long long)nnz * nr;
  // the chunk's vectors, transposed into [dof][vector], and neighbour 0's slots: asynchronous copies
  for (int t = threadIdx.x; t < kSpVB * nr; t += blockDim.x) {
    const int v = t / nr, q = t - v * nr;
    if (v < vb && FD_INB(base + (long long)(v0 + v) * nr + q, ext, 207))
      cp_async4(uss + q * kSpLd + v, u + base + (long long)(v0 + v) * nr + q);
    else
      uss[q * kSpLd + v] = 0.f;
  }
  for (int t = threadIdx.x; t < sl; t += blockDim.x) cp_async4(evs + t, ev + t);   // neighbour 0
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  const long long ybase = rhs * y_rs + cell * y_cs;
  const int n = threadIdx.x;                      // one node per thread (the host launches >= nnode threads)
  const bool live = n < nnode;
  float acc[D][kSpVB];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int v = 0; v < kSpVB; ++v) acc[a][v] = 0.f;
  int m_next = live ? __ldg(nbr + n) : 0;
  for (int k = 0; k < nk; ++k) {
    if (k + 1 < nk) {
      const float* src = ev + (long long)(k + 1) * sl;
      float* dst = evs + ((k + 1) & 1) * sl;
      for (int t = threadIdx.x; t < sl; t += blockDim.x) cp_async4(dst + t, src + t);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();                              // neighbour k's slots (and the vectors) are in place
    const int m = m_next;
    if (live && k + 1 < nk) m_next = __ldg(nbr + (long long)(k + 1) * nnode + n);
    if (live) {
      const float* e = evs + (k & 1) * sl;
#pragma unroll
      for (int cq = 0; cq < D; ++cq) {
        float av[D];
#pragma unroll
        for (int a = 0; a < D; ++a) av[a] = e[cq * nr + D * n + a];
        const float4* xs = reinterpret_cast<const float4*>(uss + (D * m + cq) * kSpLd);
#pragma unroll
        for (int v4 = 0; v4 < kSpVB / 4; ++v4) {
          const float4 x = xs[v4];
#pragma unroll
          for (int a = 0; a < D; ++a) {
            acc[a][4 * v4] = fmaf(av[a], x.x, acc[a][4 * v4]);
            acc[a][4 * v4 + 1] = fmaf(av[a], x.y, acc[a][4 * v4 + 1]);
            acc[a][4 * v4 + 2] = fmaf(av[a], x.z, acc[a][4 * v4 + 2]);
            acc[a][4 * v4 + 3] = fmaf(av[a], x.w, acc[a][4 * v4 + 3]);
          }
        }
      }
    }
    __syncthreads();                              // buffer k & 1 is refilled at step k + 1
  }
  if (!live) return;
#pragma unroll
  for (int v = 0; v < kSpVB; ++v)
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const long long o = ybase + (long long)(v0 + v) * nr + D * n + a;
      if (v < vb && FD_INB(o, ext, 208)) y[o] = acc[a][v];
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

// Narrow per-cell operators with a compile-time column count MC (n_p: 8 in 2D, 24 in 3D): one
// thread per (cell, row); the row's MC entries arrive as 16-byte loads issued before any use, so
// each thread waits for memory once.  Rows must be 16-byte aligned (ld and the base even).
template <int MC>
__global__ void cell_gemv_narrow_fixed(const double* __restrict__ mats, long long mstride, int ld, int mrows,
                                       const double* __restrict__ x, long long x_rs, int x_cs,
                                       double* __restrict__ y, long long y_rs, int y_cs, double alpha,
                                       double beta, int nrhs, long long ncell) {
  const int total = (int)(ncell * mrows);             // < 2^31, checked by the host
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int cell = t / mrows;
    const int row = t - cell * mrows;
    const double2* Mr = reinterpret_cast<const double2*>(mats + (long long)cell * mstride + (long long)row * ld);
    double mv[MC];
#pragma unroll
    for (int q = 0; q < MC / 2; ++q) {
      const double2 v = Mr[q];
      mv[2 * q] = v.x;
      mv[2 * q + 1] = v.y;
    }
    for (int r = 0; r < nrhs; ++r) {
      const double* xc = x + r * x_rs + (long long)cell * x_cs;
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < MC; ++q) acc = fma(mv[q], xc[q], acc);
      double* dst = y + r * y_rs + (long long)cell * y_cs + row;
      *dst = (beta == 0.0) ? alpha * acc : alpha * acc + beta * (*dst);
    }
  }
}

// Narrow per-cell operators (at most 32 columns, e.g. the n_r x n_p prolongations): one thread
// per (cell, row), so consecutive threads read consecutive rows; x entries are shared by the
// threads of a cell (cache broadcast).
__global__ void cell_gemv_narrow_kernel(const double* __restrict__ mats, long long mstride, int ld,
                                        int mrows, int mcols, const double* __restrict__ x, long long x_rs,
                                        int x_cs, double* __restrict__ y, long long y_rs, int y_cs,
                                        double alpha, double beta, int nrhs, long long ncell) {
  const long long total = ncell * mrows;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long cell = t / mrows;
    const int row = (int)(t - cell * mrows);
    const double* Mr = mats + cell * mstride + (long long)row * ld;
    for (int r0 = 0; r0 < nrhs; r0 += kMaxRhsGemv) {
      const int rb = min(kMaxRhsGemv, nrhs - r0);
      double acc[kMaxRhsGemv];
#pragma unroll
      for (int r = 0; r < kMaxRhsGemv; ++r) acc[r] = 0.0;
      for (int q = 0; q < mcols; ++q) {
        const double mv = Mr[q];
#pragma unroll
        for (int r = 0; r < kMaxRhsGemv; ++r)
          if (r < rb) acc[r] += mv * x[(r0 + r) * x_rs + cell * x_cs + q];
      }
#pragma unroll
      for (int r = 0; r < kMaxRhsGemv; ++r) {
        if (r < rb) {
          double* dst = y + (r0 + r) * y_rs + cell * y_cs + row;
          *dst = (beta == 0.0) ? alpha * acc[r] : alpha * acc[r] + beta * (*dst);
        }
      }
    }
  }
}

// ---- assembled per-cell ROM operators in FP32 (mixed path, large cells)
// F_dd_ring^(s) = sum_k delta_k F_dd^(sigma_k) and S_dd_ring^(s) = sum_k alpha_k S_dd^(sigma_k)
// (Eqs. 43, 48, 49) formed once per setup.  Applying the principal form costs 2 N_rb n_d^2 flops
// per column (three BF16 products with the hi/lo split); the assembled operator costs 4 n_d^2
// bytes per cell, shared by the cell's m columns.  At n_d = 630 the streamed operator is the
// cheaper of the two on GB300, and it is HBM-bound.

// out[cell][r][c] (row stride ldo, FP32) = sum_k coef[cell][k] src[k][(r0 + r) * ld + c0 + c].
// A thread owns one entry (r, c): its NRBM principal values sit in registers and are reused for
// kCombCells cells, whose coefficients are staged in shared memory (FP32 arithmetic).
constexpr int kCombCells = 32;
// symT > 0: the output is the packed symmetric tile form (upper-triangle 32 x 32 tiles of a
// symT x symT tile grid, sym_tile_offset) and entries below the diagonal tiles are not written.
__host__ __device__ inline long long sym_tile_index(int I, int J, int T) {
  return (long long)I * T - (long long)I * (I - 1) / 2 + (J - I);
}
// element (r, c) of a 32 x 32 tile: quad c / 4 of row r at float4 slot 32 (c / 4) + r, so a warp
// whose lane r loads quad k reads 512 contiguous bytes
__host__ __device__ inline int sym_in_tile(int r, int c) { return (((c >> 2) * 32 + r) << 2) + (c & 3); }
template <int NRBM>
__global__ void __launch_bounds__(256) rom_combine_f32_kernel(const double* __restrict__ src, long long kstride,
                                                              int ld, int r0, int c0, int rows, int cols,
                                                              const double* __restrict__ coef, int nrb,
                                                              long long ncell, float* __restrict__ out, int ldo,
                                                              int symT) {
  __shared__ float cs[kCombCells][NRBM];
  const long long per = (long long)rows * cols;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int r_ = t < per ? (int)(t / cols) : 0, c_ = t < per ? (int)(t - (long long)r_ * cols) : 0;
  const bool live = t < per && (symT == 0 || (r_ >> 5) <= (c_ >> 5));
  const int r = r_, cc = c_;
  const long long cell_stride = symT ? 1024LL * symT * (symT + 1) / 2 : (long long)rows * ldo;
  const long long eoff = symT ? 1024LL * sym_tile_index(r >> 5, cc >> 5, symT) + sym_in_tile(r & 31, cc & 31)
                              : (long long)r * ldo + cc;
  float p[NRBM];
#pragma unroll
  for (int k = 0; k < NRBM; ++k)
    p[k] = (live && k < nrb) ? (float)src[k * kstride + (long long)(r0 + r) * ld + c0 + cc] : 0.f;
  for (long long cell0 = (long long)blockIdx.y * kCombCells; cell0 < ncell; cell0 += (long long)gridDim.y * kCombCells) {
    const int nc = (int)min((long long)kCombCells, ncell - cell0);
    __syncthreads();
    for (int q = threadIdx.x; q < kCombCells * NRBM; q += blockDim.x) {
      const int ci = q / NRBM, k = q - ci * NRBM;
      cs[ci][k] = (ci < nc && k < nrb) ? (float)coef[(cell0 + ci) * nrb + k] : 0.f;
    }
    __syncthreads();
    if (!live) continue;
    for (int ci = 0; ci < nc; ++ci) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < NRBM; ++k) acc = fmaf(cs[ci][k], p[k], acc);
      out[(cell0 + ci) * cell_stride + eoff] = acc;
    }
  }
}

// y[rhs][cell][0..nout) = alpha M[cell]^T x[rhs][cell][0..nin) + beta y for per-cell FP32 matrices
// M[cell] of nin stored rows of nout entries (row stride ldm, a multiple of 4, >= nout): row j of M
// multiplies x_j.  For the symmetric F_dd_ring and S_dd_ring (combinations of symmetric principal
// operators) this is M x.  One CTA per cell; a thread owns four consecutive outputs, so for each
// stored row j it issues one 16-byte streaming load of M[j][4t..4t+3] (a warp reads 512 contiguous
// bytes), and the row's x values for every RHS arrive as two broadcast 16-byte reads from shared
// memory ([row][8] layout).  kAsmU rows' loads are issued before their arithmetic.
constexpr int kMaxRhsF32 = 8;
constexpr int kAsmU = 8;
constexpr int kAsmMaxThreads = 256;    // rows <= 1024
__global__ void __launch_bounds__(kAsmMaxThreads) cell_gemm_f32_kernel(const float* __restrict__ mats, int ldm,
                                                                       int nout, int nin,
                                                                       const double* __restrict__ x, long long x_rs,
                                                                       int x_cs, double* __restrict__ y,
                                                                       long long y_rs, int y_cs, double alpha,
                                                                       double beta, int nrhs) {
  extern __shared__ __align__(16) float xsf[];   // [nin][kMaxRhsF32]
  const long long cell = blockIdx.x;
  const int tid = threadIdx.x;
  const int rows = nout, cols = nin;             // outputs, stored rows
  const float* M = mats + cell * (long long)nin * ldm;
  const int r0 = 4 * tid;                        // ldm is a multiple of 4 and >= nout: the load stays in row j
  const bool live = r0 < rows;
  for (int rb0 = 0; rb0 < nrhs; rb0 += kMaxRhsF32) {
    const int rb = min(kMaxRhsF32, nrhs - rb0);
    __syncthreads();
    for (int t = tid; t < cols * kMaxRhsF32; t += blockDim.x) {
      const int j = t / kMaxRhsF32, q = t - j * kMaxRhsF32;
      xsf[t] = q < rb ? (float)x[(rb0 + q) * x_rs + cell * x_cs + j] : 0.f;
    }
    __syncthreads();
    float acc[4][kMaxRhsF32];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int q = 0; q < kMaxRhsF32; ++q) acc[a][q] = 0.f;
    for (int j0 = 0; j0 < cols; j0 += kAsmU) {
      float4 m[kAsmU];
#pragma unroll
      for (int u = 0; u < kAsmU; ++u)
        m[u] = (live && j0 + u < cols) ? __ldcs(reinterpret_cast<const float4*>(M + (long long)(j0 + u) * ldm + r0))
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < kAsmU; ++u) {
        if (j0 + u >= cols) break;
        const float4 x0 = reinterpret_cast<const float4*>(xsf)[(j0 + u) * 2];
        const float4 x1 = reinterpret_cast<const float4*>(xsf)[(j0 + u) * 2 + 1];
        const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        const float mv[4] = {m[u].x, m[u].y, m[u].z, m[u].w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int q = 0; q < kMaxRhsF32; ++q) acc[a][q] = fmaf(mv[a], xv[q], acc[a][q]);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (r0 + a >= rows) continue;
#pragma unroll
      for (int q = 0; q < kMaxRhsF32; ++q) {
        if (q < rb) {
          double* dst = y + (rb0 + q) * y_rs + cell * y_cs + r0 + a;
          *dst = (beta == 0.0) ? alpha * (double)acc[a][q] : alpha * (double)acc[a][q] + beta * (*dst);
        }
      }
    }
  }
}

// y = alpha M x + beta y for the SYMMETRIC per-cell operators stored as packed upper-triangle tiles
// (32 x 32, T tile rows, sym_in_tile layout): every stored tile (I, J), I < J, is read from memory
// once and used twice, y_I += M_IJ x_J and y_J += M_IJ^T x_I; a diagonal tile gives y_I += M_II x_I.
// One CTA per cell with T'/2 warps (T' = T rounded up to even).  The off-diagonal tiles are visited
// in the T' - 1 rounds of the circle schedule -- in each round the warps hold disjoint block pairs,
// so every y block has one writer per round and the summation order is fixed (deterministic, no
// atomics) -- then the diagonal tiles.  A warp loads its tile with lane r owning row r (eight
// 16-byte loads of 512 contiguous bytes) and the next round's tile while it computes; the column
// products read the tile transposed through a 32 x 33 shared buffer.  x and y are staged in
// shared memory in FP32 ([row][8] and [row][9]), up to eight RHS at a time.
__device__ __forceinline__ bool sym_round_pair(int round, int w, int Tp, int T, int& I, int& J) {
  int a, b;
  if (w == 0) {
    a = round;
    b = Tp - 1;
  } else {
    a = (round + w) % (Tp - 1);
    b = (round - w + (Tp - 1)) % (Tp - 1);
  }
  I = min(a, b);
  J = max(a, b);
  return J < T;                                   // block T of an odd T is the empty pad block
}
__global__ void __launch_bounds__(320, 2) cell_symv_f32_kernel(const float* __restrict__ mats, int T, int n,
                                                               const double* __restrict__ x, long long x_rs,
                                                               int x_cs, double* __restrict__ y, long long y_rs,
                                                               int y_cs, double alpha, double beta, int nrhs) {
  extern __shared__ __align__(16) float symsm[];
  const int NP = T * 32;
  float* xs = symsm;                              // [NP][8]
  float* ys = xs + (size_t)NP * 8;                // [NP][9]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  float* tb = ys + (size_t)NP * 9 + (size_t)warp * 32 * 33;
  const int Tp = (T + 1) & ~1;
  const long long cell = blockIdx.x;
  const float4* Mc = reinterpret_cast<const float4*>(mats + cell * 1024LL * T * (T + 1) / 2);
  const int nrounds = Tp - 1;
  for (int rb0 = 0; rb0 < nrhs; rb0 += 8) {
    const int rb = min(8, nrhs - rb0);
    __syncthreads();
    for (int t = tid; t < NP * 8; t += blockDim.x) {
      const int q = t / NP, j = t - q * NP;
      xs[j * 8 + q] = (q < rb && j < n) ? (float)x[(rb0 + q) * x_rs + cell * x_cs + j] : 0.f;
    }
    for (int t = tid; t < NP * 9; t += blockDim.x) ys[t] = 0.f;
    __syncthreads();
    // rounds 0 .. nrounds-1: off-diagonal pairs; round nrounds + s: diagonal tiles w + s * nw
    int I, J;
    bool have = nrounds > 0 ? sym_round_pair(0, warp, Tp, T, I, J) : false;
    float4 m[8];
    if (have)
#pragma unroll
      for (int k = 0; k < 8; ++k) m[k] = __ldcs(Mc + sym_tile_index(I, J, T) * 256 + k * 32 + lane);
    const int ndiag_steps = (T + nw - 1) / nw;
    for (int step = 0; step < nrounds + ndiag_steps; ++step) {
      // the next step's tile, loaded before this one is used
      int In = 0, Jn = 0;
      bool have_n = false;
      if (step + 1 < nrounds) have_n = sym_round_pair(step + 1, warp, Tp, T, In, Jn);
      else if (step + 1 < nrounds + ndiag_steps) {
        In = Jn = warp + (step + 1 - nrounds) * nw;
        have_n = In < T;
      }
      float4 mn[8];
      if (have_n)
#pragma unroll
        for (int k = 0; k < 8; ++k) mn[k] = __ldcs(Mc + sym_tile_index(In, Jn, T) * 256 + k * 32 + lane);
      if (have) {
        // y_I[lane] += sum_c M[lane][c] x_J[c]
        float ar[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const float4* xJ = reinterpret_cast<const float4*>(xs + (size_t)J * 32 * 8);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float mv[4] = {m[k].x, m[k].y, m[k].z, m[k].w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float4 x0 = xJ[(4 * k + e) * 2], x1 = xJ[(4 * k + e) * 2 + 1];
            ar[0] = fmaf(mv[e], x0.x, ar[0]);
            ar[1] = fmaf(mv[e], x0.y, ar[1]);
            ar[2] = fmaf(mv[e], x0.z, ar[2]);
            ar[3] = fmaf(mv[e], x0.w, ar[3]);
            ar[4] = fmaf(mv[e], x1.x, ar[4]);
            ar[5] = fmaf(mv[e], x1.y, ar[5]);
            ar[6] = fmaf(mv[e], x1.z, ar[6]);
            ar[7] = fmaf(mv[e], x1.w, ar[7]);
          }
        }
        float* yI = ys + (size_t)(I * 32 + lane) * 9;
#pragma unroll
        for (int q = 0; q < 8; ++q) yI[q] += ar[q];
        if (I != J) {
          // y_J[lane] += sum_r M[r][lane] x_I[r], column lane of the tile through the buffer
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            tb[lane * 33 + 4 * k] = m[k].x;
            tb[lane * 33 + 4 * k + 1] = m[k].y;
            tb[lane * 33 + 4 * k + 2] = m[k].z;
            tb[lane * 33 + 4 * k + 3] = m[k].w;
          }
          __syncwarp();
          float ac[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          const float4* xI = reinterpret_cast<const float4*>(xs + (size_t)I * 32 * 8);
#pragma unroll 8
          for (int r = 0; r < 32; ++r) {
            const float tv = tb[r * 33 + lane];
            const float4 x0 = xI[r * 2], x1 = xI[r * 2 + 1];
            ac[0] = fmaf(tv, x0.x, ac[0]);
            ac[1] = fmaf(tv, x0.y, ac[1]);
            ac[2] = fmaf(tv, x0.z, ac[2]);
            ac[3] = fmaf(tv, x0.w, ac[3]);
            ac[4] = fmaf(tv, x1.x, ac[4]);
            ac[5] = fmaf(tv, x1.y, ac[5]);
            ac[6] = fmaf(tv, x1.z, ac[6]);
            ac[7] = fmaf(tv, x1.w, ac[7]);
          }
          __syncwarp();                           // the buffer is rewritten by the next tile
          float* yJ = ys + (size_t)(J * 32 + lane) * 9;
#pragma unroll
          for (int q = 0; q < 8; ++q) yJ[q] += ac[q];
        }
      }
      __syncthreads();                            // this round's y blocks are complete
      have = have_n;
      I = In;
      J = Jn;
#pragma unroll
      for (int k = 0; k < 8; ++k) m[k] = mn[k];
    }
    const bool plain = alpha == 1.0, overwrite = beta == 0.0;
    for (int t = tid; t < n * 8; t += blockDim.x) {
      const int q = t / n, r = t - q * n;
      if (q >= rb) continue;
      double* dst = y + (rb0 + q) * y_rs + cell * y_cs + r;
      const double v = plain ? (double)ys[r * 9 + q] : alpha * (double)ys[r * 9 + q];
      *dst = overwrite ? v : v + beta * (*dst);
    }
  }
}

// Coarse restriction and prolongation of the inner iterations (the coarse term of Eq. 48) with the
// FP32 copy of U_dp_ring (the dual rows of U_rp_ring), [cell][n_d][NP] row-major:
//   udp_t:  cp[rhs][cell][p] = sum_d U[d][p] g[rhs][cell][d]
//   udp_n:  y[rhs][cell][d]  = alpha sum_p U[d][p] cp[rhs][cell][p] + beta y
// One CTA per cell.  In udp_t a thread owns four consecutive p of every RG-th row (one 16-byte
// load per row), accumulates them for up to eight RHS in FP32 and the RG row groups are summed in
// shared memory; in udp_n a thread owns a row.
template <int NP>
__global__ void __launch_bounds__(256, 3) udp_t_f32_kernel(const float* __restrict__ U, int nd,
                                                        const double* __restrict__ g, long long g_rs, int g_cs,
                                                        double* __restrict__ cp, long long c_rs, int c_cs,
                                                        int nrhs) {
  constexpr int G = NP / 4;          // 16-byte groups per row
  constexpr int RG = 256 / G;        // row groups
  extern __shared__ __align__(16) float smu[];   // gs[nd][8], red[RG * G][32]
  float* gs = smu;
  float* red = smu + (size_t)nd * 8;
  const long long cell = blockIdx.x;
  const int tid = threadIdx.x;
  const int grp = tid % G, rg = tid / G;
  const float4* Uc = reinterpret_cast<const float4*>(U + cell * (long long)nd * NP);
  for (int rb0 = 0; rb0 < nrhs; rb0 += 8) {
    const int rb = min(8, nrhs - rb0);
    __syncthreads();
    for (int t = tid; t < nd * 8; t += blockDim.x) {
      const int q = t / nd, d = t - q * nd;
      gs[d * 8 + q] = q < rb ? (float)g[(rb0 + q) * g_rs + cell * g_cs + d] : 0.f;
    }
    __syncthreads();
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[a][q] = 0.f;
    if (rg < RG) {
#pragma unroll 4
      for (int d = rg; d < nd; d += RG) {
        const float4 u = __ldcs(Uc + (long long)d * G + grp);
        const float4 x0 = reinterpret_cast<const float4*>(gs)[d * 2];
        const float4 x1 = reinterpret_cast<const float4*>(gs)[d * 2 + 1];
        const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        const float uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int q = 0; q < 8; ++q) acc[a][q] = fmaf(uv[a], xv[q], acc[a][q]);
      }
      float4* rd = reinterpret_cast<float4*>(red + (size_t)(rg * G + grp) * 32);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        rd[2 * a] = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
        rd[2 * a + 1] = make_float4(acc[a][4], acc[a][5], acc[a][6], acc[a][7]);
      }
    }
    __syncthreads();
    for (int o = tid; o < NP * 8; o += blockDim.x) {
      const int p = o >> 3, q = o & 7;
      const int gp = p >> 2, a = p & 3;
      float sum = 0.f;
      for (int k = 0; k < RG; ++k) sum += red[(size_t)(k * G + gp) * 32 + a * 8 + q];
      if (q < rb) cp[(rb0 + q) * c_rs + cell * c_cs + p] = (double)sum;
    }
  }
}

template <int NP>
__global__ void __launch_bounds__(1024) udp_n_f32_kernel(const float* __restrict__ U, int nd,
                                                         const double* __restrict__ cp, long long c_rs, int c_cs,
                                                         double* __restrict__ y, long long y_rs, int y_cs,
                                                         double alpha, double beta, int nrhs) {
  constexpr int G = NP / 4;
  __shared__ __align__(16) float cs[NP][8];
  const long long cell = blockIdx.x;
  const int tid = threadIdx.x;
  const float4* Uc = reinterpret_cast<const float4*>(U + cell * (long long)nd * NP);
  for (int rb0 = 0; rb0 < nrhs; rb0 += 8) {
    const int rb = min(8, nrhs - rb0);
    __syncthreads();
    for (int t = tid; t < NP * 8; t += blockDim.x) {
      const int p = t >> 3, q = t & 7;
      cs[p][q] = q < rb ? (float)cp[(rb0 + q) * c_rs + cell * c_cs + p] : 0.f;
    }
    __syncthreads();
    for (int d = tid; d < nd; d += blockDim.x) {
      float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int gq = 0; gq < G; ++gq) {
        const float4 u = __ldcs(Uc + (long long)d * G + gq);
        const float uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float4 x0 = reinterpret_cast<const float4*>(cs[4 * gq + a])[0];
          const float4 x1 = reinterpret_cast<const float4*>(cs[4 * gq + a])[1];
          acc[0] = fmaf(uv[a], x0.x, acc[0]);
          acc[1] = fmaf(uv[a], x0.y, acc[1]);
          acc[2] = fmaf(uv[a], x0.z, acc[2]);
          acc[3] = fmaf(uv[a], x0.w, acc[3]);
          acc[4] = fmaf(uv[a], x1.x, acc[4]);
          acc[5] = fmaf(uv[a], x1.y, acc[5]);
          acc[6] = fmaf(uv[a], x1.z, acc[6]);
          acc[7] = fmaf(uv[a], x1.w, acc[7]);
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q < rb) {
          double* dst = y + (rb0 + q) * y_rs + cell * y_cs + d;
          *dst = (beta == 0.0) ? alpha * (double)acc[q] : alpha * (double)acc[q] + beta * (*dst);
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

// Eq. 46b for one (rhs, cell) per warp.
//  1. G = R^T (K R) and h = R^T v.  G is formed in 32 x 32 blocks (upper blocks only, then
//     mirrored): lane r owns row r of the block.  Chunks of 32 entries of the basis vectors are
//     staged in shared memory, the R rows with a padded stride (each lane reads its own row,
//     conflict-free) and the K R chunk transposed with 16-byte rows (all lanes read the same
//     address: broadcast, four values per load).  Products in the basis type, chunk sums in FP64.
//  2. Diagonal-pivoted Cholesky, right-looking: each step takes the largest remaining Schur
//     diagonal (lowest index on ties), stops when it is not above drop_rel * max diag(G), stores
//     the scaled pivot column as the next column of L and applies the rank-1 update (lanes own
//     matrix columns, so the row-major updates are conflict-free).
//  3. L y = h(piv), L^T c(piv) = y (column-oriented, lane-parallel), c = 0 off the pivots,
//     and x = R c.
// Scratch per warp (doubles): S (nrb x (nrb + 1)), h, y, c, pivot column (nrb each), nrb pivot
// ints (in nrb doubles), 2 scalars, two v chunks (2 x 32), then one region shared by the two
// buffers of the two staging tiles (32 rows x kGramLd values of the basis type each; phase 1)
// and L (nrb x (nrb + 1); phase 2), padded to an even count.
constexpr int kMaxRb = 64;
constexpr int kGramQ = 32;     // basis-vector entries per staged chunk
constexpr int kGramLd = 36;    // row stride of a staged tile (16-byte rows, 4-bank row offset)
__host__ __device__ inline int gram_warp_head(int nrb) {
  const int fixed = nrb * (nrb + 1) + 5 * nrb + 2 + 2 * kGramQ;
  return fixed + (fixed & 1);   // the shared region starts 16-byte aligned
}
__host__ __device__ inline int gram_warp_doubles(int nrb, int tb_bytes) {
  const int tiles = (2 * 2 * kGramQ * kGramLd * tb_bytes + 7) / 8;
  const int lmat = nrb * (nrb + 1);
  const int tot = gram_warp_head(nrb) + (tiles > lmat ? tiles : lmat);
  return tot + (tot & 1);
}

// One element (4 or 8 bytes) global -> shared without waiting; zero-filled when !valid.
template <typename TB>
__device__ __forceinline__ void cp_async_elem(TB* dst, const TB* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? (int)sizeof(TB) : 0;
  if (sizeof(TB) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}

__device__ __forceinline__ void load4(const float* p, float (&o)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void load4(const double* p, double (&o)[4]) {
  const double2 t0 = *reinterpret_cast<const double2*>(p);
  const double2 t1 = *reinterpret_cast<const double2*>(p + 2);
  o[0] = t0.x; o[1] = t0.y; o[2] = t1.x; o[3] = t1.y;
}

// Diagonal-pivoted Cholesky solve of one symmetric nrb x nrb system by one warp, on the warp's
// shared scratch (row stride ld = nrb + 1): S holds G (overwritten), hs the right-hand side; the
// coefficients land in cs (0 off the pivots).  Each step takes the largest remaining Schur
// diagonal (lowest index on ties) and stops when it is not above drop_rel * max diag(G); the
// scaled pivot column is the next column of L and the rank-1 update runs with lanes over columns.
// Then L y = h(piv), L^T c(piv) = y, column-oriented and lane-parallel.
__device__ void warp_pivoted_gram_solve(double* S, double* Lc, const double* hs, double* ys, double* cs,
                                        double* colv, int* piv, int nrb, int ld, double drop_rel, int lane) {
  double dmax = 0.0;
  for (int i = 0; i < nrb; ++i) dmax = fmax(dmax, S[i * ld + i]);
  unsigned long long used = 0ull;                   // identical in every lane
  int np = 0;
  while (np < nrb) {
    // largest remaining Schur diagonal, lowest index on ties (lane-parallel, then a warp argmax)
    int jb = -1;
    double best = 0.0;
    for (int i = lane; i < nrb; i += 32) {
      if ((used >> i) & 1ull) continue;
      const double dv = S[i * ld + i];
      if (jb < 0 || dv > best) { best = dv; jb = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, jb, o);
      if (oj >= 0 && (jb < 0 || ob > best || (ob == best && oj < jb))) { best = ob; jb = oj; }
    }
    if (jb < 0 || !(best > drop_rel * dmax)) break;   // uniform across the warp
    used |= 1ull << jb;
    if (lane == 0) piv[np] = jb;
    const double inv = 1.0 / sqrt(best);
    for (int i = lane; i < nrb; i += 32) {
      const double cv = S[i * ld + jb] * inv;
      colv[i] = cv;
      Lc[np * ld + i] = cv;
    }
    __syncwarp();
    for (int i = 0; i < nrb; ++i) {                    // lanes own columns j
      if ((used >> i) & 1ull) continue;                // pivoted rows are not read again
      const double ci = colv[i];
      for (int j = lane; j < nrb; j += 32) S[i * ld + j] -= ci * colv[j];
    }
    ++np;
    __syncwarp();
  }

  for (int i = lane; i < nrb; i += 32) { ys[i] = hs[i]; cs[i] = 0.0; }
  __syncwarp();
  for (int a = 0; a < np; ++a) {                       // forward: column a of L
    const int pa = piv[a];
    const double ya = ys[pa] / Lc[a * ld + pa];
    __syncwarp();
    for (int r = a + 1 + lane; r < np; r += 32) ys[piv[r]] -= Lc[a * ld + piv[r]] * ya;
    if (lane == 0) colv[a] = ya;                       // y in pivot order
    __syncwarp();
  }
  for (int a = np - 1; a >= 0; --a) {                  // backward: row a of L^T = column a of L
    const int pa = piv[a];
    const double ca = colv[a] / Lc[a * ld + pa];
    __syncwarp();
    for (int r = lane; r < a; r += 32) colv[r] -= Lc[r * ld + pa] * ca;
    if (lane == 0) cs[pa] = ca;
    __syncwarp();
  }
}

// The same diagonal-pivoted Cholesky solve by a whole CTA (nthreads threads, all of them calling):
// warp 0 picks the pivot, every thread forms part of the pivot column and of the rank-1 update,
// which touches only the upper triangle of the unpivoted rows and columns (S stays symmetric there;
// each entry receives the same FP64 operations in the same order as in the warp solve, and the
// pivot's scale is one rsqrt instead of a square root and a division, the step's latency on
// GB300's FP64 unit).  The substitutions run on warp 0.  sh holds a double and an int of
// block-shared scratch.  nthreads is a multiple of 64 and nrb <= 64.
__device__ void block_pivoted_gram_solve(double* S, double* Lc, const double* hs, double* ys, double* cs,
                                         double* colv, int* piv, double* sh_inv, int* sh_jb, int nrb, int ld,
                                         double drop_rel, int tid, int nthreads) {
  const int lane = tid & 31, warp = tid >> 5;
  double dmax = 0.0;                                 // needed by warp 0 only
  if (warp == 0) {
    for (int i = lane; i < nrb; i += 32) dmax = fmax(dmax, S[i * ld + i]);
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  }
  unsigned long long used = 0ull;                   // identical in every thread
  int np = 0;
  while (np < nrb) {
    if (warp == 0) {
      int jb = -1;
      double best = 0.0;
      for (int i = lane; i < nrb; i += 32) {
        if ((used >> i) & 1ull) continue;
        const double dv = S[i * ld + i];
        if (jb < 0 || dv > best) { best = dv; jb = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, jb, o);
        if (oj >= 0 && (jb < 0 || ob > best || (ob == best && oj < jb))) { best = ob; jb = oj; }
      }
      if (lane == 0) {
        const bool take = jb >= 0 && best > drop_rel * dmax;
        *sh_jb = take ? jb : -1;
        if (take) { *sh_inv = rsqrt(best); piv[np] = jb; }   // one call on the pivot chain
      }
    }
    __syncthreads();
    const int jb = *sh_jb;
    if (jb < 0) break;                                 // uniform across the block
    const double inv = *sh_inv;
    used |= 1ull << jb;
    for (int i = tid; i < nrb; i += nthreads) {
      const double cv = S[min(i, jb) * ld + max(i, jb)] * inv;
      colv[i] = cv;
      Lc[np * ld + i] = cv;
    }
    __syncthreads();
    // nrb <= 64 and nthreads a multiple of 64: the thread's column j is fixed, its rows step by
    // nthreads / 64 up to the diagonal
    {
      const int j = tid & 63, rs = nthreads >> 6;
      if (j < nrb && !((used >> j) & 1ull)) {
        const double cj = colv[j];
        for (int i = tid >> 6; i <= j; i += rs)
          if (!((used >> i) & 1ull)) S[i * ld + j] -= colv[i] * cj;
      }
    }
    ++np;
    __syncthreads();
  }
  if (warp != 0) return;
  for (int i = lane; i < nrb; i += 32) { ys[i] = hs[i]; cs[i] = 0.0; }
  __syncwarp();
  for (int a = 0; a < np; ++a) {
    const int pa = piv[a];
    const double ya = ys[pa] / Lc[a * ld + pa];
    __syncwarp();
    for (int r = a + 1 + lane; r < np; r += 32) ys[piv[r]] -= Lc[a * ld + piv[r]] * ya;
    if (lane == 0) colv[a] = ya;
    __syncwarp();
  }
  for (int a = np - 1; a >= 0; --a) {
    const int pa = piv[a];
    const double ca = colv[a] / Lc[a * ld + pa];
    __syncwarp();
    for (int r = lane; r < a; r += 32) colv[r] -= Lc[r * ld + pa] * ca;
    if (lane == 0) cs[pa] = ca;
    __syncwarp();
  }
}

// s + c += x with Neumaier's compensation (c collects the rounding error of every addition)
template <typename T>
__device__ __forceinline__ void neumaier_add(T& s, T& c, T x) {
  if (sizeof(T) == 8) {   // FP64 sums need no compensation at these lengths
    s += x;
    return;
  }
  const T t = s + x;
  c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

// Eq. 46b in FP32 for one (rhs, cell) per block of 256 threads: G = R^T (K R) and h = R^T v from
// 32-entry chunks of the basis staged in shared memory, each thread a strided 4 x 4 tile of G
// (rows ti + 16a, columns tj + 16b: a broadcast read of R and a conflict-free read of K R per
// product), FP32 chunk sums accumulated with Neumaier's compensation; then warp 0 runs the same
// diagonal-pivoted Cholesky solve as the warp kernel, and all threads form x = R c.
constexpr int kGbQ = 32;
constexpr int kGbLd = 36;   // 16-byte rows; a warp's 16 distinct K R rows take the minimum two wavefronts
// The two staging stages of R, K R and v (filled by cp.async one chunk ahead) live inside the L
// factor's region, used only after the Gram matrix is complete: a 64-basis block needs 74 KB and
// three blocks fit an SM.
__host__ __device__ inline size_t gram_block_stage_floats(int nrb) { return 2 * (size_t)nrb * kGbLd + kGbQ; }
__host__ __device__ inline size_t gram_block_smem(int nrb) {
  const size_t ld = (size_t)nrb + 1;
  const size_t stage = 2 * sizeof(float) * gram_block_stage_floats(nrb);
  const size_t lc = sizeof(double) * nrb * ld;
  return sizeof(double) * (nrb * ld + 6 * (size_t)nrb + 2) + (stage > lc ? stage : lc);
}
__global__ void __launch_bounds__(256, 3) gram_block_f32_kernel(const float* __restrict__ R, const float* __restrict__ KR,
                                                             const double* __restrict__ v, long long v_rs, int v_cs,
                                                             double* __restrict__ x, long long x_rs, int x_cs, int nr,
                                                             int nrb, long long ncell, double drop_rel) {
  extern __shared__ __align__(16) double gbsm[];
  const int ld = nrb + 1;
  double* S = gbsm;                                  // [nrb][ld]
  double* hs = S + (size_t)nrb * ld;
  double* ys = hs + nrb;
  double* cs = ys + nrb;
  double* colv = cs + nrb;
  int* piv = reinterpret_cast<int*>(colv + nrb);     // nrb ints in 2 nrb doubles of room
  double* sh_inv = colv + 3 * nrb;
  int* sh_jb = reinterpret_cast<int*>(sh_inv + 1);
  double* Lc = sh_inv + 2;                           // [nrb][ld], after the Gram matrix is formed
  float* stage0 = reinterpret_cast<float*>(Lc);      // two staging stages while it is formed
  const size_t stage_f = gram_block_stage_floats(nrb);
  const long long col = blockIdx.x;                  // rhs * ncell + cell
  const int rhs = (int)(col / ncell);
  const long long cell = col - (long long)rhs * ncell;
  const float* Rc = R + col * (long long)nrb * nr;
  const float* KRc = KR + col * (long long)nrb * nr;
  const double* vc = v + rhs * v_rs + cell * v_cs;
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  float acc[4][4], cmp[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b] = 0.f; cmp[a][b] = 0.f; }
  float hacc = 0.f, hcmp = 0.f;
  // chunk k of R and K R goes to stage k & 1 by cp.async (zero-filled past n_r), one chunk ahead
  auto issue = [&](int q0, float* st) {
    float* Rs_ = st;
    float* Ks_ = st + (size_t)nrb * kGbLd;
    for (int t = tid; t < nrb * kGbQ; t += blockDim.x) {
      const int i = t / kGbQ, qq = t - i * kGbQ, q = q0 + qq;
      const bool in = q < nr;
      cp_async_elem(Rs_ + i * kGbLd + qq, Rc + (size_t)i * nr + (in ? q : 0), in);
      cp_async_elem(Ks_ + i * kGbLd + qq, KRc + (size_t)i * nr + (in ? q : 0), in);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  const int nchunk = (nr + kGbQ - 1) / kGbQ;
  issue(0, stage0);
  float part[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) part[a][b] = 0.f;
  float hp = 0.f;
  for (int ck = 0; ck < nchunk; ++ck) {
    const int q0 = ck * kGbQ;
    float* Rs = stage0 + (ck & 1) * stage_f;
    float* Ks = Rs + (size_t)nrb * kGbLd;
    float* vs = Ks + (size_t)nrb * kGbLd;
    if (ck + 1 < nchunk) {
      issue(q0 + kGbQ, stage0 + ((ck + 1) & 1) * stage_f);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    if (tid < kGbQ) vs[tid] = q0 + tid < nr ? (float)vc[q0 + tid] : 0.f;
    __syncthreads();                                  // chunk ck (and its v) is in place
#pragma unroll 2
    for (int qq = 0; qq < kGbQ; qq += 4) {
      float4 rv[4], kv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int i = ti + 16 * a, j = tj + 16 * a;
        rv[a] = i < nrb ? *reinterpret_cast<const float4*>(Rs + i * kGbLd + qq) : make_float4(0.f, 0.f, 0.f, 0.f);
        kv[a] = j < nrb ? *reinterpret_cast<const float4*>(Ks + j * kGbLd + qq) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          float p = part[a][b];
          p = fmaf(rv[a].x, kv[b].x, p);
          p = fmaf(rv[a].y, kv[b].y, p);
          p = fmaf(rv[a].z, kv[b].z, p);
          p = fmaf(rv[a].w, kv[b].w, p);
          part[a][b] = p;
        }
    }
    if (tid < nrb)
      for (int qq = 0; qq < kGbQ; ++qq) hp = fmaf(Rs[tid * kGbLd + qq], vs[qq], hp);
    // the partial sums of two chunks (64 terms) are added with Neumaier's compensation
    if ((ck & 1) || ck + 1 == nchunk) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          neumaier_add(acc[a][b], cmp[a][b], part[a][b]);
          part[a][b] = 0.f;
        }
      if (tid < nrb) neumaier_add(hacc, hcmp, hp);
      hp = 0.f;
    }
    __syncthreads();                                  // stage ck & 1 is refilled at chunk ck + 2
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = ti + 16 * a, j = tj + 16 * b;
      if (i < nrb && j < nrb && i <= j) S[i * ld + j] = (double)acc[a][b] + (double)cmp[a][b];
    }
  if (tid < nrb) hs[tid] = (double)hacc + (double)hcmp;
  __syncthreads();
  for (int t = tid; t < nrb * nrb; t += blockDim.x) {   // the upper triangle, mirrored
    const int i = t / nrb, j = t - (t / nrb) * nrb;
    if (i > j) S[i * ld + j] = S[j * ld + i];
  }
  __syncthreads();
  block_pivoted_gram_solve(S, Lc, hs, ys, cs, colv, piv, sh_inv, sh_jb, nrb, ld, drop_rel, tid, blockDim.x);
  __syncthreads();
  float* csf = reinterpret_cast<float*>(ys);         // the coefficients in FP32, converted once
  if (tid < nrb) csf[tid] = (float)cs[tid];
  __syncthreads();
  double* xc = x + rhs * x_rs + cell * x_cs;
  for (int q = tid; q < nr; q += blockDim.x) {
    float sx = 0.f;
#pragma unroll 8
    for (int i = 0; i < nrb; ++i) sx = fmaf(csf[i], Rc[(size_t)i * nr + q], sx);
    xc[q] = (double)sx;
  }
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
  const int ld = nrb + 1;
  double* S = gwsm + (size_t)wib * gram_warp_doubles(nrb, (int)sizeof(TB));
  double* hs = S + nrb * ld;
  double* ys = hs + nrb;
  double* cs = ys + nrb;
  double* colv = cs + nrb;
  int* piv = reinterpret_cast<int*>(colv + nrb);
  double* sc = colv + 2 * nrb;
  double* vq = sc + 2;                              // [2][32]: v chunks
  double* region = S + gram_warp_head(nrb);
  TB* Rs = reinterpret_cast<TB*>(region);           // phase 1: [2][32 rows][kGramLd]
  TB* Ks = Rs + 2 * kGramQ * kGramLd;               // phase 1: [2][32 rows][kGramLd]
  double* Lc = region;                              // phase 2: column a of L at Lc[a * ld + i]
  const int rhs = (int)(col / ncell);
  const long long cell = col - (long long)rhs * ncell;
  const TB* Rc = R + col * (long long)nrb * nr;
  const TB* KRc = KR + col * (long long)nrb * nr;
  const double* vc = v + rhs * v_rs + cell * v_cs;
  const int nchunk = (nr + kGramQ - 1) / kGramQ;

  // ---- 1. G (upper blocks) and h.  Rows of R and K R are staged chunk by chunk (row-major,
  // lane = entry q, one async copy per element), the next chunk in flight while this one is
  // used.  Lane j accumulates column j of the block: per row i and 4 entries one broadcast
  // 16-byte read of R and 4 FMAs against the lane's own K R values.
  for (int ib = 0; ib < nrb; ib += 32) {
    const int ni = min(32, nrb - ib);
    for (int jb = ib; jb < nrb; jb += 32) {
      const int nj = min(32, nrb - jb);
      const bool diag = (jb == ib);
      // chunk sums in the basis type, accumulated over chunks with Neumaier compensation (as
      // accurate as FP64 chunk sums, with no FP64 pipe work in the FP32 path)
      TB gacc[32], gcmp[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) { gacc[i] = TB(0); gcmp[i] = TB(0); }
      TB hacc = TB(0), hcmp = TB(0);
      auto stage = [&](int buf, int ch) {
        const int q = ch * kGramQ + lane;
        const bool in = q < nr;
        TB* rs = Rs + buf * kGramQ * kGramLd;
        TB* ks = Ks + buf * kGramQ * kGramLd;
        for (int r = 0; r < 32; ++r) {
          cp_async_elem(rs + r * kGramLd + lane, Rc + (size_t)(ib + (r < ni ? r : 0)) * nr + (in ? q : 0),
                        in && r < ni);
          cp_async_elem(ks + r * kGramLd + lane, KRc + (size_t)(jb + (r < nj ? r : 0)) * nr + (in ? q : 0),
                        in && r < nj);
        }
        if (diag) vq[buf * kGramQ + lane] = in ? vc[q] : 0.0;
        asm volatile("cp.async.commit_group;\n" ::: "memory");
      };
      __syncwarp();
      stage(0, 0);
      for (int ch = 0; ch < nchunk; ++ch) {
        const int buf = ch & 1;
        if (ch + 1 < nchunk) {
          stage(buf ^ 1, ch + 1);
          asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
          asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncwarp();
        const TB* rs = Rs + buf * kGramQ * kGramLd;
        const TB* ks = Ks + buf * kGramQ * kGramLd;
        TB acc[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] = TB(0);
#pragma unroll
        for (int q = 0; q < kGramQ; q += 4) {
          TB k4[4];
          load4(ks + lane * kGramLd + q, k4);
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            TB r4[4];
            load4(rs + i * kGramLd + q, r4);   // broadcast
            acc[i] = fma(r4[0], k4[0], acc[i]);
            acc[i] = fma(r4[1], k4[1], acc[i]);
            acc[i] = fma(r4[2], k4[2], acc[i]);
            acc[i] = fma(r4[3], k4[3], acc[i]);
          }
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) neumaier_add(gacc[i], gcmp[i], acc[i]);
        if (diag) {   // h_i, lane i
          TB hsum = TB(0);
          for (int q = 0; q < kGramQ; ++q) hsum += rs[lane * kGramLd + q] * (TB)vq[buf * kGramQ + q];
          neumaier_add(hacc, hcmp, hsum);
        }
        __syncwarp();   // this buffer is refilled by the next stage call
      }
      if (lane < nj) {
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i < ni && (!diag || i <= lane)) S[(ib + i) * ld + jb + lane] = (double)gacc[i] + (double)gcmp[i];
      }
      if (diag && lane < ni) hs[ib + lane] = (double)hacc + (double)hcmp;
    }
  }
  __syncwarp();
  for (int t = lane; t < nrb * nrb; t += 32) {      // mirror the upper triangle
    const int i = t / nrb, j = t - (t / nrb) * nrb;
    if (i > j) S[i * ld + j] = S[j * ld + i];
  }
  __syncwarp();

  warp_pivoted_gram_solve(S, Lc, hs, ys, cs, colv, piv, nrb, ld, drop_rel, lane);
  __syncwarp();
  double* xc = x + rhs * x_rs + cell * x_cs;
  for (int q = lane; q < nr; q += 32) {
    TB sx = TB(0);
    for (int i = 0; i < nrb; ++i) sx += (TB)cs[i] * Rc[(size_t)i * nr + q];
    xc[q] = (double)sx;
  }
}

// The two Eq. 42 systems of every cell from its traces Y[cell] = [A upper (npair), b (nrb),
// M upper (npair)]: pi solves A pi = b, delta solves M delta = dvec (shared right-hand side).
// One warp per (cell, system); same pivoted solve as Eq. 46b.
__global__ void gram_direct_kernel(const double* __restrict__ Y, int ntab, int nrb,
                                   const double* __restrict__ dvec, double* __restrict__ pi,
                                   double* __restrict__ delta, long long ncell, double drop_rel) {
  extern __shared__ double gdsm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long task = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
  if (task >= 2 * ncell) return;                    // the whole warp leaves together
  const long long cell = task >> 1;
  const int sys = (int)(task & 1);                  // 0: pi, 1: delta
  const int ld = nrb + 1;
  const int per = 2 * nrb * ld + 6 * nrb;
  double* S = gdsm + (size_t)wib * (per + (per & 1));
  double* Lc = S + nrb * ld;
  double* hs = Lc + nrb * ld;
  double* ys = hs + nrb;
  double* cs = ys + nrb;
  double* colv = cs + nrb;
  int* piv = reinterpret_cast<int*>(colv + nrb);
  const int npair = nrb * (nrb + 1) / 2;
  const double* y = Y + cell * ntab;
  const double* g = y + (sys == 0 ? 0 : npair + nrb);
  for (int p = lane; p < npair; p += 32) {
    int i = 0, rem = p;
    while (rem >= nrb - i) { rem -= nrb - i; ++i; }
    const int j = i + rem;
    S[i * ld + j] = g[p];
    S[j * ld + i] = g[p];
  }
  for (int i = lane; i < nrb; i += 32) hs[i] = (sys == 0) ? y[npair + i] : dvec[i];
  __syncwarp();
  warp_pivoted_gram_solve(S, Lc, hs, ys, cs, colv, piv, nrb, ld, drop_rel, lane);
  __syncwarp();
  double* out = (sys == 0 ? pi : delta) + cell * nrb;
  for (int i = lane; i < nrb; i += 32) out[i] = cs[i];
}

// g[rhs][cell] = - sum_e sum_gp w G(w)^T dC_hat/dr G(u), one block per (rhs, cell).
template <int D>
__global__ void grad_kernel(Geo g, const double* __restrict__ r_cell, long long ncell, int n,
                            const double* __restrict__ u, const double* __restrict__ w, long long u_rs,
                            double* __restrict__ out, long long out_rs, double wq, double inv_h) {
  extern __shared__ double sm[];
  constexpr int NA = 1 << D;
  constexpr int NI = D * D;
  const long long col = blockIdx.x;
  const int rhs = (int)(col / ncell);
  const long long cell = col - (long long)rhs * ncell;   // cell within this launch's lattice
  const double* uc = u + rhs * u_rs + cell * n;
  const double* wc = w + rhs * u_rs + cell * n;
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
    out[rhs * out_rs + cell] = -s;
  }
}

}  // namespace

fetidp_status k_snapshots(Ctx& c) {
  ProfScope ps(c, FETIDP_K_SETUP, 0.0, (double)c.N * c.nsnap * 8.0);
  const long long total = c.N * c.nelem * c.ngp;
  int grid = ceil_div(total, 256);
  if (grid > 152 * 32) grid = 152 * 32;
  for (const LatticeSpan& ls : c.lat) {   // one launch per lattice: its own geometry and radii
    snapshot_kernel<<<grid, 256, 0, c.stream>>>(ls.geo, c.r_dev + ls.cell0, ls.ncell, c.nelem, c.ngp, c.nc,
                                                c.snap + ls.cell0 * c.nsnap);
    FD_CHECK_LAUNCH();
  }
  return FETIDP_OK;
}

// u, y: column (rhs, cell) holds nvec vectors of length len (n, or n_r when r_only).
fetidp_status k_apply_K(Ctx& c, CCellVec u, CellVec y, int nvec, int nrhs, bool idp, bool r_only,
                        const double* chat, double /*unused*/, int len_override) {
  const int len = len_override > 0 ? len_override : (r_only ? c.nr : c.n);
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

// FP32 element matrices of every cell (mixed path), formed once per setup.
fetidp_status k_krr_ell_assemble(Ctx& c, const int* cnt, const int* idx, int cmax) {
  const int NA = 1 << c.d, ND = NA * c.d;
  FD_TRY(dalloc_t(c, &c.krr_val, (size_t)c.N * c.krr_nnz * c.nr));
  ProfScope ps(c, FETIDP_K_SETUP, 0.0, 4.0 * (double)c.N * c.krr_nnz * c.nr * 2.0);
  const long long work = c.N * (long long)c.krr_nnz * c.nr;
  const int grid = (int)std::min<long long>((work + 255) / 256, 152LL * 64);
  krr_ell_assemble_kernel<<<grid, 256, 0, c.stream>>>(c.Ke_all, (long long)c.nelem * ND * ND, cnt, idx, cmax,
                                                     c.krr_nnz, c.nr, c.N, c.krr_val);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_element_matrices_f32(Ctx& c) {
  const int NA = 1 << c.d, ND = NA * c.d;
  FD_TRY(dalloc_t(c, &c.Ke_all, (size_t)c.N * c.nelem * ND * ND));
  ProfScope ps(c, FETIDP_K_SETUP, 0.0, (double)c.N * (c.nsnap * 8.0 + (double)c.nelem * ND * ND * 4.0));
  const float h = 1.0f / c.e;
  const float wq = (float)pow(0.5 / c.e, c.d);
  const long long work = c.N * c.nelem * ND;
  const int grid = (int)std::min<long long>((work + 255) / 256, 152LL * 64);
  if (c.d == 2)
    element_matrices_f32_kernel<2><<<grid, 256, 0, c.stream>>>(c.snap, c.N, c.e, c.nc, wq, 1.0f / h, c.Ke_all);
  else
    element_matrices_f32_kernel<3><<<grid, 256, 0, c.stream>>>(c.snap, c.N, c.e, c.nc, wq, 1.0f / h, c.Ke_all);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

// FP32 variant (local ROM bases of the mixed path): u, y float with the same view strides.
fetidp_status k_apply_K_f32(Ctx& c, const float* u, long long u_rs, int u_cs, float* y, long long y_rs,
                            int y_cs, int nvec, int nrhs, bool idp, bool r_only, long long ext) {
  if (idp && r_only && c.krr_val) {   // sparse K_rr in ELL form
    const int nchunk = (nvec + kSpVB - 1) / kSpVB;
    const size_t smem = (size_t)c.nr * kSpLd * sizeof(float);
    // algorithmic work: one FMA per stored entry and vector; bytes: the values once per cell, the
    // vectors in and out
    ProfScope ps(c, FETIDP_K_MULTI_K, 2.0 * (double)c.N * nrhs * nvec * c.krr_nnz * c.nr,
                 4.0 * (double)c.N * c.krr_nnz * c.nr + 8.0 * (double)c.N * nrhs * nvec * c.nr);
    const int nnode = c.nr / c.d;
    const size_t smem_n = smem + sizeof(float) * 2 * (size_t)c.d * c.nr;
    if (c.krr_nbr && nnode <= 352 && smem_n <= 113 * 1024) {
      const int threads = (nnode + 31) / 32 * 32;
      if (c.d == 3) {
        cudaFuncSetAttribute(krr_spmm_nodal_f32_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_n);
        krr_spmm_nodal_f32_kernel<3><<<(unsigned)(c.N * nrhs * nchunk), threads, smem_n, c.stream>>>(
            c.krr_nbr, c.krr_val, c.krr_nnz, c.nr, nrhs, nchunk, u, u_rs, u_cs, y, y_rs, y_cs, nvec, ext);
      } else {
        cudaFuncSetAttribute(krr_spmm_nodal_f32_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_n);
        krr_spmm_nodal_f32_kernel<2><<<(unsigned)(c.N * nrhs * nchunk), threads, smem_n, c.stream>>>(
            c.krr_nbr, c.krr_val, c.krr_nnz, c.nr, nrhs, nchunk, u, u_rs, u_cs, y, y_rs, y_cs, nvec, ext);
      }
    } else {
      cudaFuncSetAttribute(krr_spmm_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      krr_spmm_f32_kernel<<<(unsigned)(c.N * nrhs * nchunk), 256, smem, c.stream>>>(
          c.krr_col, c.krr_val, c.krr_nnz, c.nr, nrhs, nchunk, u, u_rs, u_cs, y, y_rs, y_cs, nvec, ext);
    }
    FD_CHECK_LAUNCH();
    return FETIDP_OK;
  }
  if (!c.Ke_all) {
    set_error("multi-vector K_s: element matrices not formed");
    return FETIDP_EINVAL;
  }
  const int len = r_only ? c.nr : c.n;
  const int NA = 1 << c.d, ND = NA * c.d;
  const int half = (c.e + 1) / 2;
  const int nelc_max = half * half * (c.d == 3 ? half : 1);
  const int kes = c.d == 2 ? multi_ke_stride(2) : multi_ke_stride(3);
  const size_t fixed = (size_t)nelc_max * kes * sizeof(float) + 16 + (size_t)c.n * sizeof(int);
  // vectors per chunk: as many as fit beside one colour's element matrices (<= 16) with two
  // blocks per SM (one block's global loads and stores overlap the other's arithmetic), else
  // as many as fit with one
  auto bytes = [&](int vb) { return fixed + 2 * (size_t)c.n * (vb + 1) * sizeof(float); };
  size_t budget = 110 * 1024;
  int VB = (int)std::min<long long>(16, nvec);
  while (VB > 1 && bytes(VB) > budget) --VB;
  if (bytes(VB) > budget) {
    budget = 220 * 1024;
    VB = (int)std::min<long long>(32, nvec);
    while (VB > 1 && bytes(VB) > budget) --VB;
  }
  if (bytes(VB) > budget) {
    set_error("multi-vector K_s: cell too large for shared memory");
    return FETIDP_EINVAL;
  }
  {
    // algorithmic work: one K_e product (ND^2 FMA) per element and vector; bytes: the element
    // matrices once per cell, the vectors in and out
    const double cols = (double)c.N * nrhs;
    c.prof_pending_flops = 2.0 * cols * c.nelem * (double)nvec * ND * ND;
    c.prof_pending_bytes = (double)c.N * c.nelem * (double)ND * ND * 4.0 + cols * 2.0 * nvec * len * 4.0;
  }
  ProfScope ps(c, FETIDP_K_MULTI_K, c.prof_pending_flops, c.prof_pending_bytes);
  const size_t smem = bytes(VB);
  const int nchunk = (nvec + VB - 1) / VB;
  const dim3 grid((unsigned)(c.N * nrhs * nchunk));
  if (c.d == 2) {
    cudaFuncSetAttribute(apply_K_multi_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    apply_K_multi_kernel<2><<<grid, kMultiThreads, smem, c.stream>>>(
        c.e, c.N, c.n, len, c.perm, idp, u, u_rs, u_cs, y, y_rs, y_cs, nvec, VB, nchunk, nrhs, c.Ke_all, nelc_max,
        ext, ext);
  } else {
    cudaFuncSetAttribute(apply_K_multi_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    apply_K_multi_kernel<3><<<grid, kMultiThreads, smem, c.stream>>>(
        c.e, c.N, c.n, len, c.perm, idp, u, u_rs, u_cs, y, y_rs, y_cs, nvec, VB, nchunk, nrhs, c.Ke_all, nelc_max,
        ext, ext);
  }
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_rom_combine_f32(Ctx& c, const double* src, long long kstride, int ld, int r0, int c0, int rows,
                                int cols, const double* coef, float* out, int ldo, int symT) {
  if (c.nrb > 64) { set_error("n_rb above 64"); return FETIDP_EINVAL; }
  const long long per = (long long)rows * cols;
  long long gy = (c.N + kCombCells - 1) / kCombCells;
  if (gy > 64) gy = 64;
  const dim3 grid((unsigned)((per + 255) / 256), (unsigned)gy);
  ProfScope ps(c, FETIDP_K_SETUP, 2.0 * c.nrb * per * (double)c.N, 4.0 * per * (double)c.N);
  if (c.nrb <= 16)
    rom_combine_f32_kernel<16><<<grid, 256, 0, c.stream>>>(src, kstride, ld, r0, c0, rows, cols, coef, c.nrb, c.N, out, ldo,
                                                             symT);
  else if (c.nrb <= 32)
    rom_combine_f32_kernel<32><<<grid, 256, 0, c.stream>>>(src, kstride, ld, r0, c0, rows, cols, coef, c.nrb, c.N, out, ldo,
                                                             symT);
  else
    rom_combine_f32_kernel<64><<<grid, 256, 0, c.stream>>>(src, kstride, ld, r0, c0, rows, cols, coef, c.nrb, c.N, out, ldo,
                                                             symT);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_cell_gemm_f32(Ctx& c, const float* mats, int ldm, int nout, int nin, CCellVec x, CellVec y,
                              double alpha, double beta, int nrhs) {
  // algorithmic bytes: the operators once (padded rows as stored), the FP64 vectors in and out
  ProfScope ps(c, FETIDP_K_ASM_OP, 2.0 * nout * nin * (double)c.N * nrhs,
               4.0 * c.N * (double)nin * ldm + 8.0 * c.N * (double)nrhs * (nout + nin));
  if (nout < 1 || nin < 1 || nout > 4 * kAsmMaxThreads || ldm % 4 != 0 || ldm < nout ||
      (size_t)nin * kMaxRhsF32 * sizeof(float) > 200 * 1024 || (reinterpret_cast<uintptr_t>(mats) & 15) != 0) {
    set_error("FP32 cell operators: at most 1024 outputs, rows padded to 16 bytes");
    return FETIDP_EINVAL;
  }
  const size_t smem = (size_t)nin * kMaxRhsF32 * sizeof(float);
  const int threads = ((nout + 3) / 4 + 31) / 32 * 32;
  cudaFuncSetAttribute(cell_gemm_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cell_gemm_f32_kernel<<<(unsigned)c.N, threads, smem, c.stream>>>(mats, ldm, nout, nin, x.p, x.rs, x.cs, y.p,
                                                                   y.rs, y.cs, alpha, beta, nrhs);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_cell_symv_f32(Ctx& c, const float* mats, CCellVec x, CellVec y, double alpha, double beta,
                              int nrhs) {
  const int T = c.sym_T, n = c.nd;
  const long long ntile = (long long)T * (T + 1) / 2;
  // algorithmic bytes: the packed operator once, the FP64 vectors in and out
  ProfScope ps(c, FETIDP_K_ASM_OP, 2.0 * n * n * (double)c.N * nrhs,
               4096.0 * ntile * c.N + 8.0 * c.N * (double)nrhs * 2.0 * n);
  const int nw = (T + 1) / 2;
  if (T < 1 || n > 32 * T || nw > 10 || (reinterpret_cast<uintptr_t>(mats) & 15) != 0) {
    set_error("packed FP32 cell operators: at most 20 tile rows");
    return FETIDP_EINVAL;
  }
  const size_t smem = sizeof(float) * ((size_t)T * 32 * 17 + (size_t)nw * 32 * 33);
  cudaFuncSetAttribute(cell_symv_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cell_symv_f32_kernel<<<(unsigned)c.N, 32 * nw, smem, c.stream>>>(mats, T, n, x.p, x.rs, x.cs, y.p, y.rs, y.cs,
                                                                   alpha, beta, nrhs);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_udp_f32(Ctx& c, bool trans, CCellVec x, CellVec y, double alpha, double beta, int nrhs) {
  const int nd = c.nd, np = c.np;
  if (!c.Udp_f || (np != 8 && np != 24) || nd < 1) { set_error("FP32 U_dp needs n_p of 8 or 24"); return FETIDP_EINVAL; }
  ProfScope ps(c, FETIDP_K_CELL_GEMV, 2.0 * nd * np * (double)c.N * nrhs,
               4.0 * c.N * nd * np + 8.0 * c.N * nrhs * (nd + np + (beta != 0.0 ? nd : 0)));
  if (trans) {
    const int G = np / 4, RG = 256 / G;
    const size_t smem = sizeof(float) * ((size_t)nd * 8 + (size_t)RG * G * 32);
    if (smem > 227 * 1024) { set_error("FP32 U_dp: n_d too large"); return FETIDP_EINVAL; }
    if (np == 8) {
      cudaFuncSetAttribute(udp_t_f32_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      udp_t_f32_kernel<8><<<(unsigned)c.N, 256, smem, c.stream>>>(c.Udp_f, nd, x.p, x.rs, x.cs, y.p, y.rs, y.cs, nrhs);
    } else {
      cudaFuncSetAttribute(udp_t_f32_kernel<24>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      udp_t_f32_kernel<24><<<(unsigned)c.N, 256, smem, c.stream>>>(c.Udp_f, nd, x.p, x.rs, x.cs, y.p, y.rs, y.cs, nrhs);
    }
  } else {
    const int threads = std::min(1024, (nd + 31) / 32 * 32);
    if (np == 8)
      udp_n_f32_kernel<8><<<(unsigned)c.N, threads, 0, c.stream>>>(c.Udp_f, nd, x.p, x.rs, x.cs, y.p, y.rs, y.cs,
                                                                   alpha, beta, nrhs);
    else
      udp_n_f32_kernel<24><<<(unsigned)c.N, threads, 0, c.stream>>>(c.Udp_f, nd, x.p, x.rs, x.cs, y.p, y.rs, y.cs,
                                                                    alpha, beta, nrhs);
  }
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_cell_gemv_strided(Ctx& c, const double* mats, long long mstride, int ld, int mrows,
                                  int mcols, CCellVec x, CellVec y, double alpha, double beta,
                                  int nrhs) {
  ProfScope ps(c, FETIDP_K_CELL_GEMV, 2.0 * mrows * mcols * (double)c.N * nrhs,
               8.0 * c.N * ((double)mrows * mcols + (double)nrhs * (mrows + mcols)));
  const bool aligned16 = (ld % 2 == 0) && (mstride % 2 == 0) && ((reinterpret_cast<uintptr_t>(mats) & 15) == 0);
  if ((mcols == 8 || mcols == 24) && aligned16 && c.N * mrows < (1LL << 31)) {
    const long long total = c.N * mrows;
    long long grid = (total + 255) / 256;
    if (grid > 152LL * 32) grid = 152LL * 32;
    if (mcols == 8)
      cell_gemv_narrow_fixed<8><<<(unsigned)grid, 256, 0, c.stream>>>(mats, mstride, ld, mrows, x.p, x.rs, x.cs, y.p,
                                                                     y.rs, y.cs, alpha, beta, nrhs, c.N);
    else
      cell_gemv_narrow_fixed<24><<<(unsigned)grid, 256, 0, c.stream>>>(mats, mstride, ld, mrows, x.p, x.rs, x.cs,
                                                                      y.p, y.rs, y.cs, alpha, beta, nrhs, c.N);
    FD_CHECK_LAUNCH();
    return FETIDP_OK;
  }
  if (mcols <= 32) {
    const long long total = c.N * mrows;
    long long grid = (total + 255) / 256;
    if (grid > 152LL * 16) grid = 152LL * 16;
    cell_gemv_narrow_kernel<<<(unsigned)grid, 256, 0, c.stream>>>(mats, mstride, ld, mrows, mcols, x.p, x.rs,
                                                                 x.cs, y.p, y.rs, y.cs, alpha, beta, nrhs, c.N);
    FD_CHECK_LAUNCH();
    return FETIDP_OK;
  }
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
                               long long y_k_stride, int prof_class) {
  const long long ncols = ncell * nrhs;
  ProfScope ps(c, prof_class, 2.0 * M * K * nk * (double)ncols,
               8.0 * ((double)nk * M * K + (double)ncols * K + (double)ncols * M * (separate ? nk : 1)));
  dim3 grid((unsigned)ceil_div(ncols, GT), (unsigned)ceil_div(M, GT));
  grouped_gemm_kernel<<<grid, 256, 0, c.stream>>>(A, a_stride_k, lda, M, K, nk, X.p, X.rs, X.cs,
                                                  Y.p, Y.rs, Y.cs, coef, alpha, beta, ncell, nrhs,
                                                  separate, y_k_stride);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

template <typename TB>
static fetidp_status gram_solve_t(Ctx& c, const TB* R, const TB* KR, CCellVec v, CellVec x, int nrhs,
                                  double drop_rel, int len = -1) {
  if (len < 0) len = c.nr;
  if (c.nrb > kMaxRb) {
    set_error("n_rb above 64 is not supported by the Gram solve");
    return FETIDP_EINVAL;
  }
  const long long cols = c.N * nrhs;
  ProfScope ps(c, FETIDP_K_GRAM, cols * 2.0 * len * (c.nrb * (c.nrb + 1) / 2.0 + 2.0 * c.nrb),
               cols * (double)sizeof(TB) * (2.0 * c.nrb * len) + cols * 16.0 * len);
  const size_t per_warp = (size_t)gram_warp_doubles(c.nrb, (int)sizeof(TB)) * sizeof(double);
  int wpb = (int)std::min<size_t>(8, (200 * 1024) / per_warp);
  if (wpb < 1) wpb = 1;
  const size_t smem = per_warp * wpb;
  cudaFuncSetAttribute(gram_warp_kernel<TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  gram_warp_kernel<TB><<<(unsigned)ceil_div(cols, wpb), 32 * wpb, smem, c.stream>>>(
      R, KR, v.p, v.rs, v.cs, x.p, x.rs, x.cs, len, c.nrb, c.N, nrhs, drop_rel);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_gram_solve(Ctx& c, const double* R, const double* KR, CCellVec v, CellVec x,
                           int nrhs, int len) {
  return gram_solve_t<double>(c, R, KR, v, x, nrhs, 1e-12, len);
}

fetidp_status k_gram_solve_f32(Ctx& c, const float* R, const float* KR, CCellVec v, CellVec x,
                               int nrhs, long long r_ext) {
  (void)r_ext;
  if (c.nrb > kMaxRb) {
    set_error("n_rb above 64 is not supported by the Gram solve");
    return FETIDP_EINVAL;
  }
  const long long cols = c.N * nrhs;
  ProfScope ps(c, FETIDP_K_GRAM, cols * 2.0 * c.nr * ((double)c.nrb * c.nrb + c.nrb) + cols * 2.0 * c.nr * c.nrb,
               cols * 4.0 * (2.0 * c.nrb * c.nr) + cols * 16.0 * c.nr);
  const size_t smem = gram_block_smem(c.nrb);
  cudaFuncSetAttribute(gram_block_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  gram_block_f32_kernel<<<(unsigned)cols, 256, smem, c.stream>>>(R, KR, v.p, v.rs, v.cs, x.p, x.rs, x.cs, c.nr,
                                                                  c.nrb, c.N, c.opt.gram_drop_mixed);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_grad(Ctx& c, const double* u, const double* w, double* g) {
  const double h = 1.0 / c.e;
  const double wq = pow(0.5 * h, c.d);
  const size_t smem = 2 * (size_t)c.n * sizeof(double);
  for (const LatticeSpan& ls : c.lat) {   // one launch per lattice: its own geometry and radii
    const dim3 grid((unsigned)(ls.ncell * c.m));
    const long long off = ls.cell0 * c.n;
    if (c.d == 2)
      grad_kernel<2><<<grid, 256, smem, c.stream>>>(ls.geo, c.r_dev + ls.cell0, ls.ncell, c.n, u + off, w + off,
                                                    c.N * c.n, g + ls.cell0, c.N, wq, 1.0 / h);
    else
      grad_kernel<3><<<grid, 256, smem, c.stream>>>(ls.geo, c.r_dev + ls.cell0, ls.ncell, c.n, u + off, w + off,
                                                    c.N * c.n, g + ls.cell0, c.N, wq, 1.0 / h);
    FD_CHECK_LAUNCH();
  }
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

FD_DEFINE_CHECK(fd_check_cell)

fetidp_status k_gram_direct(Ctx& c, const double* Y, int ntab, const double* dvec, double* pi, double* delta,
                           double drop_rel) {
  const int nrb = c.nrb, ld = nrb + 1;
  const int per = 2 * nrb * ld + 6 * nrb;
  const size_t per_warp = (size_t)(per + (per & 1)) * sizeof(double);
  int wpb = (int)std::min<size_t>(8, (200 * 1024) / per_warp);
  if (wpb < 1) wpb = 1;
  const size_t smem = per_warp * wpb;
  cudaFuncSetAttribute(gram_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  gram_direct_kernel<<<(unsigned)ceil_div(2 * c.N, wpb), 32 * wpb, smem, c.stream>>>(Y, ntab, nrb, dvec, pi, delta,
                                                                                      c.N, drop_rel);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

}  // namespace fetidp
