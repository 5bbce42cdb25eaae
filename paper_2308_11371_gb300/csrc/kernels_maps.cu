// Integer-indexed maps of the FETI-DP hot path and FP64 vector kernels.
//
// * B_d^T gather and B_d scatter (Eq. 15; used in Eqs. 48-49 and Algorithm 3):
//   both are written as row-wise gathers over at most two signed terms in a
//   fixed order, so they are bit-exact and need no atomics.
// * A_p assembly / extraction of corner values (Eq. 18).
// * Deterministic FP64 reductions for the Krylov recurrences: a fixed
//   partition into kRedBlocks blocks, warp-shuffle trees, then the partials
//   summed in block order by a second kernel.
#include "common.cuh"

namespace fetidp {

namespace {

constexpr int kRedBlocks = kReductionBlocks;
constexpr int kRedThreads = 256;

// Dirichlet-preconditioner scaling D = (B B^T)^{-1} (Eq. 30: sum_s B_d B_d^T D = I_L).
// B B^T is block diagonal over the rows of one node and component.  dinfo[row] = (n << 8) | q:
// the row is chain row q of the n chain rows of its node (rows of one node and component lie d
// apart), n = 0 for a Dirichlet row (block 1).  The block is the inverse of the n x n matrix
// tridiag(-1, 2, -1), (T^{-1})_ab = (min(a, b) + 1)(n - max(a, b)) / (n + 1): 1/2 for n = 1
// (every 2D row, 3D face rows), quarters for the n = 3 rows of a 3D cell edge (exact in binary).
// The blocks for n = 1, 2, 3 as constants (each the correctly rounded quotient, as a run-time FP64
// division would give): GB300's FP64 divide is a long software sequence on its slow FP64 pipe.
__device__ __forceinline__ double tinv(int a, int b, int n) {
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  const int num = (lo + 1) * (n - hi);
  if (n == 1) return 0.5;
  if (n == 2) return num == 2 ? 2.0 / 3.0 : 1.0 / 3.0;
  if (n == 3) return 0.25 * num;
  return (double)num / (double)(n + 1);
}


// -x when neg is 1, by the sign bit alone (no FP64 instruction: GB300 runs FP64 at 1/64 of FP32)
__device__ __forceinline__ double flip_sign(double x, int neg) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)neg << 63));
}

// x_d = B_d^T lambda, or B_d^T D lambda when dinfo is given.  One thread per (cell, dual DOF):
// the (multiplier row, weight) terms of the entry -- at most two signed rows, each expanded into
// at most three rows by the D block -- are decoded once, then applied to every RHS.  Entries whose
// terms all have weight +-1 (every entry of the unscaled map) take one FP64 addition per RHS, the
// signs applied to the bits.
__global__ void gather_BT_kernel(const int* __restrict__ gath, const double* __restrict__ lam,
                                 long long lam_rs, const int* __restrict__ dinfo, int d,
                                 double* __restrict__ out, long long out_rs, int out_cs, int nd,
                                 long long ncell, int nrhs, double beta) {
  const int total = (int)(ncell * nd);               // < 2^31, checked by the host
  const bool overwrite = beta == 0.0;
  for (int cj = blockIdx.x * blockDim.x + threadIdx.x; cj < total; cj += gridDim.x * blockDim.x) {
    const int cell = cj / nd;
    const int j = cj - cell * nd;
    const int2 cc = reinterpret_cast<const int2*>(gath)[cj];
    // six term slots in registers (fixed trip counts); live / neg are bit masks over the slots
    int idx[6];
    double w[6];
    int live = 0, neg = 0;
    bool unit = true;
#pragma unroll
    for (int k = 0; k < 6; ++k) { idx[k] = 0; w[k] = 0.0; }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int code = h ? cc.y : cc.x;
      if (code == 0) continue;
      const int row = (code > 0 ? code : -code) - 1;
      const int sg = code < 0 ? 1 : 0;
      const int dc = dinfo ? dinfo[row] : 0;
      const int n = dc >> 8, q = dc & 0xff;
      if (n == 0) {
        idx[3 * h] = row;
        w[3 * h] = sg ? -1.0 : 1.0;
        live |= 1 << (3 * h);
        neg |= sg << (3 * h);
        continue;
      }
      unit = false;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (b < n) {
          const int k = 3 * h + b;
          idx[k] = row + (b - q) * d;
          const double t = tinv(q, b, n);
          w[k] = sg ? -t : t;
          live |= 1 << k;
        }
      }
    }
    for (int rhs = 0; rhs < nrhs; ++rhs) {
      const double* l = lam + rhs * lam_rs;
      double v;
      if (unit) {
        const double a = (live & 1) ? l[idx[0]] : 0.0, bv = (live & 8) ? l[idx[3]] : 0.0;
        v = flip_sign(a, neg & 1) + flip_sign(bv, (neg >> 3) & 1);
      } else {
        v = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k)
          if ((live >> k) & 1) v = fma(w[k], l[idx[k]], v);
      }
      double* o = out + rhs * out_rs + (long long)cell * out_cs + j;
      *o = overwrite ? v : v + beta * (*o);
    }
  }
}

// z = alpha B y + beta z, or alpha D B y + beta z when dinfo is given.  One thread per row: the
// (cell entry, weight) terms -- two signed copies of each of at most three chain rows -- are decoded
// once, then applied to every RHS (a signed FP64 sum for the unscaled rows, as in the gather).
__global__ void scatter_B_kernel(const int* __restrict__ scat, const double* __restrict__ yd,
                                 long long y_rs, int y_cs, int nd, const int* __restrict__ dinfo,
                                 int d, double* __restrict__ out, long long out_rs, long long L,
                                 double alpha, double beta, int nrhs) {
  const int Li = (int)L;                             // < 2^31, checked by the host
  const bool overwrite = beta == 0.0, unscaled = alpha == 1.0;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < Li; row += gridDim.x * blockDim.x) {
    const int code = dinfo ? dinfo[row] : 0;
    const int n = code >> 8, q = code & 0xff;
    long long idx[6];
    double w[6];
    int live = 0, neg = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) { idx[k] = 0; w[k] = 0.0; }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b > 0 && b >= n) break;
      const int r = n == 0 ? row : row + (b - q) * d;
      const double wr = n == 0 ? 1.0 : tinv(q, b, n);
      const int2 sc = reinterpret_cast<const int2*>(scat)[r];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = h ? sc.y : sc.x;
        if (c == 0) continue;
        const int e = (c > 0 ? c : -c) - 1;
        const int cell = e / nd;
        const int k = 2 * b + h;
        idx[k] = (long long)cell * y_cs + (e - cell * nd);
        w[k] = c > 0 ? wr : -wr;
        live |= 1 << k;
        neg |= (c < 0 ? 1 : 0) << k;
      }
    }
    for (int rhs = 0; rhs < nrhs; ++rhs) {
      const double* y = yd + rhs * y_rs;
      double v;
      if (n == 0) {   // weights +-1
        const double a = (live & 1) ? y[idx[0]] : 0.0, bv = (live & 2) ? y[idx[1]] : 0.0;
        v = flip_sign(a, neg & 1) + flip_sign(bv, (neg >> 1) & 1);
      } else {
        v = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k)
          if ((live >> k) & 1) v = fma(w[k], y[idx[k]], v);
      }
      double* o = out + rhs * out_rs + row;
      const double av = unscaled ? v : alpha * v;
      *o = overwrite ? av : av + beta * (*o);
    }
  }
}

__global__ void primal_assemble_kernel(const int* __restrict__ vert_cells, int ncorner, int d,
                                       const double* __restrict__ cp, long long c_rs, int c_cs,
                                       double* __restrict__ out, long long out_rs, int nV,
                                       double alpha, double beta, int nrhs) {
  const long long total = (long long)nV * d;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total * nrhs;
       t += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / total);
    const long long vc = t - rhs * total;
    const int v = (int)(vc / d), comp = (int)(vc - (long long)v * d);
    double s = 0.0;
    for (int q = 0; q < ncorner; ++q) {
      const int code = vert_cells[v * ncorner + q];
      if (code < 0) continue;
      const long long cell = code / ncorner;
      const int k = code - (int)cell * ncorner;
      s += cp[rhs * c_rs + cell * c_cs + k * d + comp];
    }
    double* o = out + rhs * out_rs + vc;
    *o = (beta == 0.0) ? alpha * s : alpha * s + beta * (*o);
  }
}

__global__ void primal_extract_kernel(const int* __restrict__ corner_v, int ncorner, int d,
                                      const double* __restrict__ uP, long long uP_rs,
                                      double* __restrict__ cp, long long c_rs, int c_cs,
                                      long long ncell, int nrhs) {
  const int npc = ncorner * d;
  const long long total = ncell * npc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total * nrhs;
       t += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / total);
    const long long ck = t - rhs * total;
    const long long cell = ck / npc;
    const int q = (int)(ck - cell * npc);
    const int k = q / d, comp = q - k * d;
    const int v = corner_v[cell * ncorner + k];
    cp[rhs * c_rs + cell * c_cs + q] = v >= 0 ? uP[rhs * uP_rs + (long long)v * d + comp] : 0.0;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

// partial[(rhs*nv + i)*kRedBlocks + blk] = sum over this block's fixed slice of V_i . w
__global__ void multi_dot_partial(const double* __restrict__ Vb, long long vstride, long long vrs,
                                  const double* __restrict__ w, long long wrs, long long len,
                                  int nv, double* __restrict__ partial) {
  __shared__ double sh[32];
  const int i = blockIdx.z, rhs = blockIdx.y, blk = blockIdx.x;
  const double* v = Vb + i * vstride + rhs * vrs;
  const double* x = w + rhs * wrs;
  const long long chunk = (len + kRedBlocks - 1) / kRedBlocks;
  const long long beg = blk * chunk;
  const long long end = beg + chunk < len ? beg + chunk : len;
  double s = 0.0;
  for (long long t = beg + threadIdx.x; t < end; t += blockDim.x) s += v[t] * x[t];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[((long long)rhs * nv + i) * kRedBlocks + blk] = s;
}

__global__ void reduce_partials(const double* __restrict__ partial, int count,
                                double* __restrict__ out) {
  __shared__ double sh[32];
  const int k = blockIdx.x;
  double s = 0.0;
  // fixed assignment of partials to threads, then a fixed tree
  for (int t = threadIdx.x; t < kRedBlocks; t += blockDim.x) s += partial[(long long)k * kRedBlocks + t];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[k] = s;
  (void)count;
}

// Compliance partial sums: sum over (cell, local dof) of f . u for one load case, with f the
// remaining-DOF part of the outer right-hand side and the cells' own corner loads, and u in
// natural cell order.  Fixed chunk per block, fixed tree in the block (deterministic).
__global__ void compliance_partial(const double* __restrict__ rhs, long long ntot, const double* __restrict__ fp,
                                   const double* __restrict__ u, const int* __restrict__ perm, int n, int nr,
                                   long long ncell, double* __restrict__ partial) {
  __shared__ double sh[32];
  const int rhs_i = blockIdx.y, blk = blockIdx.x;
  const long long len = ncell * n;
  const long long chunk = (len + kRedBlocks - 1) / kRedBlocks;
  const long long beg = blk * chunk;
  const long long end = beg + chunk < len ? beg + chunk : len;
  const double* fr = rhs + rhs_i * ntot;
  const double* fq = fp + rhs_i * ncell * (n - nr);
  const double* uc = u + rhs_i * len;
  double acc = 0.0;
  for (long long t = beg + threadIdx.x; t < end; t += blockDim.x) {
    const long long s = t / n;
    const int li = (int)(t - s * n);
    const double f = li < nr ? fr[s * nr + li] : fq[s * (n - nr) + (li - nr)];
    acc += f * uc[s * n + perm[li]];
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[(long long)rhs_i * kRedBlocks + blk] = acc;
}

__global__ void multi_axpy_kernel(const double* __restrict__ Vb, long long vstride, long long vrs,
                                  int nv, const double* __restrict__ coef, double* __restrict__ w,
                                  long long wrs, long long len, int nrhs, double sign) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len * nrhs;
       t += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / len);
    const long long q = t - rhs * len;
    double s = 0.0;
    for (int i = 0; i < nv; ++i) s += coef[rhs * nv + i] * Vb[i * vstride + rhs * vrs + q];
    w[rhs * wrs + q] += sign * s;
  }
}

__global__ void copy_scale_kernel(const double* __restrict__ x, double* __restrict__ y,
                                  long long len, int nrhs, long long xs, long long ys,
                                  const double* __restrict__ s_dev, double s_host) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len * nrhs;
       t += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / len);
    const long long q = t - rhs * len;
    const double s = s_dev ? s_dev[rhs] : s_host;
    y[rhs * ys + q] = s * x[rhs * xs + q];
  }
}

// flag |= 1 if any x[i] is NaN or +-Inf (input validation of the C entry points)
__global__ void nonfinite_kernel(const double* __restrict__ x, long long n, int* __restrict__ flag) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) {
      atomicOr(flag, 1);
      return;
    }
}

inline int grid_for(long long work, int threads = 256) {
  long long g = (work + threads - 1) / threads;
  if (g > 152LL * 16) g = 152LL * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

fetidp_status k_gather_BT(Ctx& c, const double* lam, long long lam_rs, const int* dinfo,
                          CellVec out, int nrhs, double beta) {
  const long long work = c.N * c.nd;
  if (work >= (1LL << 31) || c.L >= (1LL << 31)) { set_error("lattice too large for 32-bit map indices"); return FETIDP_EINVAL; }
  ProfScope ps(c, FETIDP_K_MAPS, 0.0, (double)nrhs * (c.L * 8.0 + c.N * c.nd * 8.0) + c.N * c.nd * 8.0);
  gather_BT_kernel<<<grid_for(work), 256, 0, c.stream>>>(c.gath, lam, lam_rs, dinfo, c.d, out.p, out.rs,
                                                          out.cs, c.nd, c.N, nrhs, beta);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_scatter_B(Ctx& c, CCellVec yd, double* out, long long out_rs, const int* dinfo,
                          double alpha, double beta, int nrhs) {
  if (c.L >= (1LL << 31) || c.N * c.nd >= (1LL << 31)) { set_error("lattice too large for 32-bit map indices"); return FETIDP_EINVAL; }
  ProfScope ps(c, FETIDP_K_MAPS, 0.0, (double)nrhs * (c.L * 8.0 + c.N * c.nd * 8.0) + c.L * 8.0);
  scatter_B_kernel<<<grid_for(c.L), 256, 0, c.stream>>>(
      c.scat, yd.p, yd.rs, yd.cs, c.nd, dinfo, c.d, out, out_rs, c.L, alpha, beta, nrhs);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_primal_assemble(Ctx& c, CCellVec cp, double* out, long long out_rs, double alpha,
                                double beta, int nrhs) {
  ProfScope ps(c, FETIDP_K_MAPS, 0.0, (double)nrhs * (c.N * c.np * 8.0 + c.nP * 8.0));
  primal_assemble_kernel<<<grid_for((long long)c.nV * c.d * nrhs), 256, 0, c.stream>>>(
      c.vert_cells, c.ncorner, c.d, cp.p, cp.rs, cp.cs, out, out_rs, c.nV, alpha, beta, nrhs);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_primal_extract(Ctx& c, const double* uP, long long uP_rs, CellVec cp, int nrhs) {
  ProfScope ps(c, FETIDP_K_MAPS, 0.0, (double)nrhs * (c.N * c.np * 8.0 + c.nP * 8.0));
  primal_extract_kernel<<<grid_for(c.N * c.np * nrhs), 256, 0, c.stream>>>(
      c.corner_v, c.ncorner, c.d, uP, uP_rs, cp.p, cp.rs, cp.cs, c.N, nrhs);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

// out[rhs*nv + i] = V_i[rhs] . w[rhs]; V_i at Vb + i*vstride + rhs*len_rs.
static fetidp_status multi_dot_impl(Ctx& c, const double* Vb, long long vstride, long long vrs,
                                    int nv, const double* w, long long wrs, long long len,
                                    int nrhs, double* out) {
  ProfScope ps(c, FETIDP_K_VECTOR, 2.0 * nv * len * nrhs, 8.0 * (nv + 1) * len * nrhs);
  dim3 grid(kRedBlocks, nrhs, nv);
  multi_dot_partial<<<grid, kRedThreads, 0, c.stream>>>(Vb, vstride, vrs, w, wrs, len, nv, c.red);
  FD_CHECK_LAUNCH();
  reduce_partials<<<nrhs * nv, kRedThreads, 0, c.stream>>>(c.red, nrhs * nv, out);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_dot(Ctx& c, const double* x, long long xs, const double* y, long long ys,
                    long long len, int nrhs, double* out) {
  return multi_dot_impl(c, x, 0, xs, 1, y, ys, len, nrhs, out);
}

fetidp_status k_multi_dot(Ctx& c, const double* Vb, long long vstride, int nv, const double* w,
                          long long len, int nrhs, double* out) {
  // Krylov vectors: V_i[rhs] at Vb + i*vstride + rhs*len; w[rhs] at w + rhs*len
  return multi_dot_impl(c, Vb, vstride, len, nv, w, len, len, nrhs, out);
}

fetidp_status k_multi_axpy(Ctx& c, const double* Vb, long long vstride, int nv, const double* coef,
                           double* w, long long len, int nrhs, double sign) {
  ProfScope ps(c, FETIDP_K_VECTOR, 2.0 * nv * len * nrhs, 8.0 * (nv + 2) * len * nrhs);
  multi_axpy_kernel<<<grid_for(len * nrhs), 256, 0, c.stream>>>(Vb, vstride, len, nv, coef, w, len,
                                                                 len, nrhs, sign);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_compliance(Ctx& c, const double* u, double* out, double* partial) {
  compliance_partial<<<dim3(kRedBlocks, c.m), 256, 0, c.stream>>>(c.rhs, c.ntot, c.rhs_p_cells, u, c.perm, c.n, c.nr,
                                                                 c.N, partial);
  FD_CHECK_LAUNCH();
  reduce_partials<<<c.m, 256, 0, c.stream>>>(partial, kRedBlocks, out);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_copy_scale(Ctx& c, const double* x, double* y, long long len, int nrhs,
                           long long xs, long long ys, const double* s_dev, double s_host) {
  ProfScope ps(c, FETIDP_K_VECTOR, (double)len * nrhs, 16.0 * len * nrhs);
  copy_scale_kernel<<<grid_for(len * nrhs), 256, 0, c.stream>>>(x, y, len, nrhs, xs, ys, s_dev,
                                                                 s_host);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

}  // namespace fetidp

namespace fetidp {

fetidp_status k_nonfinite(Ctx& c, const double* x, long long n, int* flag) {
  if (n <= 0) return FETIDP_OK;
  nonfinite_kernel<<<grid_for(n), 256, 0, c.stream>>>(x, n, flag);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

}  // namespace fetidp
