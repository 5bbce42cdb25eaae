// Setup kernels: greedy selection (Algorithm 4), trace tables for the
// projections of Eq. 42, and assembly of the ROM local operators (Eq. 43).
//
// The projections use that K^(s) is linear in C_hat (Eq. 52): every trace
// tr(U_i^T K^(s) U_j) equals sum over Gauss points and tensor entries of
// C_hat^(s) times a cell-independent table built from the gradients of the
// principal columns, so all cells' Gram matrices come out of one GEMM
// against the snapshot matrix.
#include "common.cuh"

namespace fetidp {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double bsum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double bmax(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r = fmax(r, sh[k]);
  __syncthreads();
  return r;
}

// out[row] = ||X[row]||_2 (mode 0), ||X[row]||_inf (mode 1), X[row] . z (mode 2), ||X[row]||_2^2 (mode 3)
__global__ void row_reduce_kernel(const double* __restrict__ X, long long len,
                                  const double* __restrict__ z, int mode, double* __restrict__ out) {
  __shared__ double sh[32];
  const double* x = X + blockIdx.x * len;
  double acc = 0.0;
  for (long long t = threadIdx.x; t < len; t += blockDim.x) {
    const double v = x[t];
    if (mode == 0 || mode == 3) acc += v * v;
    else if (mode == 1) acc = fmax(acc, fabs(v));
    else acc += v * z[t];
  }
  const double r = (mode == 1) ? bmax(acc, sh) : bsum(acc, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = (mode == 0) ? sqrt(r) : r;
}

// Delta = A / norm (rows)
__global__ void row_normalise_kernel(const double* __restrict__ A, const double* __restrict__ nrm,
                                     double* __restrict__ D, long long len, long long rows) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < rows * len;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / len;
    D[t] = A[t] / nrm[r];
  }
}

// Delta[row] -= beta[row] * zeta
__global__ void row_update_kernel(double* __restrict__ D, const double* __restrict__ beta,
                                  const double* __restrict__ zeta, long long len, long long rows) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < rows * len;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / len;
    D[t] -= beta[r] * zeta[t - r * len];
  }
}

// Selection of step i of Algorithm 4 (one block): the largest infinity norm of the current
// residual snapshots; the selected cell is the lowest index within relative `tie` of it, and the
// 2-norm of its residual row is kept for the normalisation.  Stops (and every later kernel of the
// loop returns at once) when the maximum is not above tol_rb (from the second step on) or is zero.
__global__ void greedy_select_kernel(const double* __restrict__ inf, long long n, const double* __restrict__ D,
                                     long long len, int i, double tol_rb, double tie, GreedyState* __restrict__ st) {
  __shared__ double sh[32];
  __shared__ double smx;
  __shared__ long long sidx[32];
  __shared__ long long sbest;
  if (st->stop) return;                             // uniform across the block
  double mx = 0.0;
  for (long long t = threadIdx.x; t < n; t += blockDim.x) mx = fmax(mx, inf[t]);
  const double m = bmax(mx, sh);
  if (threadIdx.x == 0) smx = m;
  __syncthreads();
  const double M = smx;
  if ((i > 0 && M <= tol_rb) || M == 0.0) {
    if (threadIdx.x == 0) st->stop = 1;
    return;
  }
  long long best = n;
  for (long long t = threadIdx.x; t < n; t += blockDim.x)
    if (inf[t] >= M * (1.0 - tie)) { best = t; break; }
  for (int o = 16; o > 0; o >>= 1) {
    const long long ob = __shfl_down_sync(0xffffffffu, best, o);
    best = ob < best ? ob : best;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sidx[w] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) best = sidx[k] < best ? sidx[k] : best;
    sbest = best;
    st->sigma[i] = (int)best;
    st->count = i + 1;
  }
  __syncthreads();
  const double* x = D + sbest * len;
  double acc = 0.0;
  for (long long t = threadIdx.x; t < len; t += blockDim.x) acc = fma(x[t], x[t], acc);
  const double q = bsum(acc, sh);
  if (threadIdx.x == 0) st->znrm = sqrt(q);
}

// zeta_i = Delta[sigma_i] / ||Delta[sigma_i]||_2 (grid-stride over the row).
__global__ void greedy_zeta_kernel(const double* __restrict__ D, long long len, int i,
                                   const GreedyState* __restrict__ st, double* __restrict__ zeta) {
  if (st->count <= i) return;
  const int sig = st->sigma[i];
  const double* x = D + (long long)sig * len;
  const double nrm = st->znrm;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len; t += (long long)gridDim.x * blockDim.x)
    zeta[t] = x[t] / nrm;
}

// T[i][j] = zeta_i . A^(sigma_j) (the change of basis of Eq. 56), one block per (i, j).
__global__ void greedy_T_kernel(const double* __restrict__ Z, const double* __restrict__ snap, long long len, int nrb,
                                const GreedyState* __restrict__ st, double* __restrict__ T) {
  __shared__ double sh[32];
  const int i = blockIdx.x / nrb, j = blockIdx.x - (blockIdx.x / nrb) * nrb;
  const double* z = Z + (long long)i * len;
  const double* a = snap + (long long)st->sigma[j] * len;
  double acc = 0.0;
  for (long long t = threadIdx.x; t < len; t += blockDim.x) acc += z[t] * a[t];
  const double r = bsum(acc, sh);
  if (threadIdx.x == 0) T[i * nrb + j] = r;
}

// alpha^(s) from T alpha = ||A^(s)|| beta^(s), T upper triangular (Eq. 56); one thread per cell.
__global__ void greedy_alpha_kernel(const double* __restrict__ T, const double* __restrict__ nrm,
                                    const double* __restrict__ beta, long long ncell, int nrb,
                                    double* __restrict__ alpha) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < ncell;
       s += (long long)gridDim.x * blockDim.x) {
    double* a = alpha + s * nrb;
    for (int i = nrb - 1; i >= 0; --i) {
      double v = nrm[s] * beta[(long long)i * ncell + s];
      for (int j = i + 1; j < nrb; ++j) v -= T[i * nrb + j] * a[j];
      a[i] = v / T[i * nrb + i];
    }
  }
}

// One greedy step of Algorithm 4 for every row, fused: beta = Delta[row] . zeta,
// Delta[row] -= beta zeta, and the infinity norm of the updated row (the next step's
// selection).  Two FP64 FMAs per entry: at GB300's FP64 rate (2 FMA/clk/SM) they, not the
// 16 B of HBM traffic, bound the kernel, so the maximum of |v| runs on the integer pipe (the bit
// patterns of non-negative doubles order like the values).  One block per row; the second pass
// re-reads the row from L2.
__device__ __forceinline__ unsigned long long bmax_u64(unsigned long long v, unsigned long long* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_down_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  unsigned long long r = 0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r = sh[k] > r ? sh[k] : r;
  __syncthreads();
  return r;
}

__global__ void greedy_step_kernel(double* __restrict__ D, const double* __restrict__ zeta, long long len,
                                   double* __restrict__ beta_out, double* __restrict__ inf_out,
                                   const GreedyState* __restrict__ st, int i) {
  __shared__ double sh[32];
  __shared__ unsigned long long shu[32];
  __shared__ double sbeta;
  if (st->count <= i) return;                       // the greedy stopped before step i
  double* x = D + blockIdx.x * len;
  const long long stride = blockDim.x;
  double a0 = 0.0, a1 = 0.0;
  long long t = threadIdx.x;
  for (; t + stride < len; t += 2 * stride) {
    a0 = fma(x[t], zeta[t], a0);
    a1 = fma(x[t + stride], zeta[t + stride], a1);
  }
  if (t < len) a0 = fma(x[t], zeta[t], a0);
  const double beta = bsum(a0 + a1, sh);
  if (threadIdx.x == 0) sbeta = beta;
  __syncthreads();
  const double bt = sbeta;
  unsigned long long mx = 0;
  for (t = threadIdx.x; t < len; t += stride) {
    const double v = fma(-bt, zeta[t], x[t]);
    x[t] = v;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
    mx = b > mx ? b : mx;
  }
  const unsigned long long m = bmax_u64(mx, shu);
  if (threadIdx.x == 0) {
    beta_out[blockIdx.x] = bt;
    inf_out[blockIdx.x] = __longlong_as_double((long long)m);
  }
}

// ---------------------------------------------------------------- double-float greedy (mixed path)
// The residual snapshots Delta are kept as float planes (hi, lo) with |lo| <= ulp(hi) / 2, so a
// greedy step runs on the FP32 pipe (dot product and update in double-float, ~2^-46 relative)
// and is bound by its 16 B per entry of HBM traffic instead of GB300's FP64 rate.  |hi + lo|
// orders like the 64-bit key (bits of |hi|, order-preserving bits of sign(hi) lo), so the
// infinity norm is an integer maximum.
__device__ __forceinline__ unsigned long long df_abs_key(float h, float l) {
  const unsigned hb = __float_as_uint(h);
  const float ls = (hb >> 31) ? -l : l;                   // lo in the direction of |hi|
  const unsigned lb = __float_as_uint(ls);
  const unsigned lkey = (lb >> 31) ? ~lb : (lb | 0x80000000u);
  return ((unsigned long long)(hb & 0x7fffffffu) << 32) | lkey;
}
__device__ __forceinline__ double df_key_value(unsigned long long key) {
  const float ah = __uint_as_float((unsigned)(key >> 32));
  const unsigned lkey = (unsigned)key;
  const unsigned lb = (lkey >> 31) ? (lkey & 0x7fffffffu) : ~lkey;
  return (double)ah + (double)__uint_as_float(lb);
}
__device__ __forceinline__ void df_fma_acc(float ah, float al, float bh, float bl, float& s, float& c) {
  const float p = ah * bh;
  const float e = fmaf(ah, bh, -p);
  c = fmaf(ah, bl, c);
  c = fmaf(al, bh, c);
  const float t = s + p;
  const float bv = t - s;
  const float err = (s - (t - bv)) + (p - bv);
  s = t;
  c = c + (err + e);
}

// Delta[row] = A[row] / ||A[row]|| as planes, and its infinity norm; one block per row.
__global__ void greedy_init_df_kernel(const double* __restrict__ A, const double* __restrict__ nrm, long long len,
                                      float* __restrict__ Dh, float* __restrict__ Dl, double* __restrict__ inf_out) {
  __shared__ double sinv;
  __shared__ unsigned long long shu[32];
  if (threadIdx.x == 0) sinv = 1.0 / nrm[blockIdx.x];
  __syncthreads();
  const double inv = sinv;
  const long long o = (long long)blockIdx.x * len;
  unsigned long long mx = 0;
  for (long long t = threadIdx.x; t < len; t += blockDim.x) {
    const double v = A[o + t] * inv;
    const float h = (float)v, l = (float)(v - (double)h);
    Dh[o + t] = h;
    Dl[o + t] = l;
    const unsigned long long k = df_abs_key(h, l);
    mx = k > mx ? k : mx;
  }
  const unsigned long long m = bmax_u64(mx, shu);
  if (threadIdx.x == 0) inf_out[blockIdx.x] = df_key_value(m);
}

// Selection (as greedy_select_kernel) with the selected row's 2-norm from the planes.
__global__ void greedy_select_df_kernel(const double* __restrict__ inf, long long n, const float* __restrict__ Dh,
                                        const float* __restrict__ Dl, long long len, int i, double tol_rb,
                                        double tie, GreedyState* __restrict__ st) {
  __shared__ double sh[32];
  __shared__ double smx;
  __shared__ long long sidx[32];
  __shared__ long long sbest;
  if (st->stop) return;
  double mx = 0.0;
  for (long long t = threadIdx.x; t < n; t += blockDim.x) mx = fmax(mx, inf[t]);
  const double m = bmax(mx, sh);
  if (threadIdx.x == 0) smx = m;
  __syncthreads();
  const double M = smx;
  if ((i > 0 && M <= tol_rb) || M == 0.0) {
    if (threadIdx.x == 0) st->stop = 1;
    return;
  }
  long long best = n;
  for (long long t = threadIdx.x; t < n; t += blockDim.x)
    if (inf[t] >= M * (1.0 - tie)) { best = t; break; }
  for (int o = 16; o > 0; o >>= 1) {
    const long long ob = __shfl_down_sync(0xffffffffu, best, o);
    best = ob < best ? ob : best;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sidx[w] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) best = sidx[k] < best ? sidx[k] : best;
    sbest = best;
    st->sigma[i] = (int)best;
    st->count = i + 1;
  }
  __syncthreads();
  const long long o = sbest * len;
  float s = 0.f, c = 0.f;
  for (long long t = threadIdx.x; t < len; t += blockDim.x) df_fma_acc(Dh[o + t], Dl[o + t], Dh[o + t], Dl[o + t], s, c);
  const double q = bsum((double)s + (double)c, sh);
  if (threadIdx.x == 0) st->znrm = sqrt(q);
}

// zeta_i = Delta[sigma_i] / ||Delta[sigma_i]||_2 as planes and in FP64 (for Eq. 56).
__global__ void greedy_zeta_df_kernel(const float* __restrict__ Dh, const float* __restrict__ Dl, long long len, int i,
                                      const GreedyState* __restrict__ st, float* __restrict__ zh,
                                      float* __restrict__ zl, double* __restrict__ zeta) {
  if (st->count <= i) return;
  const long long o = (long long)st->sigma[i] * len;
  const double nrm = st->znrm;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len; t += (long long)gridDim.x * blockDim.x) {
    const double v = ((double)Dh[o + t] + (double)Dl[o + t]) / nrm;
    const float h = (float)v;
    zh[t] = h;
    zl[t] = (float)(v - (double)h);
    zeta[t] = v;
  }
}

// One greedy step in double-float: beta = Delta[row] . zeta (per-thread pairs summed in FP64),
// Delta[row] -= beta zeta (TwoSum on the leading parts, renormalised), next infinity norm.
// 16-byte loads and stores (4 entries per thread and pass; len is a multiple of 4: 2^d Gauss
// points per element), so enough bytes are in flight to approach the HBM rate.
__device__ __forceinline__ void df_axpy_entry(float bh, float bl, float qh, float ql, float& xh, float& xl,
                                              unsigned long long& mx) {
  const float p = bh * qh;
  const float e = fmaf(bh, qh, -p);
  const float cr = fmaf(bh, ql, bl * qh);
  const float t1 = xh - p;                             // TwoSum(xh, -p)
  const float bv = t1 - xh;
  const float err = (xh - (t1 - bv)) + (-p - bv);
  const float low = (xl - (e + cr)) + err;
  const float vh = t1 + low;                           // renormalise
  const float vl = low - (vh - t1);
  xh = vh;
  xl = vl;
  const unsigned long long k = df_abs_key(vh, vl);
  mx = k > mx ? k : mx;
}

__global__ void greedy_step_df_kernel(float* __restrict__ Dh, float* __restrict__ Dl, const float* __restrict__ zh,
                                      const float* __restrict__ zl, long long len, double* __restrict__ beta_out,
                                      double* __restrict__ inf_out, const GreedyState* __restrict__ st, int i) {
  __shared__ double sh[32];
  __shared__ unsigned long long shu[32];
  __shared__ double sbeta;
  if (st->count <= i) return;
  const long long o = (long long)blockIdx.x * len;
  const long long n4 = len / 4;
  const float4* xh4 = reinterpret_cast<const float4*>(Dh + o);
  const float4* xl4 = reinterpret_cast<const float4*>(Dl + o);
  const float4* zh4 = reinterpret_cast<const float4*>(zh);
  const float4* zl4 = reinterpret_cast<const float4*>(zl);
  float s = 0.f, c = 0.f;
  for (long long q = threadIdx.x; q < n4; q += blockDim.x) {
    const float4 a = xh4[q], b = xl4[q], u = zh4[q], w = zl4[q];
    df_fma_acc(a.x, b.x, u.x, w.x, s, c);
    df_fma_acc(a.y, b.y, u.y, w.y, s, c);
    df_fma_acc(a.z, b.z, u.z, w.z, s, c);
    df_fma_acc(a.w, b.w, u.w, w.w, s, c);
  }
  const double beta = bsum((double)s + (double)c, sh);
  if (threadIdx.x == 0) sbeta = beta;
  __syncthreads();
  const double bt = sbeta;
  const float bh = (float)bt, bl = (float)(bt - (double)bh);
  unsigned long long mx = 0;
  float4* wh4 = reinterpret_cast<float4*>(Dh + o);
  float4* wl4 = reinterpret_cast<float4*>(Dl + o);
  for (long long q = threadIdx.x; q < n4; q += blockDim.x) {
    float4 a = wh4[q], b = wl4[q];
    const float4 u = zh4[q], w = zl4[q];
    df_axpy_entry(bh, bl, u.x, w.x, a.x, b.x, mx);
    df_axpy_entry(bh, bl, u.y, w.y, a.y, b.y, mx);
    df_axpy_entry(bh, bl, u.z, w.z, a.z, b.z, mx);
    df_axpy_entry(bh, bl, u.w, w.w, a.w, b.w, mx);
    wh4[q] = a;
    wl4[q] = b;
  }
  const unsigned long long m = bmax_u64(mx, shu);
  if (threadIdx.x == 0) {
    beta_out[blockIdx.x] = bt;
    inf_out[blockIdx.x] = df_key_value(m);
  }
}

__global__ void scale_copy_kernel(const double* __restrict__ x, const double* __restrict__ s,
                                  double* __restrict__ y, long long len) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = x[t] / s[0];
}

// Reference gradients G_ia (xi-derivatives) of column vectors at every Gauss point.
// Column (k, l): values at local (i,d,p) index li taken from
//   mode 0: src[k*kstride + l*lstride + li] for li < len_in, 0 otherwise
//   mode 1: unit vector at local index unit_base + l
// out[((k*ncol + l)*nelem + el)*ngp + gp][d*d]
template <int D>
__global__ void column_gradients_kernel(int e, int n, const int* __restrict__ iperm,
                                        const double* __restrict__ src, long long kstride,
                                        long long lstride, int len_in, int mode, int unit_base,
                                        int nk, int ncol, double inv_h, double* __restrict__ out) {
  constexpr int NA = 1 << D;
  const int nelem = e * e * (D == 3 ? e : 1);
  const long long total = (long long)nk * ncol * nelem * NA;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int gp = (int)(t % NA);
    long long r = t / NA;
    const int el = (int)(r % nelem);
    r /= nelem;
    const int l = (int)(r % ncol);
    const int k = (int)(r / ncol);
    const int ex = el % e, ey = (el / e) % e, ez = el / (e * e);
    double tq[D];
    for (int q = 0; q < D; ++q) tq[q] = gauss_t((gp >> q) & 1);
    double G[D * D];
    for (int q = 0; q < D * D; ++q) G[q] = 0.0;
    for (int A = 0; A < NA; ++A) {
      const int ax = A & 1, ay = (A >> 1) & 1, az = (A >> 2) & 1;
      const int node = (ex + ax) + (e + 1) * ((ey + ay) + (e + 1) * (D == 3 ? (ez + az) : 0));
      double dn[D];
      for (int a = 0; a < D; ++a) {
        double v = inv_h;
        for (int q = 0; q < D; ++q) {
          const int off = (A >> q) & 1;
          if (q == a) v *= off ? 1.0 : -1.0;
          else v *= off ? tq[q] : 1.0 - tq[q];
        }
        dn[a] = v;
      }
      for (int i = 0; i < D; ++i) {
        const int li = iperm[node * D + i];
        double uv;
        if (mode == 0) uv = li < len_in ? src[k * kstride + l * lstride + li] : 0.0;
        else uv = (li == unit_base + l) ? 1.0 : 0.0;
        for (int a = 0; a < D; ++a) G[i * D + a] += uv * dn[a];
      }
    }
    (void)n;
    double* o = out + t * (D * D);
    for (int q = 0; q < D * D; ++q) o[q] = G[q];
  }
}

// Table row t = (i, j): T[t][(el*ngp + gp)*nc + c] = wq sum_l [Gi_I Gj_J + (I != J) Gi_J Gj_I]
// for every table in one launch (grid.y = table).
__global__ void trace_tables_kernel(const TraceTableSpec* __restrict__ specs, int nqp, int d,
                                    double wq, double* __restrict__ T, long long tstride) {
  const TraceTableSpec sp = specs[blockIdx.y];
  const int dd = d * d;
  const int nc = dd * (dd + 1) / 2;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nqp; t += gridDim.x * blockDim.x) {
    double acc[45];
    for (int c = 0; c < nc; ++c) acc[c] = 0.0;
    for (int l = 0; l < sp.ncol; ++l) {
      const double* gi = sp.Gi + ((long long)l * nqp + t) * dd;
      const double* gj = sp.Gj + ((long long)l * nqp + t) * dd;
      double a[9], b[9];
      for (int I = 0; I < dd; ++I) { a[I] = gi[I]; b[I] = gj[I]; }
      int c = 0;
      for (int I = 0; I < dd; ++I)
        for (int J = I; J < dd; ++J) {
          double v = a[I] * b[J];
          if (J != I) v += a[J] * b[I];
          acc[c++] += v;
        }
    }
    double* o = T + blockIdx.y * tstride + (long long)t * nc;
    for (int c = 0; c < nc; ++c) o[c] = wq * acc[c];
  }
}

// Double-float variant for the mixed path: the same table rows from gradients kept as float
// planes (hi = fl(g), lo = fl(g - hi)), every product made exact by an FMA residual plus the two
// cross products, sums kept as (s, c) pairs with TwoSum (~2^-46 relative per term, all on the
// FP32 pipe).  Rows are written scaled by wq and split into the padded float planes that the
// double-float trace GEMM reads: Th/Tl[row * ldt + gp * nc + comp].
__device__ __forceinline__ void df_acc_prod(float ah, float al, float bh, float bl, float& s, float& c) {
  const float p = ah * bh;
  const float e = fmaf(ah, bh, -p);
  c = fmaf(ah, bl, c);
  c = fmaf(al, bh, c);
  const float t = s + p;
  const float bv = t - s;
  const float err = (s - (t - bv)) + (p - bv);
  s = t;
  c = c + (err + e);
}

template <int D>
__global__ void trace_tables_df_kernel(const TraceTableSpecDF* __restrict__ specs, int nqp, double wq,
                                       float* __restrict__ Th, float* __restrict__ Tl, long long ldt) {
  constexpr int DD = D * D;
  constexpr int NC = DD * (DD + 1) / 2;
  const TraceTableSpecDF sp = specs[blockIdx.y];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nqp; t += gridDim.x * blockDim.x) {
    float s[NC], cc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) { s[k] = 0.f; cc[k] = 0.f; }
    for (int l = 0; l < sp.ncol; ++l) {
      const long long o = ((long long)l * nqp + t) * DD;
      float ah[DD], al[DD], bh[DD], bl[DD];
#pragma unroll
      for (int I = 0; I < DD; ++I) { ah[I] = sp.Gih[o + I]; al[I] = sp.Gil[o + I]; bh[I] = sp.Gjh[o + I]; bl[I] = sp.Gjl[o + I]; }
      int k = 0;
#pragma unroll
      for (int I = 0; I < DD; ++I)
#pragma unroll
        for (int J = I; J < DD; ++J, ++k) {
          df_acc_prod(ah[I], al[I], bh[J], bl[J], s[k], cc[k]);
          if (J != I) df_acc_prod(ah[J], al[J], bh[I], bl[I], s[k], cc[k]);
        }
    }
    const long long row = (long long)blockIdx.y * ldt + (long long)t * NC;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const double v = ((double)s[k] + (double)cc[k]) * wq;
      const float h = (float)v;
      Th[row + k] = h;
      Tl[row + k] = (float)(v - (double)h);
    }
  }
}

// hi / lo float planes of n doubles
__global__ void split_planes_kernel(const double* __restrict__ x, long long n, float* __restrict__ hi,
                                    float* __restrict__ lo) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double v = x[t];
    const float h = (float)v;
    hi[t] = h;
    lo[t] = (float)(v - (double)h);
  }
}

// out[cell][r][c] = sum_k coef[cell][k] src[k*kstride + (r0 + r)*ld + c0 + c]
__global__ void rom_combine_kernel(const double* __restrict__ src, long long kstride, int ld,
                                   int r0, int c0, int rows, int cols,
                                   const double* __restrict__ coef, int nrb, long long ncell,
                                   double* __restrict__ out, bool transpose) {
  const long long per = (long long)rows * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncell * per;
       t += (long long)gridDim.x * blockDim.x) {
    const long long cell = t / per;
    const long long q = t - cell * per;
    const int r = (int)(q / cols), cc = (int)(q - (long long)r * cols);
    double s = 0.0;
    for (int k = 0; k < nrb; ++k)
      s += coef[cell * nrb + k] * src[k * kstride + (long long)(r0 + r) * ld + c0 + cc];
    if (transpose) out[cell * per + (long long)cc * rows + r] = s;
    else out[t] = s;
  }
}

inline int gridn(long long work) {
  long long g = (work + kThreads - 1) / kThreads;
  if (g > 152LL * 32) g = 152LL * 32;
  return (int)(g < 1 ? 1 : g);
}


// Body-force loads (Eq. 5b) of every cell for the body-force load cases: f_a = sum over the elements
// and Gauss points of w detJ N_a(gp) times the load's direction.  One CTA per cell: the w detJ of
// every (element, Gauss point) in shared memory, then each node's sum of w detJ N_a over its
// elements, then every local DOF (natural index perm[li]) of every body load written into the
// remaining-DOF right-hand side (li < nr) or the cell's corner loads (li >= nr).
__global__ void body_loads_kernel(Geo g, int nelem, const int* __restrict__ perm, int n, int nr, int np,
                                  const double* __restrict__ dirs, const int* __restrict__ body, int m,
                                  double* __restrict__ rhs, long long rhs_rs, double* __restrict__ fpc,
                                  long long ncell) {
  extern __shared__ double blsm[];
  const int d = g.dim, e = g.e, NA = 1 << d, nn1 = e + 1;
  double* wq = blsm;                                  // [nelem][NA]
  double* mn = blsm + (size_t)nelem * NA;             // [(e+1)^d]
  const long long s = blockIdx.x;
  const int nx = g.nc[0], ny = g.nc[1];
  const int cx = (int)(s % nx), cy = (int)((s / nx) % ny), cz = (int)(s / ((long long)nx * ny));
  const double h = 1.0 / e;
  double hw = 1.0;
  for (int k = 0; k < d; ++k) hw *= 0.5 * h;
  for (int t = threadIdx.x; t < nelem * NA; t += blockDim.x) {
    const int el = t / NA, gp = t - el * NA;
    const int ex = el % e, ey = (el / e) % e, ez = el / (e * e);
    double eta[3], xi[3], J[3][3];
    gauss_point(g, cx, cy, cz, ex, ey, ez, gp, eta, xi);
    macro_jacobian(g, xi, J);
    const double det = d == 2 ? J[0][0] * J[1][1] - J[0][1] * J[1][0]
                              : J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                                    J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                                    J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    wq[t] = hw * det;
  }
  __syncthreads();
  const int nnode = d == 2 ? nn1 * nn1 : nn1 * nn1 * nn1;
  for (int node = threadIdx.x; node < nnode; node += blockDim.x) {
    const int ix = node % nn1, iy = (node / nn1) % nn1, iz = d == 3 ? node / (nn1 * nn1) : 0;
    double acc = 0.0;
    for (int A = 0; A < NA; ++A) {                    // the element in which this node is local node A
      const int ex = ix - (A & 1), ey = iy - ((A >> 1) & 1), ez = d == 3 ? iz - ((A >> 2) & 1) : 0;
      if (ex < 0 || ex >= e || ey < 0 || ey >= e || ez < 0 || (d == 3 && ez >= e)) continue;
      const int el = ex + e * (ey + e * ez);
      for (int gp = 0; gp < NA; ++gp) {
        double Nv = 1.0;
        for (int k = 0; k < d; ++k) {
          const double tk = gauss_t((gp >> k) & 1);
          Nv *= ((A >> k) & 1) ? tk : 1.0 - tk;
        }
        acc += wq[el * NA + gp] * Nv;
      }
    }
    mn[node] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < m * n; t += blockDim.x) {
    const int l = t / n, li = t - l * n;
    if (!body[l]) continue;
    const int nat = perm[li];
    const double v = mn[nat / d] * dirs[l * d + nat % d];
    if (li < nr) rhs[l * rhs_rs + s * nr + li] += v;
    else fpc[((long long)l * ncell + s) * np + (li - nr)] += v;
  }
}

}  // namespace

fetidp_status k_row_reduce(Ctx& c, const double* X, long long rows, long long len, const double* z,
                           int mode, double* out) {
  row_reduce_kernel<<<(unsigned)rows, kThreads, 0, c.stream>>>(X, len, z, mode, out);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_row_normalise(Ctx& c, const double* A, const double* nrm, double* D, long long rows,
                              long long len) {
  row_normalise_kernel<<<gridn(rows * len), kThreads, 0, c.stream>>>(A, nrm, D, len, rows);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_row_update(Ctx& c, double* D, const double* beta, const double* zeta,
                           long long rows, long long len) {
  row_update_kernel<<<gridn(rows * len), kThreads, 0, c.stream>>>(D, beta, zeta, len, rows);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_greedy_step(Ctx& c, double* D, const double* zeta, long long rows, long long len, double* beta,
                            double* inf, const GreedyState* st, int i) {
  ProfScope ps(c, FETIDP_K_GREEDY, 4.0 * rows * (double)len, 16.0 * rows * (double)len);
  greedy_step_kernel<<<(unsigned)rows, kThreads, 0, c.stream>>>(D, zeta, len, beta, inf, st, i);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_greedy_init_df(Ctx& c, const double* A, const double* nrm, long long rows, long long len, float* Dh,
                               float* Dl, double* inf) {
  ProfScope ps(c, FETIDP_K_GREEDY, 0.0, 16.0 * rows * (double)len);
  greedy_init_df_kernel<<<(unsigned)rows, kThreads, 0, c.stream>>>(A, nrm, len, Dh, Dl, inf);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_greedy_select_df(Ctx& c, const double* inf, long long n, const float* Dh, const float* Dl,
                                 long long len, int i, double tol_rb, double tie, GreedyState* st) {
  ProfScope ps(c, FETIDP_K_GREEDY, 0.0, 8.0 * (double)(n + len));
  greedy_select_df_kernel<<<1, 1024, 0, c.stream>>>(inf, n, Dh, Dl, len, i, tol_rb, tie, st);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_greedy_zeta_df(Ctx& c, const float* Dh, const float* Dl, long long len, int i, const GreedyState* st,
                               float* zh, float* zl, double* zeta) {
  ProfScope ps(c, FETIDP_K_GREEDY, 0.0, 24.0 * (double)len);
  greedy_zeta_df_kernel<<<gridn(len), kThreads, 0, c.stream>>>(Dh, Dl, len, i, st, zh, zl, zeta);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_greedy_step_df(Ctx& c, float* Dh, float* Dl, const float* zh, const float* zl, long long rows,
                               long long len, double* beta, double* inf, const GreedyState* st, int i) {
  if (len % 4 != 0) {
    set_error("double-float greedy: snapshot length not a multiple of 4");
    return FETIDP_EINVAL;
  }
  ProfScope ps(c, FETIDP_K_GREEDY, 4.0 * rows * (double)len, 16.0 * rows * (double)len);
  greedy_step_df_kernel<<<(unsigned)rows, kThreads, 0, c.stream>>>(Dh, Dl, zh, zl, len, beta, inf, st, i);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_greedy_select(Ctx& c, const double* inf, long long n, const double* D, long long len, int i,
                              double tol_rb, double tie, GreedyState* st) {
  ProfScope ps(c, FETIDP_K_GREEDY, 0.0, 8.0 * (double)(n + len));
  greedy_select_kernel<<<1, 1024, 0, c.stream>>>(inf, n, D, len, i, tol_rb, tie, st);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_greedy_zeta(Ctx& c, const double* D, long long len, int i, const GreedyState* st, double* zeta) {
  ProfScope ps(c, FETIDP_K_GREEDY, 0.0, 16.0 * (double)len);
  greedy_zeta_kernel<<<gridn(len), kThreads, 0, c.stream>>>(D, len, i, st, zeta);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_greedy_alpha(Ctx& c, const double* Z, const double* nrm, const double* beta, int nrb,
                             const GreedyState* st, double* T, double* alpha) {
  greedy_T_kernel<<<(unsigned)(nrb * nrb), kThreads, 0, c.stream>>>(Z, c.snap, c.nsnap, nrb, st, T);
  FD_CHECK_LAUNCH();
  greedy_alpha_kernel<<<gridn(c.N), kThreads, 0, c.stream>>>(T, nrm, beta, c.N, nrb, alpha);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_scale_copy(Ctx& c, const double* x, const double* s, double* y, long long len) {
  scale_copy_kernel<<<gridn(len), kThreads, 0, c.stream>>>(x, s, y, len);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_column_gradients(Ctx& c, const double* src, long long kstride, long long lstride,
                                 int len_in, int mode, int unit_base, int nk, int ncol,
                                 double* out) {
  const double inv_h = (double)c.e;
  const long long work = (long long)nk * ncol * c.nelem * c.ngp;
  if (c.d == 2)
    column_gradients_kernel<2><<<gridn(work), kThreads, 0, c.stream>>>(
        c.e, c.n, c.perm + c.n, src, kstride, lstride, len_in, mode, unit_base, nk, ncol, inv_h, out);
  else
    column_gradients_kernel<3><<<gridn(work), kThreads, 0, c.stream>>>(
        c.e, c.n, c.perm + c.n, src, kstride, lstride, len_in, mode, unit_base, nk, ncol, inv_h, out);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_split_planes(Ctx& c, const double* x, long long n, float* hi, float* lo) {
  ProfScope ps(c, FETIDP_K_SETUP, 0.0, 16.0 * (double)n);
  split_planes_kernel<<<gridn(n), kThreads, 0, c.stream>>>(x, n, hi, lo);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_trace_tables_df(Ctx& c, const TraceTableSpecDF* specs_dev, int ntab, float* Th, float* Tl,
                                long long ldt) {
  const int nqp = c.nelem * c.ngp;
  const double wq = pow(0.5 / c.e, c.d);
  ProfScope ps(c, FETIDP_K_SETUP, 0.0, 0.0);
  dim3 grid((unsigned)((nqp + 127) / 128), (unsigned)ntab);
  if (c.d == 2)
    trace_tables_df_kernel<2><<<grid, 128, 0, c.stream>>>(specs_dev, nqp, wq, Th, Tl, ldt);
  else
    trace_tables_df_kernel<3><<<grid, 128, 0, c.stream>>>(specs_dev, nqp, wq, Th, Tl, ldt);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_trace_tables(Ctx& c, const TraceTableSpec* specs_dev, int ntab, double* T,
                             long long tstride) {
  const int nqp = c.nelem * c.ngp;
  const double wq = pow(0.5 / c.e, c.d);
  ProfScope ps(c, FETIDP_K_SETUP, 0.0, 0.0);
  dim3 grid((unsigned)((nqp + 127) / 128), (unsigned)ntab);
  trace_tables_kernel<<<grid, 128, 0, c.stream>>>(specs_dev, nqp, c.d, wq, T, tstride);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_rom_combine(Ctx& c, const double* src, long long kstride, int ld, int r0, int c0,
                            int rows, int cols, const double* coef, double* out, bool transpose) {
  rom_combine_kernel<<<gridn(c.N * rows * cols), kThreads, 0, c.stream>>>(
      src, kstride, ld, r0, c0, rows, cols, coef, c.nrb, c.N, out, transpose);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status k_body_loads(Ctx& c, const Geo& g, const int* perm_dev, const double* dirs_dev, const int* body_dev,
                           double* rhs, long long rhs_rs, double* fpc) {
  const int NA = 1 << c.d;
  const int nnode = c.d == 2 ? (c.e + 1) * (c.e + 1) : (c.e + 1) * (c.e + 1) * (c.e + 1);
  const size_t smem = sizeof(double) * ((size_t)c.nelem * NA + nnode);
  ProfScope ps(c, FETIDP_K_SETUP, 0.0, 8.0 * (double)c.N * c.m * c.n);
  cudaFuncSetAttribute(body_loads_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  body_loads_kernel<<<(unsigned)c.N, 256, smem, c.stream>>>(g, c.nelem, perm_dev, c.n, c.nr, c.np, dirs_dev,
                                                             body_dev, c.m, rhs, rhs_rs, fpc, c.N);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

}  // namespace fetidp
