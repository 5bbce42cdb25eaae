// Corner coarse problem (Sec. 3.2.1): S_PP_ring assembled from the ROM local
// primal Schur complements S_pp_ring^(s) (Eq. 43), factorised once at setup and
// solved exactly (FP64) at every use.
//
// GB300 design: in lattice-vertex slabs along the longest lattice axis the
// assembled S_PP is block tridiagonal (every cell couples two neighbouring
// vertex slabs).  It is factorised by block cyclic reduction -- the exact
// block Gaussian elimination of the SPD matrix in odd/even order -- so a
// solve is 2 log2(slabs) + 1 level-parallel sweeps of dense b x b FP64
// matrix-vector products (one warp per output row, all RHS per row) instead
// of a sequential sparse triangular substitution.
#include <cstring>

#include "common.cuh"
#include "host_linalg.h"

namespace fetidp {

namespace {

__global__ void bcr_gather_kernel(const int* __restrict__ perm, const double* __restrict__ b,
                                  long long b_rs, double* __restrict__ bl, long long bl_rs,
                                  long long len, int nrhs) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len * nrhs;
       t += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / len);
    const long long q = t - rhs * len;
    const int pq = perm[q];   // < 0: padding position of a smaller lattice's slab
    bl[rhs * bl_rs + q] = pq >= 0 ? b[rhs * b_rs + pq] : 0.0;
  }
}

__global__ void bcr_scatter_kernel(const int* __restrict__ perm, const double* __restrict__ xl,
                                   long long xl_rs, double* __restrict__ x, long long x_rs,
                                   long long len, int nrhs) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len * nrhs;
       t += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / len);
    const long long q = t - rhs * len;
    const int pq = perm[q];
    if (pq >= 0) x[rhs * x_rs + pq] = xl[rhs * xl_rs + q];
  }
}

// Identity on the padding positions of every slab block (positions past the slab's own size).
__global__ void bcr_pad_identity_kernel(double* __restrict__ A, long long bb, int b, const int* __restrict__ real,
                                        int nslab) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nslab * b;
       t += (long long)gridDim.x * blockDim.x) {
    const int sl = (int)(t / b), p = (int)(t - (long long)sl * b);
    if (p >= real[sl]) A[sl * bb + (long long)p * b + p] = 1.0;
  }
}

// Forward level: for even i of level l (new index i/2):
//   bl[l+1][i/2] = bl[l][i] - U_{i-1}^T bl[l][i-1] - V_{i+1}^T bl[l][i+1]
// Backward level: for odd j of level l:
//   xl[l][j] = Ainv_j bl[l][j] - V_j xl[l][j-1] - U_j xl[l][j+1], xl[l][even i] = xl[l+1][i/2]
struct BcrLevel {
  int b, n, nrhs;
  long long rs;                 // per-RHS stride of bl / xl
  const double* mats;
  const long long* offA;        // device tables, indexed by block j (-1 = absent)
  const long long* offU;
  const long long* offUT;
  const long long* offV;
  const long long* offVT;
  double* bl_l;                 // level l right-hand sides
  double* bl_n;                 // level l+1 right-hand sides
  double* xl_l;                 // level l solutions
  const double* xl_n;           // level l+1 solutions
};

constexpr int kMaxRhsBcr = 8;

__global__ void bcr_forward_kernel(BcrLevel P) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n_new = (P.n + 1) / 2;
  if (gw >= (long long)n_new * P.b) return;
  const int inew = (int)(gw / P.b), row = (int)(gw - (long long)inew * P.b);
  const int i = 2 * inew;
  const int b = P.b;
  for (int r0 = 0; r0 < P.nrhs; r0 += kMaxRhsBcr) {
    const int rb = min(kMaxRhsBcr, P.nrhs - r0);
    double acc[kMaxRhsBcr];
    for (int r = 0; r < kMaxRhsBcr; ++r) acc[r] = 0.0;
    if (i - 1 >= 0 && P.offUT[i - 1] >= 0) {
      const double* M = P.mats + P.offUT[i - 1] + (size_t)row * b;
      const double* v = P.bl_l + (size_t)(i - 1) * b;
      for (int q = lane; q < b; q += 32) {
        const double mv = M[q];
        for (int r = 0; r < rb; ++r) acc[r] += mv * v[(r0 + r) * P.rs + q];
      }
    }
    if (i + 1 < P.n) {
      const double* M = P.mats + P.offVT[i + 1] + (size_t)row * b;
      const double* v = P.bl_l + (size_t)(i + 1) * b;
      for (int q = lane; q < b; q += 32) {
        const double mv = M[q];
        for (int r = 0; r < rb; ++r) acc[r] += mv * v[(r0 + r) * P.rs + q];
      }
    }
    for (int r = 0; r < rb; ++r) {
      double s = acc[r];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) {
        const long long rr = (long long)(r0 + r) * P.rs;
        P.bl_n[rr + (size_t)inew * b + row] = P.bl_l[rr + (size_t)i * b + row] - s;
      }
    }
  }
}

__global__ void bcr_backward_kernel(BcrLevel P) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= (long long)P.n * P.b) return;
  const int j = (int)(gw / P.b), row = (int)(gw - (long long)j * P.b);
  const int b = P.b;
  if ((j & 1) == 0) {
    // even block: copy from the reduced level
    if (lane == 0)
      for (int r = 0; r < P.nrhs; ++r)
        P.xl_l[(long long)r * P.rs + (size_t)j * b + row] =
            P.xl_n[(long long)r * P.rs + (size_t)(j / 2) * b + row];
    return;
  }
  for (int r0 = 0; r0 < P.nrhs; r0 += kMaxRhsBcr) {
    const int rb = min(kMaxRhsBcr, P.nrhs - r0);
    double acc[kMaxRhsBcr];
    for (int r = 0; r < kMaxRhsBcr; ++r) acc[r] = 0.0;
    {
      const double* M = P.mats + P.offA[j] + (size_t)row * b;
      const double* v = P.bl_l + (size_t)j * b;
      for (int q = lane; q < b; q += 32) {
        const double mv = M[q];
        for (int r = 0; r < rb; ++r) acc[r] += mv * v[(r0 + r) * P.rs + q];
      }
    }
    {  // - V_j x_{j-1}; x_{j-1} (even) lives at level l+1 index (j-1)/2
      const double* M = P.mats + P.offV[j] + (size_t)row * b;
      const double* v = P.xl_n + (size_t)((j - 1) / 2) * b;
      for (int q = lane; q < b; q += 32) {
        const double mv = M[q];
        for (int r = 0; r < rb; ++r) acc[r] -= mv * v[(r0 + r) * P.rs + q];
      }
    }
    if (j + 1 < P.n) {
      const double* M = P.mats + P.offU[j] + (size_t)row * b;
      const double* v = P.xl_n + (size_t)((j + 1) / 2) * b;
      for (int q = lane; q < b; q += 32) {
        const double mv = M[q];
        for (int r = 0; r < rb; ++r) acc[r] -= mv * v[(r0 + r) * P.rs + q];
      }
    }
    for (int r = 0; r < rb; ++r) {
      double s = acc[r];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) P.xl_l[(long long)(r0 + r) * P.rs + (size_t)j * b + row] = s;
    }
  }
}

__global__ void bcr_final_kernel(const double* __restrict__ Ainv, int b, const double* bl,
                                 double* xl, long long rs, int nrhs) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= b) return;
  const int row = (int)gw;
  for (int r = 0; r < nrhs; ++r) {
    double s = 0.0;
    for (int q = lane; q < b; q += 32) s += Ainv[(size_t)row * b + q] * bl[r * rs + q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) xl[r * rs + row] = s;
  }
}

// ---- FP32 copy for the mixed path's inner iterations: the whole solve is one cooperative launch.
//      The level vectors hold up to eight RHS interleaved ([chunk][vec_len][8] floats), so one lane
//      reads all RHS of a column as two 16-byte loads; a warp forms four output rows, each lane
//      summing every 32nd column of them in FP32, and the 32 (row, RHS) lane partials are summed by
//      halving exchanges.  The levels are separated by grid-wide barriers whose waits are bounded.
constexpr int kBcrMaxLevels = 24;
struct BcrCoopF {
  int b, L, nch, nrhs;
  long long rs;                         // per-chunk stride of the level vectors, in 8-float entries
  long long len0;                       // nb * b
  const float* mats;
  const long long* tables;              // per level: A, U, UT, V, VT offset arrays of n_at[l] entries
  long long off_final;
  int n_at[kBcrMaxLevels + 1];
  long long vec_off[kBcrMaxLevels + 1];
  long long tab_off[kBcrMaxLevels];
  float* bl;
  float* xl;
  const int* perm;
  const double* bin;
  long long b_rs;
  double* xout;
  long long x_rs;
  unsigned* bar;                        // [0] arrivals, [1] generation (arrivals zeroed before launch)
  int* err;
  unsigned long long wait_ns;
};

__device__ __forceinline__ unsigned long long bcr_gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative launch.  The last block to arrive resets the arrival count
// and advances the generation; the others spin on the generation until the kernel's deadline, after
// which they record error 7 and go on (every later wait then ends at once, so the kernel finishes).
__device__ __forceinline__ void bcr_grid_sync(unsigned* bar, unsigned nblocks, unsigned long long deadline,
                                              int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      while (*gen == g) {
        if (bcr_gtime() > deadline) {
          atomicExch(err, 7);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// acc[a][r] += sgn * sum_q M[(row0 + a) b + q] v[q][r] over this lane's columns q (every 32nd),
// for the rows row0 + a < b.  One pair of 16-byte reads of v serves the four rows.
__device__ __forceinline__ void bcr_rows4_f32(const float* __restrict__ M, int row0, const float* __restrict__ v,
                                              int b, int lane, float sgn, float acc[4][8]) {
  const int na = min(4, b - row0);
#pragma unroll 2
  for (int q = lane; q < b; q += 32) {
    const float4 x0 = *reinterpret_cast<const float4*>(v + (size_t)q * 8);
    const float4 x1 = *reinterpret_cast<const float4*>(v + (size_t)q * 8 + 4);
    const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float mv = a < na ? sgn * __ldcs(M + (size_t)(row0 + a) * b + q) : 0.f;
#pragma unroll
      for (int r = 0; r < 8; ++r) acc[a][r] = fmaf(mv, xv[r], acc[a][r]);
    }
  }
}

// Sum of the 32 values acc[a][r] over the warp by halving exchanges (31 shuffles): lane l ends
// with the total of value l = 8 a + r.
__device__ __forceinline__ float bcr_warp_reduce32(float acc[4][8], int lane) {
  float v[32];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int r = 0; r < 8; ++r) v[8 * a + r] = acc[a][r];
#pragma unroll
  for (int o = 16, n = 32; o > 0; o >>= 1, n >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < n / 2; ++k) {
      const float send = up ? v[k] : v[k + n / 2];
      const float keep = up ? v[k + n / 2] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

__device__ __forceinline__ void bcr_zero(float acc[4][8]) {
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 8; ++y) acc[x][y] = 0.f;
}

__global__ void __launch_bounds__(256) bcr_coop_f32_kernel(BcrCoopF P) {
  const unsigned long long deadline = bcr_gtime() + P.wait_ns;
  const unsigned nblocks = gridDim.x;
  const int lane = threadIdx.x & 31;
  const long long gthreads = (long long)gridDim.x * blockDim.x;
  const long long gt0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nwarps = gthreads >> 5, gw0 = gt0 >> 5;
  const int b = P.b, g4 = (b + 3) / 4;
  const int a = lane >> 3, r = lane & 7;
  // level-0 right-hand sides: bl[ch][q][r8] = b[8 ch + r8][perm[q]] (0 on padding and absent RHS)
  for (long long t = gt0; t < (long long)P.nch * P.len0 * 8; t += gthreads) {
    const int r8 = (int)(t & 7);
    const long long e = t >> 3;
    const int ch = (int)(e / P.len0);
    const long long q = e - (long long)ch * P.len0;
    const int rr = ch * 8 + r8;
    const int pq = P.perm[q];
    P.bl[((size_t)ch * P.rs + q) * 8 + r8] = (pq >= 0 && rr < P.nrhs) ? (float)P.bin[rr * P.b_rs + pq] : 0.f;
  }
  bcr_grid_sync(P.bar, nblocks, deadline, P.err);
  // forward: bl[l+1][i/2] = bl[l][i] - U_{i-1}^T bl[l][i-1] - V_{i+1}^T bl[l][i+1]
  for (int l = 0; l < P.L; ++l) {
    const int n = P.n_at[l], n_new = (n + 1) / 2;
    const long long* tUT = P.tables + P.tab_off[l] + 2LL * n;
    const long long* tVT = P.tables + P.tab_off[l] + 4LL * n;
    for (long long task = gw0; task < (long long)n_new * g4 * P.nch; task += nwarps) {
      const int ch = (int)(task / ((long long)n_new * g4));
      const long long tr = task - (long long)ch * n_new * g4;
      const int inew = (int)(tr / g4), row0 = 4 * (int)(tr - (long long)inew * g4);
      const int i = 2 * inew;
      const float* vl = P.bl + ((size_t)ch * P.rs + P.vec_off[l]) * 8;
      float acc[4][8];
      bcr_zero(acc);
      if (i - 1 >= 0 && tUT[i - 1] >= 0)
        bcr_rows4_f32(P.mats + tUT[i - 1], row0, vl + (size_t)(i - 1) * b * 8, b, lane, 1.f, acc);
      if (i + 1 < n) bcr_rows4_f32(P.mats + tVT[i + 1], row0, vl + (size_t)(i + 1) * b * 8, b, lane, 1.f, acc);
      const float s = bcr_warp_reduce32(acc, lane);
      if (row0 + a < b) {
        const size_t o = (size_t)(row0 + a) * 8 + r;
        P.bl[((size_t)ch * P.rs + P.vec_off[l + 1]) * 8 + (size_t)inew * b * 8 + o] = vl[(size_t)i * b * 8 + o] - s;
      }
    }
    bcr_grid_sync(P.bar, nblocks, deadline, P.err);
  }
  // the last remaining block: x = A^{-1} bl
  for (long long task = gw0; task < (long long)g4 * P.nch; task += nwarps) {
    const int ch = (int)(task / g4), row0 = 4 * (int)(task - (long long)ch * g4);
    float acc[4][8];
    bcr_zero(acc);
    bcr_rows4_f32(P.mats + P.off_final, row0, P.bl + ((size_t)ch * P.rs + P.vec_off[P.L]) * 8, b, lane, 1.f, acc);
    const float s = bcr_warp_reduce32(acc, lane);
    if (row0 + a < b) P.xl[((size_t)ch * P.rs + P.vec_off[P.L]) * 8 + (size_t)(row0 + a) * 8 + r] = s;
  }
  bcr_grid_sync(P.bar, nblocks, deadline, P.err);
  // backward: x[l][j] = Ainv_j bl[l][j] - V_j x[l][j-1] - U_j x[l][j+1] (odd j), x[l][j] = x[l+1][j/2]
  for (int l = P.L - 1; l >= 0; --l) {
    const int n = P.n_at[l];
    const long long* tA = P.tables + P.tab_off[l];
    const long long* tU = tA + n;
    const long long* tV = tA + 3LL * n;
    for (long long task = gw0; task < (long long)n * g4 * P.nch; task += nwarps) {
      const int ch = (int)(task / ((long long)n * g4));
      const long long tr = task - (long long)ch * n * g4;
      const int j = (int)(tr / g4), row0 = 4 * (int)(tr - (long long)j * g4);
      const size_t cl = ((size_t)ch * P.rs + P.vec_off[l]) * 8, cn = ((size_t)ch * P.rs + P.vec_off[l + 1]) * 8;
      const size_t o = (size_t)(row0 + a) * 8 + r;
      if ((j & 1) == 0) {
        if (row0 + a < b) P.xl[cl + (size_t)j * b * 8 + o] = P.xl[cn + (size_t)(j / 2) * b * 8 + o];
        continue;
      }
      float acc[4][8];
      bcr_zero(acc);
      bcr_rows4_f32(P.mats + tA[j], row0, P.bl + cl + (size_t)j * b * 8, b, lane, 1.f, acc);
      bcr_rows4_f32(P.mats + tV[j], row0, P.xl + cn + (size_t)((j - 1) / 2) * b * 8, b, lane, -1.f, acc);
      if (j + 1 < n)
        bcr_rows4_f32(P.mats + tU[j], row0, P.xl + cn + (size_t)((j + 1) / 2) * b * 8, b, lane, -1.f, acc);
      const float s = bcr_warp_reduce32(acc, lane);
      if (row0 + a < b) P.xl[cl + (size_t)j * b * 8 + o] = s;
    }
    bcr_grid_sync(P.bar, nblocks, deadline, P.err);
  }
  // scatter of level 0 back to the primal DOF
  for (long long t = gt0; t < P.len0 * P.nrhs; t += gthreads) {
    const int rr = (int)(t / P.len0);
    const long long q = t - rr * P.len0;
    const int pq = P.perm[q];
    if (pq >= 0) P.xout[rr * P.x_rs + pq] = (double)P.xl[((size_t)(rr >> 3) * P.rs + q) * 8 + (rr & 7)];
  }
}

// dst[dst_off[k] + e] = (float) src[src_off[k] + e] for e < bb, block k = blockIdx.y
__global__ void bcr_convert_blocks_kernel(const double* __restrict__ src, const long long* __restrict__ src_off,
                                          float* __restrict__ dst, const long long* __restrict__ dst_off,
                                          long long bb) {
  const double* s = src + src_off[blockIdx.y];
  float* d = dst + dst_off[blockIdx.y];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < bb; e += (long long)gridDim.x * blockDim.x)
    d[e] = (float)s[e];
}

// grid-stride kernels may cap the grid; the warp-per-row kernels may not
inline int gridn(long long work, int threads = 256) {
  long long g = (work + threads - 1) / threads;
  if (g > 152LL * 16) g = 152LL * 16;
  return (int)(g < 1 ? 1 : g);
}
inline unsigned grid_exact(long long threads_total, int threads = 256) {
  const long long g = (threads_total + threads - 1) / threads;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

fetidp_status coarse_setup(Ctx& c, const double* Spp_dev) {
  const int d = c.d;
  CoarseBCR& B = c.bcr;
  // ---- slabs of every lattice (the vertex planes normal to its longest axis, ties -> highest
  //      axis; a fully clamped plane is skipped), concatenated lattice after lattice.  The coarse
  //      matrix is block-diagonal over lattices, so the chains of slab blocks simply follow each
  //      other with zero coupling; slabs are padded to the largest size with identity.
  struct SlabMap {
    std::vector<int> vslab, vpos;   // per local vertex: global slab, position in it (-1: clamped)
  };
  std::vector<SlabMap> maps(c.lat.size());
  std::vector<int> slab_real;       // DOF per slab (before padding)
  std::vector<std::vector<int>> slab_dofs;   // per slab: global primal DOF at each position
  int nb = 0, bmax = 0;
  for (size_t bl = 0; bl < c.lat.size(); ++bl) {
    const LatticeSpan& ls = c.lat[bl];
    int vd[3] = {1, 1, 1};
    for (int k = 0; k < d; ++k) vd[k] = ls.geo.nc[k] + 1;
    int ax = 0;
    for (int k = 1; k < d; ++k)
      if (vd[k] >= vd[ax]) ax = k;
    const int ca = ls.clamp_axis, cs = ls.clamp_side;
    const int clamp_val = cs == 0 ? 0 : vd[ca] - 1;
    const long long nvert = (long long)vd[0] * vd[1] * vd[2];
    std::vector<int> vnum(nvert, -1);
    {
      int q = 0;   // free vertex numbering (lexicographic, x fastest) as in setup, then + V0
      for (long long v = 0; v < nvert; ++v) {
        const int ijk[3] = {(int)(v % vd[0]), (int)((v / vd[0]) % vd[1]), (int)(v / ((long long)vd[0] * vd[1]))};
        if (ijk[ca] != clamp_val) vnum[v] = (int)ls.V0 + q++;
      }
    }
    std::vector<int> slab_of(vd[ax], -1);
    const int nb0 = nb;
    for (int sl = 0; sl < vd[ax]; ++sl) {
      if (ax == ca && sl == clamp_val) continue;
      slab_of[sl] = nb++;
    }
    slab_real.resize(nb, 0);
    slab_dofs.resize(nb);
    SlabMap& mp = maps[bl];
    mp.vslab.assign(nvert, -1);
    mp.vpos.assign(nvert, -1);
    for (long long v = 0; v < nvert; ++v) {
      if (vnum[v] < 0) continue;
      const int ijk[3] = {(int)(v % vd[0]), (int)((v / vd[0]) % vd[1]), (int)(v / ((long long)vd[0] * vd[1]))};
      const int sl = slab_of[ijk[ax]];
      mp.vslab[v] = sl;
      mp.vpos[v] = slab_real[sl] / d;
      for (int comp = 0; comp < d; ++comp) slab_dofs[sl].push_back(vnum[v] * d + comp);
      slab_real[sl] += d;
    }
    for (int sl = nb0; sl < nb; ++sl) bmax = std::max(bmax, slab_real[sl]);
  }
  const int b = bmax;
  B.b = b;
  B.nb = nb;
  std::vector<int> perm((size_t)nb * b, -1);
  for (int sl = 0; sl < nb; ++sl)
    for (size_t q = 0; q < slab_dofs[sl].size(); ++q) perm[(size_t)sl * b + q] = slab_dofs[sl][q];
  // ---- level structure and the device pool: per level l with n_l blocks, regions
  //      A (Ainv at odd slots after the level), U, U^T, V, V^T of n_l blocks each; the reduced
  //      block of the last level (then its inverse) follows.
  const long long bb = (long long)b * b;
  std::vector<int> nl;
  for (int n = nb; n > 1; n = (n + 1) / 2) nl.push_back(n);
  const int levels = (int)nl.size();
  std::vector<long long> base(levels + 1, 0);
  for (int l = 0; l < levels; ++l) base[l + 1] = base[l] + 5LL * nl[l] * bb;
  const long long pool = base[levels] + bb;
  FD_TRY(dalloc_t(c, &B.mats, (size_t)pool));
  B.mat_bytes = (size_t)pool * sizeof(double);
  double* P = B.mats;
  double* Cbuf[2] = {nullptr, nullptr};
  int *vslab_d = nullptr, *vpos_d = nullptr, *st_d = nullptr;
  const long long cmax = nb > 1 ? (long long)(nb - 1) * bb : bb;
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&Cbuf[0]), sizeof(double) * cmax));
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&Cbuf[1]), sizeof(double) * cmax));
  size_t nvert_all = 0;
  for (const SlabMap& mp : maps) nvert_all += mp.vslab.size();
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&vslab_d), sizeof(int) * nvert_all));
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&vpos_d), sizeof(int) * nvert_all));
  int* real_d = nullptr;
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&real_d), sizeof(int) * nb));
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&st_d), sizeof(int)));
  std::vector<size_t> voff(maps.size() + 1, 0);
  for (size_t bl = 0; bl < maps.size(); ++bl) {
    FD_CUDA(cudaMemcpyAsync(vslab_d + voff[bl], maps[bl].vslab.data(), sizeof(int) * maps[bl].vslab.size(),
                            cudaMemcpyHostToDevice, c.stream));
    FD_CUDA(cudaMemcpyAsync(vpos_d + voff[bl], maps[bl].vpos.data(), sizeof(int) * maps[bl].vpos.size(),
                            cudaMemcpyHostToDevice, c.stream));
    voff[bl + 1] = voff[bl] + maps[bl].vslab.size();
  }
  FD_CUDA(cudaMemcpyAsync(real_d, slab_real.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c.stream));
  FD_CUDA(cudaMemsetAsync(st_d, 0, sizeof(int), c.stream));
  FD_CUDA(cudaMemsetAsync(P, 0, sizeof(double) * (size_t)nb * bb, c.stream));
  FD_CUDA(cudaMemsetAsync(Cbuf[0], 0, sizeof(double) * cmax, c.stream));
  // ---- diagonal blocks A_i and couplings C_i = S(slab i, slab i+1) from the per-cell S_pp
  for (size_t bl = 0; bl < maps.size(); ++bl)
    FD_TRY(k_coarse_assemble(c, c.lat[bl], Spp_dev + c.lat[bl].cell0 * c.np * c.np, vslab_d + voff[bl],
                             vpos_d + voff[bl], b, P + base[0], Cbuf[0]));
  bcr_pad_identity_kernel<<<gridn((long long)nb * b), 256, 0, c.stream>>>(P + base[0], bb, b, real_d, nb);
  FD_CHECK_LAUNCH();
  // ---- block cyclic reduction on the device
  B.off_Ainv.assign(levels, {}); B.off_U.assign(levels, {}); B.off_UT.assign(levels, {});
  B.off_V.assign(levels, {}); B.off_VT.assign(levels, {});
  fetidp_status st = FETIDP_OK;
  for (int l = 0; l < levels && st == FETIDP_OK; ++l) {
    const int n = nl[l], nn = (n + 1) / 2;
    double* Al = P + base[l];
    double* Ul = Al + n * bb;
    double* UTl = Al + 2 * n * bb;
    double* Vl = Al + 3 * n * bb;
    double* VTl = Al + 4 * n * bb;
    double* An = P + base[l + 1];
    double* Cl = Cbuf[l & 1];
    double* Cn = Cbuf[(l + 1) & 1];
    const int nodd = n / 2, nu = (n - 1) / 2;
    // Ainv_j (odd j) in place; V_j = Ainv_j C_{j-1}^T; U_j = Ainv_j C_j (j + 1 < n)
    st = k_spd_inverse_batched(c, Al + bb, 2 * bb, b, b, nodd, st_d);
    if (st == FETIDP_OK)
      st = k_batched_gemm(c, false, true, b, b, b, 1.0, Al + bb, 2 * bb, b, Cl, 2 * bb, b, 0.0, Vl + bb, 2 * bb, b, nodd);
    if (st == FETIDP_OK)
      st = k_batched_gemm(c, false, false, b, b, b, 1.0, Al + bb, 2 * bb, b, Cl + bb, 2 * bb, b, 0.0, Ul + bb, 2 * bb,
                          b, nu);
    if (st == FETIDP_OK)
      st = k_batched_block_copy(c, Vl + bb, 2 * bb, b, 0, 0, VTl + bb, 2 * bb, b, b, b, nodd, true);
    if (st == FETIDP_OK)
      st = k_batched_block_copy(c, Ul + bb, 2 * bb, b, 0, 0, UTl + bb, 2 * bb, b, b, b, nu, true);
    // A'_q = A_2q - C_{2q-1}^T U_{2q-1} - C_2q V_{2q+1};  C'_q = - C_2q U_{2q+1}
    if (st == FETIDP_OK) st = k_batched_block_copy(c, Al, 2 * bb, b, 0, 0, An, bb, b, b, b, nn, false);
    if (st == FETIDP_OK)
      st = k_batched_gemm(c, true, false, b, b, b, -1.0, Cl + bb, 2 * bb, b, Ul + bb, 2 * bb, b, 1.0, An + bb, bb, b,
                          nn - 1);
    if (st == FETIDP_OK)
      st = k_batched_gemm(c, false, false, b, b, b, -1.0, Cl, 2 * bb, b, Vl + bb, 2 * bb, b, 1.0, An, bb, b, nodd);
    if (st == FETIDP_OK && nn > 1)
      st = k_batched_gemm(c, false, false, b, b, b, -1.0, Cl, 2 * bb, b, Ul + bb, 2 * bb, b, 0.0, Cn, bb, b, nu);
    if (st == FETIDP_OK) st = k_batched_symmetrize(c, An, bb, b, b, nn);   // against rounding drift
    std::vector<long long> oA(n, -1), oU(n, -1), oUT(n, -1), oV(n, -1), oVT(n, -1);
    for (int j = 1; j < n; j += 2) {
      oA[j] = base[l] + j * bb;
      oV[j] = base[l] + 3 * n * bb + j * bb;
      oVT[j] = base[l] + 4 * n * bb + j * bb;
      if (j + 1 < n) {
        oU[j] = base[l] + n * bb + j * bb;
        oUT[j] = base[l] + 2 * n * bb + j * bb;
      }
    }
    B.off_Ainv[l] = oA; B.off_U[l] = oU; B.off_UT[l] = oUT; B.off_V[l] = oV; B.off_VT[l] = oVT;
  }
  if (st == FETIDP_OK) st = k_spd_inverse_batched(c, P + base[levels], bb, b, b, 1, st_d);
  int hst = 0;
  if (st == FETIDP_OK) {
    FD_CUDA(cudaMemcpyAsync(&hst, st_d, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    FD_CUDA(cudaStreamSynchronize(c.stream));
  }
  tmp_free(c, Cbuf[0]); tmp_free(c, Cbuf[1]); tmp_free(c, vslab_d); tmp_free(c, vpos_d); tmp_free(c, real_d); tmp_free(c, st_d);
  FD_TRY(st);
  if (hst != 0) {
    set_error("coarse S_PP is not positive definite");
    return FETIDP_ESINGULAR;
  }
  B.off_final = base[levels];
  B.levels = levels;
  B.n_at.assign(nl.begin(), nl.end());
  B.n_at.push_back(1);
  B.vec_off.assign(B.levels + 1, 0);
  long long acc = 0;
  for (int l = 0; l <= B.levels; ++l) {
    B.vec_off[l] = acc;
    acc += (long long)B.n_at[l] * b;
  }
  B.vec_len = acc;
  // offset tables (device): per level the A, U, UT, V, VT arrays of n entries
  std::vector<long long> tab;
  for (int l = 0; l < B.levels; ++l)
    for (auto* v : {&B.off_Ainv[l], &B.off_U[l], &B.off_UT[l], &B.off_V[l], &B.off_VT[l]})
      tab.insert(tab.end(), v->begin(), v->end());
  FD_TRY(dalloc_t(c, &B.tables, tab.size() + 1));
  if (!tab.empty())
    FD_CUDA(cudaMemcpyAsync(B.tables, tab.data(), tab.size() * sizeof(long long), cudaMemcpyHostToDevice, c.stream));
  FD_TRY(dalloc_t(c, &B.perm, perm.size()));
  FD_CUDA(cudaMemcpyAsync(B.perm, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  FD_TRY(dalloc_t(c, &B.bl, (size_t)c.m * B.vec_len));
  FD_TRY(dalloc_t(c, &B.xl, (size_t)c.m * B.vec_len));
  if (c.mixed) {
    // FP32 copy of every used block, packed in table order; tab_f mirrors tab with the new offsets
    std::vector<long long> tab_f(tab.size(), -1), src_off, dst_off;
    long long pos = 0;
    for (size_t k = 0; k < tab.size(); ++k) {
      if (tab[k] < 0) continue;
      tab_f[k] = pos;
      src_off.push_back(tab[k]);
      dst_off.push_back(pos);
      pos += bb;
    }
    B.off_final_f = pos;
    src_off.push_back(B.off_final);
    dst_off.push_back(pos);
    pos += bb;
    FD_TRY(dalloc_t(c, &B.mats_f, (size_t)pos));
    B.mat_bytes_f = (size_t)pos * sizeof(float);
    FD_TRY(dalloc_t(c, &B.tables_f, tab_f.size() + 1));
    if (!tab_f.empty())
      FD_CUDA(cudaMemcpyAsync(B.tables_f, tab_f.data(), tab_f.size() * sizeof(long long), cudaMemcpyHostToDevice,
                              c.stream));
    long long* offs = nullptr;
    const size_t nblk = src_off.size();
    FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&offs), sizeof(long long) * 2 * nblk));
    FD_CUDA(cudaMemcpyAsync(offs, src_off.data(), sizeof(long long) * nblk, cudaMemcpyHostToDevice, c.stream));
    FD_CUDA(cudaMemcpyAsync(offs + nblk, dst_off.data(), sizeof(long long) * nblk, cudaMemcpyHostToDevice, c.stream));
    for (size_t k0 = 0; k0 < nblk; k0 += 65535) {
      const unsigned ny = (unsigned)std::min<size_t>(65535, nblk - k0);
      bcr_convert_blocks_kernel<<<dim3((unsigned)std::min<long long>((bb + 255) / 256, 1024), ny), 256, 0,
                                  c.stream>>>(B.mats, offs + k0, B.mats_f, offs + nblk + k0, bb);
      FD_CHECK_LAUNCH();
    }
    const int nch = (c.m + 7) / 8;
    FD_TRY(dalloc_t(c, &B.bl_f, (size_t)nch * B.vec_len * 8));
    FD_TRY(dalloc_t(c, &B.xl_f, (size_t)nch * B.vec_len * 8));
    // cooperative grid: every block resident (occupancy x SMs), no more than the widest level needs
    int dev = 0, nsm = 0, per_sm = 0;
    FD_CUDA(cudaGetDevice(&dev));
    FD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bcr_coop_f32_kernel, 256, 0));
    int coop_ok = 0;
    FD_CUDA(cudaDeviceGetAttribute(&coop_ok, cudaDevAttrCooperativeLaunch, dev));
    if (coop_ok && per_sm > 0) {
      // up to two CTAs per SM (measured faster than one at both the 2D and the 3D benchmark sizes),
      // no more than one warp per task of the widest level
      const long long widest = (long long)std::max(nb, 1) * ((b + 3) / 4) * nch;   // warp tasks
      const long long want = (widest * 32 + 255) / 256;
      B.coop_grid = (int)std::max<long long>(1, std::min<long long>((long long)std::min(per_sm, 2) * nsm, want));
      FD_TRY(dalloc_t(c, &B.coop_bar, 2));
      FD_CUDA(cudaMemsetAsync(B.coop_bar, 0, 2 * sizeof(unsigned), c.stream));
    }
    FD_CUDA(cudaStreamSynchronize(c.stream));   // host offset lists go out of scope
    tmp_free(c, offs);
  }
  FD_CUDA(cudaStreamSynchronize(c.stream));   // host tables go out of scope
  return FETIDP_OK;
}

fetidp_status coarse_solve(Ctx& c, const double* b, long long b_rs, double* x, long long x_rs,
                           int nrhs) {
  CoarseBCR& B = c.bcr;
  const long long len0 = (long long)B.nb * B.b;
  const long long rs = B.vec_len;
  ProfScope ps(c, FETIDP_K_COARSE, 2.0 * (B.mat_bytes / 8.0) * nrhs,
               (double)B.mat_bytes + 8.0 * nrhs * 4.0 * B.vec_len);
  bcr_gather_kernel<<<gridn(len0 * nrhs), 256, 0, c.stream>>>(B.perm, b, b_rs, B.bl, rs, len0, nrhs);
  FD_CHECK_LAUNCH();
  // device offset tables: per level 5 arrays of n entries, in order A, U, UT, V, VT
  std::vector<const long long*> tA(B.levels), tU(B.levels), tUT(B.levels), tV(B.levels), tVT(B.levels);
  {
    const long long* p = B.tables;
    for (int l = 0; l < B.levels; ++l) {
      const int n = B.n_at[l];
      tA[l] = p; p += n;
      tU[l] = p; p += n;
      tUT[l] = p; p += n;
      tV[l] = p; p += n;
      tVT[l] = p; p += n;
    }
  }
  for (int l = 0; l < B.levels; ++l) {
    BcrLevel P{B.b, B.n_at[l], nrhs, rs, B.mats, tA[l], tU[l], tUT[l], tV[l], tVT[l],
               B.bl + B.vec_off[l], B.bl + B.vec_off[l + 1], nullptr, nullptr};
    const long long warps = (long long)((B.n_at[l] + 1) / 2) * B.b;
    bcr_forward_kernel<<<grid_exact(warps * 32), 256, 0, c.stream>>>(P);
    FD_CHECK_LAUNCH();
  }
  {
    const int L = B.levels;
    bcr_final_kernel<<<grid_exact((long long)B.b * 32), 256, 0, c.stream>>>(
        B.mats + B.off_final, B.b, B.bl + B.vec_off[L], B.xl + B.vec_off[L], rs, nrhs);
    FD_CHECK_LAUNCH();
  }
  for (int l = B.levels - 1; l >= 0; --l) {
    BcrLevel P{B.b, B.n_at[l], nrhs, rs, B.mats, tA[l], tU[l], tUT[l], tV[l], tVT[l],
               B.bl + B.vec_off[l], nullptr, B.xl + B.vec_off[l], B.xl + B.vec_off[l + 1]};
    const long long warps = (long long)B.n_at[l] * B.b;
    bcr_backward_kernel<<<grid_exact(warps * 32), 256, 0, c.stream>>>(P);
    FD_CHECK_LAUNCH();
  }
  bcr_scatter_kernel<<<gridn(len0 * nrhs), 256, 0, c.stream>>>(B.perm, B.xl, rs, x, x_rs, len0, nrhs);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

// The same solve on the FP32 copy (mixed path): FP32 factor and level vectors, FP32 products summed
// per lane and over the warp, one cooperative launch for the whole solve (gather, levels, scatter).
// The rounding of the copy is a fixed linear perturbation of S_PP^{-1}.
fetidp_status coarse_solve_f32(Ctx& c, const double* b, long long b_rs, double* x, long long x_rs, int nrhs) {
  CoarseBCR& B = c.bcr;
  if (!B.mats_f || !B.coop_bar || !c.tc_err) return coarse_solve(c, b, b_rs, x, x_rs, nrhs);
  const int nch = (nrhs + 7) / 8;
  if (nch > (c.m + 7) / 8 || B.levels > kBcrMaxLevels) {
    set_error("coarse solve: more RHS or levels than the FP32 copy holds");
    return FETIDP_EINVAL;
  }
  ProfScope ps(c, FETIDP_K_COARSE, 2.0 * (B.mat_bytes_f / 4.0) * 8.0 * nch,
               (double)B.mat_bytes_f + 4.0 * 8.0 * nch * 4.0 * B.vec_len);
  BcrCoopF P;
  P.b = B.b;
  P.L = B.levels;
  P.nch = nch;
  P.nrhs = nrhs;
  P.rs = B.vec_len;
  P.len0 = (long long)B.nb * B.b;
  P.mats = B.mats_f;
  P.tables = B.tables_f;
  P.off_final = B.off_final_f;
  long long toff = 0;
  for (int l = 0; l <= B.levels; ++l) {
    P.n_at[l] = B.n_at[l];
    P.vec_off[l] = B.vec_off[l];
    if (l < B.levels) {
      P.tab_off[l] = toff;
      toff += 5LL * B.n_at[l];
    }
  }
  P.bl = B.bl_f;
  P.xl = B.xl_f;
  P.perm = B.perm;
  P.bin = b;
  P.b_rs = b_rs;
  P.xout = x;
  P.x_rs = x_rs;
  P.bar = B.coop_bar;
  P.err = c.tc_err;
  P.wait_ns = c.wait_ns;
  FD_CUDA(cudaMemsetAsync(B.coop_bar, 0, sizeof(unsigned), c.stream));   // arrivals (the generation runs on)
  void* args[] = {&P};
  FD_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(bcr_coop_f32_kernel), dim3((unsigned)B.coop_grid),
                                      dim3(256), args, 0, c.stream));
  count_launch();
  return FETIDP_OK;
}

}  // namespace fetidp
