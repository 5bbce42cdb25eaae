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
    bl[rhs * bl_rs + q] = b[rhs * b_rs + perm[q]];
  }
}

__global__ void bcr_scatter_kernel(const int* __restrict__ perm, const double* __restrict__ xl,
                                   long long xl_rs, double* __restrict__ x, long long x_rs,
                                   long long len, int nrhs) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len * nrhs;
       t += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / len);
    const long long q = t - rhs * len;
    x[rhs * x_rs + perm[q]] = xl[rhs * xl_rs + q];
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

fetidp_status coarse_setup(Ctx& c, const std::vector<double>& Spp_cells) {
  using namespace host;
  const int d = c.d;
  CoarseBCR& B = c.bcr;
  // ---- slab axis: longest vertex axis, ties -> highest axis index
  int vd[3] = {1, 1, 1};
  for (int k = 0; k < d; ++k) vd[k] = c.geo.nc[k] + 1;
  int ax = 0;
  for (int k = 1; k < d; ++k)
    if (vd[k] >= vd[ax]) ax = k;
  const int ca = c.clamp_axis, cs = c.clamp_side;
  const int clamp_val = cs == 0 ? 0 : vd[ca] - 1;
  // free vertex numbering (lexicographic, x fastest) must match setup's
  const long long nvert = (long long)vd[0] * vd[1] * vd[2];
  std::vector<int> vnum(nvert, -1);
  {
    int q = 0;
    for (long long v = 0; v < nvert; ++v) {
      const int ijk[3] = {(int)(v % vd[0]), (int)((v / vd[0]) % vd[1]), (int)(v / ((long long)vd[0] * vd[1]))};
      if (ijk[ca] != clamp_val) vnum[v] = q++;
    }
  }
  // slabs along ax (skipping a fully clamped slab), position of each free vertex in its slab
  std::vector<int> slab_of(vd[ax], -1);
  int nb = 0;
  for (int s = 0; s < vd[ax]; ++s) {
    if (ax == ca && s == clamp_val) continue;
    slab_of[s] = nb++;
  }
  std::vector<int> vslab(nvert, -1), vpos(nvert, -1);
  std::vector<int> count(nb, 0);
  for (long long v = 0; v < nvert; ++v) {
    if (vnum[v] < 0) continue;
    const int ijk[3] = {(int)(v % vd[0]), (int)((v / vd[0]) % vd[1]), (int)(v / ((long long)vd[0] * vd[1]))};
    const int sl = slab_of[ijk[ax]];
    vslab[v] = sl;
    vpos[v] = count[sl]++;
  }
  const int bv = count[0];
  for (int s = 1; s < nb; ++s)
    if (count[s] != bv) {
      set_error("coarse: unequal slab sizes");
      return FETIDP_EINVAL;
    }
  const int b = bv * d;
  B.b = b;
  B.nb = nb;
  std::vector<int> perm((size_t)nb * b);
  for (long long v = 0; v < nvert; ++v) {
    if (vnum[v] < 0) continue;
    for (int comp = 0; comp < d; ++comp)
      perm[(size_t)vslab[v] * b + vpos[v] * d + comp] = vnum[v] * d + comp;
  }
  // ---- assemble diagonal blocks A_i and couplings C_i = S(slab i, slab i+1)
  const size_t bb = (size_t)b * b;
  std::vector<std::vector<double>> A(nb, std::vector<double>(bb, 0.0));
  std::vector<std::vector<double>> C(nb > 1 ? nb - 1 : 0, std::vector<double>(bb, 0.0));
  const int nck = c.ncorner, npc = c.np;
  for (long long s = 0; s < c.N; ++s) {
    const int cijk[3] = {(int)(s % c.geo.nc[0]), (int)((s / c.geo.nc[0]) % c.geo.nc[1]),
                         (int)(s / ((long long)c.geo.nc[0] * c.geo.nc[1]))};
    long long vid[8];
    for (int k = 0; k < nck; ++k) {
      const int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
      long long v = 0, stride = 1;
      for (int q = 0; q < 3; ++q) {
        const int coord = cijk[q] + (q < d ? o[q] : 0);
        v += coord * stride;
        stride *= vd[q];
      }
      vid[k] = v;
    }
    const double* S = Spp_cells.data() + (size_t)s * npc * npc;
    for (int k1 = 0; k1 < nck; ++k1) {
      if (vnum[vid[k1]] < 0) continue;
      for (int k2 = 0; k2 < nck; ++k2) {
        if (vnum[vid[k2]] < 0) continue;
        const int s1 = vslab[vid[k1]], s2 = vslab[vid[k2]];
        for (int c1 = 0; c1 < d; ++c1)
          for (int c2 = 0; c2 < d; ++c2) {
            const double val = S[(size_t)(k1 * d + c1) * npc + k2 * d + c2];
            const int r = vpos[vid[k1]] * d + c1, q = vpos[vid[k2]] * d + c2;
            if (s1 == s2) A[s1][(size_t)r * b + q] += val;
            else if (s2 == s1 + 1) C[s1][(size_t)r * b + q] += val;
          }
      }
    }
  }
  // ---- block cyclic reduction, host FP64
  struct Lvl {
    int n;
    std::vector<long long> oA, oU, oUT, oV, oVT;
  };
  std::vector<Lvl> lv;
  std::vector<double> pool;   // matrices appended here
  auto push = [&](const std::vector<double>& M) {
    const long long off = (long long)pool.size();
    pool.insert(pool.end(), M.begin(), M.end());
    return off;
  };
  int n = nb;
  bool ok = true;
  std::vector<std::vector<double>> Acur = std::move(A), Ccur = std::move(C);
  while (n > 1) {
    Lvl L;
    L.n = n;
    L.oA.assign(n, -1); L.oU.assign(n, -1); L.oUT.assign(n, -1); L.oV.assign(n, -1); L.oVT.assign(n, -1);
    std::vector<std::vector<double>> Ainv(n), U(n), V(n);
    std::vector<char> fail(n, 0);
    parallel_for(n / 2, [&](int q) {
      const int j = 2 * q + 1;
      Ainv[j].assign(bb, 0.0);
      if (!spd_inverse(b, Acur[j].data(), b, Ainv[j].data(), b)) { fail[j] = 1; return; }
      V[j].assign(bb, 0.0);   // V_j = Ainv_j C_{j-1}^T
      gemm(false, true, b, b, b, 1.0, Ainv[j].data(), b, Ccur[j - 1].data(), b, 0.0, V[j].data(), b);
      if (j + 1 < n) {        // U_j = Ainv_j C_j
        U[j].assign(bb, 0.0);
        gemm(false, false, b, b, b, 1.0, Ainv[j].data(), b, Ccur[j].data(), b, 0.0, U[j].data(), b);
      }
    });
    for (int j = 1; j < n; j += 2) ok = ok && !fail[j];
    if (!ok) break;
    const int nn = (n + 1) / 2;
    std::vector<std::vector<double>> An(nn), Cn(nn > 1 ? nn - 1 : 0);
    parallel_for(nn, [&](int q) {
      const int i = 2 * q;
      An[q] = Acur[i];
      if (i - 1 >= 0)   // - C_{i-1}^T U_{i-1}
        gemm(true, false, b, b, b, -1.0, Ccur[i - 1].data(), b, U[i - 1].data(), b, 1.0, An[q].data(), b);
      if (i + 1 < n)    // - C_i V_{i+1}
        gemm(false, false, b, b, b, -1.0, Ccur[i].data(), b, V[i + 1].data(), b, 1.0, An[q].data(), b);
      if (i + 2 < n) {  // C'_q = - C_i U_{i+1}
        Cn[q].assign(bb, 0.0);
        gemm(false, false, b, b, b, -1.0, Ccur[i].data(), b, U[i + 1].data(), b, 0.0, Cn[q].data(), b);
      }
    });
    // symmetrise the reduced diagonal blocks against rounding drift
    for (int q = 0; q < nn; ++q)
      for (int r = 0; r < b; ++r)
        for (int s2 = r + 1; s2 < b; ++s2) {
          const double avg = 0.5 * (An[q][(size_t)r * b + s2] + An[q][(size_t)s2 * b + r]);
          An[q][(size_t)r * b + s2] = avg;
          An[q][(size_t)s2 * b + r] = avg;
        }
    for (int j = 1; j < n; j += 2) {
      L.oA[j] = push(Ainv[j]);
      L.oV[j] = push(V[j]);
      std::vector<double> T(bb);
      for (int r = 0; r < b; ++r)
        for (int s2 = 0; s2 < b; ++s2) T[(size_t)s2 * b + r] = V[j][(size_t)r * b + s2];
      L.oVT[j] = push(T);
      if (j + 1 < n) {
        L.oU[j] = push(U[j]);
        for (int r = 0; r < b; ++r)
          for (int s2 = 0; s2 < b; ++s2) T[(size_t)s2 * b + r] = U[j][(size_t)r * b + s2];
        L.oUT[j] = push(T);
      }
    }
    lv.push_back(std::move(L));
    Acur = std::move(An);
    Ccur = std::move(Cn);
    n = nn;
  }
  if (!ok) {
    set_error("coarse S_PP is not positive definite");
    return FETIDP_ESINGULAR;
  }
  {
    std::vector<double> Af(bb);
    if (!spd_inverse(b, Acur[0].data(), b, Af.data(), b)) {
      set_error("coarse S_PP is not positive definite");
      return FETIDP_ESINGULAR;
    }
    B.off_final = push(Af);
  }
  B.levels = (int)lv.size();
  B.n_at.clear();
  for (auto& L : lv) B.n_at.push_back(L.n);
  B.n_at.push_back(1);
  B.vec_off.assign(B.levels + 1, 0);
  long long acc = 0;
  for (int l = 0; l <= B.levels; ++l) {
    B.vec_off[l] = acc;
    acc += (long long)B.n_at[l] * b;
  }
  B.vec_len = acc;
  // offset tables appended after the matrices as raw long longs (device side)
  std::vector<long long> tab;
  B.off_Ainv.assign(B.levels, {}); B.off_U.assign(B.levels, {}); B.off_UT.assign(B.levels, {});
  B.off_V.assign(B.levels, {}); B.off_VT.assign(B.levels, {});
  for (int l = 0; l < B.levels; ++l) {
    B.off_Ainv[l] = lv[l].oA; B.off_U[l] = lv[l].oU; B.off_UT[l] = lv[l].oUT;
    B.off_V[l] = lv[l].oV; B.off_VT[l] = lv[l].oVT;
    for (auto* v : {&lv[l].oA, &lv[l].oU, &lv[l].oUT, &lv[l].oV, &lv[l].oVT})
      tab.insert(tab.end(), v->begin(), v->end());
  }
  B.mat_bytes = pool.size() * sizeof(double);
  FD_TRY(dalloc_t(c, &B.mats, pool.size()));
  FD_CUDA(cudaMemcpyAsync(B.mats, pool.data(), B.mat_bytes, cudaMemcpyHostToDevice, c.stream));
  FD_TRY(dalloc_t(c, &B.tables, tab.size() + 1));
  if (!tab.empty())
    FD_CUDA(cudaMemcpyAsync(B.tables, tab.data(), tab.size() * sizeof(long long),
                            cudaMemcpyHostToDevice, c.stream));
  FD_TRY(dalloc_t(c, &B.perm, perm.size()));
  FD_CUDA(cudaMemcpyAsync(B.perm, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice,
                          c.stream));
  FD_TRY(dalloc_t(c, &B.bl, (size_t)c.m * B.vec_len));
  FD_TRY(dalloc_t(c, &B.xl, (size_t)c.m * B.vec_len));
  FD_CUDA(cudaStreamSynchronize(c.stream));   // host pool / tables go out of scope
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

}  // namespace fetidp
