// Operators and Krylov drivers of the ROM-based inexact FETI-DP solver, and
// the C ABI (include/fetidp.h).
//
// * op_apply_F   -- Eq. 48: gather, F_dd_ring, coarse correction, scatter.
// * op_apply_MD  -- Eq. 49: D-scaled gather, S_dd_ring, D-scaled scatter.
// * U_apply      -- Algorithm 3 (U_ring v); UT_apply its transpose.
// * K_rom_inv    -- Algorithm 2 / Eq. 45 with the local ROM solve of Eq. 46.
// * precondition -- Algorithm 1 (the block preconditioner of Eq. 44).
// * pcg          -- inner PCG on F_ring preconditioned by M_D_ring (Sec. 3.2.3).
// * fgmres       -- outer right-preconditioned flexible GMRES on Eq. 16.
// Every step runs in the kernels of this library; the host only keeps the
// Krylov scalars (Hessenberg, Givens rotations, convergence decisions).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include <initializer_list>

#include "common.cuh"

namespace fetidp {

namespace {
thread_local std::string g_last_error;

constexpr int S_RZ0 = 0, S_RZ1 = 1, S_PQ = 2, S_RR = 3, S_ACT = 4, S_R0 = 5, S_ERR = 6, S_ITS = 7,
              S_NSLOT = 8;

__global__ void copy_cells_kernel(const double* __restrict__ x, long long x_rs, int x_cs,
                                  double* __restrict__ y, long long y_rs, int y_cs, int len,
                                  long long ncell, int nrhs, double scale) {
  const long long per = ncell * len;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < per * nrhs;
       t += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / per);
    const long long q = t - rhs * per;
    const long long cell = q / len;
    const int i = (int)(q - cell * len);
    const double v = x[rhs * x_rs + cell * x_cs + i];
    y[rhs * y_rs + cell * y_cs + i] = scale == 1.0 ? v : scale * v;
  }
}

__global__ void axpby_kernel(const double* __restrict__ x, long long xs, const double* __restrict__ y,
                             long long ys, double* __restrict__ out, long long os, double a, double b,
                             long long len, int nrhs) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len * nrhs;
       t += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / len);
    const long long q = t - rhs * len;
    out[rhs * os + q] = a * x[rhs * xs + q] + b * y[rhs * ys + q];
  }
}

// out[rhs][cell][perm[li]] = in[rhs][cell][li]
__global__ void permute_out_kernel(const int* __restrict__ perm, const double* __restrict__ in,
                                   double* __restrict__ out, int n, long long ncell, int nrhs) {
  const long long per = ncell * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < per * nrhs;
       t += (long long)gridDim.x * blockDim.x) {
    const long long cn = t / n;
    const int li = (int)(t - cn * n);
    out[cn * n + perm[li]] = in[t];
  }
}

// x += alpha p, r -= alpha q with alpha = rz / pq per active RHS
__global__ void pcg_xr_kernel(double* __restrict__ X, double* __restrict__ R,
                              const double* __restrict__ P, const double* __restrict__ Q,
                              const double* __restrict__ scal, int rz_slot, long long L, int nrhs) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < L * nrhs;
       t += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / L);
    const double act = scal[S_ACT * nrhs + rhs];
    if (act == 0.0) continue;
    const double alpha = scal[rz_slot * nrhs + rhs] / scal[S_PQ * nrhs + rhs];
    X[t] += alpha * P[t];
    R[t] -= alpha * Q[t];
  }
}

// Convergence test of one PCG iteration on the device (one thread per RHS): counts the iteration,
// flags a breakdown (p^T F p <= 0 or a non-finite residual) and clears the RHS's active flag when
// ||r|| / ||r_0|| <= tol or r = 0.  Lets whole iterations run without a host round trip.
__global__ void pcg_check_kernel(double* __restrict__ scal, int nrhs, double tol) {
  const int r = threadIdx.x;
  if (r >= nrhs || scal[S_ACT * nrhs + r] == 0.0) return;
  const double pq = scal[S_PQ * nrhs + r], rr = scal[S_RR * nrhs + r];
  scal[S_ITS * nrhs + r] += 1.0;
  if (!(pq > 0.0) || !isfinite(rr)) {
    scal[S_ERR * nrhs + r] = 1.0;
    scal[S_ACT * nrhs + r] = 0.0;
    return;
  }
  if (sqrt(rr / scal[S_R0 * nrhs + r]) <= tol || rr == 0.0) scal[S_ACT * nrhs + r] = 0.0;
}

// p = z + beta p, beta = rz_new / rz_old per active RHS
__global__ void pcg_p_kernel(double* __restrict__ P, const double* __restrict__ Zv,
                             const double* __restrict__ scal, int new_slot, int old_slot, long long L,
                             int nrhs) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < L * nrhs;
       t += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / L);
    if (scal[S_ACT * nrhs + rhs] == 0.0) continue;
    const double beta = scal[new_slot * nrhs + rhs] / scal[old_slot * nrhs + rhs];
    P[t] = Zv[t] + beta * P[t];
  }
}

inline int gridn(long long work) {
  long long g = (work + 255) / 256;
  if (g > 152LL * 16) g = 152LL * 16;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Device memory comes from the device's stream-ordered pool, whose release threshold is raised
// once per device: freed blocks stay in the pool, so a context set up after another reuses its
// memory without the device-wide synchronisation of cudaMalloc / cudaFree.
static std::mutex g_pool_mu;
static bool g_pool_ready[64];
static void ensure_pool(int dev) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (dev < 0 || dev >= 64 || g_pool_ready[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  g_pool_ready[dev] = true;
}

// Timing events outlive contexts, per device: a profiled context borrows them and gives them
// back when it is destroyed, so profiling a new context costs no event creation.
static std::vector<cudaEvent_t> g_events[64];
cudaEvent_t event_take(int dev) {
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (dev >= 0 && dev < 64 && !g_events[dev].empty()) {
      cudaEvent_t e = g_events[dev].back();
      g_events[dev].pop_back();
      return e;
    }
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void event_give(int dev, cudaEvent_t e) {
  if (!e) return;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (dev >= 0 && dev < 64) g_events[dev].push_back(e);
  else cudaEventDestroy(e);
}

// 256 more event pairs for profiled launches, up to 16384 pairs per context (later launches of a
// profiled class are counted but not timed).
bool prof_grow(Ctx& c) {
  Prof& P = c.prof;
  if (P.capacity >= 16384) return false;
  for (int i = 0; i < 256; ++i) {
    cudaEvent_t a = event_take(c.device), b = event_take(c.device);
    if (!a || !b) {
      event_give(c.device, a);
      event_give(c.device, b);
      break;
    }
    P.ev.push_back(a);
    P.ev.push_back(b);
    P.cls.push_back(0);
    ++P.capacity;
  }
  return P.used < P.capacity;
}

fetidp_status tmp_alloc(Ctx& c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 8;
  ensure_pool(c.device);
  cudaError_t e = cudaMallocAsync(p, bytes, c.stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error(std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FETIDP_ENOMEM : FETIDP_ECUDA;
  }
  return FETIDP_OK;
}

void tmp_free(Ctx& c, void* p) {
  if (p) cudaFreeAsync(p, c.stream);
}

fetidp_status dalloc(Ctx& c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 8;
  ensure_pool(c.device);
  cudaError_t e = cudaMallocAsync(p, bytes, c.stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FETIDP_ENOMEM : FETIDP_ECUDA;
  }
  c.allocations.push_back(*p);
  c.device_bytes += bytes;
  return FETIDP_OK;
}

namespace {

fetidp_status copy_cells(Ctx& c, CCellVec x, CellVec y, int len, int nrhs, double scale = 1.0) {
  copy_cells_kernel<<<gridn(c.N * len * nrhs), 256, 0, c.stream>>>(x.p, x.rs, x.cs, y.p, y.rs, y.cs,
                                                                   len, c.N, nrhs, scale);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

fetidp_status axpby(Ctx& c, const double* x, long long xs, const double* y, long long ys, double* out,
                    long long os, double a, double b, long long len, int nrhs) {
  axpby_kernel<<<gridn(len * nrhs), 256, 0, c.stream>>>(x, xs, y, ys, out, os, a, b, len, nrhs);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

// Per-cell operator sub-blocks (FP64 path): y = alpha M x + beta y, M rows x cols with
// row stride ld and per-cell stride mstride.
fetidp_status cell_op(Ctx& c, const double* mats, long long mstride, int ld, int rows, int cols,
                      CCellVec x, CellVec y, double alpha, double beta) {
  return k_cell_gemv_strided(c, mats, mstride, ld, rows, cols, x, y, alpha, beta, c.m);
}

}  // namespace

// ------------------------------------------------------------------ Eq. 48
fetidp_status op_apply_F(Ctx& c, const double* lam, long long lam_rs, double* y, long long y_rs) {
  const int m = c.m, nd = c.nd, np = c.np, nr = c.nr, ni = c.ni;
  CellVec g{c.w_d1, c.N * nd, nd}, yd{c.w_d2, c.N * nd, nd}, cp{c.w_p1, c.N * np, np};
  FD_TRY(k_gather_BT(c, lam, lam_rs, nullptr, g, m, 0.0));
  if (c.asm_f32 && c.sym_T)
    FD_TRY(k_cell_symv_f32(c, c.Fdd_f, cview(g), yd, 1.0, 0.0, m));
  else if (c.asm_f32)
    FD_TRY(k_cell_gemm_f32(c, c.Fdd_f, c.ld_f, nd, nd, cview(g), yd, 1.0, 0.0, m));
  else if (c.mixed)
    FD_TRY(tc_comb_apply(c, c.cFdd, cview(g), c.delta, c.delta, yd.p, true, yd.rs, yd.cs, 1.0, 0.0, m, c.N));
  else
    FD_TRY(cell_op(c, c.Fdd_c, (long long)nd * nd, nd, nd, nd, cview(g), yd, 1.0, 0.0));
  // coarse correction: c_p = (T_dr U_rp_ring)^T g, assembled, S_PP^{-1}, prolonged.  The mixed path
  // applies it with FP32 copies of U_dp_ring and of the S_PP factor (a fixed perturbation of the
  // operator of the inner iterations, well inside their 1e-6 tolerance; the outer FGMRES is FP64).
  if (c.Udp_f)
    FD_TRY(k_udp_f32(c, true, cview(g), cp, 1.0, 0.0, m));
  else
    FD_TRY(cell_op(c, c.UrpT_c + ni, (long long)np * nr, nr, np, nd, cview(g), cp, 1.0, 0.0));
  FD_TRY(k_primal_assemble(c, cview(cp), c.w_P1, c.nP, 1.0, 0.0, m));
  if (c.bcr.mats_f)
    FD_TRY(coarse_solve_f32(c, c.w_P1, c.nP, c.w_P2, c.nP, m));
  else
    FD_TRY(coarse_solve(c, c.w_P1, c.nP, c.w_P2, c.nP, m));
  FD_TRY(k_primal_extract(c, c.w_P2, c.nP, cp, m));
  if (c.Udp_f)
    FD_TRY(k_udp_f32(c, false, cview(cp), yd, 1.0, 1.0, m));
  else
    FD_TRY(cell_op(c, c.Urp_c + (size_t)ni * np, (long long)nr * np, np, nd, np, cview(cp), yd, 1.0, 1.0));
  FD_TRY(k_scatter_B(c, cview(yd), y, y_rs, nullptr, 1.0, 0.0, m));
  return FETIDP_OK;
}

// ------------------------------------------------------------------ Eq. 49
fetidp_status op_apply_MD(Ctx& c, const double* r, long long r_rs, double* z, long long z_rs) {
  const int m = c.m, nd = c.nd;
  CellVec g{c.w_d1, c.N * nd, nd}, yd{c.w_d2, c.N * nd, nd};
  FD_TRY(k_gather_BT(c, r, r_rs, c.dinfo, g, m, 0.0));
  if (c.asm_f32 && c.sym_T)
    FD_TRY(k_cell_symv_f32(c, c.Sdd_f, cview(g), yd, 1.0, 0.0, m));
  else if (c.asm_f32)
    FD_TRY(k_cell_gemm_f32(c, c.Sdd_f, c.ld_f, nd, nd, cview(g), yd, 1.0, 0.0, m));
  else if (c.mixed)
    FD_TRY(tc_comb_apply(c, c.cSdd, cview(g), c.alpha, c.alpha, yd.p, true, yd.rs, yd.cs, 1.0, 0.0, m, c.N));
  else
    FD_TRY(cell_op(c, c.Sdd_c, (long long)nd * nd, nd, nd, nd, cview(g), yd, 1.0, 0.0));
  FD_TRY(k_scatter_B(c, cview(yd), z, z_rs, c.dinfo, 1.0, 0.0, m));
  return FETIDP_OK;
}

// ------------------------------------------------------------------ Eq. 47
// z = M_D^{-ROM} r: the Dirichlet preconditioner of Eq. 30 whose interior solves K_ii^(s)^{-1} are
// approximated like Eq. 46 approximates K_rr^(s)^{-1}: R = [K_ii^(sigma_k)^{-1} v_i]_k and the
// K_ii^(s)-orthogonal projection x_i = R (R^T K_ii R)^{-1} R^T v_i.  Every product with the cell's
// own stiffness is the matrix-free K_s of Eq. 52 on full local vectors.
fetidp_status op_apply_MD_rom(Ctx& c, const double* r, long long r_rs, double* z, long long z_rs) {
  if (!c.Kii_inv) { set_error("the context was set up without the Eq. 47 interface option"); return FETIDP_EINVAL; }
  const int m = c.m, nd = c.nd, ni = c.ni, n = c.n, nrb = c.nrb;
  CellVec g{c.w_d1, c.N * nd, nd};
  FD_TRY(k_gather_BT(c, r, r_rs, c.dinfo, g, m, 0.0));
  // K_s (0; g; 0): its interior part is K_id g, its dual part K_dd g
  CellVec ua{c.w_cell_a, c.N * n, n}, kb{c.w_cell_b, c.N * n, n};
  FD_CUDA(cudaMemsetAsync(c.w_cell_a, 0, sizeof(double) * (size_t)m * c.N * n, c.stream));
  FD_TRY(copy_cells(c, cview(g), CellVec{c.w_cell_a + ni, c.N * n, n}, nd, m));
  FD_TRY(k_apply_K(c, cview(ua), kb, 1, m, true, false, c.snap, 0.0));
  // x_i ~ K_ii^{-1} K_id g
  CCellVec vi{c.w_cell_b, c.N * n, n};
  CellVec R{c.w_R, c.N * nrb * ni, nrb * ni}, KR{c.w_KR, c.N * nrb * ni, nrb * ni}, xi{c.w_i, c.N * ni, ni};
  FD_TRY(k_grouped_gemm(c, c.Kii_inv, (long long)ni * ni, ni, ni, ni, vi, R, nullptr, 1.0, 0.0, m, true, ni));
  FD_TRY(k_apply_K(c, cview(R), KR, nrb, m, true, false, c.snap, 0.0, ni));
  FD_TRY(k_gram_solve(c, c.w_R, c.w_KR, vi, xi, m, ni));
  // y_d = K_dd g - K_di x_i = [K_s (-x_i; g; 0)]_d
  FD_TRY(copy_cells(c, cview(xi), ua, ni, m, -1.0));
  FD_TRY(k_apply_K(c, cview(ua), kb, 1, m, true, false, c.snap, 0.0));
  FD_TRY(k_scatter_B(c, CCellVec{c.w_cell_b + ni, c.N * n, n}, z, z_rs, c.dinfo, 1.0, 0.0, m));
  return FETIDP_OK;
}

namespace {

// Algorithm 3: out_L = U_ring v,  zP (= S_PP^{-1} (v_P - U_RP^T v_R)) kept in c.w_zP.
fetidp_status U_apply(Ctx& c, CCellVec vR, const double* vP, long long vP_rs, double* out_L,
                      long long out_rs) {
  const int m = c.m, nd = c.nd, np = c.np, nr = c.nr, ni = c.ni;
  CellVec cp{c.w_p1, c.N * np, np}, td{c.w_d1, c.N * nd, nd};
  FD_TRY(cell_op(c, c.UrpT_c, (long long)np * nr, nr, np, nr, vR, cp, 1.0, 0.0));
  FD_TRY(k_copy_scale(c, vP, c.w_P1, c.nP, m, vP_rs, c.nP, nullptr, 1.0));
  FD_TRY(k_primal_assemble(c, cview(cp), c.w_P1, c.nP, -1.0, 1.0, m));
  FD_TRY(coarse_solve(c, c.w_P1, c.nP, c.w_zP, c.nP, m));
  // t_d = U_rd_ring^T v_r - T_dr U_rp_ring A_p^T z_P
  if (c.exact)   // standard FETI-DP: rows d of each cell's own K_rr^{-1} (symmetric)
    FD_TRY(cell_op(c, c.Kinv + (size_t)ni * nr, (long long)nr * nr, nr, nd, nr, vR, td, 1.0, 0.0));
  else if (c.Uid_f) {   // assembled FP32 blocks: U_id^T v_i + F_dd v_d
    FD_TRY(k_cell_gemm_f32(c, c.Uid_f, c.ld_id, nd, ni, vR, td, 1.0, 0.0, m));
    const CCellVec vd{vR.p + ni, vR.rs, vR.cs};
    if (c.sym_T)
      FD_TRY(k_cell_symv_f32(c, c.Fdd_f, vd, td, 1.0, 1.0, m));
    else
      FD_TRY(k_cell_gemm_f32(c, c.Fdd_f, c.ld_f, nd, nd, vd, td, 1.0, 1.0, m));
  } else if (c.mixed)
    FD_TRY(tc_comb_apply(c, c.cUrdT, vR, c.delta, c.delta, td.p, true, td.rs, td.cs, 1.0, 0.0, m, c.N));
  else
    FD_TRY(k_grouped_gemm(c, c.Kinv + (size_t)ni * nr, (long long)nr * nr, nr, nd, nr, vR, td, c.delta,
                          1.0, 0.0, m, false, 0));
  FD_TRY(k_primal_extract(c, c.w_zP, c.nP, cp, m));
  FD_TRY(cell_op(c, c.Urp_c + (size_t)ni * np, (long long)nr * np, np, nd, np, cview(cp), td, -1.0, 1.0));
  FD_TRY(k_scatter_B(c, cview(td), out_L, out_rs, nullptr, 1.0, 0.0, m));
  return FETIDP_OK;
}

// Eq. 46 for every (rhs, cell): x_r = R (R^T K_s R)^{-1} R^T v_r, R = [K_rr^(sigma_k)^{-1} v_r]_k;
// standard FETI-DP: x_r = K_rr^(s)^{-1} v_r with the cell's own inverse
fetidp_status local_rom(Ctx& c, CCellVec vR, CellVec xR) {
  const int m = c.m, nr = c.nr, nrb = c.nrb;
  if (c.exact) return cell_op(c, c.Kinv, (long long)nr * nr, nr, nr, nr, vR, xR, 1.0, 0.0);
  if (c.mixed) {
    float* Rf = reinterpret_cast<float*>(c.w_R);
    float* KRf = reinterpret_cast<float*>(c.w_KR);
    const long long rs = c.N * nrb * nr;
    const long long rext = (long long)m * rs;       // floats held by each buffer
    FD_TRY(tc_apply(c, c.opKinv, vR, nullptr, Rf, false, rs, nrb * nr, nr, 1.0, 0.0, m, c.N, rext));
    FD_TRY(fd_check_tc("local ROM basis (tensor cores)"));
    FD_TRY(k_apply_K_f32(c, Rf, rs, nrb * nr, KRf, rs, nrb * nr, nrb, m, true, true, rext));
    FD_TRY(fd_check_cell("local ROM K_s products"));
    FD_TRY(k_gram_solve_f32(c, Rf, KRf, vR, xR, m, rext));
    FD_TRY(fd_check_cell("local ROM Gram solve"));
    return FETIDP_OK;
  }
  CellVec R{c.w_R, c.N * nrb * nr, nrb * nr};
  FD_TRY(k_grouped_gemm(c, c.Kinv, (long long)nr * nr, nr, nr, nr, vR, R, nullptr, 1.0, 0.0, m, true,
                        nr));
  CellVec KR{c.w_KR, c.N * nrb * nr, nrb * nr};
  FD_TRY(k_apply_K(c, cview(R), KR, nrb, m, true, true, c.snap, 0.0));
  FD_TRY(k_gram_solve(c, c.w_R, c.w_KR, vR, xR, m));
  return FETIDP_OK;
}

}  // namespace

// inner PCG on F_ring y = b (Sec. 3.2.3); x: output [m][L] with row stride x_rs
fetidp_status pcg_solve(Ctx& c, const double* b, long long b_rs, double* x, long long x_rs) {
  const int m = c.m;
  const long long L = c.L, mL = (long long)m * L;
  double *X = c.pcg, *R = c.pcg + mL, *Zv = c.pcg + 2 * mL, *P = c.pcg + 3 * mL, *Q = c.pcg + 4 * mL;
  double* sc = c.scal;
  double* hs = c.h_scal;
  FD_TRY(k_copy_scale(c, b, R, L, m, b_rs, L, nullptr, 1.0));
  FD_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * mL, c.stream));
  FD_TRY(k_dot(c, R, L, R, L, L, m, sc + S_R0 * m));
  FD_CUDA(cudaMemcpyAsync(hs, sc, sizeof(double) * S_NSLOT * m, cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  std::vector<double> rr0(m), act(m, 0.0);
  int nact = 0;
  for (int r = 0; r < m; ++r) {
    rr0[r] = hs[S_R0 * m + r];
    if (!std::isfinite(rr0[r])) { set_error("non-finite PCG right-hand side"); return FETIDP_EBREAKDOWN; }
    act[r] = rr0[r] > 0.0 ? 1.0 : 0.0;
    nact += act[r] > 0.0;
  }
  if (nact > 0) {
    FD_CUDA(cudaMemcpyAsync(sc + S_ACT * m, act.data(), sizeof(double) * m, cudaMemcpyHostToDevice, c.stream));
    FD_TRY(op_apply_MD(c, R, L, Zv, L));
    FD_CUDA(cudaMemcpyAsync(P, Zv, sizeof(double) * mL, cudaMemcpyDeviceToDevice, c.stream));
    FD_TRY(k_dot(c, R, L, Zv, L, L, m, sc + S_RZ0 * m));
  }
  const int max_it = c.opt.fixed_inner > 0 ? c.opt.fixed_inner : c.opt.max_inner;
  int cur = S_RZ0, it = 0;
  // Graph path (no fixed iteration count): two iterations (one per rho slot) are captured once
  // per context and replayed; the convergence test runs on the device and the host reads the
  // flags once per replay.  A replay may run one iteration past convergence: the converged
  // right-hand sides are frozen (their x, r, p do not change), only time is spent.  Profiled
  // launches keep their event pairs as event nodes of the graph, read after every replay.
  const bool graph_ok = nact > 0 && c.opt.fixed_inner <= 0 && !c.pcg_graph_failed;
  // The graph runs on the context's own non-blocking stream (capture is not possible on the
  // legacy default stream), ordered after and before the caller's stream by events.
  struct StreamSwap {
    Ctx& c;
    cudaStream_t user;
    bool on = false;
    ~StreamSwap() {
      if (!on) return;
      cudaEventRecord(c.ev_out, c.ws);
      cudaStreamWaitEvent(user, c.ev_out, 0);
      c.stream = user;
    }
  } swap{c, c.stream};
  if (graph_ok) {
    if (!c.ws) {
      FD_CUDA(cudaStreamCreateWithFlags(&c.ws, cudaStreamNonBlocking));
      FD_CUDA(cudaEventCreateWithFlags(&c.ev_in, cudaEventDisableTiming));
      FD_CUDA(cudaEventCreateWithFlags(&c.ev_out, cudaEventDisableTiming));
    }
    FD_CUDA(cudaEventRecord(c.ev_in, c.stream));
    FD_CUDA(cudaStreamWaitEvent(c.ws, c.ev_in, 0));
    c.stream = c.ws;
    swap.on = true;
  }
  if (graph_ok) {
    const double tol = c.mixed ? c.opt.tol_inner_mixed : c.opt.tol_inner;
    Prof& pf = c.prof;
    if (c.pcg_graph && c.pcg_graph_mask != pf.mask) {   // profiled classes changed: capture again
      FD_CUDA(cudaGraphExecDestroy(c.pcg_graph));
      c.pcg_graph = nullptr;
    }
    if (!c.pcg_graph) {
      const long long l0 = g_launches.load();
      pf.captured.clear();
      if (pf.mask != 0 && pf.gev.empty())
        for (int i = 0; i < 512; ++i) {
          cudaEvent_t e = event_take(c.device);
          if (!e) break;
          pf.gev.push_back(e);
        }
      c.pcg_graph_mask = pf.mask;
      FD_CUDA(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
      pf.capturing = true;
      fetidp_status cap = FETIDP_OK;
      for (int half = 0; half < 2 && cap == FETIDP_OK; ++half) {
        const int rz = half == 0 ? S_RZ0 : S_RZ1, rzn = half == 0 ? S_RZ1 : S_RZ0;
        cap = op_apply_F(c, P, L, Q, L);
        if (cap == FETIDP_OK) cap = k_dot(c, P, L, Q, L, L, m, sc + S_PQ * m);
        if (cap == FETIDP_OK) {
          pcg_xr_kernel<<<gridn(mL), 256, 0, c.stream>>>(X, R, P, Q, sc, rz, L, m);
          count_launch();
          cap = k_dot(c, R, L, R, L, L, m, sc + S_RR * m);
        }
        if (cap == FETIDP_OK) {
          pcg_check_kernel<<<1, 32, 0, c.stream>>>(sc, m, tol);
          count_launch();
          cap = op_apply_MD(c, R, L, Zv, L);
        }
        if (cap == FETIDP_OK) cap = k_dot(c, R, L, Zv, L, L, m, sc + rzn * m);
        if (cap == FETIDP_OK) {
          pcg_p_kernel<<<gridn(mL), 256, 0, c.stream>>>(P, Zv, sc, rzn, rz, L, m);
          count_launch();
        }
      }
      cudaGraph_t graph = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(c.stream, &graph);
      pf.capturing = false;
      // captured kernels have not run: they are counted when the graph is replayed
      c.pcg_graph_kernels = g_launches.load() - l0;
      g_launches.fetch_sub(c.pcg_graph_kernels);
      cudaError_t ie = cudaErrorUnknown;
      if (cap == FETIDP_OK && ce == cudaSuccess) ie = cudaGraphInstantiate(&c.pcg_graph, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (ie != cudaSuccess) {   // capture not possible here: run the iterations one by one
        cudaGetLastError();
        c.pcg_graph = nullptr;
        c.pcg_graph_failed = true;
        pf.captured.clear();
      }
    }
  }
  if (graph_ok && c.pcg_graph) {
    // counters and error flags start at zero, active flags are set above
    FD_CUDA(cudaMemsetAsync(sc + S_ERR * m, 0, sizeof(double) * 2 * m, c.stream));
    while (true) {
      FD_CUDA(cudaGraphLaunch(c.pcg_graph, c.stream));
      g_launches.fetch_add(c.pcg_graph_kernels);
      c.graph_kernels_run += c.pcg_graph_kernels;
      ++c.graph_replays;
      FD_CUDA(cudaMemcpyAsync(hs, sc, sizeof(double) * S_NSLOT * m, cudaMemcpyDeviceToHost, c.stream));
      FD_CUDA(cudaStreamSynchronize(c.stream));
      for (const Prof::Captured& g : c.prof.captured) {
        c.prof.launches[g.cls] += 1;
        float v = 0.f;
        if (cudaEventElapsedTime(&v, g.e0, g.e1) != cudaSuccess) { cudaGetLastError(); continue; }
        c.prof.ms[g.cls] += v;
        c.prof.flops[g.cls] += g.flops;
        c.prof.bytes[g.cls] += g.bytes;
      }
      nact = 0;
      it = 0;
      for (int r = 0; r < m; ++r) {
        if (hs[S_ERR * m + r] != 0.0) {
          set_error("PCG breakdown: p^T F p <= 0 or non-finite residual");
          return FETIDP_EBREAKDOWN;
        }
        nact += hs[S_ACT * m + r] != 0.0;
        it = std::max(it, (int)hs[S_ITS * m + r]);
      }
      if (nact == 0 || it >= max_it) break;
    }
    c.inner_total += it;
    FD_TRY(k_copy_scale(c, X, x, L, m, L, x_rs, nullptr, 1.0));
    return FETIDP_OK;
  }
  while (nact > 0 && it < max_it) {
    FD_TRY(op_apply_F(c, P, L, Q, L));
    FD_TRY(k_dot(c, P, L, Q, L, L, m, sc + S_PQ * m));
    pcg_xr_kernel<<<gridn(mL), 256, 0, c.stream>>>(X, R, P, Q, sc, cur, L, m);
    FD_CHECK_LAUNCH();
    FD_TRY(k_dot(c, R, L, R, L, L, m, sc + S_RR * m));
    FD_CUDA(cudaMemcpyAsync(hs, sc, sizeof(double) * S_NSLOT * m, cudaMemcpyDeviceToHost, c.stream));
    FD_CUDA(cudaStreamSynchronize(c.stream));
    ++it;
    nact = 0;
    for (int r = 0; r < m; ++r) {
      if (act[r] == 0.0) continue;
      const double pq = hs[S_PQ * m + r], rr = hs[S_RR * m + r];
      if (!(pq > 0.0) || !std::isfinite(rr)) {
        set_error("PCG breakdown: p^T F p <= 0 or non-finite residual");
        return FETIDP_EBREAKDOWN;
      }
      const double rel = std::sqrt(rr / rr0[r]);
      const double tol = c.mixed ? c.opt.tol_inner_mixed : c.opt.tol_inner;
      if (c.opt.fixed_inner <= 0 && rel <= tol) act[r] = 0.0;
      if (rr == 0.0) act[r] = 0.0;
      nact += act[r] > 0.0;
    }
    if (nact == 0 || it >= max_it) break;
    FD_CUDA(cudaMemcpyAsync(sc + S_ACT * m, act.data(), sizeof(double) * m, cudaMemcpyHostToDevice, c.stream));
    FD_TRY(op_apply_MD(c, R, L, Zv, L));
    const int nxt = cur == S_RZ0 ? S_RZ1 : S_RZ0;
    FD_TRY(k_dot(c, R, L, Zv, L, L, m, sc + nxt * m));
    pcg_p_kernel<<<gridn(mL), 256, 0, c.stream>>>(P, Zv, sc, nxt, cur, L, m);
    FD_CHECK_LAUNCH();
    cur = nxt;
  }
  c.inner_total += it;
  FD_TRY(k_copy_scale(c, X, x, L, m, L, x_rs, nullptr, 1.0));
  return FETIDP_OK;
}

// ------------------------------------------------------------------ Eq. 16 operator
fetidp_status op_apply_A(Ctx& c, const double* x, double* y) {
  const int m = c.m, n = c.n, nr = c.nr, ni = c.ni;
  const long long nt = c.ntot, NR = c.N * nr;
  CellVec ua{c.w_cell_a, c.N * n, n}, ub{c.w_cell_b, c.N * n, n};
  FD_TRY(copy_cells(c, CCellVec{x, nt, nr}, ua, nr, m));
  FD_TRY(k_primal_extract(c, x + NR, nt, CellVec{c.w_cell_a + nr, c.N * n, n}, m));
  FD_TRY(k_apply_K(c, cview(ua), ub, 1, m, true, false, c.snap, 0.0));
  FD_TRY(copy_cells(c, cview(ub), CellVec{y, nt, nr}, nr, m));
  FD_TRY(k_gather_BT(c, x + NR + c.nP, nt, nullptr, CellVec{y + ni, nt, nr}, m, 1.0));
  FD_TRY(k_primal_assemble(c, CCellVec{c.w_cell_b + nr, c.N * n, n}, y + NR, nt, 1.0, 0.0, m));
  FD_TRY(k_scatter_B(c, CCellVec{x + ni, nt, nr}, y + NR + c.nP, nt, nullptr, 1.0, 0.0, m));
  return FETIDP_OK;
}

// ------------------------------------------------------------------ Algorithm 1 (Eq. 44)
fetidp_status op_precondition(Ctx& c, const double* x, double* y) {
  const int m = c.m, nd = c.nd, np = c.np, nr = c.nr, ni = c.ni;
  const long long nt = c.ntot, NR = c.N * nr;
  CCellVec vR{x, nt, nr};
  const double* vP = x + NR;
  const double* w = x + NR + c.nP;
  CellVec yR{y, nt, nr};
  double* yP = y + NR;
  double* yL = y + NR + c.nP;
  double* pcg_b = c.pcg + 5LL * m * c.L;
  // w_bar = w - U_ring v  (Algorithm 3; keeps z_P = x_P of Algorithm 2 in w_zP)
  FD_TRY(U_apply(c, vR, vP, nt, c.w_L1, c.L));
  FD_TRY(axpby(c, w, nt, c.w_L1, c.L, pcg_b, c.L, 1.0, -1.0, c.L, m));
  // y = -F_ring^{-pcg} w_bar, or y = -M_D^{-ROM} w_bar (Eq. 47)
  if (c.opt.interface == 1)
    FD_TRY(op_apply_MD_rom(c, pcg_b, c.L, yL, nt));
  else
    FD_TRY(pcg_solve(c, pcg_b, c.L, yL, nt));
  FD_TRY(k_copy_scale(c, yL, yL, c.L, m, nt, nt, nullptr, -1.0));
  // x = K_ring^{-ROM} v - U_ring^T y   (Algorithm 2 with Eq. 46)
  FD_TRY(local_rom(c, vR, yR));
  CellVec cp{c.w_p1, c.N * np, np};
  FD_TRY(k_primal_extract(c, c.w_zP, c.nP, cp, m));
  FD_TRY(cell_op(c, c.Urp_c, (long long)nr * np, np, nr, np, cview(cp), yR, -1.0, 1.0));
  // U_ring^T y = (U_RD B_R^T y - U_RP z'_P, z'_P), z'_P = S_PP^{-1}(-U_RP^T B_R^T y)
  CellVec g{c.w_d1, c.N * nd, nd};
  FD_TRY(k_gather_BT(c, yL, nt, nullptr, g, m, 0.0));
  FD_TRY(cell_op(c, c.UrpT_c + ni, (long long)np * nr, nr, np, nd, cview(g), cp, 1.0, 0.0));
  FD_TRY(k_primal_assemble(c, cview(cp), c.w_P1, c.nP, -1.0, 0.0, m));
  FD_TRY(coarse_solve(c, c.w_P1, c.nP, c.w_P1, c.nP, m));
  if (c.exact)   // columns d of each cell's own K_rr^{-1}
    FD_TRY(cell_op(c, c.Kinv + ni, (long long)nr * nr, nr, nr, nd, cview(g), yR, -1.0, 1.0));
  else if (c.Uid_f) {   // assembled FP32 blocks: y_i -= U_id g, y_d -= F_dd g
    FD_TRY(k_cell_gemm_f32(c, c.Udi_f, c.ld_di, ni, nd, cview(g), yR, -1.0, 1.0, m));
    const CellVec yd{yR.p + ni, yR.rs, yR.cs};
    if (c.sym_T)
      FD_TRY(k_cell_symv_f32(c, c.Fdd_f, cview(g), yd, -1.0, 1.0, m));
    else
      FD_TRY(k_cell_gemm_f32(c, c.Fdd_f, c.ld_f, nd, nd, cview(g), yd, -1.0, 1.0, m));
  } else if (c.mixed)
    FD_TRY(tc_comb_apply(c, c.cUrd, cview(g), c.delta, c.delta, yR.p, true, yR.rs, yR.cs, -1.0, 1.0, m, c.N));
  else
    FD_TRY(k_grouped_gemm(c, c.Kinv + ni, (long long)nr * nr, nr, nr, nd, cview(g), yR, c.delta, -1.0,
                          1.0, m, false, 0));
  FD_TRY(k_primal_extract(c, c.w_P1, c.nP, cp, m));
  FD_TRY(cell_op(c, c.Urp_c, (long long)nr * np, np, nr, np, cview(cp), yR, 1.0, 1.0));
  FD_TRY(axpby(c, c.w_zP, c.nP, c.w_P1, c.nP, yP, nt, 1.0, -1.0, c.nP, m));
  return FETIDP_OK;
}

// ------------------------------------------------------------------ outer FGMRES
struct OuterResult {
  int its = 0;
  double rel_res = 0.0;
  bool converged = false;
};

// Restarted flexible GMRES: each cycle runs the Arnoldi process on the current residual;
// after a cycle the true residual b - A x is recomputed and the solver restarts from x
// while it is above tol_outer (the least-squares estimate and the true residual drift
// apart when the preconditioner changes between applications).
fetidp_status fgmres(Ctx& c, double* xout, OuterResult& res) {
  const int m = c.m, mo = c.kry;      // cycle length = Krylov storage
  const long long nt = c.ntot, mnt = (long long)m * nt;
  const bool fixed = c.opt.fixed_outer > 0;
  const int max_total = fixed ? c.opt.fixed_outer : c.opt.max_outer;
  double* dots1 = c.scal + 64 * m;
  double* dots2 = dots1 + (size_t)m * (mo + 2);
  double* rcur = c.w_tot + mnt;        // residual of the current cycle
  double* rbuf = c.w_tot + 2 * mnt;    // A x
  std::vector<double> hbuf((size_t)m * (mo + 2));
  FD_TRY(k_dot(c, c.rhs, nt, c.rhs, nt, nt, m, dots1));
  FD_CUDA(cudaMemcpyAsync(hbuf.data(), dots1, sizeof(double) * m, cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  std::vector<double> bnorm(m), rnorm(m), inv(m);
  for (int r = 0; r < m; ++r) bnorm[r] = std::sqrt(hbuf[r]);
  FD_CUDA(cudaMemsetAsync(xout, 0, sizeof(double) * mnt, c.stream));
  FD_CUDA(cudaMemcpyAsync(rcur, c.rhs, sizeof(double) * mnt, cudaMemcpyDeviceToDevice, c.stream));
  rnorm = bnorm;
  int total_its = 0;
  res.converged = false;
  std::vector<std::vector<double>> H(m, std::vector<double>((size_t)(mo + 1) * mo, 0.0));
  std::vector<std::vector<double>> g(m, std::vector<double>(mo + 1, 0.0)), cs(m, std::vector<double>(mo)),
      sn(m, std::vector<double>(mo));
  auto Hij = [&](int r, int i, int j) -> double& { return H[r][(size_t)i * mo + j]; };
  while (total_its < max_total) {
    std::vector<char> active(m, 0);
    std::vector<double> target(m, 0.0);
    int nact = 0;
    for (int r = 0; r < m; ++r) {
      // batch: every lattice b must reach tol against its own load; ||r|| <= tol min_b ||f_b||
      // guarantees ||r_b|| <= tol ||f_b|| for all b (tol_scale = min_b ||f_b|| / ||f||, 1 alone)
      const double tol_r = c.opt.tol_outer * c.tol_scale[r];
      const bool done = bnorm[r] == 0.0 || rnorm[r] == 0.0 || (!fixed && rnorm[r] <= tol_r * bnorm[r]);
      active[r] = !done;
      target[r] = tol_r * bnorm[r] / std::max(rnorm[r], 1e-300);
      inv[r] = active[r] ? 1.0 / rnorm[r] : 0.0;
      nact += active[r];
      std::fill(H[r].begin(), H[r].end(), 0.0);
      std::fill(g[r].begin(), g[r].end(), 0.0);
      g[r][0] = rnorm[r];
    }
    if (nact == 0) { res.converged = true; break; }
    FD_CUDA(cudaMemcpyAsync(dots2, inv.data(), sizeof(double) * m, cudaMemcpyHostToDevice, c.stream));
    FD_TRY(k_copy_scale(c, rcur, c.V, nt, m, nt, nt, dots2, 0.0));
    std::vector<int> k_used(m, 0);
    std::vector<char> live = active;
    int j = 0;
    for (j = 0; j < mo && nact > 0 && total_its < max_total; ++j) {
      double* Vj = c.V + (size_t)j * mnt;
      double* Zj = c.Z + (size_t)j * mnt;
      double* w = c.V + (size_t)(j + 1) * mnt;
      FD_TRY(op_precondition(c, Vj, Zj));
      FD_TRY(op_apply_A(c, Zj, w));
      // classical Gram-Schmidt with one reorthogonalisation
      FD_TRY(k_multi_dot(c, c.V, mnt, j + 1, w, nt, m, dots1));
      FD_TRY(k_multi_axpy(c, c.V, mnt, j + 1, dots1, w, nt, m, -1.0));
      FD_TRY(k_multi_dot(c, c.V, mnt, j + 1, w, nt, m, dots2));
      FD_TRY(k_multi_axpy(c, c.V, mnt, j + 1, dots2, w, nt, m, -1.0));
      std::vector<double> h1((size_t)m * (j + 1)), h2((size_t)m * (j + 1));
      FD_CUDA(cudaMemcpyAsync(h1.data(), dots1, sizeof(double) * h1.size(), cudaMemcpyDeviceToHost, c.stream));
      FD_CUDA(cudaMemcpyAsync(h2.data(), dots2, sizeof(double) * h2.size(), cudaMemcpyDeviceToHost, c.stream));
      FD_TRY(k_dot(c, w, nt, w, nt, nt, m, dots1));
      FD_CUDA(cudaMemcpyAsync(hbuf.data(), dots1, sizeof(double) * m, cudaMemcpyDeviceToHost, c.stream));
      FD_CUDA(cudaStreamSynchronize(c.stream));
      ++total_its;
      for (int r = 0; r < m; ++r) {
        inv[r] = 0.0;
        if (!live[r]) continue;
        const double hn = std::sqrt(hbuf[r]);
        for (int i = 0; i <= j; ++i) Hij(r, i, j) = h1[(size_t)r * (j + 1) + i] + h2[(size_t)r * (j + 1) + i];
        Hij(r, j + 1, j) = hn;
        for (int i = 0; i < j; ++i) {
          const double a = Hij(r, i, j), b = Hij(r, i + 1, j);
          Hij(r, i, j) = cs[r][i] * a + sn[r][i] * b;
          Hij(r, i + 1, j) = -sn[r][i] * a + cs[r][i] * b;
        }
        const double rho = std::hypot(Hij(r, j, j), Hij(r, j + 1, j));
        if (!(rho > 0.0) || !std::isfinite(rho)) {
          set_error("FGMRES breakdown");
          return FETIDP_EBREAKDOWN;
        }
        cs[r][j] = Hij(r, j, j) / rho;
        sn[r][j] = Hij(r, j + 1, j) / rho;
        Hij(r, j, j) = rho;
        Hij(r, j + 1, j) = 0.0;
        g[r][j + 1] = -sn[r][j] * g[r][j];
        g[r][j] = cs[r][j] * g[r][j];
        k_used[r] = j + 1;
        const double est = std::fabs(g[r][j + 1]) / rnorm[r];
        if ((!fixed && est <= target[r]) || hn == 0.0 || (fixed && j + 1 >= c.opt.fixed_outer))
          live[r] = 0;
        inv[r] = (live[r] && hn > 0.0) ? 1.0 / hn : 0.0;
      }
      nact = 0;
      for (int r = 0; r < m; ++r) nact += live[r];
      if (nact > 0) {
        FD_CUDA(cudaMemcpyAsync(dots2, inv.data(), sizeof(double) * m, cudaMemcpyHostToDevice, c.stream));
        FD_TRY(k_copy_scale(c, w, w, nt, m, nt, nt, dots2, 0.0));
      }
    }
    // x += sum_i y_i Z_i with y from the triangular least-squares system
    int kmax = 0;
    for (int r = 0; r < m; ++r) kmax = std::max(kmax, k_used[r]);
    if (kmax > 0) {
      std::vector<double> coef((size_t)m * kmax, 0.0);
      for (int r = 0; r < m; ++r) {
        const int k = k_used[r];
        std::vector<double> yv(k, 0.0);
        for (int i = k - 1; i >= 0; --i) {
          double sacc = g[r][i];
          for (int q = i + 1; q < k; ++q) sacc -= Hij(r, i, q) * yv[q];
          yv[i] = sacc / Hij(r, i, i);
        }
        for (int i = 0; i < k; ++i) coef[(size_t)r * kmax + i] = yv[i];
      }
      FD_CUDA(cudaMemcpyAsync(dots1, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, c.stream));
      FD_TRY(k_multi_axpy(c, c.Z, mnt, kmax, dots1, xout, nt, m, 1.0));
    }
    // true residual
    FD_TRY(op_apply_A(c, xout, rbuf));
    FD_TRY(axpby(c, c.rhs, nt, rbuf, nt, rcur, nt, 1.0, -1.0, nt, m));
    FD_TRY(k_dot(c, rcur, nt, rcur, nt, nt, m, dots1));
    FD_CUDA(cudaMemcpyAsync(hbuf.data(), dots1, sizeof(double) * m, cudaMemcpyDeviceToHost, c.stream));
    FD_CUDA(cudaStreamSynchronize(c.stream));
    for (int r = 0; r < m; ++r) rnorm[r] = std::sqrt(hbuf[r]);
    if (fixed) { res.converged = true; break; }
  }
  res.rel_res = 0.0;
  bool conv = true;
  for (int r = 0; r < m; ++r) {
    // ||r|| / min_b ||f_b||: the combined relative residual alone, an upper bound of the worst
    // lattice's relative residual in a batch
    const double rr = bnorm[r] > 0.0 ? rnorm[r] / (bnorm[r] * c.tol_scale[r]) : 0.0;
    res.rel_res = std::max(res.rel_res, rr);
    if (!fixed && rr > c.opt.tol_outer) conv = false;
  }
  res.converged = fixed ? true : conv;
  res.its = total_its;
  return FETIDP_OK;
}

// u_out natural [m][N][n] from an outer vector x [m][ntot]
fetidp_status to_cells_natural(Ctx& c, const double* x, double* u_out) {
  const int m = c.m, n = c.n, nr = c.nr;
  CellVec ua{c.w_cell_a, c.N * n, n};
  FD_TRY(copy_cells(c, CCellVec{x, c.ntot, nr}, ua, nr, m));
  FD_TRY(k_primal_extract(c, x + c.N * nr, c.ntot, CellVec{c.w_cell_a + nr, c.N * n, n}, m));
  permute_out_kernel<<<gridn(c.N * n * m), 256, 0, c.stream>>>(c.perm, c.w_cell_a, u_out, n, c.N, m);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

}  // namespace fetidp

// ======================================================================== C ABI
using namespace fetidp;

struct fetidp_ctx {
  Ctx c;
};

static fetidp_status enter(fetidp_ctx* ctx) {
  if (!ctx) { set_error("null context"); return FETIDP_EINVAL; }
  cudaError_t e = cudaSetDevice(ctx->c.device);
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return FETIDP_ECUDA; }
  return FETIDP_OK;
}

// Input validation of the vector entry points (option check_inputs): null pointers, then NaN/Inf
// in each input of n doubles.  Synchronises the stream.
struct InVec { const double* p; long long n; const char* name; };
static fetidp_status check_inputs(Ctx& c, std::initializer_list<InVec> ins, const void* out) {
  for (const InVec& v : ins)
    if (!v.p) { set_error(std::string("null input ") + v.name); return FETIDP_EINVAL; }
  if (!out) { set_error("null output"); return FETIDP_EINVAL; }
  if (!c.opt.check_inputs) return FETIDP_OK;
  for (const InVec& v : ins) {
    FD_CUDA(cudaMemsetAsync(c.chk, 0, sizeof(int), c.stream));
    FD_TRY(k_nonfinite(c, v.p, v.n, c.chk));
    int h = 0;
    FD_CUDA(cudaMemcpyAsync(&h, c.chk, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    FD_CUDA(cudaStreamSynchronize(c.stream));
    if (h) { set_error(std::string("non-finite value in ") + v.name); return FETIDP_EINVAL; }
  }
  return FETIDP_OK;
}

// After a call that ran tensor-core kernels: an expired device wait gives ETIMEOUT (the flag is
// cleared, so the context stays usable).  Only with check_inputs, which already synchronises.
static fetidp_status check_waits(Ctx& c, fetidp_status st) {
  if (!c.mixed || !c.tc_err || !c.opt.check_inputs) return st;
  int h = 0;
  FD_CUDA(cudaMemcpyAsync(&h, c.tc_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  if (h) {
    FD_CUDA(cudaMemsetAsync(c.tc_err, 0, sizeof(int), c.stream));
    set_error("a device wait (tensor-core pipeline or coarse-solve barrier) exceeded wait_budget_ns (code " + std::to_string(h) + ")");
    return FETIDP_ETIMEOUT;
  }
  return st;
}

extern "C" {

void fetidp_default_options(fetidp_options* o) {
  if (!o) return;
  o->tol_outer = 1e-8;
  o->tol_inner = 1e-11;
  o->max_outer = 100;
  o->max_inner = 1000;
  o->precision = FETIDP_FP64;
  o->fixed_outer = 0;
  o->fixed_inner = 0;
  o->tc_split = 3;
  o->tol_inner_mixed = 1e-6;
  o->gram_drop_mixed = 1e-9;
  o->profile_mask = 0;
  o->restart = 0;
  o->wait_budget_ns = 1000000000LL;
  o->check_inputs = 1;
  o->mixed_assembled = -1;
  o->interface = 0;
  o->method = 0;
  o->tc_bn = 0;
}

const char* fetidp_status_string(fetidp_status s) {
  switch (s) {
    case FETIDP_OK: return "ok";
    case FETIDP_EINVAL: return "invalid argument";
    case FETIDP_ENOMEM: return "out of memory";
    case FETIDP_ECUDA: return "CUDA error";
    case FETIDP_ENOTCONV: return "not converged";
    case FETIDP_ETIMEOUT: return "device wait timed out";
    case FETIDP_ESINGULAR: return "singular (not SPD)";
    case FETIDP_EBREAKDOWN: return "Krylov breakdown";
  }
  return "unknown status";
}

const char* fetidp_last_error(void) { return g_last_error.c_str(); }

long long fetidp_kernel_launches(void) { return g_launches.load(); }

fetidp_status fetidp_tc_comb_selfcheck(int M0, int M1, int K, int N, int nops, double* rel_err) {
  if (M0 < 1 || M1 < 0 || K < 1 || N < 1 || nops < 1 || !rel_err) {
    set_error("bad self-check sizes");
    return FETIDP_EINVAL;
  }
  fetidp_ctx tmp;
  Ctx& c = tmp.c;
  cudaGetDevice(&c.device);
  c.stream = nullptr;
  fetidp_status st = dalloc(c, reinterpret_cast<void**>(&c.tc_err), sizeof(int));
  if (st == FETIDP_OK) {
    cudaMemset(c.tc_err, 0, sizeof(int));
    st = tc_comb_selfcheck(c, M0, M1, K, N, nops, rel_err);
  }
  for (void* p : c.allocations) cudaFreeAsync(p, c.stream);
  cudaStreamSynchronize(nullptr);
  c.allocations.clear();
  return st;
}

fetidp_status fetidp_tc_selfcheck(int M, int K, int N, double* rel_err) {
  if (M < 1 || K < 1 || N < 1 || !rel_err) { set_error("bad self-check sizes"); return FETIDP_EINVAL; }
  fetidp_ctx tmp;
  Ctx& c = tmp.c;
  cudaGetDevice(&c.device);
  c.stream = nullptr;
  const int m_tiles = (M + 127) / 128, k_tiles = (K + 63) / 64;
  const int bn = tc_bn_for(N, m_tiles, 1);
  const long long n_tiles = (N + bn - 1) / bn;
  c.tc_bbuf_bytes = (size_t)n_tiles * k_tiles * bn * 64 * 2;
  fetidp_status st = dalloc(c, reinterpret_cast<void**>(&c.tc_bbuf), c.tc_bbuf_bytes);
  if (st == FETIDP_OK) st = dalloc(c, reinterpret_cast<void**>(&c.tc_err), sizeof(int));
  if (st == FETIDP_OK) {
    cudaMemset(c.tc_err, 0, sizeof(int));
    st = tc_selfcheck(c, M, K, N, rel_err);
  }
  for (void* p : c.allocations) cudaFreeAsync(p, c.stream);
  cudaStreamSynchronize(nullptr);
  c.allocations.clear();
  return st;
}

fetidp_status fetidp_tc_selfcheck_static(int M, int K, int N, double* rel_err, void* stream) {
  if (M < 1 || K < 1 || N < 1 || !rel_err) { set_error("bad self-check sizes"); return FETIDP_EINVAL; }
  // the size check needs no device: an oversized request fails before any CUDA call
  const size_t need = tc_selfcheck_static_bytes(M, K, N);
  if (need > (size_t)FETIDP_TC_STATIC_SCRATCH_BYTES) {
    set_error("tensor-core probe M=" + std::to_string(M) + " K=" + std::to_string(K) + " N=" +
              std::to_string(N) + " needs " + std::to_string(need) + " bytes of scratch; the static scratch holds " +
              std::to_string((size_t)FETIDP_TC_STATIC_SCRATCH_BYTES) + " (fetidp_tc_selfcheck takes any size)");
    return FETIDP_EINVAL;
  }
  fetidp_ctx tmp;
  Ctx& c = tmp.c;
  FD_CUDA(cudaGetDevice(&c.device));
  c.stream = static_cast<cudaStream_t>(stream);
  return tc_selfcheck_static(c, M, K, N, rel_err);
}

fetidp_status fetidp_tc_time(fetidp_ctx* ctx, int bn, int reps, double* ms) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  if (!ms || reps < 1 || (bn != 64 && bn != 128 && bn != 256)) {
    set_error("fetidp_tc_time: bn must be 64, 128 or 256, reps >= 1, ms non-null");
    return FETIDP_EINVAL;
  }
  if (!c.mixed || c.exact || !c.opKinv.tiles) {
    set_error("fetidp_tc_time: a mixed-precision ROM context is required");
    return FETIDP_EINVAL;
  }
  // the Eq. 46a GEMM of the local ROM solve, on zeroed workspace columns, into the bases' buffer
  const int m = c.m, nr = c.nr, nrb = c.nrb;
  const long long rs = c.N * nrb * nr;
  float* Rf = reinterpret_cast<float*>(c.w_R);
  FD_CUDA(cudaMemsetAsync(c.w_cell_a, 0, sizeof(double) * (size_t)m * c.N * nr, c.stream));
  const CCellVec vR{c.w_cell_a, c.N * nr, nr};
  const int saved = c.opt.tc_bn;
  c.opt.tc_bn = bn;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  fetidp_status st = FETIDP_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_error("fetidp_tc_time: event creation failed");
    st = FETIDP_ECUDA;
  }
  if (st == FETIDP_OK) st = tc_apply(c, c.opKinv, vR, nullptr, Rf, false, rs, nrb * nr, nr, 1.0, 0.0, m, c.N, m * rs);
  if (st == FETIDP_OK && cudaEventRecord(e0, c.stream) != cudaSuccess) st = FETIDP_ECUDA;
  for (int r = 0; r < reps && st == FETIDP_OK; ++r)
    st = tc_apply(c, c.opKinv, vR, nullptr, Rf, false, rs, nrb * nr, nr, 1.0, 0.0, m, c.N, m * rs);
  if (st == FETIDP_OK && cudaEventRecord(e1, c.stream) != cudaSuccess) st = FETIDP_ECUDA;
  c.opt.tc_bn = saved;
  if (st == FETIDP_OK && cudaEventSynchronize(e1) != cudaSuccess) st = FETIDP_ECUDA;
  float t = 0.f;
  if (st == FETIDP_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) st = FETIDP_ECUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st == FETIDP_ECUDA) set_error("fetidp_tc_time: CUDA event failure");
  FD_TRY(st);
  *ms = t / reps;
  return check_waits(c, FETIDP_OK);
}

fetidp_status fetidp_wait_selfcheck(long long wait_budget_ns, void* stream, double* waited_s) {
  if (wait_budget_ns <= 0 || wait_budget_ns > 10000000000LL) {
    set_error("wait_budget_ns must lie in (0, 1e10]");
    return FETIDP_EINVAL;
  }
  const auto t0 = std::chrono::steady_clock::now();
  const fetidp_status st = wait_selfcheck((unsigned long long)wait_budget_ns, static_cast<cudaStream_t>(stream));
  if (waited_s) *waited_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

static fetidp_status profile_enable(Ctx& c, unsigned mask) {
  Prof& P = c.prof;
  P.mask = mask;
  P.used = 0;
  for (int k = 0; k < FETIDP_K_NCLASS; ++k) { P.flops[k] = 0; P.bytes[k] = 0; P.launches[k] = 0; P.ms[k] = 0; }
  return FETIDP_OK;
}

fetidp_status fetidp_profile_enable(fetidp_ctx* ctx, unsigned mask) {
  FD_TRY(enter(ctx));
  FD_CUDA(cudaStreamSynchronize(ctx->c.stream));
  return profile_enable(ctx->c, mask);
}

fetidp_status fetidp_profile_read(fetidp_ctx* ctx, double* ms, long long* launches, double* flops,
                                  double* bytes) {
  FD_TRY(enter(ctx));
  Prof& P = ctx->c.prof;
  FD_CUDA(cudaStreamSynchronize(ctx->c.stream));
  double t[FETIDP_K_NCLASS] = {};
  for (int k = 0; k < FETIDP_K_NCLASS; ++k) t[k] = P.ms[k];
  for (int i = 0; i < P.used; ++i) {
    float v = 0.f;
    FD_CUDA(cudaEventElapsedTime(&v, P.ev[2 * i], P.ev[2 * i + 1]));
    t[P.cls[i]] += v;
  }
  for (int k = 0; k < FETIDP_K_NCLASS; ++k) {
    if (ms) ms[k] = t[k];
    if (launches) launches[k] = P.launches[k];
    if (flops) flops[k] = P.flops[k];
    if (bytes) bytes[k] = P.bytes[k];
    P.flops[k] = 0; P.bytes[k] = 0; P.launches[k] = 0; P.ms[k] = 0;
  }
  P.used = 0;
  return FETIDP_OK;
}

void fetidp_destroy(fetidp_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->c.device);
  cudaStreamSynchronize(ctx->c.stream);
  if (ctx->c.pcg_graph) cudaGraphExecDestroy(ctx->c.pcg_graph);
  for (auto& e : ctx->c.prof.ev) event_give(ctx->c.device, e);
  for (auto& e : ctx->c.prof.gev) event_give(ctx->c.device, e);
  if (ctx->c.ws) {
    cudaStreamSynchronize(ctx->c.ws);
    cudaStreamDestroy(ctx->c.ws);
    cudaEventDestroy(ctx->c.ev_in);
    cudaEventDestroy(ctx->c.ev_out);
  }
  for (void* p : ctx->c.allocations) cudaFreeAsync(p, ctx->c.stream);
  cudaStreamSynchronize(ctx->c.stream);
  if (ctx->c.h_scal) cudaFreeHost(ctx->c.h_scal);
  delete ctx;
}

fetidp_status fetidp_setup(const fetidp_problem* probs, int n_problems, const fetidp_options* opt,
                           void* cuda_stream, fetidp_ctx** out) {
  if (!out) { set_error("null output pointer"); return FETIDP_EINVAL; }
  *out = nullptr;
  if (!probs || n_problems < 1) {
    set_error("at least one problem per context");
    return FETIDP_EINVAL;
  }
  fetidp_options o;
  fetidp_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != FETIDP_FP64 && o.precision != FETIDP_MIXED_BF16) {
    set_error("unknown precision");
    return FETIDP_EINVAL;
  }
  fetidp_ctx* ctx = new fetidp_ctx();
  cudaGetDevice(&ctx->c.device);
  ctx->c.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  fetidp_status s = o.profile_mask ? profile_enable(ctx->c, o.profile_mask) : FETIDP_OK;
  if (s == FETIDP_OK) s = setup_context(ctx->c, probs, n_problems, o);
  if (s != FETIDP_OK) {
    fetidp_destroy(ctx);
    return s;
  }
  *out = ctx;
  return FETIDP_OK;
}

fetidp_status fetidp_batch_layout(const fetidp_ctx* ctx, long long* cell0, long long* L0, long long* P0) {
  if (!ctx) { set_error("null argument"); return FETIDP_EINVAL; }
  const Ctx& c = ctx->c;
  const size_t B = c.lat.size();
  for (size_t b = 0; b <= B; ++b) {
    const bool end = b == B;
    if (cell0) cell0[b] = end ? c.N : c.lat[b].cell0;
    if (L0) L0[b] = end ? c.L : c.lat[b].L0;
    if (P0) P0[b] = end ? c.nP : c.lat[b].V0 * c.d;
  }
  return FETIDP_OK;
}

fetidp_status fetidp_sizes(const fetidp_ctx* ctx, long long o[12]) {
  if (!ctx || !o) { set_error("null argument"); return FETIDP_EINVAL; }
  const Ctx& c = ctx->c;
  o[0] = c.N; o[1] = c.n; o[2] = c.ni; o[3] = c.nd; o[4] = c.np; o[5] = c.nr;
  o[6] = c.L; o[7] = c.nP; o[8] = c.m; o[9] = c.nrb; o[10] = c.nsnap; o[11] = c.ntot;
  return FETIDP_OK;
}

fetidp_status fetidp_apply_F(fetidp_ctx* ctx, const double* lambda, double* y) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  FD_TRY(check_inputs(c, {{lambda, (long long)c.m * c.L, "lambda"}}, y));
  return check_waits(c, op_apply_F(c, lambda, c.L, y, c.L));
}

fetidp_status fetidp_precond(fetidp_ctx* ctx, const double* r, double* z) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  FD_TRY(check_inputs(c, {{r, (long long)c.m * c.L, "r"}}, z));
  return check_waits(c, op_apply_MD(c, r, c.L, z, c.L));
}

fetidp_status fetidp_precond_rom(fetidp_ctx* ctx, const double* r, double* z) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  FD_TRY(check_inputs(c, {{r, (long long)c.m * c.L, "r"}}, z));
  return op_apply_MD_rom(c, r, c.L, z, c.L);
}

fetidp_status fetidp_gather_BT(fetidp_ctx* ctx, const double* lambda, double* x_d) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  FD_TRY(check_inputs(c, {{lambda, (long long)c.m * c.L, "lambda"}}, x_d));
  return k_gather_BT(c, lambda, c.L, nullptr, CellVec{x_d, c.N * c.nd, c.nd}, c.m, 0.0);
}

fetidp_status fetidp_scatter_B(fetidp_ctx* ctx, const double* y_d, double* z) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  FD_TRY(check_inputs(c, {{y_d, (long long)c.m * c.N * c.nd, "y_d"}}, z));
  return k_scatter_B(c, CCellVec{y_d, c.N * c.nd, c.nd}, z, c.L, nullptr, 1.0, 0.0, c.m);
}

fetidp_status fetidp_apply_K(fetidp_ctx* ctx, const double* u, double* y) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  FD_TRY(check_inputs(c, {{u, (long long)c.m * c.N * c.n, "u"}}, y));
  return k_apply_K(c, CCellVec{u, c.N * c.n, c.n}, CellVec{y, c.N * c.n, c.n}, 1, c.m, false, false,
                   c.snap, 0.0);
}

fetidp_status fetidp_coarse_solve(fetidp_ctx* ctx, const double* b, double* x) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  FD_TRY(check_inputs(c, {{b, (long long)c.m * c.nP, "b"}}, x));
  return coarse_solve(c, b, c.nP, x, c.nP, c.m);
}

fetidp_status fetidp_local_rom_solve(fetidp_ctx* ctx, const double* v, double* x) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  const long long ext = (long long)c.m * c.N * c.nr;
  FD_TRY(check_inputs(c, {{v, ext, "v"}}, x));
  return check_waits(c, local_rom(c, CCellVec{v, c.N * c.nr, c.nr, ext}, CellVec{x, c.N * c.nr, c.nr, ext}));
}

fetidp_status fetidp_apply_A(fetidp_ctx* ctx, const double* x, double* y) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  FD_TRY(check_inputs(c, {{x, (long long)c.m * c.ntot, "x"}}, y));
  return op_apply_A(c, x, y);
}

fetidp_status fetidp_apply_P(fetidp_ctx* ctx, const double* x, double* y) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  FD_TRY(check_inputs(c, {{x, (long long)c.m * c.ntot, "x"}}, y));
  return check_waits(c, op_precondition(c, x, y));
}

fetidp_status fetidp_rom_data(fetidp_ctx* ctx, int* sigma, double* alpha, double* pi, double* delta) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  if (sigma) std::memcpy(sigma, c.sigma.data(), sizeof(int) * c.nrb);
  const size_t bytes = sizeof(double) * c.N * c.nrb;
  if (c.exact) { set_error("standard FETI-DP has no reduced-order model"); return FETIDP_EINVAL; }
  if (alpha) FD_CUDA(cudaMemcpyAsync(alpha, c.alpha, bytes, cudaMemcpyDeviceToHost, c.stream));
  if (pi) FD_CUDA(cudaMemcpyAsync(pi, c.pi, bytes, cudaMemcpyDeviceToHost, c.stream));
  if (delta) FD_CUDA(cudaMemcpyAsync(delta, c.delta, bytes, cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  return FETIDP_OK;
}

static fetidp_status solve_common(fetidp_ctx* ctx, fetidp_info* info, OuterResult& r) {
  Ctx& c = ctx->c;
  auto t0 = std::chrono::steady_clock::now();
  c.inner_total = 0;
  const long long l0 = g_launches.load(), gk0 = c.graph_kernels_run, gr0 = c.graph_replays;
  if (c.mixed) FD_CUDA(cudaMemsetAsync(c.tc_err, 0, sizeof(int), c.stream));
  const fetidp_status st = fgmres(c, c.w_tot, r);
  FD_CUDA(cudaStreamSynchronize(c.stream));
  if (c.mixed) {
    // an expired device wait explains whatever else went wrong (e.g. a breakdown on the garbage it
    // left behind), so it is reported first; the flag is cleared for the next call
    int herr = 0;
    FD_CUDA(cudaMemcpy(&herr, c.tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr != 0) {
      FD_CUDA(cudaMemsetAsync(c.tc_err, 0, sizeof(int), c.stream));
      FD_CUDA(cudaStreamSynchronize(c.stream));
      set_error("a device wait (tensor-core pipeline or coarse-solve barrier) exceeded wait_budget_ns (code " + std::to_string(herr) + ")");
      return FETIDP_ETIMEOUT;
    }
  }
  FD_TRY(st);
  if (info) {
    info->outer_its = r.its;
    info->inner_its_total = c.inner_total;
    info->n_rb = c.nrb;
    info->rel_residual = r.rel_res;
    info->t_setup_s = c.t_setup_s;
    info->t_solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->device_bytes = c.device_bytes;
    const long long kl = g_launches.load() - l0;
    info->kernel_launches = kl;
    info->host_launches = kl - (c.graph_kernels_run - gk0) + (c.graph_replays - gr0);
    info->inner_graph = c.pcg_graph != nullptr && !c.pcg_graph_failed ? 1 : 0;
  }
  return FETIDP_OK;
}

fetidp_status fetidp_solve(fetidp_ctx* ctx, double* u, double* lambda, fetidp_info* info) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  OuterResult r;
  FD_TRY(solve_common(ctx, info, r));
  if (u) FD_TRY(to_cells_natural(c, c.w_tot, u));
  if (lambda)
    FD_TRY(k_copy_scale(c, c.w_tot + c.N * c.nr + c.nP, lambda, c.L, c.m, c.ntot, c.L, nullptr, 1.0));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  return r.converged ? FETIDP_OK : FETIDP_ENOTCONV;
}

fetidp_status fetidp_solve_host(fetidp_ctx* ctx, double* u_host, double* lambda_host,
                                fetidp_info* info) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  OuterResult r;
  FD_TRY(solve_common(ctx, info, r));
  if (u_host) {
    FD_TRY(to_cells_natural(c, c.w_tot, c.w_cell_b));
    FD_CUDA(cudaMemcpyAsync(u_host, c.w_cell_b, sizeof(double) * c.m * c.N * c.n,
                            cudaMemcpyDeviceToHost, c.stream));
  }
  if (lambda_host)
    for (int q = 0; q < c.m; ++q)
      FD_CUDA(cudaMemcpyAsync(lambda_host + (size_t)q * c.L, c.w_tot + (size_t)q * c.ntot + c.N * c.nr + c.nP,
                              sizeof(double) * c.L, cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  return r.converged ? FETIDP_OK : FETIDP_ENOTCONV;
}

fetidp_status fetidp_compliance(fetidp_ctx* ctx, const double* u, double* c_out) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  FD_TRY(check_inputs(c, {{u, (long long)c.m * c.N * c.n, "u"}}, c_out));
  // scratch: the partial sums and the results live in the reduction workspace
  FD_TRY(k_compliance(c, u, c.red + (size_t)c.m * kReductionBlocks, c.red));
  FD_CUDA(cudaMemcpyAsync(c_out, c.red + (size_t)c.m * kReductionBlocks, sizeof(double) * c.m, cudaMemcpyDefault,
                          c.stream));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  return FETIDP_OK;
}

fetidp_status fetidp_grad(fetidp_ctx* ctx, const double* u, const double* w, double* g) {
  FD_TRY(enter(ctx));
  Ctx& c = ctx->c;
  const long long nu = (long long)c.m * c.N * c.n;
  FD_TRY(check_inputs(c, {{u, nu, "u"}, {w ? w : u, nu, "w"}}, g));
  return k_grad(c, u, w ? w : u, g);
}

}  // extern "C"
