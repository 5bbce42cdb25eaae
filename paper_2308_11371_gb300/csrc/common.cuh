// Internal declarations of the FETI-DP library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fetidp.h"
#include "geometry.cuh"

namespace fetidp {

void set_error(const std::string& msg);
struct Ctx;
// blocks of the deterministic two-stage reductions (2 x 152 SMs)
constexpr int kReductionBlocks = 304;
// stream-ordered temporaries of the setup phase (not tracked by the context)
fetidp_status tmp_alloc(Ctx& c, void** p, size_t bytes);
void tmp_free(Ctx& c, void* p);
void count_launch();

#define FD_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      ::fetidp::set_error(std::string(#call) + ": " + cudaGetErrorString(e_)); \
      return FETIDP_ECUDA;                                                   \
    }                                                                        \
  } while (0)

#define FD_CHECK_LAUNCH()                                                    \
  do {                                                                       \
    ::fetidp::count_launch();                                                \
    cudaError_t e_ = cudaGetLastError();                                     \
    if (e_ != cudaSuccess) {                                                 \
      ::fetidp::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_)); \
      return FETIDP_ECUDA;                                                   \
    }                                                                        \
  } while (0)

#define FD_TRY(expr)                              \
  do {                                            \
    fetidp_status s_ = (expr);                    \
    if (s_ != FETIDP_OK) return s_;               \
  } while (0)

// One Eq. 42 trace table: gradients of two column sets of ncol columns each.
struct TraceTableSpec {
  const double* Gi;
  const double* Gj;
  int ncol;
};
struct TraceTableSpecDF {   // the same rows from gradient float planes (double-float path)
  const float* Gih;
  const float* Gil;
  const float* Gjh;
  const float* Gjl;
  int ncol;
};

// ---------------------------------------------------------------- debug bounds checks
// Built with -DFETIDP_BOUNDS_CHECK, the kernels of the mixed local-ROM chain compare their
// global accesses with the extent of the buffer they touch; a violation is recorded in
// g_fd_violation (kernel code, offending index, extent) and the access is skipped.
struct FdViolation {
  int code;
  long long index;
  long long extent;
};
#ifdef FETIDP_BOUNDS_CHECK
static __device__ FdViolation g_fd_violation;   // one record per translation unit
__device__ __forceinline__ bool fd_in_bounds(long long idx, long long extent, int code) {
  if (extent < 0 || (idx >= 0 && idx < extent)) return true;   // extent < 0: unknown, unchecked
  if (atomicCAS(&g_fd_violation.code, 0, code) == 0) {
    g_fd_violation.index = idx;
    g_fd_violation.extent = extent;
  }
  return false;
}
#define FD_INB(idx, extent, code) fd_in_bounds((long long)(idx), (long long)(extent), (code))
#define FD_CHECKED_BUILD 1
#else
#define FD_INB(idx, extent, code) ((void)(idx), (void)(extent), true)
#define FD_CHECKED_BUILD 0
#endif
// per-translation-unit readers of the violation record (FETIDP_OK in unchecked builds)
fetidp_status fd_check_cell(const char* where);
fetidp_status fd_check_tc(const char* where);
#ifdef FETIDP_BOUNDS_CHECK
#define FD_DEFINE_CHECK(fname)                                                                  \
  fetidp_status fname(const char* where) {                                                       \
    FdViolation h{};                                                                             \
    const cudaError_t se = cudaDeviceSynchronize();                                              \
    if (se != cudaSuccess) {                                                                     \
      set_error(std::string("after ") + where + ": " + cudaGetErrorString(se));                  \
      return FETIDP_ECUDA;                                                                       \
    }                                                                                            \
    cudaMemcpyFromSymbol(&h, g_fd_violation, sizeof(h));                                         \
    if (h.code != 0) {                                                                           \
      FdViolation z{};                                                                           \
      cudaMemcpyToSymbol(g_fd_violation, &z, sizeof(z));                                         \
      set_error(std::string("bounds check in ") + where + ": code " + std::to_string(h.code) +   \
                " index " + std::to_string(h.index) + " extent " + std::to_string(h.extent));    \
      return FETIDP_ECUDA;                                                                       \
    }                                                                                            \
    return FETIDP_OK;                                                                            \
  }
#else
#define FD_DEFINE_CHECK(fname) \
  fetidp_status fname(const char*) { return FETIDP_OK; }
#endif

// Per-cell vector view: element (rhs, cell, i) at p[rhs*rs + cell*cs + i].
struct CellVec {
  double* p;
  long long rs;   // RHS stride
  int cs;         // cell stride
  long long ext = -1;   // elements addressable from p (checked builds; -1 = unknown)
};
struct CCellVec {
  const double* p;
  long long rs;
  int cs;
  long long ext = -1;
};
inline CCellVec cview(const CellVec& v) { return {v.p, v.rs, v.cs, v.ext}; }

// Block cyclic reduction of the block-tridiagonal coarse matrix (slab ordering).
struct CoarseBCR {
  int b = 0;                       // block (slab) size in DOF
  int nb = 0;                      // slabs at level 0
  int levels = 0;                  // reductions until one block remains
  std::vector<int> n_at;           // blocks at level l (levels + 1 entries)
  std::vector<long long> vec_off;  // offset of level l in the per-RHS level vectors
  long long vec_len = 0;           // per-RHS length of all level vectors
  // matrices, FP64 row-major b x b; per level l and odd j:
  //   Ainv_j at mat_off[l][j], U_j (if j+1 < n), U_j^T, V_j, V_j^T
  std::vector<std::vector<long long>> off_Ainv, off_U, off_UT, off_V, off_VT;
  long long off_final = 0;         // Ainv of the last remaining block
  double* mats = nullptr;          // device
  long long* tables = nullptr;     // device offsets: per level A, U, UT, V, VT arrays of n entries
  int* perm = nullptr;             // device [nb*b]: slab-ordered position -> primal DOF
  double* bl = nullptr;            // device [m][vec_len] right-hand sides per level
  double* xl = nullptr;            // device [m][vec_len] solutions per level
  size_t mat_bytes = 0;
  // mixed path: an FP32 copy of the used blocks (compact pool, same per-level table layout) and
  // level vectors [rhs chunk of 8][vec_len][8] for the inner iterations' coarse correction
  float* mats_f = nullptr;
  long long* tables_f = nullptr;
  long long off_final_f = 0;
  float* bl_f = nullptr;
  float* xl_f = nullptr;
  size_t mat_bytes_f = 0;
  unsigned* coop_bar = nullptr;    // grid barrier of the cooperative FP32 solve (arrivals, generation)
  int coop_grid = 0;
};

// A principal-operator set packed for the tensor-core GEMM (BF16, SW128 K-major tiles).
struct TcOperator {
  uint8_t* tiles = nullptr;
  int M = 0, K = 0, nops = 0, nterm = 1;
  bool separate = false;
  int m_tiles = 0, k_tiles_op = 0, k_tiles = 0;
  long long batch_bytes = 0;
};

// Principal-operator set for the fused combine kernel (operator tiles with hi/lo parts; rows
// [0, msplit) combined with coef0, the rest with coef1).
struct TcComb {
  uint8_t* tiles = nullptr;
  int M = 0, msplit = 0, K = 0, nops = 0, nA = 1, nX = 1, m_tiles = 0, kto = 0;
  long long bytes = 0;
};

// Kernel-class profiler: CUDA event pairs on the context stream plus the algorithmic
// FLOP / byte counts of every timed launch.
struct Prof {
  unsigned mask = 0;
  int capacity = 0;
  std::vector<cudaEvent_t> ev;   // 2 * capacity events
  std::vector<int> cls;          // class of each used pair
  int used = 0;
  double flops[FETIDP_K_NCLASS] = {};
  double bytes[FETIDP_K_NCLASS] = {};
  long long launches[FETIDP_K_NCLASS] = {};
  double ms[FETIDP_K_NCLASS] = {};   // time of launches inside replayed graphs (read per replay)
  // Launches captured into a graph: their event pair is recorded by the graph's own event nodes
  // on every replay; the host adds their time after each replay.
  struct Captured { int cls; double flops, bytes; cudaEvent_t e0, e1; };
  bool capturing = false;
  std::vector<Captured> captured;
  std::vector<cudaEvent_t> gev;   // events for captured launches, created before a capture
};

// One lattice of a batch: its geometry and where its cells, multipliers and free vertices sit in
// the concatenated vectors of the context.
struct LatticeSpan {
  Geo geo{};
  long long cell0 = 0, ncell = 0;   // cells [cell0, cell0 + ncell)
  long long L0 = 0, nL = 0;         // multiplier rows
  long long V0 = 0, nV = 0;         // free vertices (primal DOF = vertex * d + component)
  int clamp_axis = 0, clamp_side = 0;
};

struct Ctx {
  Prof prof;
  double prof_pending_flops = 0.0, prof_pending_bytes = 0.0;
  int device = 0;
  cudaStream_t stream = nullptr;
  Geo geo{};
  fetidp_options opt{};
  // sizes
  int d = 0, e = 0, n = 0, ni = 0, nd = 0, np = 0, nr = 0, ncorner = 0;
  int nelem = 0, ngp = 0, nc = 0;
  long long nsnap = 0;
  long long N = 0, L = 0, nP = 0, ntot = 0;
  int m = 0;        // RHS
  int kry = 0;      // FGMRES cycle length (Krylov storage)
  int nrb = 0;      // principal cells selected
  int nV = 0;       // free lattice vertices (all lattices)
  int clamp_axis = 0, clamp_side = 0;
  std::vector<LatticeSpan> lat;   // the lattices of the context (one unless batched)
  cudaGraphExec_t pcg_graph = nullptr;   // two inner PCG iterations, captured on first use
  long long pcg_graph_kernels = 0;       // kernels in that graph
  bool pcg_graph_failed = false;         // capture not possible: iterations run one by one
  long long graph_replays = 0;           // graph launches issued by the host
  long long graph_kernels_run = 0;       // kernels run inside those replays
  unsigned pcg_graph_mask = 0;           // profiled kernel classes when the graph was captured
  cudaStream_t ws = nullptr;             // the context's own stream for graph capture and replay
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // per RHS: min over lattices of ||f_b|| / ||f||; the outer solve targets tol * this so that
  // every lattice meets tol relative to its own load
  std::vector<double> tol_scale;
  std::vector<int> sigma;
  std::vector<double> r_cell;
  double t_setup_s = 0.0;
  size_t device_bytes = 0;
  std::vector<void*> allocations;

  // reference-cell tables
  int* perm = nullptr;        // [2n]: local (i,d,p) index -> natural index node*d + c,
                              //       then the inverse permutation
  // lattice maps
  int* gath = nullptr;        // [N*nd*2] signed (row+1) codes, 0 = none (B_d^T)
  int* scat = nullptr;        // [L*2] signed (cell*nd + j + 1) codes, 0 = none (B_d)
  int* dinfo = nullptr;       // [L] (n << 8) | q: chain row q of n at the row's node (Eq. 30 D)
  int* corner_v = nullptr;    // [N*ncorner] free vertex index or -1 (A_p)
  int* vert_cells = nullptr;  // [nV*ncorner] (cell*ncorner + k) or -1 (A_p^T gather)
  double* r_dev = nullptr;    // [N]
  // snapshots = C_hat at every Gauss point, [N][nsnap]
  double* snap = nullptr;
  // mixed path: FP32 element matrices [N][nelem][ND][ND] for the Eq. 46b K_s products
  float* Ke_all = nullptr;
  // sparse K_rr of every cell in ELL form (mixed path, Eq. 46b): columns [nnz][nr] shared by all
  // cells, FP32 values [N][nnz][nr]
  int* krr_col = nullptr;
  float* krr_val = nullptr;
  int krr_nnz = 0;
  int* krr_nbr = nullptr;       // [nnz/d][nr/d] neighbour node of each node-level slot (nodal pattern)
  // Eq. 47 interface option: principal K_ii^{-1} [nrb][ni][ni] and the interior work vector
  double* Kii_inv = nullptr;
  double* w_i = nullptr;        // [m][N][ni]
  // ROM coefficients [N][nrb]
  double* alpha = nullptr;
  double* pi = nullptr;
  double* delta = nullptr;
  // principal operators (FP64)
  double* Kinv = nullptr;     // [nrb][nr][nr]  K_rr^(sigma_k)^{-1}
  double* Urp = nullptr;      // [nrb][nr][np]
  double* UrpT = nullptr;     // [nrb][np][nr]
  double* Sdd = nullptr;      // [nrb][nd][nd]  = F_dd^{-1}
  // ROM per-cell operators (assembled, Eq. 43)
  double* Fdd_c = nullptr;    // [N][nd][nd]
  double* Sdd_c = nullptr;    // [N][nd][nd]
  // mixed path, large cells: the same operators assembled in FP32, rows padded to ld_f (16 bytes)
  float* Fdd_f = nullptr;     // [N][nd][ld_f]
  float* Sdd_f = nullptr;     // [N][nd][ld_f]
  // mixed path, large cells: U_id_ring = the (i, d) block of the delta-combined K_rr^{-1} (Algorithm
  // 3), in FP32 in both orientations, [N][n_i][ld_id] and [N][n_d][ld_di]
  float* Uid_f = nullptr;
  float* Udi_f = nullptr;
  int ld_id = 0, ld_di = 0;
  int ld_f = 0;                // 0: packed symmetric tiles (sym_T tile rows of 32), else dense row stride
  int sym_T = 0;
  bool asm_f32 = false;
  bool exact = false;         // standard FETI-DP: every cell's own K_rr^{-1} (nrb = N, no ROM)
  float* Udp_f = nullptr;     // [N][nd][np] mixed path: the dual rows of U_rp_ring in FP32
  double* Urp_c = nullptr;    // [N][nr][np]
  double* UrpT_c = nullptr;   // [N][np][nr]
  // coarse solve
  CoarseBCR bcr;
  // right-hand side of Eq. 16: [m][ntot] = (f_R, f_P, d = 0)
  double* rhs = nullptr;
  double* rhs_p_cells = nullptr;   // [m][N][n_p] each cell's own corner loads (local corner order)
  // workspace
  double* w_cell_a = nullptr;   // [m][N][max(n, nr)]
  double* w_cell_b = nullptr;   // [m][N][max(n, nr)]
  double* w_d1 = nullptr;       // [m][N][nd]
  double* w_d2 = nullptr;       // [m][N][nd]
  double* w_p1 = nullptr;       // [m][N][np]
  double* w_P1 = nullptr;       // [m][nP]
  double* w_P2 = nullptr;       // [m][nP]
  double* w_zP = nullptr;       // [m][nP]  coarse solution shared by Algorithms 2 and 3
  double* w_L1 = nullptr;       // [m][L]
  double* w_R = nullptr;        // [m][N][nrb][nr]  local ROM bases (Eq. 46a)
  double* w_KR = nullptr;       // [m][N][nrb][nr]  K_s R
  double* w_tot = nullptr;      // [m][ntot] x 3 (preconditioner scratch)
  // Krylov storage
  double* V = nullptr;          // [(max_outer+1)][m][ntot]
  double* Z = nullptr;          // [max_outer][m][ntot]
  double* pcg = nullptr;        // [6][m][L]: x, r, z, p, q, right-hand side
  double* red = nullptr;        // reduction scratch (partials + scalars)
  unsigned int* red_count = nullptr;
  double* scal = nullptr;       // device scalars [64][m]
  double* h_scal = nullptr;     // pinned host mirror
  int inner_total = 0;
  // tensor-core path (mixed precision)
  bool mixed = false;           // FETIDP_MIXED_BF16
  TcOperator opKinv;            // K_rr^(k)^{-1}, separate (Eq. 46a)
  TcComb cFdd;                  // F_dd^(k) combined with delta (Eq. 48)
  TcComb cSdd;                  // S_dd^(k) combined with alpha (Eq. 49)
  TcComb cUrdT;                 // U_rd^(k)T combined with delta (Algorithm 3)
  TcComb cUrd;                  // U_rd^(k) combined with delta (transpose of Algorithm 3)
  uint8_t* tc_bbuf = nullptr;   // packed B operand staging
  size_t tc_bbuf_bytes = 0;
  float* tc_xf = nullptr;       // resident-operator combination: x in FP32
  size_t tc_xf_bytes = 0;
  float* tc_yp = nullptr;       // resident-operator combination: partial sums per principal group
  size_t tc_yp_bytes = 0;
  int* tc_err = nullptr;        // device error flag of the bounded waits
  unsigned long long wait_ns = 1000000000ull;   // budget of every device-side wait
  int* chk = nullptr;           // device flag of the input checks
};

// RAII timing of one launch (or one multi-kernel step) of a kernel class.
bool prof_grow(Ctx& c);
cudaEvent_t event_take(int dev);
void event_give(int dev, cudaEvent_t e);

struct ProfScope {
  Ctx& c;
  int slot = -1, gslot = -1;
  ProfScope(Ctx& ctx, int cls, double flops, double bytes) : c(ctx) {
    Prof& P = c.prof;
    if (!(P.mask >> cls & 1u)) return;
    if (P.capturing) {   // becomes a pair of event nodes of the graph being captured
      const size_t k = 2 * P.captured.size();
      if (k + 2 > P.gev.size()) return;
      gslot = (int)P.captured.size();
      P.captured.push_back({cls, flops, bytes, P.gev[k], P.gev[k + 1]});
      cudaEventRecordWithFlags(P.gev[k], c.stream, cudaEventRecordExternal);
      return;
    }
    P.launches[cls] += 1;
    if (P.used >= P.capacity && !prof_grow(c)) return;   // totals below cover the timed launches only
    P.flops[cls] += flops;
    P.bytes[cls] += bytes;
    slot = P.used++;
    P.cls[slot] = cls;
    cudaEventRecord(P.ev[2 * slot], c.stream);
  }
  ~ProfScope() {
    if (slot >= 0) cudaEventRecord(c.prof.ev[2 * slot + 1], c.stream);
    if (gslot >= 0) cudaEventRecordWithFlags(c.prof.captured[gslot].e1, c.stream, cudaEventRecordExternal);
  }
};

// ---------------------------------------------------------------- allocation
fetidp_status dalloc(Ctx& c, void** p, size_t bytes);
template <typename T>
fetidp_status dalloc_t(Ctx& c, T** p, size_t count) {
  return dalloc(c, reinterpret_cast<void**>(p), count * sizeof(T));
}

// ---------------------------------------------------------------- kernels (maps, vectors)
fetidp_status k_gather_BT(Ctx& c, const double* lam, long long lam_rs, const int* dinfo,
                          CellVec out_d, int nrhs, double beta);
fetidp_status k_nonfinite(Ctx& c, const double* x, long long n, int* flag);
fetidp_status wait_selfcheck(unsigned long long wait_ns, cudaStream_t stream);
fetidp_status k_scatter_B(Ctx& c, CCellVec yd, double* out, long long out_rs, const int* dinfo,
                          double alpha, double beta, int nrhs);
fetidp_status k_primal_assemble(Ctx& c, CCellVec cp, double* out, long long out_rs, double alpha,
                                double beta, int nrhs);
fetidp_status k_primal_extract(Ctx& c, const double* uP, long long uP_rs, CellVec cp, int nrhs);
fetidp_status k_dot(Ctx& c, const double* x, long long xs, const double* y, long long ys,
                    long long len, int nrhs, double* out);
fetidp_status k_multi_dot(Ctx& c, const double* Vb, long long vstride, int nv, const double* w,
                          long long len, int nrhs, double* out);
fetidp_status k_multi_axpy(Ctx& c, const double* Vb, long long vstride, int nv, const double* coef,
                           double* w, long long len, int nrhs, double sign);
fetidp_status k_copy_scale(Ctx& c, const double* x, double* y, long long len, int nrhs,
                           long long xs, long long ys, const double* s_dev, double s_host);

// ---------------------------------------------------------------- kernels (cell-level compute)
fetidp_status k_snapshots(Ctx& c);
fetidp_status k_body_loads(Ctx& c, const Geo& g, const int* perm_dev, const double* dirs_dev, const int* body_dev,
                           double* rhs, long long rhs_rs, double* fpc);
// c[l] = sum_s f_l^(s) . u_l^(s) (u natural cell order); partial: [m][kRedBlocks] scratch
fetidp_status k_compliance(Ctx& c, const double* u, double* out, double* partial);
// Device state of the greedy loop (Algorithm 4): selected cells and a stop flag.
constexpr int kMaxRbGreedy = 64;
struct GreedyState {
  int stop;
  int count;
  int sigma[kMaxRbGreedy];
  double znrm;   // 2-norm of the residual row selected at the current step
};
fetidp_status k_greedy_step(Ctx& c, double* D, const double* zeta, long long rows, long long len, double* beta,
                            double* inf, const GreedyState* st, int i);
fetidp_status k_greedy_select(Ctx& c, const double* inf, long long n, const double* D, long long len, int i,
                              double tol_rb, double tie, GreedyState* st);
fetidp_status k_greedy_init_df(Ctx& c, const double* A, const double* nrm, long long rows, long long len, float* Dh,
                               float* Dl, double* inf);
fetidp_status k_greedy_select_df(Ctx& c, const double* inf, long long n, const float* Dh, const float* Dl,
                                 long long len, int i, double tol_rb, double tie, GreedyState* st);
fetidp_status k_greedy_zeta_df(Ctx& c, const float* Dh, const float* Dl, long long len, int i, const GreedyState* st,
                               float* zh, float* zl, double* zeta);
fetidp_status k_greedy_step_df(Ctx& c, float* Dh, float* Dl, const float* zh, const float* zl, long long rows,
                               long long len, double* beta, double* inf, const GreedyState* st, int i);
fetidp_status k_greedy_zeta(Ctx& c, const double* D, long long len, int i, const GreedyState* st, double* zeta);
fetidp_status k_greedy_alpha(Ctx& c, const double* Z, const double* nrm, const double* beta, int nrb,
                             const GreedyState* st, double* T, double* alpha);
// dense batched setup kernels (principal blocks, SPD inverses by sweeps)
fetidp_status k_assemble_principal(Ctx& c, const int* sigma_dev, int nrb, double* Krr, double* Krp, double* Kpp);
fetidp_status k_spd_inverse_batched(Ctx& c, double* A, long long stride, int n, int lda, int batch, int* status);
fetidp_status k_batched_gemm_nn(Ctx& c, const double* A, long long sa, int lda, const double* B, long long sb,
                                int ldb, double* C, long long sc, int ldc, int M, int N, int K, int batch);
fetidp_status k_batched_block_copy(Ctx& c, const double* in, long long si, int ldi, int r0, int c0, double* out,
                                   long long so, int ldo, int M, int N, int batch, bool transpose);
fetidp_status k_df_gemm_planes(Ctx& c, const float* Ah, const float* Al, int M, int K, const double* X, int x_cs,
                               long long ncols, double* Y, int y_cs);
int df_pad_rows(long long rows);
int df_pad_k(int K);
fetidp_status k_df_gemm(Ctx& c, const double* A, int lda, int M, int K, const double* X, int x_cs, long long ncols,
                        double* Y, int y_cs);
fetidp_status k_batched_gemm(Ctx& c, bool ta, bool tb, int M, int N, int K, double alpha, const double* A,
                             long long sa, int lda, const double* B, long long sb, int ldb, double beta, double* C,
                             long long sc, int ldc, int batch);
fetidp_status k_batched_symmetrize(Ctx& c, double* A, long long stride, int n, int lda, int batch);
fetidp_status k_principal_pairs(Ctx& c, const double* Krp, double* P);   // P_kj = K_rp^(k)T U_rp^(j)
fetidp_status k_spp_cells(Ctx& c, const double* Kpp, const double* P, double* out);
struct LatticeSpan;
fetidp_status k_coarse_assemble(Ctx& c, const LatticeSpan& ls, const double* Spp, const int* vslab, const int* vpos,
                                int b, double* A, double* C);
fetidp_status k_gram_direct(Ctx& c, const double* Y, int ntab, const double* dvec, double* pi, double* delta,
                           double drop_rel);
fetidp_status k_batched_diag_sum(Ctx& c, const double* A, long long stride, int lda, int r0, int m, int batch,
                                 double* out);
fetidp_status k_apply_K(Ctx& c, CCellVec u, CellVec y, int nvec_per_col, int ncols, bool idp,
                        bool r_only, const double* chat, double chat_scale_dr, int len_override = 0);
fetidp_status k_rom_combine_f32(Ctx& c, const double* src, long long kstride, int ld, int r0, int c0, int rows,
                                int cols, const double* coef, float* out, int ldo, int symT = 0);
fetidp_status k_cell_symv_f32(Ctx& c, const float* mats, CCellVec x, CellVec y, double alpha, double beta, int nrhs);
fetidp_status k_cell_gemm_f32(Ctx& c, const float* mats, int ldm, int nout, int nin, CCellVec x, CellVec y,
                              double alpha, double beta, int nrhs);
fetidp_status k_cell_gemv_strided(Ctx& c, const double* mats, long long mstride, int ld, int mrows,
                                  int mcols, CCellVec x, CellVec y, double alpha, double beta,
                                  int nrhs);
fetidp_status k_grouped_gemm(Ctx& c, const double* A, long long a_stride_k, int lda, int M, int K,
                             CCellVec X, CellVec Y, const double* coef, double alpha, double beta,
                             int nrhs, bool separate, long long y_k_stride);
fetidp_status k_grouped_gemm_n(Ctx& c, const double* A, long long a_stride_k, int lda, int M,
                               int K, int nk, CCellVec X, CellVec Y, const double* coef,
                               double alpha, double beta, long long ncell, int nrhs, bool separate,
                               long long y_k_stride, int prof_class = FETIDP_K_GROUPED_GEMM);
fetidp_status k_gram_solve(Ctx& c, const double* R, const double* KR, CCellVec v, CellVec x,
                           int nrhs, int len = -1);
fetidp_status k_grad(Ctx& c, const double* u, const double* w, double* g);
fetidp_status k_element_matrices_f32(Ctx& c);
fetidp_status k_krr_ell_assemble(Ctx& c, const int* cnt, const int* idx, int cmax);
fetidp_status k_apply_K_f32(Ctx& c, const float* u, long long u_rs, int u_cs, float* y, long long y_rs,
                            int y_cs, int nvec, int nrhs, bool idp, bool r_only, long long ext = -1);
fetidp_status k_gram_solve_f32(Ctx& c, const float* R, const float* KR, CCellVec v, CellVec x,
                               int nrhs, long long r_ext = -1);

// ---------------------------------------------------------------- tensor cores (tc_gemm.cu)
int tc_bn_for(long long ncols, int m_tiles, int batch);
fetidp_status tc_pack_operator(Ctx& c, TcOperator& op, const double* src, long long op_stride, int lda,
                               int r0, int c0, int M, int K, int nops, bool separate, int nterm);
fetidp_status tc_apply(Ctx& c, const TcOperator& op, CCellVec X, const double* coef, void* Y,
                       bool y_f64, long long y_rs, int y_cs, long long y_b_stride, double alpha,
                       double beta, int nrhs, long long ncell, long long y_ext = -1);
fetidp_status tc_selfcheck(Ctx& c, int M, int K, int N, double* rel_err);
fetidp_status tc_selfcheck_static(Ctx& c, int M, int K, int N, double* rel_err);
size_t tc_selfcheck_static_bytes(int M, int K, int N);
void tc_free_operator(Ctx& c, TcOperator& op);
int tc_comb_bn(long long ncols, int m_tiles, int kto, int nX, int nops, bool two_sets);
bool tc_comb_fits(int K, int split, long long ncols, int m_tiles, int nops, bool two_sets);
fetidp_status tc_comb_pack(Ctx& c, TcComb& op, const double* src0, long long st0, int lda0, int r00, int c00,
                           int M0, const double* src1, long long st1, int lda1, int r01, int c01, int M1,
                           int K, int nops, int split);
size_t tc_comb_staging_bytes(const TcComb& op, long long ncols);
bool tc_comb2_ok(const TcComb& op);
size_t tc_comb2_xf_bytes(const TcComb& op, long long ncols);
size_t tc_comb2_yp_bytes(const TcComb& op, long long ncols);
fetidp_status tc_comb_selfcheck(Ctx& c, int M0, int M1, int K, int N, int nops, double* rel_err);
fetidp_status tc_comb_apply(Ctx& c, const TcComb& op, CCellVec X, const double* coef0, const double* coef1,
                            void* Y, bool y_f64, long long y_rs, int y_cs, double alpha, double beta, int nrhs,
                            long long ncell);

// ---------------------------------------------------------------- setup / coarse
fetidp_status setup_context(Ctx& c, const fetidp_problem* probs, int nprob, const fetidp_options& o);
fetidp_status coarse_setup(Ctx& c, const double* Spp_dev);   // per-cell S_pp_ring on the device
fetidp_status coarse_solve_f32(Ctx& c, const double* b, long long b_rs, double* x, long long x_rs, int nrhs);
fetidp_status k_udp_f32(Ctx& c, bool trans, CCellVec x, CellVec y, double alpha, double beta, int nrhs);
fetidp_status coarse_solve(Ctx& c, const double* b, long long b_rs, double* x, long long x_rs,
                           int nrhs);

// ---------------------------------------------------------------- operators (solver.cu)
fetidp_status op_apply_F(Ctx& c, const double* lam, long long lam_rs, double* y, long long y_rs);
fetidp_status op_apply_MD(Ctx& c, const double* r, long long r_rs, double* z, long long z_rs);
fetidp_status op_apply_A(Ctx& c, const double* x, double* y);
fetidp_status op_precondition(Ctx& c, const double* x, double* y);
fetidp_status pcg_solve(Ctx& c, const double* b, long long b_rs, double* x, long long x_rs);

}  // namespace fetidp
