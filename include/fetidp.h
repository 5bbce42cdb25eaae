/*
 * fetidp.h -- C ABI of the GB300 (sm_103a) ROM-based inexact FETI-DP hot path.
 *
 * Method: Hirschler, Bouclier, Antolin, Buffa, "Reduced Order Modeling based
 * Inexact FETI-DP solver for lattice structures" (arXiv 2308.11371).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Ownership   The caller owns every buffer it passes.  A context owns all of
 *             its device workspace; it is allocated in fetidp_setup and freed
 *             in fetidp_destroy.  No other entry point allocates device
 *             memory.
 * Pointers    Vectors are FP64.  Unless stated otherwise they are DEVICE
 *             pointers on the device that was current at fetidp_setup.
 * Streams     All work is enqueued on the stream given to fetidp_setup
 *             (NULL = legacy default stream).  Entry points that return
 *             host-visible results (fetidp_solve's info, fetidp_rom_data)
 *             synchronise that stream; the others are asynchronous.
 * Errors      Every call returns a fetidp_status and never aborts the process.
 *             A CUDA error is reported as FETIDP_ECUDA.  Non-finite host data
 *             given to fetidp_setup (radii, loads, map parameters, material)
 *             give FETIDP_EINVAL; so do non-finite input vectors when the
 *             context's check_inputs option is set (the default).  A device
 *             wait that exceeds wait_budget_ns gives FETIDP_ETIMEOUT.
 * Layouts     n_rhs load cases ("RHS") are stored RHS-major:
 *               multiplier vectors   lambda[rhs][L]
 *               cell vectors         u[rhs][cell][n_dof]  (cell-duplicated,
 *                                    local node-lexicographic order, x fastest,
 *                                    displacement components interleaved)
 *               primal vectors       uP[rhs][n_P]
 *             Cell s = cx + nx*(cy + ny*cz).  Multiplier rows are ordered by
 *             global node (lexicographic, x fastest), then by the chain pair,
 *             then by component; see fetidp_problem for the row definition.
 */
#ifndef FETIDP_H
#define FETIDP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fetidp_ctx fetidp_ctx;

typedef enum {
  FETIDP_OK = 0,
  FETIDP_EINVAL = -1,      /* invalid argument or unsupported problem */
  FETIDP_ENOMEM = -2,      /* device or host allocation failed */
  FETIDP_ECUDA = -3,       /* a CUDA call failed (message: fetidp_last_error) */
  FETIDP_ENOTCONV = -4,    /* iteration limit reached before the tolerance */
  FETIDP_ETIMEOUT = -5,    /* a device-side wait exceeded its budget */
  FETIDP_ESINGULAR = -6,   /* a principal factorisation or the coarse problem is not SPD */
  FETIDP_EBREAKDOWN = -7   /* Krylov breakdown (p^T F p <= 0 or non-finite) */
} fetidp_status;

typedef enum {
  FETIDP_FP64 = 0,         /* every step in FP64 */
  FETIDP_MIXED_BF16 = 1    /* grouped principal contractions on tcgen05 in BF16 with FP32
                              accumulation; Krylov recurrences, reductions, coarse solve,
                              outer operator in FP64.  There is no TF32 precision: one TF32
                              product keeps 11 significand bits, fewer than the 16 of the
                              three-product BF16 split used here, at half its MMA rate */
} fetidp_precision;

/* One lattice problem (Sec. 2.1-2.2.1, Eqs. 1-6).  Host memory; copied at setup.
 *
 * Cells are images of one reference cell [0,1]^dim carrying elems^dim Q1
 * elements (Eq. 6).  Lattice coordinate xi = (cx,cy,cz) + eta, physical
 * x = F(xi) with the analytic macro map selected by map_kind:
 *   0 identity
 *   1 2D bend        x = (xi_x, xi_y + a sin(pi xi_x / L))          params a, L
 *   2 3D shear+bend  x = xi + (g1 xi_z, g2 xi_z, a sin(pi xi_x / L))  params a, L, g1, g2
 *   3 3D twist+bend  rotate (xi_y, xi_z) about (yc, zc) by tau xi_x / L, then add
 *                    a sin(pi xi_x / L) to z                          params a, L, tau, yc, zc
 * Material: isotropic, Poisson ratio nu (plane strain in 2D); Young's modulus
 * at each Gauss point from the strut mask in cell-local eta (mask_kind
 * 0 = 2D frame + diagonals, E_solid where distance <= r_cell[s] else E_void;
 * 1 = 3D body-centred-cubic diagonals, same rule; 2 = BCC with
 * E = E_void + (E_solid - E_void) sigmoid((r - dist) / mask_width)).
 * Dirichlet: all DOF on the face xi_{clamp_axis} = (clamp_side ? n : 0) are 0.
 * Loads: load_kind[l] = 0 traction of load_dir[l*dim..] per unit physical area
 * on the face xi_{load_axis[l]} = (load_side[l] ? n : 0); 1 body force per unit
 * physical volume.
 * Multipliers (Eq. 14-15, P. 156): non-redundant -- for a non-corner interface
 * node shared by cells s_1 < ... < s_m, rows u(s_j) - u(s_{j+1}) per component;
 * every cell copy of a clamped non-corner node gets one row u(s) = 0.
 * Primal DOF (Eq. 18): cell corners, assembled over free lattice vertices.
 * ROM (Sec. 4.2, Algorithm 4): at most n_rb principal cells, greedy stops early
 * when max ||Delta||_inf <= tol_rb.                                                 */
typedef struct {
  int dim;                  /* 2 or 3 */
  int cells[3];             /* nx, ny, nz (nz = 1 in 2D) */
  int elems;                /* Q1 elements per cell edge (>= 2) */
  double nu, E_solid, E_void;
  int mask_kind;
  double mask_width;
  const double *r_cell;     /* [N] strut radius per cell */
  int map_kind;
  double map_params[8];
  int clamp_axis, clamp_side;
  int n_loads;              /* number of load cases = RHS (>= 1) */
  const int *load_kind;     /* [n_loads] */
  const int *load_axis;     /* [n_loads] */
  const int *load_side;     /* [n_loads] */
  const double *load_dir;   /* [n_loads * dim] */
  int n_rb;                 /* principal cells requested (1..64) */
  double tol_rb;
} fetidp_problem;

/* Solver options.  fetidp_default_options fills the defaults shown. */
typedef struct {
  double tol_outer;         /* stop when the TRUE ||b - A x|| / ||b|| <= tol_outer (1e-8) */
  double tol_inner;         /* inner PCG stop: ||r_k|| / ||r_0|| <= tol_inner (1e-11; P. 579) */
  int max_outer;            /* FGMRES iterations in total, over all restart cycles (100)    */
  int max_inner;            /* PCG iterations per preconditioner application (1000) */
  int precision;            /* fetidp_precision (FETIDP_FP64) */
  int fixed_outer;          /* > 0: run exactly this many outer iterations (iterate-locked) */
  int fixed_inner;          /* > 0: run exactly this many PCG iterations per application */
  int tc_split;             /* mixed: 1 = one BF16 x BF16 product per contraction; 3 = operands
                               split into hi + lo BF16 parts, three products (hi hi, hi lo,
                               lo hi) for ~16-bit input precision (default 3)                */
  double tol_inner_mixed;   /* inner PCG tolerance used by the mixed path (1e-6)             */
  double gram_drop_mixed;   /* mixed path, Eq. 46b: pivots of the FP32 Gram matrix whose Schur
                               diagonal is not above this fraction of its largest diagonal are
                               dropped (1e-9; the FP64 path drops below 1e-12).  The Gram data
                               carry ~1e-5 relative noise (BF16 split products, FP32 K_s), so
                               Schur diagonals below ~1e-10 are noise                        */
  unsigned profile_mask;    /* kernel classes (bit k = fetidp_kernel_class k) timed from the
                               start of fetidp_setup, as fetidp_profile_enable does from the
                               call on; read with fetidp_profile_read (0)                     */
  int restart;              /* FGMRES cycle length: the Krylov storage holds restart + 1 basis
                               vectors and restart preconditioned ones per RHS (2 x restart x
                               n_tot x n_rhs x 8 bytes).  After a cycle the true residual is
                               recomputed and a new cycle starts from the current iterate.
                               0 = min(max_outer, 30) (0); fixed_outer > restart raises it    */
  long long wait_budget_ns; /* bound of every device-side wait of the tensor-core kernels and
                               of the grid barriers of the mixed path's one-launch coarse solve,
                               in ns of the GPU's global timer (1e9).  On expiry a tensor-core
                               kernel stops, lets its own copies and MMAs finish (a separate
                               fixed 1 s bound), frees its tensor memory and returns; a coarse
                               solve runs its remaining levels without waiting; the call reports
                               FETIDP_ETIMEOUT and the context stays usable.  Must be > 0     */
  int check_inputs;         /* 1: entry points that take input vectors (all but fetidp_solve)
                               check them for NaN/Inf first (FETIDP_EINVAL) and, in the mixed
                               precision, report an expired device wait (FETIDP_ETIMEOUT);
                               both synchronise the stream.  0: no check, fully asynchronous
                               calls (1)                                                     */
  int mixed_assembled;      /* mixed path, operators of the inner PCG (Eqs. 48, 49): 1 = each
                               cell's F_dd_ring and S_dd_ring assembled once in FP32 and streamed
                               (4 n_d^2 bytes per cell per application, shared by the RHS);
                               0 = principal form on the tensor cores (2 N_rb n_d^2 flops per
                               column); 2 = assembled in FP32 as packed upper-triangle 32 x 32
                               tiles, each read once and used for both triangles (about half
                               the memory of 1; n_d <= 640); -1 = 1 when n_d > 128, i.e. for 3D
                               cells, else 0 (-1)                                              */
  int interface;            /* interface sub-preconditioner of Algorithm 1 (Sec. 3.2.3): 0 = PCG on
                               F_ring (Eq. 48) preconditioned by M_D_ring (Eq. 49); 1 = one
                               application of M_D^{-ROM} (Eq. 47), the Dirichlet preconditioner
                               whose interior solves K_ii^(s)^{-1} are ROM approximations built
                               from the principal K_ii^{-1} as Eq. 46 builds the K_rr solves;
                               FP64 arithmetic in both precisions (0)                         */
  int method;               /* 0 = ROM-based inexact FETI-DP (Secs. 3-4); 1 = standard FETI-DP
                               (Sec. 2.2.4, the paper's comparison system): every cell's K_rr is
                               factorised (dense inverse, N n_r^2 doubles), F and M_D are exact and
                               the block preconditioner of Eq. 44 is exact, so FGMRES takes one
                               outer iteration and the inner PCG is standard FETI-DP's.  FP64 with
                               interface 0 only; fetidp_rom_data answers EINVAL (0)           */
  int tc_bn;                /* mixed path: column-tile width of the Eq. 46a tensor-core GEMM, 64,
                               128 or 256; 0 = the library's rule (the widest tile that still
                               gives a wave of CTAs).  fetidp_tc_time measures the candidates and
                               the Python tuner stores the best per problem shape (0)          */
} fetidp_options;

typedef struct {
  int outer_its;            /* FGMRES iterations (max over RHS) */
  int inner_its_total;      /* PCG iterations summed over preconditioner applications */
  int n_rb;                 /* principal cells selected */
  double rel_residual;      /* max over RHS of the true ||b - A x|| / ||b|| (a batch: divided by
                               min over lattices of ||b_lattice||, which bounds the worst lattice) */
  double t_setup_s, t_solve_s;
  size_t device_bytes;      /* device workspace held by the context */
  long long kernel_launches;   /* kernels of this library run by the solve (graph replays included;
                                  a process-wide counter, so concurrent calls on other contexts
                                  are counted too) */
  long long host_launches;     /* launch calls the host issued for them (a graph replay is one) */
  int inner_graph;             /* 1: the inner PCG iterations ran as a captured CUDA graph */
} fetidp_info;

/* Sizes of a context: out[0..11] = N cells, n_dof, n_i, n_d, n_p, n_r per cell,
 * L multipliers, n_P primal DOF, n_rhs, n_rb selected, n_snap snapshot length,
 * n_tot = N*n_r + n_P + L (outer Krylov vector length per RHS).             */
fetidp_status fetidp_sizes(const fetidp_ctx *ctx, long long out[12]);

void fetidp_default_options(fetidp_options *opt);

/* Where each lattice of a batch sits: cell0[b], L0[b], P0[b] (b = 0..B) are the first cell,
 * multiplier row and primal DOF of lattice b, and [B] the totals (N, L, n_P).  Arrays of B + 1
 * entries (host memory), any may be NULL; B = n_problems of fetidp_setup. */
fetidp_status fetidp_batch_layout(const fetidp_ctx *ctx, long long *cell0, long long *L0, long long *P0);

/* Build the context for n_problems >= 1 lattices: maps B, A_p, D (Eqs. 14-18);
 * snapshots of C_hat at every Gauss point (Eq. 52); greedy principal cells and
 * alpha (Algorithm 4, Eqs. 55-56); principal factorisations and operators
 * (Eq. 39); pi, delta (Eqs. 40-42); ROM local operators and the coarse S_PP
 * factorisation (Eq. 43, Sec. 3.2.1).  cuda_stream is a cudaStream_t (may be
 * NULL).  On success *out owns all workspace.
 * Batch (n_problems > 1): the lattices are solved together as one block-diagonal
 * system.  They share the reference cell (dim, elems), the material law and mask
 * and the number of load cases; sizes, radii, macro maps, clamped faces and loads
 * are their own.  One reduced basis is selected from the snapshots of all cells
 * (n_rb, tol_rb of probs[0]); the principal operators serve every lattice.  Cells,
 * multipliers and primal DOF of the lattices follow each other in the context's
 * vectors (fetidp_batch_layout).  The outer solve stops when every lattice's
 * relative residual is <= tol_outer.
 * Errors: EINVAL (bad sizes, incompatible lattices), ENOMEM, ECUDA, ESINGULAR. */
fetidp_status fetidp_setup(const fetidp_problem *probs, int n_problems,
                           const fetidp_options *opt, void *cuda_stream, fetidp_ctx **out);

/* y = F_ring lambda (Eq. 48) for every RHS column: gather B_d^T, grouped
 * principal contraction with delta, coarse correction through S_PP^{-1},
 * scatter B_d.  lambda, y: device [n_rhs][L]; may not alias.                */
fetidp_status fetidp_apply_F(fetidp_ctx *ctx, const double *lambda, double *y);

/* z = M_D_ring^{-1} r (Eq. 49): D-scaled gather, alpha-combined principal
 * Dirichlet Schur complements, D-scaled scatter.  r, z: device [n_rhs][L].  */
fetidp_status fetidp_precond(fetidp_ctx *ctx, const double *r, double *z);

/* z = M_D^{-ROM} r (Eq. 47): D-scaled gather, per cell K_dd g - K_di x_i with x_i the ROM
 * approximation of K_ii^(s)^{-1} K_id g (basis [K_ii^(sigma_k)^{-1} K_id g]_k, K_ii^(s)-orthogonal
 * projection), D-scaled scatter; K_s matrix-free (Eq. 52), FP64.  The context must have been set
 * up with the option interface = 1 (EINVAL otherwise).  r, z: device [n_rhs][L].            */
fetidp_status fetidp_precond_rom(fetidp_ctx *ctx, const double *r, double *z);

/* Solve the saddle-point system of Eq. 16 by right-preconditioned flexible
 * GMRES with the block preconditioner of Eq. 44 (Algorithms 1-3), x_0 = 0,
 * restarted from the current iterate while the true residual is above tol.
 * u: device [n_rhs][N][n_dof] cell-duplicated displacements (out);
 * lambda: device [n_rhs][L] multipliers (out), may be NULL.  info (host, may
 * be NULL) receives iteration counts, residual and timings.
 * Returns ENOTCONV when max_outer is reached above tol_outer (u still holds
 * the last iterate), EBREAKDOWN on a Krylov breakdown.                       */
fetidp_status fetidp_solve(fetidp_ctx *ctx, double *u, double *lambda, fetidp_info *info);

/* Same as fetidp_solve with HOST output buffers (pageable or pinned); copies
 * the results back inside the call (end-to-end measurement).               */
fetidp_status fetidp_solve_host(fetidp_ctx *ctx, double *u_host, double *lambda_host,
                                fetidp_info *info);

/* Compliance c[l] = sum_s f_l^(s)T u_l^(s) per load case (the objective whose gradient
 * fetidp_grad returns).  u: device, cell-duplicated natural order [rhs][cell][n_dof] as written by
 * fetidp_solve; c: n_rhs doubles, host or device.  Deterministic reduction order. */
fetidp_status fetidp_compliance(fetidp_ctx *ctx, const double *u, double *c);

/* Gradient of compliance w.r.t. the per-cell radii r_s: for every RHS,
 * g[rhs][s] = - w_s^T (dK_s / dr_s) u_s with w = u when w == NULL (the
 * compliance c = f^T u is self-adjoint).  u, w: device [n_rhs][N][n_dof] as
 * returned by fetidp_solve; g: device [n_rhs][N].  Zero for hard masks.    */
fetidp_status fetidp_grad(fetidp_ctx *ctx, const double *u, const double *w, double *g);

/* ---- component entry points (the individual steps of the hot path) ---- */

/* x_d = B_d^T lambda for every cell (Eq. 15): x_d device [n_rhs][N][n_d]
 * (dual DOF in local order), lambda device [n_rhs][L].  Bit-exact.          */
fetidp_status fetidp_gather_BT(fetidp_ctx *ctx, const double *lambda, double *x_d);

/* z = sum_s B_d^(s) y_d^(s) (Eq. 15): y_d device [n_rhs][N][n_d], z device
 * [n_rhs][L].  Row-wise, no atomics, bit-exact.                            */
fetidp_status fetidp_scatter_B(fetidp_ctx *ctx, const double *y_d, double *z);

/* y_s = K_s u_s for every cell (Eq. 5a with Eq. 52), matrix-free from the
 * Gauss-point field C_hat: u, y device [n_rhs][N][n_dof] (natural order).   */
fetidp_status fetidp_apply_K(fetidp_ctx *ctx, const double *u, double *y);

/* x = S_PP_ring^{-1} b, the coarse solve of Sec. 3.2.1 (FP64 block cyclic
 * reduction of the Cholesky-equivalent block factorisation): b, x device
 * [n_rhs][n_P]; may alias.                                                   */
fetidp_status fetidp_coarse_solve(fetidp_ctx *ctx, const double *b, double *x);

/* x_r = K_rr_ring^{-ROM} v_r (Eq. 46a-b) for every cell: v, x device
 * [n_rhs][N][n_r] in local (i, d) order.                                     */
fetidp_status fetidp_local_rom_solve(fetidp_ctx *ctx, const double *v, double *x);

/* y = A x with A the saddle-point matrix of Eq. 16, and y = P x with P the
 * preconditioner of Eq. 44 (Algorithm 1).  x, y device [n_rhs][n_tot] laid
 * out as (u_R [N][n_r] local (i,d) order, u_P [n_P], lambda [L]).           */
fetidp_status fetidp_apply_A(fetidp_ctx *ctx, const double *x, double *y);
fetidp_status fetidp_apply_P(fetidp_ctx *ctx, const double *x, double *y);

/* Copy the ROM data to HOST buffers (any may be NULL): sigma [n_rb] principal
 * cells, alpha / pi / delta [N][n_rb] (Eqs. 38, 41).  Synchronises.          */
fetidp_status fetidp_rom_data(fetidp_ctx *ctx, int *sigma, double *alpha, double *pi,
                              double *delta);

/* ---- diagnostics ---- */

/* Kernel classes timed by the profiler. */
enum {
  FETIDP_K_GROUPED_GEMM = 0,  /* principal-operator contraction, FP64 CUDA cores (Eqs. 43, 46a) */
  FETIDP_K_APPLY_K = 1,       /* matrix-free K_s (Eq. 52) */
  FETIDP_K_MAPS = 2,          /* B_d gather / scatter, A_p assembly / extraction (Eqs. 15, 18) */
  FETIDP_K_COARSE = 3,        /* coarse block cyclic reduction sweeps (Sec. 3.2.1) */
  FETIDP_K_CELL_GEMV = 4,     /* per-cell ROM operators (Eq. 43) */
  FETIDP_K_VECTOR = 5,        /* Krylov reductions and vector updates */
  FETIDP_K_GRAM = 6,          /* Eq. 46b Gram solves */
  FETIDP_K_TC_GEMM = 7,       /* principal contraction on tcgen05 tensor cores (BF16) */
  FETIDP_K_SETUP = 8,         /* setup kernels not in the classes below */
  FETIDP_K_SWEEP = 9,         /* setup: blocked sweep SPD inverses (K_rr, S_dd, coarse blocks) */
  FETIDP_K_TRACES = 10,       /* setup: Eq. 42 snapshot traces (FP64 or double-float GEMM) */
  FETIDP_K_GREEDY = 11,       /* setup: Algorithm 4 greedy steps */
  FETIDP_K_MULTI_K = 12,      /* mixed: K_rr^(s) times the N_rb local ROM basis vectors (Eq. 46b) */
  FETIDP_K_ASM_OP = 13,       /* mixed: assembled FP32 F_dd_ring / S_dd_ring of the inner PCG */
  FETIDP_K_NCLASS = 16
};

/* Start (mask != 0) or stop (mask == 0) timing the kernel classes whose bit is set in
 * mask: a CUDA event pair on the context stream around every launch of those classes
 * (at most 65536 launches until the next read), plus the algorithmic FLOP and byte
 * counts of each launch computed from its shapes.  Resets the accumulators.       */
fetidp_status fetidp_profile_enable(fetidp_ctx *ctx, unsigned mask);

/* Synchronise the stream and return per-class totals since the last enable/read
 * (host arrays of FETIDP_K_NCLASS entries, any may be NULL): device milliseconds,
 * launches, algorithmic FLOPs and algorithmic bytes.  Milliseconds, FLOPs and bytes
 * cover the launches that got an event pair (the first 16384); launches counts all.
 * Resets the accumulators.                                                          */
fetidp_status fetidp_profile_read(fetidp_ctx *ctx, double *ms, long long *launches,
                                  double *flops, double *bytes);

/* Self-check of the tcgen05 tensor-core GEMM on the current device: random A (M x K) and
 * N columns X, packed to BF16, multiplied on the tensor cores with FP32 accumulation and
 * compared with an FP64 GEMM of the same BF16-rounded inputs.  *rel_err receives
 * max |Y_tc - Y_ref| / max |Y_ref|.  Allocates and frees its own scratch (diagnostic only).
 * ETIMEOUT if a bounded device wait expired.                                           */
fetidp_status fetidp_tc_selfcheck(int M, int K, int N, double *rel_err);

/* Self-check of the fused combine kernel: nops random operators of M0 + M1 rows, rows below M0
 * combined with one random coefficient set and the others with a second set, random N
 * columns X; compared with FP64 on the same BF16-rounded inputs.  Diagnostic only.        */
fetidp_status fetidp_tc_comb_selfcheck(int M0, int M1, int K, int N, int nops, double *rel_err);

/* Size in bytes of the static device scratch behind fetidp_tc_selfcheck_static (4 MiB). */
#define FETIDP_TC_STATIC_SCRATCH_BYTES 4194304

/* Allocation-free variant of fetidp_tc_selfcheck.  The paper has no counterpart: this is a
 * health probe of the tensor-core path for callers that must not allocate device memory.
 *
 * Who cannot allocate, and why: a process whose device memory is held by a caching allocator
 * (PyTorch's, for one) can see a raw cudaMalloc fail while the cache still has room, and
 * cudaFree waits for the whole device, so a probe that frees stalls every stream other host
 * threads have queued work on.  A long-running solver or serving process that wants to check
 * its tensor cores between jobs is such a caller.
 *
 * Computes exactly what fetidp_tc_selfcheck(M, K, N, rel_err) computes (same seeded inputs,
 * same kernels; *rel_err = max |Y_tc - Y_ref| / max |Y_ref|), but every buffer (A, X, both
 * outputs, packed tiles, staging, error flag, result slot) is carved from one fixed device array
 * of FETIDP_TC_STATIC_SCRATCH_BYTES bytes inside this library.  No cudaMalloc / cudaFree or
 * other allocating routine is called; the error flag and result slot are cleared on the stream
 * at the start of each call, and every other buffer is fully written before it is read.
 *
 * M, K, N >= 1.  The scratch needed is about 8 (M K + N K + 2 N M) bytes plus the packed BF16
 * tiles; a shape that does not fit returns FETIDP_EINVAL with the required and available
 * byte counts in fetidp_last_error(), before any CUDA call.
 * stream: a cudaStream_t, or NULL for the legacy default stream; the call returns after that
 * stream has finished the probe.  rel_err: host pointer.
 *
 * Setup: the first call on each device looks the scratch address up with cudaGetSymbolAddress
 * (this may load the library's device code on that device), with that device current, and keeps
 * it; later calls reuse it.  Make the first call on a device before any stream capture begins.
 *
 * Concurrency: all callers on a device share the one scratch array.  Calls that overlap in time
 * (from two host threads, or on two streams with no ordering between them) race on it and may
 * return wrong results; the caller must serialise them.
 * Errors: EINVAL (sizes, or scratch too small), ECUDA, ETIMEOUT (a bounded device wait expired). */
fetidp_status fetidp_tc_selfcheck_static(int M, int K, int N, double *rel_err, void *stream);

/* Probe of the bounded device waits (the paper has no counterpart): one thread of a one-block
 * kernel waits, through the same bounded wait the tensor-core kernels use, on an mbarrier phase
 * that nothing completes.  The wait expires after wait_budget_ns (0 < budget <= 1e10 ns) and the
 * call returns FETIDP_ETIMEOUT -- the status a solve or an entry point returns when one of its
 * kernels' waits expires -- with the device and every context still usable.  FETIDP_OK would mean
 * the wait completed, which it cannot.  stream: cudaStream_t or NULL; the call synchronises it.
 * waited_s (host, may be NULL): wall time of the call.  The flag it uses is one static device int
 * of this library, so calls that overlap in time race on it.  EINVAL for a budget out of range. */
/* Mean device time (ms, CUDA events on the context's stream) of `reps` launches of the context's
 * Eq. 46a tensor-core GEMM (all principal inverses against every cell's column, into the local
 * bases' buffer) with column-tile width bn (64, 128 or 256), after one untimed launch.  Mixed
 * contexts only (EINVAL otherwise); the inputs are the context's workspace, so the call changes no
 * solver state that a later solve reads.  Synchronises the stream.                               */
fetidp_status fetidp_tc_time(fetidp_ctx *ctx, int bn, int reps, double *ms);

fetidp_status fetidp_wait_selfcheck(long long wait_budget_ns, void *stream, double *waited_s);

/* Number of kernels this library has launched in the calling process. *//* Number of kernels this library has launched in the calling process. */
long long fetidp_kernel_launches(void);

void fetidp_destroy(fetidp_ctx *ctx);
const char *fetidp_status_string(fetidp_status s);
/* Last error message of this thread (CUDA error text or argument check). */
const char *fetidp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FETIDP_H */
