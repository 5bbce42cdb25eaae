// Setup phase of the ROM-based inexact FETI-DP solver.
//
// Host C++ builds the integer maps (Eqs. 12-18), the loads (Eq. 5b) and the
// O(N_rb) principal work (Eq. 39 factorisations); the O(N) work runs on the
// GPU: snapshots (Eq. 52), the greedy passes of Algorithm 4, the projection
// traces of Eq. 42 (one GEMM against the snapshot matrix) and the ROM local
// operators of Eq. 43.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <thread>

#include "common.cuh"
#include "host_linalg.h"

namespace fetidp {

fetidp_status k_row_reduce(Ctx& c, const double* X, long long rows, long long len, const double* z,
                           int mode, double* out);
fetidp_status k_row_normalise(Ctx& c, const double* A, const double* nrm, double* D, long long rows,
                              long long len);
fetidp_status k_row_update(Ctx& c, double* D, const double* beta, const double* zeta,
                           long long rows, long long len);
fetidp_status k_scale_copy(Ctx& c, const double* x, const double* s, double* y, long long len);
fetidp_status k_column_gradients(Ctx& c, const double* src, long long kstride, long long lstride,
                                 int len_in, int mode, int unit_base, int nk, int ncol, double* out);
fetidp_status k_trace_tables(Ctx& c, const TraceTableSpec* specs_dev, int ntab, double* T,
                             long long tstride);
fetidp_status k_split_planes(Ctx& c, const double* x, long long n, float* hi, float* lo);
fetidp_status k_trace_tables_df(Ctx& c, const TraceTableSpecDF* specs_dev, int ntab, float* Th, float* Tl,
                                long long ldt);
fetidp_status k_rom_combine(Ctx& c, const double* src, long long kstride, int ld, int r0, int c0,
                            int rows, int cols, const double* coef, double* out, bool transpose);

namespace {

constexpr double kTieRel = 1e-12;     // greedy argmax ties (lowest cell index wins)
constexpr double kDropRel = 1e-12;    // pivot drop of the N_rb x N_rb Gram systems

struct RefCell {
  std::vector<int> perm;        // idp -> natural
  std::vector<int> iperm;       // natural -> idp
  std::vector<int> dual_pos;    // node -> position among dual nodes, or -1
  std::vector<int> corner_pos;  // node -> corner index, or -1
};

RefCell build_ref(int d, int e, int& ni, int& nd, int& np) {
  RefCell R;
  const int nn1 = e + 1;
  const int nnode = d == 2 ? nn1 * nn1 : nn1 * nn1 * nn1;
  std::vector<int> cls(nnode);
  for (int nidx = 0; nidx < nnode; ++nidx) {
    const int ijk[3] = {nidx % nn1, (nidx / nn1) % nn1, nidx / (nn1 * nn1)};
    int nb = 0;
    for (int k = 0; k < d; ++k) nb += (ijk[k] == 0 || ijk[k] == e) ? 1 : 0;
    cls[nidx] = nb == d ? 2 : (nb > 0 ? 1 : 0);
  }
  R.dual_pos.assign(nnode, -1);
  R.corner_pos.assign(nnode, -1);
  int cnt[3] = {0, 0, 0};
  for (int nidx = 0; nidx < nnode; ++nidx) {
    if (cls[nidx] == 1) R.dual_pos[nidx] = cnt[1];
    if (cls[nidx] == 2) R.corner_pos[nidx] = cnt[2];
    cnt[cls[nidx]]++;
  }
  for (int cl = 0; cl < 3; ++cl)
    for (int nidx = 0; nidx < nnode; ++nidx)
      if (cls[nidx] == cl)
        for (int comp = 0; comp < d; ++comp) R.perm.push_back(nidx * d + comp);
  R.iperm.assign(R.perm.size(), 0);
  for (size_t i = 0; i < R.perm.size(); ++i) R.iperm[R.perm[i]] = (int)i;
  ni = cnt[0] * d;
  nd = cnt[1] * d;
  np = cnt[2] * d;
  return R;
}

// f^(s) of one load case for one cell (natural order), Eq. 5b.
void cell_load(const Ctx& c, const Geo& g, const fetidp_problem& p, int load, int cx, int cy, int cz,
               std::vector<double>& f) {
  const int d = c.d, e = c.e, NA = 1 << d;
  const double h = 1.0 / e;
  const double* dir = p.load_dir + (size_t)load * d;
  const int cc[3] = {cx, cy, cz};
  std::fill(f.begin(), f.end(), 0.0);
  if (p.load_kind[load] == 1) {   // body force per unit physical volume
    for (int el = 0; el < c.nelem; ++el) {
      const int ec[3] = {el % e, (el / e) % e, el / (e * e)};
      for (int gp = 0; gp < NA; ++gp) {
        double eta[3], xi[3], J[3][3];
        gauss_point(g, cx, cy, cz, ec[0], ec[1], ec[2], gp, eta, xi);
        macro_jacobian(g, xi, J);
        double det;
        if (d == 2) det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        else
          det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        const double wq = std::pow(0.5 * h, d) * det;
        for (int A = 0; A < NA; ++A) {
          double NAv = 1.0;
          for (int k = 0; k < d; ++k) {
            const double tk = gauss_t((gp >> k) & 1);
            NAv *= ((A >> k) & 1) ? tk : 1.0 - tk;
          }
          const int node = (ec[0] + (A & 1)) + (e + 1) * ((ec[1] + ((A >> 1) & 1)) +
                                                          (e + 1) * (d == 3 ? ec[2] + ((A >> 2) & 1) : 0));
          for (int i = 0; i < d; ++i) f[(size_t)node * d + i] += wq * NAv * dir[i];
        }
      }
    }
    return;
  }
  const int ax = p.load_axis[load], side = p.load_side[load];
  if (cc[ax] != (side ? g.nc[ax] - 1 : 0)) return;
  int tang[2], nt = 0;
  for (int k = 0; k < d; ++k)
    if (k != ax) tang[nt++] = k;
  for (int el = 0; el < c.nelem; ++el) {
    const int ec[3] = {el % e, (el / e) % e, el / (e * e)};
    if (ec[ax] != (side ? e - 1 : 0)) continue;
    for (int fg = 0; fg < (1 << (d - 1)); ++fg) {
      double t[3] = {0.0, 0.0, 0.0};
      t[ax] = side ? 1.0 : 0.0;
      for (int q = 0; q < nt; ++q) t[tang[q]] = gauss_t((fg >> q) & 1);
      double xi[3] = {0.0, 0.0, 0.0};
      for (int k = 0; k < d; ++k) xi[k] = cc[k] + (ec[k] + t[k]) * h;
      double J[3][3];
      macro_jacobian(g, xi, J);
      double meas;
      if (d == 2) {
        meas = std::sqrt(J[0][tang[0]] * J[0][tang[0]] + J[1][tang[0]] * J[1][tang[0]]);
      } else {
        const double a[3] = {J[0][tang[0]], J[1][tang[0]], J[2][tang[0]]};
        const double b[3] = {J[0][tang[1]], J[1][tang[1]], J[2][tang[1]]};
        const double cr[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2],
                              a[0] * b[1] - a[1] * b[0]};
        meas = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
      }
      const double wq = std::pow(0.5 * h, d - 1) * meas;
      for (int A = 0; A < NA; ++A) {
        if (((A >> ax) & 1) != (side ? 1 : 0)) continue;
        double NAv = 1.0;
        for (int k = 0; k < d; ++k) NAv *= ((A >> k) & 1) ? t[k] : 1.0 - t[k];
        const int node = (ec[0] + (A & 1)) + (e + 1) * ((ec[1] + ((A >> 1) & 1)) +
                                                        (e + 1) * (d == 3 ? ec[2] + ((A >> 2) & 1) : 0));
        for (int i = 0; i < d; ++i) f[(size_t)node * d + i] += wq * NAv * dir[i];
      }
    }
  }
}

template <typename T>
fetidp_status upload(Ctx& c, T** dst, const std::vector<T>& src) {
  FD_TRY(dalloc_t(c, dst, src.size() ? src.size() : 1));
  if (!src.empty())
    FD_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice,
                            c.stream));
  return FETIDP_OK;
}

}  // namespace

fetidp_status setup_context(Ctx& c, const fetidp_problem* probs, int nprob, const fetidp_options& o) {
  using namespace host;
  auto t0 = std::chrono::steady_clock::now();
  // FETIDP_VERBOSE=1: synchronise after each phase and print its wall time to stderr
  const bool verbose = std::getenv("FETIDP_VERBOSE") != nullptr;
  auto tp = t0;
  auto phase = [&](const char* name) {
    if (!verbose) return;
    cudaStreamSynchronize(c.stream);
    const auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "[fetidp setup] %-28s %8.2f ms\n", name,
                 std::chrono::duration<double, std::milli>(now - tp).count());
    tp = now;
  };
  // ---------------------------------------------------------------- validation
  // A batch shares the reference cell (dim, elems), the material law and mask, the load count
  // and the reduced basis (n_rb, tol_rb of the first lattice); sizes, radii, macro maps, clamped
  // faces and load cases are per lattice.
  if (nprob < 1 || !probs) { set_error("no lattice"); return FETIDP_EINVAL; }
  const fetidp_problem& p = probs[0];
  for (int bl = 0; bl < nprob; ++bl) {
    const fetidp_problem& q = probs[bl];
    if (q.dim != 2 && q.dim != 3) { set_error("dim must be 2 or 3"); return FETIDP_EINVAL; }
    if (q.elems < 2) { set_error("elems must be >= 2"); return FETIDP_EINVAL; }
    for (int k = 0; k < 3; ++k)
      if (q.cells[k] < 1 || (q.dim == 2 && k == 2 && q.cells[2] != 1)) {
        set_error("bad cell counts"); return FETIDP_EINVAL;
      }
    if (q.n_loads < 1 || !q.load_kind || !q.load_dir || !q.r_cell) {
      set_error("missing loads or radii"); return FETIDP_EINVAL;
    }
    if (q.n_rb < 1 || q.n_rb > 64) { set_error("n_rb must be in [1, 64]"); return FETIDP_EINVAL; }
    if (q.E_solid < 0.0 || q.E_void < 0.0) { set_error("negative Young's modulus"); return FETIDP_EINVAL; }
    if (q.E_solid == 0.0 && q.E_void == 0.0) {
      set_error("E_solid = E_void = 0: every cell stiffness is zero");
      return FETIDP_ESINGULAR;
    }
    {
      // non-finite host data would propagate silently into every operator
      bool fin = std::isfinite(q.nu) && std::isfinite(q.E_solid) && std::isfinite(q.E_void) &&
                 std::isfinite(q.mask_width) && std::isfinite(q.tol_rb);
      for (int k = 0; k < 8; ++k) fin = fin && std::isfinite(q.map_params[k]);
      const long long nq = (long long)q.cells[0] * q.cells[1] * q.cells[2];
      for (long long k = 0; k < nq && fin; ++k) fin = std::isfinite(q.r_cell[k]);
      for (int k = 0; k < q.n_loads * q.dim && fin; ++k) fin = std::isfinite(q.load_dir[k]);
      if (!fin) { set_error("non-finite value in the problem data"); return FETIDP_EINVAL; }
    }
    if (q.clamp_axis < 0 || q.clamp_axis >= q.dim) { set_error("bad clamp axis"); return FETIDP_EINVAL; }
    if (!(q.nu > -1.0 && q.nu < 0.5)) { set_error("nu out of range"); return FETIDP_EINVAL; }
    if (q.mask_kind < 0 || q.mask_kind > 2 || (q.dim == 2) != (q.mask_kind == 0)) {
      set_error("mask kind does not match the dimension"); return FETIDP_EINVAL;
    }
    if (q.dim != p.dim || q.elems != p.elems || q.mask_kind != p.mask_kind || q.nu != p.nu ||
        q.E_solid != p.E_solid || q.E_void != p.E_void || q.mask_width != p.mask_width ||
        q.n_loads != p.n_loads) {
      set_error("lattices of a batch must share dim, elems, material, mask and the number of loads");
      return FETIDP_EINVAL;
    }
  }
  if (o.max_outer < 1 || o.max_inner < 1 || o.restart < 0 || o.fixed_outer < 0 || o.fixed_inner < 0) {
    set_error("bad iteration limits");
    return FETIDP_EINVAL;
  }
  if (o.wait_budget_ns <= 0) { set_error("wait_budget_ns must be > 0"); return FETIDP_EINVAL; }
  if (o.mixed_assembled < -1 || o.mixed_assembled > 2) { set_error("mixed_assembled must be -1, 0, 1 or 2"); return FETIDP_EINVAL; }
  if (o.interface < 0 || o.interface > 1) { set_error("interface must be 0 or 1"); return FETIDP_EINVAL; }
  if (o.method < 0 || o.method > 1) { set_error("method must be 0 or 1"); return FETIDP_EINVAL; }
  if (o.tc_bn != 0 && o.tc_bn != 64 && o.tc_bn != 128 && o.tc_bn != 256) {
    set_error("tc_bn must be 0, 64, 128 or 256");
    return FETIDP_EINVAL;
  }
  if (o.method == 1 && (o.precision != FETIDP_FP64 || o.interface != 0)) {
    set_error("standard FETI-DP (method 1) runs in FP64 with the PCG interface solve");
    return FETIDP_EINVAL;
  }
  if (!(std::isfinite(o.tol_outer) && std::isfinite(o.tol_inner) && std::isfinite(o.tol_inner_mixed) &&
        o.tol_outer >= 0.0 && o.tol_inner >= 0.0 && o.tol_inner_mixed >= 0.0)) {
    set_error("tolerances must be finite and >= 0");
    return FETIDP_EINVAL;
  }
  c.opt = o;
  c.kry = o.restart > 0 ? o.restart : std::min(o.max_outer, 30);
  if (o.fixed_outer > c.kry) c.kry = o.fixed_outer;
  c.wait_ns = (unsigned long long)o.wait_budget_ns;
  c.mixed = o.precision == FETIDP_MIXED_BF16;
  if (c.mixed && o.tc_split != 1 && o.tc_split != 3) { set_error("tc_split must be 1 or 3"); return FETIDP_EINVAL; }
  if (!(o.gram_drop_mixed >= 0.0 && o.gram_drop_mixed < 1.0)) {
    set_error("gram_drop_mixed must lie in [0, 1)");
    return FETIDP_EINVAL;
  }
  const int d = p.dim, e = p.elems;
  c.lat.assign(nprob, LatticeSpan{});
  c.N = 0;
  for (int bl = 0; bl < nprob; ++bl) {
    const fetidp_problem& q = probs[bl];
    LatticeSpan& ls = c.lat[bl];
    Geo& g = ls.geo;
    g.dim = d; g.e = e;
    for (int k = 0; k < 3; ++k) g.nc[k] = q.cells[k];
    g.mask_kind = q.mask_kind; g.map_kind = q.map_kind;
    g.mask_width = q.mask_width; g.E_solid = q.E_solid; g.E_void = q.E_void; g.nu = q.nu;
    for (int k = 0; k < 8; ++k) g.mp[k] = q.map_params[k];
    ls.cell0 = c.N;
    ls.ncell = (long long)q.cells[0] * q.cells[1] * q.cells[2];
    ls.clamp_axis = q.clamp_axis;
    ls.clamp_side = q.clamp_side;
    c.N += ls.ncell;
  }
  c.geo = c.lat[0].geo;
  c.d = d; c.e = e;
  c.clamp_axis = p.clamp_axis; c.clamp_side = p.clamp_side;
  c.m = p.n_loads;
  c.ncorner = 1 << d;
  c.nelem = d == 2 ? e * e : e * e * e;
  c.ngp = 1 << d;
  c.nc = d == 2 ? 10 : 45;
  c.nsnap = (long long)c.nelem * c.ngp * c.nc;
  RefCell ref = build_ref(d, e, c.ni, c.nd, c.np);
  c.n = (int)ref.perm.size();
  c.nr = c.ni + c.nd;
  c.r_cell.clear();
  for (int bl = 0; bl < nprob; ++bl) c.r_cell.insert(c.r_cell.end(), probs[bl].r_cell, probs[bl].r_cell + c.lat[bl].ncell);
  {
    std::vector<int> pp(ref.perm);
    pp.insert(pp.end(), ref.iperm.begin(), ref.iperm.end());
    FD_TRY(upload(c, &c.perm, pp));
  }
  FD_TRY(upload(c, &c.r_dev, c.r_cell));
  phase("reference tables");

  // ---------------------------------------------------------------- multipliers (Eqs. 14-15)
  const int nn1 = e + 1;
  std::vector<int> gath((size_t)c.N * c.nd * 2, 0);
  std::vector<int> scat;
  std::vector<int> dinfo;   // per row: (chain rows n of its node << 8) | chain position q
  {
    // about one multiplier per dual DOF of every cell and component (upper bound for reserve)
    const size_t est = (size_t)c.N * c.nd;
    scat.reserve(2 * est);
    dinfo.reserve(est);
  }
  for (int bl = 0; bl < nprob; ++bl) {
  const fetidp_problem& pl = probs[bl];
  const long long cell0 = c.lat[bl].cell0;
  c.lat[bl].L0 = (long long)dinfo.size();
  const int nx = pl.cells[0], ny = pl.cells[1], nz = pl.cells[2];
  const long long gd[3] = {(long long)nx * e + 1, (long long)ny * e + 1, d == 3 ? (long long)nz * e + 1 : 1};
  const long long clamp_coord = pl.clamp_side ? (long long)pl.cells[pl.clamp_axis] * e : 0;
  for (long long gz = 0; gz < gd[2]; ++gz)
    for (long long gy = 0; gy < gd[1]; ++gy)
      for (long long gx = 0; gx < gd[0]; ++gx) {
        const long long gc[3] = {gx, gy, gz};
        int on = 0;
        for (int k = 0; k < d; ++k) on += (gc[k] % e == 0) ? 1 : 0;
        if (on == 0 || on == d) continue;   // cell interior or lattice vertex (primal)
        // owner cells: Cartesian product of candidate cell coordinates
        int cand[3][2], ncand[3];
        for (int k = 0; k < 3; ++k) {
          if (k >= d) { cand[k][0] = 0; ncand[k] = 1; continue; }
          const int nk = pl.cells[k];
          if (gc[k] % e == 0) {
            const int q = (int)(gc[k] / e);
            ncand[k] = 0;
            if (q - 1 >= 0) cand[k][ncand[k]++] = q - 1;
            if (q < nk) cand[k][ncand[k]++] = q;
          } else {
            cand[k][0] = (int)(gc[k] / e);
            ncand[k] = 1;
          }
        }
        std::pair<long long, int> own[8];   // (cell, dual node position), sorted by cell
        int mult = 0;
        for (int a = 0; a < ncand[0]; ++a)
          for (int b = 0; b < ncand[1]; ++b)
            for (int q = 0; q < ncand[2]; ++q) {
              const int cx = cand[0][a], cy = cand[1][b], cz = cand[2][q];
              const long long s = cell0 + cx + (long long)nx * (cy + (long long)ny * cz);
              const int lx = (int)(gx - (long long)cx * e), ly = (int)(gy - (long long)cy * e);
              const int lz = d == 3 ? (int)(gz - (long long)cz * e) : 0;
              const int lnode = lx + nn1 * (ly + nn1 * lz);
              int pos = mult++;
              while (pos > 0 && own[pos - 1].first > s) { own[pos] = own[pos - 1]; --pos; }
              own[pos] = {s, ref.dual_pos[lnode]};
            }
        const bool clamped = gc[pl.clamp_axis] == clamp_coord;
        auto add_gath = [&](long long s, int j, int code) {
          int* gp2 = &gath[((size_t)s * c.nd + j) * 2];
          if (gp2[0] == 0) gp2[0] = code;
          else gp2[1] = code;
        };
        if (clamped) {
          for (int q = 0; q < mult; ++q)
            for (int comp = 0; comp < d; ++comp) {
              const auto& ow = own[q];
              const long long row = (long long)dinfo.size();
              const int j = ow.second * d + comp;
              scat.push_back((int)(ow.first * c.nd + j + 1));
              scat.push_back(0);
              dinfo.push_back(0);
              add_gath(ow.first, j, (int)(row + 1));
            }
        } else {
          for (int q = 0; q + 1 < mult; ++q)
            for (int comp = 0; comp < d; ++comp) {
              const long long row = (long long)dinfo.size();
              const int j1 = own[q].second * d + comp, j2 = own[q + 1].second * d + comp;
              scat.push_back((int)(own[q].first * c.nd + j1 + 1));
              scat.push_back(-(int)(own[q + 1].first * c.nd + j2 + 1));
              dinfo.push_back(((mult - 1) << 8) | q);
              add_gath(own[q].first, j1, (int)(row + 1));
              add_gath(own[q + 1].first, j2, -(int)(row + 1));
            }
        }
      }
  c.lat[bl].nL = (long long)dinfo.size() - c.lat[bl].L0;
  }
  c.L = (long long)dinfo.size();
  FD_TRY(upload(c, &c.gath, gath));
  FD_TRY(upload(c, &c.scat, scat));
  FD_TRY(upload(c, &c.dinfo, dinfo));
  phase("multiplier maps");

  // ---------------------------------------------------------------- primal DOF (Eq. 18)
  // free vertices numbered lattice by lattice, lexicographic (x fastest) inside each lattice
  std::vector<int> corner_v((size_t)c.N * c.ncorner);
  std::vector<int> vert_cells;
  int nV = 0;
  for (int bl = 0; bl < nprob; ++bl) {
    const fetidp_problem& pl = probs[bl];
    const long long cell0 = c.lat[bl].cell0;
    const int nx = pl.cells[0], ny = pl.cells[1], nz = pl.cells[2];
    const int vd[3] = {nx + 1, ny + 1, d == 3 ? nz + 1 : 1};
    const long long nvert = (long long)vd[0] * vd[1] * vd[2];
    const int cvert = pl.clamp_side ? vd[pl.clamp_axis] - 1 : 0;
    std::vector<int> vnum(nvert, -1);
    const int V0 = nV;
    for (long long v = 0; v < nvert; ++v) {
      const int ijk[3] = {(int)(v % vd[0]), (int)((v / vd[0]) % vd[1]), (int)(v / ((long long)vd[0] * vd[1]))};
      if (ijk[pl.clamp_axis] != cvert) vnum[v] = nV++;
    }
    c.lat[bl].V0 = V0;
    c.lat[bl].nV = nV - V0;
    vert_cells.resize((size_t)nV * c.ncorner, -1);
    std::vector<int> vfill(nV - V0, 0);
    for (long long sl = 0; sl < c.lat[bl].ncell; ++sl) {
      const long long s = cell0 + sl;
      const int cijk[3] = {(int)(sl % nx), (int)((sl / nx) % ny), (int)(sl / ((long long)nx * ny))};
      for (int k = 0; k < c.ncorner; ++k) {
        const int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
        long long v = 0, stride = 1;
        for (int q = 0; q < 3; ++q) {
          v += (cijk[q] + (q < d ? o[q] : 0)) * stride;
          stride *= vd[q];
        }
        const int vn = vnum[v];
        corner_v[(size_t)s * c.ncorner + k] = vn;
        if (vn >= 0) vert_cells[(size_t)vn * c.ncorner + vfill[vn - V0]++] = (int)(s * c.ncorner + k);
      }
    }
  }
  c.nV = nV;
  c.nP = (long long)nV * d;
  FD_TRY(upload(c, &c.corner_v, corner_v));
  FD_TRY(upload(c, &c.vert_cells, vert_cells));
  c.ntot = c.N * c.nr + c.nP + c.L;

  // ---------------------------------------------------------------- loads: rhs = (f_R, f_P, 0)
  {
    std::vector<double> rhs((size_t)c.m * c.ntot, 0.0), fpc((size_t)c.m * c.N * c.np, 0.0);
    // a single lattice's body-force loads are integrated on the GPU (every cell's Gauss points);
    // tractions (face cells only) and batches stay on the host threads
    bool any_body = false;
    for (int l = 0; l < c.m; ++l) any_body = any_body || probs[0].load_kind[l] == 1;
    const bool gpu_body = nprob == 1 && any_body;
    // each cell's loads (Eq. 5b) on the host threads; every cell writes only its own entries
    auto cells_range = [&](long long s0, long long s1) {
      std::vector<double> f(c.n);
      for (int l = 0; l < c.m; ++l) {
        if (gpu_body && probs[0].load_kind[l] == 1) continue;
        double* rl = rhs.data() + (size_t)l * c.ntot;
        for (long long s = s0; s < s1; ++s) {
          int bl = 0;
          while (bl + 1 < nprob && s >= c.lat[bl + 1].cell0) ++bl;
          const fetidp_problem& pl = probs[bl];
          const long long sl = s - c.lat[bl].cell0;
          const int nx = pl.cells[0], ny = pl.cells[1];
          const int cx = (int)(sl % nx), cy = (int)((sl / nx) % ny), cz = (int)(sl / ((long long)nx * ny));
          cell_load(c, c.lat[bl].geo, pl, l, cx, cy, cz, f);
          for (int li = 0; li < c.nr; ++li) rl[s * c.nr + li] = f[ref.perm[li]];
          for (int q = 0; q < c.np; ++q) fpc[((size_t)l * c.N + s) * c.np + q] = f[ref.perm[c.nr + q]];
        }
      }
    };
    {
      const long long nthr = std::max(1LL, std::min<long long>(std::thread::hardware_concurrency(), 32));
      const long long per = (c.N + nthr - 1) / nthr;
      std::vector<std::thread> pool;
      for (long long t = 0; t < nthr; ++t) {
        const long long s0 = t * per, s1 = std::min(c.N, s0 + per);
        if (s0 < s1) pool.emplace_back(cells_range, s0, s1);
      }
      for (auto& th : pool) th.join();
    }
    // primal loads f_P = sum_s A_p f_p (Eq. 18), assembled in cell order (on the GPU below when the
    // body forces are integrated there)
    for (int l = 0; l < c.m && !gpu_body; ++l) {
      double* rl = rhs.data() + (size_t)l * c.ntot;
      for (long long s = 0; s < c.N; ++s)
        for (int k = 0; k < c.ncorner; ++k) {
          const int vn = corner_v[(size_t)s * c.ncorner + k];
          if (vn < 0) continue;
          for (int comp = 0; comp < d; ++comp)
            rl[c.N * c.nr + (size_t)vn * d + comp] += fpc[((size_t)l * c.N + s) * c.np + k * d + comp];
        }
    }
    FD_TRY(upload(c, &c.rhs, rhs));
    FD_TRY(upload(c, &c.rhs_p_cells, fpc));
    if (gpu_body) {
      std::vector<int> body(c.m);
      std::vector<double> dirs((size_t)c.m * d);
      for (int l = 0; l < c.m; ++l) {
        body[l] = probs[0].load_kind[l] == 1 ? 1 : 0;
        for (int i = 0; i < d; ++i) dirs[(size_t)l * d + i] = probs[0].load_dir[(size_t)l * d + i];
      }
      int *perm_d = nullptr, *body_d = nullptr;
      double* dirs_d = nullptr;
      FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&perm_d), sizeof(int) * c.n));
      FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&body_d), sizeof(int) * c.m));
      FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&dirs_d), sizeof(double) * dirs.size()));
      FD_CUDA(cudaMemcpyAsync(perm_d, ref.perm.data(), sizeof(int) * c.n, cudaMemcpyHostToDevice, c.stream));
      FD_CUDA(cudaMemcpyAsync(body_d, body.data(), sizeof(int) * c.m, cudaMemcpyHostToDevice, c.stream));
      FD_CUDA(cudaMemcpyAsync(dirs_d, dirs.data(), sizeof(double) * dirs.size(), cudaMemcpyHostToDevice, c.stream));
      FD_TRY(k_body_loads(c, c.lat[0].geo, perm_d, dirs_d, body_d, c.rhs, c.ntot, c.rhs_p_cells));
      // f_P from every cell's corner loads (tractions and body forces)
      FD_TRY(k_primal_assemble(c, CCellVec{c.rhs_p_cells, c.N * c.np, c.np}, c.rhs + c.N * c.nr, c.ntot, 1.0,
                               1.0, c.m));
      FD_CUDA(cudaStreamSynchronize(c.stream));   // host vectors go out of scope
      tmp_free(c, perm_d);
      tmp_free(c, body_d);
      tmp_free(c, dirs_d);
    }
    // per RHS: min over lattices of ||f_b|| / ||f|| (f_b: the lattice's remaining and primal loads)
    c.tol_scale.assign(c.m, 1.0);
    if (nprob > 1)
      for (int l = 0; l < c.m; ++l) {
        const double* rl = rhs.data() + (size_t)l * c.ntot;
        double all = 0.0, mn = -1.0;
        std::vector<double> nb(nprob, 0.0);
        for (int bl = 0; bl < nprob; ++bl) {
          for (long long t = c.lat[bl].cell0 * c.nr; t < (c.lat[bl].cell0 + c.lat[bl].ncell) * c.nr; ++t)
            nb[bl] += rl[t] * rl[t];
          for (long long t = c.N * c.nr + c.lat[bl].V0 * d; t < c.N * c.nr + (c.lat[bl].V0 + c.lat[bl].nV) * d; ++t)
            nb[bl] += rl[t] * rl[t];
          all += nb[bl];
        }
        for (int bl = 0; bl < nprob; ++bl)
          if (nb[bl] > 0.0 && (mn < 0.0 || nb[bl] < mn)) mn = nb[bl];
        c.tol_scale[l] = (all > 0.0 && mn > 0.0) ? std::sqrt(mn / all) : 1.0;
      }
  }
  phase("primal maps + loads");

  // ---------------------------------------------------------------- snapshots (Eq. 52)
  FD_TRY(dalloc_t(c, &c.snap, (size_t)c.N * c.nsnap));
  FD_TRY(k_snapshots(c));
  phase("snapshots");

  // ---------------------------------------------------------------- Algorithm 4 (greedy)
  // The whole loop is enqueued without host round trips: each step selects on the device (or
  // sets the stop flag, after which the remaining kernels return at once); sigma is read back
  // once at the end.
  c.exact = o.method == 1;
  const int nrb_req = c.exact ? 0 : p.n_rb;
  if (nrb_req > kMaxRbGreedy) { set_error("n_rb above 64 is not supported"); return FETIDP_EINVAL; }
  if (!c.exact) {
  double *Delta = nullptr, *nrm = nullptr, *vals = nullptr, *beta_d = nullptr, *Z = nullptr, *T = nullptr;
  GreedyState* gst = nullptr;
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&Delta), sizeof(double) * c.N * c.nsnap));
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&nrm), sizeof(double) * c.N));
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&vals), sizeof(double) * c.N));
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&beta_d), sizeof(double) * c.N * nrb_req));
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&Z), sizeof(double) * c.nsnap * nrb_req));
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&T), sizeof(double) * nrb_req * nrb_req));
  FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&gst), sizeof(GreedyState)));
  auto free_greedy = [&]() {
    tmp_free(c, Delta); tmp_free(c, nrm); tmp_free(c, vals); tmp_free(c, beta_d); tmp_free(c, Z); tmp_free(c, T); tmp_free(c, gst);
  };
  FD_CUDA(cudaMemsetAsync(gst, 0, sizeof(GreedyState), c.stream));
  FD_TRY(k_row_reduce(c, c.snap, c.N, c.nsnap, nullptr, 0, nrm));
  if (c.mixed) {
    // mixed path: Delta as double-float planes (the Delta buffer holds them), steps on the FP32
    // pipe; zeta also as planes (zp) beside its FP64 row in Z
    float* Dh = reinterpret_cast<float*>(Delta);
    float* Dl = Dh + (size_t)c.N * c.nsnap;
    float* zp = nullptr;
    FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&zp), sizeof(float) * 2 * (size_t)c.nsnap));
    FD_TRY(k_greedy_init_df(c, c.snap, nrm, c.N, c.nsnap, Dh, Dl, vals));
    for (int i = 0; i < nrb_req; ++i) {
      double* zeta = Z + (size_t)i * c.nsnap;
      FD_TRY(k_greedy_select_df(c, vals, c.N, Dh, Dl, c.nsnap, i, p.tol_rb, kTieRel, gst));
      FD_TRY(k_greedy_zeta_df(c, Dh, Dl, c.nsnap, i, gst, zp, zp + c.nsnap, zeta));
      FD_TRY(k_greedy_step_df(c, Dh, Dl, zp, zp + c.nsnap, c.N, c.nsnap, beta_d + (size_t)i * c.N, vals, gst, i));
    }
    tmp_free(c, zp);
  } else {
    FD_TRY(k_row_normalise(c, c.snap, nrm, Delta, c.N, c.nsnap));
    FD_TRY(k_row_reduce(c, Delta, c.N, c.nsnap, nullptr, 1, vals));
    for (int i = 0; i < nrb_req; ++i) {
      double* zeta = Z + (size_t)i * c.nsnap;
      FD_TRY(k_greedy_select(c, vals, c.N, Delta, c.nsnap, i, p.tol_rb, kTieRel, gst));
      FD_TRY(k_greedy_zeta(c, Delta, c.nsnap, i, gst, zeta));
      // beta_i = Delta . zeta_i, Delta -= beta_i zeta_i and the next infinity norms, one pass
      FD_TRY(k_greedy_step(c, Delta, zeta, c.N, c.nsnap, beta_d + (size_t)i * c.N, vals, gst, i));
    }
  }
  GreedyState hst{};
  FD_CUDA(cudaMemcpyAsync(&hst, gst, sizeof(GreedyState), cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  c.sigma.assign(hst.sigma, hst.sigma + hst.count);
  c.nrb = hst.count;
  // ---------------------------------------------------------------- alpha (Eq. 56)
  FD_TRY(dalloc_t(c, &c.alpha, (size_t)c.N * c.nrb));
  FD_TRY(k_greedy_alpha(c, Z, nrm, beta_d, c.nrb, gst, T, c.alpha));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  free_greedy();
  phase("greedy + alpha");
  } else {
    // standard FETI-DP (Sec. 2.2.4): every cell is factorised; the "principal" operators below
    // are every cell's own, and no ROM coefficient is formed
    c.sigma.resize(c.N);
    for (long long s = 0; s < c.N; ++s) c.sigma[s] = (int)s;
    c.nrb = (int)c.N;
  }
  const int nrb = c.nrb;

  // ---------------------------------------------------------------- principal operators (Eq. 39)
  const int nr = c.nr, ni = c.ni, nd = c.nd, np = c.np;
  // All on the device: the principal K blocks assembled from their C_hat snapshots, K_rr^{-1} and
  // S_dd = F_dd^{-1} (F_dd = T_dr K_rr^{-1} T_rd, Sec. 3.1.1) by batched sweeps, U_rp = K_rr^{-1} K_rp.
  std::vector<double> dvec(nrb, 0.0);
  double *Krp_d = nullptr, *Kpp_d = nullptr;   // principal K_rp, K_pp: kept for S_pp_ring (Eq. 43)
  {
    FD_TRY(dalloc_t(c, &c.Kinv, (size_t)nrb * nr * nr));
    FD_TRY(dalloc_t(c, &c.Urp, (size_t)nrb * nr * np));
    FD_TRY(dalloc_t(c, &c.UrpT, (size_t)nrb * np * nr));
    FD_TRY(dalloc_t(c, &c.Sdd, (size_t)nrb * nd * nd));
    int* sigma_dev = nullptr;
    int* st_dev = nullptr;
    double* dvec_d = nullptr;
    FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&sigma_dev), sizeof(int) * nrb));
    FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&st_dev), sizeof(int)));
    FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&Krp_d), sizeof(double) * (size_t)nrb * nr * np));
    FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&Kpp_d), sizeof(double) * (size_t)nrb * np * np));
    FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&dvec_d), sizeof(double) * nrb));
    FD_CUDA(cudaMemcpyAsync(sigma_dev, c.sigma.data(), sizeof(int) * nrb, cudaMemcpyHostToDevice, c.stream));
    FD_CUDA(cudaMemsetAsync(st_dev, 0, sizeof(int), c.stream));
    FD_TRY(k_assemble_principal(c, sigma_dev, nrb, c.Kinv, Krp_d, Kpp_d));
    if (o.interface == 1) {   // Eq. 47: the principal interior blocks K_ii, inverted below
      FD_TRY(dalloc_t(c, &c.Kii_inv, (size_t)nrb * ni * ni));
      FD_TRY(k_batched_block_copy(c, c.Kinv, (long long)nr * nr, nr, 0, 0, c.Kii_inv, (long long)ni * ni, ni, ni,
                                  ni, nrb, false));
      FD_TRY(k_spd_inverse_batched(c, c.Kii_inv, (long long)ni * ni, ni, ni, nrb, st_dev));
    }
    phase("  principal assembly");
    FD_TRY(k_spd_inverse_batched(c, c.Kinv, (long long)nr * nr, nr, nr, nrb, st_dev));
    phase("  principal K_rr inverse");
    FD_TRY(k_batched_gemm_nn(c, c.Kinv, (long long)nr * nr, nr, Krp_d, (long long)nr * np, np, c.Urp,
                             (long long)nr * np, np, nr, np, nr, nrb));
    FD_TRY(k_batched_block_copy(c, c.Urp, (long long)nr * np, np, 0, 0, c.UrpT, (long long)np * nr, nr, nr, np,
                                nrb, true));
    FD_TRY(k_batched_diag_sum(c, c.Kinv, (long long)nr * nr, nr, ni, nd, nrb, dvec_d));
    FD_TRY(k_batched_block_copy(c, c.Kinv, (long long)nr * nr, nr, ni, ni, c.Sdd, (long long)nd * nd, nd, nd, nd,
                                nrb, false));
    FD_TRY(k_spd_inverse_batched(c, c.Sdd, (long long)nd * nd, nd, nd, nrb, st_dev));
    int hst = 0;
    FD_CUDA(cudaMemcpyAsync(dvec.data(), dvec_d, sizeof(double) * nrb, cudaMemcpyDeviceToHost, c.stream));
    FD_CUDA(cudaMemcpyAsync(&hst, st_dev, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    FD_CUDA(cudaStreamSynchronize(c.stream));
    tmp_free(c, sigma_dev); tmp_free(c, st_dev); tmp_free(c, dvec_d);
    if (hst != 0) {
      tmp_free(c, Krp_d); tmp_free(c, Kpp_d);
      set_error("principal K_rr is not positive definite");
      return FETIDP_ESINGULAR;
    }
  }
  phase("principal factorisations");

  // ---------------------------------------------------------------- projections pi, delta (Eqs. 41-42)
  if (!c.exact) {
    const int nqp = c.nelem * c.ngp, dd = d * d;
    const int npair = nrb * (nrb + 1) / 2;
    const int ntab = 2 * npair + nrb;
    double *Gd = nullptr, *Gp = nullptr, *Ge = nullptr, *Tab = nullptr, *Y = nullptr;
    FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&Gd), sizeof(double) * (size_t)nrb * nd * nqp * dd));
    FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&Gp), sizeof(double) * (size_t)nrb * np * nqp * dd));
    FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&Ge), sizeof(double) * (size_t)np * nqp * dd));
    FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&Y), sizeof(double) * (size_t)c.N * ntab));
    // columns of U_rd^(k) = K_rr^{-1} T_rd: rows ni+l of the symmetric inverse
    FD_TRY(k_column_gradients(c, c.Kinv + (size_t)ni * nr, (long long)nr * nr, nr, nr, 0, 0, nrb, nd, Gd));
    // columns of U_rp^(k): rows of U_rp^T
    FD_TRY(k_column_gradients(c, c.UrpT, (long long)np * nr, nr, nr, 0, 0, nrb, np, Gp));
    // unit corner vectors e_p (columns of K_rp)
    FD_TRY(k_column_gradients(c, nullptr, 0, 0, 0, 1, nr, 1, np, Ge));
    const size_t gstride_d = (size_t)nd * nqp * dd, gstride_p = (size_t)np * nqp * dd;
    // Both trace systems of Eq. 42 are Gram matrices of nearly dependent principal fields; their
    // pivoted solves decide which directions to drop at 1e-12 of the largest pivot and amplify
    // trace errors by ~1e5, so a BF16-split contraction is far too coarse.  The FP64 path takes
    // the tables and traces in FP64; the mixed path (whose operators carry ~1e-5 BF16 error) in
    // double-float arithmetic on the FP32 pipe (~1e-13), the tables written straight into the
    // padded float planes of the trace GEMM.
    void* specs_dev = nullptr;
    float* planes = nullptr;
    if (c.mixed) {
      const size_t nGd = (size_t)nrb * gstride_d, nGp = (size_t)nrb * gstride_p, nGe = gstride_p;
      const int Mp = df_pad_rows(ntab), Kp = df_pad_k((int)c.nsnap);
      const size_t nT = (size_t)Mp * Kp;
      FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&planes), sizeof(float) * 2 * (nGd + nGp + nGe + nT)));
      float *Gdh = planes, *Gdl = Gdh + nGd, *Gph = Gdl + nGd, *Gpl = Gph + nGp, *Geh = Gpl + nGp, *Gel = Geh + nGe;
      float *Th = Gel + nGe, *Tl = Th + nT;
      FD_TRY(k_split_planes(c, Gd, (long long)nGd, Gdh, Gdl));
      FD_TRY(k_split_planes(c, Gp, (long long)nGp, Gph, Gpl));
      FD_TRY(k_split_planes(c, Ge, (long long)nGe, Geh, Gel));
      std::vector<TraceTableSpecDF> specs;
      for (int i = 0; i < nrb; ++i)
        for (int j = i; j < nrb; ++j)
          specs.push_back({Gph + i * gstride_p, Gpl + i * gstride_p, Gph + j * gstride_p, Gpl + j * gstride_p, np});
      for (int i = 0; i < nrb; ++i) specs.push_back({Gph + i * gstride_p, Gpl + i * gstride_p, Geh, Gel, np});
      for (int i = 0; i < nrb; ++i)
        for (int j = i; j < nrb; ++j)
          specs.push_back({Gdh + i * gstride_d, Gdl + i * gstride_d, Gdh + j * gstride_d, Gdl + j * gstride_d, nd});
      FD_TRY(tmp_alloc(c, &specs_dev, sizeof(TraceTableSpecDF) * specs.size()));
      FD_CUDA(cudaMemcpyAsync(specs_dev, specs.data(), sizeof(TraceTableSpecDF) * specs.size(),
                              cudaMemcpyHostToDevice, c.stream));
      FD_CUDA(cudaMemsetAsync(Th, 0, sizeof(float) * 2 * nT, c.stream));   // zero padding
      FD_TRY(k_trace_tables_df(c, static_cast<const TraceTableSpecDF*>(specs_dev), (int)specs.size(), Th, Tl, Kp));
      phase("  gradients + trace tables");
      FD_TRY(k_df_gemm_planes(c, Th, Tl, ntab, (int)c.nsnap, c.snap, (int)c.nsnap, c.N, Y, ntab));
    } else {
      FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&Tab), sizeof(double) * (size_t)ntab * c.nsnap));
      std::vector<TraceTableSpec> specs;
      for (int i = 0; i < nrb; ++i)
        for (int j = i; j < nrb; ++j) specs.push_back({Gp + i * gstride_p, Gp + j * gstride_p, np});
      for (int i = 0; i < nrb; ++i) specs.push_back({Gp + i * gstride_p, Ge, np});
      for (int i = 0; i < nrb; ++i)
        for (int j = i; j < nrb; ++j) specs.push_back({Gd + i * gstride_d, Gd + j * gstride_d, nd});
      FD_TRY(tmp_alloc(c, &specs_dev, sizeof(TraceTableSpec) * specs.size()));
      FD_CUDA(cudaMemcpyAsync(specs_dev, specs.data(), sizeof(TraceTableSpec) * specs.size(),
                              cudaMemcpyHostToDevice, c.stream));
      FD_TRY(k_trace_tables(c, static_cast<const TraceTableSpec*>(specs_dev), (int)specs.size(), Tab, c.nsnap));
      phase("  gradients + trace tables");
      FD_TRY(k_grouped_gemm_n(c, Tab, 0, (int)c.nsnap, ntab, (int)c.nsnap, 1, CCellVec{c.snap, 0, (int)c.nsnap},
                              CellVec{Y, 0, ntab}, nullptr, 1.0, 0.0, c.N, 1, false, 0, FETIDP_K_TRACES));
    }
    phase("  trace contraction");
    // the two Gram systems of every cell, solved on the device (one warp per system)
    double* dvec_d = nullptr;
    FD_TRY(dalloc_t(c, &c.pi, (size_t)c.N * nrb));
    FD_TRY(dalloc_t(c, &c.delta, (size_t)c.N * nrb));
    FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&dvec_d), sizeof(double) * nrb));
    FD_CUDA(cudaMemcpyAsync(dvec_d, dvec.data(), sizeof(double) * nrb, cudaMemcpyHostToDevice, c.stream));
    FD_TRY(k_gram_direct(c, Y, ntab, dvec_d, c.pi, c.delta, kDropRel));
    FD_CUDA(cudaStreamSynchronize(c.stream));
    tmp_free(c, Gd); tmp_free(c, Gp); tmp_free(c, Ge); tmp_free(c, Tab); tmp_free(c, Y); tmp_free(c, specs_dev); tmp_free(c, planes); tmp_free(c, dvec_d);
  }
  phase("projections pi, delta");

  // ---------------------------------------------------------------- ROM local operators (Eq. 43)
  if (c.exact) {    // standard FETI-DP: every cell's own F_dd and S_dd
    FD_TRY(dalloc_t(c, &c.Fdd_c, (size_t)c.N * nd * nd));
    FD_TRY(k_batched_block_copy(c, c.Kinv, (long long)nr * nr, nr, ni, ni, c.Fdd_c, (long long)nd * nd, nd, nd, nd,
                                nrb, false));
    c.Sdd_c = c.Sdd;
  } else if (!c.mixed) {   // FP64 path: per-cell assembled F_dd_ring, S_dd_ring
    FD_TRY(dalloc_t(c, &c.Fdd_c, (size_t)c.N * nd * nd));
    FD_TRY(dalloc_t(c, &c.Sdd_c, (size_t)c.N * nd * nd));
    FD_TRY(k_rom_combine(c, c.Kinv, (long long)nr * nr, nr, ni, ni, nd, nd, c.delta, c.Fdd_c, false));
    FD_TRY(k_rom_combine(c, c.Sdd, (long long)nd * nd, nd, 0, 0, nd, nd, c.alpha, c.Sdd_c, false));
  } else {          // mixed path: principal operators packed for the tensor cores
    FD_TRY(k_element_matrices_f32(c));
    {
      // ELL pattern of K_rr on the reference cell (remaining DOF, local order) and, for each
      // stored entry, the element-matrix entries that sum into it (at most 2^d, fixed order)
      const int d = c.d, e = c.e, NA = 1 << d, ND = NA * d, nn1 = e + 1;
      std::vector<std::map<int, std::vector<int>>> rows(nr);
      for (int el = 0; el < c.nelem; ++el) {
        const int ex = el % e, ey = (el / e) % e, ez = d == 3 ? el / (e * e) : 0;
        for (int a = 0; a < ND; ++a) {
          const int A = a / d, ia = a % d;
          const int na = (ex + (A & 1)) + nn1 * ((ey + ((A >> 1) & 1)) + nn1 * (d == 3 ? ez + ((A >> 2) & 1) : 0));
          const int ga = ref.iperm[na * d + ia];
          if (ga >= nr) continue;
          for (int b = 0; b < ND; ++b) {
            const int B = b / d, ib = b % d;
            const int nb = (ex + (B & 1)) + nn1 * ((ey + ((B >> 1) & 1)) + nn1 * (d == 3 ? ez + ((B >> 2) & 1) : 0));
            const int gb = ref.iperm[nb * d + ib];
            if (gb >= nr) continue;
            rows[ga][gb].push_back(el * ND * ND + a * ND + b);
          }
        }
      }
      int nnz = 0;
      for (const auto& r : rows) nnz = std::max(nnz, (int)r.size());
      const int cmax = NA;
      std::vector<int> col((size_t)nnz * nr), cnt((size_t)nnz * nr, 0), idx((size_t)nnz * nr * cmax, 0);
      for (int r = 0; r < nr; ++r) {
        int sl = 0;
        for (const auto& kv : rows[r]) {
          col[(size_t)sl * nr + r] = kv.first;
          cnt[(size_t)sl * nr + r] = (int)kv.second.size();
          for (size_t q = 0; q < kv.second.size() && q < (size_t)cmax; ++q)
            idx[((size_t)sl * nr + r) * cmax + q] = kv.second[q];
          ++sl;
        }
        for (; sl < nnz; ++sl) col[(size_t)sl * nr + r] = r;   // padding: value 0 on the diagonal column
      }
      c.krr_nnz = nnz;
      // nodal structure: the d rows of a node share their neighbour nodes, slot d k + c' of row
      // d n + a holding component c' of the k-th neighbour (columns sorted, components interleaved)
      bool nodal = nr % d == 0 && nnz % d == 0;
      const int nnode = nr / d, nk = nnz / d;
      std::vector<int> nbr;
      if (nodal) nbr.assign((size_t)nk * nnode, 0);
      for (int n = 0; nodal && n < nnode; ++n)
        for (int k = 0; nodal && k < nk; ++k) {
          const size_t e0 = (size_t)(d * k) * nr + (size_t)d * n;
          const bool pad = cnt[e0] == 0;
          const int c0 = col[e0];
          if (!pad && c0 % d != 0) nodal = false;
          for (int a = 0; nodal && a < d; ++a)
            for (int cq = 0; cq < d; ++cq) {
              const size_t e = (size_t)(d * k + cq) * nr + (size_t)d * n + a;
              if ((cnt[e] == 0) != pad || (!pad && col[e] != c0 + cq)) { nodal = false; break; }
            }
          if (nodal) nbr[(size_t)k * nnode + n] = pad ? n : c0 / d;
        }
      if (nodal) FD_TRY(upload(c, &c.krr_nbr, nbr));
      int *cnt_d = nullptr, *idx_d = nullptr;
      FD_TRY(upload(c, &c.krr_col, col));
      FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&cnt_d), sizeof(int) * cnt.size()));
      FD_TRY(tmp_alloc(c, reinterpret_cast<void**>(&idx_d), sizeof(int) * idx.size()));
      FD_CUDA(cudaMemcpyAsync(cnt_d, cnt.data(), sizeof(int) * cnt.size(), cudaMemcpyHostToDevice, c.stream));
      FD_CUDA(cudaMemcpyAsync(idx_d, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, c.stream));
      FD_TRY(k_krr_ell_assemble(c, cnt_d, idx_d, cmax));
      FD_CUDA(cudaStreamSynchronize(c.stream));
      tmp_free(c, cnt_d);
      tmp_free(c, idx_d);
    }
    const int split = o.tc_split == 3 ? 3 : 1;
    const long long ncols = c.N * c.m;
    FD_TRY(tc_pack_operator(c, c.opKinv, c.Kinv, (long long)nr * nr, nr, 0, 0, nr, nr, nrb, true, split));
    // F_dd_ring and S_dd_ring of the inner PCG: assembled per cell in FP32 for large cells (streamed,
    // HBM-bound), principal form on the tensor cores otherwise
    c.asm_f32 = o.mixed_assembled > 0 || (o.mixed_assembled < 0 && nd > 128);
    if (c.asm_f32) {
      // dense rows padded to 16 bytes (streamed at the HBM rate), or with mixed_assembled = 2 the
      // packed upper-triangle 32 x 32 tiles of these symmetric operators (about half the bytes, up to
      // 20 tile rows; on GB300 that kernel is bound by its shared-memory traffic and is not faster)
      const int T = (nd + 31) / 32;
      c.sym_T = (o.mixed_assembled == 2 && T <= 20) ? T : 0;
      c.ld_f = c.sym_T ? 0 : (nd + 3) & ~3;
      const size_t fbytes = c.sym_T ? sizeof(float) * (size_t)c.N * 1024 * T * (T + 1) / 2
                                    : sizeof(float) * (size_t)c.N * nd * c.ld_f;
      FD_TRY(dalloc(c, reinterpret_cast<void**>(&c.Fdd_f), fbytes));
      FD_TRY(dalloc(c, reinterpret_cast<void**>(&c.Sdd_f), fbytes));
      FD_CUDA(cudaMemsetAsync(c.Fdd_f, 0, fbytes, c.stream));   // padding stays zero
      FD_CUDA(cudaMemsetAsync(c.Sdd_f, 0, fbytes, c.stream));
      FD_TRY(k_rom_combine_f32(c, c.Kinv, (long long)nr * nr, nr, ni, ni, nd, nd, c.delta, c.Fdd_f, c.ld_f, c.sym_T));
      FD_TRY(k_rom_combine_f32(c, c.Sdd, (long long)nd * nd, nd, 0, 0, nd, nd, c.alpha, c.Sdd_f, c.ld_f, c.sym_T));
      // Algorithm 3's U_rd_ring = [U_id_ring; F_dd_ring]: the (i, d) block in FP32, stored once per
      // orientation so that both of its products stream rows (K_rr^{-1} is symmetric, so the (d, i)
      // block is its transpose)
      c.ld_id = (nd + 3) & ~3;
      c.ld_di = (ni + 3) & ~3;
      FD_TRY(dalloc_t(c, &c.Uid_f, (size_t)c.N * ni * c.ld_id));
      FD_TRY(dalloc_t(c, &c.Udi_f, (size_t)c.N * nd * c.ld_di));
      FD_CUDA(cudaMemsetAsync(c.Uid_f, 0, sizeof(float) * (size_t)c.N * ni * c.ld_id, c.stream));
      FD_CUDA(cudaMemsetAsync(c.Udi_f, 0, sizeof(float) * (size_t)c.N * nd * c.ld_di, c.stream));
      FD_TRY(k_rom_combine_f32(c, c.Kinv, (long long)nr * nr, nr, 0, ni, ni, nd, c.delta, c.Uid_f, c.ld_id));
      FD_TRY(k_rom_combine_f32(c, c.Kinv, (long long)nr * nr, nr, ni, 0, nd, ni, c.delta, c.Udi_f, c.ld_di));
    }
    FD_TRY(tc_comb_pack(c, c.cFdd, c.Kinv, (long long)nr * nr, nr, ni, ni, nd, nullptr, 0, 0, 0, 0, 0, nd, nrb,
                        split));
    FD_TRY(tc_comb_pack(c, c.cSdd, c.Sdd, (long long)nd * nd, nd, 0, 0, nd, nullptr, 0, 0, 0, 0, 0, nd, nrb, split));
    FD_TRY(tc_comb_pack(c, c.cUrdT, c.Kinv, (long long)nr * nr, nr, ni, 0, nd, nullptr, 0, 0, 0, 0, 0, nr, nrb,
                        split));
    FD_TRY(tc_comb_pack(c, c.cUrd, c.Kinv, (long long)nr * nr, nr, 0, ni, nr, nullptr, 0, 0, 0, 0, 0, nd, nrb,
                        split));
    for (const TcComb* cb : {&c.cFdd, &c.cSdd, &c.cUrdT, &c.cUrd})
      if (!tc_comb_fits(cb->K, split, ncols, cb->m_tiles, cb->nops, cb->msplit < cb->M)) {
        set_error("combine kernel does not fit this cell size");
        return FETIDP_EINVAL;
      }
    size_t mx = 0;
    for (int bn : {64, 128, 256}) {   // room for every tile width (fetidp_tc_time, option tc_bn)
      const TcOperator* op = &c.opKinv;
      const long long n_tiles = (ncols + bn - 1) / bn;
      mx = std::max(mx, (size_t)n_tiles * op->k_tiles * bn * 64 * 2);
    }
    for (const TcComb* cb : {&c.cFdd, &c.cSdd, &c.cUrdT, &c.cUrd})
      mx = std::max(mx, tc_comb_staging_bytes(*cb, ncols));
    c.tc_bbuf_bytes = mx;
    FD_TRY(dalloc(c, reinterpret_cast<void**>(&c.tc_bbuf), mx));
    // resident-operator combination (every combined operator with one row tile and K <= 128:
    // F_dd, S_dd of the inner PCG, and U_rd for small cells): FP32 x and group partials
    size_t xf = 0, yp = 0;
    for (const TcComb* cb : {&c.cFdd, &c.cSdd, &c.cUrdT, &c.cUrd})
      if (tc_comb2_ok(*cb)) {
        xf = std::max(xf, tc_comb2_xf_bytes(*cb, ncols));
        yp = std::max(yp, tc_comb2_yp_bytes(*cb, ncols));
      }
    if (xf > 0) {
      c.tc_xf_bytes = xf;
      c.tc_yp_bytes = yp;
      FD_TRY(dalloc(c, reinterpret_cast<void**>(&c.tc_xf), xf));
      FD_TRY(dalloc(c, reinterpret_cast<void**>(&c.tc_yp), yp));
    }
    if (!c.tc_err) FD_TRY(dalloc(c, reinterpret_cast<void**>(&c.tc_err), sizeof(int)));
    FD_CUDA(cudaMemsetAsync(c.tc_err, 0, sizeof(int), c.stream));
  }
  if (c.exact) {
    c.Urp_c = c.Urp;
    c.UrpT_c = c.UrpT;
  } else {
    FD_TRY(dalloc_t(c, &c.Urp_c, (size_t)c.N * nr * np));
    FD_TRY(dalloc_t(c, &c.UrpT_c, (size_t)c.N * nr * np));
    FD_TRY(k_rom_combine(c, c.Urp, (long long)nr * np, np, 0, 0, nr, np, c.pi, c.Urp_c, false));
    FD_TRY(k_rom_combine(c, c.Urp, (long long)nr * np, np, 0, 0, nr, np, c.pi, c.UrpT_c, true));
  }
  if (c.mixed && (np == 8 || np == 24)) {   // the inner iterations' coarse term (Eq. 48) in FP32
    FD_TRY(dalloc_t(c, &c.Udp_f, (size_t)c.N * nd * np));
    FD_TRY(k_rom_combine_f32(c, c.Urp, (long long)nr * np, np, ni, 0, nd, np, c.pi, c.Udp_f, np));
  }

  phase("ROM operators / packing");

  // ---------------------------------------------------------------- coarse S_PP (Eq. 43, Sec. 3.2.1)
  {
    // P_kj = K_rp^(k)T U_rp^(j), then per cell S_pp_ring = sym(K_pp_ring - K_rp_ring^T U_rp_ring)
    double *Pkj = nullptr, *Spp = nullptr;
    fetidp_status st = FETIDP_OK;
    if (c.exact) {   // every cell's exact S_pp = K_pp - K_rp^T U_rp (Eq. 22)
      st = tmp_alloc(c, reinterpret_cast<void**>(&Spp), sizeof(double) * (size_t)c.N * np * np);
      if (st == FETIDP_OK && cudaMemcpyAsync(Spp, Kpp_d, sizeof(double) * (size_t)c.N * np * np, cudaMemcpyDeviceToDevice,
                                             c.stream) != cudaSuccess)
        st = FETIDP_ECUDA;
      if (st == FETIDP_OK)
        st = k_batched_gemm(c, true, false, np, np, nr, -1.0, Krp_d, (long long)nr * np, np, c.Urp, (long long)nr * np,
                            np, 1.0, Spp, (long long)np * np, np, (int)c.N);
      if (st == FETIDP_OK) st = k_batched_symmetrize(c, Spp, (long long)np * np, np, np, (int)c.N);
    } else {
      st = tmp_alloc(c, reinterpret_cast<void**>(&Pkj), sizeof(double) * (size_t)nrb * nrb * np * np);
      if (st == FETIDP_OK) st = tmp_alloc(c, reinterpret_cast<void**>(&Spp), sizeof(double) * (size_t)c.N * np * np);
      if (st == FETIDP_OK) st = k_principal_pairs(c, Krp_d, Pkj);
      if (st == FETIDP_OK) st = k_spp_cells(c, Kpp_d, Pkj, Spp);
    }
    if (st == FETIDP_OK) phase("S_pp per cell");
    if (st == FETIDP_OK) st = coarse_setup(c, Spp);
    cudaStreamSynchronize(c.stream);
    tmp_free(c, Pkj); tmp_free(c, Spp); tmp_free(c, Krp_d); tmp_free(c, Kpp_d);
    FD_TRY(st);
    phase("coarse factorisation");
  }

  // ---------------------------------------------------------------- workspace
  const size_t m = c.m;
  const size_t ncell_max = (size_t)c.N * std::max(c.n, c.nr);
  FD_TRY(dalloc_t(c, &c.w_cell_a, m * ncell_max));
  FD_TRY(dalloc_t(c, &c.w_cell_b, m * ncell_max));
  FD_TRY(dalloc_t(c, &c.w_d1, m * c.N * nd));
  FD_TRY(dalloc_t(c, &c.w_d2, m * c.N * nd));
  FD_TRY(dalloc_t(c, &c.w_p1, m * c.N * np));
  FD_TRY(dalloc_t(c, &c.w_P1, m * c.nP + 1));
  FD_TRY(dalloc_t(c, &c.w_P2, m * c.nP + 1));
  FD_TRY(dalloc_t(c, &c.w_zP, m * c.nP + 1));
  FD_TRY(dalloc_t(c, &c.w_L1, m * c.L + 1));
  // local ROM bases R and K_s R (Eq. 46): FP64 in the FP64 path, FP32 in the mixed path
  const size_t rom_elems = c.exact ? 1 : m * c.N * nrb * nr;
  const bool rom_f32 = c.mixed && o.interface != 1;   // the Eq. 47 interior bases are FP64
  FD_TRY(dalloc_t(c, &c.w_R, rom_f32 ? (rom_elems + 1) / 2 : rom_elems));
  FD_TRY(dalloc_t(c, &c.w_KR, rom_f32 ? (rom_elems + 1) / 2 : rom_elems));
  FD_TRY(dalloc_t(c, &c.w_tot, 3 * m * c.ntot));
  // Krylov storage: one restart cycle (c.kry basis vectors and preconditioned vectors per RHS)
  FD_TRY(dalloc_t(c, &c.V, (size_t)(c.kry + 1) * m * c.ntot));
  FD_TRY(dalloc_t(c, &c.Z, (size_t)c.kry * m * c.ntot));
  FD_TRY(dalloc_t(c, &c.pcg, 6 * m * c.L + 1));
  FD_TRY(dalloc(c, reinterpret_cast<void**>(&c.chk), sizeof(int)));
  if (o.interface == 1) FD_TRY(dalloc_t(c, &c.w_i, m * c.N * c.ni));
  FD_TRY(dalloc_t(c, &c.red, (size_t)m * (c.kry + 2) * 304));
  FD_TRY(dalloc_t(c, &c.scal, 64 * m + (size_t)m * (c.kry + 2) * 2));
  FD_CUDA(cudaMallocHost(&c.h_scal, sizeof(double) * (64 * m + (size_t)m * (c.kry + 2) * 2)));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  phase("workspace");
  c.t_setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return FETIDP_OK;
}

}  // namespace fetidp
