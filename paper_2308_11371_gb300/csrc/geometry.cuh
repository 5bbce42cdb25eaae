// Cell geometry and material shared by host setup and device kernels.
//
// Every cell is the image of the reference cell [0,1]^d under xi -> F(xi)
// with xi = cell index + eta (Sec. 2.2.1, Eq. 6; Sec. 4.1, Eq. 51 composed
// with an analytic macro map).  The pulled-back tensor C_hat (Eq. 52) holds
// all dependence on the map and the material:
//   C_hat_(ia)(jb) = E det J [ lam Jinv_ai Jinv_bj + mu d_ij (Jinv_a . Jinv_b)
//                              + mu Jinv_aj Jinv_bi ],
// acting on the reference gradient G_ia = du_i / dxi_a (isotropic C, plane
// strain in 2D).  Stored as the upper triangle of the symmetric d^2 x d^2
// matrix, row-major over I = i*d + a.
#pragma once
#include <cmath>

#ifdef __CUDACC__
#define FD_HD __host__ __device__ __forceinline__
#else
#define FD_HD inline
#endif

namespace fetidp {

struct Geo {
  int dim, e;
  int nc[3];            // cells per axis (nz = 1 in 2D)
  int mask_kind;        // 0 frame+diag (2D, hard), 1 BCC hard, 2 BCC sigmoid
  int map_kind;         // 0 identity, 1 bend 2D, 2 shear+bend 3D, 3 twist+bend 3D
  double mask_width, E_solid, E_void, nu;
  double mp[8];
};

constexpr double kGaussLo = 0.21132486540518711775;   // 1/2 - 1/(2 sqrt 3)
constexpr double kGaussHi = 0.78867513459481288225;   // 1/2 + 1/(2 sqrt 3)
constexpr double kPi = 3.14159265358979323846;

FD_HD double gauss_t(int bit) { return bit ? kGaussHi : kGaussLo; }

// J = dx/dxi at lattice coordinate xi (row = x component, column = xi direction).
FD_HD void macro_jacobian(const Geo& g, const double* xi, double J[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) J[a][b] = (a == b) ? 1.0 : 0.0;
  const double* p = g.mp;
  switch (g.map_kind) {
    case 1: {  // (xi_x, xi_y + a sin(pi xi_x / L))
      J[1][0] = p[0] * kPi / p[1] * cos(kPi * xi[0] / p[1]);
      break;
    }
    case 2: {  // xi + (g1 xi_z, g2 xi_z, a sin(pi xi_x / L))
      J[0][2] = p[2];
      J[1][2] = p[3];
      J[2][0] = p[0] * kPi / p[1] * cos(kPi * xi[0] / p[1]);
      break;
    }
    case 3: {  // twist about x through (yc, zc) by tau xi_x / L, then bend along z
      const double a = p[0], L = p[1], tau = p[2], yc = p[3], zc = p[4];
      const double th = tau * xi[0] / L, dth = tau / L;
      const double c = cos(th), s = sin(th);
      const double dy = xi[1] - yc, dz = xi[2] - zc;
      J[1][0] = dth * (-s * dy - c * dz);
      J[1][1] = c;
      J[1][2] = -s;
      J[2][0] = dth * (c * dy - s * dz) + a * kPi / L * cos(kPi * xi[0] / L);
      J[2][1] = s;
      J[2][2] = c;
      break;
    }
    default:
      break;
  }
}

// Distance from the cell-local point eta to the strut skeleton of the mask.
FD_HD double strut_distance(const Geo& g, const double* eta) {
  if (g.mask_kind == 0) {
    const double x = eta[0], y = eta[1];
    double m = fmin(fmin(x, 1.0 - x), fmin(y, 1.0 - y));
    const double r2 = 0.70710678118654752440;
    m = fmin(m, fabs(x - y) * r2);
    m = fmin(m, fabs(x + y - 1.0) * r2);
    return m;
  }
  // four body diagonals of the unit cube: through corner c with direction (+-1,+-1,+-1)/sqrt3
  const double inv3 = 0.57735026918962576451;
  double best = 1e300;
  for (int q = 0; q < 4; ++q) {
    double a[3] = {0.0, 0.0, 0.0};
    if (q > 0) a[q - 1] = 1.0;
    double u[3];
    for (int k = 0; k < 3; ++k) u[k] = (a[k] == 0.0 ? 1.0 : -1.0) * inv3;
    double w[3] = {eta[0] - a[0], eta[1] - a[1], eta[2] - a[2]};
    const double t = w[0] * u[0] + w[1] * u[1] + w[2] * u[2];
    double p2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double pk = w[k] - t * u[k];
      p2 += pk * pk;
    }
    best = fmin(best, sqrt(p2));
  }
  return best;
}

FD_HD double youngs(const Geo& g, double dist, double r) {
  if (g.mask_kind == 2) {
    const double z = (r - dist) / g.mask_width;
    return g.E_void + (g.E_solid - g.E_void) / (1.0 + exp(-z));
  }
  return dist <= r ? g.E_solid : g.E_void;
}

FD_HD double youngs_dr(const Geo& g, double dist, double r) {
  if (g.mask_kind != 2) return 0.0;
  const double z = (r - dist) / g.mask_width;
  const double sg = 1.0 / (1.0 + exp(-z));
  return (g.E_solid - g.E_void) * sg * (1.0 - sg) / g.mask_width;
}

// Upper triangle of C_hat (unit E scaled by E) from the Jacobian; returns count.
FD_HD int chat_upper(int d, double nu, const double J[3][3], double E, double* out) {
  double Ji[3][3];
  double det;
  if (d == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double id = 1.0 / det;
    Ji[0][0] = J[1][1] * id; Ji[0][1] = -J[0][1] * id;
    Ji[1][0] = -J[1][0] * id; Ji[1][1] = J[0][0] * id;
  } else {
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    const double id = 1.0 / det;
    Ji[0][0] = c00 * id;
    Ji[1][0] = c01 * id;
    Ji[2][0] = c02 * id;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  }
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  const double s = E * det;
  const int n = d * d;
  int c = 0;
  for (int I = 0; I < n; ++I) {
    const int i = I / d, a = I % d;
    for (int Jx = I; Jx < n; ++Jx) {
      const int j = Jx / d, b = Jx % d;
      double gab = 0.0;
      for (int k = 0; k < d; ++k) gab += Ji[a][k] * Ji[b][k];
      double v = lam * Ji[a][i] * Ji[b][j] + mu * Ji[a][j] * Ji[b][i];
      if (i == j) v += mu * gab;
      out[c++] = s * v;
    }
  }
  return c;
}

// Lattice coordinate of Gauss point gp of element (ex,ey,ez) in cell (cx,cy,cz).
FD_HD void gauss_point(const Geo& g, int cx, int cy, int cz, int ex, int ey, int ez, int gp,
                       double* eta, double* xi) {
  const double h = 1.0 / g.e;
  const int ec[3] = {ex, ey, ez};
  const int cc[3] = {cx, cy, cz};
  for (int k = 0; k < g.dim; ++k) {
    eta[k] = (ec[k] + gauss_t((gp >> k) & 1)) * h;
    xi[k] = cc[k] + eta[k];
  }
  if (g.dim == 2) { eta[2] = 0.0; xi[2] = 0.0; }
}

}  // namespace fetidp
