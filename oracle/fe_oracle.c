/*
 * CPU ORACLE -- test infrastructure only.  Nothing in the product library
 * links, includes or calls this file; only the tests, the benchmark's CPU
 * baseline and the smoke check use it.  Plain FP64 C, written for
 * obviousness, not speed.
 *
 * What it computes (Mandel et al., "Simple finite elements and multigrid
 * for efficient mass-consistent wind downscaling", Sec. 2):
 *
 *  - standard isoparametric 8-node hexahedra (Sec. 2, discretization
 *    paragraph): N_n(xi) = 1/8 prod_d (1 + xi_d xi_{n,d}), the node
 *    positions mapped by the same shape functions;
 *  - left-hand side of Eq. 5, int A^{-1} grad lambda . grad mu, with
 *    A = diag(a1^2, a2^2, a3^2) (Sec. 2, after Eq. 1), by the 2x2x2
 *    tensor Gauss rule (points +-1/sqrt(3), weights 1);
 *  - right-hand side of Eq. 5, -int grad mu . u0, by the 2x2x2 rule with u0
 *    interpolated from the nodes (primary), or by the one-point rule at the
 *    element center that the paper uses (variant);
 *  - recovery u = u0 + A^{-1} grad lambda, Eq. 3, at the element center
 *    (the same derivative code, as the paper says) or at the Gauss points;
 *  - the discrete weak divergence (B u)_m = sum_g detJ grad N_m(g) . u(g),
 *    the operator whose null space Eq. 5 enforces.
 *
 * Grid: nodes (i, j, k), 0 <= i <= nx, 0 <= j <= ny, 0 <= k <= nz, arrays
 * [k][j][i] with i fastest.  Element (i, j, k) has local node
 * n = a + 2b + 4c at grid node (i+a, j+b, k+c), reference corner
 * (2a-1, 2b-1, 2c-1).
 *
 * Return codes: 0 ok, -2 an element with detJ <= 0 at a quadrature point.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_EGEOM (-2)

static void corner(int n, double c[3]) {
  c[0] = (n & 1) ? 1.0 : -1.0;
  c[1] = (n & 2) ? 1.0 : -1.0;
  c[2] = (n & 4) ? 1.0 : -1.0;
}

/* shape functions and their reference derivatives dN[n][a] = dN_n/dxi_a */
static void shape(const double xi[3], double N[8], double dN[8][3]) {
  for (int n = 0; n < 8; ++n) {
    double c[3];
    corner(n, c);
    double f0 = 1.0 + c[0] * xi[0], f1 = 1.0 + c[1] * xi[1], f2 = 1.0 + c[2] * xi[2];
    N[n] = 0.125 * f0 * f1 * f2;
    dN[n][0] = 0.125 * c[0] * f1 * f2;
    dN[n][1] = 0.125 * f0 * c[1] * f2;
    dN[n][2] = 0.125 * f0 * f1 * c[2];
  }
}

/* J[d][a] = dx_d / dxi_a;  returns det J; Jinv = J^{-1} (Jinv[a][d] = dxi_a/dx_d) */
static double jacobian(const double xe[8][3], const double dN[8][3], double Jinv[3][3]) {
  double J[3][3] = {{0}};
  for (int n = 0; n < 8; ++n)
    for (int d = 0; d < 3; ++d)
      for (int a = 0; a < 3; ++a) J[d][a] += xe[n][d] * dN[n][a];
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  /* inverse by the cofactor formula */
  Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  return det;
}

/* physical gradients grad[n][d] = sum_a dN_n/dxi_a * dxi_a/dx_d */
static void phys_grad(const double dN[8][3], const double Jinv[3][3], double grad[8][3]) {
  for (int n = 0; n < 8; ++n)
    for (int d = 0; d < 3; ++d) {
      double s = 0.0;
      for (int a = 0; a < 3; ++a) s += dN[n][a] * Jinv[a][d];
      grad[n][d] = s;
    }
}

static void gauss_point(int g, double xi[3]) {
  double p = 1.0 / sqrt(3.0);
  xi[0] = (g & 1) ? p : -p;
  xi[1] = (g & 2) ? p : -p;
  xi[2] = (g & 4) ? p : -p;
}

static int64_t nid(int nx, int ny, int i, int j, int k) {
  return ((int64_t)k * (ny + 1) + j) * (nx + 1) + i;
}

static void gather_xe(int nx, int ny, const double* X, const double* Y, const double* Z,
                      int i, int j, int k, double xe[8][3]) {
  for (int n = 0; n < 8; ++n) {
    int64_t id = nid(nx, ny, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1));
    xe[n][0] = X[id];
    xe[n][1] = Y[id];
    xe[n][2] = Z[id];
  }
}

static void gather_u(int nx, int ny, int nz, const double* u0, int i, int j, int k,
                     double ue[8][3]) {
  int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  for (int n = 0; n < 8; ++n) {
    int64_t id = nid(nx, ny, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1));
    for (int d = 0; d < 3; ++d) ue[n][d] = u0[d * N + id];
  }
}

/* Element stiffness Ke[m][n] = sum_g detJ grad N_m . A^{-1} grad N_n (Eq. 5 left side). */
int oracle_element_stiffness(const double* xe_flat, const double* a, double* Ke) {
  const double(*xe)[3] = (const double(*)[3])xe_flat;
  memset(Ke, 0, 64 * sizeof(double));
  for (int g = 0; g < 8; ++g) {
    double xi[3], N[8], dN[8][3], Jinv[3][3], grad[8][3];
    gauss_point(g, xi);
    shape(xi, N, dN);
    double det = jacobian(xe, dN, Jinv);
    if (!(det > 0.0)) return ORACLE_EGEOM;
    phys_grad(dN, Jinv, grad);
    for (int m = 0; m < 8; ++m)
      for (int n = 0; n < 8; ++n) {
        double s = 0.0;
        for (int d = 0; d < 3; ++d) s += grad[m][d] * grad[n][d] / (a[d] * a[d]);
        Ke[m * 8 + n] += det * s;
      }
  }
  return 0;
}

/* Element load fe[m] = -int grad N_m . u0 (Eq. 5 right side).
 * quad 0: 2x2x2 Gauss with u0(g) = sum_n N_n(g) u0_n.
 * quad 1: one point at the center, weight 8, u0 at the center (mean of corners). */
int oracle_element_rhs(const double* xe_flat, const double* ue_flat, int quad, double* fe) {
  const double(*xe)[3] = (const double(*)[3])xe_flat;
  const double(*ue)[3] = (const double(*)[3])ue_flat;
  memset(fe, 0, 8 * sizeof(double));
  int ng = quad == 0 ? 8 : 1;
  for (int g = 0; g < ng; ++g) {
    double xi[3] = {0.0, 0.0, 0.0}, w = 8.0;
    if (quad == 0) { gauss_point(g, xi); w = 1.0; }
    double N[8], dN[8][3], Jinv[3][3], grad[8][3];
    shape(xi, N, dN);
    double det = jacobian(xe, dN, Jinv);
    if (!(det > 0.0)) return ORACLE_EGEOM;
    phys_grad(dN, Jinv, grad);
    double ug[3] = {0.0, 0.0, 0.0};
    for (int n = 0; n < 8; ++n)
      for (int d = 0; d < 3; ++d) ug[d] += N[n] * ue[n][d];
    for (int m = 0; m < 8; ++m) {
      double s = 0.0;
      for (int d = 0; d < 3; ++d) s += grad[m][d] * ug[d];
      fe[m] -= w * det * s;
    }
  }
  return 0;
}

/* Global stiffness as COO triplets, 64 per element, element order
 * (i fastest, then j, then k); duplicates are summed by the caller.
 * This is the full matrix before any boundary condition. */
int oracle_assemble_coo(int nx, int ny, int nz, const double* X, const double* Y,
                        const double* Z, const double* a, int64_t* rows, int64_t* cols,
                        double* vals) {
  int64_t t = 0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double xe[8][3], Ke[64];
        gather_xe(nx, ny, X, Y, Z, i, j, k, xe);
        int rc = oracle_element_stiffness(&xe[0][0], a, Ke);
        if (rc) return rc;
        for (int m = 0; m < 8; ++m) {
          int64_t r = nid(nx, ny, i + (m & 1), j + ((m >> 1) & 1), k + ((m >> 2) & 1));
          for (int n = 0; n < 8; ++n) {
            int64_t c = nid(nx, ny, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1));
            rows[t] = r;
            cols[t] = c;
            vals[t] = Ke[m * 8 + n];
            ++t;
          }
        }
      }
  return 0;
}

/* Global load vector f (all nodes, before boundary conditions). */
int oracle_assemble_rhs(int nx, int ny, int nz, const double* X, const double* Y,
                        const double* Z, const double* u0, int quad, double* f) {
  int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  memset(f, 0, N * sizeof(double));
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double xe[8][3], ue[8][3], fe[8];
        gather_xe(nx, ny, X, Y, Z, i, j, k, xe);
        gather_u(nx, ny, nz, u0, i, j, k, ue);
        int rc = oracle_element_rhs(&xe[0][0], &ue[0][0], quad, fe);
        if (rc) return rc;
        for (int m = 0; m < 8; ++m)
          f[nid(nx, ny, i + (m & 1), j + ((m >> 1) & 1), k + ((m >> 2) & 1))] += fe[m];
      }
  return 0;
}

/* One row of the full stiffness matrix at node (i, j, k): row27[s] with
 * s = (di+1) + 3(dj+1) + 9(dk+1) the coefficient of neighbor (i+di, j+dj, k+dk),
 * summed over the (up to 8) elements that contain the node. */
int oracle_stencil_row(int nx, int ny, int nz, const double* X, const double* Y,
                       const double* Z, const double* a, int i, int j, int k, double* row27) {
  memset(row27, 0, 27 * sizeof(double));
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int aa = 0; aa < 2; ++aa) {
        int ei = i - aa, ej = j - b, ek = k - c;
        if (ei < 0 || ej < 0 || ek < 0 || ei >= nx || ej >= ny || ek >= nz) continue;
        double xe[8][3], Ke[64];
        gather_xe(nx, ny, X, Y, Z, ei, ej, ek, xe);
        int rc = oracle_element_stiffness(&xe[0][0], a, Ke);
        if (rc) return rc;
        int m = aa + 2 * b + 4 * c;
        for (int n = 0; n < 8; ++n) {
          int di = (n & 1) - aa, dj = ((n >> 1) & 1) - b, dk = ((n >> 2) & 1) - c;
          row27[(di + 1) + 3 * (dj + 1) + 9 * (dk + 1)] += Ke[m * 8 + n];
        }
      }
  return 0;
}

/* y = K x with the full matrix, element by element (no matrix stored).
 * Elements are visited in 4 classes by the parities of (j, k); two element
 * rows (j, k) of one class share no node, so the rows of a class may run in
 * parallel. */
int oracle_apply_K(int nx, int ny, int nz, const double* X, const double* Y, const double* Z,
                   const double* a, const double* x, double* y) {
  int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  memset(y, 0, N * sizeof(double));
  int bad = 0;
  for (int cls = 0; cls < 4; ++cls) {
    int pj = cls & 1, pk = cls >> 1;
    int nj = (ny - pj + 1) / 2, nk = (nz - pk + 1) / 2;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (int64_t q = 0; q < (int64_t)nj * nk; ++q) {
      int j = pj + 2 * (int)(q % nj), k = pk + 2 * (int)(q / nj);
      for (int i = 0; i < nx; ++i) {
        double xe[8][3], Ke[64];
        gather_xe(nx, ny, X, Y, Z, i, j, k, xe);
        if (oracle_element_stiffness(&xe[0][0], a, Ke)) { bad = 1; continue; }
        int64_t id[8];
        for (int n = 0; n < 8; ++n)
          id[n] = nid(nx, ny, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1));
        for (int m = 0; m < 8; ++m) {
          double sum = 0.0;
          for (int n = 0; n < 8; ++n) sum += Ke[m * 8 + n] * x[id[n]];
          y[id[m]] += sum;
        }
      }
    }
  }
  return bad ? ORACLE_EGEOM : 0;
}

/* Same as oracle_assemble_rhs, the element rows in 4 parity classes of
 * (j, k) as in oracle_apply_K, rows of a class in parallel. */
int oracle_assemble_rhs_par(int nx, int ny, int nz, const double* X, const double* Y,
                            const double* Z, const double* u0, int quad, double* f) {
  int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  memset(f, 0, N * sizeof(double));
  int bad = 0;
  for (int cls = 0; cls < 4; ++cls) {
    int pj = cls & 1, pk = cls >> 1;
    int nj = (ny - pj + 1) / 2, nk = (nz - pk + 1) / 2;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (int64_t q = 0; q < (int64_t)nj * nk; ++q) {
      int j = pj + 2 * (int)(q % nj), k = pk + 2 * (int)(q / nj);
      for (int i = 0; i < nx; ++i) {
        double xe[8][3], ue[8][3], fe[8];
        gather_xe(nx, ny, X, Y, Z, i, j, k, xe);
        gather_u(nx, ny, nz, u0, i, j, k, ue);
        if (oracle_element_rhs(&xe[0][0], &ue[0][0], quad, fe)) { bad = 1; continue; }
        for (int m = 0; m < 8; ++m)
          f[nid(nx, ny, i + (m & 1), j + ((m >> 1) & 1), k + ((m >> 2) & 1))] += fe[m];
      }
    }
  }
  return bad ? ORACLE_EGEOM : 0;
}

/* u = u0 + A^{-1} grad lambda (Eq. 3).
 * where 0: at element centers, u[3][nz][ny][nx].
 * where 1: at the 8 Gauss points, u[3][8][nz][ny][nx] (g = gx + 2gy + 4gz,
 *          gx = 0 for xi = -1/sqrt(3)). */
int oracle_recover(int nx, int ny, int nz, const double* X, const double* Y, const double* Z,
                   const double* u0, const double* lam, const double* a, int where, double* u) {
  int64_t NE = (int64_t)nx * ny * nz;
  int ng = where == 0 ? 1 : 8;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double xe[8][3], ue[8][3], le[8];
        gather_xe(nx, ny, X, Y, Z, i, j, k, xe);
        gather_u(nx, ny, nz, u0, i, j, k, ue);
        for (int n = 0; n < 8; ++n)
          le[n] = lam[nid(nx, ny, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1))];
        int64_t e = ((int64_t)k * ny + j) * nx + i;
        for (int g = 0; g < ng; ++g) {
          double xi[3] = {0.0, 0.0, 0.0}, N[8], dN[8][3], Jinv[3][3], grad[8][3];
          if (where == 1) gauss_point(g, xi);
          shape(xi, N, dN);
          double det = jacobian(xe, dN, Jinv);
          if (!(det > 0.0)) { bad = 1; continue; }
          phys_grad(dN, Jinv, grad);
          for (int d = 0; d < 3; ++d) {
            double u0p = 0.0, gl = 0.0;
            for (int n = 0; n < 8; ++n) {
              u0p += N[n] * ue[n][d];
              gl += le[n] * grad[n][d];
            }
            u[((int64_t)d * ng + g) * NE + e] = u0p + gl / (a[d] * a[d]);
          }
        }
      }
  return bad ? ORACLE_EGEOM : 0;
}

/* (B u)_m = sum_e sum_g detJ grad N_m(g) . u_e(g), u given at the Gauss
 * points as u[3][8][nz][ny][nx]; out is nodal, all nodes. */
int oracle_weak_div(int nx, int ny, int nz, const double* X, const double* Y, const double* Z,
                    const double* ug, double* out) {
  int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  int64_t NE = (int64_t)nx * ny * nz;
  memset(out, 0, N * sizeof(double));
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double xe[8][3];
        gather_xe(nx, ny, X, Y, Z, i, j, k, xe);
        int64_t e = ((int64_t)k * ny + j) * nx + i;
        for (int g = 0; g < 8; ++g) {
          double xi[3], N[8], dN[8][3], Jinv[3][3], grad[8][3];
          gauss_point(g, xi);
          shape(xi, N, dN);
          double det = jacobian(xe, dN, Jinv);
          if (!(det > 0.0)) return ORACLE_EGEOM;
          phys_grad(dN, Jinv, grad);
          for (int m = 0; m < 8; ++m) {
            double s = 0.0;
            for (int d = 0; d < 3; ++d) s += grad[m][d] * ug[((int64_t)d * 8 + g) * NE + e];
            out[nid(nx, ny, i + (m & 1), j + ((m >> 1) & 1), k + ((m >> 2) & 1))] += det * s;
          }
        }
      }
  return 0;
}

/* Gauss-Seidel smoothing sweep of the multigrid cycle (Sec. 3): vertical
 * sweeps through each column of nodes, the columns taken in 4 horizontal
 * groups by the parities of (i, j): group (i mod 2) + 2 (j mod 2).
 * direction 0: groups 0,1,2,3 and each column bottom-up;
 * direction 1: groups 3,2,1,0 and each column top-down (the reverse order).
 * Only free nodes are updated: 1 <= i <= Nx-2, 1 <= j <= Ny-2,
 * 0 <= k <= Nz-2 on a grid of Nx x Ny x Nz nodes.  The matrix is CSR over
 * all nodes with node id (k*Ny + j)*Nx + i; entries that couple to fixed
 * (Dirichlet) nodes multiply their stored value, which the caller keeps 0. */
void oracle_gs_sweep(int Nx, int Ny, int Nz, const int64_t* indptr, const int64_t* indices,
                     const double* data, const double* f, double* x, int direction) {
  for (int gi = 0; gi < 4; ++gi) {
    int group = direction == 0 ? gi : 3 - gi;
    int pi = group & 1, pj = group >> 1;
    for (int j = 1; j <= Ny - 2; ++j) {
      if ((j & 1) != pj) continue;
      for (int i = 1; i <= Nx - 2; ++i) {
        if ((i & 1) != pi) continue;
        for (int kk = 0; kk <= Nz - 2; ++kk) {
          int k = direction == 0 ? kk : Nz - 2 - kk;
          int64_t r = ((int64_t)k * Ny + j) * Nx + i;
          double diag = 0.0, s = f[r];
          for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p) {
            if (indices[p] == r) diag += data[p];
            else s -= data[p] * x[indices[p]];
          }
          x[r] = s / diag;
        }
      }
    }
  }
}

/* detJ at the 8 Gauss points of every element: detj[8][nz][ny][nx]. */
int oracle_gauss_detj(int nx, int ny, int nz, const double* X, const double* Y, const double* Z,
                      double* detj) {
  int64_t NE = (int64_t)nx * ny * nz;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double xe[8][3];
        gather_xe(nx, ny, X, Y, Z, i, j, k, xe);
        int64_t e = ((int64_t)k * ny + j) * nx + i;
        for (int g = 0; g < 8; ++g) {
          double xi[3], N[8], dN[8][3], Jinv[3][3];
          gauss_point(g, xi);
          shape(xi, N, dN);
          detj[(int64_t)g * NE + e] = jacobian(xe, dN, Jinv);
        }
      }
  return 0;
}

/* nodal field interpolated to the Gauss points: ug[3][8][nz][ny][nx]. */
int oracle_interp_gauss(int nx, int ny, int nz, const double* u0, double* ug) {
  int64_t NE = (int64_t)nx * ny * nz;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double ue[8][3];
        gather_u(nx, ny, nz, u0, i, j, k, ue);
        int64_t e = ((int64_t)k * ny + j) * nx + i;
        for (int g = 0; g < 8; ++g) {
          double xi[3], N[8], dN[8][3];
          gauss_point(g, xi);
          shape(xi, N, dN);
          for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int n = 0; n < 8; ++n) s += N[n] * ue[n][d];
            ug[((int64_t)d * 8 + g) * NE + e] = s;
          }
        }
      }
  return 0;
}

/* Load vector for a wind given at the element centers, uc[3][nz][ny][nx]
 * (the paper's representation of the wind, Sec. 2): the wind is constant over
 * each element, so the element routine gets the center value at all 8 nodes. */
int oracle_assemble_rhs_centers(int nx, int ny, int nz, const double* X, const double* Y,
                                const double* Z, const double* uc, int quad, double* f) {
  int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  int64_t NE = (int64_t)nx * ny * nz;
  memset(f, 0, N * sizeof(double));
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double xe[8][3], ue[8][3], fe[8];
        int64_t e = ((int64_t)k * ny + j) * nx + i;
        gather_xe(nx, ny, X, Y, Z, i, j, k, xe);
        for (int n = 0; n < 8; ++n)
          for (int d = 0; d < 3; ++d) ue[n][d] = uc[d * NE + e];
        int rc = oracle_element_rhs(&xe[0][0], &ue[0][0], quad, fe);
        if (rc) return rc;
        for (int m = 0; m < 8; ++m)
          f[nid(nx, ny, i + (m & 1), j + ((m >> 1) & 1), k + ((m >> 2) & 1))] += fe[m];
      }
  return 0;
}
