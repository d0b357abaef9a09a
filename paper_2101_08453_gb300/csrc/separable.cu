// Separable (column x layer) operator of a terrain-following grid in shift
// form, z = z_s(x, y) + zeta_k (Sec. 2), and the float32 cycle kernels that
// rebuild the 27-point rows from it (MCWIND_OP_SEPARABLE).
//
// Why it is exact.  In an element of layer l (thickness h = zeta_{l+1} -
// zeta_l) the isoparametric map is x = X(xi1, xi2), y = Y(xi1, xi2),
// z = Z_s(xi1, xi2) + zeta_l + h (1 + xi3) / 2, so with J2 the 2 x 2
// horizontal Jacobian, j2 = det J2, adj its adjugate, D = diag(a^-2) and
// z' = (dZ_s/dxi1, dZ_s/dxi2):
//   det J = (h/2) j2,  d/dz = (2/h) d/dxi3,
//   d/d(x, y) = J2^-T (d/d(xi1, xi2) - z' (2/h) d/dxi3),
// and the 2x2x2-Gauss stiffness integrand of Eq. 5 splits into
//   (h/2) grad_h N_m . W grad_h N_n - (grad_h N_m . W z') N_n,3
//     - N_m,3 (z' . W grad_h N_n) + (2/h) (z' . W z' + c3 j2) N_m,3 N_n,3,
// W = adj D adj^T / j2, every horizontal factor a function of (xi1, xi2) and
// every vertical one a fixed 1-D integral.  Hence K_e = (h/2) Phat (x) m -
// Qhat (x) g - Qhat^T (x) g^T + (2/h) Rhat (x) kappa, m = [[2,1],[1,2]]/3,
// g = [[-1,1],[-1,1]]/2, kappa = [[1,-1],[-1,1]]/2, and after assembly
//   K = H_P (x) V_M + H_Q (x) V_G + H_Q^T (x) V_G^T + H_R (x) V_K,
// a sum the tensor-product prolongation of Sec. 3 keeps on every level
// (P^T (H (x) V) P = (Ph^T H Ph) (x) (Pv^T V Pv)).  The factor layout is
// described in internal.cuh.
#include "async.cuh"
#include "kernels.cuh"

namespace mcw {
namespace {

constexpr int kShiftFlag = 8;

__device__ __forceinline__ bool free_column(const Grid& g, int i, int j) {
  return i >= 1 && i <= g.Nx - 2 && j >= 1 && j <= g.Ny - 2;
}

// ---------------------------------------------------------------- set-up

// flag |= 8 unless X and Y do not depend on k and Z(i,j,k) - Z(i,j,0) equals
// Z(0,0,k) - Z(0,0,0), to 1e-10 of the coordinates' magnitude (the
// generator's rounding of z_s + zeta is far below it).  Standard layout.
__global__ void k_shift_check(int Nx, int Ny, int Nz, const double* __restrict__ X,
                              const double* __restrict__ Y, const double* __restrict__ Z,
                              int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= Nx || j >= Ny) return;
  const int64_t lay = (int64_t)Nx * Ny;
  const int64_t c = (int64_t)j * Nx + i;
  const double x0 = X[c], y0 = Y[c], z0 = Z[c], zb = Z[0];
  bool ok = true;
  for (int k = 1; k < Nz; ++k) {
    const double xk = X[k * lay + c], yk = Y[k * lay + c], zk = Z[k * lay + c], zr = Z[k * lay];
    const double tol = 1e-10 * (fabs(x0) + fabs(y0) + fabs(zk) + fabs(z0) + fabs(zr) + fabs(zb));
    ok = ok && fabs(xk - x0) <= tol && fabs(yk - y0) <= tol && fabs((zk - z0) - (zr - zb)) <= tol;
  }
  if (!ok) atomicOr(flag, kShiftFlag);
}

// Horizontal factors of the cells of one parity class (cell (ci, cj) with
// ci & 1 = cls & 1, cj & 1 = cls >> 1), added into the float64 planes of
// their 4 corner columns: cells of one class share no corner, and the four
// classes run in order, so every sum is formed in one fixed order.  2 x 2
// Gauss points in (xi1, xi2), float64.  Corner p = a + 2b is node
// (ci + a, cj + b) of the ground layer (standard layout).
__global__ void __launch_bounds__(128) k_hfactor_cells(Grid g, int cls, const double* __restrict__ X,
                                                       const double* __restrict__ Y,
                                                       const double* __restrict__ Z, double c1,
                                                       double c2, double c3,
                                                       double* __restrict__ H, int* flag) {
  const int ci = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + (cls & 1);
  const int cj = 2 * (blockIdx.y * blockDim.y + threadIdx.y) + (cls >> 1);
  if (ci >= g.Nx - 1 || cj >= g.Ny - 1) return;
  double xs[4], ys[4], zs[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int64_t n = (int64_t)(cj + (p >> 1)) * g.Nx + ci + (p & 1);
    xs[p] = X[n]; ys[p] = Y[n]; zs[p] = Z[n];
  }
  double P[4][4], Q[4][4], R[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) P[p][q] = Q[p][q] = R[p][q] = 0.0;
  const double gp = 0.57735026918962576451;  // 1/sqrt(3)
  bool bad = false;
#pragma unroll
  for (int gq = 0; gq < 4; ++gq) {
    const double e1 = (gq & 1) ? gp : -gp, e2 = (gq & 2) ? gp : -gp;
    double phi[4], d1[4], d2[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const double sx = (p & 1) ? 1.0 : -1.0, sy = (p & 2) ? 1.0 : -1.0;
      phi[p] = 0.25 * (1.0 + sx * e1) * (1.0 + sy * e2);
      d1[p] = 0.25 * sx * (1.0 + sy * e2);
      d2[p] = 0.25 * sy * (1.0 + sx * e1);
    }
    double J00 = 0, J01 = 0, J10 = 0, J11 = 0, z1 = 0, z2 = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      J00 += xs[p] * d1[p]; J01 += xs[p] * d2[p];
      J10 += ys[p] * d1[p]; J11 += ys[p] * d2[p];
      z1 += zs[p] * d1[p]; z2 += zs[p] * d2[p];
    }
    const double j2 = J00 * J11 - J01 * J10;
    bad = bad || !(j2 > 0.0);
    const double ij = 1.0 / j2;
    // W = adj D adj^T / j2 with adj = [[J11, -J01], [-J10, J00]]
    const double W00 = (c1 * J11 * J11 + c2 * J01 * J01) * ij;
    const double W01 = -(c1 * J11 * J10 + c2 * J01 * J00) * ij;
    const double W11 = (c1 * J10 * J10 + c2 * J00 * J00) * ij;
    const double v1 = W00 * z1 + W01 * z2, v2 = W01 * z1 + W11 * z2;  // W z'
    const double s = z1 * v1 + z2 * v2 + c3 * j2;
    double wg1[4], wg2[4], u[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      wg1[p] = W00 * d1[p] + W01 * d2[p];
      wg2[p] = W01 * d1[p] + W11 * d2[p];
      u[p] = d1[p] * v1 + d2[p] * v2;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        P[p][q] += d1[p] * wg1[q] + d2[p] * wg2[q];
        Q[p][q] += u[p] * phi[q];
        R[p][q] += s * phi[p] * phi[q];
      }
  }
  if (bad) atomicOr(flag, 1);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int64_t col = gidx(g, ci + (p & 1), cj + (p >> 1), 0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int s2 = ((q & 1) - (p & 1) + 1) + 3 * ((q >> 1) - (p >> 1) + 1);
      H[(0 * 9 + s2) * g.PP + col] += P[p][q];
      H[(1 * 9 + s2) * g.PP + col] -= Q[p][q];
      H[(2 * 9 + s2) * g.PP + col] -= Q[q][p];
      H[(3 * 9 + s2) * g.PP + col] += R[p][q];
    }
  }
}

// Zero the couplings that touch a fixed column (and everything of padding
// columns) in the float64 planes and write the float32 tiles.  One thread
// per split-layout column: blockIdx.z = parity of i.
__global__ void __launch_bounds__(128) k_hfactor_finalize(Grid g, double* __restrict__ H,
                                                          float* __restrict__ H32) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int par = (int)blockIdx.z;
  if (h >= g.H || j >= g.Ny) return;
  const int i = 2 * h + par;
  const int64_t col = (int64_t)j * g.RP + (int64_t)par * g.H + h;
  const bool fc = i < g.Nx && free_column(g, i, j);
#pragma unroll
  for (int q = 0; q < kHF; ++q) {
    const int s2 = q % 9;
    const bool keep = fc && free_column(g, i + s2 % 3 - 1, j + s2 / 3 - 1);
    const double v = keep ? H[q * g.PP + col] : 0.0;
    H[q * g.PP + col] = v;
    H32[hidx(col, q)] = (float)v;
  }
}

// One direction (DIM 0: x, 1: y) of the horizontal Galerkin product
// Ph^T H_t Ph, for all four terms: out(I; D, e) = sum_a w_a sum_d
// H(f_I + a; d, e) P(f_I + a + d, I + D) with the interpolation weights of
// Sec. 3 (a, d, D in {-1, 0, 1}; e the offset in the other direction).  One
// thread per output column, float64; inputs outside the grid have weight 0.
template <int DIM>
__global__ void __launch_bounds__(128) k_hgalerkin(Grid gin, Grid gout,
                                                   const double* __restrict__ Hin,
                                                   double* __restrict__ Hout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= gout.Nx || j >= gout.Ny) return;
  const int Iout = DIM == 0 ? i : j;
  const int Nf = DIM == 0 ? gin.Nx : gin.Ny;
  const int Nc = DIM == 0 ? gout.Nx : gout.Ny;
  int f;
  double wa[3];
  hcoarse(1, Nf, Nc, Iout, f, wa[0], wa[2]);
  wa[1] = 1.0;
  double Pw[5][3];  // Pw[q][D] = P(f + q - 2, Iout + D - 1)
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int b = f + q - 2;
    int c0 = -100, c1 = -100;
    double w0 = 0.0, w1 = 0.0;
    if (b >= 0 && b <= Nf - 1) hpair(1, Nf, Nc, b, c0, w0, c1, w1);
#pragma unroll
    for (int D = 0; D < 3; ++D) {
      const int J = Iout + D - 1;
      Pw[q][D] = (c0 == J ? w0 : 0.0) + (c1 == J && c1 != c0 ? w1 : 0.0);
    }
  }
  const int64_t o = gidx(gout, i, j, 0);
  for (int t = 0; t < 4; ++t) {
    double acc[9];
#pragma unroll
    for (int s = 0; s < 9; ++s) acc[s] = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (wa[a] == 0.0) continue;
      const int ii = DIM == 0 ? f + a - 1 : i, jj = DIM == 1 ? f + a - 1 : j;
      const int64_t in = gidx(gin, ii, jj, 0);
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        const int d = DIM == 0 ? s % 3 : s / 3, e = DIM == 0 ? s / 3 : s % 3;
        const double v = wa[a] * Hin[(t * 9 + s) * gin.PP + in];
#pragma unroll
        for (int D = 0; D < 3; ++D) {
          const double w = Pw[a + d][D];
          if (w != 0.0) acc[DIM == 0 ? D + 3 * e : e + 3 * D] += v * w;
        }
      }
    }
#pragma unroll
    for (int s = 0; s < 9; ++s) Hout[(t * 9 + s) * gout.PP + o] = acc[s];
  }
}

// Vertical factors of the finest level from the layer thicknesses of
// column (0, 0) (standard layout Z): element l adds (h/2) m, g and (2/h)
// kappa to layers l, l+1.  One thread.  Couplings to the top layer (fixed)
// are zero.
__global__ void k_vfactor0(int Nx, int Ny, int Nz, const double* __restrict__ Z,
                           double* __restrict__ V, float* __restrict__ V32) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int64_t lay = (int64_t)Nx * Ny;
  for (int q = 0; q < Nz * kVF; ++q) V[q] = 0.0;
  for (int l = 0; l + 1 < Nz; ++l) {
    const double h = Z[(int64_t)(l + 1) * lay] - Z[(int64_t)l * lay];
    double* lo = V + l * kVF;        // row l
    double* up = V + (l + 1) * kVF;  // row l + 1
    // term 0: (h/2) [[2,1],[1,2]]/3
    lo[1] += h / 3.0; lo[2] += h / 6.0; up[0] += h / 6.0; up[1] += h / 3.0;
    // term 1: g = [[-1,1],[-1,1]]/2; term 2: its transpose
    lo[3 + 1] -= 0.5; lo[3 + 2] += 0.5; up[3 + 0] -= 0.5; up[3 + 1] += 0.5;
    lo[6 + 1] -= 0.5; lo[6 + 2] -= 0.5; up[6 + 0] += 0.5; up[6 + 1] += 0.5;
    // term 3: (2/h) [[1,-1],[-1,1]]/2
    lo[9 + 1] += 1.0 / h; lo[9 + 2] -= 1.0 / h; up[9 + 0] -= 1.0 / h; up[9 + 1] += 1.0 / h;
  }
  for (int t = 0; t < 4; ++t) {
    V[(Nz - 2) * kVF + 3 * t + 2] = 0.0;
    for (int d = 0; d < 3; ++d) V[(Nz - 1) * kVF + 3 * t + d] = 0.0;
  }
  for (int q = 0; q < Nz * kVF; ++q) V32[q] = (float)V[q];
}

// Vertical Galerkin product Pv^T V_t Pv with the layer map of the transfer
// (same form as the horizontal stage); one thread per coarse layer.
__global__ void k_vgalerkin(Transfer tr, const double* __restrict__ Vf, double* __restrict__ Vc,
                            float* __restrict__ Vc32) {
  const int K = threadIdx.x;
  if (K >= tr.Nzc) return;
  const int f = tr.kf[K];
  double wa[3];
  wa[0] = (K > 0 && tr.kf[K] - tr.kf[K - 1] == 2) ? 0.5 : 0.0;
  wa[1] = 1.0;
  wa[2] = (K < tr.Nzc - 1 && tr.kf[K + 1] - tr.kf[K] == 2) ? 0.5 : 0.0;
  double Pw[5][3];
  for (int q = 0; q < 5; ++q) {
    const int b = f + q - 2;
    int c0 = -100, c1 = -100;
    double w0 = 0.0, w1 = 0.0;
    if (b >= 0 && b <= tr.Nzf - 1) { c0 = tr.kc0[b]; c1 = tr.kc1[b]; w0 = tr.kw0[b]; w1 = tr.kw1[b]; }
    for (int D = 0; D < 3; ++D) {
      const int J = K + D - 1;
      Pw[q][D] = (c0 == J ? w0 : 0.0) + (c1 == J && c1 != c0 ? w1 : 0.0);
    }
  }
  double acc[kVF];
  for (int q = 0; q < kVF; ++q) acc[q] = 0.0;
  for (int a = 0; a < 3; ++a) {
    if (wa[a] == 0.0) continue;
    const int k = f + a - 1;
    for (int t = 0; t < 4; ++t)
      for (int d = 0; d < 3; ++d) {
        const double v = wa[a] * Vf[k * kVF + 3 * t + d];
        for (int D = 0; D < 3; ++D) acc[3 * t + D] += v * Pw[a + d][D];
      }
  }
  for (int t = 0; t < 4; ++t) {
    if (K == tr.Nzc - 1) acc[3 * t] = acc[3 * t + 1] = acc[3 * t + 2] = 0.0;
    if (K == tr.Nzc - 2) acc[3 * t + 2] = 0.0;
  }
  for (int q = 0; q < kVF; ++q) {
    Vc[K * kVF + q] = acc[q];
    Vc32[K * kVF + q] = (float)acc[q];
  }
}

// Expanded 27-point rows from float64 factors into the tiled float64
// operator (planes 0..26; plane 27 is set by the stencil finalization).
// One thread per node, blockIdx.z = 2 k + parity.
__global__ void __launch_bounds__(128) k_sep_expand64(Grid g, const double* __restrict__ H,
                                                      const double* __restrict__ V,
                                                      double* __restrict__ C) {
  const int hh = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z >> 1, par = blockIdx.z & 1;
  if (hh >= g.H || j >= g.Ny) return;
  const int64_t col = (int64_t)j * g.RP + (int64_t)par * g.H + hh;
  const int64_t b = (int64_t)k * g.PP + col;
#pragma unroll
  for (int s = 0; s < 27; ++s) {
    const int s2 = s % 9, dk = s / 9;
    double c = 0.0;
#pragma unroll
    for (int t = 0; t < 4; ++t) c += H[(t * 9 + s2) * g.PP + col] * V[k * kVF + 3 * t + dk];
    C[cidx(b, s)] = c;
  }
}

// Rows from the factors in the standard layout [27][Nz][Ny][Nx] (the level
// stencil export): float64 factors in float64, float32 factors in float32.
template <typename T>
__global__ void __launch_bounds__(128) k_sep_export(Grid g, const T* __restrict__ H,
                                                    const T* __restrict__ V,
                                                    double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.Nx || j >= g.Ny) return;
  const int64_t col = gidx(g, i, j, 0);
  const int64_t n = (int64_t)g.Nx * g.Ny * g.Nz;
  const int64_t o = ((int64_t)k * g.Ny + j) * g.Nx + i;
#pragma unroll
  for (int s = 0; s < 27; ++s) {
    const int s2 = s % 9, dk = s / 9;
    T c = T(0);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const T hv = sizeof(T) == 8 ? H[(t * 9 + s2) * g.PP + col] : H[hidx(col, t * 9 + s2)];
      c += hv * V[k * kVF + 3 * t + dk];
    }
    out[s * n + o] = (double)c;
  }
}

// ---------------------------------------------------------------- cycle

// In-row offsets of the 9 columns around split-layout column (i, j):
// c = (di+1) + 3 (dj+1).  A neighbour across i flips the parity half.
__device__ __forceinline__ void column_offsets(const Grid& g, int i, int off[9]) {
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const int ii = i + c % 3 - 1, dj = c / 3 - 1;
    off[c] = dj * (int)g.RP + ((ii & 1) - (i & 1)) * g.H + ((ii >> 1) - (i >> 1));
  }
}

// Gauss-Seidel of Sec. 3 on the separable float32 operator, one column
// group per launch, one thread per column, the layers bottom-up (UP) or
// top-down.  Per layer k' the thread forms the four neighbour sums
// y_t(k') = sum_{d != 0} H_t(c, c + d) x(c + d, k') once (they serve rows
// k'-1, k', k'+1), so a row costs 32 + 12 products plus the center column's
// three couplings sum_t H_t(c, c) V_t(k, k + dk).  The column's 36 factors
// stay in registers; per node the launch reads f, the 9 x values of the
// layer two ahead (issued before the row's store) and writes one value.
template <bool UP>
__global__ void __launch_bounds__(256) k_gs_sep(Grid g, const float* __restrict__ H,
                                                const float* __restrict__ V,
                                                const float* __restrict__ f,
                                                float* __restrict__ x, int pi, int pj) {
  const int ih = blockIdx.x * blockDim.x + threadIdx.x;
  const int jh = blockIdx.y * blockDim.y + threadIdx.y;
  const int i = 2 * ih + pi, j = 2 * jh + pj;
  if (i < 1 || i > g.Nx - 2 || j < 1 || j > g.Ny - 2) return;
  int off[9];
  column_offsets(g, i, off);
  const int64_t own = (int64_t)j * g.RP + (int64_t)(i & 1) * g.H + (i >> 1);
  float hf[4][9];
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int c = 0; c < 9; ++c) hf[t][c] = H[hidx(own, 9 * t + c)];
  const int64_t PP = g.PP;
  const int Nz = g.Nz;
  float nb[9];
  auto load = [&](int k) {
    const float* xl = x + (int64_t)k * PP + own;
#pragma unroll
    for (int c = 0; c < 9; ++c) nb[c] = xl[off[c]];
  };
  auto nsum = [&](float y[4]) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float s = 0.0f;
#pragma unroll
      for (int c = 0; c < 9; ++c)
        if (c != 4) s = fmaf(hf[t][c], nb[c], s);
      y[t] = s;
    }
  };
  float Yn[4], Y0[4], Yf[4];  // neighbour sums: the layer behind, this one, the one ahead
  float xn_behind = 0.0f, x_ahead = 0.0f;
  const int kfirst = UP ? 0 : Nz - 2;
  const int step = UP ? 1 : -1;
#pragma unroll
  for (int t = 0; t < 4; ++t) Yn[t] = 0.0f;
  if (UP) {
    load(0);
    nsum(Y0);
    load(1);
    nsum(Yf);
    x_ahead = nb[4];
  } else {
    // the top layer is fixed: x = 0 there and its couplings are zero
#pragma unroll
    for (int t = 0; t < 4; ++t) Yn[t] = 0.0f;
    load(kfirst);
    nsum(Y0);
    if (kfirst >= 1) {
      load(kfirst - 1);
      nsum(Yf);
      x_ahead = nb[4];
    } else {
#pragma unroll
      for (int t = 0; t < 4; ++t) Yf[t] = 0.0f;
    }
  }
  // behind / ahead in V's offsets: UP reads dk = -1 behind, +1 ahead
  const int vb = UP ? 0 : 2, va = UP ? 2 : 0;
  for (int q = 0, k = kfirst; q <= Nz - 2; ++q, k += step) {
    const int k2 = k + 2 * step;
    const bool more = UP ? (k2 <= Nz - 1) : (k2 >= 0);
    if (more) load(k2);
    const float* v = V + k * kVF;
    float acc = f[(int64_t)k * PP + own];
    // the layer behind the sweep first, the layer ahead (loaded last) last
#pragma unroll
    for (int t = 0; t < 4; ++t) acc = fmaf(-v[3 * t + vb], Yn[t], acc);
#pragma unroll
    for (int t = 0; t < 4; ++t) acc = fmaf(-v[3 * t + 1], Y0[t], acc);
#pragma unroll
    for (int t = 0; t < 4; ++t) acc = fmaf(-v[3 * t + va], Yf[t], acc);
    float kb = 0.0f, dg = 0.0f, ka = 0.0f;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      kb = fmaf(hf[t][4], v[3 * t + vb], kb);
      dg = fmaf(hf[t][4], v[3 * t + 1], dg);
      ka = fmaf(hf[t][4], v[3 * t + va], ka);
    }
    acc = fmaf(-kb, xn_behind, acc);
    acc = fmaf(-ka, x_ahead, acc);
    const float xn = acc / dg;
    x[(int64_t)k * PP + own] = xn;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      Yn[t] = Y0[t];
      Y0[t] = Yf[t];
    }
    xn_behind = xn;
    if (more) {
      nsum(Yf);
      x_ahead = nb[4];
    } else {
#pragma unroll
      for (int t = 0; t < 4; ++t) Yf[t] = 0.0f;
      x_ahead = 0.0f;
    }
  }
}

// The same sweep with the x values staged through shared memory.  A block
// owns kGsR rows x 32 same-group columns; for every free layer it needs the
// x values of rows j0-1 .. j0+2kGsR-1, both parity halves, half-row indices
// [h0-4, h0+36) (the 9 columns around each of its columns; 16-byte aligned
// windows), and f of its own columns.  Warp 0 copies those with bulk
// asynchronous copies (one per half-row segment) into a ring of kStages
// shared-memory stages, kStages-1 layers ahead of the layer in use, each
// stage's arrival counted in bytes on its mbarrier.  The threads read their
// 9 neighbours from the stage, so a block keeps about 10 KB of loads in
// flight with no registers held for them.  Only this group's columns are
// written in the launch, and a thread needs the old x of other groups' columns
// and of its own column above (below) the row it updates, so the staged
// values are the ones the sweep must read.  A wait that runs out sets the
// status bit and ends the block (after waiting, bounded, for its copies).
constexpr int kGsR = 4;
constexpr int kTileRows = 2 * kGsR + 1;
constexpr int kTileW = 40;
constexpr int kStageX = kTileRows * 2 * kTileW;
constexpr int kStage = kStageX + kGsR * 32;
constexpr int kStages = 8;

template <bool UP>
__global__ void __launch_bounds__(32 * kGsR) k_gs_sep_staged(Grid g, const float* __restrict__ H,
                                                            const float* __restrict__ V,
                                                            const float* __restrict__ f,
                                                            float* __restrict__ x, int pi, int pj,
                                                            int* status) {
  __shared__ __align__(128) float tile[kStages][kStage];
  __shared__ __align__(8) uint64_t bar[kStages];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int h0 = blockIdx.x * 32;
  const int j0 = 2 * kGsR * blockIdx.y + pj;
  const int h = h0 + tx, j = j0 + 2 * ty, i = 2 * h + pi;
  const bool active = i >= 1 && i <= g.Nx - 2 && j >= 1 && j <= g.Ny - 2;
  const int nlay = g.Nz - 1;  // free layers; the top layer is fixed (x = 0)
  const int64_t PP = g.PP;
  if (ty == 0 && tx == 0) {
    for (int q = 0; q < kStages; ++q) mbar_init(&bar[q], 1);
    fence_barrier_init();
  }
  __syncthreads();
  // warp 0: the copies of free layer number t (sweep order) into stage t % kStages
  auto issue = [&](int t) {
    const int k = UP ? t : nlay - 1 - t;
    float* st = tile[t % kStages];
    const int q = tx;
    const float* src = nullptr;
    float* dst = nullptr;
    uint32_t bytes = 0;
    if (q < 2 * kTileRows) {
      const int r = q >> 1, par = q & 1, jj = j0 - 1 + r;
      const int lo = max(h0 - 4, 0), hi = min(h0 + 36, g.H);
      if (jj >= 0 && jj < g.Ny) {
        src = x + (int64_t)k * PP + (int64_t)jj * g.RP + (int64_t)par * g.H + lo;
        dst = st + (r * 2 + par) * kTileW + (lo - (h0 - 4));
        bytes = (uint32_t)(hi - lo) * 4u;
      }
    } else if (q < 2 * kTileRows + kGsR) {
      const int r = q - 2 * kTileRows, jj = j0 + 2 * r;
      if (jj < g.Ny) {
        src = f + (int64_t)k * PP + (int64_t)jj * g.RP + (int64_t)pi * g.H + h0;
        dst = st + kStageX + r * 32;
        bytes = 128u;
      }
    }
    const uint32_t total = __reduce_add_sync(0xffffffffu, bytes);
    if (q == 0) mbar_arrive_expect_tx(&bar[t % kStages], total);
    __syncwarp();
    if (bytes) bulk_copy_g2s(dst, src, bytes, &bar[t % kStages]);
  };
  int issued = 0;
  if (ty == 0) {
    for (int t = 0; t < kStages - 1 && t < nlay; ++t) issue(t);
    issued = min(kStages - 1, nlay);
  }
  const int64_t own = (int64_t)j * g.RP + (int64_t)pi * g.H + h;
  float hf[4][9];
  int toff[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const int ii = i + c % 3 - 1, r = 2 * ty + 1 + c / 3 - 1;
    toff[c] = (r * 2 + (ii & 1)) * kTileW + ((ii >> 1) - (h0 - 4));
  }
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int c = 0; c < 9; ++c) hf[t][c] = active ? H[hidx(own, 9 * t + c)] : 0.0f;
  const int vb = UP ? 0 : 2, va = UP ? 2 : 0;
  float Yb[4], Yc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) Yb[q] = Yc[q] = 0.0f;
  float xb = 0.0f;
  for (int t = 0; t <= nlay; ++t) {
    float Yt[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float xt = 0.0f;
    if (t < nlay) {
      const bool ok = wait_parity(&bar[t % kStages], (uint32_t)(t / kStages) & 1u, status,
                                  kWaitLimitNs);
      if (__syncthreads_or(!ok)) {
        // bounded wait for the copies still in flight, then leave
        if (ty == 0 && tx == 0)
          for (int u = t + 1; u < issued; ++u)
            wait_parity(&bar[u % kStages], (uint32_t)(u / kStages) & 1u, status, kWaitLimitNs);
        return;
      }
      if (active) {
        const float* st = tile[t % kStages];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float sum = 0.0f;
#pragma unroll
          for (int c = 0; c < 9; ++c)
            if (c != 4) sum = fmaf(hf[q][c], st[toff[c]], sum);
          Yt[q] = sum;
        }
        xt = st[toff[4]];
      }
    }
    if (t >= 1 && active) {
      // row of free layer number t-1: behind = t-2, ahead = t
      const int kr = UP ? t - 1 : nlay - t;
      const float* v = V + kr * kVF;
      float acc = tile[(t - 1) % kStages][kStageX + ty * 32 + tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc = fmaf(-v[3 * q + vb], Yb[q], acc);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc = fmaf(-v[3 * q + 1], Yc[q], acc);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc = fmaf(-v[3 * q + va], Yt[q], acc);
      float kb = 0.0f, dg = 0.0f, ka = 0.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        kb = fmaf(hf[q][4], v[3 * q + vb], kb);
        dg = fmaf(hf[q][4], v[3 * q + 1], dg);
        ka = fmaf(hf[q][4], v[3 * q + va], ka);
      }
      acc = fmaf(-kb, xb, acc);
      acc = fmaf(-ka, xt, acc);
      xb = acc / dg;
      x[(int64_t)kr * PP + own] = xb;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Yb[q] = Yc[q];
      Yc[q] = Yt[q];
    }
    __syncthreads();  // stage (t - 1) % kStages is free
    if (ty == 0 && issued < nlay && issued == t + kStages - 1) {
      fence_proxy_async_shared();
      issue(issued);
      ++issued;
    }
  }
}

// First group of a forward sweep from x = 0: every neighbour is still zero
// except the node just below, so x_k = (f_k - K(k, k-1) x_{k-1}) / K_kk with
// the center column's couplings from the factors.  Every other entry of x
// (other groups, fixed nodes, padding) is written 0.
__global__ void __launch_bounds__(128) k_gs_sep_zero_start(Grid g, const float* __restrict__ H,
                                                           const float* __restrict__ V,
                                                           const float* __restrict__ f,
                                                           float* __restrict__ x, int pi, int pj) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int par = (int)blockIdx.z;
  if (h >= g.H || j >= g.Ny) return;
  const int i = 2 * h + par;
  const int64_t own = (int64_t)j * g.RP + (int64_t)par * g.H + h;
  const int64_t PP = g.PP;
  const bool mine = par == pi && (j & 1) == pj && i < g.Nx && free_column(g, i, j);
  if (!mine) {
    for (int k = 0; k < g.Nz; ++k) x[(int64_t)k * PP + own] = 0.0f;
    return;
  }
  float hc[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) hc[t] = H[hidx(own, 9 * t + 4)];
  float prev = 0.0f;
  for (int k = 0; k <= g.Nz - 2; ++k) {
    const float* v = V + k * kVF;
    float kb = 0.0f, dg = 0.0f;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      kb = fmaf(hc[t], v[3 * t], kb);
      dg = fmaf(hc[t], v[3 * t + 1], dg);
    }
    const float acc = fmaf(-kb, prev, f[(int64_t)k * PP + own]);
    prev = acc / dg;
    x[(int64_t)k * PP + own] = prev;
  }
  x[(int64_t)(g.Nz - 1) * PP + own] = 0.0f;
}

// r = f - K x on the separable float32 operator, one thread per column
// (blockIdx.z = parity of i), with the full 9-column sums
// y_t(k') = sum_d H_t(c, c + d) x(c + d, k') formed once per layer.
// FUSE = false: writes r (0 at fixed nodes).  FUSE = true, for a transfer
// that keeps the columns (vertical coarsening only): restricts on the fly,
// f_c(K) = sum_k P(k, K) r(k) (Eq. 7 first row) with the layer weights of
// the transfer, so r is never stored; fc is on the coarse grid (same
// columns, tr.Nzc layers).
template <bool FUSE>
__global__ void __launch_bounds__(128) k_residual_sep(Grid g, Transfer tr,
                                                      const float* __restrict__ H,
                                                      const float* __restrict__ V,
                                                      const float* __restrict__ f,
                                                      const float* __restrict__ x,
                                                      float* __restrict__ out) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int par = (int)blockIdx.z;
  if (h >= g.H || j >= g.Ny) return;
  const int i = 2 * h + par;
  const int64_t own = (int64_t)j * g.RP + (int64_t)par * g.H + h;
  const int64_t PP = g.PP;
  const int Nz = g.Nz;
  const int Nout = FUSE ? tr.Nzc : Nz;
  if (!(i < g.Nx && free_column(g, i, j))) {
    for (int k = 0; k < Nout; ++k) out[(int64_t)k * PP + own] = 0.0f;
    return;
  }
  int off[9];
  column_offsets(g, i, off);
  float hf[4][9];
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int c = 0; c < 9; ++c) hf[t][c] = H[hidx(own, 9 * t + c)];
  float nb[9];
  auto load = [&](int k) {
    const float* xl = x + (int64_t)k * PP + own;
#pragma unroll
    for (int c = 0; c < 9; ++c) nb[c] = xl[off[c]];
  };
  auto fsum = [&](float y[4]) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float s = 0.0f;
#pragma unroll
      for (int c = 0; c < 9; ++c) s = fmaf(hf[t][c], nb[c], s);
      y[t] = s;
    }
  };
  float Yb[4], Y0[4], Y1[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) Yb[t] = 0.0f;
  load(0);
  fsum(Y0);
  load(1);
  fsum(Y1);
  int Kcur = 0;
  float accLo = 0.0f, accHi = 0.0f;
  for (int k = 0; k <= Nz - 2; ++k) {
    const bool more = k + 2 <= Nz - 1;
    if (more) load(k + 2);
    const float* v = V + k * kVF;
    float r = f[(int64_t)k * PP + own];
#pragma unroll
    for (int t = 0; t < 4; ++t) r = fmaf(-v[3 * t], Yb[t], r);
#pragma unroll
    for (int t = 0; t < 4; ++t) r = fmaf(-v[3 * t + 1], Y0[t], r);
#pragma unroll
    for (int t = 0; t < 4; ++t) r = fmaf(-v[3 * t + 2], Y1[t], r);
    if (FUSE) {
      const int c0 = tr.kc0[k], c1 = tr.kc1[k];
      if (c0 > Kcur) {  // coarse layer Kcur has all its fine contributions
        out[(int64_t)Kcur * PP + own] = accLo;
        accLo = accHi;
        accHi = 0.0f;
        Kcur = c0;
      }
      accLo = fmaf(tr.kw0[k], r, accLo);
      if (c1 != c0) accHi = fmaf(tr.kw1[k], r, accHi);
    } else {
      out[(int64_t)k * PP + own] = r;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      Yb[t] = Y0[t];
      Y0[t] = Y1[t];
    }
    if (more) {
      fsum(Y1);
    } else {
#pragma unroll
      for (int t = 0; t < 4; ++t) Y1[t] = 0.0f;
    }
  }
  if (FUSE) {
    // the last fine free layer ends coarse layer Nzc - 2; the top is fixed
    out[(int64_t)Kcur * PP + own] = accLo;
    for (int K = Kcur + 1; K < Nout; ++K) out[(int64_t)K * PP + own] = 0.0f;
  } else {
    out[(int64_t)(Nz - 1) * PP + own] = 0.0f;
  }
}

}  // namespace

cudaError_t launch_shift_check(int Nx, int Ny, int Nz, const double* X, const double* Y,
                               const double* Z, int* flag, cudaStream_t st) {
  k_shift_check<<<dim3((Nx + 31) / 32, (Ny + 3) / 4), dim3(32, 4), 0, st>>>(Nx, Ny, Nz, X, Y, Z,
                                                                          flag);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_hfactors(const Grid& g, const double* X, const double* Y, const double* Z,
                            const double* a, double* H64, float* H32, int* flag,
                            cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(H64, 0, sizeof(double) * kHF * (size_t)g.PP, st);
  const double c1 = 1.0 / (a[0] * a[0]), c2 = 1.0 / (a[1] * a[1]), c3 = 1.0 / (a[2] * a[2]);
  // cells (Nx - 1) x (Ny - 1), a quarter of them per class
  const dim3 grd((g.Nx / 2 + 31) / 32, (g.Ny / 2 + 3) / 4);
  for (int cls = 0; cls < 4 && e == cudaSuccess; ++cls) {
    k_hfactor_cells<<<grd, dim3(32, 4), 0, st>>>(g, cls, X, Y, Z, c1, c2, c3, H64, flag);
    count_launches(1);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? launch_hfactor_finalize(g, H64, H32, st) : e;
}

cudaError_t launch_hfactor_finalize(const Grid& g, double* H64, float* H32, cudaStream_t st) {
  k_hfactor_finalize<<<dim3((g.H + 31) / 32, (g.Ny + 3) / 4, 2), dim3(32, 4), 0, st>>>(g, H64, H32);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_hgalerkin(int dim, const Grid& gin, const Grid& gout, const double* Hin,
                             double* Hout, cudaStream_t st) {
  const dim3 grd((gout.Nx + 31) / 32, (gout.Ny + 3) / 4), blk(32, 4);
  if (dim == 0) k_hgalerkin<0><<<grd, blk, 0, st>>>(gin, gout, Hin, Hout);
  else k_hgalerkin<1><<<grd, blk, 0, st>>>(gin, gout, Hin, Hout);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_vfactor0(int Nx, int Ny, int Nz, const double* Z, double* V64, float* V32,
                            cudaStream_t st) {
  k_vfactor0<<<1, 32, 0, st>>>(Nx, Ny, Nz, Z, V64, V32);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_vgalerkin(const Transfer& tr, const double* Vf, double* Vc, float* Vc32,
                             cudaStream_t st) {
  k_vgalerkin<<<1, kMaxZ, 0, st>>>(tr, Vf, Vc, Vc32);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sep_expand64(const Grid& g, const double* H64, const double* V64, double* C,
                                cudaStream_t st) {
  k_sep_expand64<<<dim3((g.H + 31) / 32, (g.Ny + 3) / 4, 2 * g.Nz), dim3(32, 4), 0, st>>>(g, H64,
                                                                                     V64, C);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sep_export(const Grid& g, const T* H, const T* V, double* out,
                              cudaStream_t st) {
  k_sep_export<T><<<dim3((g.Nx + 31) / 32, (g.Ny + 3) / 4, g.Nz), dim3(32, 4), 0, st>>>(g, H, V,
                                                                                     out);
  count_launches(1);
  return cudaGetLastError();
}
template cudaError_t launch_sep_export<double>(const Grid&, const double*, const double*, double*,
                                               cudaStream_t);
template cudaError_t launch_sep_export<float>(const Grid&, const float*, const float*, double*,
                                              cudaStream_t);

cudaError_t launch_gs_sep(const Grid& g, const float* H32, const float* V32, const float* f,
                          float* x, int group, int up, int rows, cudaStream_t st) {
  const int pi = group & 1, pj = group >> 1;
  const dim3 blk(32, rows);
  const dim3 grd(((g.Nx + 1) / 2 + 31) / 32, ((g.Ny + 1) / 2 + rows - 1) / rows);
  if (up) k_gs_sep<true><<<grd, blk, 0, st>>>(g, H32, V32, f, x, pi, pj);
  else k_gs_sep<false><<<grd, blk, 0, st>>>(g, H32, V32, f, x, pi, pj);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gs_sep_staged(const Grid& g, const float* H32, const float* V32,
                                 const float* f, float* x, int group, int up, int* status,
                                 cudaStream_t st) {
  const int pi = group & 1, pj = group >> 1;
  const dim3 blk(32, kGsR);
  const dim3 grd(((g.Nx + 1) / 2 + 31) / 32, ((g.Ny + 1) / 2 + kGsR - 1) / kGsR);
  if (up) k_gs_sep_staged<true><<<grd, blk, 0, st>>>(g, H32, V32, f, x, pi, pj, status);
  else k_gs_sep_staged<false><<<grd, blk, 0, st>>>(g, H32, V32, f, x, pi, pj, status);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gs_sep_zero_start(const Grid& g, const float* H32, const float* V32,
                                     const float* f, float* x, int group, cudaStream_t st) {
  const dim3 grd((g.H + 31) / 32, (g.Ny + 3) / 4, 2);
  k_gs_sep_zero_start<<<grd, dim3(32, 4), 0, st>>>(g, H32, V32, f, x, group & 1, group >> 1);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_residual_sep(const Grid& g, const Transfer* fuse, const float* H32,
                                const float* V32, const float* f, const float* x, float* out,
                                cudaStream_t st) {
  const dim3 grd((g.H + 31) / 32, (g.Ny + 3) / 4, 2), blk(32, 4);
  if (fuse) {
    k_residual_sep<true><<<grd, blk, 0, st>>>(g, *fuse, H32, V32, f, x, out);
  } else {
    Transfer none;
    none.Nzc = g.Nz;
    k_residual_sep<false><<<grd, blk, 0, st>>>(g, none, H32, V32, f, x, out);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mcw
