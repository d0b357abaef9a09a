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
#include <cudaTypedefs.h>

#include "async.cuh"
#include "cellgeom.cuh"
#include "dfloat.cuh"
#include "kernels.cuh"

namespace mcw {
namespace {

constexpr int kShiftFlag = 8;

__device__ __forceinline__ bool free_column(const Grid& g, int i, int j) {
  return i >= 1 && i <= g.Nx - 2 && j >= 1 && j <= g.Ny - 2;
}

// acc += a * b in float pairs: the product's rounding error kept by the FMA,
// the sum's by a two-sum; the low part is renormalized by the caller
__device__ __forceinline__ void pmac2(float& sh, float& sl, float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float s = sh + p;
  const float bb = s - sh;
  const float t = (sh - (s - bb)) + (p - bb);
  sh = s;
  sl += t + e;
}

// ---------------------------------------------------------------- set-up

// flag |= 8 unless X and Y do not depend on k and Z(i,j,k) - Z(i,j,0) equals
// zeta_k = Z(0,0,k) - Z(0,0,0), each to about 1e-10 of the largest
// coordinate magnitude involved (the generator's rounding of z_s + zeta is
// far below it).  Standard layout.  One thread per node above the ground
// layer (blockIdx.z = k - 1); equal X and Y are recognised by their bits,
// and "small" is decided on the exponents, |d| < 2^-33 max, in 32-bit
// integer arithmetic on the high words (on GB300 the double pipe, which
// also issues some 64-bit integer instructions, runs at 1/64 of the float
// rate): two float64 subtractions per node for the z test.
__device__ __forceinline__ unsigned mag_hi(double v) { return (unsigned)__double2hiint(v) & 0x7FFFFFFFu; }

__global__ void k_shift_check(int Nx, int Ny, int Nz, const double* __restrict__ X,
                              const double* __restrict__ Y, const double* __restrict__ Z,
                              int* flag) {
  __shared__ double zeta;
  __shared__ unsigned mlay;
  const int k = (int)blockIdx.z + 1;
  const int64_t lay = (int64_t)Nx * Ny;
  if (threadIdx.x == 0) {
    const double zr = Z[k * lay], zb = Z[0];
    zeta = zr - zb;
    mlay = max(mag_hi(zr), mag_hi(zb));
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= Nx || j >= Ny || k >= Nz) return;
  const int64_t c = (int64_t)j * Nx + i;
  const double x0 = X[c], y0 = Y[c], z0 = Z[c];
  const double xk = X[k * lay + c], yk = Y[k * lay + c], zk = Z[k * lay + c];
  const unsigned m = max(max(mag_hi(x0), mag_hi(y0)), max(max(mag_hi(z0), mag_hi(zk)), mlay));
  const int lim = (int)(m >> 20) - 34;  // biased exponent bound of a small difference
  auto small = [lim](double d) { return (int)(mag_hi(d) >> 20) <= lim; };
  bool ok = small((zk - z0) - zeta);
  if (__double2hiint(xk) != __double2hiint(x0) || __double2loint(xk) != __double2loint(x0))
    ok = ok && small(xk - x0);
  if (__double2hiint(yk) != __double2hiint(y0) || __double2loint(yk) != __double2loint(y0))
    ok = ok && small(yk - y0);
  if (!ok) atomicOr(flag, kShiftFlag);
}

// Horizontal factors of the cells of one parity class (cell (ci, cj) with
// ci & 1 = cls & 1, cj & 1 = cls >> 1), added into the float64 planes of
// their 4 corner columns: cells of one class share no corner, and the four
// classes run in order, so every sum is formed in one fixed order (the adds
// are L2 reductions, one per address and launch: the same sums, bitwise).  2 x 2
// Gauss points in (xi1, xi2), in arithmetic R (float64 or float pairs).
// Corner p = a + 2b is node (ci + a, cj + b) of the ground layer (standard
// layout).  P and R are symmetric, so only their upper triangles are formed.
template <typename R>
__global__ void __launch_bounds__(128) k_hfactor_cells(Grid g, int cls, const double* __restrict__ X,
                                                       const double* __restrict__ Y,
                                                       const double* __restrict__ Z, double c1d,
                                                       double c2d, double c3d,
                                                       double* __restrict__ H, int* flag) {
  using A = Arith<R>;
  const int ci = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + (cls & 1);
  const int cj = 2 * (blockIdx.y * blockDim.y + threadIdx.y) + (cls >> 1);
  if (ci >= g.Nx - 1 || cj >= g.Ny - 1) return;
  double xs[4], ys[4], zs[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int64_t n = (int64_t)(cj + (p >> 1)) * g.Nx + ci + (p & 1);
    xs[p] = X[n]; ys[p] = Y[n]; zs[p] = Z[n];
  }
  const CellEdges<R> ce = cell_edges<R>(xs, ys, zs);
  const R c1 = A::from(c1d), c2 = A::from(c2d), c3 = A::from(c3d);
  R P[10], Q[4][4], Rr[10];  // P, R: upper triangles, index tri(p, q)
#pragma unroll
  for (int u = 0; u < 10; ++u) P[u] = Rr[u] = A::zero();
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) Q[p][q] = A::zero();
  bool bad = false;
#pragma unroll
  for (int gq = 0; gq < 4; ++gq) {
    const GaussGeom<R> G = gauss_geom(ce, gq);
    const R j2 = G.J00 * G.J11 - G.J01 * G.J10;
    bad = bad || !A::pos(j2);
    const R ij = A::rcp(j2);
    // W = adj D adj^T / j2 with adj = [[J11, -J01], [-J10, J00]]
    const R W00 = (c1 * (G.J11 * G.J11) + c2 * (G.J01 * G.J01)) * ij;
    const R W01 = -((c1 * (G.J11 * G.J10) + c2 * (G.J01 * G.J00)) * ij);
    const R W11 = (c1 * (G.J10 * G.J10) + c2 * (G.J00 * G.J00)) * ij;
    const R v1 = W00 * G.z1 + W01 * G.z2, v2 = W01 * G.z1 + W11 * G.z2;  // W z'
    const R s = G.z1 * v1 + G.z2 * v2 + c3 * j2;
    R wg1[4], wg2[4], u[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const R d1 = A::from(gauss_d1(gq, p)), d2 = A::from(gauss_d2(gq, p));
      wg1[p] = W00 * d1 + W01 * d2;
      wg2[p] = W01 * d1 + W11 * d2;
      u[p] = d1 * v1 + d2 * v2;
    }
    int t = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const R d1 = A::from(gauss_d1(gq, p)), d2 = A::from(gauss_d2(gq, p));
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        Q[p][q] = Q[p][q] + u[p] * A::from(gauss_phi(gq, q));
        if (q >= p) {
          P[t] = P[t] + (d1 * wg1[q] + d2 * wg2[q]);
          Rr[t] = Rr[t] + s * A::from(gauss_phi(gq, p) * gauss_phi(gq, q));
          ++t;
        }
      }
    }
  }
  if (bad) atomicOr(flag, 1);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int64_t col = gidx(g, ci + (p & 1), cj + (p >> 1), 0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int s2 = ((q & 1) - (p & 1) + 1) + 3 * ((q >> 1) - (p >> 1) + 1);
      const int lo = p < q ? p : q, hi = p < q ? q : p;
      const int t = lo * 4 - lo * (lo - 1) / 2 + (hi - lo);  // tri(lo, hi)
      // one add per address and launch (cells of a class share no column),
      // issued as reductions in L2 so the cell does not wait for the reads
      atomicAdd(&H[(0 * 9 + s2) * g.PP + col], A::to_double(P[t]));
      atomicAdd(&H[(1 * 9 + s2) * g.PP + col], -A::to_double(Q[p][q]));
      atomicAdd(&H[(2 * 9 + s2) * g.PP + col], -A::to_double(Q[q][p]));
      atomicAdd(&H[(3 * 9 + s2) * g.PP + col], A::to_double(Rr[t]));
    }
  }
}

// Zero the couplings that touch a fixed column (and everything of padding
// columns) in the float64 planes and write the float32 tiles in the form
// the float32 kernels read: terms P, S = H_Q - H_Q^T, T = H_Q + H_Q^T, R
// (S(c, c) = 0 exactly).  With V_G = A + B, A = (V_G - V_G^T)/2
// antisymmetric and B = (V_G + V_G^T)/2, the two mixed terms are
// H_Q (x) V_G + H_Q^T (x) V_G^T = S (x) A + T (x) B, and B is -1/2 on the
// ground layer's diagonal and 0 elsewhere on every level (the ground layer
// is a node layer of every level), so above the ground three terms remain.
// One thread per split-layout column: blockIdx.z = parity of i.
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
  for (int s2 = 0; s2 < 9; ++s2) {
    const bool keep = fc && free_column(g, i + s2 % 3 - 1, j + s2 / 3 - 1);
    double v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      v[t] = keep ? H[(t * 9 + s2) * g.PP + col] : 0.0;
      H[(t * 9 + s2) * g.PP + col] = v[t];
    }
    H32[hidx(col, s2)] = (float)v[0];
    H32[hidx(col, 9 + s2)] = (float)(v[1] - v[2]);
    H32[hidx(col, 18 + s2)] = (float)(v[1] + v[2]);
    H32[hidx(col, 27 + s2)] = (float)v[3];
  }
}

// float32 vertical factors of one layer from its float64 ones (order M, G,
// G^T, K, 3 offsets each): [0..2] V_M(k, k-1..k+1), [3..5] V_K, [6] A(k, k-1),
// [7] A(k, k+1), [8] B(k, k), [9..11] 0.
__device__ __forceinline__ void write_v32(const double* v, float* o) {
  o[0] = (float)v[0]; o[1] = (float)v[1]; o[2] = (float)v[2];
  o[3] = (float)v[9]; o[4] = (float)v[10]; o[5] = (float)v[11];
  o[6] = (float)(0.5 * (v[3] - v[6]));
  o[7] = (float)(0.5 * (v[5] - v[8]));
  o[8] = (float)(0.5 * (v[4] + v[7]));
  o[9] = o[10] = o[11] = 0.0f;
}

// coefficient of offset (s2, dk) in a row, from float32 factors: hq[t] =
// term t of the column at s2 (P, S, T, R), v = the layer's float32 factors
__device__ __forceinline__ float sep32_coef(const float hq[4], const float* v, int dk) {
  float c = hq[0] * v[dk] + hq[3] * v[3 + dk];
  if (dk == 0) c += hq[1] * v[6];
  if (dk == 2) c += hq[1] * v[7];
  if (dk == 1) c += hq[2] * v[8];
  return c;
}

// One direction (DIM 0: x, 1: y) of the horizontal Galerkin product
// Ph^T H_t Ph, for all four terms: out(I; D, e) = sum_a w_a sum_d
// H(f_I + a; d, e) P(f_I + a + d, I + D) with the interpolation weights of
// Sec. 3 (a, d, D in {-1, 0, 1}; e the offset in the other direction).  One
// thread per output column; inputs outside the grid have weight 0.  The
// weights are 0, 1/2 and 1, so every product w_a P v is exact; the sums run
// in float pairs (about 48 significant bits, FP32 pipe) and each output is
// rounded to float64 once.
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
  float wa[3];
  hcoarse(1, Nf, Nc, Iout, f, wa[0], wa[2]);
  wa[1] = 1.0f;
  float Pw[5][3];  // Pw[q][D] = P(f + q - 2, Iout + D - 1)
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int b = f + q - 2;
    int c0 = -100, c1 = -100;
    float w0 = 0.0f, w1 = 0.0f;
    if (b >= 0 && b <= Nf - 1) hpair(1, Nf, Nc, b, c0, w0, c1, w1);
#pragma unroll
    for (int D = 0; D < 3; ++D) {
      const int J = Iout + D - 1;
      Pw[q][D] = (c0 == J ? w0 : 0.0f) + (c1 == J && c1 != c0 ? w1 : 0.0f);
    }
  }
  const int64_t o = gidx(gout, i, j, 0);
  for (int t = 0; t < 4; ++t) {
    dflt acc[9];
#pragma unroll
    for (int s = 0; s < 9; ++s) acc[s] = dflt{0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (wa[a] == 0.0f) continue;
      const int ii = DIM == 0 ? f + a - 1 : i, jj = DIM == 1 ? f + a - 1 : j;
      const int64_t in = gidx(gin, ii, jj, 0);
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        const int d = DIM == 0 ? s % 3 : s / 3, e = DIM == 0 ? s / 3 : s % 3;
        const float2 v2 = split_bits(Hin[(t * 9 + s) * gin.PP + in]);
#pragma unroll
        for (int D = 0; D < 3; ++D) {
          const float w = wa[a] * Pw[a + d][D];  // 0, 1/4, 1/2 or 1: exact
          if (w != 0.0f) {
            dflt& r = acc[DIM == 0 ? D + 3 * e : e + 3 * D];
            r = r + dflt{v2.x * w, v2.y * w};
          }
        }
      }
    }
#pragma unroll
    for (int s = 0; s < 9; ++s) Hout[(t * 9 + s) * gout.PP + o] = pair_to_double(acc[s].hi, acc[s].lo);
  }
}

// Vertical factors of the finest level from the layer thicknesses of
// column (0, 0) (standard layout Z): element l adds (h/2) m, g and (2/h)
// kappa to layers l, l+1.  One thread.  Couplings to the top layer (fixed)
// are zero.
__global__ void k_vfactor0(int Nx, int Ny, int Nz, const double* __restrict__ Z,
                           double* __restrict__ V, float* __restrict__ V32, float2* __restrict__ VR,
                           int* flag) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int64_t lay = (int64_t)Nx * Ny;
  for (int q = 0; q < Nz * kVF; ++q) V[q] = 0.0;
  for (int l = 0; l + 1 < Nz; ++l) {
    const double h = Z[(int64_t)(l + 1) * lay] - Z[(int64_t)l * lay];
    if (!(h > 0.0)) atomicOr(flag, 1);  // det J = (h/2) j2 must be positive
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
  // the load vector's vertical factors, V_M and V_G^T with the top layer
  // kept (u0 of the top nodes enters the rows below them)
  if (VR)
    for (int k = 0; k < Nz; ++k)
      for (int d = 0; d < 3; ++d) {
        VR[k * kRV + d] = split_bits(V[k * kVF + d]);
        VR[k * kRV + 3 + d] = split_bits(V[k * kVF + 6 + d]);
      }
  for (int t = 0; t < 4; ++t) {
    V[(Nz - 2) * kVF + 3 * t + 2] = 0.0;
    for (int d = 0; d < 3; ++d) V[(Nz - 1) * kVF + 3 * t + d] = 0.0;
  }
  for (int k = 0; k < Nz; ++k) write_v32(V + k * kVF, V32 + k * kVF);
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
  for (int q = 0; q < kVF; ++q) Vc[K * kVF + q] = acc[q];
  write_v32(acc, Vc32 + K * kVF);
}

// Expanded 27-point rows from float64 factors into the tiled float64
// operator, planes 0..26, and plane 27 = 1/K_nn (0 at fixed nodes; flag |= 2
// if a free diagonal is not positive).  The factors already zero every
// coupling that touches a fixed node, so no further masking is needed.
// Three-term form: coefficient (s2, dk) = P V_M + R V_K + S A (+ T B on the
// ground layer's diagonal), S = H_Q - H_Q^T, T = H_Q + H_Q^T,
// A = (V_G - V_G^T)/2, B = (V_G + V_G^T)/2 (B is exactly -1/2 at (0, 0) and 0
// elsewhere, A(k, k) exactly 0).  PAIRS: the products and sums run in float
// pairs (about 48 significant bits, FP32 pipe; each coefficient is rounded
// to float64 once); otherwise in float64, as sum_t H_t V_t over the four
// terms.  The reciprocal of the diagonal is float64.  One thread per column
// (blockIdx.z = parity), walking the layers; the block first turns the
// level's vertical factors into float pairs in shared memory.
template <bool PAIRS>
__global__ void __launch_bounds__(128) k_sep_expand(Grid g, const double* __restrict__ H,
                                                    const double* __restrict__ V,
                                                    double* __restrict__ C, int* flag) {
  if (!PAIRS) {
    const int hh = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int par = blockIdx.z;
    if (hh >= g.H || j >= g.Ny) return;
    const int i = 2 * hh + par;
    const int64_t col = (int64_t)j * g.RP + (int64_t)par * g.H + hh;
    const bool fcol = i >= 1 && i <= g.Nx - 2 && j >= 1 && j <= g.Ny - 2;
    for (int k = 0; k < g.Nz; ++k) {
      const int64_t b = (int64_t)k * g.PP + col;
      double diag = 0.0;
#pragma unroll
      for (int s = 0; s < 27; ++s) {
        const int s2 = s % 9, dk = s / 9;
        double c = 0.0;
#pragma unroll
        for (int t = 0; t < 4; ++t) c += H[(t * 9 + s2) * g.PP + col] * V[k * kVF + 3 * t + dk];
        C[cidx(b, s)] = c;
        if (s == 13) diag = c;
      }
      const bool fr = fcol && k <= g.Nz - 2;
      if (fr && !(diag > 0.0)) atomicOr(flag, 2);
      C[cidx(b, kInvDiag)] = fr ? 1.0 / diag : 0.0;
    }
    return;
  }
  __shared__ float2 vs[kMaxZ][9];  // M(3), K(3), A(k,k-1), A(k,k+1), B(k,k)
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int q = tid; q < g.Nz * 9; q += blockDim.x * blockDim.y) {
    const int k = q / 9, e = q % 9;
    const double* v = V + k * kVF;
    double x;
    if (e < 3) x = v[e];
    else if (e < 6) x = v[9 + e - 3];
    else if (e == 6) x = 0.5 * (v[3] - v[6]);
    else if (e == 7) x = 0.5 * (v[5] - v[8]);
    else x = 0.5 * (v[4] + v[7]);
    vs[k][e] = split_bits(x);
  }
  __syncthreads();
  const int hh = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int par = blockIdx.z;
  if (hh >= g.H || j >= g.Ny) return;
  const int i = 2 * hh + par;
  const int64_t col = (int64_t)j * g.RP + (int64_t)par * g.H + hh;
  float2 P[9], S[9], T[9], R[9];
#pragma unroll
  for (int s2 = 0; s2 < 9; ++s2) {
    const double q = H[(9 + s2) * g.PP + col], qt = H[(18 + s2) * g.PP + col];
    P[s2] = split_bits(H[s2 * g.PP + col]);
    S[s2] = split_bits(q - qt);
    T[s2] = split_bits(q + qt);
    R[s2] = split_bits(H[(27 + s2) * g.PP + col]);
  }
  const bool fcol = i >= 1 && i <= g.Nx - 2 && j >= 1 && j <= g.Ny - 2;
  for (int k = 0; k < g.Nz; ++k) {
    const float2* v = vs[k];
    const int64_t b = (int64_t)k * g.PP + col;
    double diag = 0.0;
#pragma unroll
    for (int s2 = 0; s2 < 9; ++s2) {
#pragma unroll
      for (int dk = 0; dk < 3; ++dk) {
        // the first product seeds the sum: its rounding error is the low part
        float sh = P[s2].x * v[dk].x;
        float sl = fmaf(P[s2].x, v[dk].x, -sh);
        sl = fmaf(P[s2].x, v[dk].y, sl);
        sl = fmaf(P[s2].y, v[dk].x, sl);
        pmac2(sh, sl, R[s2], v[3 + dk]);
        if (dk == 0) pmac2(sh, sl, S[s2], v[6]);
        if (dk == 2) pmac2(sh, sl, S[s2], v[7]);
        if (dk == 1 && k == 0) pmac2(sh, sl, T[s2], v[8]);
        const float hi = sh + sl, lo = sl - (hi - sh);
        const double c = pair_to_double(hi, lo);
        C[cidx(b, dk * 9 + s2)] = c;
        if (dk == 1 && s2 == 4) diag = c;
      }
    }
    const bool fr = fcol && k <= g.Nz - 2;
    if (fr && !(diag > 0.0)) atomicOr(flag, 2);
    C[cidx(b, kInvDiag)] = fr ? 1.0 / diag : 0.0;
  }
}

// Rows from the factors in the standard layout [27][Nz][Ny][Nx] (the level
// stencil export): float64 factors (planes, terms M, G, G^T, K) in float64,
// float32 factors (tiles, the float32 form) in float32.
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
    double c;
    if (sizeof(T) == 8) {
      c = 0.0;
#pragma unroll
      for (int t = 0; t < 4; ++t) c += (double)H[(t * 9 + s2) * g.PP + col] * (double)V[k * kVF + 3 * t + dk];
    } else {
      float hq[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) hq[t] = (float)H[hidx(col, t * 9 + s2)];
      c = sep32_coef(hq, (const float*)V + k * kVF, dk);
    }
    out[s * n + o] = c;
  }
}

// ---------------------------------------------------------------- cycle
//
// The float32 kernels stage x and f through shared memory.  A block owns
// kGsR rows x 32 columns of the split layout; a producer warp loads, per
// free layer and in sweep order, a tile of x around them (rows j0-1 ..
// j0+span, both parity halves, half-row indices [h0-4, h0+36): the 9
// columns around each owned column, the window starting on a 16-byte
// boundary) and the owned f, as two TMA tiles of the level's tensor maps,
// into a ring of kStages shared-memory stages, as far ahead of the
// consumers as the ring allows; entries outside the grid arrive as zeros.
// Each stage has a "full" mbarrier (one arrival + the tiles' bytes) and an
// "empty" one (one arrival per consumer warp once its rows no longer read
// the stage).  The consumer warps (one thread per column) never wait on each
// other.  Per layer a thread forms its neighbour sums once -- they serve the
// rows below, at and above -- so a row costs about 40 products.  Every wait
// is bounded: one that runs out sets the status bit and its warp leaves; the
// producer waits (bounded) for the tiles it issued before it leaves.
constexpr int kGsR = 4;
constexpr int kTileW = 40;
constexpr int kStages = 8;
// smoother: owned rows j0, j0+2, ..., j0+2(kGsR-1) (one column group)
constexpr int kGsTileRows = 2 * kGsR + 1;
constexpr int kGsX = 768;                         // 720 used; f 128-byte aligned
constexpr int kGsFRows = 2 * kGsR - 1;
constexpr int kGsStage = kGsX + kGsFRows * 32;    // 992 floats = 31 x 128 bytes
constexpr uint32_t kGsBytes = (kGsTileRows * 2 * kTileW + kGsFRows * 32) * 4;
// residual: owned rows j0 .. j0+kGsR-1 (one parity half)
constexpr int kResTileRows = kGsR + 2;
constexpr int kResX = 512;                        // 480 used
constexpr int kResStage = kResX + kGsR * 32;      // 640 floats = 20 x 128 bytes
constexpr uint32_t kResBytes = (kResTileRows * 2 * kTileW + kGsR * 32) * 4;

// producer side of the ring: tile t of nlay into stage t % kStages
template <int STAGE>
__device__ __forceinline__ bool produce(float (*tile)[STAGE], uint64_t* full, uint64_t* empty,
                                        int nlay, bool up, uint32_t bytes, int fx,
                                        const CUtensorMap* tmx, const CUtensorMap* tmf, int cx0,
                                        int cx2, int cf0, int cf1, int cf2, int* status) {
  const int lane = threadIdx.x;
  int issued = 0;
  bool ok = true;
  for (int t = 0; t < nlay; ++t) {
    const int sidx = t & (kStages - 1);
    if (t >= kStages) {
      ok = wait_parity(&empty[sidx], (uint32_t)(t / kStages - 1) & 1u, status, kWaitLimitNs);
      if (__any_sync(0xffffffffu, !ok)) break;  // the warp leaves together
    }
    if (lane == 0) {
      const int k = up ? t : nlay - 1 - t;
      fence_proxy_async_shared();
      mbar_arrive_expect_tx(&full[sidx], bytes);
      tensor_copy_4d(tile[sidx], tmx, cx0, 0, cx2, k, &full[sidx]);
      tensor_copy_4d(tile[sidx] + fx, tmf, cf0, cf1, cf2, k, &full[sidx]);
    }
    __syncwarp();
    issued = t + 1;
  }
  // the block's shared memory must outlive the tiles this warp issued
  if (lane == 0)
    for (int u = max(0, issued - kStages); u < issued; ++u)
      wait_parity(&full[u & (kStages - 1)], (uint32_t)(u / kStages) & 1u, status, kWaitLimitNs);
  return ok;
}

// Gauss-Seidel of Sec. 3 on the separable float32 operator, one column
// group (pi, pj) per launch, one thread per column, the layers bottom-up
// (UP) or top-down.  A row needs the new x of the layer behind the sweep,
// the old x of the layer ahead (its own column) and the other groups' old x
// (the neighbour sums), all staged.
template <bool UP>
__global__ void __launch_bounds__(32 * (kGsR + 1)) k_gs_sep_staged(
    Grid g, const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmf,
    const float* __restrict__ H, const float* __restrict__ V, float* __restrict__ x, int pi, int pj,
    int* status) {
  __shared__ __align__(128) float tile[kStages][kGsStage];
  __shared__ __align__(16) float vsh[kMaxZ * kVF];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int h0 = blockIdx.x * 32;
  const int j0 = 2 * kGsR * blockIdx.y + pj;
  const int nlay = g.Nz - 1;  // free layers; the top layer is fixed (x = 0)
  if (ty == 0 && tx == 0) {
    for (int q = 0; q < kStages; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kGsR);
    }
    fence_barrier_init();
  }
  for (int q = ty * 32 + tx; q < nlay * kVF; q += 32 * (kGsR + 1)) vsh[q] = V[q];
  __syncthreads();
  if (ty == kGsR) {
    produce<kGsStage>(tile, full, empty, nlay, UP, kGsBytes, kGsX, &tmx, &tmf, h0 - 4, j0 - 1,
                      h0, pi, j0, status);
    return;
  }
  const int h = h0 + tx, j = j0 + 2 * ty, i = 2 * h + pi;
  const bool active = i >= 1 && i <= g.Nx - 2 && j >= 1 && j <= g.Ny - 2;
  const int64_t own = (int64_t)j * g.RP + (int64_t)pi * g.H + h;
  float hf[4][9];  // P, S, T, R
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
  // vertical offsets of the layer behind / ahead of the sweep
  const int vb = UP ? 0 : 2, va = UP ? 2 : 0;
  const int ab = UP ? 6 : 7, aa = UP ? 7 : 6;
  const int fo = kGsX + 2 * ty * 32 + tx;
  float Pb = 0.0f, Sb = 0.0f, Rb = 0.0f, Pc = 0.0f, Sc = 0.0f, Rc = 0.0f;
  float yT0 = 0.0f;  // T-sum of the ground layer (its only row with B != 0)
  float xb = 0.0f;
  // unrolled by the period of the behind / current / ahead window, so the
  // window moves by renaming registers
#pragma unroll 3
  for (int t = 0; t <= nlay; ++t) {
    float Pt = 0.0f, St = 0.0f, Rt = 0.0f, xt = 0.0f;
    if (t < nlay) {
      const bool ok = wait_parity(&full[t & (kStages - 1)], (uint32_t)(t / kStages) & 1u, status,
                                  kWaitLimitNs);
      if (__any_sync(0xffffffffu, !ok)) return;  // the warp leaves together
      if (active) {
        const float* st = tile[t & (kStages - 1)];
        float nb[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) nb[c] = st[toff[c]];
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          if (c == 4) continue;
          Pt = fmaf(hf[0][c], nb[c], Pt);
          St = fmaf(hf[1][c], nb[c], St);
          Rt = fmaf(hf[3][c], nb[c], Rt);
        }
        if ((UP ? t : nlay - 1 - t) == 0) {
#pragma unroll
          for (int c = 0; c < 9; ++c)
            if (c != 4) yT0 = fmaf(hf[2][c], nb[c], yT0);
        }
        xt = nb[4];
      }
    }
    if (t >= 1) {
      if (active) {
        // row of free layer number t-1: behind = t-2, ahead = t
        const int kr = UP ? t - 1 : nlay - t;
        const float4 v0 = *reinterpret_cast<const float4*>(vsh + kr * kVF);
        const float4 v1 = *reinterpret_cast<const float4*>(vsh + kr * kVF + 4);
        const float v[9] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, vsh[kr * kVF + 8]};
        float acc = tile[(t - 1) & (kStages - 1)][fo];
        acc = fmaf(-v[vb], Pb, acc);
        acc = fmaf(-v[3 + vb], Rb, acc);
        acc = fmaf(-v[ab], Sb, acc);
        acc = fmaf(-v[1], Pc, acc);
        acc = fmaf(-v[4], Rc, acc);
        acc = fmaf(-v[8], yT0, acc);
        acc = fmaf(-v[va], Pt, acc);
        acc = fmaf(-v[3 + va], Rt, acc);
        acc = fmaf(-v[aa], St, acc);
        const float kb = fmaf(hf[0][4], v[vb], hf[3][4] * v[3 + vb]);
        const float ka = fmaf(hf[0][4], v[va], hf[3][4] * v[3 + va]);
        const float dg = fmaf(hf[0][4], v[1], fmaf(hf[3][4], v[4], hf[2][4] * v[8]));
        acc = fmaf(-ka, xt, acc);
        acc = fmaf(-kb, xb, acc);
        xb = __fdividef(acc, dg);
        x[(int64_t)kr * g.PP + own] = xb;
      }
      // this warp no longer reads the stage of layer t-1
      __syncwarp();
      if (tx == 0) mbar_arrive(&empty[(t - 1) & (kStages - 1)]);
    }
    Pb = Pc; Sb = Sc; Rb = Rc;
    Pc = Pt; Sc = St; Rc = Rt;
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
  const float Pc = H[hidx(own, 4)], Tc = H[hidx(own, 22)], Rc = H[hidx(own, 31)];
  float prev = 0.0f;
  for (int k = 0; k <= g.Nz - 2; ++k) {
    const float* v = V + k * kVF;
    const float kb = fmaf(Pc, v[0], Rc * v[3]);
    const float dg = fmaf(Pc, v[1], fmaf(Rc, v[4], Tc * v[8]));
    prev = __fdividef(fmaf(-kb, prev, f[(int64_t)k * PP + own]), dg);
    x[(int64_t)k * PP + own] = prev;
  }
  x[(int64_t)(g.Nz - 1) * PP + own] = 0.0f;
}

// r = f - K x on the separable float32 operator, one thread per column of
// one parity half (blockIdx.z), owned rows j0 .. j0+kGsR-1, with the full
// 9-column sums formed once per layer.  FUSE = false: writes r (0 at fixed
// nodes and padding).  FUSE = true, for a transfer that keeps the columns
// (vertical coarsening only): restricts on the fly, f_c(K) = sum_k P(k, K)
// r(k) (Eq. 7 first row) with the layer weights of the transfer, so r is
// never stored; out is then the coarse f (same columns, tr.Nzc layers).
template <bool FUSE>
__global__ void __launch_bounds__(32 * (kGsR + 1)) k_residual_sep_staged(
    Grid g, const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmf,
    const __grid_constant__ Transfer tr, const float* __restrict__ H, const float* __restrict__ V,
    float* __restrict__ out, int* status) {
  __shared__ __align__(128) float tile[kStages][kResStage];
  __shared__ __align__(16) float vsh[kMaxZ * kVF];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int par = (int)blockIdx.z;
  const int h0 = blockIdx.x * 32;
  const int j0 = kGsR * blockIdx.y;
  const int nlay = g.Nz - 1;
  const int64_t PP = g.PP;
  if (ty == 0 && tx == 0) {
    for (int q = 0; q < kStages; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kGsR);
    }
    fence_barrier_init();
  }
  for (int q = ty * 32 + tx; q < nlay * kVF; q += 32 * (kGsR + 1)) vsh[q] = V[q];
  __syncthreads();
  if (ty == kGsR) {
    produce<kResStage>(tile, full, empty, nlay, true, kResBytes, kResX, &tmx, &tmf, h0 - 4,
                       j0 - 1, h0, par, j0, status);
    return;
  }
  const int h = h0 + tx, j = j0 + ty, i = 2 * h + par;
  const bool inrow = j < g.Ny;
  const bool active = inrow && i < g.Nx && free_column(g, i, j);
  const int64_t own = (int64_t)j * g.RP + (int64_t)par * g.H + h;
  float hf[4][9];
  int toff[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const int ii = i + c % 3 - 1, r = ty + 1 + c / 3 - 1;
    toff[c] = (r * 2 + (ii & 1)) * kTileW + ((ii >> 1) - (h0 - 4));
  }
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int c = 0; c < 9; ++c) hf[t][c] = active ? H[hidx(own, 9 * t + c)] : 0.0f;
  const int fo = kResX + ty * 32 + tx;
  float Pb = 0.0f, Sb = 0.0f, Rb = 0.0f, Pc = 0.0f, Sc = 0.0f, Rc = 0.0f;
  float T0 = 0.0f;
  int Kcur = 0;
  float accLo = 0.0f, accHi = 0.0f;
  // unrolled by the window's period (the unfused form keeps its registers)
#pragma unroll (FUSE ? 3 : 1)
  for (int t = 0; t <= nlay; ++t) {
    float Pt = 0.0f, St = 0.0f, Rt = 0.0f;
    if (t < nlay) {
      const bool ok = wait_parity(&full[t & (kStages - 1)], (uint32_t)(t / kStages) & 1u, status,
                                  kWaitLimitNs);
      if (__any_sync(0xffffffffu, !ok)) return;
      if (active) {
        const float* st = tile[t & (kStages - 1)];
        float nb[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) nb[c] = st[toff[c]];
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          Pt = fmaf(hf[0][c], nb[c], Pt);
          if (c != 4) St = fmaf(hf[1][c], nb[c], St);
          Rt = fmaf(hf[3][c], nb[c], Rt);
        }
        if (t == 0) {
#pragma unroll
          for (int c = 0; c < 9; ++c) T0 = fmaf(hf[2][c], nb[c], T0);
        }
      }
    }
    if (t >= 1) {
      const int k = t - 1;
      float r = 0.0f;
      if (active) {
        const float4 v0 = *reinterpret_cast<const float4*>(vsh + k * kVF);
        const float4 v1 = *reinterpret_cast<const float4*>(vsh + k * kVF + 4);
        r = tile[k & (kStages - 1)][fo];
        r = fmaf(-v0.x, Pb, r);
        r = fmaf(-v0.w, Rb, r);
        r = fmaf(-v1.z, Sb, r);
        r = fmaf(-v0.y, Pc, r);
        r = fmaf(-v1.x, Rc, r);
        r = fmaf(-vsh[k * kVF + 8], T0, r);
        r = fmaf(-v0.z, Pt, r);
        r = fmaf(-v1.y, Rt, r);
        r = fmaf(-v1.w, St, r);
      }
      __syncwarp();
      if (tx == 0) mbar_arrive(&empty[k & (kStages - 1)]);
      if (inrow) {
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
      }
    }
    Pb = Pc; Sb = Sc; Rb = Rc;
    Pc = Pt; Sc = St; Rc = Rt;
  }
  if (!inrow) return;
  if (FUSE) {
    // the last fine free layer ends coarse layer Nzc - 2; the top is fixed
    out[(int64_t)Kcur * PP + own] = accLo;
    for (int K = Kcur + 1; K < tr.Nzc; ++K) out[(int64_t)K * PP + own] = 0.0f;
  } else {
    out[(int64_t)(g.Nz - 1) * PP + own] = 0.0f;
  }
}

}  // namespace

cudaError_t launch_shift_check(int Nx, int Ny, int Nz, const double* X, const double* Y,
                               const double* Z, int* flag, cudaStream_t st) {
  if (Nz < 2) return cudaSuccess;
  k_shift_check<<<dim3((Nx + 255) / 256, Ny, Nz - 1), dim3(256, 1), 0, st>>>(Nx, Ny, Nz, X, Y, Z,
                                                                           flag);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_hfactors(const Grid& g, const double* X, const double* Y, const double* Z,
                            const double* a, double* H64, float* H32, int* flag, bool pairs,
                            cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(H64, 0, sizeof(double) * kHF * (size_t)g.PP, st);
  const double c1 = 1.0 / (a[0] * a[0]), c2 = 1.0 / (a[1] * a[1]), c3 = 1.0 / (a[2] * a[2]);
  // cells (Nx - 1) x (Ny - 1), a quarter of them per class
  const dim3 grd((g.Nx / 2 + 31) / 32, (g.Ny / 2 + 3) / 4);
  for (int cls = 0; cls < 4 && e == cudaSuccess; ++cls) {
    if (pairs)
      k_hfactor_cells<dflt><<<grd, dim3(32, 4), 0, st>>>(g, cls, X, Y, Z, c1, c2, c3, H64, flag);
    else
      k_hfactor_cells<double><<<grd, dim3(32, 4), 0, st>>>(g, cls, X, Y, Z, c1, c2, c3, H64, flag);
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
                            float2* VR2, int* flag, cudaStream_t st) {
  k_vfactor0<<<1, 32, 0, st>>>(Nx, Ny, Nz, Z, V64, V32, VR2, flag);
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
                               int* flag, bool pairs, cudaStream_t st) {
  const dim3 grd((g.H + 31) / 32, (g.Ny + 3) / 4, 2);
  if (pairs) k_sep_expand<true><<<grd, dim3(32, 4), 0, st>>>(g, H64, V64, C, flag);
  else k_sep_expand<false><<<grd, dim3(32, 4), 0, st>>>(g, H64, V64, C, flag);
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

cudaError_t launch_gs_sep_staged(const Level& L, const float* H32, const float* V32, float* x,
                                 int group, int up, int* status, cudaStream_t st) {
  const Grid& g = L.g;
  const int pi = group & 1, pj = group >> 1;
  const dim3 blk(32, kGsR + 1);
  const dim3 grd(((g.Nx + 1) / 2 + 31) / 32, ((g.Ny + 1) / 2 + kGsR - 1) / kGsR);
  if (up) k_gs_sep_staged<true><<<grd, blk, 0, st>>>(g, L.tm_x, L.tm_f, H32, V32, x, pi, pj, status);
  else k_gs_sep_staged<false><<<grd, blk, 0, st>>>(g, L.tm_x, L.tm_f, H32, V32, x, pi, pj, status);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_residual_sep_staged(const Level& L, bool fuse, const float* H32,
                                       const float* V32, float* out, int* status,
                                       cudaStream_t st) {
  const Grid& g = L.g;
  const dim3 blk(32, kGsR + 1);
  const dim3 grd((g.H + 31) / 32, (g.Ny + kGsR - 1) / kGsR, 2);
  if (fuse)
    k_residual_sep_staged<true><<<grd, blk, 0, st>>>(g, L.tm_rx, L.tm_rf, L.tr, H32, V32, out, status);
  else
    k_residual_sep_staged<false><<<grd, blk, 0, st>>>(g, L.tm_rx, L.tm_rf, L.tr, H32, V32, out, status);
  count_launches(1);
  return cudaGetLastError();
}

// Tensor maps of a level's float32 x and f for the staged kernels: each
// array as a 4-D tensor [Nz][Ny][2][H] (half-row index innermost, then the
// parity half, the row and the layer); boxes of 40 x 2 x 9 (smoother) or
// 40 x 2 x 6 (residual) x values and 32 x 1 x 7 or 32 x 1 x 4 f values,
// zero fill outside.
cudaError_t make_tile_maps(Level& L, float* x32, float* f32) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&encode,
                                                     12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !encode) return cudaErrorNotSupported;
  }
  const Grid& g = L.g;
  const cuuint64_t dims[4] = {(cuuint64_t)g.H, 2, (cuuint64_t)g.Ny, (cuuint64_t)g.Nz};
  const cuuint64_t strides[3] = {(cuuint64_t)g.H * 4, (cuuint64_t)g.RP * 4, (cuuint64_t)g.PP * 4};
  const cuuint32_t ones[4] = {1, 1, 1, 1};
  struct Map { CUtensorMap* m; float* base; cuuint32_t box[4]; };
  const Map maps[4] = {
      {&L.tm_x, x32, {(cuuint32_t)kTileW, 2, (cuuint32_t)kGsTileRows, 1}},
      {&L.tm_f, f32, {32, 1, (cuuint32_t)kGsFRows, 1}},
      {&L.tm_rx, x32, {(cuuint32_t)kTileW, 2, (cuuint32_t)kResTileRows, 1}},
      {&L.tm_rf, f32, {32, 1, (cuuint32_t)kGsR, 1}}};
  for (const Map& mp : maps) {
    const CUresult r = encode(mp.m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, mp.base, dims, strides,
                              mp.box, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t launch_gs_sep_zero_start(const Grid& g, const float* H32, const float* V32,
                                     const float* f, float* x, int group, cudaStream_t st) {
  const dim3 grd((g.H + 31) / 32, (g.Ny + 3) / 4, 2);
  k_gs_sep_zero_start<<<grd, dim3(32, 4), 0, st>>>(g, H32, V32, f, x, group & 1, group >> 1);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mcw
