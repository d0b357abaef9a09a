// Element kernels: isoparametric 8-node hexahedra (Sec. 2 of the paper).
//
// Local node n = a + 2b + 4c of element (i, j, k) is grid node
// (i+a, j+b, k+c) with reference corner (2a-1, 2b-1, 2c-1).  The Jacobian
// J[d][r] = dx_d/dxi_r of the trilinear map is evaluated from the 12 edge
// vectors: column r at a point depends only on the other two reference
// coordinates, through a bilinear blend of the 4 edges parallel to r.
// With adj = det(J) J^{-1}:
//   detJ grad N_m . A^{-1} grad N_n = dN_m^T (adj D adj^T / detJ) dN_n,
//   detJ grad N_m . v               = dN_m^T (adj v),       D = diag(a^-2).
// The 2x2x2 Gauss sums are taken in the modal (Walsh) basis of the trilinear
// space: with phi_S = prod_{b in S} xi_b (S a subset of {0,1,2}) the shape
// functions are N_n = 1/8 sum_S eps_n^S phi_S, eps_n^S = prod_{b in S} eps_{n,b},
// so with the Gauss-point sign sums  C^_q = sum_g sigma_q(g) C_g
// (sigma_q(g) = prod_{b in q} sign(xi_{g,b}), xi_g = +-1/sqrt(3) =: +-s):
//   K^[S][T] = s^(|S|+|T|-2) sum_{a in S, b in T} C^_{(S) xor (T)}[a][b],
//   K_e      = 1/64 H K^ H^T,   H[n][S] = eps_n^S = (-1)^|S| W[n][S],
// W the 8-point Walsh-Hadamard matrix: two fast transforms instead of the
// 8 x 36 three-term products of the nodal form.  The load vector is done the
// same way with w_g = adj(J_g) u0(g).  The shape-function values at the
// Gauss points are compile-time constants (sign patterns and powers of
// 1/sqrt(3)).  The float64 kernels unroll every loop; the float-pair kernels
// (the default) keep the Gauss points and transforms in loops over
// per-thread shared memory, because their unrolled code is too long for the
// instruction cache.
//
// Assembly scatters element contributions in 8 launches, one per element
// parity class (i mod 2, j mod 2, k mod 2): elements of one class share no
// node, so there are no atomics and the sums are deterministic.
#include "dfloat.cuh"
#include "kernels.cuh"

namespace mcw {
namespace {

constexpr double kGp = 0.57735026918962576451;  // 1/sqrt(3), the 2-point Gauss abscissa

template <typename R>
struct GeoT {
  R e[3][4][3];  // e[r][q][d]: edge vectors parallel to reference axis r
};
using Geo = GeoT<double>;

__device__ __forceinline__ int64_t sidx(int nx1, int ny1, int i, int j, int k) {
  return ((int64_t)k * ny1 + j) * nx1 + i;
}

// Edge vectors of element (i, j, k).  For axis r the 4 parallel edges are
// indexed q = q1 + 2 q2 by the node bits of the other two axes (in
// increasing axis order).
__device__ __forceinline__ void load_geo(const double* X, const double* Y, const double* Z,
                                         int nx1, int ny1, int i, int j, int k, Geo& G) {
  double xe[8][3];
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    int64_t id = sidx(nx1, ny1, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1));
    xe[n][0] = X[id];
    xe[n][1] = Y[id];
    xe[n][2] = Z[id];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int q1 = q & 1, q2 = q >> 1;
    int nx0 = 0 + 2 * q1 + 4 * q2;   // axis 0 edge: b = q1, c = q2
    int ny0 = q1 + 0 + 4 * q2;       // axis 1 edge: a = q1, c = q2
    int nz0 = q1 + 2 * q2 + 0;       // axis 2 edge: a = q1, b = q2
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      G.e[0][q][d] = xe[nx0 + 1][d] - xe[nx0][d];
      G.e[1][q][d] = xe[ny0 + 2][d] - xe[ny0][d];
      G.e[2][q][d] = xe[nz0 + 4][d] - xe[nz0][d];
    }
  }
}

// Edge vectors from the 8 corner positions xe[n][d] (any arithmetic type).
template <typename R>
__device__ __forceinline__ void edges_of(const R xe[8][3], GeoT<R>& G) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int q1 = q & 1, q2 = q >> 1;
    const int nx0 = 2 * q1 + 4 * q2, ny0 = q1 + 4 * q2, nz0 = q1 + 2 * q2;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      G.e[0][q][d] = xe[nx0 + 1][d] - xe[nx0][d];
      G.e[1][q][d] = xe[ny0 + 2][d] - xe[ny0][d];
      G.e[2][q][d] = xe[nz0 + 4][d] - xe[nz0][d];
    }
  }
}

// Jacobian at reference point xi: J[d][r] = 1/8 sum_q e[r][q][d] (1+s1 t1)(1+s2 t2),
// (t1, t2) = the other two coordinates of xi, s = -1/+1 by the edge's node bits.
__device__ __forceinline__ void jacobian_at(const Geo& G, const double xi[3], double J[3][3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    double t1 = (r == 0) ? xi[1] : xi[0];
    double t2 = (r == 2) ? xi[1] : xi[2];
    double w[4];
    w[0] = 0.125 * (1.0 - t1) * (1.0 - t2);
    w[1] = 0.125 * (1.0 + t1) * (1.0 - t2);
    w[2] = 0.125 * (1.0 - t1) * (1.0 + t2);
    w[3] = 0.125 * (1.0 + t1) * (1.0 + t2);
#pragma unroll
    for (int d = 0; d < 3; ++d)
      J[d][r] = w[0] * G.e[r][0][d] + w[1] * G.e[r][1][d] + w[2] * G.e[r][2][d] +
                w[3] * G.e[r][3][d];
  }
}

// adj[r][d] = det(J) * (J^{-1})[r][d]; returns det(J).
__device__ __forceinline__ double adjugate(const double J[3][3], double adj[3][3]) {
  adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
}

// reference gradient of shape function n at xi
__device__ __forceinline__ void dshape(int n, const double xi[3], double dN[3]) {
  double c0 = (n & 1) ? 1.0 : -1.0, c1 = (n & 2) ? 1.0 : -1.0, c2 = (n & 4) ? 1.0 : -1.0;
  double f0 = 1.0 + c0 * xi[0], f1 = 1.0 + c1 * xi[1], f2 = 1.0 + c2 * xi[2];
  dN[0] = 0.125 * c0 * f1 * f2;
  dN[1] = 0.125 * f0 * c1 * f2;
  dN[2] = 0.125 * f0 * f1 * c2;
}

__device__ __forceinline__ double shape(int n, const double xi[3]) {
  double c0 = (n & 1) ? 1.0 : -1.0, c1 = (n & 2) ? 1.0 : -1.0, c2 = (n & 4) ? 1.0 : -1.0;
  return 0.125 * (1.0 + c0 * xi[0]) * (1.0 + c1 * xi[1]) * (1.0 + c2 * xi[2]);
}

__device__ __forceinline__ void gauss_xi(int g, double xi[3]) {
  xi[0] = (g & 1) ? kGp : -kGp;
  xi[1] = (g & 2) ? kGp : -kGp;
  xi[2] = (g & 4) ? kGp : -kGp;
}

// Thread -> element of parity class (pi, pj, pk).
__device__ __forceinline__ bool elem_of_thread(int nx, int ny, int nz, int cls, int& i, int& j,
                                               int& k) {
  i = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x) + (cls & 1);
  j = 2 * (int)(blockIdx.y * blockDim.y + threadIdx.y) + ((cls >> 1) & 1);
  k = 2 * (int)blockIdx.z + ((cls >> 2) & 1);
  return i < nx && j < ny && k < nz;
}

// The 8 element-parity classes are assembled in the order 0..7.  Among the
// elements that hold both local nodes m and n of element (i, j, k) (m == n:
// the elements around node m), the first to be assembled has parity 0, and
// the last parity 1, along every axis where the two nodes share their
// coordinate and the element on the other side of that coordinate exists;
// along the other axes all of them have this element's parity.
__device__ __forceinline__ bool class_is(int nx, int ny, int nz, int i, int j, int k, int m, int n,
                                         int want) {
  bool ok = true;
  if (((m ^ n) & 1) == 0) {
    const int o = (m & 1) ? i + 1 : i - 1;
    if (o >= 0 && o < nx && (i & 1) != want) ok = false;
  }
  if (((m ^ n) & 2) == 0) {
    const int o = (m & 2) ? j + 1 : j - 1;
    if (o >= 0 && o < ny && (j & 1) != want) ok = false;
  }
  if (((m ^ n) & 4) == 0) {
    const int o = (m & 4) ? k + 1 : k - 1;
    if (o >= 0 && o < nz && (k & 1) != want) ok = false;
  }
  return ok;
}

__host__ __device__ constexpr int popc3(int q) { return (q & 1) + ((q >> 1) & 1) + ((q >> 2) & 1); }
// index of the symmetric 3x3 component (a, b) in (00, 01, 02, 11, 12, 22)
__host__ __device__ constexpr int sym6(int a, int b) {
  return (a < b ? a : b) == 0 ? (a < b ? b : a) : ((a < b ? a : b) == 1 ? 2 + (a < b ? b : a) : 5);
}
__host__ __device__ constexpr double spow(int e) {
  return e == 0 ? 1.0 : (e == 1 ? kGp : (e == 2 ? kGp * kGp : (e == 3 ? kGp * kGp * kGp : kGp * kGp * kGp * kGp)));
}

// Element arithmetic in type R: double (the FP64 pipe) or dflt (float pairs
// on the FP32 pipe, about 48 significant bits).
template <typename R>
struct Num;
template <>
struct Num<double> {
  __device__ static double from(double v) { return v; }
  __device__ static double to(double v) { return v; }
  __device__ static double rcp(double v) { return 1.0 / v; }
  __device__ static bool pos(double v) { return v > 0.0; }
};
template <>
struct Num<dflt> {
  __device__ static dflt from(double v) {
    const float2 t = split_bits(v);
    return {t.x, t.y};
  }
  __device__ static double to(dflt v) { return pair_to_double(v.hi, v.lo); }
  __device__ static dflt rcp(dflt v) { return reciprocal(v); }
  __device__ static bool pos(dflt v) { return positive(v); }
};

// Jacobian columns of the trilinear map at the 2-point Gauss abscissae:
// column r at sign combination q (bit 0: first other axis positive, bit 1:
// second) is 1/8 (S + s sig1 D1 + s sig2 D2 + s^2 sig1 sig2 D12), with S, D1,
// D2, D12 the sum and signed sums of the 4 edges parallel to axis r.
template <typename R>
__device__ __forceinline__ void jac_columns(const GeoT<R>& G, R Jc[3][4][3]) {
  const R cs = Num<R>::from(0.125 * kGp), cs2 = Num<R>::from(0.125 * kGp * kGp);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const R e0 = G.e[r][0][d], e1 = G.e[r][1][d];
      const R e2 = G.e[r][2][d], e3 = G.e[r][3][d];
      const R p0 = e0 + e1, p1 = e2 + e3, m0 = e1 - e0, m1 = e3 - e2;
      const R A = (p0 + p1) * 0.125f, B1 = (m0 + m1) * cs, B2 = (p1 - p0) * cs;
      const R B12 = (m1 - m0) * cs2;
      const R ApB = A + B12, AmB = A - B12, P = B1 + B2, M = B1 - B2;
      Jc[r][3][d] = ApB + P;
      Jc[r][0][d] = ApB - P;
      Jc[r][1][d] = AmB + M;
      Jc[r][2][d] = AmB - M;
    }
}

// Element geometry in arithmetic R: float64 from X, Y, Z; float pairs from the
// pre-split copy xyz2 ([3][nodes] of (hi, lo)).
template <typename R>
__device__ __forceinline__ void load_geo_t(const double* X, const double* Y, const double* Z,
                                           const float2* xyz2, int64_t N, int nx1, int ny1, int i,
                                           int j, int k, GeoT<R>& G) {
  R xe[8][3];
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const int64_t id = sidx(nx1, ny1, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1));
    if constexpr (sizeof(R) == sizeof(double) && !__is_same(R, dflt)) {
      xe[n][0] = X[id];
      xe[n][1] = Y[id];
      xe[n][2] = Z[id];
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float2 v = xyz2[d * N + id];
        xe[n][d] = R{v.x, v.y};
      }
    }
  }
  edges_of<R>(xe, G);
}

// J[d][r] at Gauss point gp from the columns
template <typename R>
__device__ __forceinline__ void jac_at_gauss(const R Jc[3][4][3], int gp, R J[3][3]) {
  const int gx = gp & 1, gy = (gp >> 1) & 1, gz = (gp >> 2) & 1;
  const int q0 = gy + 2 * gz, q1 = gx + 2 * gz, q2 = gx + 2 * gy;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    J[d][0] = Jc[0][q0][d];
    J[d][1] = Jc[1][q1][d];
    J[d][2] = Jc[2][q2][d];
  }
}

template <typename R>
__device__ __forceinline__ R adjugate_t(const R J[3][3], R adj[3][3]) {
  adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
}

template <typename R>
__device__ __forceinline__ void wht8_t(R x[8]) {
#pragma unroll
  for (int h = 1; h < 8; h <<= 1)
#pragma unroll
    for (int i = 0; i < 8; i += 2 * h)
#pragma unroll
      for (int j = i; j < i + h; ++j) {
        const R a = x[j], b = x[j + h];
        x[j] = a + b;
        x[j + h] = a - b;
      }
}

// in-place 8-point Walsh-Hadamard transform y[n] = sum_S (-1)^popcount(n & S) x[S]
__device__ __forceinline__ void wht8(double x[8]) {
#pragma unroll
  for (int h = 1; h < 8; h <<= 1)
#pragma unroll
    for (int i = 0; i < 8; i += 2 * h)
#pragma unroll
      for (int j = i; j < i + h; ++j) {
        const double a = x[j], b = x[j + h];
        x[j] = a + b;
        x[j + h] = a - b;
      }
}

// Stiffness in arithmetic R, fully unrolled; instantiated for float64 (the
// float-pair form is k_assemble_stencil_df below).
template <typename R>
__global__ void __launch_bounds__(128, 4) k_assemble_stencil(Grid g, int nx, int ny, int nz,
                                                          const double* __restrict__ X,
                                                          const double* __restrict__ Y,
                                                          const double* __restrict__ Z,
                                                          const float2* __restrict__ xyz2,
                                                          double d0, double d1, double d2,
                                                          double* __restrict__ C, int* flag,
                                                          int cls) {
  int i, j, k;
  if (!elem_of_thread(nx, ny, nz, cls, i, j, k)) return;
  R Ch[8][6];
  bool bad = false;
  {
    GeoT<R> G;
    load_geo_t<R>(X, Y, Z, xyz2, (int64_t)(nx + 1) * (ny + 1) * (nz + 1), nx + 1, ny + 1, i, j, k, G);
    R Jc[3][4][3];
    jac_columns<R>(G, Jc);
    const R D[3] = {Num<R>::from(d0), Num<R>::from(d1), Num<R>::from(d2)};
    // C_g = adj D adj^T / det at the 8 Gauss points (6 symmetric components)
#pragma unroll
    for (int gp = 0; gp < 8; ++gp) {
      R J[3][3], adj[3][3];
      jac_at_gauss<R>(Jc, gp, J);
      const R det = adjugate_t<R>(J, adj);
      bad |= !Num<R>::pos(det);
      const R inv = Num<R>::rcp(det);
      R aD[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int t = 0; t < 3; ++t) aD[r][t] = adj[r][t] * D[t];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int t = r; t < 3; ++t)
          Ch[gp][sym6(r, t)] = (aD[r][0] * adj[t][0] + aD[r][1] * adj[t][1] + aD[r][2] * adj[t][2]) * inv;
    }
  }
  if (bad) atomicOr(flag, 1);
  // sign sums over the Gauss points: sum_g sigma_q(g) C_g = (-1)^|q| (W C)[q]
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    R v[8];
#pragma unroll
    for (int gp = 0; gp < 8; ++gp) v[gp] = Ch[gp][c];
    wht8_t<R>(v);
#pragma unroll
    for (int q = 0; q < 8; ++q) Ch[q][c] = (popc3(q) & 1) ? -v[q] : v[q];
  }
  // K~ = D K^ D / 64 (D[S] = (-1)^|S|), upper triangle; row and column 0 vanish
  R Kt[8][8];
#pragma unroll
  for (int S = 1; S < 8; ++S)
#pragma unroll
    for (int T = S; T < 8; ++T) {
      R v = Num<R>::from(0.0);
      bool first = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (!((S >> a) & 1)) continue;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          if (!((T >> b) & 1)) continue;
          const R t = Ch[(S & ~(1 << a)) ^ (T & ~(1 << b))][sym6(a, b)];
          v = first ? t : v + t;
          first = false;
        }
      }
      const int e = popc3(S) + popc3(T);
      Kt[S][T] = v * Num<R>::from(spow(e - 2) * ((e & 1) ? -1.0 : 1.0) / 64.0);
    }
  // K_e = W K~ W: transform the rows, then the columns (only m <= n is kept)
#pragma unroll
  for (int S = 0; S < 8; ++S)
#pragma unroll
    for (int T = 0; T < 8; ++T) {
      if (S == 0 || T == 0) Kt[S][T] = Num<R>::from(0.0);
      else if (T < S) Kt[S][T] = Kt[T][S];
    }
#pragma unroll
  for (int S = 1; S < 8; ++S) wht8_t<R>(Kt[S]);
  R Ke[8][8];  // m <= n
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    R col[8];
#pragma unroll
    for (int S = 0; S < 8; ++S) col[S] = Kt[S][n];
    wht8_t<R>(col);
#pragma unroll
    for (int m = 0; m <= n; ++m) Ke[m][n] = col[m];
  }
  // scatter: row of local node m gets Ke[m][n] at offset (n - m).  The 8
  // targets of a row are distinct, so their loads are issued together
  // before the stores (a plain += per target would wait for each round trip).
  bool fr[8];
#pragma unroll
  for (int n = 0; n < 8; ++n)
    fr[n] = is_free(g, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1));
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    if (!fr[m]) continue;
    const int64_t row = gidx(g, i + (m & 1), j + ((m >> 1) & 1), k + ((m >> 2) & 1));
    double cur[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int s = ((n & 1) - (m & 1) + 1) + 3 * (((n >> 1) & 1) - ((m >> 1) & 1) + 1) +
                    9 * (((n >> 2) & 1) - ((m >> 2) & 1) + 1);
      cur[n] = fr[n] ? C[cidx(row, s)] : 0.0;
    }
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int s = ((n & 1) - (m & 1) + 1) + 3 * (((n >> 1) & 1) - ((m >> 1) & 1) + 1) +
                    9 * (((n >> 2) & 1) - ((m >> 2) & 1) + 1);
      if (fr[n]) C[cidx(row, s)] = cur[n] + ((n >= m) ? Ke[m][n] : Ke[n][m]);
    }
  }
}

// The float-pair stiffness kernel with its repeated work in loops.  Fully
// unrolled, the per-element code is about 16 k instructions executed once
// each, and fetching them bounds the kernel (ncu: about half of the stall
// cycles waited for an instruction).  Here the Gauss points, the 6 sign sums, the 15 transforms
// of the 8 x 8 modal matrix and the 8 scatter rows are loops, and the values
// they index by the loop counter live in shared memory (64 float pairs per
// thread, each thread touching only its own column: no barrier).
constexpr int kAsmThreads = 128;
constexpr int kAsmSlots = 64;

__device__ __forceinline__ dflt sel4(const dflt& v0, const dflt& v1, const dflt& v2, const dflt& v3,
                                     int q) {
  const dflt a = (q & 1) ? v1 : v0, b = (q & 1) ? v3 : v2;
  return (q & 2) ? b : a;
}

__global__ void __launch_bounds__(kAsmThreads, 3) k_assemble_stencil_df(
    Grid g, int nx, int ny, int nz, const float2* __restrict__ xyz2, float2 d0, float2 d1,
    float2 d2, double* __restrict__ C, int* flag, int cls) {
  extern __shared__ float2 sm_asm[];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  float2* my = sm_asm + tid;  // slot q of this thread: my[q * kAsmThreads]
  int i, j, k;
  if (!elem_of_thread(nx, ny, nz, cls, i, j, k)) return;
  const dflt D[3] = {{d0.x, d0.y}, {d1.x, d1.y}, {d2.x, d2.y}};
  dflt Jc[3][4][3];
  {
    GeoT<dflt> G;
    load_geo_t<dflt>(nullptr, nullptr, nullptr, xyz2, (int64_t)(nx + 1) * (ny + 1) * (nz + 1),
                     nx + 1, ny + 1, i, j, k, G);
    jac_columns<dflt>(G, Jc);
  }
  // C_g = adj D adj^T / det at Gauss point gp -> slots gp * 6 + c
  bool bad = false;
#pragma unroll 1
  for (int gp = 0; gp < 8; ++gp) {
    const int gx = gp & 1, gy = (gp >> 1) & 1, gz = gp >> 2;
    const int q0 = gy + 2 * gz, q1 = gx + 2 * gz, q2 = gx + 2 * gy;
    dflt J[3][3], adj[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      J[d][0] = sel4(Jc[0][0][d], Jc[0][1][d], Jc[0][2][d], Jc[0][3][d], q0);
      J[d][1] = sel4(Jc[1][0][d], Jc[1][1][d], Jc[1][2][d], Jc[1][3][d], q1);
      J[d][2] = sel4(Jc[2][0][d], Jc[2][1][d], Jc[2][2][d], Jc[2][3][d], q2);
    }
    const dflt det = adjugate_t<dflt>(J, adj);
    bad |= !positive(det);
    const dflt inv = reciprocal(det);
    dflt aD[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int t = 0; t < 3; ++t) aD[r][t] = adj[r][t] * D[t];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int t = r; t < 3; ++t) {
        const dflt v = (aD[r][0] * adj[t][0] + aD[r][1] * adj[t][1] + aD[r][2] * adj[t][2]) * inv;
        my[(gp * 6 + sym6(r, t)) * kAsmThreads] = make_float2(v.hi, v.lo);
      }
  }
  if (bad) atomicOr(flag, 1);
  // sign sums over the Gauss points, in place: sum_g sigma_q(g) C_g = (-1)^|q| (W C)[q]
#pragma unroll 1
  for (int c = 0; c < 6; ++c) {
    dflt v[8];
#pragma unroll
    for (int gp = 0; gp < 8; ++gp) {
      const float2 t = my[(gp * 6 + c) * kAsmThreads];
      v[gp] = dflt{t.x, t.y};
    }
    wht8_t<dflt>(v);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const dflt t = (popc3(q) & 1) ? -v[q] : v[q];
      my[(q * 6 + c) * kAsmThreads] = make_float2(t.hi, t.lo);
    }
  }
  // K~ = D K^ D / 64 (D[S] = (-1)^|S|), upper triangle; row and column 0 vanish
  dflt Kt[28];
#pragma unroll
  for (int S = 1; S < 8; ++S)
#pragma unroll
    for (int T = S; T < 8; ++T) {
      dflt v = dflt{0.0f, 0.0f};
      bool first = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (!((S >> a) & 1)) continue;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          if (!((T >> b) & 1)) continue;
          const float2 w = my[(((S & ~(1 << a)) ^ (T & ~(1 << b))) * 6 + sym6(a, b)) * kAsmThreads];
          v = first ? dflt{w.x, w.y} : v + dflt{w.x, w.y};
          first = false;
        }
      }
      const int e = popc3(S) + popc3(T);
      // upper-triangle index of (S, T), 1 <= S <= T <= 7
      Kt[(S - 1) * (16 - S) / 2 + (T - S)] =
          v * Num<dflt>::from(spow(e - 2) * ((e & 1) ? -1.0 : 1.0) / 64.0);
    }
  // the full symmetric 8 x 8 matrix, slot S * 8 + T
#pragma unroll
  for (int S = 0; S < 8; ++S)
#pragma unroll
    for (int T = 0; T < 8; ++T) {
      const int lo = S < T ? S : T, hi = S < T ? T : S;
      const dflt v = (lo == 0) ? dflt{0.0f, 0.0f} : Kt[(lo - 1) * (16 - lo) / 2 + (hi - lo)];
      my[(S * 8 + T) * kAsmThreads] = make_float2(v.hi, v.lo);
    }
  // K_e = W K~ W: transform the rows (row 0 stays zero), then the columns
#pragma unroll 1
  for (int S = 1; S < 8; ++S) {
    dflt r[8];
#pragma unroll
    for (int T = 0; T < 8; ++T) {
      const float2 t = my[(S * 8 + T) * kAsmThreads];
      r[T] = dflt{t.x, t.y};
    }
    wht8_t<dflt>(r);
#pragma unroll
    for (int T = 0; T < 8; ++T) my[(S * 8 + T) * kAsmThreads] = make_float2(r[T].hi, r[T].lo);
  }
#pragma unroll 1
  for (int n = 0; n < 8; ++n) {
    dflt col[8];
#pragma unroll
    for (int S = 0; S < 8; ++S) {
      const float2 t = my[(S * 8 + n) * kAsmThreads];
      col[S] = dflt{t.x, t.y};
    }
    wht8_t<dflt>(col);
#pragma unroll
    for (int m = 0; m < 8; ++m) my[(m * 8 + n) * kAsmThreads] = make_float2(col[m].hi, col[m].lo);
  }
  // scatter: row of local node m gets K_e[m][n] at offset (n - m), summed in
  // float pairs until the last element class that touches the entry stores
  // it as a double (the first class writes without reading)
  float2* C2 = reinterpret_cast<float2*>(C);
  unsigned freem = 0u;
#pragma unroll
  for (int n = 0; n < 8; ++n)
    if (is_free(g, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1))) freem |= 1u << n;
#pragma unroll 1
  for (int m = 0; m < 8; ++m) {
    if (!((freem >> m) & 1u)) continue;
    const int64_t row = gidx(g, i + (m & 1), j + ((m >> 1) & 1), k + ((m >> 2) & 1));
    float2 cur[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int s = ((n & 1) - (m & 1) + 1) + 3 * (((n >> 1) & 1) - ((m >> 1) & 1) + 1) +
                    9 * (((n >> 2) & 1) - ((m >> 2) & 1) + 1);
      cur[n] = (((freem >> n) & 1u) && !class_is(nx, ny, nz, i, j, k, m, n, 0))
                   ? C2[cidx(row, s)]
                   : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      if (!((freem >> n) & 1u)) continue;
      const int s = ((n & 1) - (m & 1) + 1) + 3 * (((n >> 1) & 1) - ((m >> 1) & 1) + 1) +
                    9 * (((n >> 2) & 1) - ((m >> 2) & 1) + 1);
      const float2 ke = my[((m < n ? m : n) * 8 + (m < n ? n : m)) * kAsmThreads];
      const dflt v = dflt{cur[n].x, cur[n].y} + dflt{ke.x, ke.y};
      if (class_is(nx, ny, nz, i, j, k, m, n, 1))
        C[cidx(row, s)] = pair_to_double(v.hi, v.lo);
      else
        C2[cidx(row, s)] = make_float2(v.hi, v.lo);
    }
  }
}

// out[m] = sum_g dN_m(g) . (adj(J_g) v_g) for the 8 local nodes, v_g given at
// the Gauss points: with w^_q = sum_g sigma_q(g) w_g the modal load is
// f^[S] = s^(|S|-1) sum_{a in S} w^_{S\a}[a] and out = 1/8 H f^.
template <typename R>
__device__ __forceinline__ void weak_div_modal_t(const GeoT<R>& G, const R vg[8][3], R fv[8]) {
  R Jc[3][4][3];
  jac_columns<R>(G, Jc);
  R wh[8][3];
#pragma unroll
  for (int gp = 0; gp < 8; ++gp) {
    R J[3][3], adj[3][3];
    jac_at_gauss<R>(Jc, gp, J);
    adjugate_t<R>(J, adj);
#pragma unroll
    for (int r = 0; r < 3; ++r)
      wh[gp][r] = adj[r][0] * vg[gp][0] + adj[r][1] * vg[gp][1] + adj[r][2] * vg[gp][2];
  }
  // sign sums over the Gauss points, (-1)^|q| (W w)[q]
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    R t[8];
#pragma unroll
    for (int gp = 0; gp < 8; ++gp) t[gp] = wh[gp][r];
    wht8_t<R>(t);
#pragma unroll
    for (int q = 0; q < 8; ++q) wh[q][r] = (popc3(q) & 1) ? -t[q] : t[q];
  }
  // f~[S] = (-1)^|S| f^[S] / 8, then out = W f~
  fv[0] = Num<R>::from(0.0);
#pragma unroll
  for (int S = 1; S < 8; ++S) {
    R v = Num<R>::from(0.0);
    bool first = true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if ((S >> a) & 1) {
        v = first ? wh[S & ~(1 << a)][a] : v + wh[S & ~(1 << a)][a];
        first = false;
      }
    const int e = popc3(S);
    fv[S] = v * Num<R>::from(spow(e - 1) * ((e & 1) ? -1.0 : 1.0) * 0.125);
  }
  wht8_t<R>(fv);
}

template <typename R>
__device__ __forceinline__ void weak_div_modal(const GeoT<R>& G, const R vg[8][3], double out[8]) {
  R fv[8];
  weak_div_modal_t<R>(G, vg, fv);
#pragma unroll
  for (int m = 0; m < 8; ++m) out[m] = Num<R>::to(fv[m]);
}

// one-point rule at the center (weight 8): out[m] = eps_m . (adj(J_0) v_0)
__device__ __forceinline__ void weak_div_center(const Geo& G, const double v[3], double out[8]) {
  double xi[3] = {0.0, 0.0, 0.0}, J[3][3], adj[3][3], w[3];
  jacobian_at(G, xi, J);
  adjugate(J, adj);
#pragma unroll
  for (int r = 0; r < 3; ++r) w[r] = adj[r][0] * v[0] + adj[r][1] * v[1] + adj[r][2] * v[2];
#pragma unroll
  for (int m = 0; m < 8; ++m)
    out[m] = ((m & 1) ? w[0] : -w[0]) + ((m & 2) ? w[1] : -w[1]) + ((m & 4) ? w[2] : -w[2]);
}

__device__ __forceinline__ void load_u(const double* u0, int64_t N, int nx1, int ny1, int i,
                                       int j, int k, double ue[8][3]) {
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    int64_t id = sidx(nx1, ny1, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1));
    ue[n][0] = u0[id];
    ue[n][1] = u0[N + id];
    ue[n][2] = u0[2 * N + id];
  }
}

// nodal values -> values at the 8 Gauss points, u(g) = 1/8 W (s^|S| (W u)):
// the trilinear interpolant's modal coefficients evaluated at xi = +-s.
template <typename R>
__device__ __forceinline__ void interp_gauss_modal(const R ue[8][3], R vg[8][3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R t[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) t[n] = ue[n][d];
    wht8_t<R>(t);
#pragma unroll
    for (int S = 0; S < 8; ++S) t[S] = t[S] * Num<R>::from(spow(popc3(S)) * 0.125);
    wht8_t<R>(t);
#pragma unroll
    for (int gp = 0; gp < 8; ++gp) vg[gp][d] = t[gp];
  }
}

// The float-pair load vector (2x2x2 Gauss, nodal u0: the default mode)
// with its Gauss-point loop and sign sums rolled like the stiffness kernel;
// u0 at the Gauss points and adj(J_g) u0(g) live in shared memory (24 float
// pairs per thread, own column only: no barrier).
constexpr int kRhsSlots = 24;

__global__ void __launch_bounds__(kAsmThreads, 4) k_assemble_rhs_df(
    Grid g, int nx, int ny, int nz, const float2* __restrict__ xyz2, const float2* __restrict__ u2,
    double* __restrict__ f, int cls) {
  extern __shared__ float2 sm_rhs[];
  float2* my = sm_rhs + (threadIdx.y * blockDim.x + threadIdx.x);  // slot q: my[q * kAsmThreads]
  int i, j, k;
  if (!elem_of_thread(nx, ny, nz, cls, i, j, k)) return;
  const int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  // u0 at the Gauss points, 1/8 W (s^|S| (W u)), component d -> slots gp * 3 + d
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dflt t[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const float2 v =
          u2[d * N + sidx(nx + 1, ny + 1, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1))];
      t[n] = dflt{v.x, v.y};
    }
    wht8_t<dflt>(t);
#pragma unroll
    for (int S = 0; S < 8; ++S) t[S] = t[S] * Num<dflt>::from(spow(popc3(S)) * 0.125);
    wht8_t<dflt>(t);
#pragma unroll
    for (int gp = 0; gp < 8; ++gp) my[(gp * 3 + d) * kAsmThreads] = make_float2(t[gp].hi, t[gp].lo);
  }
  dflt Jc[3][4][3];
  {
    GeoT<dflt> G;
    load_geo_t<dflt>(nullptr, nullptr, nullptr, xyz2, N, nx + 1, ny + 1, i, j, k, G);
    jac_columns<dflt>(G, Jc);
  }
  // w_g = adj(J_g) u0(g), written over u0(g)
#pragma unroll 1
  for (int gp = 0; gp < 8; ++gp) {
    const int gx = gp & 1, gy = (gp >> 1) & 1, gz = gp >> 2;
    const int q0 = gy + 2 * gz, q1 = gx + 2 * gz, q2 = gx + 2 * gy;
    dflt J[3][3], adj[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      J[d][0] = sel4(Jc[0][0][d], Jc[0][1][d], Jc[0][2][d], Jc[0][3][d], q0);
      J[d][1] = sel4(Jc[1][0][d], Jc[1][1][d], Jc[1][2][d], Jc[1][3][d], q1);
      J[d][2] = sel4(Jc[2][0][d], Jc[2][1][d], Jc[2][2][d], Jc[2][3][d], q2);
    }
    adjugate_t<dflt>(J, adj);
    dflt v[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float2 t = my[(gp * 3 + d) * kAsmThreads];
      v[d] = dflt{t.x, t.y};
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const dflt w = adj[r][0] * v[0] + adj[r][1] * v[1] + adj[r][2] * v[2];
      my[(gp * 3 + r) * kAsmThreads] = make_float2(w.hi, w.lo);
    }
  }
  // sign sums over the Gauss points, in place: (-1)^|q| (W w)[q]
#pragma unroll 1
  for (int r = 0; r < 3; ++r) {
    dflt t[8];
#pragma unroll
    for (int gp = 0; gp < 8; ++gp) {
      const float2 v = my[(gp * 3 + r) * kAsmThreads];
      t[gp] = dflt{v.x, v.y};
    }
    wht8_t<dflt>(t);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const dflt v = (popc3(q) & 1) ? -t[q] : t[q];
      my[(q * 3 + r) * kAsmThreads] = make_float2(v.hi, v.lo);
    }
  }
  // f~[S] = (-1)^|S| f^[S] / 8, then the nodal load = W f~
  dflt fv[8];
  fv[0] = dflt{0.0f, 0.0f};
#pragma unroll
  for (int S = 1; S < 8; ++S) {
    dflt v = dflt{0.0f, 0.0f};
    bool first = true;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if ((S >> a) & 1) {
        const float2 t = my[((S & ~(1 << a)) * 3 + a) * kAsmThreads];
        v = first ? dflt{t.x, t.y} : v + dflt{t.x, t.y};
        first = false;
      }
    const int e = popc3(S);
    fv[S] = v * Num<dflt>::from(spow(e - 1) * ((e & 1) ? -1.0 : 1.0) * 0.125);
  }
  wht8_t<dflt>(fv);
  // the 8 node rows are distinct: all loads first, then the stores
  double cur[8];
  bool fr[8];
  int64_t at[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int im = i + (m & 1), jm = j + ((m >> 1) & 1), km = k + ((m >> 2) & 1);
    fr[m] = is_free(g, im, jm, km);
    at[m] = gidx(g, im, jm, km);
    cur[m] = fr[m] ? f[at[m]] : 0.0;
  }
#pragma unroll
  for (int m = 0; m < 8; ++m)
    if (fr[m]) f[at[m]] = cur[m] - to_double(fv[m]);  // 8 per element: the double pipe is idle here
}

// QUAD: bit 0 = one-point rule at the center, bit 1 = u0 given at the
// element centers (a compile-time choice, so that each kernel carries only
// its own code).
template <typename R, int QUAD>
__global__ void __launch_bounds__(128, 3) k_assemble_rhs(Grid g, int nx, int ny, int nz,
                                                      const double* __restrict__ X,
                                                      const double* __restrict__ Y,
                                                      const double* __restrict__ Z,
                                                      const float2* __restrict__ xyz2,
                                                      const double* __restrict__ u0,
                                                      const float2* __restrict__ u2,
                                                      double* __restrict__ f, int cls) {
  constexpr int quad = QUAD;
  int i, j, k;
  if (!elem_of_thread(nx, ny, nz, cls, i, j, k)) return;
  R fe[8];
  const int64_t NE = (int64_t)nx * ny * nz, e = ((int64_t)k * ny + j) * nx + i;
  const int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  if constexpr ((quad & 1) != 0) {
    Geo G;
    load_geo(X, Y, Z, nx + 1, ny + 1, i, j, k, G);
    double v[3];
    if constexpr ((quad & 2) != 0) {
      v[0] = u0[e]; v[1] = u0[NE + e]; v[2] = u0[2 * NE + e];
    } else {
      double ue[8][3];
      load_u(u0, N, nx + 1, ny + 1, i, j, k, ue);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double sum = 0.0;
#pragma unroll
        for (int n = 0; n < 8; ++n) sum += ue[n][d];
        v[d] = 0.125 * sum;
      }
    }
    double fd[8];
    weak_div_center(G, v, fd);
#pragma unroll
    for (int m = 0; m < 8; ++m) fe[m] = Num<R>::from(fd[m]);
  } else {
    GeoT<R> G;
    load_geo_t<R>(X, Y, Z, xyz2, N, nx + 1, ny + 1, i, j, k, G);
    R vg[8][3];
    if constexpr ((quad & 2) != 0) {
      // u0 given at the element centers: constant over the element
      const R c0 = Num<R>::from(u0[e]), c1 = Num<R>::from(u0[NE + e]), c2 = Num<R>::from(u0[2 * NE + e]);
#pragma unroll
      for (int gp = 0; gp < 8; ++gp) { vg[gp][0] = c0; vg[gp][1] = c1; vg[gp][2] = c2; }
    } else {
      R ue[8][3];
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        const int64_t id = sidx(nx + 1, ny + 1, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1));
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if constexpr (__is_same(R, dflt)) {
            const float2 v = u2[d * N + id];
            ue[n][d] = R{v.x, v.y};
          } else {
            ue[n][d] = u0[d * N + id];
          }
        }
      }
      interp_gauss_modal<R>(ue, vg);
    }
    weak_div_modal_t<R>(G, vg, fe);
  }
  // the 8 node rows are distinct: all loads first, then the stores.  (Float
  // pairs for these 8 sums, as in the stiffness scatter, measured slower:
  // the double adds here are few.)
  double cur[8];
  bool fr[8];
  int64_t at[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int im = i + (m & 1), jm = j + ((m >> 1) & 1), km = k + ((m >> 2) & 1);
    fr[m] = is_free(g, im, jm, km);
    at[m] = gidx(g, im, jm, km);
    cur[m] = fr[m] ? f[at[m]] : 0.0;
  }
#pragma unroll
  for (int m = 0; m < 8; ++m)
    if (fr[m]) f[at[m]] = cur[m] - Num<R>::to(fe[m]);
}

// float64 -> (hi, lo) float pairs, n values, split in integer arithmetic
// (the double pipe would bound this copy), 4 values per thread and turn
__global__ void k_split_pairs(const double* __restrict__ a, float2* __restrict__ b, int64_t n) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; t + 3 * st < n; t += 4 * st) {
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = a[t + q * st];
#pragma unroll
    for (int q = 0; q < 4; ++q) b[t + q * st] = split_bits(v[q]);
  }
  for (; t < n; t += st) b[t] = split_bits(a[t]);
}

__global__ void __launch_bounds__(128) k_weak_div(int nx, int ny, int nz,
                                                  const double* __restrict__ X,
                                                  const double* __restrict__ Y,
                                                  const double* __restrict__ Z,
                                                  const double* __restrict__ ug,
                                                  double* __restrict__ out, int cls) {
  int i, j, k;
  if (!elem_of_thread(nx, ny, nz, cls, i, j, k)) return;
  Geo G;
  load_geo(X, Y, Z, nx + 1, ny + 1, i, j, k, G);
  const int64_t NE = (int64_t)nx * ny * nz, e = ((int64_t)k * ny + j) * nx + i;
  double vg[8][3];
#pragma unroll
  for (int gp = 0; gp < 8; ++gp)
#pragma unroll
    for (int d = 0; d < 3; ++d) vg[gp][d] = ug[((int64_t)d * 8 + gp) * NE + e];
  double be[8];
  weak_div_modal<double>(G, vg, be);
#pragma unroll
  for (int m = 0; m < 8; ++m)
    out[sidx(nx + 1, ny + 1, i + (m & 1), j + ((m >> 1) & 1), k + ((m >> 2) & 1))] += be[m];
}

template <int NG>
__global__ void __launch_bounds__(128) k_recover(Grid g, int nx, int ny, int nz,
                                                 const double* __restrict__ X,
                                                 const double* __restrict__ Y,
                                                 const double* __restrict__ Z,
                                                 const double* __restrict__ u0,
                                                 const double* __restrict__ lam, double d0,
                                                 double d1, double d2, int u0_centers,
                                                 double* __restrict__ u) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z;
  if (i >= nx || j >= ny || k >= nz) return;
  Geo G;
  load_geo(X, Y, Z, nx + 1, ny + 1, i, j, k, G);
  double ue[8][3], le[8];
  const int64_t NEc = (int64_t)nx * ny * nz, ec = ((int64_t)k * ny + j) * nx + i;
  if (u0_centers) {
    // u0 given at the element centers: the same value at every corner
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int d = 0; d < 3; ++d) ue[n][d] = u0[d * NEc + ec];
  } else {
    int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
    load_u(u0, N, nx + 1, ny + 1, i, j, k, ue);
  }
#pragma unroll
  for (int n = 0; n < 8; ++n) le[n] = lam[gidx(g, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1))];
  int64_t NE = (int64_t)nx * ny * nz, e = ((int64_t)k * ny + j) * nx + i;
  const int ng = NG;
  const double dd[3] = {d0, d1, d2};
#pragma unroll
  for (int gp = 0; gp < NG; ++gp) {
    double xi[3] = {0.0, 0.0, 0.0}, J[3][3], adj[3][3];
    if (NG == 8) gauss_xi(gp, xi);
    jacobian_at(G, xi, J);
    double det = adjugate(J, adj);
    double gr[3] = {0.0, 0.0, 0.0}, up[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      double dN[3], N = shape(n, xi);
      dshape(n, xi, dN);
#pragma unroll
      for (int r = 0; r < 3; ++r) gr[r] += le[n] * dN[r];
#pragma unroll
      for (int d = 0; d < 3; ++d) up[d] += N * ue[n][d];
    }
    double inv = 1.0 / det;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // grad lambda_d = sum_r (J^{-1})[r][d] * gr[r]
      double gd = (adj[0][d] * gr[0] + adj[1][d] * gr[1] + adj[2][d] * gr[2]) * inv;
      u[((int64_t)d * ng + gp) * NE + e] = up[d] + gd * dd[d];
    }
  }
}

// Recovery at the element centers in float pairs: coordinates, lambda and a
// nodal u0 pre-split into (hi, lo) pairs in the [k][j][i] layout.  At the
// center the Jacobian columns are the edge means, dN_n/dxi_r = eps_{n,r}/8 and
// N_n = 1/8.
__global__ void __launch_bounds__(128) k_recover_center_df(int nx, int ny, int nz,
                                                           const float2* __restrict__ xyz2,
                                                           const float2* __restrict__ u2,
                                                           const double* __restrict__ u0c,
                                                           const float2* __restrict__ lam2,
                                                           float2 d0, float2 d1, float2 d2,
                                                           double* __restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= nx || j >= ny || k >= nz) return;
  const int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  GeoT<dflt> G;
  load_geo_t<dflt>(nullptr, nullptr, nullptr, xyz2, N, nx + 1, ny + 1, i, j, k, G);
  dflt J[3][3], adj[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int d = 0; d < 3; ++d)
      J[d][r] = ((G.e[r][0][d] + G.e[r][1][d]) + (G.e[r][2][d] + G.e[r][3][d])) * 0.125f;
  const dflt inv = reciprocal(adjugate_t<dflt>(J, adj));
  dflt le[8];
  int64_t id[8];
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    id[n] = sidx(nx + 1, ny + 1, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1));
    const float2 v = lam2[id[n]];
    le[n] = dflt{v.x, v.y};
  }
  // reference gradient at the center: 1/8 sum_n eps_{n,r} lambda_n, i.e. 1/8 the
  // sum of the 4 differences along the edges parallel to axis r
  dflt gr[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int b = 1 << r;
    dflt acc = le[b] - le[0];
#pragma unroll
    for (int n = 0; n < 8; ++n)
      if (((n >> r) & 1) && n != b) acc = acc + (le[n] - le[n ^ b]);
    gr[r] = acc * 0.125f;
  }
  const int64_t NE = (int64_t)nx * ny * nz, e = ((int64_t)k * ny + j) * nx + i;
  const dflt dd[3] = {{d0.x, d0.y}, {d1.x, d1.y}, {d2.x, d2.y}};
  // no double-pipe instruction: inputs split and the output formed in
  // integer arithmetic
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dflt uc;
    if (u0c) {
      const float2 v = split_bits(u0c[d * NE + e]);
      uc = dflt{v.x, v.y};
    } else {
      float2 v = u2[d * N + id[0]];
      uc = dflt{v.x, v.y};
#pragma unroll
      for (int n = 1; n < 8; ++n) {
        v = u2[d * N + id[n]];
        uc = uc + dflt{v.x, v.y};
      }
      uc = uc * 0.125f;
    }
    const dflt gd = (adj[0][d] * gr[0] + adj[1][d] * gr[1] + adj[2][d] * gr[2]) * inv;
    const dflt ud = uc + gd * dd[d];
    u[(int64_t)d * NE + e] = pair_to_double(ud.hi, ud.lo);
  }
}

// ---- adjoint of the recovery and of the load vector (gradients) ----------
//
// Forward at element centers: u = C u0 + A^{-1} G lambda, lambda = K^{-1} f,
// f = -B I u0 (I: nodes -> Gauss points, B: weak divergence, C: nodes ->
// centers, G: gradient at the centers).  For a loss with dl/du = gu:
//   dl/du0 = C^T gu - I^T B^T mu,   mu = K^{-1} h,   h = G^T A^{-1} gu,
//   dl/dlog a_d = 2 a_d^-2 (E_d - T_d),
//   E_d = mu^T K_d lambda = sum_e sum_g detJ (d_d mu)(d_d lambda),
//   T_d = sum_centers gu_d (d_d lambda)(center).

// h = G^T A^{-1} gu and du0 = C^T gu (u0 at a center is the mean of the 8
// corners), scattered per element class; h, du0 in the [k][j][i] layout.
__global__ void __launch_bounds__(128) k_recover_adjoint(int nx, int ny, int nz,
                                                         const double* __restrict__ X,
                                                         const double* __restrict__ Y,
                                                         const double* __restrict__ Z,
                                                         const double* __restrict__ gu, double d0,
                                                         double d1, double d2,
                                                         double* __restrict__ h,
                                                         double* __restrict__ du0, int cls) {
  int i, j, k;
  if (!elem_of_thread(nx, ny, nz, cls, i, j, k)) return;
  const int64_t NE = (int64_t)nx * ny * nz, e = ((int64_t)k * ny + j) * nx + i;
  const double g0 = gu[e], g1 = gu[NE + e], g2 = gu[2 * NE + e];
  if (g0 == 0.0 && g1 == 0.0 && g2 == 0.0) return;
  Geo G;
  load_geo(X, Y, Z, nx + 1, ny + 1, i, j, k, G);
  const double xi[3] = {0.0, 0.0, 0.0};
  double J[3][3], adj[3][3];
  jacobian_at(G, xi, J);
  const double inv = 1.0 / adjugate(J, adj);
  const double v[3] = {g0 * d0, g1 * d1, g2 * d2};
  double w[3];  // J^{-1} v
#pragma unroll
  for (int r = 0; r < 3; ++r) w[r] = (adj[r][0] * v[0] + adj[r][1] * v[1] + adj[r][2] * v[2]) * inv;
  const int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    double dN[3];
    dshape(n, xi, dN);
    const int64_t id = sidx(nx + 1, ny + 1, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1));
    h[id] += dN[0] * w[0] + dN[1] * w[1] + dN[2] * w[2];
    du0[id] += 0.125 * g0;
    du0[N + id] += 0.125 * g1;
    du0[2 * N + id] += 0.125 * g2;
  }
}

// du0 -= I^T B^T mu per element class, and block partials of (E_0..2, T_0..2).
__global__ void __launch_bounds__(128) k_adjoint_finish(int nx, int ny, int nz,
                                                        const double* __restrict__ X,
                                                        const double* __restrict__ Y,
                                                        const double* __restrict__ Z,
                                                        const double* __restrict__ mu,
                                                        const double* __restrict__ lam,
                                                        const double* __restrict__ gu,
                                                        double* __restrict__ du0,
                                                        double* __restrict__ partials, int cls) {
  int i, j, k;
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (elem_of_thread(nx, ny, nz, cls, i, j, k)) {
    Geo G;
    load_geo(X, Y, Z, nx + 1, ny + 1, i, j, k, G);
    double me[8], le[8];
    int64_t id[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      id[n] = sidx(nx + 1, ny + 1, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1));
      me[n] = mu[id[n]];
      le[n] = lam[id[n]];
    }
    double out[8][3];
#pragma unroll
    for (int n = 0; n < 8; ++n) out[n][0] = out[n][1] = out[n][2] = 0.0;
#pragma unroll
    for (int gp = 0; gp < 8; ++gp) {
      double xi[3], J[3][3], adj[3][3];
      gauss_xi(gp, xi);
      jacobian_at(G, xi, J);
      const double inv = 1.0 / adjugate(J, adj);
      double dm[3] = {0.0, 0.0, 0.0}, dl[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        double dN[3];
        dshape(n, xi, dN);
#pragma unroll
        for (int r = 0; r < 3; ++r) { dm[r] += me[n] * dN[r]; dl[r] += le[n] * dN[r]; }
      }
      double gm[3], gl[3];  // detJ grad mu, detJ grad lambda (adj^T times the reference gradient)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        gm[d] = adj[0][d] * dm[0] + adj[1][d] * dm[1] + adj[2][d] * dm[2];
        gl[d] = adj[0][d] * dl[0] + adj[1][d] * dl[1] + adj[2][d] * dl[2];
        acc[d] += gm[d] * gl[d] * inv;
      }
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        const double Nn = shape(n, xi);
#pragma unroll
        for (int d = 0; d < 3; ++d) out[n][d] -= Nn * gm[d];
      }
    }
    const int64_t NE = (int64_t)nx * ny * nz, e = ((int64_t)k * ny + j) * nx + i;
    const double gc[3] = {gu[e], gu[NE + e], gu[2 * NE + e]};
    if (gc[0] != 0.0 || gc[1] != 0.0 || gc[2] != 0.0) {
      const double xi[3] = {0.0, 0.0, 0.0};
      double J[3][3], adj[3][3], dl[3] = {0.0, 0.0, 0.0};
      jacobian_at(G, xi, J);
      const double inv = 1.0 / adjugate(J, adj);
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        double dN[3];
        dshape(n, xi, dN);
#pragma unroll
        for (int r = 0; r < 3; ++r) dl[r] += le[n] * dN[r];
      }
#pragma unroll
      for (int d = 0; d < 3; ++d)
        acc[3 + d] += gc[d] * (adj[0][d] * dl[0] + adj[1][d] * dl[1] + adj[2][d] * dl[2]) * inv;
    }
    const int64_t N = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int d = 0; d < 3; ++d) du0[d * N + id[n]] += out[n][d];
  }
  __shared__ double red[6][4];
#pragma unroll
  for (int q = 0; q < 6; ++q)
    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  if ((t & 31) == 0)
#pragma unroll
    for (int q = 0; q < 6; ++q) red[q][t >> 5] = acc[q];
  __syncthreads();
  if (t == 0) {
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
    for (int q = 0; q < 6; ++q) partials[blk * 6 + q] = red[q][0] + red[q][1] + red[q][2] + red[q][3];
  }
}

// fixed-order sum of n six-component partials
__global__ void __launch_bounds__(32) k_sum6(const double* __restrict__ p, int n, double* out) {
  const int q = threadIdx.x;
  if (q >= 6) return;
  double s = 0.0;
  for (int b = 0; b < n; ++b) s += p[(int64_t)b * 6 + q];
  out[q] = s;
}

dim3 elem_grid(int nx, int ny, int nz, int cls, dim3 blk) {
  int ci = (nx - (cls & 1) + 1) / 2, cj = (ny - ((cls >> 1) & 1) + 1) / 2;
  int ck = (nz - ((cls >> 2) & 1) + 1) / 2;
  return dim3((ci + blk.x - 1) / blk.x, (cj + blk.y - 1) / blk.y, ck);
}

}  // namespace

cudaError_t launch_split_pairs(const double* a, float2* b, int64_t n, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_split_pairs<<<blocks, 256, 0, st>>>(a, b, n);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_assemble_stencil(const Grid& g, int nx, int ny, int nz, const double* X,
                                    const double* Y, const double* Z, const float2* xyz2,
                                    const double* a, double* C, int* flag, int dfloat,
                                    cudaStream_t st) {
  dim3 blk(32, 4, 1);
  const size_t smem = sizeof(float2) * kAsmSlots * kAsmThreads;
  if (dfloat) {
    const cudaError_t e = cudaFuncSetAttribute(k_assemble_stencil_df,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  for (int cls = 0; cls < 8; ++cls) {
    dim3 grd = elem_grid(nx, ny, nz, cls, blk);
    if (grd.x == 0 || grd.y == 0 || grd.z == 0) continue;
    const double d0 = 1.0 / (a[0] * a[0]), d1 = 1.0 / (a[1] * a[1]), d2 = 1.0 / (a[2] * a[2]);
    if (dfloat)
      k_assemble_stencil_df<<<grd, blk, smem, st>>>(g, nx, ny, nz, xyz2, split_bits(d0), split_bits(d1),
                                                    split_bits(d2), C, flag, cls);
    else
      k_assemble_stencil<double><<<grd, blk, 0, st>>>(g, nx, ny, nz, X, Y, Z, xyz2, d0, d1, d2, C, flag, cls);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_assemble_rhs(const Grid& g, int nx, int ny, int nz, const double* X,
                                const double* Y, const double* Z, const float2* xyz2,
                                const double* u0, const float2* u2, int quad, double* f,
                                int dfloat, cudaStream_t st) {
  dim3 blk(32, 4, 1);
  for (int cls = 0; cls < 8; ++cls) {
    dim3 grd = elem_grid(nx, ny, nz, cls, blk);
    if (grd.x == 0 || grd.y == 0 || grd.z == 0) continue;
#define MCW_RHS(Q)                                                                            \
  do {                                                                                        \
    if (dfloat)                                                                               \
      k_assemble_rhs<dflt, Q><<<grd, blk, 0, st>>>(g, nx, ny, nz, X, Y, Z, xyz2, u0, u2, f, cls); \
    else                                                                                      \
      k_assemble_rhs<double, Q><<<grd, blk, 0, st>>>(g, nx, ny, nz, X, Y, Z, xyz2, u0, u2, f, cls); \
  } while (0)
    switch (quad & 3) {
      case 0:
        if (dfloat)
          k_assemble_rhs_df<<<grd, blk, sizeof(float2) * kRhsSlots * kAsmThreads, st>>>(
              g, nx, ny, nz, xyz2, u2, f, cls);
        else
          MCW_RHS(0);
        break;
      case 1: MCW_RHS(1); break;
      case 2: MCW_RHS(2); break;
      default: MCW_RHS(3); break;
    }
#undef MCW_RHS
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_weak_div(int nx, int ny, int nz, const double* X, const double* Y,
                            const double* Z, const double* ug, double* out, cudaStream_t st) {
  dim3 blk(32, 4, 1);
  for (int cls = 0; cls < 8; ++cls) {
    dim3 grd = elem_grid(nx, ny, nz, cls, blk);
    if (grd.x == 0 || grd.y == 0 || grd.z == 0) continue;
    k_weak_div<<<grd, blk, 0, st>>>(nx, ny, nz, X, Y, Z, ug, out, cls); count_launches(1);
  }
  return cudaGetLastError();
}

int adjoint_partials(int nx, int ny, int nz) {
  dim3 blk(32, 4, 1);
  int total = 0;
  for (int cls = 0; cls < 8; ++cls) {
    dim3 grd = elem_grid(nx, ny, nz, cls, blk);
    total += (int)(grd.x * grd.y * grd.z);
  }
  return total;
}

cudaError_t launch_recover_adjoint(int nx, int ny, int nz, const double* X, const double* Y,
                                   const double* Z, const double* gu, const double* a, double* h,
                                   double* du0, cudaStream_t st) {
  dim3 blk(32, 4, 1);
  for (int cls = 0; cls < 8; ++cls) {
    dim3 grd = elem_grid(nx, ny, nz, cls, blk);
    if (grd.x == 0 || grd.y == 0 || grd.z == 0) continue;
    k_recover_adjoint<<<grd, blk, 0, st>>>(nx, ny, nz, X, Y, Z, gu, 1.0 / (a[0] * a[0]),
                                           1.0 / (a[1] * a[1]), 1.0 / (a[2] * a[2]), h, du0, cls);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_adjoint_finish(int nx, int ny, int nz, const double* X, const double* Y,
                                  const double* Z, const double* mu, const double* lam,
                                  const double* gu, double* du0, double* partials, int cap,
                                  double* sums6, cudaStream_t st) {
  dim3 blk(32, 4, 1);
  const int total = adjoint_partials(nx, ny, nz);
  if (total > cap) return cudaErrorInvalidValue;
  int off = 0;
  for (int cls = 0; cls < 8; ++cls) {
    dim3 grd = elem_grid(nx, ny, nz, cls, blk);
    const int nb = (int)(grd.x * grd.y * grd.z);
    if (nb == 0) continue;
    k_adjoint_finish<<<grd, blk, 0, st>>>(nx, ny, nz, X, Y, Z, mu, lam, gu, du0,
                                          partials + (int64_t)off * 6, cls);
    count_launches(1);
    off += nb;
  }
  k_sum6<<<1, 32, 0, st>>>(partials, off, sums6);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_recover_center_df(int nx, int ny, int nz, const float2* xyz2, const float2* u2,
                                     const double* u0c, const float2* lam2, const double* a,
                                     double* u, cudaStream_t st) {
  dim3 blk(32, 4, 1);
  dim3 grd((nx + 31) / 32, (ny + 3) / 4, nz);
  k_recover_center_df<<<grd, blk, 0, st>>>(nx, ny, nz, xyz2, u2, u0c, lam2,
                                           split_bits(1.0 / (a[0] * a[0])),
                                           split_bits(1.0 / (a[1] * a[1])),
                                           split_bits(1.0 / (a[2] * a[2])), u);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_recover(const Grid& g, int nx, int ny, int nz, const double* X,
                           const double* Y, const double* Z, const double* u0,
                           const double* lam, const double* a, int where, int u0_centers,
                           double* u, cudaStream_t st) {
  dim3 blk(32, 4, 1);
  dim3 grd((nx + 31) / 32, (ny + 3) / 4, nz);
  if (where == 0)
    k_recover<1><<<grd, blk, 0, st>>>(g, nx, ny, nz, X, Y, Z, u0, lam, 1.0 / (a[0] * a[0]),
                                      1.0 / (a[1] * a[1]), 1.0 / (a[2] * a[2]), u0_centers, u);
  else
    k_recover<8><<<grd, blk, 0, st>>>(g, nx, ny, nz, X, Y, Z, u0, lam, 1.0 / (a[0] * a[0]),
                                      1.0 / (a[1] * a[1]), 1.0 / (a[2] * a[2]), u0_centers, u);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mcw
