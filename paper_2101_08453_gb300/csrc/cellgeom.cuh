// Geometry of one horizontal cell of a shift-form grid at the 2 x 2 Gauss
// points in (xi1, xi2), in a chosen arithmetic: float64, or float pairs
// (dflt, about 48 significant bits on the float pipe).  The bilinear map's
// derivatives are taken from the cell's edge vectors, whose differences of
// neighbouring coordinates are formed in float64 first (exact for nearby
// values), so the pairs never see the cancellation of large coordinates.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dfloat.cuh"

namespace mcw {

template <typename R>
struct Arith;

template <>
struct Arith<double> {
  static __device__ __forceinline__ double from(double v) { return v; }
  static __device__ __forceinline__ double to_double(double v) { return v; }
  static __device__ __forceinline__ double rcp(double v) { return 1.0 / v; }
  static __device__ __forceinline__ bool pos(double v) { return v > 0.0; }
  static __device__ __forceinline__ double zero() { return 0.0; }
};

template <>
struct Arith<dflt> {
  static __device__ __forceinline__ dflt from(double v) {
    const float2 p = split_bits(v);
    return {p.x, p.y};
  }
  static __device__ __forceinline__ double to_double(dflt v) { return pair_to_double(v.hi, v.lo); }
  static __device__ __forceinline__ dflt rcp(dflt v) { return reciprocal(v); }
  static __device__ __forceinline__ bool pos(dflt v) { return positive(v); }
  static __device__ __forceinline__ dflt zero() { return {0.0f, 0.0f}; }
};

// The 2 x 2 Gauss abscissa 1/sqrt(3) in float64.
constexpr double kGauss2 = 0.57735026918962576451;

// Edge vectors of a cell with corners p = a + 2b (node (ci + a, cj + b)):
// e[0] = c1 - c0 and e[1] = c3 - c2 run along xi1, e[2] = c2 - c0 and
// e[3] = c3 - c1 along xi2, for each coordinate.
template <typename R>
struct CellEdges {
  R x[4], y[4], z[4];
};

template <typename R>
__device__ __forceinline__ CellEdges<R> cell_edges(const double* xs, const double* ys,
                                                   const double* zs) {
  CellEdges<R> c;
  const int lo[4] = {0, 2, 0, 1}, hi[4] = {1, 3, 2, 3};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    c.x[e] = Arith<R>::from(xs[hi[e]] - xs[lo[e]]);
    c.y[e] = Arith<R>::from(ys[hi[e]] - ys[lo[e]]);
    c.z[e] = Arith<R>::from(zs[hi[e]] - zs[lo[e]]);
  }
  return c;
}

// Shape values and derivatives of corner p at the Gauss point gq (xi1 =
// -+1/sqrt(3) by bit 0, xi2 by bit 1), in float64 (constants once unrolled).
__device__ __forceinline__ double gauss_phi(int gq, int p) {
  const double e1 = (gq & 1) ? kGauss2 : -kGauss2, e2 = (gq & 2) ? kGauss2 : -kGauss2;
  const double sx = (p & 1) ? 1.0 : -1.0, sy = (p & 2) ? 1.0 : -1.0;
  return 0.25 * (1.0 + sx * e1) * (1.0 + sy * e2);
}
__device__ __forceinline__ double gauss_d1(int gq, int p) {
  const double e2 = (gq & 2) ? kGauss2 : -kGauss2;
  const double sx = (p & 1) ? 1.0 : -1.0, sy = (p & 2) ? 1.0 : -1.0;
  return 0.25 * sx * (1.0 + sy * e2);
}
__device__ __forceinline__ double gauss_d2(int gq, int p) {
  const double e1 = (gq & 1) ? kGauss2 : -kGauss2;
  const double sx = (p & 1) ? 1.0 : -1.0, sy = (p & 2) ? 1.0 : -1.0;
  return 0.25 * sy * (1.0 + sx * e1);
}

// Derivatives of the bilinear map at Gauss point gq from the edges:
// d/dxi1 = ((1 - xi2) e[0] + (1 + xi2) e[1]) / 4, d/dxi2 = ((1 - xi1) e[2] +
// (1 + xi1) e[3]) / 4.  J = [[x1, x2], [y1, y2]], z' = (z1, z2).
template <typename R>
struct GaussGeom {
  R J00, J01, J10, J11, z1, z2;
};

template <typename R>
__device__ __forceinline__ GaussGeom<R> gauss_geom(const CellEdges<R>& c, int gq) {
  const double e1 = (gq & 1) ? kGauss2 : -kGauss2, e2 = (gq & 2) ? kGauss2 : -kGauss2;
  const R a0 = Arith<R>::from(0.25 * (1.0 - e2)), a1 = Arith<R>::from(0.25 * (1.0 + e2));
  const R b0 = Arith<R>::from(0.25 * (1.0 - e1)), b1 = Arith<R>::from(0.25 * (1.0 + e1));
  GaussGeom<R> G;
  G.J00 = a0 * c.x[0] + a1 * c.x[1];
  G.J01 = b0 * c.x[2] + b1 * c.x[3];
  G.J10 = a0 * c.y[0] + a1 * c.y[1];
  G.J11 = b0 * c.y[2] + b1 * c.y[3];
  G.z1 = a0 * c.z[0] + a1 * c.z[1];
  G.z2 = b0 * c.z[2] + b1 * c.z[3];
  return G;
}

}  // namespace mcw
