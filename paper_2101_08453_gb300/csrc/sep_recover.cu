// Recovery of the wind at the element centers, u = u0 + A^-1 grad lambda
// (Eq. 3), on a terrain-following grid in shift form (MCWIND_OP_SEPARABLE
// with float-pair element arithmetic).
//
// In shift form x and y do not depend on the layer and z = z_s(x, y) +
// zeta_k, so at an element's center the Jacobian of the trilinear map is
//   J = [[J2, 0], [z'^T, h/2]]
// with J2 the horizontal Jacobian and z' the terrain slope of the column
// (both at the cell center, the same in every layer) and h the layer's
// thickness.  With g = grad_xi lambda at the center,
//   d lambda/dz = (2/h) g_3,   (d lambda/dx, d lambda/dy) = J2^-T (g_h - z' d lambda/dz),
// so the column's J2^-T and z' are formed once and each element needs only
// its layer's 2/h.  One thread per element column walks the layers; the
// reference gradient and u0's center value come from per-layer sums over
// the 4 corners of a node layer, each formed once and used by the element
// below and the one above:
//   g_1 = (D1(k) + D1(k+1)) / 8, D1 = (l1 - l0) + (l3 - l2)  (corner p = a + 2b),
//   g_2 = (D2(k) + D2(k+1)) / 8, D2 = (l2 - l0) + (l3 - l1),
//   g_3 = (S(k+1) - S(k)) / 8,    S = l0 + l1 + l2 + l3,
//   u0(center) = (S_u(k) + S_u(k+1)) / 8.
// Everything after reading runs in float pairs (about 48 significant bits);
// lambda and u0 are split in integer arithmetic and u is formed in integer
// arithmetic, so the kernel takes no double-pipe instruction but the layer
// thicknesses' reciprocals.
#include "cellgeom.cuh"
#include "dfloat.cuh"
#include "kernels.cuh"

namespace mcw {
namespace {

__device__ __forceinline__ dflt pair_of(double v) {
  const float2 p = split_bits(v);
  return {p.x, p.y};
}

// per node layer of one element column: the lambda sums D1, D2, S and u0's
// corner sums
struct LayerSums {
  dflt d1, d2, s, su[3];
};

__device__ __forceinline__ LayerSums layer_sums(const double* __restrict__ lam,
                                                const double* __restrict__ u0, int64_t N,
                                                const int64_t* c, bool with_u0) {
  LayerSums L;
  dflt l[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) l[p] = pair_of(lam[c[p]]);
  L.d1 = (l[1] - l[0]) + (l[3] - l[2]);
  L.d2 = (l[2] - l[0]) + (l[3] - l[1]);
  L.s = (l[0] + l[1]) + (l[2] + l[3]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (with_u0) {
      dflt v[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) v[p] = pair_of(u0[d * N + c[p]]);
      L.su[d] = (v[0] + v[1]) + (v[2] + v[3]);
    } else {
      L.su[d] = dflt{0.0f, 0.0f};
    }
  }
  return L;
}

__global__ void __launch_bounds__(128) k_recover_center_sep(int nx, int ny, int nz,
                                                            const double* __restrict__ X,
                                                            const double* __restrict__ Y,
                                                            const double* __restrict__ Z,
                                                            const double* __restrict__ u0,
                                                            const double* __restrict__ u0c,
                                                            const double* __restrict__ lam,
                                                            float2 a0, float2 a1, float2 a2,
                                                            double* __restrict__ u) {
  __shared__ float2 rh[kMaxZ];  // 2 / h of each element layer
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int k = tid; k < nz; k += blockDim.x * blockDim.y)
    rh[k] = split_bits(2.0 / (Z[(int64_t)(k + 1) * (nx + 1) * (ny + 1)] - Z[(int64_t)k * (nx + 1) * (ny + 1)]));
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const int64_t lay = (int64_t)(nx + 1) * (ny + 1);
  const int64_t N = lay * (nz + 1);
  int64_t c[4];
  double xs[4], ys[4], zs[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    c[p] = (int64_t)(j + (p >> 1)) * (nx + 1) + i + (p & 1);
    xs[p] = X[c[p]]; ys[p] = Y[c[p]]; zs[p] = Z[c[p]];
  }
  // the column's center geometry from the ground layer's edge vectors
  const CellEdges<dflt> ce = cell_edges<dflt>(xs, ys, zs);
  const dflt J00 = (ce.x[0] + ce.x[1]) * 0.25f, J01 = (ce.x[2] + ce.x[3]) * 0.25f;
  const dflt J10 = (ce.y[0] + ce.y[1]) * 0.25f, J11 = (ce.y[2] + ce.y[3]) * 0.25f;
  const dflt z1 = (ce.z[0] + ce.z[1]) * 0.25f, z2 = (ce.z[2] + ce.z[3]) * 0.25f;
  const dflt ij = reciprocal(J00 * J11 - J01 * J10);
  // J2^-T = [[J11, -J10], [-J01, J00]] / j2
  const dflt m00 = J11 * ij, m01 = -(J10 * ij), m10 = -(J01 * ij), m11 = J00 * ij;
  const dflt dd[3] = {{a0.x, a0.y}, {a1.x, a1.y}, {a2.x, a2.y}};
  const bool nodal = u0c == nullptr;
  LayerSums lo = layer_sums(lam, u0, N, c, nodal);
  const int64_t NE = (int64_t)nx * ny * nz;
  for (int k = 0; k < nz; ++k) {
    int64_t cu[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) cu[p] = c[p] + (int64_t)(k + 1) * lay;
    const LayerSums up = layer_sums(lam, u0, N, cu, nodal);
    const dflt g1 = (lo.d1 + up.d1) * 0.125f, g2 = (lo.d2 + up.d2) * 0.125f;
    const dflt g3 = (up.s - lo.s) * 0.125f;
    const dflt gz = g3 * dflt{rh[k].x, rh[k].y};
    const dflt h1 = g1 - z1 * gz, h2 = g2 - z2 * gz;
    const dflt gr[3] = {m00 * h1 + m01 * h2, m10 * h1 + m11 * h2, gz};
    const int64_t e = ((int64_t)k * ny + j) * nx + i;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const dflt uc = nodal ? (lo.su[d] + up.su[d]) * 0.125f : pair_of(u0c[d * NE + e]);
      const dflt ud = uc + gr[d] * dd[d];
      u[d * NE + e] = pair_to_double(ud.hi, ud.lo);
    }
    lo = up;
  }
}

}  // namespace

cudaError_t launch_recover_center_sep(int nx, int ny, int nz, const double* X, const double* Y,
                                      const double* Z, const double* u0, const double* u0c,
                                      const double* lam, const double* a, double* u,
                                      cudaStream_t st) {
  if (nz > kMaxZ) return cudaErrorInvalidValue;
  dim3 blk(32, 4, 1);
  dim3 grd((nx + 31) / 32, (ny + 3) / 4, 1);
  k_recover_center_sep<<<grd, blk, 0, st>>>(nx, ny, nz, X, Y, Z, u0, u0c, lam,
                                            split_bits(1.0 / (a[0] * a[0])),
                                            split_bits(1.0 / (a[1] * a[1])),
                                            split_bits(1.0 / (a[2] * a[2])), u);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mcw
