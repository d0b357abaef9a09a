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
// the 4 corners of a node layer, each formed once (with the neighbouring
// lane's half) and used by the element below and the one above:
//   g_1 = (D1(k) + D1(k+1)) / 8, D1 = (l1 - l0) + (l3 - l2)  (corner p = a + 2b),
//   g_2 = (D2(k) + D2(k+1)) / 8, D2 = (l2 - l0) + (l3 - l1),
//   g_3 = (S(k+1) - S(k)) / 8,    S = l0 + l1 + l2 + l3,
//   u0(center) = (S_u(k) + S_u(k+1)) / 8.
// Everything after reading runs in float pairs (about 48 significant bits);
// lambda and u0 are split and u is formed in integer arithmetic, so the only
// double arithmetic is the layer thicknesses' reciprocals.
#include "cellgeom.cuh"
#include "dfloat.cuh"
#include "kernels.cuh"

namespace mcw {
namespace {

__device__ __forceinline__ dflt pair_of(double v) {
  const float2 p = split_bits(v);
  return {p.x, p.y};
}

// The per-layer sums of one element column, formed by the warp: a lane
// owns the node column pair (i_n, j) and (i_n, j+1) of one node layer and
// forms a = l(j) + l(j+1), b = l(j+1) - l(j) and c_d = u0_d(j) + u0_d(j+1);
// the element of lane L (corners i_n = i .. i+1) takes lane L+1's as its
// corners p = 1, 3:  S = a + a', D1 = a' - a, D2 = b + b', S_u = c + c'.
// So each node of a layer is read and split once per element row.
struct LayerSums {
  dflt d1, d2, s, su[3];
};

__device__ __forceinline__ dflt shfl_next(dflt v) {
  return {__shfl_down_sync(0xffffffffu, v.hi, 1), __shfl_down_sync(0xffffffffu, v.lo, 1)};
}

__device__ __forceinline__ LayerSums layer_sums(const double* __restrict__ lam,
                                                const double* __restrict__ u0, int64_t N,
                                                int64_t c0, int64_t c2, bool node, bool with_u0) {
  const dflt z = {0.0f, 0.0f};
  const dflt l0 = node ? pair_of(lam[c0]) : z;
  const dflt l2 = node ? pair_of(lam[c2]) : z;
  const dflt a = l0 + l2, b = l2 - l0;
  const dflt an = shfl_next(a), bn = shfl_next(b);
  LayerSums L;
  L.d1 = an - a;
  L.d2 = b + bn;
  L.s = a + an;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dflt cu = z;
    if (with_u0 && node) cu = pair_of(u0[d * N + c0]) + pair_of(u0[d * N + c2]);
    L.su[d] = cu + shfl_next(cu);
  }
  return L;
}

// Lanes 0..30 of a warp own the element columns i0 .. i0+30 (i0 = 31 per
// warp), lane 31 only supplies node column i0 + 31; threadIdx.y is the
// element row j.
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
  const int lane = threadIdx.x;
  const int i = blockIdx.x * 31 + lane;  // element column, and this lane's node column
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (j >= ny) return;  // whole warps: a warp is one row j
  const bool node = i <= nx;                 // the lane's node column exists
  const bool elem = lane < 31 && i < nx;     // the lane owns an element column
  const int64_t lay = (int64_t)(nx + 1) * (ny + 1);
  const int64_t N = lay * (nz + 1);
  const int64_t c0 = (int64_t)j * (nx + 1) + (node ? i : 0), c2 = c0 + (nx + 1);
  // the column's center geometry from the ground layer's edge vectors
  dflt m00 = {0.0f, 0.0f}, m01 = m00, m10 = m00, m11 = m00, z1 = m00, z2 = m00;
  if (elem) {
    double xs[4], ys[4], zs[4];
    const int64_t cc[4] = {c0, c0 + 1, c2, c2 + 1};
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      xs[p] = X[cc[p]]; ys[p] = Y[cc[p]]; zs[p] = Z[cc[p]];
    }
    const CellEdges<dflt> ce = cell_edges<dflt>(xs, ys, zs);
    const dflt J00 = (ce.x[0] + ce.x[1]) * 0.25f, J01 = (ce.x[2] + ce.x[3]) * 0.25f;
    const dflt J10 = (ce.y[0] + ce.y[1]) * 0.25f, J11 = (ce.y[2] + ce.y[3]) * 0.25f;
    z1 = (ce.z[0] + ce.z[1]) * 0.25f;
    z2 = (ce.z[2] + ce.z[3]) * 0.25f;
    const dflt ij = reciprocal(J00 * J11 - J01 * J10);
    // J2^-T = [[J11, -J10], [-J01, J00]] / j2
    m00 = J11 * ij; m01 = -(J10 * ij); m10 = -(J01 * ij); m11 = J00 * ij;
  }
  const dflt dd[3] = {{a0.x, a0.y}, {a1.x, a1.y}, {a2.x, a2.y}};
  const bool nodal = u0c == nullptr;
  LayerSums lo = layer_sums(lam, u0, N, c0, c2, node, nodal);
  const int64_t NE = (int64_t)nx * ny * nz;
  for (int k = 0; k < nz; ++k) {
    const int64_t up0 = c0 + (int64_t)(k + 1) * lay, up2 = c2 + (int64_t)(k + 1) * lay;
    const LayerSums up = layer_sums(lam, u0, N, up0, up2, node, nodal);
    if (elem) {
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
  dim3 grd((nx + 30) / 31, (ny + 3) / 4, 1);
  k_recover_center_sep<<<grd, blk, 0, st>>>(nx, ny, nz, X, Y, Z, u0, u0c, lam,
                                            split_bits(1.0 / (a[0] * a[0])),
                                            split_bits(1.0 / (a[1] * a[1])),
                                            split_bits(1.0 / (a[2] * a[2])), u);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mcw
