// Load vector of Eq. 5 (right side, 2x2x2 Gauss, u0 interpolated from the
// nodes) on a terrain-following grid in shift form, from column x layer
// factors (MCWIND_OP_SEPARABLE with float-pair element arithmetic).
//
// With the horizontal Jacobian J2, its adjugate adj, j2 = det J2 and the
// terrain slope z' of a column (see separable.cu), det J grad N_m =
//   ((h/2) adj^T grad_h phi_a psi_a - adj^T z' phi_a psi_a', j2 phi_a psi_a')
// and u0 = sum_n phi_b psi_b u0_n, so the Gauss sums split into horizontal
// 4 x 4 factors E_d = sum (adj^T grad_h phi_a)_d phi_b, F_d = sum (adj^T z')_d
// phi_a phi_b, M_z = sum j2 phi_a phi_b and the 1-D integrals of a linear
// element, (h/2) m and int psi_a' psi_b (the transpose of g):
//   f = -[(E_x (x) V_M) u_x + (E_y (x) V_M) u_y - (F_x (x) V_G^T) u_x
//         - (F_y (x) V_G^T) u_y + (M_z (x) V_G^T) u_z].
// The factors are formed and kept as float pairs, and the load vector is
// summed in float pairs (about 48 significant bits), as the element kernels
// of this arithmetic do.
#include <cudaTypedefs.h>

#include "async.cuh"
#include "cellgeom.cuh"
#include "dfloat.cuh"
#include "kernels.cuh"

namespace mcw {
namespace {

constexpr int kRR = 4;                        // owned rows per block
constexpr int kRTileRows = kRR + 2;
constexpr int kRTileW = 40;
constexpr int kRStage = 3 * kRTileRows * 2 * kRTileW;   // float2 values (11520 bytes)
constexpr uint32_t kRBytes = kRStage * 8;
constexpr int kRStages = 4;

__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
  const dflt s = dflt{a.x, a.y} + dflt{b.x, b.y};
  return make_float2(s.hi, s.lo);
}

// acc += a * u in float pairs: the product's rounding error is kept by the
// FMA (e), the sum's by a two-sum (t); the low part is renormalized at the end
__device__ __forceinline__ void pmac(float& sh, float& sl, float2 a, float2 u) {
  const float p = a.x * u.x;
  float e = fmaf(a.x, u.x, -p);
  e = fmaf(a.x, u.y, e);
  e = fmaf(a.y, u.x, e);
  const float s = sh + p;
  const float bb = s - sh;
  const float t = (sh - (s - bb)) + (p - bb);
  sh = s;
  sl += t + e;
}

__device__ __forceinline__ float2 pnorm(float sh, float sl) {
  const float s = sh + sl;
  return make_float2(s, sl - (s - sh));
}

// Factors of the cells of one parity class added, as float pairs, into the
// tiles of their 4 corner columns (classes in order: fixed summation order).
// The Gauss sums run in float pairs from the cell's edge vectors; F_x, F_y
// and M_z are symmetric in (p, q), so their upper triangles are formed.
__global__ void __launch_bounds__(128) k_rhs_cells(Grid g, int cls, const double* __restrict__ X,
                                                   const double* __restrict__ Y,
                                                   const double* __restrict__ Z,
                                                   float2* __restrict__ R) {
  using A = Arith<dflt>;
  const int ci = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + (cls & 1);
  const int cj = 2 * (blockIdx.y * blockDim.y + threadIdx.y) + (cls >> 1);
  if (ci >= g.Nx - 1 || cj >= g.Ny - 1) return;
  double xs[4], ys[4], zs[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int64_t n = (int64_t)(cj + (p >> 1)) * g.Nx + ci + (p & 1);
    xs[p] = X[n]; ys[p] = Y[n]; zs[p] = Z[n];
  }
  const CellEdges<dflt> ce = cell_edges<dflt>(xs, ys, zs);
  dflt Ex[4][4], Ey[4][4], Fx[10], Fy[10], Mz[10];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) Ex[p][q] = Ey[p][q] = A::zero();
#pragma unroll
  for (int u = 0; u < 10; ++u) Fx[u] = Fy[u] = Mz[u] = A::zero();
#pragma unroll
  for (int gq = 0; gq < 4; ++gq) {
    const GaussGeom<dflt> G = gauss_geom(ce, gq);
    const dflt j2 = G.J00 * G.J11 - G.J01 * G.J10;
    const dflt zx = G.J11 * G.z1 - G.J10 * G.z2, zy = G.J00 * G.z2 - G.J01 * G.z1;  // adj^T z'
    int t = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const dflt d1 = A::from(gauss_d1(gq, p)), d2 = A::from(gauss_d2(gq, p));
      const dflt gx = G.J11 * d1 - G.J10 * d2, gy = G.J00 * d2 - G.J01 * d1;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const dflt phq = A::from(gauss_phi(gq, q));
        Ex[p][q] = Ex[p][q] + gx * phq;
        Ey[p][q] = Ey[p][q] + gy * phq;
        if (q >= p) {
          const dflt pp = A::from(gauss_phi(gq, p) * gauss_phi(gq, q));
          Fx[t] = Fx[t] + zx * pp;
          Fy[t] = Fy[t] + zy * pp;
          Mz[t] = Mz[t] + j2 * pp;
          ++t;
        }
      }
    }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int64_t col = gidx(g, ci + (p & 1), cj + (p >> 1), 0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int s2 = ((q & 1) - (p & 1) + 1) + 3 * ((q >> 1) - (p >> 1) + 1);
      const int lo = p < q ? p : q, hi = p < q ? q : p;
      const int t = lo * 4 - lo * (lo - 1) / 2 + (hi - lo);  // upper-triangle index
      const dflt v[5] = {Ex[p][q], Ey[p][q], Fx[t], Fy[t], Mz[t]};
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        float2& r = R[ridx(col, 9 * c + s2)];
        r = pair_add(r, make_float2(v[c].hi, v[c].lo));
      }
    }
  }
}

// u0 [3][Nz][Ny][Nx] (float64) -> float pairs in the split layout, 3 components
// of g.total each; padding entries 0.  One thread per split-layout node.
__global__ void __launch_bounds__(128) k_u0_split_pairs(Grid g, const double* __restrict__ u0,
                                                        float2* __restrict__ u2) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z >> 1, par = blockIdx.z & 1;
  if (h >= g.H || j >= g.Ny) return;
  const int i = 2 * h + par;
  const int64_t o = (int64_t)k * g.PP + (int64_t)j * g.RP + (int64_t)par * g.H + h;
  const int64_t n = (int64_t)g.Nx * g.Ny * g.Nz;
  const int64_t s = ((int64_t)k * g.Ny + j) * g.Nx + i;
#pragma unroll
  for (int c = 0; c < 3; ++c)
    u2[c * g.total + o] = i < g.Nx ? split_bits(u0[c * n + s]) : make_float2(0.0f, 0.0f);
}

// f = load vector at every node of the split layout (0 at fixed nodes and
// padding), float64.  One thread per column of one parity half (blockIdx.z),
// owned rows j0 .. j0+kRR-1; a producer warp stages the three components of
// u0 around them, all Nz layers (u0 of the fixed top layer enters the rows
// below it), by TMA into a ring of stages; per layer a thread forms
// a = sum (E_x u_x + E_y u_y) and b = sum (F_x u_x + F_y u_y - M_z u_z) over
// its 9 columns, and row k takes a and b of layers k-1, k, k+1.
__global__ void __launch_bounds__(32 * (kRR + 1)) k_rhs_sep(Grid g,
                                                           const __grid_constant__ CUtensorMap tmu,
                                                           const float2* __restrict__ R,
                                                           const float2* __restrict__ VR,
                                                           double* __restrict__ f, int* status) {
  __shared__ __align__(128) float2 tile[kRStages][kRStage];
  __shared__ __align__(8) uint64_t full[kRStages], empty[kRStages];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int par = (int)blockIdx.z;
  const int h0 = blockIdx.x * 32;
  const int j0 = kRR * blockIdx.y;
  const int nlay = g.Nz;
  const int64_t PP = g.PP;
  if (ty == 0 && tx == 0) {
    for (int q = 0; q < kRStages; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kRR);
    }
    fence_barrier_init();
  }
  __syncthreads();
  if (ty == kRR) {
    int issued = 0;
    for (int t = 0; t < nlay; ++t) {
      const int sidx = t % kRStages;
      if (t >= kRStages) {
        const bool ok = wait_parity(&empty[sidx], (uint32_t)(t / kRStages - 1) & 1u, status,
                                    kWaitLimitNs);
        if (__any_sync(0xffffffffu, !ok)) break;
      }
      if (tx == 0) {
        fence_proxy_async_shared();
        mbar_arrive_expect_tx(&full[sidx], kRBytes);
        asm volatile(
            "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(tile[sidx])),
            "l"((unsigned long long)&tmu), "r"(h0 - 4), "r"(0), "r"(j0 - 1), "r"(t), "r"(0),
            "r"(smem_u32(&full[sidx]))
            : "memory");
      }
      __syncwarp();
      issued = t + 1;
    }
    if (tx == 0)
      for (int u = max(0, issued - kRStages); u < issued; ++u)
        wait_parity(&full[u % kRStages], (uint32_t)(u / kRStages) & 1u, status, kWaitLimitNs);
    return;
  }
  const int h = h0 + tx, j = j0 + ty, i = 2 * h + par;
  const bool inrow = j < g.Ny;
  const bool active = inrow && i >= 1 && i <= g.Nx - 2 && j >= 1 && j <= g.Ny - 2;
  const int64_t own = (int64_t)j * g.RP + (int64_t)par * g.H + h;
  float2 fac[kRF];
#pragma unroll
  for (int q = 0; q < kRF; ++q) fac[q] = active ? R[ridx(own, q)] : make_float2(0.0f, 0.0f);
  int toff[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const int ii = i + c % 3 - 1, r = ty + 1 + c / 3 - 1;
    toff[c] = (r * 2 + (ii & 1)) * kRTileW + ((ii >> 1) - (h0 - 4));
  }
  constexpr int kComp = kRTileRows * 2 * kRTileW;
  float2 ab = make_float2(0.0f, 0.0f), bb = ab, ac = ab, bc = ab;  // layers k-1, k
  for (int t = 0; t <= nlay; ++t) {
    float2 at = make_float2(0.0f, 0.0f), bt = at;
    if (t < nlay) {
      const bool ok = wait_parity(&full[t % kRStages], (uint32_t)(t / kRStages) & 1u, status,
                                  kWaitLimitNs);
      if (__any_sync(0xffffffffu, !ok)) return;
      if (active) {
        const float2* st = tile[t % kRStages];
        float ah = 0.0f, al = 0.0f, bh = 0.0f, bl = 0.0f;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          const float2 ux = st[toff[c]], uy = st[kComp + toff[c]], uz = st[2 * kComp + toff[c]];
          pmac(ah, al, fac[c], ux);
          pmac(ah, al, fac[9 + c], uy);
          pmac(bh, bl, fac[18 + c], ux);
          pmac(bh, bl, fac[27 + c], uy);
          pmac(bh, bl, make_float2(-fac[36 + c].x, -fac[36 + c].y), uz);
        }
        at = pnorm(ah, al);
        bt = pnorm(bh, bl);
      }
      __syncwarp();
      if (tx == 0) mbar_arrive(&empty[t % kRStages]);
    }
    if (t >= 1 && inrow) {
      const int k = t - 1;
      double fk = 0.0;
      if (active && k <= g.Nz - 2) {
        const float2* v = VR + k * kRV;
        float sh = 0.0f, sl = 0.0f;
        pmac(sh, sl, v[0], ab);
        pmac(sh, sl, v[1], ac);
        pmac(sh, sl, v[2], at);
        pmac(sh, sl, make_float2(-v[3].x, -v[3].y), bb);
        pmac(sh, sl, make_float2(-v[4].x, -v[4].y), bc);
        pmac(sh, sl, make_float2(-v[5].x, -v[5].y), bt);
        const float2 s = pnorm(sh, sl);
        fk = -pair_to_double(s.x, s.y);
      }
      f[(int64_t)k * PP + own] = fk;
    }
    ab = ac; bb = bc;
    ac = at; bc = bt;
  }
}

}  // namespace

cudaError_t launch_rhs_factors(const Grid& g, const double* X, const double* Y, const double* Z,
                               float2* R, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(R, 0, sizeof(float2) * kRF * (size_t)g.PP, st);
  const dim3 grd((g.Nx / 2 + 31) / 32, (g.Ny / 2 + 3) / 4);
  for (int cls = 0; cls < 4 && e == cudaSuccess; ++cls) {
    k_rhs_cells<<<grd, dim3(32, 4), 0, st>>>(g, cls, X, Y, Z, R);
    count_launches(1);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t make_u0_map(Level& L, float2* u2) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&encode,
                                                     12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !encode) return cudaErrorNotSupported;
  }
  const Grid& g = L.g;
  // [3][Nz][Ny][2][H] float pairs (8 bytes): half-row index innermost
  const cuuint64_t dims[5] = {(cuuint64_t)g.H, 2, (cuuint64_t)g.Ny, (cuuint64_t)g.Nz, 3};
  const cuuint64_t strides[4] = {(cuuint64_t)g.H * 8, (cuuint64_t)g.RP * 8, (cuuint64_t)g.PP * 8,
                                 (cuuint64_t)g.total * 8};
  const cuuint32_t box[5] = {(cuuint32_t)kRTileW, 2, (cuuint32_t)kRTileRows, 1, 3};
  const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
  const CUresult r = encode(&L.tm_u, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, u2, dims, strides, box, ones,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_rhs_sep(const Level& L, const float2* R2, const float2* VR2, const double* u0,
                           float2* u2, double* f, int* status, cudaStream_t st) {
  const Grid& g = L.g;
  k_u0_split_pairs<<<dim3((g.H + 31) / 32, (g.Ny + 3) / 4, 2 * g.Nz), dim3(32, 4), 0, st>>>(g, u0,
                                                                                        u2);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const dim3 grd((g.H + 31) / 32, (g.Ny + kRR - 1) / kRR, 2), blk(32, kRR + 1);
  k_rhs_sep<<<grd, blk, 0, st>>>(g, L.tm_u, R2, VR2, f, status);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mcw
