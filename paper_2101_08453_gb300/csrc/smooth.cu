// Gauss-Seidel smoother of Sec. 3: vertical sweeps through the columns of
// nodes, the columns in 4 horizontal groups (i mod 2) + 2 (j mod 2).  One
// launch updates one group; one thread owns one column and walks it from
// the ground up (or the top down) with the 27 values of x it needs held in a
// sliding 3-layer x 9-column register window: per node it loads the 9 new
// neighbours of the next layer, the 26 off-diagonal coefficients, 1/K_nn
// and f, and stores one value.  Same-group columns are two apart in i or j
// and so never neighbours: the threads of a launch are independent.  The
// sum over the stencil takes the layer behind the sweep first, so that the
// loads of the layer ahead have the rest of the sum to arrive.
#include "kernels.cuh"

namespace mcw {
namespace {

template <typename T, bool UP>
__global__ void __launch_bounds__(256) k_gs(Grid g, const T* __restrict__ C,
                                            const T* __restrict__ f, T* __restrict__ x, int pi,
                                            int pj) {
  const int ih = blockIdx.x * blockDim.x + threadIdx.x;
  const int jh = blockIdx.y * blockDim.y + threadIdx.y;
  const int i = 2 * ih + pi, j = 2 * jh + pj;
  if (i < 1 || i > g.Nx - 2 || j < 1 || j > g.Ny - 2) return;
  int64_t col[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const int ii = i + c % 3 - 1, jj = j + c / 3 - 1;
    col[c] = (int64_t)jj * g.RP + (int64_t)(ii & 1) * g.H + (ii >> 1);
  }
  const int64_t PP = g.PP, tot = g.total;
  const int Nz = g.Nz;
  T w[3][9];
  if (UP) {
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      w[0][c] = T(0);
      w[1][c] = x[col[c]];
      w[2][c] = x[PP + col[c]];
    }
    for (int k = 0; k <= Nz - 2; ++k) {
      const int64_t b = (int64_t)k * PP + col[4];
      T acc = f[b];
      // the layer above (w[2], loaded last) enters the sum last
#pragma unroll
      for (int s = 0; s < 27; ++s)
        if (s != kDiag) acc -= coef(C, tot, b, s) * w[s / 9][s % 9];
      const T xn = acc * coef(C, tot, b, kInvDiag);
      x[b] = xn;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        w[0][c] = w[1][c];
        w[1][c] = w[2][c];
      }
      w[0][4] = xn;
      if (k + 2 <= Nz - 1) {
#pragma unroll
        for (int c = 0; c < 9; ++c) w[2][c] = x[(int64_t)(k + 2) * PP + col[c]];
      } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) w[2][c] = T(0);
      }
    }
  } else {
    const int k0 = Nz - 2;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      w[2][c] = x[(int64_t)(k0 + 1) * PP + col[c]];
      w[1][c] = x[(int64_t)k0 * PP + col[c]];
      w[0][c] = k0 >= 1 ? x[(int64_t)(k0 - 1) * PP + col[c]] : T(0);
    }
    for (int k = k0; k >= 0; --k) {
      const int64_t b = (int64_t)k * PP + col[4];
      T acc = f[b];
      // the layer below (w[0], loaded last) enters the sum last
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        const int s = 26 - t;
        if (s != kDiag) acc -= coef(C, tot, b, s) * w[s / 9][s % 9];
      }
      const T xn = acc * coef(C, tot, b, kInvDiag);
      x[b] = xn;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        w[2][c] = w[1][c];
        w[1][c] = w[0][c];
      }
      w[2][4] = xn;
      if (k - 2 >= 0) {
#pragma unroll
        for (int c = 0; c < 9; ++c) w[0][c] = x[(int64_t)(k - 2) * PP + col[c]];
      } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) w[0][c] = T(0);
      }
    }
  }
}

// The first group of a forward sweep from x = 0: in each group-(pi, pj)
// column every neighbour is still zero except the node just below, so the
// update reduces to x_k = (f_k - K(k, k-1) x_{k-1}) / K_kk, the same value
// the full stencil gives.  Every other entry of x (other groups, boundary
// nodes, padding) is written 0, which replaces zeroing x beforehand.
template <typename T>
__global__ void __launch_bounds__(128) k_gs_zero_start(Grid g, const T* __restrict__ C,
                                                       const T* __restrict__ f,
                                                       T* __restrict__ x, int pi, int pj) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int par = (int)blockIdx.z;
  if (h >= g.H || j >= g.Ny) return;
  const int i = 2 * h + par;
  const int64_t own = (int64_t)j * g.RP + (int64_t)par * g.H + h;
  const int64_t PP = g.PP, tot = g.total;
  const bool mine = par == pi && (j & 1) == pj && i >= 1 && i <= g.Nx - 2 && j >= 1 &&
                    j <= g.Ny - 2;
  if (!mine) {
    for (int k = 0; k < g.Nz; ++k) x[(int64_t)k * PP + own] = T(0);
    return;
  }
  constexpr int kBelow = 4;  // stencil offset (0, 0, -1)
  T prev = T(0);
#pragma unroll 4
  for (int k = 0; k <= g.Nz - 2; ++k) {
    const int64_t b = (int64_t)k * PP + own;
    T acc = f[b];
    acc -= coef(C, tot, b, kBelow) * prev;
    prev = acc * coef(C, tot, b, kInvDiag);
    x[b] = prev;
  }
  x[(int64_t)(g.Nz - 1) * PP + own] = T(0);
}

}  // namespace

template <typename T>
cudaError_t launch_gs_zero_start(const Grid& g, const T* C, const T* f, T* x, int group,
                                 cudaStream_t st) {
  dim3 grd((g.H + 31) / 32, (g.Ny + 3) / 4, 2);
  k_gs_zero_start<T><<<grd, dim3(32, 4), 0, st>>>(g, C, f, x, group & 1, group >> 1);
  count_launches(1);
  return cudaGetLastError();
}
template cudaError_t launch_gs_zero_start<double>(const Grid&, const double*, const double*,
                                                  double*, int, cudaStream_t);
template cudaError_t launch_gs_zero_start<float>(const Grid&, const float*, const float*, float*,
                                                 int, cudaStream_t);

template <typename T>
cudaError_t launch_gs_group(const Grid& g, const T* C, const T* f, T* x, int group, int up,
                            int rows, cudaStream_t st) {
  const int pi = group & 1, pj = group >> 1;
  dim3 blk(32, rows);
  dim3 grd(((g.Nx + 1) / 2 + 31) / 32, ((g.Ny + 1) / 2 + rows - 1) / rows);
  if (up)
    k_gs<T, true><<<grd, blk, 0, st>>>(g, C, f, x, pi, pj);
  else
    k_gs<T, false><<<grd, blk, 0, st>>>(g, C, f, x, pi, pj);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_gs_group<double>(const Grid&, const double*, const double*, double*,
                                             int, int, int, cudaStream_t);
template cudaError_t launch_gs_group<float>(const Grid&, const float*, const float*, float*, int,
                                            int, int, cudaStream_t);

}  // namespace mcw
