// Gauss-Seidel smoother of Sec. 3: vertical sweeps through the columns of
// nodes, the columns in 4 horizontal groups (i mod 2) + 2 (j mod 2).  One
// launch updates one group; one thread owns one column and walks it from
// the ground up (or the top down) with the 27 values of x it needs held in a
// sliding 3-layer x 9-column register window: per node it loads the 9 new
// neighbours of the next layer, the 26 off-diagonal coefficients, 1/K_nn
// and f, and stores one value.  Same-group columns are two apart in i or j
// and so never neighbours: the threads of a launch are independent.
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
#pragma unroll
      for (int s = 0; s < 27; ++s)
        if (s != kDiag) acc -= coef(C, tot, b, s) * w[s / 9][s % 9];
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

}  // namespace

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
