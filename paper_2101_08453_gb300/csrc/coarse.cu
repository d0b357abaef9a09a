// Direct solve on the coarsest grid (Sec. 3: "solved by a direct method").
// The free block of the coarsest operator (n <= 4096 unknowns, numbered
// k-major over the free nodes) is gathered into a dense matrix and inverted
// once, at assembly, by Gauss-Jordan elimination without pivoting (the
// matrix is symmetric positive definite), one launch per pivot.  Each cycle
// then applies the inverse as a dense matrix-vector product in float64.
#include "kernels.cuh"

namespace mcw {
namespace {

__global__ void k_coarse_index(Grid g, int* cfree) {
  const int n1 = g.Nx - 2, n2 = g.Ny - 2, n3 = g.Nz - 1;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n1 * n2 * n3) return;
  int i = q % n1 + 1, j = (q / n1) % n2 + 1, k = q / (n1 * n2);
  cfree[q] = (int)gidx(g, i, j, k);
}

__global__ void k_dense_gather(Grid g, const double* __restrict__ C, int n,
                               double* __restrict__ A) {
  const int n1 = g.Nx - 2, n2 = g.Ny - 2;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * 27) return;
  const int row = q / 27, s = q % 27;
  const int i = row % n1 + 1, j = (row / n1) % n2 + 1, k = row / (n1 * n2);
  const int ii = i + s % 3 - 1, jj = j + (s / 3) % 3 - 1, kk = k + s / 9 - 1;
  if (!is_free(g, ii, jj, kk)) return;
  const int col = (kk * n2 + (jj - 1)) * n1 + (ii - 1);
  A[(int64_t)row * n + col] = C[cidx(gidx(g, i, j, k), s)];
}

__global__ void k_gj_step(const double* __restrict__ A, double* __restrict__ B, int n, int p) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  const int r = (int)(q / n), c = (int)(q % n);
  // one division per thread (a float64 division is a long instruction
  // sequence on the double pipe); the others multiply by the reciprocal
  const double ip = 1.0 / A[(int64_t)p * n + p];
  double v;
  if (r == p && c == p) v = ip;
  else if (r == p) v = A[(int64_t)p * n + c] * ip;
  else if (c == p) v = -A[(int64_t)r * n + p] * ip;
  else v = A[q] - A[(int64_t)r * n + p] * (A[(int64_t)p * n + c] * ip);
  B[q] = v;
}

constexpr int kRowsPerBlock = 8;

template <typename T>
__global__ void __launch_bounds__(32 * kRowsPerBlock) k_dense_solve(const double* __restrict__ Ainv,
                                                                    int n, const int* __restrict__ cfree,
                                                                    const T* __restrict__ f,
                                                                    T* __restrict__ x) {
  extern __shared__ double fs[];
  for (int q = threadIdx.x; q < n; q += blockDim.x) fs[q] = (double)f[cfree[q]];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * kRowsPerBlock + (threadIdx.x >> 5);
  if (row >= n) return;
  const double* a = Ainv + (int64_t)row * n;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) s += a[c] * fs[c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) x[cfree[row]] = (T)s;
}

}  // namespace

cudaError_t launch_coarse_index(const Grid& g, int* cfree, cudaStream_t st) {
  int n = (g.Nx - 2) * (g.Ny - 2) * (g.Nz - 1);
  k_coarse_index<<<(n + 255) / 256, 256, 0, st>>>(g, cfree); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dense_gather(const Grid& g, const double* C, const int* cfree, int n,
                                double* A, cudaStream_t st) {
  (void)cfree;
  cudaError_t e = cudaMemsetAsync(A, 0, sizeof(double) * (size_t)n * n, st);
  if (e != cudaSuccess) return e;
  k_dense_gather<<<(n * 27 + 255) / 256, 256, 0, st>>>(g, C, n, A); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dense_invert(double* A, double* B, int n, double** result, cudaStream_t st) {
  int64_t nn = (int64_t)n * n;
  int blocks = (int)((nn + 255) / 256);
  double *src = A, *dst = B;
  for (int p = 0; p < n; ++p) {
    k_gj_step<<<blocks, 256, 0, st>>>(src, dst, n, p); count_launches(1);
    double* t = src; src = dst; dst = t;
  }
  *result = src;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dense_solve(const double* Ainv, int n, const int* cfree, const T* f, T* x,
                               cudaStream_t st) {
  int blocks = (n + kRowsPerBlock - 1) / kRowsPerBlock;
  k_dense_solve<T><<<blocks, 32 * kRowsPerBlock, sizeof(double) * n, st>>>(Ainv, n, cfree, f, x); count_launches(1);
  return cudaGetLastError();
}
template cudaError_t launch_dense_solve<double>(const double*, int, const int*, const double*,
                                                double*, cudaStream_t);
template cudaError_t launch_dense_solve<float>(const double*, int, const int*, const float*,
                                               float*, cudaStream_t);

}  // namespace mcw
