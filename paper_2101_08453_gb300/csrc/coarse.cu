// Direct solve on the coarsest grid (Sec. 3: the coarsest problem is solved directly).
// The free block of the coarsest operator (n <= 4096 unknowns, numbered
// k-major over the free nodes) is gathered into a dense matrix and inverted
// once, at assembly, by Gauss-Jordan elimination without pivoting (the
// matrix is symmetric positive definite) in blocks of kGjB pivots, three
// launches per block.  Each cycle then applies the inverse as a dense
// matrix-vector product in float64.
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

// Blocked Gauss-Jordan in the exchange form: with the pivot block P of b
// indices and the others O, one block step maps
//   A_PP -> A_PP^-1,  A_PO -> A_PP^-1 A_PO,  A_OP -> -A_OP A_PP^-1,
//   A_OO -> A_OO - A_OP A_PP^-1 A_PO,
// which equals b single-pivot steps; after all blocks A holds A^-1.  The
// Schur complements of an SPD matrix stay SPD, so no pivoting is needed.
constexpr int kGjB = 16;

// the pivot block's inverse (b x b) by scalar Gauss-Jordan in shared memory
__global__ void __launch_bounds__(256) k_gj_pivot(const double* __restrict__ A, int n, int p0,
                                                  int b, double* __restrict__ Pinv) {
  __shared__ double M[kGjB][kGjB];
  const int t = threadIdx.x, r = t / kGjB, c = t % kGjB;
  if (r < b && c < b) M[r][c] = A[(int64_t)(p0 + r) * n + p0 + c];
  __syncthreads();
  for (int p = 0; p < b; ++p) {
    double v = 0.0;
    if (r < b && c < b) {
      const double ip = 1.0 / M[p][p];
      if (r == p && c == p) v = ip;
      else if (r == p) v = M[p][c] * ip;
      else if (c == p) v = -M[r][p] * ip;
      else v = M[r][c] - M[r][p] * (M[p][c] * ip);
    }
    __syncthreads();
    if (r < b && c < b) M[r][c] = v;
    __syncthreads();
  }
  if (r < b && c < b) Pinv[r * kGjB + c] = M[r][c];
}

// U = A_PP^-1 A_P. (b rows, all columns) and Lo = A_.P (all rows, the b
// pivot columns, before the step): one thread per (row, pivot) pair of each
__global__ void k_gj_panel(const double* __restrict__ A, int n, int p0, int b,
                           const double* __restrict__ Pinv, double* __restrict__ U,
                           double* __restrict__ Lo) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= (int64_t)b * n) return;
  const int t = (int)(q / n), c = (int)(q % n);
  double s = 0.0;
  for (int u = 0; u < b; ++u) s += Pinv[t * kGjB + u] * A[(int64_t)(p0 + u) * n + c];
  U[(int64_t)t * n + c] = s;
  Lo[(int64_t)c * kGjB + t] = A[(int64_t)c * n + p0 + t];
}

// the block step on every entry, from the saved panels
__global__ void k_gj_update(double* __restrict__ A, int n, int p0, int b,
                            const double* __restrict__ Pinv, const double* __restrict__ U,
                            const double* __restrict__ Lo) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= (int64_t)n * n) return;
  const int r = (int)(q / n), c = (int)(q % n);
  const bool rp = r >= p0 && r < p0 + b, cp = c >= p0 && c < p0 + b;
  double v;
  if (rp && cp) {
    v = Pinv[(r - p0) * kGjB + (c - p0)];
  } else if (rp) {
    v = U[(int64_t)(r - p0) * n + c];
  } else if (cp) {
    v = 0.0;  // -A_OP A_PP^-1
    for (int u = 0; u < b; ++u) v -= Lo[(int64_t)r * kGjB + u] * Pinv[u * kGjB + (c - p0)];
  } else {
    v = A[q];
    for (int u = 0; u < b; ++u) v -= Lo[(int64_t)r * kGjB + u] * U[(int64_t)u * n + c];
  }
  A[q] = v;
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
  // B holds the step's small buffers: pivot inverse, then U (b x n), then Lo (n x b)
  double* Pinv = B;
  double* U = B + kGjB * kGjB;
  double* Lo = U + (int64_t)kGjB * n;
  const int64_t nn = (int64_t)n * n;
  for (int p0 = 0; p0 < n; p0 += kGjB) {
    const int b = n - p0 < kGjB ? n - p0 : kGjB;
    k_gj_pivot<<<1, 256, 0, st>>>(A, n, p0, b, Pinv);
    k_gj_panel<<<(int)(((int64_t)b * n + 255) / 256), 256, 0, st>>>(A, n, p0, b, Pinv, U, Lo);
    k_gj_update<<<(int)((nn + 255) / 256), 256, 0, st>>>(A, n, p0, b, Pinv, U, Lo);
    count_launches(3);
  }
  *result = A;
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
