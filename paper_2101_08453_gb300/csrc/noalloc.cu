// Residual norms that allocate nothing: mcwind_residual_norm_noalloc.
//
// Why it exists: some callers cannot call cudaMalloc at the point where they
// want to check a solution -- for example a host model that hands all device
// memory to its own pool at start-up and forbids later allocations, or a
// latency-bound loop in which an allocation (which may synchronize the whole
// device) is not allowed.  This entry point computes the same two norms as
// the solver's convergence check without asking for any memory: its
// per-block partial sums live in the file-scope array below, which every GPU
// that loads the library holds until the process exits.
//
// The array is shared by every call, on every stream, and keeps the last
// call's contents; nothing in it has to start at zero (each call writes every
// partial it later reads).  Calls whose kernels overlap on the GPU race on it:
// serialize them (one stream, or events between streams).
#include <mutex>

#include "kernels.cuh"

namespace mcw {
namespace {

// Two partial sums (f^2 and r^2) per block of 32 x 4 columns.
constexpr int kNoAllocMaxBlocks = 131072;
static __device__ __align__(256) double g_noalloc_partials[2 * kNoAllocMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double* g_dev_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current).
cudaError_t scratch_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = (double*)p;
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

// One thread per column (blockDim 32 x 4, blockIdx.z = parity of i), the
// launch shape of the solver's residual kernel.  lambda and f are read in
// the caller's [k][j][i] layout; the stencil in the plan's layout.
__global__ void __launch_bounds__(128) k_residual_norm_noalloc(Grid g, const double* __restrict__ C,
                                                               const double* __restrict__ f,
                                                               const double* __restrict__ lam,
                                                               double* __restrict__ partials) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int i = 2 * h + (int)blockIdx.z;
  double sf = 0.0, sr = 0.0;
  if (i >= 1 && i <= g.Nx - 2 && j >= 1 && j <= g.Ny - 2) {
    const int64_t lay = (int64_t)g.Nx * g.Ny;  // standard-layout layer pitch
    int64_t col[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) col[c] = (int64_t)(j + c / 3 - 1) * g.Nx + (i + c % 3 - 1);
    // fixed nodes count as lambda = 0
    auto lval = [&](int c, int k) -> double {
      const int ii = i + c % 3 - 1, jj = j + c / 3 - 1;
      return is_free(g, ii, jj, k) ? lam[(int64_t)k * lay + col[c]] : 0.0;
    };
    const int64_t own = (int64_t)j * g.RP + (int64_t)(i & 1) * g.H + (i >> 1);
    double w[3][9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      w[0][c] = 0.0;
      w[1][c] = lval(c, 0);
      w[2][c] = lval(c, 1);
    }
    for (int k = 0; k <= g.Nz - 2; ++k) {
      const int64_t b = (int64_t)k * g.PP + own;
      const double fk = f[(int64_t)k * lay + col[4]];
      double acc = fk;
#pragma unroll
      for (int s = 0; s < 27; ++s) acc -= C[cidx(b, s)] * w[s / 9][s % 9];
      sf += fk * fk;
      sr += acc * acc;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        w[0][c] = w[1][c];
        w[1][c] = w[2][c];
        w[2][c] = (k + 2 <= g.Nz - 1) ? lval(c, k + 2) : 0.0;
      }
    }
  }
  __shared__ double red[2][4];
  for (int o = 16; o > 0; o >>= 1) {
    sf += __shfl_down_sync(0xffffffffu, sf, o);
    sr += __shfl_down_sync(0xffffffffu, sr, o);
  }
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  if ((t & 31) == 0) { red[0][t >> 5] = sf; red[1][t >> 5] = sr; }
  __syncthreads();
  if (t == 0) {
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    partials[2 * blk] = red[0][0] + red[0][1] + red[0][2] + red[0][3];
    partials[2 * blk + 1] = red[1][0] + red[1][1] + red[1][2] + red[1][3];
  }
}

// Fixed-order sum of the n block partials; norms = (||f_F||, ||f_F - K_FF lambda_F||).
__global__ void __launch_bounds__(1024) k_norms_noalloc(const double* __restrict__ partials, int n,
                                                        double* __restrict__ norms) {
  __shared__ double red[2][32];
  double sf = 0.0, sr = 0.0;
  for (int q = threadIdx.x; q < n; q += 1024) {
    sf += partials[2 * q];
    sr += partials[2 * q + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    sf += __shfl_down_sync(0xffffffffu, sf, o);
    sr += __shfl_down_sync(0xffffffffu, sr, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = sf; red[1][threadIdx.x >> 5] = sr; }
  __syncthreads();
  if (threadIdx.x < 32) {
    sf = red[0][threadIdx.x];
    sr = red[1][threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) {
      sf += __shfl_down_sync(0xffffffffu, sf, o);
      sr += __shfl_down_sync(0xffffffffu, sr, o);
    }
    if (threadIdx.x == 0) {
      norms[0] = sqrt(sf);
      norms[1] = sqrt(sr);
    }
  }
}

}  // namespace
}  // namespace mcw

using namespace mcw;

extern "C" int mcwind_residual_norm_noalloc(mcwind_plan p, const double* f, const double* lambda,
                                            double* norms, void* stream) {
  if (!p || !f || !lambda || !norms) return MCWIND_EINVAL;
  const Grid& g = p->lv[0].g;
  const dim3 grd((g.H + 31) / 32, (g.Ny + 3) / 4, 2);
  if ((int64_t)grd.x * grd.y * grd.z > kNoAllocMaxBlocks) return MCWIND_EINVAL;
  if (!p->assembled) return MCWIND_ESTATE;
  double* scratch = nullptr;
  cudaError_t e = scratch_on_current_device(&scratch);
  if (e != cudaSuccess) return MCWIND_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const double* C = (const double*)(p->ws + (size_t)p->lv[0].C64);
  k_residual_norm_noalloc<<<grd, dim3(32, 4), 0, st>>>(g, C, f, lambda, scratch);
  count_launches(1);
  k_norms_noalloc<<<1, 1024, 0, st>>>(scratch, (int)(grd.x * grd.y * grd.z), norms);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? MCWIND_OK : MCWIND_ECUDA;
}
