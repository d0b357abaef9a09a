// Conjugate gradients on K_FF lambda_F = f_F preconditioned by one V-cycle
// (the symmetric cycle of Sec. 3 with reversed post-smoothing).  Flexible
// (Polak-Ribiere) beta = z.(r - r_prev) / (z_prev.r_prev), so a float32 cycle,
// which is only nearly linear, is tolerated.  All vectors are float64 on the
// finest level in the split layout; scalars stay on the device (alpha and
// beta are formed by one-thread kernels), so an iteration needs no host
// round trip except the residual norm the driver reads for its stopping test.
#include "kernels.cuh"

namespace mcw {
namespace {

constexpr int kThreads = 128;

__device__ __forceinline__ void block_partial2(double a, double b, double* partials) {
  __shared__ double red[2][kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  if ((t & 31) == 0) { red[0][t >> 5] = a; red[1][t >> 5] = b; }
  __syncthreads();
  if (t == 0) {
    double sa = 0.0, sb = 0.0;
#pragma unroll
    for (int q = 0; q < kThreads / 32; ++q) { sa += red[0][q]; sb += red[1][q]; }
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    partials[2 * blk] = sa;
    partials[2 * blk + 1] = sb;
  }
}

// thread per free column (blockDim 32 x 4, blockIdx.z = parity of i)
__device__ __forceinline__ bool free_column(const Grid& g, int64_t& own) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int i = 2 * h + (int)blockIdx.z;
  own = (int64_t)j * g.RP + (int64_t)(i & 1) * g.H + (i >> 1);
  return i >= 1 && i <= g.Nx - 2 && j >= 1 && j <= g.Ny - 2;
}

// partials of (r . z, rp . z), z the preconditioned residual in precision TZ
template <typename TZ>
__global__ void __launch_bounds__(kThreads) k_cg_dots(Grid g, const double* __restrict__ r,
                                                      const double* __restrict__ rp,
                                                      const TZ* __restrict__ z,
                                                      double* __restrict__ partials) {
  int64_t own;
  double a = 0.0, b = 0.0;
  if (free_column(g, own))
    for (int k = 0; k <= g.Nz - 2; ++k) {
      const int64_t q = (int64_t)k * g.PP + own;
      const double zq = (double)z[q];
      a += r[q] * zq;
      b += rp[q] * zq;
    }
  block_partial2(a, b, partials);
}

// s[0] = r.z, s[1] = rp.z, s[2] = previous r.z, s[3] = beta (written), s[4] = p.Kp,
// s[5] = restart flag (set by k_cg_start, cleared here: beta = 0 after a restart)
__global__ void k_cg_beta(double* s) {
  const double rz = s[0], rpz = s[1], old = s[2];
  s[3] = s[5] != 0.0 ? 0.0 : (rz - rpz) / old;
  s[2] = rz;
  s[5] = 0.0;
}

template <typename TZ>
__global__ void __launch_bounds__(kThreads) k_cg_direction(Grid g, const TZ* __restrict__ z,
                                                           double* __restrict__ p,
                                                           const double* __restrict__ s) {
  int64_t own;
  if (!free_column(g, own)) return;
  const double beta = s[3];
  for (int k = 0; k <= g.Nz - 2; ++k) {
    const int64_t q = (int64_t)k * g.PP + own;
    p[q] = (double)z[q] + beta * p[q];
  }
}

// alpha = (r.z) / (p.Kp); x += alpha p; rp = r; r -= alpha q; the next
// preconditioner input (pf = r in precision TP, px = 0); partials of r.r.
template <typename TP>
__global__ void __launch_bounds__(kThreads) k_cg_update(Grid g, double* __restrict__ x,
                                                        double* __restrict__ r,
                                                        double* __restrict__ rp,
                                                        const double* __restrict__ p,
                                                        const double* __restrict__ qv,
                                                        TP* __restrict__ pf, TP* __restrict__ px,
                                                        const double* __restrict__ s,
                                                        double* __restrict__ partials) {
  int64_t own;
  double rr = 0.0;
  if (free_column(g, own)) {
    const double alpha = s[2] / s[4];
    for (int k = 0; k <= g.Nz - 2; ++k) {
      const int64_t q = (int64_t)k * g.PP + own;
      const double rk = r[q];
      x[q] += alpha * p[q];
      const double rn = rk - alpha * qv[q];
      rp[q] = rk;
      r[q] = rn;
      pf[q] = (TP)rn;
      px[q] = TP(0);
      rr += rn * rn;
    }
  }
  block_partial2(rr, 0.0, partials);
}

// preconditioner input from r without an update: pf = r, px = 0, rp = 0
template <typename TP>
__global__ void __launch_bounds__(kThreads) k_cg_start(Grid g, const double* __restrict__ r,
                                                       double* __restrict__ rp,
                                                       TP* __restrict__ pf, TP* __restrict__ px,
                                                       double* __restrict__ s) {
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
      threadIdx.y == 0)
    s[5] = 1.0;
  int64_t own;
  if (!free_column(g, own)) return;
  for (int k = 0; k <= g.Nz - 2; ++k) {
    const int64_t q = (int64_t)k * g.PP + own;
    pf[q] = (TP)r[q];
    px[q] = TP(0);
    rp[q] = 0.0;
  }
}

__global__ void __launch_bounds__(1024) k_reduce_pairs(const double* __restrict__ p, int n,
                                                       double* out0, double* out1) {
  __shared__ double red[2][32];
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < n; t += 1024) {
    a += p[2 * t];
    b += p[2 * t + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = a; red[1][threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x < 32) {
    a = red[0][threadIdx.x];
    b = red[1][threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
      if (out0) *out0 = a;
      if (out1) *out1 = b;
    }
  }
}

inline dim3 col_grid(const Grid& g) { return dim3((g.H + 31) / 32, (g.Ny + 3) / 4, 2); }

}  // namespace

int krylov_blocks(const Grid& g) {
  dim3 d = col_grid(g);
  return (int)(d.x * d.y * d.z);
}

template <typename TZ>
cudaError_t launch_cg_dots(const Grid& g, const double* r, const double* rp, const TZ* z,
                           double* partials, int cap, double* s, cudaStream_t st) {
  const int nb = krylov_blocks(g);
  if (2 * nb > cap) return cudaErrorInvalidValue;
  k_cg_dots<TZ><<<col_grid(g), dim3(32, 4), 0, st>>>(g, r, rp, z, partials); count_launches(1);
  k_reduce_pairs<<<1, 1024, 0, st>>>(partials, nb, s + 0, s + 1); count_launches(1);
  return cudaGetLastError();
}

template <typename TZ>
cudaError_t launch_cg_direction(const Grid& g, const TZ* z, double* p, double* s,
                                cudaStream_t st) {
  k_cg_beta<<<1, 1, 0, st>>>(s); count_launches(1);
  k_cg_direction<TZ><<<col_grid(g), dim3(32, 4), 0, st>>>(g, z, p, s); count_launches(1);
  return cudaGetLastError();
}

template <typename TP>
cudaError_t launch_cg_update(const Grid& g, double* x, double* r, double* rp, const double* p,
                             const double* q, TP* pf, TP* px, double* s, double* partials,
                             int cap, double* rr_out, cudaStream_t st) {
  const int nb = krylov_blocks(g);
  if (2 * nb > cap) return cudaErrorInvalidValue;
  k_cg_update<TP><<<col_grid(g), dim3(32, 4), 0, st>>>(g, x, r, rp, p, q, pf, px, s, partials);
  count_launches(1);
  k_reduce_pairs<<<1, 1024, 0, st>>>(partials, nb, rr_out, nullptr); count_launches(1);
  return cudaGetLastError();
}

template <typename TP>
cudaError_t launch_cg_start(const Grid& g, const double* r, double* rp, TP* pf, TP* px, double* s,
                            cudaStream_t st) {
  k_cg_start<TP><<<col_grid(g), dim3(32, 4), 0, st>>>(g, r, rp, pf, px, s); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_reduce_pairs(const double* partials, int n, double* out0, double* out1,
                                cudaStream_t st) {
  k_reduce_pairs<<<1, 1024, 0, st>>>(partials, n, out0, out1); count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_cg_dots<double>(const Grid&, const double*, const double*,
                                            const double*, double*, int, double*, cudaStream_t);
template cudaError_t launch_cg_dots<float>(const Grid&, const double*, const double*,
                                           const float*, double*, int, double*, cudaStream_t);
template cudaError_t launch_cg_direction<double>(const Grid&, const double*, double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_cg_direction<float>(const Grid&, const float*, double*, double*,
                                                cudaStream_t);
template cudaError_t launch_cg_update<double>(const Grid&, double*, double*, double*,
                                              const double*, const double*, double*, double*,
                                              double*, double*, int, double*, cudaStream_t);
template cudaError_t launch_cg_update<float>(const Grid&, double*, double*, double*, const double*,
                                             const double*, float*, float*, double*, double*, int,
                                             double*, cudaStream_t);
template cudaError_t launch_cg_start<double>(const Grid&, const double*, double*, double*,
                                             double*, double*, cudaStream_t);
template cudaError_t launch_cg_start<float>(const Grid&, const double*, double*, float*, float*,
                                            double*, cudaStream_t);

}  // namespace mcw
