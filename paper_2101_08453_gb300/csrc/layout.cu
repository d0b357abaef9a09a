// Layout conversion, stencil finalization and deterministic reductions.
#include "dfloat.cuh"
#include "kernels.cuh"

namespace mcw {
namespace {

// thread -> node (i, j, k) of grid g, node-centric kernels: blockDim (32, 4),
// x = half-row index h, y = j, z = 2k + parity.
__device__ __forceinline__ bool node_of_thread(const Grid& g, int& i, int& j, int& k) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  j = blockIdx.y * blockDim.y + threadIdx.y;
  int p = blockIdx.z & 1;
  k = blockIdx.z >> 1;
  i = 2 * h + p;
  return i < g.Nx && j < g.Ny;
}

inline dim3 node_grid(const Grid& g) {
  return dim3((g.H + 31) / 32, (g.Ny + 3) / 4, 2 * g.Nz);
}

template <typename T>
__global__ void k_std_to_split(Grid g, const double* __restrict__ src, T* __restrict__ dst,
                               int zero_fixed) {
  int i, j, k;
  if (!node_of_thread(g, i, j, k)) return;
  double v = src[((int64_t)k * g.Ny + j) * g.Nx + i];
  if (zero_fixed && !is_free(g, i, j, k)) v = 0.0;
  dst[gidx(g, i, j, k)] = (T)v;
}

template <typename T>
__global__ void k_split_to_std(Grid g, const T* __restrict__ src, double* __restrict__ dst) {
  int i, j, k;
  if (!node_of_thread(g, i, j, k)) return;
  dst[((int64_t)k * g.Ny + j) * g.Nx + i] = (double)src[gidx(g, i, j, k)];
}

template <typename T>
__global__ void k_stencil_export(Grid g, const T* __restrict__ C, double* __restrict__ out) {
  int i, j, k;
  if (!node_of_thread(g, i, j, k)) return;
  int64_t n = (int64_t)g.Nx * g.Ny * g.Nz;
  int64_t o = ((int64_t)k * g.Ny + j) * g.Nx + i;
  int64_t id = gidx(g, i, j, k);
#pragma unroll
  for (int s = 0; s < 27; ++s) out[s * n + o] = (double)coef(C, g.total, id, s);
}

// float64 operator -> float32 copy in the same tiled order: n = kPlanes x
// total values, 2 per thread and turn (16-byte loads, 8-byte stores); the
// rounding is done in integer arithmetic (float_of_bits), off the double pipe
__global__ void k_to_f32(const double2* __restrict__ a, float2* __restrict__ t, int64_t n2) {
  int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; b + 3 * st < n2; b += 4 * st) {
    double2 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = a[b + q * st];
#pragma unroll
    for (int q = 0; q < 4; ++q) t[b + q * st] = make_float2(float_of_bits(v[q].x), float_of_bits(v[q].y));
  }
  for (; b < n2; b += st) {
    const double2 v = a[b];
    t[b] = make_float2(float_of_bits(v.x), float_of_bits(v.y));
  }
}

__global__ void k_finalize(Grid g, double* __restrict__ C, int* flag) {
  int i, j, k;
  if (!node_of_thread(g, i, j, k)) return;
  int64_t id = gidx(g, i, j, k);
  bool fr = is_free(g, i, j, k);
#pragma unroll
  for (int s = 0; s < 27; ++s) {
    int di = s % 3 - 1, dj = (s / 3) % 3 - 1, dk = s / 9 - 1;
    if (!fr || !is_free(g, i + di, j + dj, k + dk)) C[cidx(id, s)] = 0.0;
  }
  double d = C[cidx(id, kDiag)];
  if (fr && !(d > 0.0)) atomicOr(flag, 2);
  C[cidx(id, kInvDiag)] = fr ? 1.0 / d : 0.0;
}

constexpr int kRedThreads = 128;

// sum of v^2 over the free nodes: one thread per column (blockDim 32 x 4,
// blockIdx.z = parity of i), the same launch shape as the residual kernel,
// so it writes exactly residual_blocks(g) partials.
__global__ void __launch_bounds__(kRedThreads) k_norm2_partials(Grid g, const double* __restrict__ v,
                                                                double* __restrict__ partials) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int i = 2 * h + (int)blockIdx.z;
  double s = 0.0;
  if (i >= 1 && i <= g.Nx - 2 && j >= 1 && j <= g.Ny - 2) {
    const int64_t own = (int64_t)j * g.RP + (int64_t)(i & 1) * g.H + (i >> 1);
    for (int k = 0; k <= g.Nz - 2; ++k) {
      const double x = v[(int64_t)k * g.PP + own];
      s += x * x;
    }
  }
  __shared__ double red[kRedThreads / 32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  if ((t & 31) == 0) red[t >> 5] = s;
  __syncthreads();
  if (t == 0) {
    double b = 0.0;
#pragma unroll
    for (int q = 0; q < kRedThreads / 32; ++q) b += red[q];
    partials[((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = b;
  }
}

// One block, fixed order: thread t sums partials t, t+1024, ...; then a
// fixed tree.  The result depends only on n and the partials.
__global__ void __launch_bounds__(1024) k_reduce_final(const double* __restrict__ p, int n,
                                                       double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += 1024) s += p[t];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = red[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_std_to_split(const Grid& g, const double* src, T* dst, bool zero_fixed,
                                cudaStream_t st) {
  k_std_to_split<T><<<node_grid(g), dim3(32, 4), 0, st>>>(g, src, dst, zero_fixed ? 1 : 0); count_launches(1);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_split_to_std(const Grid& g, const T* src, double* dst, cudaStream_t st) {
  k_split_to_std<T><<<node_grid(g), dim3(32, 4), 0, st>>>(g, src, dst); count_launches(1);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_stencil_export(const Grid& g, const T* C, double* out, cudaStream_t st) {
  k_stencil_export<T><<<node_grid(g), dim3(32, 4), 0, st>>>(g, C, out); count_launches(1);
  return cudaGetLastError();
}
template cudaError_t launch_std_to_split<double>(const Grid&, const double*, double*, bool, cudaStream_t);
template cudaError_t launch_std_to_split<float>(const Grid&, const double*, float*, bool, cudaStream_t);
template cudaError_t launch_split_to_std<double>(const Grid&, const double*, double*, cudaStream_t);
template cudaError_t launch_split_to_std<float>(const Grid&, const float*, double*, cudaStream_t);
template cudaError_t launch_stencil_export<double>(const Grid&, const double*, double*, cudaStream_t);
template cudaError_t launch_stencil_export<float>(const Grid&, const float*, double*, cudaStream_t);

cudaError_t launch_stencil_to_f32(const Grid& g, const double* C64, float* C32, cudaStream_t st) {
  const int64_t n2 = (int64_t)kPlanes * g.total / 2;  // total is a multiple of 64
  int blocks = (int)std::min<int64_t>((n2 + 255) / 256, 152 * 16);
  k_to_f32<<<blocks, 256, 0, st>>>((const double2*)C64, (float2*)C32, n2); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_stencil_finalize(const Grid& g, double* C, int* flag, cudaStream_t st) {
  k_finalize<<<node_grid(g), dim3(32, 4), 0, st>>>(g, C, flag); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_norm2_partials(const Grid& g, const double* v, double* partials, int cap,
                                  int* nblocks, cudaStream_t st) {
  dim3 grd((g.H + 31) / 32, (g.Ny + 3) / 4, 2);
  if ((int64_t)grd.x * grd.y * grd.z > cap) return cudaErrorInvalidValue;
  k_norm2_partials<<<grd, dim3(32, 4), 0, st>>>(g, v, partials); count_launches(1);
  *nblocks = (int)(grd.x * grd.y * grd.z);
  return cudaGetLastError();
}

cudaError_t launch_reduce_final(const double* partials, int n, double* out, cudaStream_t st) {
  k_reduce_final<<<1, 1024, 0, st>>>(partials, n, out); count_launches(1);
  return cudaGetLastError();
}

}  // namespace mcw

#include <atomic>

namespace mcw {
static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace mcw

extern "C" long long mcwind_launch_count(void) { return mcw::g_launches.load(); }
