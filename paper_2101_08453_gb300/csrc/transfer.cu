// Residual, restriction and prolongation (Sec. 3, Eq. 7), and the float64
// refinement kernels of the mixed-precision solve.
#include <climits>
#include "kernels.cuh"

namespace mcw {
namespace {

constexpr int kResThreads = 128;

// Sum over the block in fixed order; thread 0 writes the block's partial.
__device__ __forceinline__ void block_partial(double s, double* partials) {
  __shared__ double red[kResThreads / 32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  if ((t & 31) == 0) red[t >> 5] = s;
  __syncthreads();
  if (t == 0) {
    double b = 0.0;
#pragma unroll
    for (int q = 0; q < kResThreads / 32; ++q) b += red[q];
    partials[((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = b;
  }
}

// r = f - K x over one column, all k, both parities (blockIdx.z = parity).
// MODE 0: write r (type T) and the partials of r . r.  MODE 3: write r only
// (the residual of a cycle, before restriction: no norm, no double
// arithmetic).  MODE 1 (T = double): write (float) r into r32 and zero e32,
// the start of one float32 correction cycle.  MODE 2: r = K x (f unused) and
// the partials of x . K x instead of r . r.  MODE 4 / MODE 5: MODE 1 / MODE 0
// for x = 0 (a cold start), r = f without reading K or x (K 0 = 0 exactly,
// so the result and its partials are those of the full residual).
template <typename T, int MODE>
__global__ void __launch_bounds__(kResThreads) k_residual(Grid g, const T* __restrict__ C,
                                                          const T* __restrict__ f,
                                                          const T* __restrict__ x,
                                                          T* __restrict__ r,
                                                          float* __restrict__ r32,
                                                          float* __restrict__ e32,
                                                          double* __restrict__ partials) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int i = 2 * h + (int)blockIdx.z;
  double ss = 0.0;
  if (i < g.Nx && j < g.Ny) {
    const int64_t PP = g.PP, tot = g.total;
    const int64_t own = (int64_t)j * g.RP + (int64_t)(i & 1) * g.H + (i >> 1);
    const bool fcol = i >= 1 && i <= g.Nx - 2 && j >= 1 && j <= g.Ny - 2;
    if (!fcol) {
      for (int k = 0; k < g.Nz; ++k) {
        const int64_t b = (int64_t)k * PP + own;
        if (MODE != 1 && MODE != 4) r[b] = T(0);
        else { r32[b] = 0.0f; e32[b] = 0.0f; }
      }
    } else if (MODE >= 4) {
      for (int k = 0; k <= g.Nz - 2; ++k) {
        const int64_t b = (int64_t)k * PP + own;
        const T acc = f[b];
        ss += (double)acc * (double)acc;
        if (MODE == 5) r[b] = acc;
        else { r32[b] = (float)acc; e32[b] = 0.0f; }
      }
      const int64_t b = (int64_t)(g.Nz - 1) * PP + own;
      if (MODE == 5) r[b] = T(0);
      else { r32[b] = 0.0f; e32[b] = 0.0f; }
    } else {
      int64_t col[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const int ii = i + c % 3 - 1, jj = j + c / 3 - 1;
        col[c] = (int64_t)jj * g.RP + (int64_t)(ii & 1) * g.H + (ii >> 1);
      }
      T w[3][9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        w[0][c] = T(0);
        w[1][c] = x[col[c]];
        w[2][c] = x[PP + col[c]];
      }
      for (int k = 0; k <= g.Nz - 2; ++k) {
        const int64_t b = (int64_t)k * PP + own;
        T acc;
        if (MODE == 2) {
          acc = T(0);
#pragma unroll
          for (int s = 0; s < 27; ++s) acc += coef(C, tot, b, s) * w[s / 9][s % 9];
          ss += (double)acc * (double)w[1][4];
        } else {
          acc = f[b];
#pragma unroll
          for (int s = 0; s < 27; ++s) acc -= coef(C, tot, b, s) * w[s / 9][s % 9];
          if (MODE != 3) ss += (double)acc * (double)acc;
        }
        if (MODE != 1) r[b] = acc;
        else { r32[b] = (float)acc; e32[b] = 0.0f; }
#pragma unroll
        for (int c = 0; c < 9; ++c) {
          w[0][c] = w[1][c];
          w[1][c] = w[2][c];
        }
        if (k + 2 <= g.Nz - 1) {
#pragma unroll
          for (int c = 0; c < 9; ++c) w[2][c] = x[(int64_t)(k + 2) * PP + col[c]];
        } else {
#pragma unroll
          for (int c = 0; c < 9; ++c) w[2][c] = T(0);
        }
      }
      const int64_t b = (int64_t)(g.Nz - 1) * PP + own;
      if (MODE != 1) r[b] = T(0);
      else { r32[b] = 0.0f; e32[b] = 0.0f; }
    }
  }
  if (MODE != 3 && partials) block_partial(ss, partials);
}

__device__ __forceinline__ bool node_of_thread(const Grid& g, int& i, int& j, int& k) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  j = blockIdx.y * blockDim.y + threadIdx.y;
  k = blockIdx.z >> 1;
  i = 2 * h + (blockIdx.z & 1);
  return i < g.Nx && j < g.Ny;
}

inline dim3 node_grid(const Grid& g) { return dim3((g.H + 31) / 32, (g.Ny + 3) / 4, 2 * g.Nz); }
// one thread per column (i, j); blockIdx.z = parity of i
inline dim3 column_grid(const Grid& g) { return dim3((g.H + 31) / 32, (g.Ny + 3) / 4, 2); }

__global__ void k_update_mixed(Grid g, double* __restrict__ x, const float* __restrict__ e) {
  int i, j, k;
  if (!node_of_thread(g, i, j, k) || !is_free(g, i, j, k)) return;
  const int64_t b = gidx(g, i, j, k);
  x[b] += (double)e[b];
}

// vertical restriction weights of coarse layer K
template <typename W>
__device__ __forceinline__ void vcoarse(const Transfer& tr, int K, int& f, W& wm, W& wp) {
  f = tr.kf[K];
  wm = (K > 0 && tr.kf[K] - tr.kf[K - 1] == 2) ? W(0.5) : W(0);
  wp = (K < tr.Nzc - 1 && tr.kf[K + 1] - tr.kf[K] == 2) ? W(0.5) : W(0);
}

// a*b + c with one rounding, in the cycle's precision
__device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return fma(a, b, c); }

// f_c = P^T r (Eq. 7) over one coarse column (I, J), all K: each coarse node
// gathers up to 3 x 3 x 3 fine residuals with the interpolation weights (1
// at the coarse node, 1/2 at the half nodes around it, 0 where a coarse
// interval spans one fine cell), accumulated in the precision of the cycle
// (T).  HX, HY: the level is coarsened in x, y.  Per direction the sum is
// centre + 1/2 (minus + plus), a tap of weight 0 selected to an exact 0, so
// a coarse node costs two operations per tap and direction instead of a
// multiply-add per tap of the 27 (on GB300 the float64 pipe, not HBM, bounds
// the float64 transfers).  Every tap is loaded without a branch (a tap
// outside the stencil reads a valid neighbour), and layers go in chunks of
// U, so a thread has all loads of U nodes in flight.
template <typename T, bool HX, bool HY, typename Ix>
__global__ void __launch_bounds__(128) k_restrict(Grid gf, Grid gc, Transfer tr,
                                                  const T* __restrict__ r, T* __restrict__ fc) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int I = 2 * h + (int)blockIdx.z;
  if (I >= gc.Nx || J >= gc.Ny) return;
  const Ix own = (Ix)J * (Ix)gc.RP + (Ix)(I & 1) * (Ix)gc.H + (Ix)(I >> 1);
  if (I < 1 || I > gc.Nx - 2 || J < 1 || J > gc.Ny - 2) {
    for (int K = 0; K < gc.Nz; ++K) fc[(Ix)K * (Ix)gc.PP + own] = T(0);
    return;
  }
  constexpr int NA = HX ? 3 : 1, NB = HY ? 3 : 1;
  int fi, fj;
  float wxm, wxp, wym, wyp;
  hcoarse(HX ? 1 : 0, gf.Nx, gc.Nx, I, fi, wxm, wxp);
  hcoarse(HY ? 1 : 0, gf.Ny, gc.Ny, J, fj, wym, wyp);
  const bool mx = wxm != 0.0f, px = wxp != 0.0f, my = wym != 0.0f, py = wyp != 0.0f;
  // in-layer offsets of the taps (fine columns fi-1..fi+1 are valid: I is interior)
  Ix hoff[NB][NA];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      const int ii = HX ? fi + a - 1 : fi, jj = HY ? fj + b - 1 : fj;
      hoff[b][a] = (Ix)jj * (Ix)gf.RP + (Ix)(ii & 1) * (Ix)gf.H + (Ix)(ii >> 1);
    }
  }
  const int Kend = gc.Nz - 1;  // the top layer is Dirichlet
  constexpr int U = NA * NB >= 9 ? 1 : (NA * NB >= 3 ? 2 : 4);  // about 12 loads in flight
  for (int K0 = 0; K0 < Kend; K0 += U) {
    T v[U][3][NB][NA];
    bool mz[U], pz[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int K = min(K0 + u, Kend - 1);
      int fk;
      float wzm, wzp;
      vcoarse(tr, K, fk, wzm, wzp);
      mz[u] = wzm != 0.0f;
      pz[u] = wzp != 0.0f;
      const int kl[3] = {mz[u] ? fk - 1 : fk, fk, pz[u] ? fk + 1 : fk};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T* rl = r + (Ix)kl[c] * (Ix)gf.PP;
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int a = 0; a < NA; ++a) v[u][c][b][a] = rl[hoff[b][a]];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      T col[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T row[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          if (HX) {
            const T m = mx ? v[u][c][b][0] : T(0), pl = px ? v[u][c][b][NA - 1] : T(0);
            row[b] = madd(T(0.5), m + pl, v[u][c][b][NA / 2]);
          } else {
            row[b] = v[u][c][b][0];
          }
        }
        if (HY) {
          const T m = my ? row[0] : T(0), pl = py ? row[NB - 1] : T(0);
          col[c] = madd(T(0.5), m + pl, row[NB / 2]);
        } else {
          col[c] = row[0];
        }
      }
      const T m = mz[u] ? col[0] : T(0), pl = pz[u] ? col[2] : T(0);
      const T out = madd(T(0.5), m + pl, col[1]);
      if (K0 + u < Kend) fc[(Ix)(K0 + u) * (Ix)gc.PP + own] = out;
    }
  }
  fc[(Ix)Kend * (Ix)gc.PP + own] = T(0);
}

// x += P e_c (Eq. 7) over one fine column (i, j), all free k.  Per direction
// a fine node has one coarse tap (weight 1) or two (weight 1/2 each), so its
// n = 1..8 taps share the weight 2^-m (m = directions with two taps) and
// x + 2^-m (sum of the taps) costs n - 1 additions and one multiply-add.
// The tap pattern is the same for a whole warp (one row of one parity of i,
// one layer at a time), so the selections below do not diverge; every tap
// is loaded without a branch (a missing second tap repeats the first, an L1
// hit) and layers go in chunks of U as above.
// I: the index type of offsets within a level (int when both levels have
// fewer than 2^31 entries: 32-bit address arithmetic)
template <typename T, bool HX, bool HY, typename I>
__global__ void __launch_bounds__(128) k_prolong_add(Grid gf, Grid gc, Transfer tr,
                                                     const T* __restrict__ ec,
                                                     T* __restrict__ x) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int i = 2 * h + (int)blockIdx.z;
  if (i < 1 || i > gf.Nx - 2 || j < 1 || j > gf.Ny - 2) return;
  constexpr int NA = HX ? 2 : 1, NB = HY ? 2 : 1;
  int ci[2], cj[2];
  float ax[2], ay[2];
  hpair(HX ? 1 : 0, gf.Nx, gc.Nx, i, ci[0], ax[0], ci[1], ax[1]);
  hpair(HY ? 1 : 0, gf.Ny, gc.Ny, j, cj[0], ay[0], cj[1], ay[1]);
  const bool two_x = HX && ci[0] != ci[1], two_y = HY && cj[0] != cj[1];
  I hoff[NB][NA];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int a = 0; a < NA; ++a)
      hoff[b][a] = (I)cj[b] * (I)gc.RP + (I)(ci[a] & 1) * (I)gc.H + (I)(ci[a] >> 1);
  const I own = (I)j * (I)gf.RP + (I)(i & 1) * (I)gf.H + (I)(i >> 1);
  const int kend = gf.Nz - 1;  // free layers 0 .. Nz-2
  constexpr int U = NA * NB >= 4 ? 2 : 4;
  for (int k0 = 0; k0 < kend; k0 += U) {
    T xv[U], ev[U][2][NB][NA];
    bool two_z[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = min(k0 + u, kend - 1);
      xv[u] = x[(I)k * (I)gf.PP + own];
      const int ck[2] = {tr.kc0[k], tr.kc1[k]};
      two_z[u] = ck[0] != ck[1];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const T* el = ec + (I)ck[c] * (I)gc.PP;
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int a = 0; a < NA; ++a) ev[u][c][b][a] = el[hoff[b][a]];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      T sz[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        T sy[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b)
          sy[b] = (HX && two_x) ? ev[u][c][b][0] + ev[u][c][b][NA - 1] : ev[u][c][b][0];
        sz[c] = (HY && two_y) ? sy[0] + sy[NB - 1] : sy[0];
      }
      const T s = two_z[u] ? sz[0] + sz[1] : sz[0];
      const int m = (int)two_x + (int)two_y + (int)two_z[u];
      const T w = m == 0 ? T(1) : (m == 1 ? T(0.5) : (m == 2 ? T(0.25) : T(0.125)));
      if (k0 + u < kend) x[(I)(k0 + u) * (I)gf.PP + own] = madd(w, s, xv[u]);
    }
  }
}

}  // namespace

int residual_blocks(const Grid& g) {
  return ((g.H + 31) / 32) * ((g.Ny + 3) / 4) * 2;
}

template <typename T>
cudaError_t launch_residual(const Grid& g, const T* C, const T* f, const T* x, T* r,
                            double* partials, int cap, int* nblocks, cudaStream_t st) {
  dim3 grd((g.H + 31) / 32, (g.Ny + 3) / 4, 2);
  if (partials && (int64_t)grd.x * grd.y * grd.z > cap) return cudaErrorInvalidValue;
  if (partials && !x)  // x = 0
    k_residual<T, 5><<<grd, dim3(32, 4), 0, st>>>(g, C, f, x, r, nullptr, nullptr, partials);
  else if (partials)
    k_residual<T, 0><<<grd, dim3(32, 4), 0, st>>>(g, C, f, x, r, nullptr, nullptr, partials);
  else
    k_residual<T, 3><<<grd, dim3(32, 4), 0, st>>>(g, C, f, x, r, nullptr, nullptr, nullptr);
  count_launches(1);
  if (nblocks) *nblocks = (int)(grd.x * grd.y * grd.z);
  return cudaGetLastError();
}
template cudaError_t launch_residual<double>(const Grid&, const double*, const double*,
                                             const double*, double*, double*, int, int*,
                                             cudaStream_t);
template cudaError_t launch_residual<float>(const Grid&, const float*, const float*,
                                            const float*, float*, double*, int, int*,
                                            cudaStream_t);

cudaError_t launch_residual_mixed(const Grid& g, const double* C, const double* f,
                                  const double* x, float* r32, float* e32, double* partials,
                                  int cap, int* nblocks, cudaStream_t st) {
  dim3 grd((g.H + 31) / 32, (g.Ny + 3) / 4, 2);
  if (partials && (int64_t)grd.x * grd.y * grd.z > cap) return cudaErrorInvalidValue;
  if (x)
    k_residual<double, 1><<<grd, dim3(32, 4), 0, st>>>(g, C, f, x, nullptr, r32, e32, partials);
  else
    k_residual<double, 4><<<grd, dim3(32, 4), 0, st>>>(g, C, f, x, nullptr, r32, e32, partials);
  count_launches(1);
  if (nblocks) *nblocks = (int)(grd.x * grd.y * grd.z);
  return cudaGetLastError();
}

cudaError_t launch_apply(const Grid& g, const double* C, const double* x, double* y,
                         double* partials, int cap, int* nblocks, cudaStream_t st) {
  dim3 grd((g.H + 31) / 32, (g.Ny + 3) / 4, 2);
  if ((int64_t)grd.x * grd.y * grd.z > cap) return cudaErrorInvalidValue;
  k_residual<double, 2><<<grd, dim3(32, 4), 0, st>>>(g, C, nullptr, x, y, nullptr, nullptr, partials); count_launches(1);
  if (nblocks) *nblocks = (int)(grd.x * grd.y * grd.z);
  return cudaGetLastError();
}

cudaError_t launch_update_mixed(const Grid& g, double* x, const float* e, cudaStream_t st) {
  k_update_mixed<<<node_grid(g), dim3(32, 4), 0, st>>>(g, x, e); count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const Grid& gf, const Grid& gc, const Transfer& tr, const T* r,
                            T* fc, cudaStream_t st) {
  const dim3 grd = column_grid(gc), blk(32, 4);
  // 32-bit offsets within a level when both levels have fewer than 2^31 entries
  const bool small = gf.total < (int64_t)INT_MAX && gc.total < (int64_t)INT_MAX;
  if (small) {
    if (tr.hx && tr.hy) k_restrict<T, true, true, int><<<grd, blk, 0, st>>>(gf, gc, tr, r, fc);
    else if (tr.hx) k_restrict<T, true, false, int><<<grd, blk, 0, st>>>(gf, gc, tr, r, fc);
    else if (tr.hy) k_restrict<T, false, true, int><<<grd, blk, 0, st>>>(gf, gc, tr, r, fc);
    else k_restrict<T, false, false, int><<<grd, blk, 0, st>>>(gf, gc, tr, r, fc);
  } else {
    if (tr.hx && tr.hy) k_restrict<T, true, true, int64_t><<<grd, blk, 0, st>>>(gf, gc, tr, r, fc);
    else if (tr.hx) k_restrict<T, true, false, int64_t><<<grd, blk, 0, st>>>(gf, gc, tr, r, fc);
    else if (tr.hy) k_restrict<T, false, true, int64_t><<<grd, blk, 0, st>>>(gf, gc, tr, r, fc);
    else k_restrict<T, false, false, int64_t><<<grd, blk, 0, st>>>(gf, gc, tr, r, fc);
  }
  count_launches(1);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_prolong_add(const Grid& gf, const Grid& gc, const Transfer& tr, const T* ec,
                               T* x, cudaStream_t st) {
  const dim3 grd = column_grid(gf), blk(32, 4);
  const bool small = gf.total < (int64_t)INT_MAX && gc.total < (int64_t)INT_MAX;
  if (small) {
    if (tr.hx && tr.hy) k_prolong_add<T, true, true, int><<<grd, blk, 0, st>>>(gf, gc, tr, ec, x);
    else if (tr.hx) k_prolong_add<T, true, false, int><<<grd, blk, 0, st>>>(gf, gc, tr, ec, x);
    else if (tr.hy) k_prolong_add<T, false, true, int><<<grd, blk, 0, st>>>(gf, gc, tr, ec, x);
    else k_prolong_add<T, false, false, int><<<grd, blk, 0, st>>>(gf, gc, tr, ec, x);
  } else {
    if (tr.hx && tr.hy) k_prolong_add<T, true, true, int64_t><<<grd, blk, 0, st>>>(gf, gc, tr, ec, x);
    else if (tr.hx) k_prolong_add<T, true, false, int64_t><<<grd, blk, 0, st>>>(gf, gc, tr, ec, x);
    else if (tr.hy) k_prolong_add<T, false, true, int64_t><<<grd, blk, 0, st>>>(gf, gc, tr, ec, x);
    else k_prolong_add<T, false, false, int64_t><<<grd, blk, 0, st>>>(gf, gc, tr, ec, x);
  }
  count_launches(1);
  return cudaGetLastError();
}
template cudaError_t launch_restrict<double>(const Grid&, const Grid&, const Transfer&,
                                             const double*, double*, cudaStream_t);
template cudaError_t launch_restrict<float>(const Grid&, const Grid&, const Transfer&,
                                            const float*, float*, cudaStream_t);
template cudaError_t launch_prolong_add<double>(const Grid&, const Grid&, const Transfer&,
                                                const double*, double*, cudaStream_t);
template cudaError_t launch_prolong_add<float>(const Grid&, const Grid&, const Transfer&,
                                               const float*, float*, cudaStream_t);

}  // namespace mcw
