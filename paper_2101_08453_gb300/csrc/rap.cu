// Galerkin coarse operator K_c = P^T K P (Eq. 7, second row).
//
// P is a tensor product P = Pz (x) Py (x) Px of 1-D interpolations, so
//   P^T K P = Pz^T (Py^T (Px^T K Px) Py) Pz
// and the product is formed one direction at a time.  Each stage maps a
// 27-point operator on one grid to a 27-point operator on a grid coarsened
// in one direction:
//   S'(I; D, e) = sum_{a} sum_{d} P(f_I + a, I) S(f_I + a; d, e) P(f_I + a + d, I + D)
// (a, d, D in {-1, 0, 1}; e the offsets in the other two directions,
// unchanged).  One thread computes the 27 entries of one output node from
// the 3 x 27 input entries it depends on.
#include "dfloat.cuh"
#include "kernels.cuh"

namespace mcw {
namespace {

__device__ __forceinline__ bool node_of_thread(const Grid& g, int& i, int& j, int& k) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  j = blockIdx.y * blockDim.y + threadIdx.y;
  k = blockIdx.z >> 1;
  i = 2 * h + (blockIdx.z & 1);
  return i < g.Nx && j < g.Ny;
}

template <int DIM>
__global__ void __launch_bounds__(128) k_rap(Grid gin, Grid gout, Transfer tr,
                                             const double* __restrict__ Sin,
                                             double* __restrict__ Sout) {
  int i, j, k;
  if (!node_of_thread(gout, i, j, k)) return;
  const int Iout = DIM == 0 ? i : (DIM == 1 ? j : k);
  const int Nf = DIM == 0 ? gin.Nx : (DIM == 1 ? gin.Ny : gin.Nz);
  const int Nc = DIM == 0 ? gout.Nx : (DIM == 1 ? gout.Ny : gout.Nz);
  // weights are 0, 1/2 or 1 (products 1/4): exact in float
  int f;
  float wa[3];
  if (DIM < 2) {
    hcoarse(1, Nf, Nc, Iout, f, wa[0], wa[2]);
  } else {
    f = tr.kf[Iout];
    wa[0] = (Iout > 0 && tr.kf[Iout] - tr.kf[Iout - 1] == 2) ? 0.5f : 0.0f;
    wa[2] = (Iout < tr.Nzc - 1 && tr.kf[Iout + 1] - tr.kf[Iout] == 2) ? 0.5f : 0.0f;
  }
  wa[1] = 1.0f;
  // Pw[q][D] = P(f + q - 2, Iout + D - 1)
  float Pw[5][3];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int b = f + q - 2;
    int c0 = -100, c1 = -100;
    float w0 = 0.0f, w1 = 0.0f;
    if (b >= 0 && b <= Nf - 1) {
      if (DIM < 2) {
        hpair(1, Nf, Nc, b, c0, w0, c1, w1);
      } else {
        c0 = tr.kc0[b]; c1 = tr.kc1[b]; w0 = tr.kw0[b]; w1 = tr.kw1[b];
      }
    }
#pragma unroll
    for (int D = 0; D < 3; ++D) {
      const int J = Iout + D - 1;
      Pw[q][D] = (c0 == J ? w0 : 0.0f) + (c1 == J && c1 != c0 ? w1 : 0.0f);
    }
  }
  // The sums run in float pairs: each input is split in integer arithmetic,
  // its products with the weights are exact, and only the additions round
  // (to about 2^-48 relative); the outputs are formed as doubles in integer
  // arithmetic.  No double-pipe instruction.
  dflt acc[27];
#pragma unroll
  for (int s = 0; s < 27; ++s) acc[s] = dflt{0.0f, 0.0f};
  // Away from the ends of the direction the weights take one fixed pattern:
  // wa = (1/2, 1, 1/2) and Pw[q] = e_0, (e_0 + e_1)/2, e_1, (e_1 + e_2)/2, e_2.
  // There the products wa[a] Pw[a + d][D] are constants and only their 13
  // nonzero terms (per pair of offsets in the other two directions) are
  // formed; the general form below adds 3 weighted terms per input value.
  // Both add the same exact products (powers of two times S) in the same
  // order, zero terms aside.
  constexpr float kWa[3] = {0.5f, 1.0f, 0.5f};
  constexpr float kPw[5][3] = {{1.0f, 0.0f, 0.0f}, {0.5f, 0.5f, 0.0f}, {0.0f, 1.0f, 0.0f},
                               {0.0f, 0.5f, 0.5f}, {0.0f, 0.0f, 1.0f}};
  bool regular = wa[0] == 0.5f && wa[2] == 0.5f;
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int D = 0; D < 3; ++D) regular = regular && Pw[q][D] == kPw[q][D];
  if (regular) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ii = DIM == 0 ? f + a - 1 : i;
      const int jj = DIM == 1 ? f + a - 1 : j;
      const int kk = DIM == 2 ? f + a - 1 : k;
      const int64_t in = gidx(gin, ii, jj, kk);
      double raw[27];
#pragma unroll
      for (int s = 0; s < 27; ++s) raw[s] = Sin[cidx(in, s)];
#pragma unroll
      for (int s = 0; s < 27; ++s) {
        const int di = s % 3, dj = (s / 3) % 3, dk = s / 9;
        const int d = DIM == 0 ? di : (DIM == 1 ? dj : dk);
        const float2 v = split_bits(raw[s]);
#pragma unroll
        for (int D = 0; D < 3; ++D) {
          const float w = kWa[a] * kPw[a + d][D];
          if (w == 0.0f) continue;
          const int so = DIM == 0 ? D + 3 * dj + 9 * dk
                                  : (DIM == 1 ? di + 3 * D + 9 * dk : di + 3 * dj + 9 * D);
          acc[so] = acc[so] + dflt{v.x * w, v.y * w};
        }
      }
    }
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (wa[a] == 0.0f) continue;
      const int ii = DIM == 0 ? f + a - 1 : i;
      const int jj = DIM == 1 ? f + a - 1 : j;
      const int kk = DIM == 2 ? f + a - 1 : k;
      const int64_t in = gidx(gin, ii, jj, kk);
#pragma unroll
      for (int s = 0; s < 27; ++s) {
        const int di = s % 3, dj = (s / 3) % 3, dk = s / 9;  // 0..2
        const int d = DIM == 0 ? di : (DIM == 1 ? dj : dk);
        const float2 v = split_bits(Sin[cidx(in, s)]);
#pragma unroll
        for (int D = 0; D < 3; ++D) {
          const float w = wa[a] * Pw[a + d][D];
          const int so = DIM == 0 ? D + 3 * dj + 9 * dk
                                  : (DIM == 1 ? di + 3 * D + 9 * dk : di + 3 * dj + 9 * D);
          if (w != 0.0f) acc[so] = acc[so] + dflt{v.x * w, v.y * w};
        }
      }
    }
  }
  const int64_t o = gidx(gout, i, j, k);
#pragma unroll
  for (int s = 0; s < 27; ++s) Sout[cidx(o, s)] = pair_to_double(acc[s].hi, acc[s].lo);
}

}  // namespace

cudaError_t launch_rap_stage(int dim, const Grid& gin, const Grid& gout, const Transfer& tr,
                             const double* Sin, double* Sout, cudaStream_t st) {
  dim3 grd((gout.H + 31) / 32, (gout.Ny + 3) / 4, 2 * gout.Nz);
  dim3 blk(32, 4);
  if (dim == 0) k_rap<0><<<grd, blk, 0, st>>>(gin, gout, tr, Sin, Sout);
  else if (dim == 1) k_rap<1><<<grd, blk, 0, st>>>(gin, gout, tr, Sin, Sout);
  else k_rap<2><<<grd, blk, 0, st>>>(gin, gout, tr, Sin, Sout);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mcw
