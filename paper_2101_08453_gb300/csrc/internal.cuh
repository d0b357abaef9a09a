// Internal declarations of the mcwind CUDA library (sm_103a).
//
// Node arrays inside the workspace use a parity-split row layout: in each
// row (fixed j, k) the even-i nodes come first, then the odd-i nodes, each
// half padded to a multiple of 16 elements:
//     idx(i, j, k) = k*PP + j*RP + (i & 1)*H + (i >> 1),   RP = 2H, PP = Ny*RP.
// The smoother updates one column group (i mod 2, j mod 2) at a time, so a
// warp over consecutive same-group columns reads the stencil planes with
// unit stride instead of stride 2.
//
// A level's operator holds 28 coefficients per node: s = (di+1) + 3(dj+1)
// + 9(dk+1) (s = 13 the diagonal) holds K_FF(n, n+d), s = 27 holds
// 1/K(n, n).  Rows and columns of fixed (Dirichlet) nodes are zero, so the
// coefficients are exactly the free block K_FF of Eq. 5.  Both the float64
// operator and its float32 copy are tiled: the 28 coefficients of 32
// consecutive nodes of a half row are one contiguous tile (coefficient s of
// node b at ((b >> 5) * 28 + s) * 32 + (b & 31); 7168 or 3584 bytes), so a
// warp stepping through a layer reads one contiguous block rather than 28
// separate streams.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/mcwind.h"

namespace mcw {

constexpr int kPlanes = 28;
constexpr int kDiag = 13;
constexpr int kInvDiag = 27;
constexpr int kMaxZ = 128;          // max node layers on any level
constexpr int kMaxCoarse = 4096;    // max free unknowns of the dense coarsest solve

// every kernel launch of the library is counted here (mcwind_launch_count)
void count_launches(int n);

struct Grid {
  int Nx, Ny, Nz;
  int H;          // half-row pitch (elements, a multiple of 32)
  int64_t RP;     // row pitch = 2H
  int64_t PP;     // layer pitch = Ny*RP
  int64_t total;  // Nz*PP
};

inline Grid make_grid(int Nx, int Ny, int Nz) {
  Grid g;
  g.Nx = Nx; g.Ny = Ny; g.Nz = Nz;
  int half = (Nx + 1) / 2;
  g.H = (half + 31) / 32 * 32;
  g.RP = 2 * (int64_t)g.H;
  g.PP = (int64_t)Ny * g.RP;
  g.total = (int64_t)Nz * g.PP;
  return g;
}

__host__ __device__ inline int64_t gidx(const Grid& g, int i, int j, int k) {
  return (int64_t)k * g.PP + (int64_t)j * g.RP + (int64_t)(i & 1) * g.H + (i >> 1);
}

// Operator storage, float64 and float32 alike: tiles of 32 consecutive
// split-layout nodes, each tile holding the kPlanes coefficients of its 32
// nodes plane after plane (32 values per plane), so one warp's rows are
// one contiguous block.  cidx = position of coefficient s of node b.
__host__ __device__ constexpr int64_t cidx(int64_t b, int s) {
  return ((b >> 5) * kPlanes + s) * 32 + (b & 31);
}
__device__ __forceinline__ double coef(const double* C, int64_t, int64_t b, int s) {
  return C[cidx(b, s)];
}
__device__ __forceinline__ float coef(const float* C, int64_t, int64_t b, int s) {
  return C[cidx(b, s)];
}

__host__ __device__ inline bool is_free(const Grid& g, int i, int j, int k) {
  return i >= 1 && i <= g.Nx - 2 && j >= 1 && j <= g.Ny - 2 && k >= 0 && k <= g.Nz - 2;
}

// Transfer between level l (fine) and l+1 (coarse), passed by value.
// Horizontal directions: coarse node I sits on fine node 2I, the last coarse
// node on the last fine node; odd fine nodes interpolate half/half from
// their two coarse neighbours (Sec. 3, the weights of trilinear
// interpolation on a regular grid).  Vertical: kf[K] = fine layer of coarse
// layer K (non-uniform after per-layer semicoarsening).
// V-cycles between two float64 convergence checks: the option, or its
// default (6 in mixed precision, 1 in float64)
inline int effective_cycles_per_check(const mcwind_options& o) {
  if (o.cycles_per_check > 0) return o.cycles_per_check;
  return o.precision == MCWIND_PREC_MIXED ? 6 : 1;
}

struct Transfer {
  int hx, hy;
  int Nzf, Nzc;
  int kf[kMaxZ];             // coarse K -> fine k
  int kc0[kMaxZ], kc1[kMaxZ];  // fine k -> coarse layers (kc1 = kc0 when one)
  float kw0[kMaxZ], kw1[kMaxZ];  // their weights (0, 1/2 or 1: exact in float)
};

// 1-D interpolation pair of a horizontal fine index f (Nf fine, Nc coarse
// nodes); the weights (0, 1/2, 1) are exact in any floating type W.
template <typename W>
__host__ __device__ inline void hpair(int coarsen, int Nf, int Nc, int f, int& c0, W& w0, int& c1,
                                      W& w1) {
  if (!coarsen) { c0 = c1 = f; w0 = W(1); w1 = W(0); return; }
  if (f == Nf - 1) { c0 = c1 = Nc - 1; w0 = W(1); w1 = W(0); return; }
  if ((f & 1) == 0) { c0 = c1 = f >> 1; w0 = W(1); w1 = W(0); return; }
  c0 = (f - 1) >> 1; c1 = (f + 1) >> 1; w0 = W(0.5); w1 = W(0.5);
  if (f + 1 == Nf - 1) c1 = Nc - 1;
}

// Fine node of horizontal coarse index I and the weights of its fine
// neighbours f-1 and f+1 in the restriction.
template <typename W>
__host__ __device__ inline void hcoarse(int coarsen, int Nf, int Nc, int I, int& f, W& wm, W& wp) {
  if (!coarsen) { f = I; wm = wp = W(0); return; }
  f = (I == Nc - 1) ? Nf - 1 : 2 * I;
  wm = (f >= 1 && ((f - 1) & 1)) ? W(0.5) : W(0);
  wp = (f + 1 <= Nf - 2 && ((f + 1) & 1)) ? W(0.5) : W(0);
}

// Separable (column x layer) operator of a shift-form grid (MCWIND_OP_SEPARABLE).
// On a terrain-following grid z = z_s(x, y) + zeta_k the element stiffness
// is (h/2) Phat (x) m - Qhat (x) g - Qhat^T (x) g^T + (2/h) Rhat (x) kappa,
// with Phat, Qhat, Rhat (4 x 4) depending on the column's terrain only and
// m, g, kappa the fixed 1-D matrices of a linear element, so every level's
// K_FF = sum_t H_t (x) V_t: four horizontal 9-point operators H_t over the
// node columns and four vertical tridiagonal V_t over the layers, a form
// the tensor-product Galerkin products of Eq. 7 keep.  Terms t: 0 = (H_P,
// V_M), 1 = (H_Q, V_G), 2 = (H_Q^T, V_G^T), 3 = (H_R, V_K).
//   horizontal factor q = 9 t + s2, s2 = (di+1) + 3 (dj+1): H_t(c, c + d) of
//     column c; float64 as plain planes H64[q * PP + col], float32 in tiles of
//     32 columns H32[hidx(col, q)];
//   vertical factor 3 t + (dk+1) of layer k: V_t(k, k + dk), V[k * kVF + ...].
// Couplings to fixed columns and to the top layer are zero.
constexpr int kHF = 36;
constexpr int kVF = 12;
__host__ __device__ constexpr int64_t hidx(int64_t col, int q) {
  return ((col >> 5) * kHF + q) * 32 + (col & 31);
}
// Load vector of Eq. 5 on a shift-form grid (2x2x2 Gauss, nodal u0):
//   f = -[(E_x (x) V_M) u_x + (E_y (x) V_M) u_y - (F_x (x) V_G^T) u_x
//         - (F_y (x) V_G^T) u_y + (M_z (x) V_G^T) u_z]
// with five horizontal 9-point factors per column (no coupling zeroed: f at a
// free node takes u0 at every node around it) kept as float pairs in tiles
// of 32 columns (term q = 9 t + s2, t = E_x, E_y, F_x, F_y, M_z), and per
// layer V_M(k, k-1..k+1), V_G^T(k, k-1..k+1) as float pairs.
constexpr int kRF = 45;
constexpr int kRV = 6;
__host__ __device__ constexpr int64_t ridx(int64_t col, int q) {
  return ((col >> 5) * kRF + q) * 32 + (col & 31);
}

struct Level {
  Grid g;
  int n_free;
  // device pointers into the workspace
  double* C64 = nullptr;   // kPlanes * g.total
  float* C32 = nullptr;
  // separable form: horizontal factors (shared with the finer level when the
  // transfer keeps the columns) and vertical factors
  double* H64 = nullptr;
  float* H32 = nullptr;
  double* V64 = nullptr;
  float* V32 = nullptr;
  float2* R2 = nullptr;      // finest level: load-vector factors (float pairs)
  float2* VR2 = nullptr;     // finest level: their vertical factors
  bool h_shared = false;
  bool has_c64 = true;     // false: separable form on an intermediate level
  // separable form: tensor maps of x32 and f32 as [Nz][Ny][2][H] float tiles
  // for the staged smoother (built at assembly, tied to the workspace)
  CUtensorMap tm_x, tm_f, tm_rx, tm_rf;
  CUtensorMap tm_u;   // finest level: u0 pairs, split layout, 3 components
  double *x64 = nullptr, *f64 = nullptr, *r64 = nullptr;
  float *x32 = nullptr, *f32 = nullptr, *r32 = nullptr;
  // host description of the transfer to the next level
  int hx = 0, hy = 0;
  std::vector<int> kmap;   // coarse layer -> fine layer
  Transfer tr{};
};

}  // namespace mcw

struct mcwind_plan_s {
  int nx, ny, nz;
  double a[3];
  mcwind_options opt;
  int gs_rows = 4;                          // smoother thread-block height (tunable)
  bool sep = false;                         // MCWIND_OP_SEPARABLE: float32 cycle on factors
  int status_host = 0;                      // last device status word read
  bool in_batch = false;
  std::vector<mcw::Level> lv;
  // workspace layout (byte offsets) and sizes
  size_t ws_bytes = 0;
  size_t off_tmp = 0, tmp_bytes = 0;        // RAP intermediates, layout conversion
  size_t off_dense = 0;                     // coarsest inverse n_c x n_c, plus scratch
  size_t off_partials = 0;                  // reduction partials
  size_t off_scalars = 0;                   // device scalars / flags
  size_t off_cfree = 0;                     // coarsest free-node grid indices
  size_t off_cg = 0;                        // 6 finest-level float64 vectors of CG
  size_t off_xyz2 = 0, off_u2 = 0;          // X, Y, Z and u0 as float pairs [3][nodes]
  size_t off_adj = 0;                       // adjoint reduction partials (6 per block) + sums
  int n_adj = 0;
  int n_coarse = 0;
  int n_partials = 0;
  // bound at assemble
  char* ws = nullptr;
  const double *X = nullptr, *Y = nullptr, *Z = nullptr;
  bool assembled = false;
  // profiler: event pairs recorded around kernel classes while enabled
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct ProfMark {
    int kind;
    int launches;
    size_t idx;  // start event; idx + 1 is the end event
  };
  std::vector<ProfMark> prof_marks;
  int prof_open = 0;
  double prof_ms[MCWIND_K_KINDS] = {0};
  long long prof_n[MCWIND_K_KINDS] = {0};
  // per-plan CUDA objects: one solver iteration captured as a graph
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t iter_exec = nullptr;
  const char* iter_ws = nullptr;     // workspace the graph was captured with
  long long iter_launches = 0;       // kernels in one replay
};
