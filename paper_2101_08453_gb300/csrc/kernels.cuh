// Launch wrappers of the mcwind kernels (each returns the launch status).
#pragma once
#include "internal.cuh"

namespace mcw {

// ---- element.cu: isoparametric trilinear hexahedra (Sec. 2) ----
// Stiffness (Eq. 5 left side, 2x2x2 Gauss) scattered into the 28-plane
// stencil of level 0 (planes must be zero on entry); flag |= 1 on detJ <= 0.
// dfloat: element arithmetic in float pairs (FP32 pipe) instead of double.
// xyz2: X, Y, Z split into (hi, lo) float pairs, [3][nodes] (read when dfloat)
cudaError_t launch_assemble_stencil(const Grid& g, int nx, int ny, int nz, const double* X,
                                    const double* Y, const double* Z, const float2* xyz2,
                                    const double* a, double* C, int* flag, int dfloat,
                                    cudaStream_t st);
// float64 -> (hi, lo) float pairs
cudaError_t launch_split_pairs(const double* a, float2* b, int64_t n, cudaStream_t st);
// Load vector (Eq. 5 right side) into f (split layout, zero on entry).
// quad bit 0: one-point center rule; bit 1: u0 given at the element centers
// ([3][nz][ny][nx]) instead of at the nodes.
// u2: nodal u0 split into float pairs (read when dfloat with nodal u0)
cudaError_t launch_assemble_rhs(const Grid& g, int nx, int ny, int nz, const double* X,
                                const double* Y, const double* Z, const float2* xyz2,
                                const double* u0, const float2* u2, int quad, double* f,
                                int dfloat, cudaStream_t st);
// u = u0 + A^{-1} grad lambda (Eq. 3); lambda in split layout.
cudaError_t launch_recover(const Grid& g, int nx, int ny, int nz, const double* X,
                           const double* Y, const double* Z, const double* u0,
                           const double* lam, const double* a, int where, int u0_centers,
                           double* u, cudaStream_t st);
// recovery at the element centers in float pairs (xyz2, u2, lam2 pre-split in
// the [k][j][i] layout; u0c != nullptr: u0 given at the centers instead of u2)
// u at the element centers of a shift-form grid (Eq. 3) from the column's
// center Jacobian and each layer's thickness, in float pairs; u0 nodal
// [3][N] or, with u0 = nullptr, u0c at the centers [3][NE]
cudaError_t launch_recover_center_sep(int nx, int ny, int nz, const double* X, const double* Y,
                                      const double* Z, const double* u0, const double* u0c,
                                      const double* lam, const double* a, double* u,
                                      cudaStream_t st);
cudaError_t launch_recover_center_df(int nx, int ny, int nz, const float2* xyz2, const float2* u2,
                                     const double* u0c, const float2* lam2, const double* a,
                                     double* u, cudaStream_t st);
// adjoint of the recovery at element centers: h += G^T A^{-1} gu, du0 += C^T gu
// (standard layouts, zero on entry)
cudaError_t launch_recover_adjoint(int nx, int ny, int nz, const double* X, const double* Y,
                                   const double* Z, const double* gu, const double* a, double* h,
                                   double* du0, cudaStream_t st);
// du0 -= I^T B^T mu; sums6 = (E_0..2, T_0..2) over all elements (partials: 6 per
// block, adjoint_partials(nx, ny, nz) blocks, refused above cap blocks)
int adjoint_partials(int nx, int ny, int nz);
cudaError_t launch_adjoint_finish(int nx, int ny, int nz, const double* X, const double* Y,
                                  const double* Z, const double* mu, const double* lam,
                                  const double* gu, double* du0, double* partials, int cap,
                                  double* sums6, cudaStream_t st);
// (B u)_m at every node, out in standard layout, zero on entry.
cudaError_t launch_weak_div(int nx, int ny, int nz, const double* X, const double* Y,
                            const double* Z, const double* ug, double* out, cudaStream_t st);

// ---- layout.cu ----
template <typename T>
cudaError_t launch_std_to_split(const Grid& g, const double* src, T* dst, bool zero_fixed,
                                cudaStream_t st);
template <typename T>
cudaError_t launch_split_to_std(const Grid& g, const T* src, double* dst, cudaStream_t st);
// planes of the split layout -> [27][Nz][Ny][Nx] standard layout (float64)
template <typename T>
cudaError_t launch_stencil_export(const Grid& g, const T* C, double* out, cudaStream_t st);
cudaError_t launch_stencil_to_f32(const Grid& g, const double* C64, float* C32, cudaStream_t st);
// zero couplings to fixed nodes, rows of fixed nodes, set plane 27 = 1/diag;
// flag |= 2 if a free diagonal is not positive.
cudaError_t launch_stencil_finalize(const Grid& g, double* C, int* flag, cudaStream_t st);
// sum of n partials in fixed order -> *out
cudaError_t launch_reduce_final(const double* partials, int n, double* out, cudaStream_t st);
// sum over free nodes of v^2 (split layout) -> residual_blocks(g) partials
// (refuses to launch when that exceeds cap); block count via *nblocks
cudaError_t launch_norm2_partials(const Grid& g, const double* v, double* partials, int cap,
                                  int* nblocks, cudaStream_t st);

// ---- smooth.cu: vertical Gauss-Seidel, one column group (Sec. 3) ----
// rows: column rows per thread block (blockDim = 32 x rows, rows in 1..8)
// first group of a forward sweep on x = 0: writes every entry of x
template <typename T>
cudaError_t launch_gs_zero_start(const Grid& g, const T* C, const T* f, T* x, int group,
                                 cudaStream_t st);
template <typename T>
cudaError_t launch_gs_group(const Grid& g, const T* C, const T* f, T* x, int group, int up,
                            int rows, cudaStream_t st);

// ---- transfer.cu ----
// r = f - K x at free nodes (0 elsewhere); partials of sum r^2 if partials != nullptr
// (residual_blocks(g) of them; refuses to launch when that exceeds cap)
template <typename T>
cudaError_t launch_residual(const Grid& g, const T* C, const T* f, const T* x, T* r,
                            double* partials, int cap, int* nblocks, cudaStream_t st);
// mixed refinement: r64 = f - K64 x64; r32 = (float) r64; e32 = 0; partials of r64^2
cudaError_t launch_residual_mixed(const Grid& g, const double* C, const double* f,
                                  const double* x, float* r32, float* e32, double* partials,
                                  int cap, int* nblocks, cudaStream_t st);
// y = K x at free nodes (0 elsewhere), partials of x . K x (float64)
cudaError_t launch_apply(const Grid& g, const double* C, const double* x, double* y,
                         double* partials, int cap, int* nblocks, cudaStream_t st);
// x64 += e32 at free nodes
cudaError_t launch_update_mixed(const Grid& g, double* x, const float* e, cudaStream_t st);
template <typename T>
cudaError_t launch_restrict(const Grid& gf, const Grid& gc, const Transfer& tr, const T* r,
                            T* fc, cudaStream_t st);
template <typename T>
cudaError_t launch_prolong_add(const Grid& gf, const Grid& gc, const Transfer& tr, const T* ec,
                               T* x, cudaStream_t st);
int residual_blocks(const Grid& g);

// ---- rap.cu: K_c = P^T K P one direction at a time (Eq. 7) ----
// dim 0/1: horizontal coarsening of x/y; dim 2: vertical with tr's layer map.
cudaError_t launch_rap_stage(int dim, const Grid& gin, const Grid& gout, const Transfer& tr,
                             const double* Sin, double* Sout, cudaStream_t st);

// ---- coarse.cu: dense direct solve on the coarsest level ----
cudaError_t launch_coarse_index(const Grid& g, int* cfree, cudaStream_t st);
cudaError_t launch_dense_gather(const Grid& g, const double* C, const int* cfree, int n,
                                double* A, cudaStream_t st);
// Gauss-Jordan inversion in place in A (blocks of 16 pivots, B holds the
// step's panels: 256 + 32 n doubles); *result = A
cudaError_t launch_dense_invert(double* A, double* B, int n, double** result, cudaStream_t st);
template <typename T>
cudaError_t launch_dense_solve(const double* Ainv, int n, const int* cfree, const T* f, T* x,
                               cudaStream_t st);

// ---- krylov.cu: V-cycle-preconditioned conjugate gradients ----
// device scalars s[0..5] = (r.z, r_prev.z, previous r.z, beta, p.Kp, restart flag)
int krylov_blocks(const Grid& g);
template <typename TZ>
cudaError_t launch_cg_dots(const Grid& g, const double* r, const double* rp, const TZ* z,
                           double* partials, int cap, double* s, cudaStream_t st);
template <typename TZ>
cudaError_t launch_cg_direction(const Grid& g, const TZ* z, double* p, double* s,
                                cudaStream_t st);
template <typename TP>
cudaError_t launch_cg_update(const Grid& g, double* x, double* r, double* rp, const double* p,
                             const double* q, TP* pf, TP* px, double* s, double* partials,
                             int cap, double* rr_out, cudaStream_t st);
template <typename TP>
cudaError_t launch_cg_start(const Grid& g, const double* r, double* rp, TP* pf, TP* px, double* s,
                            cudaStream_t st);
cudaError_t launch_reduce_pairs(const double* partials, int n, double* out0, double* out1,
                                cudaStream_t st);

// ---- separable.cu: column x layer operator of a shift-form grid ----
// flag |= 8 when X, Y depend on k or Z - Z(.,.,0) differs between columns
cudaError_t launch_shift_check(int Nx, int Ny, int Nz, const double* X, const double* Y,
                               const double* Z, int* flag, cudaStream_t st);
// finest horizontal factors from the ground layer of X, Y, Z (standard
// layout), fixed couplings zeroed, float32 tiles written; flag |= 1 on j2 <= 0
// pairs: the cell sums in float pairs (else float64)
cudaError_t launch_hfactors(const Grid& g, const double* X, const double* Y, const double* Z,
                            const double* a, double* H64, float* H32, int* flag, bool pairs,
                            cudaStream_t st);
cudaError_t launch_hfactor_finalize(const Grid& g, double* H64, float* H32, cudaStream_t st);
// one direction (0: x, 1: y) of Ph^T H Ph for the 4 terms (float64)
cudaError_t launch_hgalerkin(int dim, const Grid& gin, const Grid& gout, const double* Hin,
                             double* Hout, cudaStream_t st);
// finest vertical factors from column (0, 0) of Z; Galerkin to the next level
cudaError_t launch_vfactor0(int Nx, int Ny, int Nz, const double* Z, double* V64, float* V32,
                            float2* VR2, int* flag, cudaStream_t st);
// ---- sep_rhs.cu: the load vector of Eq. 5 from column x layer factors ----
cudaError_t launch_rhs_factors(const Grid& g, const double* X, const double* Y, const double* Z,
                               float2* R2, cudaStream_t st);
cudaError_t make_u0_map(Level& L, float2* u2);
// u0 -> float pairs in the split layout (u2, 3 x g.total), then f (split layout,
// float64, 0 at fixed nodes)
cudaError_t launch_rhs_sep(const Level& L, const float2* R2, const float2* VR2, const double* u0,
                           float2* u2, double* f, int* status, cudaStream_t st);
cudaError_t launch_vgalerkin(const Transfer& tr, const double* Vf, double* Vc, float* Vc32,
                             cudaStream_t st);
// 27-point rows from float64 factors into a tiled float64 operator, planes
// 0..26 and 27 = 1/diag (flag |= 2 on a free diagonal that is not positive)
cudaError_t launch_sep_expand64(const Grid& g, const double* H64, const double* V64, double* C,
                                int* flag, bool pairs, cudaStream_t st);
// rows from the factors in the standard layout [27][N] (T = double: float64
// planes; T = float: float32 tiles)
template <typename T>
cudaError_t launch_sep_export(const Grid& g, const T* H, const T* V, double* out, cudaStream_t st);
// float32 cycle on the factors (x and f staged by TMA from the level's
// tensor maps; a wait that runs out sets bit 1 of *status): one Gauss-Seidel
// column group; the first group of a forward sweep from x = 0; r = f - K x,
// or (fuse: the level's transfer keeps the columns) f_c = P^T (f - K x) on
// the coarse grid.  make_tile_maps builds the maps of a level's x32 and f32.
cudaError_t launch_gs_sep_staged(const Level& L, const float* H32, const float* V32, float* x,
                                 int group, int up, int* status, cudaStream_t st);
cudaError_t launch_gs_sep_zero_start(const Grid& g, const float* H32, const float* V32,
                                     const float* f, float* x, int group, cudaStream_t st);
cudaError_t launch_residual_sep_staged(const Level& L, bool fuse, const float* H32,
                                       const float* V32, float* out, int* status,
                                       cudaStream_t st);
cudaError_t make_tile_maps(Level& L, float* x32, float* f32);

// ---- batch.cu: device bookkeeping of the batched solve (one graph) ----
struct BatchDev {
  int n;
  const double* const* scal;               // per domain: the plan's scalars (0: |f|^2, 1: |r|^2)
  const int* const* pstat;                 // per domain: the plan's status word
  const cudaGraphConditionalHandle* h_if;  // per domain: IF handle of its iteration
  cudaGraphConditionalHandle h_while;      // the solve loop
  int* iter;                               // checks done
  int *active, *cycles, *status, *nonfinite;
  double* nf;                              // ||f_F|| per domain
  double* hist;                            // [n][MCWIND_HIST] relative residual at the checks
};
// a bounded wait that nothing completes (sets the status bit after limit_ns)
cudaError_t launch_wait_selftest(int* status, unsigned long long limit_ns, cudaStream_t st);
// phase 0: after the set-up (first residuals); phase 1: after one iteration
cudaError_t launch_batch_step(const BatchDev& b, int phase, double rtol, int max_checks, int cpc,
                              cudaStream_t st);

}  // namespace mcw
