// C entry points and the solve driver.
#include <cmath>
#include <cstring>
#include <map>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "kernels.cuh"

using namespace mcw;

namespace {

thread_local int g_last_cuda = 0;

#define CK(expr)                                      \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) {                          \
      g_last_cuda = (int)e_;                          \
      return MCWIND_ECUDA;                            \
    }                                                 \
  } while (0)

#define CKR(expr)                                     \
  do {                                                \
    int r_ = (expr);                                  \
    if (r_ != MCWIND_OK) return r_;                   \
  } while (0)

long long launches_now() { return mcwind_launch_count(); }

// quadrature and u0 location of the load vector, as the element kernel takes them
int rhs_mode(mcwind_plan p) { return (p->opt.rhs_quad & 1) | (p->opt.u0_at ? 2 : 0); }

bool dfloat_elements(mcwind_plan p) { return p->opt.element_arith == MCWIND_ARITH_DFLOAT; }
size_t std_nodes(mcwind_plan p) { return (size_t)(p->nx + 1) * (p->ny + 1) * (p->nz + 1); }

// the separable load vector: separable plan, 2x2x2 Gauss with nodal u0,
// float-pair element arithmetic (MCWIND_ARITH_F64 keeps the element kernel)
bool sep_rhs(mcwind_plan p) {
  return p->sep && dfloat_elements(p) && rhs_mode(p) == 0;
}

int* statusp(mcwind_plan p);

// f (split layout, level 0) = load vector of Eq. 5 from u0
cudaError_t rhs_into(mcwind_plan p, const double* u0, double* f, cudaStream_t st) {
  const Level& L0 = p->lv[0];
  if (sep_rhs(p))
    return launch_rhs_sep(L0, (const float2*)(p->ws + (size_t)L0.R2),
                          (const float2*)(p->ws + (size_t)L0.VR2), u0,
                          (float2*)(p->ws + p->off_u2), f, statusp(p), st);
  const float2* xyz2 = (const float2*)(p->ws + p->off_xyz2);
  float2* u2 = (float2*)(p->ws + p->off_u2);
  const bool df = dfloat_elements(p);
  cudaError_t e = cudaMemsetAsync(f, 0, sizeof(double) * (size_t)L0.g.total, st);
  if (e == cudaSuccess && df && p->opt.u0_at == MCWIND_U0_NODES && (p->opt.rhs_quad & 1) == 0)
    e = launch_split_pairs(u0, u2, 3 * (int64_t)std_nodes(p), st);
  if (e == cudaSuccess)
    e = launch_assemble_rhs(L0.g, p->nx, p->ny, p->nz, p->X, p->Y, p->Z, xyz2, u0, u2,
                            rhs_mode(p), f, df, st);
  return e;
}

// NVTX range names of the kernel classes (the order of the MCWIND_K_* kinds)
const char* const kKindRange[MCWIND_K_KINDS] = {
    "mcwind:assemble",      "mcwind:rap",           "mcwind:setup",
    "mcwind:rhs",           "mcwind:outer_residual", "mcwind:smooth_fine",
    "mcwind:smooth_coarse", "mcwind:residual_fine",  "mcwind:residual_coarse",
    "mcwind:restrict",      "mcwind:prolong",        "mcwind:coarse_solve",
    "mcwind:update",        "mcwind:recover",        "mcwind:krylov",
    "mcwind:other"};

// Around a kernel class: an NVTX range on the host thread (always; a
// profiler can select launches by it, e.g. ncu --nvtx-include
// "mcwind:smooth_fine/"), and, while profiling is on, a CUDA event pair.
// A scope reserves its two events when it opens; finished pairs are folded
// into the per-class totals whenever the stream is idle, and the event pool
// is recycled only when no scope is open.
struct ProfScope {
  mcwind_plan p;
  int kind;
  cudaStream_t st;
  long long n0 = 0;
  size_t idx = 0;
  bool on = false;
  ProfScope(mcwind_plan p_, int kind_, cudaStream_t st_) : p(p_), kind(kind_), st(st_) {
    nvtxRangePushA(kKindRange[kind]);
    if (!p->prof) return;
    while (p->ev_used + 2 > p->ev_pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      p->ev_pool.push_back(e);
    }
    idx = p->ev_used;
    if (cudaEventRecord(p->ev_pool[idx], st) != cudaSuccess) return;
    p->ev_used += 2;
    p->prof_open += 1;
    on = true;
    n0 = launches_now();
  }
  ~ProfScope() {
    nvtxRangePop();
    if (!on) return;
    cudaEventRecord(p->ev_pool[idx + 1], st);
    p->prof_open -= 1;
    p->prof_marks.push_back({kind, (int)(launches_now() - n0), idx});
  }
};

// fold finished event pairs into the per-class totals (stream must be idle)
void prof_fold(mcwind_plan p) {
  for (const auto& mk : p->prof_marks) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p->ev_pool[mk.idx], p->ev_pool[mk.idx + 1]) == cudaSuccess)
      p->prof_ms[mk.kind] += ms;
    p->prof_n[mk.kind] += mk.launches;
  }
  p->prof_marks.clear();
  if (p->prof_open == 0) p->ev_used = 0;
}

#define PROF_CAT2(a, b) a##b
#define PROF_CAT(a, b) PROF_CAT2(a, b)
#define PROF(kind) ProfScope PROF_CAT(prof_scope_, __LINE__)(p, (kind), st)

template <typename P>
P* at(mcwind_plan p, P* offset) {
  return (P*)(p->ws + (size_t)offset);
}

double* scal(mcwind_plan p) { return (double*)(p->ws + p->off_scalars); }
int* flagp(mcwind_plan p) { return (int*)(p->ws + p->off_scalars + 128); }
// device status word: bits set by kernels whose bounded waits ran out
int* statusp(mcwind_plan p) { return (int*)(p->ws + p->off_scalars + 132); }
double* partials(mcwind_plan p) { return (double*)(p->ws + p->off_partials); }
int* cfree(mcwind_plan p) { return (int*)(p->ws + p->off_cfree); }

struct Ptr64 {
  double *C, *x, *f, *r;
};
struct Ptr32 {
  float *C, *x, *f, *r;
};

Ptr64 lv64(mcwind_plan p, int l) {
  Level& L = p->lv[l];
  return {at(p, L.C64), at(p, L.x64), at(p, L.f64), at(p, L.r64)};
}
Ptr32 lv32(mcwind_plan p, int l) {
  Level& L = p->lv[l];
  return {at(p, L.C32), at(p, L.x32), at(p, L.f32), at(p, L.r32)};
}

template <typename T>
struct Sel;
template <>
struct Sel<double> {
  static Ptr64 get(mcwind_plan p, int l) { return lv64(p, l); }
};
template <>
struct Sel<float> {
  static Ptr32 get(mcwind_plan p, int l) { return lv32(p, l); }
};

// separable float32 factors of level l
const float* sep_h32(mcwind_plan p, int l) { return at(p, p->lv[l].H32); }
const float* sep_v32(mcwind_plan p, int l) { return at(p, p->lv[l].V32); }

template <typename T>
constexpr bool is_f32() { return sizeof(T) == 4; }

double* dense_inv(mcwind_plan p) {
  // the blocked Gauss-Jordan inverts in place, in the first buffer
  return (double*)(p->ws + p->off_dense);
}

// sweeps of the column Gauss-Seidel smoother on level l; zero_start: x is 0
// on entry (or, for a forward sweep, need not be zeroed: the first group
// writes all of x)
template <typename T>
int smooth(mcwind_plan p, int l, int sweeps, int direction, cudaStream_t st,
           bool zero_start = false) {
  auto P = Sel<T>::get(p, l);
  const Grid& g = p->lv[l].g;
  PROF(l == 0 ? MCWIND_K_SMOOTH_FINE : MCWIND_K_SMOOTH_COARSE);
  const bool sep = is_f32<T>() && p->sep;
  for (int s = 0; s < sweeps; ++s)
    for (int q = 0; q < 4; ++q) {
      const int grp = direction == MCWIND_FORWARD ? q : 3 - q;
      const int up = direction == MCWIND_FORWARD ? 1 : 0;
      const bool first = s == 0 && q == 0 && zero_start && direction == MCWIND_FORWARD;
      if (sep) {
        const float* H = sep_h32(p, l);
        const float* V = sep_v32(p, l);
        if (first)
          CK(launch_gs_sep_zero_start(g, H, V, (const float*)P.f, (float*)P.x, grp, st));
        else
          CK(launch_gs_sep_staged(p->lv[l], H, V, (float*)P.x, grp, up, statusp(p), st));
      } else if (first) {
        CK(launch_gs_zero_start<T>(g, P.C, P.f, P.x, grp, st));
      } else {
        CK(launch_gs_group<T>(g, P.C, P.f, P.x, grp, up, p->gs_rows, st));
      }
    }
  return MCWIND_OK;
}

// f_c = P^T (f - K x) from level l to l+1 in the cycle's precision: the
// separable float32 operator fuses the two when the transfer keeps the
// columns (no residual stored), else r is formed and restricted.
template <typename T>
int residual_restrict(mcwind_plan p, int l, cudaStream_t st) {
  Level& L = p->lv[l];
  auto P = Sel<T>::get(p, l);
  auto Q = Sel<T>::get(p, l + 1);
  if (is_f32<T>() && p->sep) {
    const bool fuse = !L.hx && !L.hy;
    {
      PROF(l == 0 ? MCWIND_K_RESIDUAL_FINE : MCWIND_K_RESIDUAL_COARSE);
      CK(launch_residual_sep_staged(L, fuse, sep_h32(p, l), sep_v32(p, l),
                                    fuse ? (float*)Q.f : (float*)P.r, statusp(p), st));
    }
    if (fuse) return MCWIND_OK;
  } else {
    PROF(l == 0 ? MCWIND_K_RESIDUAL_FINE : MCWIND_K_RESIDUAL_COARSE);
    CK(launch_residual<T>(L.g, P.C, P.f, P.x, P.r, nullptr, 0, nullptr, st));
  }
  PROF(MCWIND_K_RESTRICT);
  CK(launch_restrict<T>(L.g, p->lv[l + 1].g, L.tr, P.r, Q.f, st));
  return MCWIND_OK;
}

// one V-cycle from level l down; x_zero: the level-0 x is 0 on entry (the
// coarser levels always start from 0)
template <typename T>
int vcycle(mcwind_plan p, int l, cudaStream_t st, bool x_zero = false) {
  const int last = (int)p->lv.size() - 1;
  auto P = Sel<T>::get(p, l);
  Level& L = p->lv[l];
  if (l == last) {
    PROF(MCWIND_K_COARSE_SOLVE);
    CK(launch_dense_solve<T>(dense_inv(p), p->n_coarse, cfree(p), P.f, P.x, st));
    return MCWIND_OK;
  }
  const bool zs = (l > 0 || x_zero) && p->opt.nu_pre >= 1;
  if (l > 0 && !zs) CK(cudaMemsetAsync(P.x, 0, sizeof(T) * (size_t)L.g.total, st));
  CKR(smooth<T>(p, l, p->opt.nu_pre, MCWIND_FORWARD, st, zs));
  CKR(residual_restrict<T>(p, l, st));
  auto Q = Sel<T>::get(p, l + 1);
  CKR(vcycle<T>(p, l + 1, st, true));
  {
    PROF(MCWIND_K_PROLONG);
    CK(launch_prolong_add<T>(L.g, p->lv[l + 1].g, L.tr, Q.x, P.x, st));
  }
  CKR(smooth<T>(p, l, p->opt.nu_post, p->opt.post_reverse ? MCWIND_BACKWARD : MCWIND_FORWARD, st));
  return MCWIND_OK;
}

// op64: the call applies the level's float64 operator (absent on the
// intermediate levels of the separable form)
int check_level(mcwind_plan p, int level, int precision, bool op64 = false) {
  if (!p) return MCWIND_EINVAL;
  if (!p->assembled) return MCWIND_ESTATE;
  if (level < 0 || level >= (int)p->lv.size()) return MCWIND_EINVAL;
  if (precision != MCWIND_PREC_F64 && precision != MCWIND_PREC_MIXED) return MCWIND_EINVAL;
  if (precision == MCWIND_PREC_MIXED && p->opt.precision != MCWIND_PREC_MIXED) return MCWIND_EINVAL;
  if (op64 && precision == MCWIND_PREC_F64 && !p->lv[level].has_c64) return MCWIND_EINVAL;
  return MCWIND_OK;
}

// ||v_F||^2 of a float64 split-layout vector into scal[slot]
int norm2(mcwind_plan p, const Grid& g, const double* v, int slot, cudaStream_t st) {
  PROF(MCWIND_K_OTHER);
  int nb = 0;
  CK(launch_norm2_partials(g, v, partials(p), p->n_partials, &nb, st));
  CK(launch_reduce_final(partials(p), nb, scal(p) + slot, st));
  return MCWIND_OK;
}

// residual of the outer float64 iteration on level 0 and its squared norm in scal[1];
// in mixed mode also the float32 right side and a zero start of the correction.
// x_zero: the iterate is known to be 0 (a cold start), so r = f without a
// product (the same values and norm as the full residual).
int outer_residual(mcwind_plan p, cudaStream_t st, bool x_zero = false) {
  Ptr64 A = lv64(p, 0);
  const Grid& g = p->lv[0].g;
  const double* x = x_zero ? nullptr : A.x;
  int nb = 0;
  {
    PROF(MCWIND_K_OUTER_RESIDUAL);
    if (p->opt.precision == MCWIND_PREC_F64) {
      CK(launch_residual<double>(g, A.C, A.f, x, A.r, partials(p), p->n_partials, &nb, st));
    } else {
      Ptr32 B = lv32(p, 0);
      CK(launch_residual_mixed(g, A.C, A.f, x, B.f, B.x, partials(p), p->n_partials, &nb, st));
    }
  }
  PROF(MCWIND_K_OTHER);
  CK(launch_reduce_final(partials(p), nb, scal(p) + 1, st));
  return MCWIND_OK;
}

// V-cycles between two convergence checks (the option, or its default)
int check_every(mcwind_plan p) { return effective_cycles_per_check(p->opt); }

// n V-cycles, then the float64 residual and its norm (one check).  Mixed
// precision: the cycles iterate on the float32 correction (the first from
// the zero the outer residual left), then x += e once.
int iteration(mcwind_plan p, cudaStream_t st, int n) {
  if (p->opt.precision == MCWIND_PREC_F64) {
    for (int q = 0; q < n; ++q) CKR(vcycle<double>(p, 0, st));
  } else {
    for (int q = 0; q < n; ++q) CKR(vcycle<float>(p, 0, st, q == 0));
    PROF(MCWIND_K_UPDATE);
    CK(launch_update_mixed(p->lv[0].g, lv64(p, 0).x, lv32(p, 0).x, st));
  }
  return outer_residual(p, st);
}

// res_hist entries c0+1 .. c1-1 between two checks: geometric interpolation
void fill_between(double* h, int c0, int c1) {
  for (int q = c0 + 1; q < c1; ++q)
    h[q] = (h[c0] > 0.0 && h[c1] > 0.0)
               ? h[c0] * std::pow(h[c1] / h[c0], (double)(q - c0) / (c1 - c0))
               : h[c1];
}

// Run one solver iteration (body(p, stream)) on st: replayed from a graph
// captured once per plan and workspace, or launched directly while profiling
// or when graphs are off.
template <typename Body>
int run_iteration(mcwind_plan p, cudaStream_t st, Body body) {
  if (p->prof || !p->opt.use_graphs) return body(p, st);
  if (!p->iter_exec || p->iter_ws != p->ws) {
    if (p->iter_exec) { cudaGraphExecDestroy(p->iter_exec); p->iter_exec = nullptr; }
    if (!p->cap_stream) CK(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    const long long n0 = mcwind_launch_count();
    const int rc = body(p, p->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p->cap_stream, &graph);
    if (rc != MCWIND_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    CK(e);
    const cudaError_t ei = cudaGraphInstantiate(&p->iter_exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ei);
    p->iter_ws = p->ws;
    p->iter_launches = mcwind_launch_count() - n0;
    count_launches(-(int)p->iter_launches);  // captured, not run: counted at replay
  }
  CK(cudaGraphLaunch(p->iter_exec, st));
  count_launches((int)p->iter_launches);
  return MCWIND_OK;
}

// copy device scalars [first, first + n) to host (synchronizes the stream);
// ETIMEOUT when a kernel's bounded wait has run out since the last assembly
int read_scalars(mcwind_plan p, double* host, int first, int n, cudaStream_t st) {
  CK(cudaMemcpyAsync(host, scal(p) + first, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&p->status_host, statusp(p), sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (p->prof) prof_fold(p);
  if (p->status_host != 0) return MCWIND_ETIMEOUT;
  return MCWIND_OK;
}

}  // namespace

extern "C" int mcwind_last_cuda_error(void) { return g_last_cuda; }

extern "C" const char* mcwind_strerror(int code) {
  switch (code) {
    case MCWIND_OK: return "ok";
    case MCWIND_EINVAL: return "invalid argument";
    case MCWIND_EGEOM: return "inverted or degenerate element (detJ <= 0)";
    case MCWIND_ENONFINITE: return "non-finite input wind";
    case MCWIND_ENOTCONV: return "not converged within max_cycles";
    case MCWIND_ECUDA: return "CUDA error";
    case MCWIND_ESTATE: return "plan not assembled";
    case MCWIND_ETIMEOUT: return "device wait timed out";
    case MCWIND_ESHIFT: return "grid not terrain-following in shift form (separable operator)";
    default: return "unknown error";
  }
}

extern "C" void mcwind_plan_destroy(mcwind_plan p) {
  if (!p) return;
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  if (p->iter_exec) cudaGraphExecDestroy(p->iter_exec);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  delete p;
}

namespace {
int assemble_hierarchy(mcwind_plan p, cudaStream_t st);
int assemble_separable(mcwind_plan p, cudaStream_t st);
}  // namespace

extern "C" int mcwind_assemble(mcwind_plan p, void* workspace, const double* X, const double* Y,
                               const double* Z, void* stream) {
  if (!p || !workspace || !X || !Y || !Z) return MCWIND_EINVAL;
  if (((uintptr_t)workspace) % 256 != 0) return MCWIND_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  p->ws = (char*)workspace;
  p->X = X; p->Y = Y; p->Z = Z;
  p->assembled = false;
  // zero level-0 planes (assembly accumulates into them) and every vector
  for (size_t l = 0; l < p->lv.size(); ++l) {
    Level& L = p->lv[l];
    const size_t t = (size_t)L.g.total;
    if (l == 0 && !p->sep) CK(cudaMemsetAsync(at(p, L.C64), 0, kPlanes * t * 8, st));
    Ptr64 A = lv64(p, (int)l);
    CK(cudaMemsetAsync(A.x, 0, 3 * ((t * 8 + 255) / 256 * 256), st));
    if (p->opt.precision == MCWIND_PREC_MIXED) {
      Ptr32 B = lv32(p, (int)l);
      CK(cudaMemsetAsync(B.x, 0, 3 * ((t * 4 + 255) / 256 * 256), st));
    }
  }
  CK(cudaMemsetAsync(p->ws + p->off_scalars, 0, 256, st));
  Level& L0 = p->lv[0];
  {
    PROF(MCWIND_K_ASSEMBLE);
    float2* xyz2 = (float2*)(p->ws + p->off_xyz2);
    const int64_t nn = (int64_t)std_nodes(p);
    // the element kernels' coordinates as float pairs (a separable plan
    // needs them only for a load vector formed element by element)
    if (dfloat_elements(p) && (!p->sep || !sep_rhs(p))) {
      CK(launch_split_pairs(X, xyz2, nn, st));
      CK(launch_split_pairs(Y, xyz2 + nn, nn, st));
      CK(launch_split_pairs(Z, xyz2 + 2 * nn, nn, st));
    }
    // the separable form expands the finest rows from its factors instead
    if (!p->sep)
      CK(launch_assemble_stencil(L0.g, p->nx, p->ny, p->nz, X, Y, Z, xyz2, p->a, at(p, L0.C64),
                                 flagp(p), dfloat_elements(p), st));
  }
  if (!p->sep) {
    PROF(MCWIND_K_SETUP);
    CK(launch_stencil_finalize(L0.g, at(p, L0.C64), flagp(p), st));
  }
  if (p->sep) {
    CKR(assemble_separable(p, st));
  } else {
    CKR(assemble_hierarchy(p, st));
  }
  // coarsest direct solver
  Level& Lc = p->lv.back();
  double* A = (double*)(p->ws + p->off_dense);
  double* B = A + (size_t)p->n_coarse * p->n_coarse;
  {
    PROF(MCWIND_K_SETUP);
    CK(launch_coarse_index(Lc.g, cfree(p), st));
    CK(launch_dense_gather(Lc.g, at(p, Lc.C64), cfree(p), p->n_coarse, A, st));
    double* res = nullptr;
    CK(launch_dense_invert(A, B, p->n_coarse, &res, st));
  }
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, flagp(p), sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (p->prof) prof_fold(p);
  if (flag & 8) return MCWIND_ESHIFT;
  if (flag) return MCWIND_EGEOM;
  p->assembled = true;
  return MCWIND_OK;
}

namespace {

// Galerkin operators of the stored form: K_c = P^T K P one direction at a
// time on every level, finalized, and their float32 copies (mixed precision).
int assemble_hierarchy(mcwind_plan p, cudaStream_t st) {
  double* tmpA = (double*)(p->ws + p->off_tmp);
  double* tmpB = (double*)(p->ws + p->off_tmp + p->tmp_bytes);
  for (size_t l = 0; l + 1 < p->lv.size(); ++l) {
    Level& F = p->lv[l];
    Level& Cl = p->lv[l + 1];
    struct Stage { int dim; Grid gout; };
    std::vector<Stage> stages;
    int nxg = F.g.Nx, nyg = F.g.Ny;
    if (F.hx) { nxg = Cl.g.Nx; stages.push_back({0, make_grid(nxg, nyg, F.g.Nz)}); }
    if (F.hy) { nyg = Cl.g.Ny; stages.push_back({1, make_grid(nxg, nyg, F.g.Nz)}); }
    if (Cl.g.Nz != F.g.Nz) stages.push_back({2, Cl.g});
    const double* src = at(p, F.C64);
    Grid gin = F.g;
    for (size_t s = 0; s < stages.size(); ++s) {
      double* dst = (s + 1 == stages.size()) ? at(p, Cl.C64) : (s == 0 ? tmpA : tmpB);
      PROF(MCWIND_K_RAP);
      CK(launch_rap_stage(stages[s].dim, gin, stages[s].gout, F.tr, src, dst, st));
      src = dst;
      gin = stages[s].gout;
    }
    PROF(MCWIND_K_SETUP);
    CK(launch_stencil_finalize(Cl.g, at(p, Cl.C64), flagp(p), st));
  }
  PROF(MCWIND_K_SETUP);
  if (p->opt.precision == MCWIND_PREC_MIXED)
    for (size_t l = 0; l < p->lv.size(); ++l)
      CK(launch_stencil_to_f32(p->lv[l].g, at(p, p->lv[l].C64), at(p, p->lv[l].C32), st));
  return MCWIND_OK;
}

// Separable form: check the shift form, build the finest factors from the
// ground layer and the layer thicknesses, carry them down the hierarchy
// (horizontal and vertical Galerkin products), and expand the coarsest
// level's float64 rows for its direct solve.
int assemble_separable(mcwind_plan p, cudaStream_t st) {
  Level& L0 = p->lv[0];
  const int Nx = p->nx + 1, Ny = p->ny + 1, Nz = p->nz + 1;
  {
    PROF(MCWIND_K_SETUP);
    CK(launch_shift_check(Nx, Ny, Nz, p->X, p->Y, p->Z, flagp(p), st));
    CK(launch_hfactors(L0.g, p->X, p->Y, p->Z, p->a, at(p, L0.H64), at(p, L0.H32), flagp(p),
                       dfloat_elements(p), st));
    CK(launch_vfactor0(Nx, Ny, Nz, p->Z, at(p, L0.V64), at(p, L0.V32), at(p, L0.VR2), flagp(p),
                       st));
    if (sep_rhs(p)) {
      CK(launch_rhs_factors(L0.g, p->X, p->Y, p->Z, at(p, L0.R2), st));
      CK(make_u0_map(L0, (float2*)(p->ws + p->off_u2)));
    }
  }
  {
    // the finest float64 rows (the refinement's residual operator): the same
    // 2x2x2-Gauss stiffness, assembled from its column and layer factors
    PROF(MCWIND_K_ASSEMBLE);
    CK(launch_sep_expand64(L0.g, at(p, L0.H64), at(p, L0.V64), at(p, L0.C64), flagp(p),
                           dfloat_elements(p), st));
  }
  for (size_t l = 0; l < p->lv.size(); ++l)
    CK(make_tile_maps(p->lv[l], at(p, p->lv[l].x32), at(p, p->lv[l].f32)));
  double* tmp = (double*)(p->ws + p->off_tmp);
  for (size_t l = 0; l + 1 < p->lv.size(); ++l) {
    Level& F = p->lv[l];
    Level& Cl = p->lv[l + 1];
    PROF(MCWIND_K_RAP);
    if (F.hx && F.hy) {
      const Grid mid = make_grid(Cl.g.Nx, F.g.Ny, 1);
      CK(launch_hgalerkin(0, F.g, mid, at(p, F.H64), tmp, st));
      CK(launch_hgalerkin(1, mid, Cl.g, tmp, at(p, Cl.H64), st));
    } else if (F.hx || F.hy) {
      CK(launch_hgalerkin(F.hx ? 0 : 1, F.g, Cl.g, at(p, F.H64), at(p, Cl.H64), st));
    }
    if (!Cl.h_shared) CK(launch_hfactor_finalize(Cl.g, at(p, Cl.H64), at(p, Cl.H32), st));
    CK(launch_vgalerkin(F.tr, at(p, F.V64), at(p, Cl.V64), at(p, Cl.V32), st));
  }
  Level& Lc = p->lv.back();
  PROF(MCWIND_K_SETUP);
  CK(launch_sep_expand64(Lc.g, at(p, Lc.H64), at(p, Lc.V64), at(p, Lc.C64), flagp(p),
                         dfloat_elements(p), st));
  return MCWIND_OK;
}

}  // namespace

extern "C" int mcwind_rhs(mcwind_plan p, const double* u0, double* f, void* stream) {
  if (!p || !u0 || !f) return MCWIND_EINVAL;
  if (!p->assembled) return MCWIND_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  Level& L0 = p->lv[0];
  Ptr64 A = lv64(p, 0);
  PROF(MCWIND_K_RHS);
  CK(rhs_into(p, u0, A.f, st));
  CK(launch_split_to_std<double>(L0.g, A.f, f, st));
  return MCWIND_OK;
}

namespace {

struct CgVec {
  double *x, *f, *r, *rp, *p, *q;
};
CgVec cg_vectors(mcwind_plan p) {
  const size_t stride = ((size_t)p->lv[0].g.total * 8 + 255) / 256 * 256;
  char* b = p->ws + p->off_cg;
  return {(double*)b, (double*)(b + stride), (double*)(b + 2 * stride), (double*)(b + 3 * stride),
          (double*)(b + 4 * stride), (double*)(b + 5 * stride)};
}

// preconditioner input from the current residual (pf = r, px = 0, rp = 0)
int cg_restart(mcwind_plan p, const CgVec& v, cudaStream_t st) {
  PROF(MCWIND_K_KRYLOV);
  const Grid& g = p->lv[0].g;
  if (p->opt.precision == MCWIND_PREC_F64)
    CK(launch_cg_start<double>(g, v.r, v.rp, lv64(p, 0).f, lv64(p, 0).x, scal(p) + 4, st));
  else
    CK(launch_cg_start<float>(g, v.r, v.rp, lv32(p, 0).f, lv32(p, 0).x, scal(p) + 4, st));
  return MCWIND_OK;
}

// r = f - K x (true residual) and ||r||^2 into scal[1]
int cg_true_residual(mcwind_plan p, const CgVec& v, cudaStream_t st) {
  const Grid& g = p->lv[0].g;
  int nb = 0;
  {
    PROF(MCWIND_K_OUTER_RESIDUAL);
    CK(launch_residual<double>(g, lv64(p, 0).C, v.f, v.x, v.r, partials(p), p->n_partials, &nb, st));
  }
  PROF(MCWIND_K_OTHER);
  CK(launch_reduce_final(partials(p), nb, scal(p) + 1, st));
  return MCWIND_OK;
}

// one preconditioned CG iteration; ||r||^2 (recursive) into scal[1]
template <typename T>
int cg_iteration(mcwind_plan p, const CgVec& v, cudaStream_t st) {
  CKR(vcycle<T>(p, 0, st, true));  // the preconditioner input starts at 0
  const Grid& g = p->lv[0].g;
  auto P = Sel<T>::get(p, 0);
  double* s = scal(p) + 4;
  {
    PROF(MCWIND_K_KRYLOV);
    CK(launch_cg_dots<T>(g, v.r, v.rp, P.x, partials(p), p->n_partials, s, st));
    CK(launch_cg_direction<T>(g, P.x, v.p, s, st));
  }
  int nb = 0;
  {
    PROF(MCWIND_K_OUTER_RESIDUAL);
    CK(launch_apply(g, lv64(p, 0).C, v.p, v.q, partials(p), p->n_partials, &nb, st));
  }
  {
    PROF(MCWIND_K_OTHER);
    CK(launch_reduce_final(partials(p), nb, s + 4, st));
  }
  PROF(MCWIND_K_KRYLOV);
  CK(launch_cg_update<T>(g, v.x, v.r, v.rp, v.p, v.q, P.f, P.x, s, partials(p), p->n_partials,
                         scal(p) + 1, st));
  return MCWIND_OK;
}

int solve_cg(mcwind_plan p, const double* u0, const double* f_given, double* lambda,
             double rtol, int max_cycles, unsigned flags, mcwind_stats& S, cudaStream_t st) {
  Level& L0 = p->lv[0];
  const CgVec v = cg_vectors(p);
  if (f_given) {
    PROF(MCWIND_K_OTHER);
    CK(launch_std_to_split<double>(L0.g, f_given, v.f, true, st));
  } else {
    PROF(MCWIND_K_RHS);
    CK(rhs_into(p, u0, v.f, st));
  }
  CKR(norm2(p, L0.g, v.f, 0, st));
  {
    PROF(MCWIND_K_OTHER);
    if (flags & MCWIND_WARM)
      CK(launch_std_to_split<double>(L0.g, lambda, v.x, true, st));
    else
      CK(cudaMemsetAsync(v.x, 0, sizeof(double) * (size_t)L0.g.total, st));
  }
  CKR(cg_true_residual(p, v, st));
  double h[2];
  CKR(read_scalars(p, h, 0, 2, st));
  const double nf = std::sqrt(h[0]);
  S.norm_f = nf;
  if (!std::isfinite(nf) || !std::isfinite(h[1])) return MCWIND_ENONFINITE;
  int status = MCWIND_OK;
  if (nf == 0.0) {
    CK(cudaMemsetAsync(v.x, 0, sizeof(double) * (size_t)L0.g.total, st));
    S.res_hist[0] = 0.0;
  } else {
    S.res_hist[0] = std::sqrt(h[1]) / nf;
    CKR(cg_restart(p, v, st));
    int c = 0;
    while (c < max_cycles) {
      if (S.res_hist[c] <= rtol) {
        // the recursive residual says converged: confirm with the true one
        CKR(cg_true_residual(p, v, st));
        CKR(read_scalars(p, h + 1, 1, 1, st));
        S.res_hist[c] = std::sqrt(h[1]) / nf;
        if (S.res_hist[c] <= rtol) break;
        CKR(cg_restart(p, v, st));
      }
      if (p->opt.precision == MCWIND_PREC_F64)
        CKR(run_iteration(p, st, [&v](mcwind_plan q, cudaStream_t s2) -> int { return cg_iteration<double>(q, v, s2); }));
      else
        CKR(run_iteration(p, st, [&v](mcwind_plan q, cudaStream_t s2) -> int { return cg_iteration<float>(q, v, s2); }));
      CKR(read_scalars(p, h + 1, 1, 1, st));
      ++c;
      S.res_hist[c] = std::sqrt(h[1]) / nf;
      if (!std::isfinite(S.res_hist[c])) break;
    }
    if (c == max_cycles && S.res_hist[c] <= rtol) {
      CKR(cg_true_residual(p, v, st));
      CKR(read_scalars(p, h + 1, 1, 1, st));
      S.res_hist[c] = std::sqrt(h[1]) / nf;
    }
    S.cycles = c;
    if (!(S.res_hist[c] <= rtol)) status = MCWIND_ENOTCONV;
  }
  {
    PROF(MCWIND_K_OTHER);
    CK(launch_split_to_std<double>(L0.g, v.x, lambda, st));
  }
  return status;
}

}  // namespace

// u0 given: load vector of Eq. 5 from it; f_given: the caller's load vector
static int solve_impl(mcwind_plan p, const double* u0, const double* f_given, double* lambda,
                      double rtol, int max_cycles, unsigned flags, mcwind_stats* stats,
                      void* stream) {
  if (!p || (!u0 && !f_given) || !lambda) return MCWIND_EINVAL;
  if (!p->assembled) return MCWIND_ESTATE;
  if (max_cycles < 0 || max_cycles >= MCWIND_HIST || !(rtol >= 0.0)) return MCWIND_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (p->opt.accel == MCWIND_ACCEL_CG) {
    mcwind_stats S;
    std::memset(&S, 0, sizeof(S));
    int status = solve_cg(p, u0, f_given, lambda, rtol, max_cycles, flags, S, st);
    if (status != MCWIND_OK && status != MCWIND_ENOTCONV && status != MCWIND_ENONFINITE) return status;
    S.rel_res = S.res_hist[S.cycles];
    if (S.cycles >= 3 && S.res_hist[2] > 0.0)
      S.rate = std::pow(S.res_hist[S.cycles] / S.res_hist[2], 1.0 / (S.cycles - 2));
    else if (S.cycles >= 1 && S.res_hist[0] > 0.0)
      S.rate = std::pow(S.res_hist[S.cycles] / S.res_hist[0], 1.0 / S.cycles);
    S.status = status;
    if (stats) *stats = S;
    return status;
  }
  Level& L0 = p->lv[0];
  Ptr64 A = lv64(p, 0);
  // load vector f (Eq. 5 right side) and its norm
  if (f_given) {
    PROF(MCWIND_K_OTHER);
    CK(launch_std_to_split<double>(L0.g, f_given, A.f, true, st));
  } else {
    PROF(MCWIND_K_RHS);
    CK(rhs_into(p, u0, A.f, st));
  }
  CKR(norm2(p, L0.g, A.f, 0, st));
  {
    PROF(MCWIND_K_OTHER);
    if (flags & MCWIND_WARM)
      CK(launch_std_to_split<double>(L0.g, lambda, A.x, true, st));
    else
      CK(cudaMemsetAsync(A.x, 0, sizeof(double) * (size_t)L0.g.total, st));
  }
  CKR(outer_residual(p, st, !(flags & MCWIND_WARM)));
  double h[2];
  CKR(read_scalars(p, h, 0, 2, st));
  const double nf = std::sqrt(h[0]);
  mcwind_stats S;
  std::memset(&S, 0, sizeof(S));
  S.norm_f = nf;
  if (!std::isfinite(nf) || !std::isfinite(h[1])) {
    if (stats) { S.status = MCWIND_ENONFINITE; *stats = S; }
    return MCWIND_ENONFINITE;
  }
  int status = MCWIND_OK;
  if (nf == 0.0) {
    CK(cudaMemsetAsync(A.x, 0, sizeof(double) * (size_t)L0.g.total, st));
    S.res_hist[0] = 0.0;
  } else {
    S.res_hist[0] = std::sqrt(h[1]) / nf;
    int c = 0;
    const int kc = check_every(p);
    while (S.res_hist[c] > rtol && c < max_cycles) {
      const int n = std::min(kc, max_cycles - c);
      if (n == kc)
        CKR(run_iteration(p, st, [kc](mcwind_plan q, cudaStream_t s2) -> int {
          return iteration(q, s2, kc);
        }));
      else
        CKR(iteration(p, st, n));  // a shorter last step runs outside the graph
      CKR(read_scalars(p, h + 1, 1, 1, st));
      S.res_hist[c + n] = std::sqrt(h[1]) / nf;
      fill_between(S.res_hist, c, c + n);
      c += n;
      if (!std::isfinite(S.res_hist[c])) break;
    }
    S.cycles = c;
    if (!(S.res_hist[c] <= rtol)) status = MCWIND_ENOTCONV;
  }
  S.rel_res = S.res_hist[S.cycles];
  if (S.cycles >= 3 && S.res_hist[2] > 0.0)
    S.rate = std::pow(S.res_hist[S.cycles] / S.res_hist[2], 1.0 / (S.cycles - 2));
  else if (S.cycles >= 1 && S.res_hist[0] > 0.0)
    S.rate = std::pow(S.res_hist[S.cycles] / S.res_hist[0], 1.0 / S.cycles);
  S.status = status;
  {
    PROF(MCWIND_K_OTHER);
    CK(launch_split_to_std<double>(L0.g, A.x, lambda, st));
  }
  if (stats) *stats = S;
  return status;
}

extern "C" int mcwind_solve(mcwind_plan p, const double* u0, double* lambda, double rtol,
                            int max_cycles, unsigned flags, mcwind_stats* stats, void* stream) {
  if (!u0) return MCWIND_EINVAL;
  return solve_impl(p, u0, nullptr, lambda, rtol, max_cycles, flags, stats, stream);
}

extern "C" int mcwind_solve_rhs(mcwind_plan p, const double* f, double* x, double rtol,
                                int max_cycles, unsigned flags, mcwind_stats* stats, void* stream) {
  if (!f) return MCWIND_EINVAL;
  return solve_impl(p, nullptr, f, x, rtol, max_cycles, flags, stats, stream);
}

extern "C" int mcwind_recover_adjoint(mcwind_plan p, const double* gu, double* h, double* du0,
                                      void* stream) {
  if (!p || !gu || !h || !du0 || p->opt.u0_at != MCWIND_U0_NODES) return MCWIND_EINVAL;
  if (!p->assembled) return MCWIND_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t N = (size_t)(p->nx + 1) * (p->ny + 1) * (p->nz + 1);
  CK(cudaMemsetAsync(h, 0, N * sizeof(double), st));
  CK(cudaMemsetAsync(du0, 0, 3 * N * sizeof(double), st));
  CK(launch_recover_adjoint(p->nx, p->ny, p->nz, p->X, p->Y, p->Z, gu, p->a, h, du0, st));
  return MCWIND_OK;
}

extern "C" int mcwind_adjoint_finish(mcwind_plan p, const double* mu, const double* lambda,
                                     const double* gu, double* du0, double* dloga, void* stream) {
  if (!p || !mu || !lambda || !gu || !du0 || !dloga || p->opt.u0_at != MCWIND_U0_NODES)
    return MCWIND_EINVAL;
  if (!p->assembled) return MCWIND_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  double* part = (double*)(p->ws + p->off_adj);
  double* sums = part + 6 * (size_t)p->n_adj;
  CK(launch_adjoint_finish(p->nx, p->ny, p->nz, p->X, p->Y, p->Z, mu, lambda, gu, du0, part,
                           p->n_adj, sums, st));
  double h6[6];
  CK(cudaMemcpyAsync(h6, sums, sizeof(h6), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int d = 0; d < 3; ++d) dloga[d] = 2.0 / (p->a[d] * p->a[d]) * (h6[d] - h6[3 + d]);
  return MCWIND_OK;
}

extern "C" int mcwind_recover(mcwind_plan p, const double* u0, const double* lambda, double* u,
                              int where, void* stream) {
  if (!p || !u0 || !lambda || !u) return MCWIND_EINVAL;
  if (where != MCWIND_AT_CENTERS && where != MCWIND_AT_GAUSS) return MCWIND_EINVAL;
  if (!p->assembled) return MCWIND_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  Level& L0 = p->lv[0];
  if (where == MCWIND_AT_CENTERS && dfloat_elements(p) && p->sep) {
    // shift form: the column's center Jacobian once, each layer's 2/h
    const bool nodal = p->opt.u0_at == MCWIND_U0_NODES;
    PROF(MCWIND_K_RECOVER);
    CK(launch_recover_center_sep(p->nx, p->ny, p->nz, p->X, p->Y, p->Z, nodal ? u0 : nullptr,
                                 nodal ? nullptr : u0, lambda, p->a, u, st));
    return MCWIND_OK;
  }
  if (where == MCWIND_AT_CENTERS && dfloat_elements(p)) {
    // float pairs: lambda and a nodal u0 split in the [k][j][i] layout
    float2* lam2 = (float2*)lv64(p, 0).r;  // scratch, >= nodes float pairs
    float2* u2 = (float2*)(p->ws + p->off_u2);
    const int64_t nn = (int64_t)std_nodes(p);
    {
      PROF(MCWIND_K_OTHER);
      CK(launch_split_pairs(lambda, lam2, nn, st));
      if (p->opt.u0_at == MCWIND_U0_NODES) CK(launch_split_pairs(u0, u2, 3 * nn, st));
    }
    PROF(MCWIND_K_RECOVER);
    CK(launch_recover_center_df(p->nx, p->ny, p->nz, (const float2*)(p->ws + p->off_xyz2), u2,
                                p->opt.u0_at == MCWIND_U0_NODES ? nullptr : u0, lam2, p->a, u, st));
    return MCWIND_OK;
  }
  double* lam = lv64(p, 0).r;  // scratch: lambda in the split layout
  {
    PROF(MCWIND_K_OTHER);
    CK(launch_std_to_split<double>(L0.g, lambda, lam, true, st));
  }
  PROF(MCWIND_K_RECOVER);
  CK(launch_recover(L0.g, p->nx, p->ny, p->nz, p->X, p->Y, p->Z, u0, lam, p->a, where, p->opt.u0_at, u, st));
  return MCWIND_OK;
}

extern "C" int mcwind_weak_div(mcwind_plan p, const double* ug, double* out, void* stream) {
  if (!p || !ug || !out) return MCWIND_EINVAL;
  if (!p->assembled) return MCWIND_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  size_t n = (size_t)(p->nx + 1) * (p->ny + 1) * (p->nz + 1);
  CK(cudaMemsetAsync(out, 0, n * sizeof(double), st));
  CK(launch_weak_div(p->nx, p->ny, p->nz, p->X, p->Y, p->Z, ug, out, st));
  return MCWIND_OK;
}

extern "C" int mcwind_level_stencil(mcwind_plan p, int level, int precision, double* out,
                                    void* stream) {
  CKR(check_level(p, level, precision));
  if (!out) return MCWIND_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const Grid& g = p->lv[level].g;
  const Level& L = p->lv[level];
  if (p->sep && precision == MCWIND_PREC_F64)
    CK(launch_sep_export<double>(g, at(p, L.H64), at(p, L.V64), out, st));
  else if (p->sep)
    CK(launch_sep_export<float>(g, at(p, L.H32), at(p, L.V32), out, st));
  else if (precision == MCWIND_PREC_F64)
    CK(launch_stencil_export<double>(g, lv64(p, level).C, out, st));
  else
    CK(launch_stencil_export<float>(g, lv32(p, level).C, out, st));
  return MCWIND_OK;
}

extern "C" int mcwind_level_residual(mcwind_plan p, int level, int precision, const double* x,
                                     const double* f, double* r, void* stream) {
  CKR(check_level(p, level, precision, true));
  if (!x || !f || !r) return MCWIND_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const Grid& g = p->lv[level].g;
  if (precision == MCWIND_PREC_F64) {
    Ptr64 P = lv64(p, level);
    CK(launch_std_to_split<double>(g, x, P.x, true, st));
    CK(launch_std_to_split<double>(g, f, P.f, true, st));
    CK(launch_residual<double>(g, P.C, P.f, P.x, P.r, nullptr, 0, nullptr, st));
    CK(launch_split_to_std<double>(g, P.r, r, st));
  } else {
    Ptr32 P = lv32(p, level);
    CK(launch_std_to_split<float>(g, x, P.x, true, st));
    CK(launch_std_to_split<float>(g, f, P.f, true, st));
    if (p->sep)
      CK(launch_residual_sep_staged(p->lv[level], false, sep_h32(p, level), sep_v32(p, level),
                                    P.r, statusp(p), st));
    else
      CK(launch_residual<float>(g, P.C, P.f, P.x, P.r, nullptr, 0, nullptr, st));
    CK(launch_split_to_std<float>(g, P.r, r, st));
  }
  return MCWIND_OK;
}

extern "C" int mcwind_level_residual_restrict(mcwind_plan p, int level, int precision,
                                              const double* x, const double* f, double* fc,
                                              void* stream) {
  CKR(check_level(p, level, precision, true));
  if (level + 1 >= (int)p->lv.size() || !x || !f || !fc) return MCWIND_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const Grid& g = p->lv[level].g;
  const Grid& gc = p->lv[level + 1].g;
  if (precision == MCWIND_PREC_F64) {
    Ptr64 P = lv64(p, level), Q = lv64(p, level + 1);
    CK(launch_std_to_split<double>(g, x, P.x, true, st));
    CK(launch_std_to_split<double>(g, f, P.f, true, st));
    CKR(residual_restrict<double>(p, level, st));
    CK(launch_split_to_std<double>(gc, Q.f, fc, st));
  } else {
    Ptr32 P = lv32(p, level), Q = lv32(p, level + 1);
    CK(launch_std_to_split<float>(g, x, P.x, true, st));
    CK(launch_std_to_split<float>(g, f, P.f, true, st));
    CKR(residual_restrict<float>(p, level, st));
    CK(launch_split_to_std<float>(gc, Q.f, fc, st));
  }
  return MCWIND_OK;
}

extern "C" int mcwind_level_smooth(mcwind_plan p, int level, int precision, double* x,
                                   const double* f, int sweeps, int direction, void* stream) {
  CKR(check_level(p, level, precision, true));
  if (!x || !f || sweeps < 0) return MCWIND_EINVAL;
  if (direction != MCWIND_FORWARD && direction != MCWIND_BACKWARD) return MCWIND_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const Grid& g = p->lv[level].g;
  if (precision == MCWIND_PREC_F64) {
    Ptr64 P = lv64(p, level);
    CK(launch_std_to_split<double>(g, x, P.x, true, st));
    CK(launch_std_to_split<double>(g, f, P.f, true, st));
    CKR(smooth<double>(p, level, sweeps, direction, st));
    CK(launch_split_to_std<double>(g, P.x, x, st));
  } else {
    Ptr32 P = lv32(p, level);
    CK(launch_std_to_split<float>(g, x, P.x, true, st));
    CK(launch_std_to_split<float>(g, f, P.f, true, st));
    CKR(smooth<float>(p, level, sweeps, direction, st));
    CK(launch_split_to_std<float>(g, P.x, x, st));
  }
  return MCWIND_OK;
}

extern "C" int mcwind_level_restrict(mcwind_plan p, int level, int precision, const double* r,
                                     double* fc, void* stream) {
  CKR(check_level(p, level, precision));
  if (level + 1 >= (int)p->lv.size() || !r || !fc) return MCWIND_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Level& F = p->lv[level];
  const Grid& gc = p->lv[level + 1].g;
  if (precision == MCWIND_PREC_F64) {
    Ptr64 P = lv64(p, level), Q = lv64(p, level + 1);
    CK(launch_std_to_split<double>(F.g, r, P.r, true, st));
    CK(launch_restrict<double>(F.g, gc, F.tr, P.r, Q.f, st));
    CK(launch_split_to_std<double>(gc, Q.f, fc, st));
  } else {
    Ptr32 P = lv32(p, level), Q = lv32(p, level + 1);
    CK(launch_std_to_split<float>(F.g, r, P.r, true, st));
    CK(launch_restrict<float>(F.g, gc, F.tr, P.r, Q.f, st));
    CK(launch_split_to_std<float>(gc, Q.f, fc, st));
  }
  return MCWIND_OK;
}

extern "C" int mcwind_level_prolong(mcwind_plan p, int level, int precision, const double* ec,
                                    double* x, void* stream) {
  CKR(check_level(p, level, precision));
  if (level + 1 >= (int)p->lv.size() || !ec || !x) return MCWIND_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Level& F = p->lv[level];
  const Grid& gc = p->lv[level + 1].g;
  if (precision == MCWIND_PREC_F64) {
    Ptr64 P = lv64(p, level), Q = lv64(p, level + 1);
    CK(launch_std_to_split<double>(gc, ec, Q.x, true, st));
    CK(launch_std_to_split<double>(F.g, x, P.x, true, st));
    CK(launch_prolong_add<double>(F.g, gc, F.tr, Q.x, P.x, st));
    CK(launch_split_to_std<double>(F.g, P.x, x, st));
  } else {
    Ptr32 P = lv32(p, level), Q = lv32(p, level + 1);
    CK(launch_std_to_split<float>(gc, ec, Q.x, true, st));
    CK(launch_std_to_split<float>(F.g, x, P.x, true, st));
    CK(launch_prolong_add<float>(F.g, gc, F.tr, Q.x, P.x, st));
    CK(launch_split_to_std<float>(F.g, P.x, x, st));
  }
  return MCWIND_OK;
}

extern "C" int mcwind_coarse_solve(mcwind_plan p, const double* f, double* x, void* stream) {
  if (!p || !f || !x) return MCWIND_EINVAL;
  if (!p->assembled) return MCWIND_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  const int last = (int)p->lv.size() - 1;
  const Grid& g = p->lv[last].g;
  Ptr64 P = lv64(p, last);
  CK(launch_std_to_split<double>(g, f, P.f, true, st));
  CK(cudaMemsetAsync(P.x, 0, sizeof(double) * (size_t)g.total, st));
  CK(launch_dense_solve<double>(dense_inv(p), p->n_coarse, cfree(p), P.f, P.x, st));
  CK(launch_split_to_std<double>(g, P.x, x, st));
  return MCWIND_OK;
}

extern "C" int mcwind_vcycle(mcwind_plan p, int precision, double* x, const double* f,
                             void* stream) {
  CKR(check_level(p, 0, precision));
  if (p->sep && precision == MCWIND_PREC_F64) return MCWIND_EINVAL;
  if (!x || !f) return MCWIND_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const Grid& g = p->lv[0].g;
  if (precision == MCWIND_PREC_F64) {
    Ptr64 P = lv64(p, 0);
    CK(launch_std_to_split<double>(g, x, P.x, true, st));
    CK(launch_std_to_split<double>(g, f, P.f, true, st));
    CKR(vcycle<double>(p, 0, st));
    CK(launch_split_to_std<double>(g, P.x, x, st));
  } else {
    Ptr32 P = lv32(p, 0);
    CK(launch_std_to_split<float>(g, x, P.x, true, st));
    CK(launch_std_to_split<float>(g, f, P.f, true, st));
    CKR(vcycle<float>(p, 0, st));
    CK(launch_split_to_std<float>(g, P.x, x, st));
  }
  return MCWIND_OK;
}

extern "C" int mcwind_profile(mcwind_plan p, int enable, void* stream) {
  if (!p) return MCWIND_EINVAL;
  if (enable) {
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    p->prof_marks.clear();
    p->ev_used = 0;
    for (int k = 0; k < MCWIND_K_KINDS; ++k) { p->prof_ms[k] = 0.0; p->prof_n[k] = 0; }
  }
  p->prof = enable != 0;
  return MCWIND_OK;
}

extern "C" int mcwind_profile_read(mcwind_plan p, double* ms, long long* launches, int nkinds,
                                   void* stream) {
  if (!p || nkinds < 0 || (nkinds > 0 && (!ms || !launches))) return MCWIND_EINVAL;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  prof_fold(p);
  for (int k = 0; k < nkinds && k < MCWIND_K_KINDS; ++k) {
    ms[k] = p->prof_ms[k];
    launches[k] = p->prof_n[k];
  }
  return MCWIND_K_KINDS;
}

// ---------------------------------------------------------------------------
// batches of independent domains: one CUDA graph per solve

namespace {

// the batch workspace: pointer and handle arrays, then the block read back
struct BatchLayout {
  size_t scal, pstat, hif, iter, out, active, cycles, status, nonfinite, nf, hist, total;
};

BatchLayout batch_layout(int n) {
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  BatchLayout L;
  size_t o = 0;
  L.scal = o; o = al(o + 8 * (size_t)n);
  L.pstat = o; o = al(o + 8 * (size_t)n);
  L.hif = o; o = al(o + 8 * (size_t)n);
  L.iter = o; o = al(o + 8);
  L.out = o;
  L.active = o; o += 4 * (size_t)n;
  L.cycles = o; o += 4 * (size_t)n;
  L.status = o; o += 4 * (size_t)n;
  L.nonfinite = o; o += 4 * (size_t)n;
  o = (o + 7) / 8 * 8;
  L.nf = o; o += 8 * (size_t)n;
  L.hist = o; o += 8 * (size_t)n * MCWIND_HIST;
  L.total = al(o);
  return L;
}

}  // namespace

struct mcwind_batch_s {
  std::vector<mcwind_plan> plans;
  char* ws = nullptr;                  // device workspace of the batch
  BatchLayout lay;
  std::vector<cudaStream_t> streams;   // one per domain (set-up and output branches)
  cudaStream_t cap = nullptr;          // the solve's capture stream
  cudaStream_t body = nullptr;         // capture stream of the loop's bodies
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraphExec_t exec = nullptr;      // the solve graph
  std::string key;                     // the arguments it was built for
  long long fixed_launches = 0;        // kernels outside the loop
  std::vector<long long> iter_launches;  // kernels of one iteration, per domain
};

namespace {

long long tuning_key(mcwind_plan p) {
  return ((long long)p->opt.nu_pre << 16) | ((long long)p->opt.nu_post << 8) | p->gs_rows;
}

// fork the batch's domain streams off st, run body(d) on the selected
// domains, join back into st
template <typename Body>
int fork_join(mcwind_batch b, cudaStream_t st, Body body) {
  CK(cudaEventRecord(b->fork, st));
  for (size_t d = 0; d < b->plans.size(); ++d) {
    CK(cudaStreamWaitEvent(b->streams[d], b->fork, 0));
    CKR(body((int)d, b->streams[d]));
    CK(cudaEventRecord(b->joins[d], b->streams[d]));
    CK(cudaStreamWaitEvent(st, b->joins[d], 0));
  }
  return MCWIND_OK;
}

void batch_clear_graph(mcwind_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->key.clear();
}

BatchDev batch_dev(mcwind_batch b, cudaGraphConditionalHandle h_while) {
  const BatchLayout& L = b->lay;
  BatchDev v;
  v.n = (int)b->plans.size();
  v.scal = (const double* const*)(b->ws + L.scal);
  v.pstat = (const int* const*)(b->ws + L.pstat);
  v.h_if = (const cudaGraphConditionalHandle*)(b->ws + L.hif);
  v.h_while = h_while;
  v.iter = (int*)(b->ws + L.iter);
  v.active = (int*)(b->ws + L.active);
  v.cycles = (int*)(b->ws + L.cycles);
  v.status = (int*)(b->ws + L.status);
  v.nonfinite = (int*)(b->ws + L.nonfinite);
  v.nf = (double*)(b->ws + L.nf);
  v.hist = (double*)(b->ws + L.hist);
  return v;
}

// The solve graph: per-domain set-up, k_batch_step(init), WHILE { per
// domain IF(active) { cycles_per_check V-cycles + update + float64
// residual }, k_batch_step(check) }, per-domain output.  Built once per set
// of arguments (tolerance, cycle limit, flags, buffers, tuning) and replayed.
int batch_build(mcwind_batch b, const double* const* u0, double* const* lambda, double rtol,
                int max_cycles, unsigned flags) {
  const int n = (int)b->plans.size();
  const int cpc = check_every(b->plans[0]);
  const int max_checks = max_cycles / cpc;
  batch_clear_graph(b);
  std::vector<const double*> sc(n);
  std::vector<const int*> ps(n);
  for (int d = 0; d < n; ++d) {
    sc[d] = scal(b->plans[d]);
    ps[d] = statusp(b->plans[d]);
  }
  CK(cudaMemcpy(b->ws + b->lay.scal, sc.data(), sizeof(void*) * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b->ws + b->lay.pstat, ps.data(), sizeof(void*) * n, cudaMemcpyHostToDevice));
  const long long n0 = mcwind_launch_count();
  CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  cudaGraph_t G = nullptr;
  std::vector<cudaGraphConditionalHandle> hif(n);
  cudaGraphConditionalHandle hw = 0;
  auto body = [&]() -> int {
    cudaStreamCaptureStatus cs;
    CK(cudaStreamGetCaptureInfo(b->cap, &cs, nullptr, &G, nullptr, nullptr, nullptr));
    CK(cudaGraphConditionalHandleCreate(&hw, G, 0, 0));
    for (int d = 0; d < n; ++d) CK(cudaGraphConditionalHandleCreate(&hif[d], G, 0, 0));
    const BatchDev dev = batch_dev(b, hw);
    // per domain: load vector, its norm, first iterate, first float64 residual
    CKR(fork_join(b, b->cap, [&](int d, cudaStream_t s) -> int {
      mcwind_plan p = b->plans[d];
      Level& L0 = p->lv[0];
      Ptr64 A = lv64(p, 0);
      CK(rhs_into(p, u0[d], A.f, s));
      CKR(norm2(p, L0.g, A.f, 0, s));
      if (flags & MCWIND_WARM)
        CK(launch_std_to_split<double>(L0.g, lambda[d], A.x, true, s));
      else
        CK(cudaMemsetAsync(A.x, 0, sizeof(double) * (size_t)L0.g.total, s));
      CKR(outer_residual(p, s, !(flags & MCWIND_WARM)));
      return (int)MCWIND_OK;
    }));
    CK(launch_batch_step(dev, 0, rtol, max_checks, cpc, b->cap));
    // the loop node after the init step
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(b->cap, &cs, nullptr, &G, &deps, nullptr, &ndeps));
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    CK(cudaGraphAddNode(&wnode, G, deps, nullptr, ndeps, &wp));
    CK(cudaStreamUpdateCaptureDependencies(b->cap, &wnode, nullptr, 1,
                                           cudaStreamSetCaptureDependencies));
    cudaGraph_t wbody = wp.conditional.phGraph_out[0];
    std::vector<cudaGraphNode_t> ifs(n);
    b->iter_launches.assign(n, 0);
    for (int d = 0; d < n; ++d) {
      cudaGraphNodeParams ip = {};
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = hif[d];
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      CK(cudaGraphAddNode(&ifs[d], wbody, nullptr, nullptr, 0, &ip));
      const long long k0 = mcwind_launch_count();
      CK(cudaStreamBeginCaptureToGraph(b->body, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal));
      const int rc = iteration(b->plans[d], b->body, cpc);
      cudaGraph_t g_if = nullptr;
      const cudaError_t e = cudaStreamEndCapture(b->body, &g_if);
      CKR(rc);
      CK(e);
      b->iter_launches[d] = mcwind_launch_count() - k0;
    }
    CK(cudaStreamBeginCaptureToGraph(b->body, wbody, ifs.data(), nullptr, n,
                                     cudaStreamCaptureModeThreadLocal));
    const cudaError_t ec = launch_batch_step(dev, 1, rtol, max_checks, cpc, b->body);
    cudaGraph_t g_w = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->body, &g_w);
    CK(ec);
    CK(ee);
    // per domain: the solution in the caller's layout
    CKR(fork_join(b, b->cap, [&](int d, cudaStream_t s) -> int {
      mcwind_plan p = b->plans[d];
      CK(launch_split_to_std<double>(p->lv[0].g, lv64(p, 0).x, lambda[d], s));
      return (int)MCWIND_OK;
    }));
    return (int)MCWIND_OK;
  };
  const int rc = body();
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
  long long loop_kernels = 1;
  for (long long k : b->iter_launches) loop_kernels += k;
  const long long captured = mcwind_launch_count() - n0;
  count_launches(-(int)captured);  // captured, not run: counted per solve
  if (rc != MCWIND_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  CK(e);
  const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(ei);
  b->fixed_launches = captured - loop_kernels;
  CK(cudaMemcpy(b->ws + b->lay.hif, hif.data(), sizeof(cudaGraphConditionalHandle) * n,
                cudaMemcpyHostToDevice));
  return MCWIND_OK;
}

std::string batch_key(mcwind_batch b, const double* const* u0, double* const* lambda, double rtol,
                      int max_cycles, unsigned flags) {
  std::string k;
  char buf[64];
  snprintf(buf, sizeof(buf), "%.17g/%d/%u", rtol, max_cycles, flags);
  k += buf;
  for (size_t d = 0; d < b->plans.size(); ++d) {
    snprintf(buf, sizeof(buf), "|%p,%p,%p,%lld", (const void*)u0[d], (void*)lambda[d],
             (void*)b->plans[d]->ws, tuning_key(b->plans[d]));
    k += buf;
  }
  return k;
}

}  // namespace

extern "C" size_t mcwind_batch_workspace_bytes(int n) {
  return n <= 0 ? 0 : batch_layout(n).total;
}

extern "C" int mcwind_batch_create(int n, const mcwind_plan* plans, void* workspace,
                                   mcwind_batch* out) {
  if (!out || n <= 0 || !plans || !workspace || ((uintptr_t)workspace) % 256 != 0) return MCWIND_EINVAL;
  *out = nullptr;
  for (int d = 0; d < n; ++d) {
    if (!plans[d]) return MCWIND_EINVAL;
    if (plans[d]->opt.accel != MCWIND_ACCEL_NONE || plans[d]->in_batch) return MCWIND_EINVAL;
    for (int e = 0; e < d; ++e)
      if (plans[e] == plans[d]) return MCWIND_EINVAL;
  }
  mcwind_batch b = new (std::nothrow) mcwind_batch_s;
  if (!b) return MCWIND_EINVAL;
  b->plans.assign(plans, plans + n);
  b->ws = (char*)workspace;
  b->lay = batch_layout(n);
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->body, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int d = 0; d < n && e == cudaSuccess; ++d) {
    cudaStream_t s;
    cudaEvent_t j;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    b->streams.push_back(s);
    e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    if (e == cudaSuccess) b->joins.push_back(j);
  }
  if (e != cudaSuccess) {
    g_last_cuda = (int)e;
    mcwind_batch_destroy(b);
    return MCWIND_ECUDA;
  }
  for (int d = 0; d < n; ++d) plans[d]->in_batch = true;
  *out = b;
  return MCWIND_OK;
}

extern "C" void mcwind_batch_destroy(mcwind_batch b) {
  if (!b) return;
  batch_clear_graph(b);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->body) cudaStreamDestroy(b->body);
  for (mcwind_plan p : b->plans)
    if (p) p->in_batch = false;
  delete b;
}

extern "C" int mcwind_batch_solve(mcwind_batch b, const double* const* u0, double* const* lambda,
                                  double rtol, int max_cycles, unsigned flags,
                                  mcwind_stats* stats, void* stream) {
  if (!b || !u0 || !lambda) return MCWIND_EINVAL;
  if (max_cycles < 0 || max_cycles >= MCWIND_HIST || !(rtol >= 0.0)) return MCWIND_EINVAL;
  const int n = (int)b->plans.size();
  for (int d = 0; d < n; ++d) {
    if (!u0[d] || !lambda[d]) return MCWIND_EINVAL;
    if (!b->plans[d]->assembled) return MCWIND_ESTATE;
    if (b->plans[d]->prof) return MCWIND_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const std::string key = batch_key(b, u0, lambda, rtol, max_cycles, flags);
  if (!b->exec || key != b->key) {
    CKR(batch_build(b, u0, lambda, rtol, max_cycles, flags));
    b->key = key;
  }
  // the whole solve: one graph launch, then one read of the bookkeeping
  CK(cudaGraphLaunch(b->exec, st));
  const BatchLayout& L = b->lay;
  std::vector<char> host(L.total - L.out);
  CK(cudaMemcpyAsync(host.data(), b->ws + L.out, host.size(), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  auto at_out = [&](size_t off) { return host.data() + (off - L.out); };
  const int* cyc = (const int*)at_out(L.cycles);
  const int* stw = (const int*)at_out(L.status);
  const int* nfin = (const int*)at_out(L.nonfinite);
  const double* hist = (const double*)at_out(L.hist);
  const double* nfv = (const double*)at_out(L.nf);
  const int cpc = check_every(b->plans[0]);
  int status = MCWIND_OK;
  long long ran = b->fixed_launches;
  for (int d = 0; d < n; ++d) {
    mcwind_stats T;
    std::memset(&T, 0, sizeof(T));
    T.cycles = cyc[d];
    T.norm_f = nfv[d];
    const double* h = hist + (size_t)d * MCWIND_HIST;
    for (int c = 0; c <= T.cycles; c += cpc) {
      T.res_hist[c] = h[c];
      if (c > 0) fill_between(T.res_hist, c - cpc, c);
    }
    ran += b->iter_launches[d] * (T.cycles / cpc);
    T.rel_res = T.res_hist[T.cycles];
    if (T.cycles >= 3 && T.res_hist[2] > 0.0)
      T.rate = std::pow(T.res_hist[T.cycles] / T.res_hist[2], 1.0 / (T.cycles - 2));
    else if (T.cycles >= 1 && T.res_hist[0] > 0.0)
      T.rate = std::pow(T.res_hist[T.cycles] / T.res_hist[0], 1.0 / T.cycles);
    if (nfin[d]) {
      T.status = MCWIND_ENONFINITE;
      if (status == MCWIND_OK || status == MCWIND_ENOTCONV) status = MCWIND_ENONFINITE;
    } else {
      T.status = T.rel_res <= rtol ? MCWIND_OK : MCWIND_ENOTCONV;
      if (T.status != MCWIND_OK && status == MCWIND_OK) status = MCWIND_ENOTCONV;
    }
    if (stw[d] != 0) status = MCWIND_ETIMEOUT;
    if (stats) stats[d] = T;
  }
  int checks = 0;
  for (int d = 0; d < n; ++d) checks = std::max(checks, cyc[d] / cpc);
  count_launches((int)(ran + checks));  // set-up + output, the iterations run, the checks
  return status;
}

extern "C" int mcwind_plan_wait_selftest(mcwind_plan p, int limit_us, void* stream) {
  if (!p || limit_us < 1 || limit_us > 1000000) return MCWIND_EINVAL;
  if (!p->assembled) return MCWIND_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  CK(launch_wait_selftest(statusp(p), 1000ull * (unsigned long long)limit_us, st));
  CK(cudaMemcpyAsync(&p->status_host, statusp(p), sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return p->status_host != 0 ? MCWIND_ETIMEOUT : MCWIND_OK;
}

extern "C" int mcwind_plan_set_tuning(mcwind_plan p, int nu_pre, int nu_post, int gs_block_rows) {
  if (!p) return MCWIND_EINVAL;
  if (nu_pre < 0 || nu_post < 0 || nu_pre > 16 || nu_post > 16 || nu_pre + nu_post == 0)
    return MCWIND_EINVAL;
  if (gs_block_rows != 1 && gs_block_rows != 2 && gs_block_rows != 4 && gs_block_rows != 8)
    return MCWIND_EINVAL;
  if (p->opt.accel == MCWIND_ACCEL_CG && nu_pre != nu_post) return MCWIND_EINVAL;
  p->opt.nu_pre = nu_pre;
  p->opt.nu_post = nu_post;
  p->gs_rows = gs_block_rows;
  if (p->iter_exec) { cudaGraphExecDestroy(p->iter_exec); p->iter_exec = nullptr; }
  return MCWIND_OK;
}
