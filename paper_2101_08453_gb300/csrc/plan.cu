// Host planner: the adaptive semicoarsening of Sec. 3 and the workspace
// layout.  No CUDA call is made here.
//
// Rule (Sec. 3).  With ratio(t) = t / (h1 a3) (MCWIND_RULE_PAPER, as
// printed) or a3 t / (a1 h1) (MCWIND_RULE_OPERATOR):
//  * coarsen both horizontal directions by 2 when ratio(bottom layer) > 1/3;
//  * then, with h1 doubled if it was coarsened, walk the layers from the
//    ground up: when ratio(layer) < 3 merge it with the layer above (the node
//    between them is dropped) and continue two layers up, else keep it.
// A coarsened horizontal direction keeps the even-index nodes and the last
// node; a direction with fewer than 3 cells is not coarsened.  The hierarchy
// ends at the first level with at most coarsest_max free nodes.  When the
// rule coarsens nothing on a level that is still too large, both horizontal
// directions are coarsened (or, if that is impossible, the level is the
// coarsest).
#include <algorithm>
#include <cmath>
#include <new>

#include "kernels.cuh"

namespace mcw {

struct PlanLevel {
  int cx, cy, cz;
  int hx = 0, hy = 0;
  std::vector<int> kmap;
};

static std::vector<PlanLevel> hierarchy(int nx, int ny, int nz, const double a[3], double h1,
                                        const double* h3, int rule, int coarsest_max) {
  std::vector<PlanLevel> out;
  const double a1 = a[0], a3 = a[2];
  auto ratio = [&](double t, double h) {
    return rule == MCWIND_RULE_PAPER ? t / (h * a3) : a3 * t / (a1 * h);
  };
  int cx = nx, cy = ny, cz = nz;
  double hh = h1;
  std::vector<double> layers(h3, h3 + nz);
  for (int guard = 0; guard < 64; ++guard) {
    PlanLevel L;
    L.cx = cx; L.cy = cy; L.cz = cz;
    const long long nfree = (long long)(cx - 1) * (cy - 1) * cz;
    if (nfree <= coarsest_max) { out.push_back(L); break; }
    const bool horiz = ratio(layers[0], hh) > 1.0 / 3.0;
    int hx = horiz && cx >= 3, hy = horiz && cy >= 3;
    double hn = (hx || hy) ? 2.0 * hh : hh;
    std::vector<int> kmap{0};
    std::vector<double> merged;
    for (size_t l = 0; l < layers.size();) {
      if (l + 1 < layers.size() && ratio(layers[l], hn) < 3.0) {
        merged.push_back(layers[l] + layers[l + 1]);
        l += 2;
      } else {
        merged.push_back(layers[l]);
        l += 1;
      }
      kmap.push_back((int)l);
    }
    if (!hx && !hy && merged.size() == layers.size()) {
      hx = cx >= 3;
      hy = cy >= 3;
      if (!hx && !hy) { out.push_back(L); break; }
      hn = 2.0 * hh;
    }
    L.hx = hx; L.hy = hy; L.kmap = kmap;
    out.push_back(L);
    cx = hx ? (cx + 1) / 2 : cx;
    cy = hy ? (cy + 1) / 2 : cy;
    cz = (int)merged.size();
    hh = hn;
    layers = merged;
  }
  return out;
}

static Transfer make_transfer(int hx, int hy, int Nzf, const std::vector<int>& kmap) {
  Transfer t;
  t.hx = hx; t.hy = hy; t.Nzf = Nzf; t.Nzc = (int)kmap.size();
  for (int K = 0; K < kMaxZ; ++K) t.kf[K] = K < t.Nzc ? kmap[K] : 0;
  for (int k = 0; k < kMaxZ; ++k) { t.kc0[k] = t.kc1[k] = 0; t.kw0[k] = t.kw1[k] = 0.0f; }
  for (int K = 0; K < t.Nzc; ++K) {
    const int k = kmap[K];
    t.kc0[k] = t.kc1[k] = K; t.kw0[k] = 1.0f; t.kw1[k] = 0.0f;
    if (K + 1 < t.Nzc && kmap[K + 1] - k == 2) {
      t.kc0[k + 1] = K; t.kc1[k + 1] = K + 1; t.kw0[k + 1] = 0.5f; t.kw1[k + 1] = 0.5f;
    }
  }
  return t;
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace mcw

using namespace mcw;

extern "C" void mcwind_default_options(mcwind_options* o) {
  if (!o) return;
  o->nu_pre = 2;
  o->nu_post = 2;
  o->coarsen_rule = MCWIND_RULE_OPERATOR;
  o->coarsest_max = 1024;
  o->precision = MCWIND_PREC_F64;
  o->rhs_quad = MCWIND_RHS_GAUSS8;
  o->post_reverse = 1;
  o->accel = MCWIND_ACCEL_NONE;
  o->use_graphs = 1;
  o->u0_at = MCWIND_U0_NODES;
  o->element_arith = MCWIND_ARITH_DFLOAT;
  o->cycles_per_check = 0;
  o->op_form = MCWIND_OP_STORED;
}

extern "C" int mcwind_plan_create(int nx, int ny, int nz, const double a[3], double h1,
                                  const double* h3, const mcwind_options* opt, mcwind_plan* out,
                                  size_t* workspace_bytes) {
  if (!out || !a || !h3) return MCWIND_EINVAL;
  *out = nullptr;
  if (nx < 2 || ny < 2 || nz < 1 || nz + 1 > kMaxZ) return MCWIND_EINVAL;
  if ((long long)(nx + 1) * (ny + 1) * (nz + 1) > (1LL << 34)) return MCWIND_EINVAL;
  if ((long long)(nx + 2) * (ny + 1) > (1LL << 31) - 1) return MCWIND_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!(a[d] > 0.0) || !std::isfinite(a[d])) return MCWIND_EINVAL;
  if (!(h1 > 0.0) || !std::isfinite(h1)) return MCWIND_EINVAL;
  for (int k = 0; k < nz; ++k)
    if (!(h3[k] > 0.0) || !std::isfinite(h3[k])) return MCWIND_EINVAL;
  mcwind_options o;
  mcwind_default_options(&o);
  if (opt) o = *opt;
  if (o.nu_pre < 0 || o.nu_post < 0 || o.nu_pre > 16 || o.nu_post > 16 ||
      o.nu_pre + o.nu_post == 0)
    return MCWIND_EINVAL;
  if (o.coarsen_rule != MCWIND_RULE_PAPER && o.coarsen_rule != MCWIND_RULE_OPERATOR)
    return MCWIND_EINVAL;
  if (o.coarsest_max < 1 || o.coarsest_max > kMaxCoarse) return MCWIND_EINVAL;
  if (o.precision != MCWIND_PREC_F64 && o.precision != MCWIND_PREC_MIXED) return MCWIND_EINVAL;
  if (o.rhs_quad != MCWIND_RHS_GAUSS8 && o.rhs_quad != MCWIND_RHS_CENTER1) return MCWIND_EINVAL;
  if (o.post_reverse != 0 && o.post_reverse != 1) return MCWIND_EINVAL;
  if (o.accel != MCWIND_ACCEL_NONE && o.accel != MCWIND_ACCEL_CG) return MCWIND_EINVAL;
  if (o.accel == MCWIND_ACCEL_CG && o.post_reverse != 1) return MCWIND_EINVAL;
  if (o.use_graphs != 0 && o.use_graphs != 1) return MCWIND_EINVAL;
  if (o.u0_at != MCWIND_U0_NODES && o.u0_at != MCWIND_U0_CENTERS) return MCWIND_EINVAL;
  if (o.element_arith != MCWIND_ARITH_F64 && o.element_arith != MCWIND_ARITH_DFLOAT) return MCWIND_EINVAL;
  if (o.cycles_per_check < 0 || o.cycles_per_check > 8) return MCWIND_EINVAL;
  if (o.op_form != MCWIND_OP_STORED && o.op_form != MCWIND_OP_SEPARABLE) return MCWIND_EINVAL;
  if (o.op_form == MCWIND_OP_SEPARABLE && o.precision != MCWIND_PREC_MIXED) return MCWIND_EINVAL;

  std::vector<PlanLevel> H = hierarchy(nx, ny, nz, a, h1, h3, o.coarsen_rule, o.coarsest_max);
  if (H.empty() || !H.back().kmap.empty()) return MCWIND_EINVAL;
  const PlanLevel& last = H.back();
  const long long nc = (long long)(last.cx - 1) * (last.cy - 1) * last.cz;
  if (nc > kMaxCoarse || nc < 1) return MCWIND_EINVAL;

  mcwind_plan p = new (std::nothrow) mcwind_plan_s;
  if (!p) return MCWIND_EINVAL;
  p->nx = nx; p->ny = ny; p->nz = nz;
  p->a[0] = a[0]; p->a[1] = a[1]; p->a[2] = a[2];
  p->opt = o;
  p->sep = o.op_form == MCWIND_OP_SEPARABLE;
  const bool mixed = o.precision == MCWIND_PREC_MIXED;
  size_t off = 0;
  int max_blocks = 0;
  for (size_t l = 0; l < H.size(); ++l) {
    Level L;
    L.g = make_grid(H[l].cx + 1, H[l].cy + 1, H[l].cz + 1);
    L.n_free = (H[l].cx - 1) * (H[l].cy - 1) * H[l].cz;
    L.hx = H[l].hx; L.hy = H[l].hy; L.kmap = H[l].kmap;
    if (l + 1 < H.size()) L.tr = make_transfer(L.hx, L.hy, L.g.Nz, L.kmap);
    const size_t t = (size_t)L.g.total;
    // separable form: float64 operator on the finest and the coarsest level
    // only, no float32 copy, factors per level (the horizontal ones shared
    // with the finer level when its transfer keeps the columns)
    L.has_c64 = !p->sep || l == 0 || l + 1 == H.size();
    if (L.has_c64) { L.C64 = (double*)off; off = align256(off + kPlanes * t * 8); }
    if (mixed && !p->sep) { L.C32 = (float*)off; off = align256(off + kPlanes * t * 4); }
    if (p->sep) {
      const Level* F = l > 0 ? &p->lv[l - 1] : nullptr;
      if (F && !F->hx && !F->hy) {
        L.H64 = F->H64; L.H32 = F->H32; L.h_shared = true;
      } else {
        const size_t cols = (size_t)L.g.PP;
        L.H64 = (double*)off; off = align256(off + kHF * cols * 8);
        L.H32 = (float*)off; off = align256(off + kHF * cols * 4);
      }
      L.V64 = (double*)off; off = align256(off + (size_t)kVF * L.g.Nz * 8);
      L.V32 = (float*)off; off = align256(off + (size_t)kVF * L.g.Nz * 4);
      if (l == 0) {
        L.R2 = (float2*)off; off = align256(off + (size_t)kRF * L.g.PP * 8);
        L.VR2 = (float2*)off; off = align256(off + (size_t)kRV * L.g.Nz * 8);
      }
    }
    L.x64 = (double*)off; off = align256(off + t * 8);
    L.f64 = (double*)off; off = align256(off + t * 8);
    L.r64 = (double*)off; off = align256(off + t * 8);
    if (mixed) {
      L.x32 = (float*)off; off = align256(off + t * 4);
      L.f32 = (float*)off; off = align256(off + t * 4);
      L.r32 = (float*)off; off = align256(off + t * 4);
    }
    max_blocks = std::max(max_blocks, residual_blocks(L.g));
    p->lv.push_back(L);
  }
  // RAP intermediates: up to two stage outputs per transition
  size_t tmpA = 0, tmpB = 0;
  for (size_t l = 0; l + 1 < p->lv.size(); ++l) {
    const Level& F = p->lv[l];
    const Level& Cl = p->lv[l + 1];
    int nxg = F.g.Nx, nyg = F.g.Ny;
    std::vector<size_t> outs;
    if (F.hx) { nxg = Cl.g.Nx; outs.push_back(make_grid(nxg, nyg, F.g.Nz).total); }
    if (F.hy) { nyg = Cl.g.Ny; outs.push_back(make_grid(nxg, nyg, F.g.Nz).total); }
    if (Cl.g.Nz != F.g.Nz) outs.push_back(Cl.g.total);
    if (outs.size() >= 2) tmpA = std::max(tmpA, outs[0]);
    if (outs.size() >= 3) tmpB = std::max(tmpB, outs[1]);
  }
  p->off_tmp = off;
  if (p->sep) {
    // horizontal factors after the x stage of a transfer that halves both directions
    size_t cols = 0;
    for (size_t l = 0; l + 1 < p->lv.size(); ++l)
      if (p->lv[l].hx && p->lv[l].hy)
        cols = std::max(cols, (size_t)make_grid(p->lv[l + 1].g.Nx, p->lv[l].g.Ny, 1).PP);
    p->tmp_bytes = align256(kHF * cols * 8);
    off = align256(off + p->tmp_bytes);
  } else {
    // stage outputs in the tiled operator layout (28 slots per node, 27 used)
    p->tmp_bytes = align256(kPlanes * tmpA * 8);
    off = align256(off + p->tmp_bytes + kPlanes * tmpB * 8);
  }
  p->n_coarse = (int)nc;
  // the inverse, then the blocked Gauss-Jordan's panels (16 x 16 + 2 x 16 n)
  p->off_dense = off; off = align256(off + ((size_t)nc * nc + 256 + 32 * (size_t)nc) * 8);
  p->off_cfree = off; off = align256(off + (size_t)nc * 4);
  if (o.accel == MCWIND_ACCEL_CG) {
    const size_t t0 = (size_t)p->lv[0].g.total;
    p->off_cg = off;
    off = align256(off + 6 * align256(t0 * 8));
  }
  {
    const size_t nodes = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
    p->off_xyz2 = off;
    off = align256(off + 3 * nodes * sizeof(float2));
    p->off_u2 = off;  // nodal u0 as float pairs: [k][j][i], or the split layout (separable)
    off = align256(off + 3 * std::max(nodes, (size_t)p->lv[0].g.total) * sizeof(float2));
  }
  p->n_adj = adjoint_partials(nx, ny, nz);
  p->off_adj = off;
  off = align256(off + (6 * (size_t)p->n_adj + 8) * 8);
  p->n_partials = 2 * max_blocks;
  p->off_partials = off; off = align256(off + (size_t)p->n_partials * 8);
  p->off_scalars = off; off = align256(off + 256);
  p->ws_bytes = off;
  *out = p;
  if (workspace_bytes) *workspace_bytes = off;
  return MCWIND_OK;
}

extern "C" int mcwind_plan_query(mcwind_plan p, mcwind_options* opt, size_t* workspace_bytes) {
  if (!p) return MCWIND_EINVAL;
  if (opt) {
    *opt = p->opt;
    opt->cycles_per_check = effective_cycles_per_check(p->opt);
  }
  if (workspace_bytes) *workspace_bytes = p->ws_bytes;
  return MCWIND_OK;
}

extern "C" int mcwind_plan_num_levels(mcwind_plan p) {
  return p ? (int)p->lv.size() : MCWIND_EINVAL;
}

extern "C" int mcwind_plan_level(mcwind_plan p, int level, int dims[3], int* hx, int* hy,
                                 int* kmap) {
  if (!p || level < 0 || level >= (int)p->lv.size()) return MCWIND_EINVAL;
  const Level& L = p->lv[level];
  if (dims) { dims[0] = L.g.Nx; dims[1] = L.g.Ny; dims[2] = L.g.Nz; }
  const bool last = level + 1 == (int)p->lv.size();
  if (hx) *hx = last ? 0 : L.hx;
  if (hy) *hy = last ? 0 : L.hy;
  if (kmap && !last)
    for (size_t K = 0; K < L.kmap.size(); ++K) kmap[K] = L.kmap[K];
  return MCWIND_OK;
}
