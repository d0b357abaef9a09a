// Device side of the batched solve of many independent domains: the
// convergence bookkeeping that lets one CUDA graph run the whole solve.
//
// The graph is: per-domain set-up (load vector, its norm, first iterate,
// first float64 residual), then k_batch_step(init), then a conditional WHILE
// node whose body holds one conditional IF node per domain (that domain's
// cycles, refinement update and float64 residual) followed by
// k_batch_step(check), then the per-domain output.  k_batch_step reads every
// domain's norms from its plan's device scalars, records the relative
// residual, decides which domains iterate again and sets the IF handles and
// the WHILE handle itself; the loop ends when no domain is above the
// tolerance or the cycle limit is reached, so it is bounded by construction.
#include "async.cuh"
#include "kernels.cuh"

namespace mcw {
namespace {

__global__ void __launch_bounds__(256) k_batch_step(BatchDev b, int phase, double rtol,
                                                    int max_checks, int cpc) {
  __shared__ int any_active;
  __shared__ int it_sh;
  if (threadIdx.x == 0) {
    any_active = 0;
    it_sh = phase == 0 ? 0 : *b.iter + 1;
  }
  __syncthreads();
  const int it = it_sh;
  const int c = it * cpc;
  for (int d = threadIdx.x; d < b.n; d += blockDim.x) {
    const double f2 = b.scal[d][0], r2 = b.scal[d][1];
    const double nf = sqrt(f2);
    const double rel = nf > 0.0 ? sqrt(r2) / nf : 0.0;
    b.status[d] = *b.pstat[d];
    if (phase == 0) {
      b.cycles[d] = 0;
      b.nf[d] = nf;
      b.hist[(int64_t)d * MCWIND_HIST] = rel;
      const bool finite = isfinite(nf) && isfinite(r2);
      b.active[d] = finite && rel > rtol ? 1 : 0;
      b.nonfinite[d] = finite ? 0 : 1;
    } else if (b.active[d]) {
      b.hist[(int64_t)d * MCWIND_HIST + c] = rel;
      b.cycles[d] = c;
      b.active[d] = isfinite(rel) && rel > rtol ? 1 : 0;
    }
    if (b.active[d]) atomicOr(&any_active, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *b.iter = it;
    // one thread sets every handle (concurrent sets are not allowed)
    for (int d = 0; d < b.n; ++d) cudaGraphSetConditional(b.h_if[d], b.active[d] ? 1u : 0u);
    cudaGraphSetConditional(b.h_while, (any_active && it + 1 <= max_checks) ? 1u : 0u);
  }
}

// One block waits on an mbarrier that nothing arrives on, with the bounded
// wait of the solver's kernels: the wait runs out after limit_ns, sets the
// status bit and the kernel returns.
__global__ void k_wait_selftest(int* status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) wait_parity(&bar, 0u, status, limit_ns);
}

}  // namespace

cudaError_t launch_wait_selftest(int* status, unsigned long long limit_ns, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(status, limit_ns);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_batch_step(const BatchDev& b, int phase, double rtol, int max_checks, int cpc,
                              cudaStream_t st) {
  k_batch_step<<<1, 256, 0, st>>>(b, phase, rtol, max_checks, cpc);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace mcw
