// svv_solve.cu -- single-value frontier solve, used for
//   * the intersection-graph bound (Section 3 Step 1; Algorithm 1 Compute(G_cap)):
//     edges present in every window snapshot, from the source;
//   * the union-graph bound, computed incrementally from the intersection
//     values as Section 6.2 describes: seed with the edges present in some but
//     not all window snapshots, then relax every edge present in any;
//   * the plain per-snapshot recompute (Fig. 2a): edges present in one snapshot.
//
// One persistent cooperative launch runs every frontier round; rounds are
// separated by a bounded team barrier instead of host round trips.  Work is a
// queue of units (vertex, chunk of 2^cshift edges), so a hub's edges spread over
// many warps.  A warp takes up to 32 units at a time (fewer when the frontier
// is small, so every warp gets work), prefix-sums their edge counts and walks
// the concatenated edge list two 32-edge steps at a time, so lanes stay busy
// whatever the degree mix and each lane keeps two load chains in flight.  Relaxation is atomicMin/atomicMax; a vertex joins
// the next frontier once per round (stamp dedupe).
#include "svv_solve.cuh"

namespace svv {

constexpr int kSolveThreads = 512;

template <class Op, int PRED>
__global__ void __launch_bounds__(kSolveThreads, 3) solve_kernel(SolveArgs a) {
  __shared__ unsigned long long s_stage[(kSolveThreads / 32) * kStageUnits];
  const Team t{a.ctl, a.qerr, gridDim.x, blockIdx.x, a.spin_ns};
  solve_team<Op, PRED>(a, t, s_stage);
}

template <class Op, int PRED>
static cudaError_t launch_one(const SolveArgs& a, LaunchCfg cfg, cudaStream_t s) {
  SolveArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)solve_kernel<Op, PRED>, dim3(cfg.blocks),
                                     dim3(cfg.threads), args, 0, s);
}

template <class Op>
static cudaError_t launch_pred(int pred, const SolveArgs& a, LaunchCfg cfg, cudaStream_t s) {
  switch (pred) {
    case kPredAll: return launch_one<Op, kPredAll>(a, cfg, s);
    case kPredAny: return launch_one<Op, kPredAny>(a, cfg, s);
    default: return launch_one<Op, kPredBit>(a, cfg, s);
  }
}

cudaError_t launch_solve(int type, int pred, const SolveArgs& a, LaunchCfg cfg, cudaStream_t s) {
  switch (type) {
    case 0: return launch_pred<OpSSSP>(pred, a, cfg, s);
    case 1: return launch_pred<OpSSWP>(pred, a, cfg, s);
    case 3: return launch_pred<OpSSNP>(pred, a, cfg, s);
    default: return launch_pred<OpBFS>(pred, a, cfg, s);
  }
}

int occupancy_solve(int threads) {
  int best = 1 << 30;
  const void* ks[] = {
      (const void*)solve_kernel<OpSSSP, kPredAll>, (const void*)solve_kernel<OpSSSP, kPredAny>,
      (const void*)solve_kernel<OpSSSP, kPredBit>, (const void*)solve_kernel<OpSSWP, kPredAll>,
      (const void*)solve_kernel<OpSSWP, kPredAny>, (const void*)solve_kernel<OpSSWP, kPredBit>,
      (const void*)solve_kernel<OpBFS, kPredAll>,  (const void*)solve_kernel<OpBFS, kPredAny>,
      (const void*)solve_kernel<OpBFS, kPredBit>,  (const void*)solve_kernel<OpSSNP, kPredAll>,
      (const void*)solve_kernel<OpSSNP, kPredAny>, (const void*)solve_kernel<OpSSNP, kPredBit>};
  for (const void* k : ks) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, 0) != cudaSuccess) return 0;
    best = n < best ? n : best;
  }
  return best;
}

}  // namespace svv
