// svv_qrs.cu -- stable-vertex compaction and Q-relevant subgraph extraction.
//
// Section 3 Step 2 (Theorem 2): v is stable iff its intersection-graph and
// union-graph values agree; Algorithm 1 collects those into `found`.
// Section 3 Steps 3-4 and Algorithm 1 RemoveIncomingEdges /
// RemoveDeltaAdditionBatches: the in-edges of stable vertices, and the
// additions whose sink is stable, are dropped.  As Section 6.2 does, the
// subgraph is built "in reverse": only in-edges of unstable vertices are
// gathered.  Stable sources keep no rows: their value is final, so their edges
// into unstable vertices only matter once, in the seeding pass of the
// relaxation (which reads the addition edges directly).  The kept edges are
// those whose source and target are both unstable and that are present in at
// least one window snapshot; per row, edges present in every window snapshot
// come first (Section 4.1), followed by the rest with masks rebased so that bit
// i is snapshot win_begin+i.
//
// One cooperative launch, five phases separated by the team barrier:
//   P1 per-CTA counts of unstable vertices and their work units;
//   P2 rows in vertex order (CTA offsets from P1), row -> vertex map, units;
//   P3 per-row edge counts (all-window / masked);
//   P4 exclusive scan of the row counts -> row descriptors and fill cursors;
//   P5 fill.
#include "svv_qrs.cuh"

namespace svv {

constexpr int kQrsThreads = 512;

__global__ void __launch_bounds__(kQrsThreads) qrs_kernel(QrsArgs a) {
  const Team t{a.ctl, a.qerr, gridDim.x, blockIdx.x, a.spin_ns};
  qrs_team(a, t);
}

cudaError_t launch_qrs(const QrsArgs& a, LaunchCfg cfg, cudaStream_t s) {
  QrsArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)qrs_kernel, dim3(cfg.blocks), dim3(cfg.threads),
                                     args, 0, s);
}

int occupancy_qrs(int threads) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void*)qrs_kernel, threads, 0) !=
      cudaSuccess)
    return 0;
  return n;
}

}  // namespace svv
