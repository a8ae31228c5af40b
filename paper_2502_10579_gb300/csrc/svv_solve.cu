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
// many warps.  A warp takes 32 units at a time, prefix-sums their edge counts
// and walks the concatenated edge list 32 edges per step, so lanes stay busy
// whatever the degree mix.  Relaxation is atomicMin/atomicMax; a vertex joins
// the next frontier once per round (stamp dedupe).
#include "svv_device.cuh"
#include "svv_push.cuh"

namespace svv {

constexpr int kSolveThreads = 512;

template <class Op, int PRED>
__global__ void __launch_bounds__(kSolveThreads) solve_kernel(SolveArgs a) {
  const DevGraph& g = a.g;
  TeamCtl* c = a.ctl;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned nthreads = gridDim.x * blockDim.x;
  const unsigned gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned gwarp = gtid >> 5, nwarps = nthreads >> 5;
  if (a.qerr && ld_acquire(a.qerr) != 0u) return;

  // round 0: starting values and stamps
  if (a.init == kInitSource) {
    for (uint32_t v = gtid; v < g.V; v += nthreads) {
      a.val[v] = Op::kIdentity;
      a.stamp[v] = 0u;
    }
  } else {
    for (uint32_t v = gtid; v < g.V; v += nthreads) {
      a.val[v] = a.base[v];
      a.stamp[v] = 0u;
    }
  }
  if (!team_sync(c, a.qerr, gridDim.x, a.spin_ns)) return;

  // round 0: first frontier (stamp 1, queue q1, count qn[1])
  if (a.init == kInitSource) {
    if (gwarp == 0) {
      uint32_t deg = 0;
      if (lane == 0) {
        a.val[a.source] = Op::kSource;
        a.stamp[a.source] = 1u;
        deg = g.rp[a.source + 1] - g.rp[a.source];
      }
      warp_push_units(lane == 0, a.source, deg, a.cshift, a.q1, &c->qn[1], a.qcap, c, a.qerr, lane);
    }
  } else {
    // edges present in some but not all window snapshots (the window's
    // addition batches); intersection edges cannot improve a fixed point of
    // the intersection graph, so they are skipped
    for (uint32_t k0 = gwarp * 32u; k0 < g.NF; k0 += nwarps * 32u) {
      const uint32_t k = k0 + lane;
      bool push = false;
      uint32_t x = 0, deg = 0;
      if (k < g.NF) {
        bool any, all;
        window_any_all(g.nfmask + (size_t)k * g.W, a.win, any, all);
        if (any && !all) {
          const uint32_t u = __ldg(g.nfsrc + k);
          const uint2 e = __ldg(g.nfcw + k);
          x = e.x;
          const uint32_t cand = Op::relax(ld_cg(a.val + u), e.y);
          if (Op::better(cand, ld_cg(a.val + x))) {
            const uint32_t old = Op::atomic(a.val + x, cand);
            if (Op::better(cand, old) && atomicExch(a.stamp + x, 1u) != 1u) {
              push = true;
              deg = g.rp[x + 1] - g.rp[x];
            }
          }
        }
      }
      warp_push_units(push, x, deg, a.cshift, a.q1, &c->qn[1], a.qcap, c, a.qerr, lane);
    }
  }
  if (!team_sync(c, a.qerr, gridDim.x, a.spin_ns)) return;

  unsigned long long relaxed = 0;
  uint32_t it = 1;
  for (;; ++it) {
    const uint32_t cur = it % 3u, nxt = (it + 1u) % 3u, clr = (it + 2u) % 3u;
    uint32_t n = ld_acquire(&c->qn[cur]);
    if (n == 0u) break;
    if (it > a.maxit) {
      if (gtid == 0) set_err(c, a.qerr, kErrTimeout);
      break;
    }
    n = min(n, a.qcap);
    if (gtid == 0) {
      atomicExch(&c->qn[clr], 0u);
      atomicExch(&c->ticket[clr], 0u);
    }
    const unsigned long long* qin = (it & 1u) ? a.q1 : a.q0;
    unsigned long long* qout = (it & 1u) ? a.q0 : a.q1;
    unsigned* qn_out = &c->qn[nxt];
    const uint32_t stamp_next = it + 1u;

    for (;;) {
      uint32_t t0 = 0;
      if (lane == 0) t0 = atomicAdd(&c->ticket[cur], 32u);
      t0 = __shfl_sync(kFullMask, t0, 0);
      if (t0 >= n) break;
      const uint32_t ui = t0 + lane;
      uint32_t beg = 0, cnt = 0, fe = 0, nfb = 0, sv = Op::kIdentity;
      if (ui < n) {
        const unsigned long long u = ld_cg(qin + ui);
        const uint32_t v = (uint32_t)u, ch = (uint32_t)(u >> 32);
        const uint32_t r0 = __ldg(g.rp + v), r1 = __ldg(g.rp + v + 1);
        const uint32_t nf0 = __ldg(g.nfp + v), nf1 = __ldg(g.nfp + v + 1);
        fe = r1 - (nf1 - nf0);
        nfb = nf0;
        beg = r0 + (ch << a.cshift);
        uint32_t end = min(r1, beg + (1u << a.cshift));
        if (PRED == kPredAll && a.skip_nf) end = min(end, fe);
        cnt = end > beg ? end - beg : 0u;
        sv = ld_cg(a.val + v);
      }
      const uint32_t incl = warp_incl_scan(cnt, lane);
      const uint32_t total = __shfl_sync(kFullMask, incl, 31);
      if (lane == 0) relaxed += total;
      for (uint32_t p0 = 0; p0 < total; p0 += 32u) {
        const uint32_t p = p0 + lane;
        const int k = warp_owner(incl, p < total ? p : total - 1u);
        const uint32_t ik = __shfl_sync(kFullMask, incl, k);
        const uint32_t ck = __shfl_sync(kFullMask, cnt, k);
        const uint32_t bk = __shfl_sync(kFullMask, beg, k);
        const uint32_t fk = __shfl_sync(kFullMask, fe, k);
        const uint32_t nk = __shfl_sync(kFullMask, nfb, k);
        const uint32_t sk = __shfl_sync(kFullMask, sv, k);
        bool push = false;
        uint32_t x = 0, deg = 0;
        if (p < total) {
          const uint32_t e = bk + (p - (ik - ck));
          const uint2 ew = __ldg(g.cw + e);
          x = ew.x;
          bool present = true;
          if (e >= fk) {
            const uint64_t* m = g.nfmask + (size_t)(nk + (e - fk)) * g.W;
            if (PRED == kPredAll) present = window_all(m, a.win);
            else if (PRED == kPredAny) present = window_any(m, a.win);
            else present = mask_bit(m, a.bit);
          }
          if (present) {
            const uint32_t cand = Op::relax(sk, ew.y);
            if (Op::better(cand, ld_cg(a.val + x))) {
              const uint32_t old = Op::atomic(a.val + x, cand);
              if (Op::better(cand, old) && atomicExch(a.stamp + x, stamp_next) != stamp_next) {
                push = true;
                deg = __ldg(g.rp + x + 1) - __ldg(g.rp + x);
              }
            }
          }
        }
        warp_push_units(push, x, deg, a.cshift, qout, qn_out, a.qcap, c, a.qerr, lane);
      }
    }
    if (!team_sync(c, a.qerr, gridDim.x, a.spin_ns)) return;
  }
  if (lane == 0 && relaxed) atomicAdd(&c->relaxed, relaxed);
  if (gtid == 0) c->iters = it - 1u;
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
      (const void*)solve_kernel<OpBFS, kPredBit>};
  for (const void* k : ks) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, 0) != cudaSuccess) return 0;
    best = n < best ? n : best;
  }
  return best;
}

}  // namespace svv
