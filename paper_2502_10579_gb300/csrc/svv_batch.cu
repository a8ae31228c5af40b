// svv_batch.cu -- many queries in one persistent launch.
//
// The cooperative grid is split into teams of `team_blocks` CTAs.  A team's
// leader takes the next instance from the device work queue (one atomic
// ticket), and the whole team runs the instance's pipeline -- intersection
// solve, union solve, stable compaction + subgraph extraction, then per slab
// the multi-snapshot relaxation and the scatter -- separated by the team's own
// bounded barrier, with the team's own scratch.  Instances of different types
// and window lengths run side by side, so one query's small frontier rounds
// overlap with another query's large ones.  In serving mode the queue grows
// while the kernel runs: the host appends instances and raises a tail index in
// host-mapped memory; an idle team waits for work with a bounded sleep and the
// kernel ends after `idle_ns` without work (the host relaunches it on the next
// arrival) or when the host sets the stop flag.
#include "svv_qrs.cuh"
#include "svv_relax.cuh"
#include "svv_solve.cuh"

namespace svv {

constexpr int kBatchThreads = 512;
constexpr uint32_t kNoInst = 0xFFFFFFFFu;
constexpr uint32_t kSlab = 128;

__device__ __forceinline__ void zero_phase(TeamCtl* p) {
  for (int k = 0; k < 3; ++k) {
    p->qn[k] = 0u;
    p->ticket[k] = 0u;
  }
  for (int k = 0; k < 14; ++k) p->aux[k] = 0u;
  p->err = 0u;
  p->iters = 0u;
  p->relaxed = 0ull;
}

// leader thread: next instance index, or kNoInst when the queue is done
__device__ uint32_t pick_instance(const BatchArgs& b) {
  if (!b.live_tail) {
    const uint32_t i = atomicAdd(b.next, 1u);
    return i < b.n_inst ? i : kNoInst;
  }
  const unsigned long long t0 = global_ns();
  unsigned ns = 256;
  for (;;) {
    const uint32_t tail = *b.live_tail;
    const uint32_t cur = ld_relaxed(b.next);  // no L1 drop per poll (other teams share the SM)
    if (cur < tail) {
      if (atomicCAS(b.next, cur, cur + 1u) == cur) {
        fence_acq_rel();
        return cur;
      }
      continue;
    }
    if (*b.live_stop) return kNoInst;
    if (global_ns() - t0 > b.idle_ns) return kNoInst;
    __nanosleep(ns);
    if (ns < 8192) ns <<= 1;
  }
}

// Out-of-line phase entry points: each phase keeps its own register
// allocation instead of the sum of all of them inlined into one body.
template <class Op, int PRED>
__device__ __noinline__ bool solve_nl(const SolveArgs a, const Team t, unsigned long long* stage) {
  return solve_team<Op, PRED>(a, t, stage);
}
__device__ __noinline__ bool qrs_nl(const QrsArgs a, const Team t) { return qrs_team(a, t); }
template <class Op, int P, int K>
__device__ __noinline__ bool relax_nl(const RelaxArgs a, const Team t, unsigned long long* stage) {
  return relax_team<Op, P, K>(a, t, stage);
}
__device__ __noinline__ void scatter_nl(const ScatterArgs a, const Team t, uint32_t* tile) {
  scatter_team(a, t, tile);
}

template <class Op>
__device__ bool run_instance(const BatchArgs& b, const BatchInstance& q, uint32_t i, const Team& t,
                             const TeamScratch& sc, TeamCtl* tc, unsigned long long* stage, uint32_t* tile) {
  SolveArgs a{};
  a.g = b.g;
  a.win = Window{q.wb, q.wl};
  a.source = q.source;
  a.stamp = sc.stamp;
  a.q0 = sc.q0;
  a.q1 = sc.q1;
  a.qcap = sc.qcap;
  a.cshift = b.solve_cs;
  a.qerr = t.qerr;
  a.delta = (q.type == 0 || q.type == 1) ? b.delta[q.type] : 0u;
  const unsigned long long cap = a.delta ? 16ull * b.g.V + 64 : (unsigned long long)b.g.V + 2;
  a.maxit = b.maxit ? b.maxit : (uint32_t)min(cap, 0xFFFFFFF0ull);
  a.spin_ns = b.spin_ns;
  a.pull_units = b.pull_units;
  a.push_verts = b.push_verts;
  if (b.skip_same && sc.procv) {
    a.procv = sc.procv;
    a.pcap = b.g.V + (b.g.E >> b.solve_cs) + 2u;
  }

  // intersection graph
  a.init = kInitSource;
  a.val = sc.rI;
  a.ctl = tc + 1;
  a.skip_nf = (q.wb == 0 && q.wl == b.g.S) ? 1 : 0;
  if (!solve_nl<Op, kPredAll>(a, t, stage)) return false;
  // union graph, incrementally
  a.init = kInitSeed;
  a.base = sc.rI;
  a.val = sc.rU;
  a.ctl = tc + 2;
  a.skip_nf = 0;
  if (!solve_nl<Op, kPredAny>(a, t, stage)) return false;
  // stable compaction + subgraph
  QrsArgs r{};
  r.g = b.g;
  r.win = Window{q.wb, q.wl};
  r.QW = (q.wl + 63u) / 64u;
  r.prune = 1;
  r.rI = sc.rI;
  r.rU = sc.rU;
  r.row = sc.row;
  r.uv = sc.uv;
  r.part = sc.part;
  r.units = sc.units;
  r.ucap = sc.ucap;
  r.cshift = b.qrs_cs;
  r.qcnt = sc.qcnt;
  r.qrow = sc.qrow;
  r.cur = sc.cur;
  r.qcw = sc.qcw;
  r.qmask = sc.qmask;
  r.ecap = sc.ecap;
  r.mcap = sc.mcap;
  r.rowcap = b.g.V;
  r.ctl = tc + 3;
  r.qerr = t.qerr;
  r.spin_ns = b.spin_ns;
  if (!qrs_nl(r, t)) return false;
  if (!t.sync()) return false;
  // relaxation + scatter per slab
  for (uint32_t s0 = 0; s0 < q.wl; s0 += kSlab) {
    const uint32_t ls = min(kSlab, q.wl - s0);
    uint32_t P, K;
    if (ls <= 8) { P = 8; K = 1; }
    else if (ls <= 16) { P = 16; K = 1; }
    else if (ls <= 32) { P = 32; K = 1; }
    else if (ls <= 64) { P = 32; K = 2; }
    else { P = 32; K = 4; }
    if (s0 > 0) {
      if (t.rank == 0 && threadIdx.x == 0) zero_phase(tc + 4);
      if (!t.sync()) return false;
    }
    RelaxArgs x{};
    x.g = b.g;
    x.win = Window{q.wb, q.wl};
    x.s0 = s0;
    x.ls = ls;
    x.QW = r.QW;
    x.rI = sc.rI;
    x.row = sc.row;
    x.uv = sc.uv;
    x.qrow = sc.qrow;
    x.qcw = sc.qcw;
    x.qmask = sc.qmask;
    x.counts = &(tc + 3)->aux[0];
    x.val = sc.val;
    x.LP = P * K;
    x.stamp = sc.stamp;
    x.q0 = sc.q0;
    x.q1 = sc.q1;
    x.qcap = sc.qcap;
    x.cshift = b.relax_cs;
    x.ctl = tc + 4;
    x.qerr = t.qerr;
    x.maxit = b.maxit ? b.maxit : b.g.V + 2u;
    x.spin_ns = b.spin_ns;
    bool ok;
    if (P == 8) ok = relax_nl<Op, 8, 1>(x, t, stage);
    else if (P == 16) ok = relax_nl<Op, 16, 1>(x, t, stage);
    else if (K == 1) ok = relax_nl<Op, 32, 1>(x, t, stage);
    else if (K == 2) ok = relax_nl<Op, 32, 2>(x, t, stage);
    else ok = relax_nl<Op, 32, 4>(x, t, stage);
    if (!ok) return false;
    ScatterArgs o{};
    o.V = b.g.V;
    o.s0 = s0;
    o.ls = ls;
    o.rI = sc.rI;
    o.row = sc.row;
    o.val = sc.val;
    o.LP = P * K;
    o.out = q.out;
    o.qerr = t.qerr;
    scatter_nl(o, t, tile);
    if (!t.sync()) return false;
  }
  return true;
}

__global__ void __launch_bounds__(kBatchThreads, 2) batch_kernel(BatchArgs b) {
  __shared__ unsigned long long s_stage[(kBatchThreads / 32) * kStageUnits];
  __shared__ uint32_t s_tile[kSlab * (kScatterTV + 1)];
  const unsigned team = blockIdx.x / b.team_blocks, rank = blockIdx.x % b.team_blocks;
  TeamCtl* tc = b.ctl + (size_t)team * kBatchCtl;
  const TeamScratch sc = b.scratch[team];
  const Team base{tc, nullptr, b.team_blocks, rank, b.spin_ns};
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) {
      const uint32_t id = pick_instance(b);
      tc->aux[0] = id;
      for (int p = 1; p < kBatchCtl; ++p) zero_phase(tc + p);
      if (id != kNoInst) b.t_start[b.ring ? id % b.ring : id] = global_ns();
    }
    if (!base.sync()) return;
    const uint32_t id = cta_read(&tc->aux[0]);
    if (id == kNoInst) return;
    const uint32_t i = b.ring ? id % b.ring : id;  // slot of the instance
    const BatchInstance q = b.inst[i];
    Team t = base;
    t.qerr = b.qerr + i;
    bool ok;
    if (q.type == 0) ok = run_instance<OpSSSP>(b, q, i, t, sc, tc, s_stage, s_tile);
    else if (q.type == 1) ok = run_instance<OpSSWP>(b, q, i, t, sc, tc, s_stage, s_tile);
    else if (q.type == 3) ok = run_instance<OpSSNP>(b, q, i, t, sc, tc, s_stage, s_tile);
    else ok = run_instance<OpBFS>(b, q, i, t, sc, tc, s_stage, s_tile);
    if (rank == 0 && threadIdx.x == 0) {
      b.t_end[i] = global_ns();
      __threadfence_system();
      b.done[i] = 1u;
      __threadfence_system();
    }
    // a failed instance may have left the team's barrier mid-round: the team
    // stops and the other teams take the remaining instances
    if (!ok) return;
  }
}

cudaError_t launch_batch(const BatchArgs& b, LaunchCfg cfg, cudaStream_t s) {
  BatchArgs copy = b;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)batch_kernel, dim3(cfg.blocks), dim3(cfg.threads), args, 0, s);
}

// Local memory the driver reserves for the batch kernel's stack frames when it
// first runs: the frame of every thread the device can hold at once.
uint64_t batch_local_bytes(int device) {
  cudaFuncAttributes fa{};
  int sms = 0, per_sm = 0;
  if (cudaFuncGetAttributes(&fa, (const void*)batch_kernel) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (uint64_t)fa.localSizeBytes * (uint64_t)per_sm * (uint64_t)sms;
}

int occupancy_batch(int threads) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void*)batch_kernel, threads, 0) != cudaSuccess)
    return 0;
  return n;
}

}  // namespace svv
