// svv_solve.cuh -- the single-value frontier solve as a team phase.
#pragma once

#include "svv_device.cuh"
#include "svv_push.cuh"
#include "svv_team.cuh"

namespace svv {


// Near-far ordering key of a value: larger = closer to the source, so one
// atomicMax per round finds the frontier's best value for both lattices.
template <class Op>
__device__ __forceinline__ uint32_t nf_key(uint32_t v) {
  return Op::better(0u, 1u) ? ~v : v;
}

template <class Op, int PRED>
__device__ bool solve_team(const SolveArgs& a, const Team& t, unsigned long long* stage) {
  const DevGraph& g = a.g;
  TeamCtl* c = a.ctl;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned nthreads = t.nthreads();
  const unsigned gtid = t.tid();
  const unsigned gwarp = gtid >> 5, nwarps = nthreads >> 5;
  if (a.qerr && cta_read(a.qerr) != 0u) return false;
  PushStage st{stage + (threadIdx.x >> 5) * kStageUnits, 0u};

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
  // no chunk has been relaxed yet: the identity is never a queued value
  if (a.procv)
    for (uint32_t k = gtid; k < a.pcap; k += nthreads) a.procv[k] = Op::kIdentity;
  if (a.skip_arrival && t.rank + 1u == a.skip_arrival) return false;  // test hook: never arrives
  if (!t.sync()) return false;
  if (a.trace && gtid == 0 && a.trace_cap) a.trace[0] = global_ns() & 0xFFFFFFFFFFull;

  // round 0: first frontier (stamp 1, queue q1, count qn[1])
  if (a.init == kInitSource) {
    if (gwarp == 0) {
      uint32_t deg = 0;
      if (lane == 0) {
        a.val[a.source] = Op::kSource;
        a.stamp[a.source] = 1u;
        deg = g.rp[a.source + 1] - g.rp[a.source];
      }
      stage_push_units(lane == 0, a.source, deg, a.cshift, st, a.q1, &c->qn[1], a.qcap, c, a.qerr, lane);
      if (lane == 0) atomicMax(&c->aux[1], nf_key<Op>(Op::kSource));
    }
  } else {
    // edges present in some but not all window snapshots (the window's
    // addition batches); intersection edges cannot improve a fixed point of
    // the intersection graph, so they are skipped
    for (uint32_t k0 = gwarp * 32u; k0 < g.NF; k0 += nwarps * 32u) {
      const uint32_t k = k0 + lane;
      bool push = false;
      uint32_t x = 0, deg = 0, cand = 0;
      if (k < g.NF) {
        bool any, all;
        window_any_all(g.nfmask + (size_t)k * g.W, a.win, any, all);
        if (any && !all) {
          const uint32_t u = __ldg(g.nfsrc + k);
          const uint2 e = __ldg(g.nfcw + k);
          x = e.x;
          cand = Op::relax(ld_val(a.val + u), e.y);
          if (Op::better(cand, ld_val(a.val + x))) {
            Op::red(a.val + x, cand);
            const uint32_t r0 = __ldg(g.rp + x), r1 = __ldg(g.rp + x + 1);
            if (atomicExch(a.stamp + x, 1u) != 1u) {
              push = true;
              deg = r1 - r0;
            }
          }
        }
      }
      stage_push_units(push, x, deg, a.cshift, st, a.q1, &c->qn[1], a.qcap, c, a.qerr, lane);
      warp_fold_max(push, nf_key<Op>(cand), &c->aux[1], lane);
    }
  }
  stage_flush_cta(st, a.q1, &c->qn[1], a.qcap, c, a.qerr, lane);
  if (!t.sync()) return false;

  unsigned long long relaxed = 0;
  uint32_t it = 1;
  for (;; ++it) {
    const uint32_t cur = it % 3u, nxt = (it + 1u) % 3u, clr = (it + 2u) % 3u;
    const bool far_on = a.delta != 0u;
    uint32_t n, slot;
    cta_read2(&c->qn[cur], far_on ? &c->aux[cur] : nullptr, n, slot);
    if (a.trace && gtid == 0 && it < a.trace_cap) a.trace[it] = ((unsigned long long)n << 40) | (global_ns() & 0xFFFFFFFFFFull);
    if (n == 0u) break;
    if (it > a.maxit) {
      if (gtid == 0) set_err(c, a.qerr, kErrTimeout);
      break;
    }
    n = min(n, a.qcap);
    // How this round runs.  After a push round the frontier is a unit queue of
    // n units; after a pull round it is the n vertices stamped with `it`.  A
    // large frontier is pulled: every vertex takes the best candidate over
    // its in-edges (no queue, one atomic per chunk); a small one is pushed.
    const bool dense = cta_read(&c->aux[3 + cur]) != 0u;
    const bool can_pull = g.ifd != nullptr && a.pull_units != 0u;
    const bool pull = can_pull && (dense ? (n > a.push_verts) : (n > a.pull_units));
    if (gtid == 0) {
      atomicExch(&c->qn[clr], 0u);
      atomicExch(&c->ticket[clr], 0u);
      atomicExch(&c->aux[clr], 0u);
      atomicExch(&c->aux[3 + nxt], pull ? 1u : 0u);
      atomicExch(&c->aux[6 + ((it + 1u) & 1u)], 0u);  // compaction counter of the next round
    }
    unsigned long long* qin = (it & 1u) ? a.q1 : a.q0;
    unsigned long long* qout = (it & 1u) ? a.q0 : a.q1;
    unsigned* qn_out = &c->qn[nxt];
    const uint32_t stamp_next = it + 1u;

    if (pull) {
      // ---- pull round: one pass over every in-edge, edge-flat.  A warp
      // takes 128 consecutive in-edges (4 per lane, all loads issued before
      // any reduction); lanes with the same target fold their candidates and
      // the lowest of them updates the target.
      uint32_t changed = 0, scanned = 0;
      // BFS from the source: round `it` sets level `it` exactly when it only
      // takes in-neighbours of level it-1; then every level already set is
      // final and a visited target skips its in-edges (bottom-up BFS)
      const bool bottom_up = Op::kLevels && a.init == kInitSource;
      const uint32_t EF = g.E - g.NF;
      const uint32_t ntot = EF + ((PRED == kPredAll && a.skip_nf) ? 0u : g.NF);
      const uint32_t nchunks = (ntot + 127u) >> 7;
      for (uint32_t ch = gwarp; ch < nchunks; ch += nwarps) {
        uint32_t d[4], src[4], w[4];
        bool live[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t idx = (ch << 7) + 32u * j + lane;
          live[j] = idx < ntot;
          d[j] = 0xFFFFFFFFu - lane;  // unique per lane when not live
          src[j] = 0;
          w[j] = 0;
          if (live[j]) d[j] = idx < EF ? ld_stream(g.ifd + idx) : ld_stream(g.ipd + (idx - EF));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t idx = (ch << 7) + 32u * j + lane;
          if (live[j] && bottom_up && ld_val(a.val + d[j]) != kInf) live[j] = false;
          if (live[j]) {
            if (idx < EF) {
              const uint2 sw = ld_stream(g.ifcw + idx);
              src[j] = sw.x;
              w[j] = sw.y;
            } else {
              const uint32_t k = idx - EF;
              const uint64_t* m = g.ipmask + (size_t)k * g.W;
              bool present;
              if (PRED == kPredAll) present = window_all(m, a.win);
              else if (PRED == kPredAny) present = window_any(m, a.win);
              else present = mask_bit(m, a.bit);
              const uint2 sw = ld_stream(g.ipcw + k);
              src[j] = sw.x;
              w[j] = sw.y;
              live[j] = present;
            }
          }
        }
        // the lowest lane of each target's run loads the target's value now,
        // alongside the source gathers, instead of after the fold
        uint32_t cand[4], tv[4];
        unsigned lead = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const unsigned grp = __match_any_sync(kFullMask, d[j]);
          const uint32_t idx = (ch << 7) + 32u * j + lane;
          const bool ld = idx < ntot && lane == (unsigned)(__ffs(grp) - 1);
          lead |= (ld ? 1u : 0u) << j;
          tv[j] = ld ? ld_val(a.val + d[j]) : 0u;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          cand[j] = Op::kIdentity;
          if (live[j]) {
            const uint32_t su = ld_val(a.val + src[j]);
            if (!bottom_up || su < it) cand[j] = Op::relax(su, w[j]);
          }
          scanned += __popc(__ballot_sync(kFullMask, live[j]));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const unsigned grp = __match_any_sync(kFullMask, d[j]);
          const uint32_t best =
              Op::better(0u, 1u) ? __reduce_min_sync(grp, cand[j]) : __reduce_max_sync(grp, cand[j]);
          if (((lead >> j) & 1u) && Op::better(best, tv[j])) {
            Op::red(a.val + d[j], best);
            // a plain store: the next round finds the changed vertices from
            // the stamps, so `changed` only needs to be zero exactly when
            // nothing changed (it may count a vertex more than once)
            a.stamp[d[j]] = stamp_next;
            ++changed;
          }
        }
      }
      if (lane == 0) relaxed += scanned;
      const uint32_t wc = __reduce_add_sync(kFullMask, changed);
      if (lane == 0 && wc) atomicAdd(qn_out, wc);
      if (!t.sync()) return false;
      continue;
    }
    if (dense) {
      // ---- the last round pulled: queue the vertices it changed (stamp == it)
      unsigned* cnt_ctr = &c->aux[6 + (it & 1u)];
      for (uint32_t v0 = gwarp * 32u; v0 < g.V; v0 += nwarps * 32u) {
        const uint32_t v = v0 + lane;
        const bool take = v < g.V && ld_cg(a.stamp + v) == it;
        const uint32_t deg = take ? (__ldg(g.rp + v + 1) - __ldg(g.rp + v)) : 0u;
        stage_push_units(take, v, deg, a.cshift, st, qin, cnt_ctr, a.qcap, c, a.qerr, lane);
      }
      stage_flush_cta(st, qin, cnt_ctr, a.qcap, c, a.qerr, lane);
      if (!t.sync()) return false;
      n = min(cta_read(cnt_ctr), a.qcap);
    }
    // near-far: relax only units whose value is within delta of the best
    // value queued for this round (that unit itself always qualifies, so every
    // round makes progress); the others are queued again unchanged
    uint32_t bound = 0;
    if (far_on) {
      if (Op::better(0u, 1u)) {
        const uint32_t best = ~slot;
        bound = best > kInf - a.delta ? kInf : best + a.delta;
      } else {
        bound = slot > a.delta ? slot - a.delta : 0u;
      }
    }

    // units per ticket: spread a small frontier over every warp, batch a
    // large one 32 units at a time
    const Batches bt{n, batch_size(n, nwarps, 32u), nwarps, gwarp, &c->ticket[cur]};
    const uint32_t tk = bt.tk;
    for (uint32_t t0 = bt.first(); t0 < n; t0 = bt.next(lane)) {
      const uint32_t ui = t0 + lane;
      uint32_t beg = 0, cnt = 0, fe = 0, nfb = 0, sv = Op::kIdentity;
      bool defer = false;
      uint32_t dv = 0, ddeg = 0;
      if (lane < tk && ui < n) {
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
        if (far_on && (Op::better(0u, 1u) ? sv > bound : sv < bound)) {
          // far: queue all of v's units again, once per round (stamp), and
          // skip this one now
          cnt = 0;
          if (atomicExch(a.stamp + v, stamp_next) != stamp_next) {
            defer = true;
            dv = v;
            ddeg = r1 - r0;
          }
        }
        if (a.procv && cnt) {
          // chunk ids v + rp[v]/C + ch are distinct across vertices; a
          // deferred chunk is not relaxed now, so it records nothing
          uint32_t* pv = a.procv + v + (r0 >> a.cshift) + ch;
          if (ld_cg(pv) == sv) cnt = 0;
          else *pv = sv;
        }
      }
      if (far_on) {
        stage_push_units(defer, dv, ddeg, a.cshift, st, qout, qn_out, a.qcap, c, a.qerr, lane);
        warp_fold_max(defer, nf_key<Op>(sv), &c->aux[nxt], lane);
      }
      const uint32_t incl = warp_incl_scan(cnt, lane);
      const uint32_t total = __shfl_sync(kFullMask, incl, 31);
      if (lane == 0) relaxed += total;
      // two 32-edge steps in flight per iteration: their loads, checks and
      // atomics are independent, so each lane keeps two chains going
      for (uint32_t p0 = 0; p0 < total; p0 += 64u) {
        bool push[2];
        uint32_t x[2], deg[2];
        uint32_t sk[2], ew_w[2];
        bool act[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const uint32_t p = p0 + 32u * j + lane;
          const int k = warp_owner(incl, p < total ? p : total - 1u);
          const uint32_t ik = __shfl_sync(kFullMask, incl, k);
          const uint32_t ck = __shfl_sync(kFullMask, cnt, k);
          const uint32_t bk = __shfl_sync(kFullMask, beg, k);
          const uint32_t fk = __shfl_sync(kFullMask, fe, k);
          const uint32_t nk = __shfl_sync(kFullMask, nfb, k);
          sk[j] = __shfl_sync(kFullMask, sv, k);
          push[j] = false;
          x[j] = 0;
          deg[j] = 0;
          act[j] = false;
          ew_w[j] = 0;
          if (p < total) {
            const uint32_t e = bk + (p - (ik - ck));
            const uint2 ew = __ldg(g.cw + e);
            x[j] = ew.x;
            ew_w[j] = ew.y;
            bool present = true;
            if (e >= fk) {
              const uint64_t* m = g.nfmask + (size_t)(nk + (e - fk)) * g.W;
              if (PRED == kPredAll) present = window_all(m, a.win);
              else if (PRED == kPredAny) present = window_any(m, a.win);
              else present = mask_bit(m, a.bit);
            }
            act[j] = present;
          }
        }
        uint32_t cand[2], curv[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          cand[j] = Op::relax(sk[j], ew_w[j]);
          curv[j] = act[j] ? ld_val(a.val + x[j]) : cand[j];
        }
        bool imp[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          imp[j] = act[j] && Op::better(cand[j], curv[j]);
          if (imp[j]) Op::red(a.val + x[j], cand[j]);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          if (imp[j]) {
            const uint32_t r0 = __ldg(g.rp + x[j]), r1 = __ldg(g.rp + x[j] + 1);
            if (atomicExch(a.stamp + x[j], stamp_next) != stamp_next) {
              push[j] = true;
              deg[j] = r1 - r0;
            }
          }
        }
        stage_push_units(push[0], x[0], deg[0], a.cshift, st, qout, qn_out, a.qcap, c, a.qerr, lane);
        stage_push_units(push[1], x[1], deg[1], a.cshift, st, qout, qn_out, a.qcap, c, a.qerr, lane);
        if (far_on) {
          const uint32_t k0v = push[0] ? nf_key<Op>(cand[0]) : 0u, k1v = push[1] ? nf_key<Op>(cand[1]) : 0u;
          warp_fold_max(push[0] || push[1], max(k0v, k1v), &c->aux[nxt], lane);
        }
      }
    }
    stage_flush_cta(st, qout, qn_out, a.qcap, c, a.qerr, lane);
    if (!t.sync()) return false;
  }
  if (lane == 0 && relaxed) atomicAdd(&c->relaxed, relaxed);
  if (gtid == 0) c->iters = it - 1u;
  return true;
}

}  // namespace svv
