// svv_group.cuh -- the bound solves of several queries in one set of frontier
// rounds (a query-oblivious frontier over a group of same-type queries).
//
// Section 4.2 relaxes every snapshot of a window with one frontier that does
// not tell snapshots apart, and cites work that shares one frontier between
// queries; this is that idea applied to the bound solves of Section 3 Step 1:
// up to KL queries of one type, each with its own source and its own window,
// keep their values side by side in one row per vertex (val[v*KL + k] is lane
// k's value of v).  A vertex joins the frontier when any lane improved, and a
// frontier vertex relaxes its out-edges for every lane in which the edge is
// present, so each round reads each edge once and ends at one team barrier for
// all the queries of the group.  Each lane computes exactly what the solve of
// its own query computes (the fixed point is per lane and unique), so lanes
// never change one another's values.
//
// Edge presence per lane: an edge present in every one of the S snapshots is
// present in every lane's intersection and union graph; for the others a
// per-edge lane word is computed once per group (group_lanes_kernel): bits
// 0..15 = lanes whose whole window holds the edge (intersection graph), bits
// 16..31 = lanes whose window holds it at least once (union graph).
#pragma once

#include "svv_device.cuh"
#include "svv_push.cuh"
#include "svv_team.cuh"

namespace svv {

// plain (L1-cacheable) load of a vertex's lane row; values only improve, so a
// stale row gives worse candidates (see ld_val)
template <int KL>
__device__ __forceinline__ void ld_row(const uint32_t* p, uint32_t (&r)[KL]) {
  if constexpr (KL == 2) {
    const uint2 x = *reinterpret_cast<const uint2*>(p);
    r[0] = x.x;
    r[1] = x.y;
  } else {
    const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int i = 0; i < KL / 4; ++i) {
      const uint4 x = q[i];
      r[4 * i] = x.x;
      r[4 * i + 1] = x.y;
      r[4 * i + 2] = x.z;
      r[4 * i + 3] = x.w;
    }
  }
}

template <int KL>
__device__ __forceinline__ void st_row(uint32_t* p, const uint32_t (&r)[KL]) {
  if constexpr (KL == 2) {
    *reinterpret_cast<uint2*>(p) = make_uint2(r[0], r[1]);
  } else {
    uint4* q = reinterpret_cast<uint4*>(p);
#pragma unroll
    for (int i = 0; i < KL / 4; ++i) q[i] = make_uint4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
  }
}

// lanes in which an edge takes part: every lane for an edge present in all S
// snapshots, else the intersection (PRED == kPredAll) or union half of its
// lane word
template <int PRED>
__device__ __forceinline__ uint32_t lanes_of(uint32_t word) {
  return PRED == kPredAll ? (word & 0xFFFFu) : (word >> 16);
}

// relax every lane of edge (u -> x, w) whose bit is set in `pm`, from the
// source row `su`, against the target row at `xr`; returns true if some lane
// of x was lowered (raised, for SSWP) by this edge
template <class Op, int KL>
__device__ __forceinline__ bool relax_lanes(const uint32_t (&su)[KL], uint32_t w, uint32_t pm, uint32_t* xr,
                                            uint32_t kinds) {
  uint32_t cur[KL];
  ld_row<KL>(xr, cur);
  bool imp = false;
#pragma unroll
  for (int k = 0; k < KL; ++k) {
    if ((pm >> k) & 1u) {
      const uint32_t cand = lane_relax<Op>(kinds, k, su[k], w);
      if (Op::better(cand, cur[k])) {
        Op::red(xr + k, cand);
        imp = true;
      }
    }
  }
  return imp;
}

template <class Op, int KL, int PRED>
__device__ bool group_solve_team(const GroupArgs& a, const Team& t, unsigned long long* stage) {
  const DevGraph& g = a.g;
  TeamCtl* c = a.ctl;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned nthreads = t.nthreads();
  const unsigned gtid = t.tid();
  const unsigned gwarp = gtid >> 5, nwarps = nthreads >> 5;
  if (a.qerr && cta_read(a.qerr) != 0u) return false;
  PushStage st{stage + (threadIdx.x >> 5) * kStageUnits, 0u};
  const uint32_t allmask = (1u << a.nlanes) - 1u;  // lanes in use (nlanes <= KL <= 8)

  // round 0: starting rows and stamps
  if (a.init == kInitSource) {
    uint32_t id[KL];
#pragma unroll
    for (int k = 0; k < KL; ++k) id[k] = Op::kIdentity;
    for (uint32_t v = gtid; v < g.V; v += nthreads) {
      st_row<KL>(a.val + (size_t)v * KL, id);
      a.stamp[v] = 0u;
    }
  } else {
    for (uint32_t v = gtid; v < g.V; v += nthreads) {
      uint32_t r[KL];
      ld_row<KL>(a.base + (size_t)v * KL, r);
      st_row<KL>(a.val + (size_t)v * KL, r);
      a.stamp[v] = 0u;
    }
  }
  if (!t.sync()) return false;
  if (a.trace && gtid == 0 && a.trace_cap) a.trace[0] = global_ns() & 0xFFFFFFFFFFull;

  // round 0: first frontier (stamp 1, queue q1, count qn[1])
  if (a.init == kInitSource) {
    if (gwarp == 0) {
      // every lane's source, queued once even when lanes share a source
      const bool mine = lane < a.nlanes;
      const uint32_t src = mine ? a.source[lane] : 0u;
      if (mine) a.val[(size_t)src * KL + lane] = Op::kSource;
      __syncwarp();
      bool push = false;
      uint32_t deg = 0;
      if (mine && atomicExch(a.stamp + src, 1u) != 1u) {
        push = true;
        deg = g.rp[src + 1] - g.rp[src];
      }
      stage_push_units(push, src, deg, a.cshift, st, a.q1, &c->qn[1], a.qcap, c, a.qerr, lane);
    }
  } else {
    // edges present in some but not all of a lane's window snapshots (that
    // lane's addition batches), from the intersection values of every lane
    for (uint32_t k0 = gwarp * 32u; k0 < g.NF; k0 += nwarps * 32u) {
      const uint32_t k = k0 + lane;
      bool push = false;
      uint32_t x = 0, deg = 0;
      if (k < g.NF) {
        const uint32_t lw = __ldg(a.nflanes + k);
        const uint32_t pm = (lw >> 16) & ~lw & allmask;  // any but not all
        if (pm) {
          const uint32_t u = __ldg(g.nfsrc + k);
          const uint2 e = __ldg(g.nfcw + k);
          x = e.x;
          uint32_t su[KL];
          ld_row<KL>(a.val + (size_t)u * KL, su);
          if (relax_lanes<Op, KL>(su, e.y, pm, a.val + (size_t)x * KL, a.kinds) && atomicExch(a.stamp + x, 1u) != 1u) {
            push = true;
            deg = __ldg(g.rp + x + 1) - __ldg(g.rp + x);
          }
        }
      }
      stage_push_units(push, x, deg, a.cshift, st, a.q1, &c->qn[1], a.qcap, c, a.qerr, lane);
    }
  }
  stage_flush_cta(st, a.q1, &c->qn[1], a.qcap, c, a.qerr, lane);
  if (!t.sync()) return false;

  unsigned long long relaxed = 0;
  uint32_t it = 1;
  for (;; ++it) {
    const uint32_t cur = it % 3u, nxt = (it + 1u) % 3u, clr = (it + 2u) % 3u;
    uint32_t n = cta_read(&c->qn[cur]);
    if (a.trace && gtid == 0 && it < a.trace_cap)
      a.trace[it] = ((unsigned long long)n << 40) | (global_ns() & 0xFFFFFFFFFFull);
    if (n == 0u) break;
    if (it > a.maxit) {
      if (gtid == 0) set_err(c, a.qerr, kErrTimeout);
      break;
    }
    n = min(n, a.qcap);
    // After a push round the frontier is a unit queue of n units; after a
    // pull round it is the n vertices stamped with `it`.  A large frontier is
    // pulled, a small one pushed.
    const bool dense = cta_read(&c->aux[3 + cur]) != 0u;
    const bool can_pull = g.ifd != nullptr && a.pull_units != 0u;
    const bool pull = can_pull && (dense ? (n > a.push_verts) : (n > a.pull_units));
    if (gtid == 0) {
      atomicExch(&c->qn[clr], 0u);
      atomicExch(&c->ticket[clr], 0u);
      atomicExch(&c->aux[3 + nxt], pull ? 1u : 0u);
      atomicExch(&c->aux[6 + ((it + 1u) & 1u)], 0u);  // compaction counter of the next round
    }
    unsigned long long* qin = (it & 1u) ? a.q1 : a.q0;
    unsigned long long* qout = (it & 1u) ? a.q0 : a.q1;
    unsigned* qn_out = &c->qn[nxt];
    const uint32_t stamp_next = it + 1u;

    if (pull && KL == 2 && !Op::kLevels) {
      // ---- pull round of a two-lane group, as the single solve's: a warp
      // takes 128 consecutive in-edges (4 per lane), the lowest lane of each
      // target's run loads the target's row alongside the source gathers, and
      // lanes with the same target fold their candidates lane by lane
      uint32_t changed = 0, scanned = 0;
      const uint32_t EF = g.E - g.NF;
      const uint32_t ntot = EF + g.NF;
      const uint32_t nchunks = (ntot + 127u) >> 7;
      for (uint32_t ch = gwarp; ch < nchunks; ch += nwarps) {
        uint32_t d[4], src[4], w[4], pm[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t idx = (ch << 7) + 32u * j + lane;
          d[j] = 0xFFFFFFFFu - lane;  // unique per lane when not live
          src[j] = 0;
          w[j] = 0;
          pm[j] = 0;
          if (idx < ntot) {
            if (idx < EF) {
              d[j] = ld_stream(g.ifd + idx);
              const uint2 sw = ld_stream(g.ifcw + idx);
              src[j] = sw.x;
              w[j] = sw.y;
              pm[j] = allmask;
            } else {
              const uint32_t k = idx - EF;
              d[j] = ld_stream(g.ipd + k);
              const uint2 sw = ld_stream(g.ipcw + k);
              src[j] = sw.x;
              w[j] = sw.y;
              pm[j] = lanes_of<PRED>(ld_stream(a.iplanes + k)) & allmask;
            }
          }
        }
        uint2 tv[4];
        unsigned lead = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const unsigned grp = __match_any_sync(kFullMask, d[j]);
          const uint32_t idx = (ch << 7) + 32u * j + lane;
          const bool ld = idx < ntot && lane == (unsigned)(__ffs(grp) - 1);
          lead |= (ld ? 1u : 0u) << j;
          tv[j] = ld ? *reinterpret_cast<const uint2*>(a.val + (size_t)d[j] * 2) : make_uint2(0u, 0u);
        }
        uint32_t c0[4], c1[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          c0[j] = c1[j] = Op::kIdentity;
          if (pm[j]) {
            const uint2 su = *reinterpret_cast<const uint2*>(a.val + (size_t)src[j] * 2);
            if (pm[j] & 1u) c0[j] = lane_relax<Op>(a.kinds, 0, su.x, w[j]);
            if (pm[j] & 2u) c1[j] = lane_relax<Op>(a.kinds, 1, su.y, w[j]);
          }
          scanned += __popc(__ballot_sync(kFullMask, pm[j] != 0u));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const unsigned grp = __match_any_sync(kFullMask, d[j]);
          const uint32_t b0 = Op::better(0u, 1u) ? __reduce_min_sync(grp, c0[j]) : __reduce_max_sync(grp, c0[j]);
          const uint32_t b1 = Op::better(0u, 1u) ? __reduce_min_sync(grp, c1[j]) : __reduce_max_sync(grp, c1[j]);
          if ((lead >> j) & 1u) {
            uint32_t* xr = a.val + (size_t)d[j] * 2;
            bool imp = false;
            if (Op::better(b0, tv[j].x)) {
              Op::red(xr, b0);
              imp = true;
            }
            if (Op::better(b1, tv[j].y)) {
              Op::red(xr + 1, b1);
              imp = true;
            }
            if (imp) {
              // a plain store, as in the other pull rounds
              a.stamp[d[j]] = stamp_next;
              ++changed;
            }
          }
        }
      }
      if (lane == 0) relaxed += scanned;
      const uint32_t wc = __reduce_add_sync(kFullMask, changed);
      if (lane == 0 && wc) atomicAdd(qn_out, wc);
      if (!t.sync()) return false;
      continue;
    }
    if (pull) {
      // ---- pull round over the edge-flat transposed graph: each lane takes
      // two in-edges per step, computes every lane's candidate from the
      // source row, and lanes with the same target fold their candidates
      // lane by lane; the lowest of them updates the target row.
      uint32_t changed = 0, scanned = 0;
      // BFS from the source: round `it` sets level `it` in every lane, so a
      // target reached in all lanes skips its in-edges, and only sources
      // reached before this round count (bottom-up BFS)
      const bool bottom_up = Op::kLevels && a.init == kInitSource;
      const uint32_t EF = g.E - g.NF;
      const uint32_t ntot = EF + g.NF;
      const uint32_t nchunks = (ntot + 63u) >> 6;
      // the next chunk's edges are loaded while this chunk's rows are gathered
      auto load_chunk = [&](uint32_t ch, bool valid, uint32_t (&d)[2], uint32_t (&src)[2], uint32_t (&w)[2],
                            uint32_t (&pm)[2]) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const uint32_t idx = (ch << 6) + 32u * j + lane;
          d[j] = 0xFFFFFFFFu - lane;  // unique per lane when not live
          src[j] = 0;
          w[j] = 0;
          pm[j] = 0;
          if (valid && idx < ntot) {
            if (idx < EF) {
              d[j] = ld_stream(g.ifd + idx);
              const uint2 sw = ld_stream(g.ifcw + idx);
              src[j] = sw.x;
              w[j] = sw.y;
              pm[j] = allmask;
            } else {
              const uint32_t k = idx - EF;
              d[j] = ld_stream(g.ipd + k);
              const uint2 sw = ld_stream(g.ipcw + k);
              src[j] = sw.x;
              w[j] = sw.y;
              pm[j] = lanes_of<PRED>(ld_stream(a.iplanes + k)) & allmask;
            }
          }
        }
      };
      uint32_t d[2], src[2], w[2], pm[2];
      load_chunk(gwarp, gwarp < nchunks, d, src, w, pm);
      for (uint32_t ch = gwarp; ch < nchunks; ch += nwarps) {
        uint32_t dn[2], srcn[2], wn[2], pmn[2];
        const bool more = ch + nwarps < nchunks;
        load_chunk(more ? ch + nwarps : ch, more, dn, srcn, wn, pmn);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const uint32_t idx = (ch << 6) + 32u * j + lane;
          if (bottom_up && pm[j]) {
            uint32_t dv[KL];
            ld_row<KL>(a.val + (size_t)d[j] * KL, dv);
            uint32_t open = 0;
#pragma unroll
            for (int k = 0; k < KL; ++k) open |= (dv[k] == kInf ? 1u : 0u) << k;
            pm[j] &= open;
          }
          // the lowest lane of the target's run loads the target's row
          // alongside the source row, not after the fold
          const unsigned grp = __match_any_sync(kFullMask, d[j]);
          const bool leader = idx < ntot && lane == (unsigned)(__ffs(grp) - 1);
          uint32_t* xr = a.val + (size_t)d[j] * KL;
          uint32_t cv[KL];
          if (leader) {
            ld_row<KL>(xr, cv);
          } else {
#pragma unroll
            for (int k = 0; k < KL; ++k) cv[k] = Op::kIdentity;
          }
          uint32_t cand[KL];
#pragma unroll
          for (int k = 0; k < KL; ++k) cand[k] = Op::kIdentity;
          if (pm[j]) {
            uint32_t su[KL];
            ld_row<KL>(a.val + (size_t)src[j] * KL, su);
#pragma unroll
            for (int k = 0; k < KL; ++k)
              if (((pm[j] >> k) & 1u) && (!bottom_up || su[k] < it)) cand[k] = lane_relax<Op>(a.kinds, k, su[k], w[j]);
          }
          scanned += __popc(__ballot_sync(kFullMask, pm[j] != 0u));
          uint32_t best[KL];
#pragma unroll
          for (int k = 0; k < KL; ++k)
            best[k] = Op::better(0u, 1u) ? __reduce_min_sync(grp, cand[k]) : __reduce_max_sync(grp, cand[k]);
          const bool any = __reduce_or_sync(grp, pm[j]) != 0u;
          if (leader && any) {
            bool imp = false;
#pragma unroll
            for (int k = 0; k < KL; ++k) {
              if (Op::better(best[k], cv[k])) {
                Op::red(xr + k, best[k]);
                imp = true;
              }
            }
            if (imp) {
              // a plain store: the next round finds the changed vertices from
              // the stamps, so `changed` only needs to be zero exactly when
              // nothing changed
              a.stamp[d[j]] = stamp_next;
              ++changed;
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          d[j] = dn[j];
          src[j] = srcn[j];
          w[j] = wn[j];
          pm[j] = pmn[j];
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

    // ---- push round: a warp takes up to 32 units, prefix-sums their edge
    // counts and walks the concatenated edges 32 at a time
    const bool levels = Op::kLevels && a.init == kInitSource;
    const Batches bt{n, batch_size(n, nwarps, 32u), nwarps, gwarp, &c->ticket[cur]};
    const uint32_t tk = bt.tk;
    for (uint32_t t0 = bt.first(); t0 < n; t0 = bt.next(lane)) {
      const uint32_t ui = t0 + lane;
      uint32_t beg = 0, cnt = 0, fe = 0, nfb = 0, vv = 0;
      if (lane < tk && ui < n) {
        const unsigned long long u = ld_cg(qin + ui);
        const uint32_t v = (uint32_t)u, ch = (uint32_t)(u >> 32);
        const uint32_t r0 = __ldg(g.rp + v), r1 = __ldg(g.rp + v + 1);
        const uint32_t nf0 = __ldg(g.nfp + v), nf1 = __ldg(g.nfp + v + 1);
        fe = r1 - (nf1 - nf0);
        nfb = nf0;
        vv = v;
        beg = r0 + (ch << a.cshift);
        const uint32_t end = min(r1, beg + (1u << a.cshift));
        cnt = end > beg ? end - beg : 0u;
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
        const uint32_t uk = __shfl_sync(kFullMask, vv, k);
        bool push = false;
        uint32_t x = 0, deg = 0;
        if (p < total) {
          const uint32_t e = bk + (p - (ik - ck));
          const uint2 ew = __ldg(g.cw + e);
          x = ew.x;
          uint32_t pm = e < fk ? allmask : (lanes_of<PRED>(__ldg(a.nflanes + nk + (e - fk))) & allmask);
          if (pm) {
            uint32_t su[KL];
            ld_row<KL>(a.val + (size_t)uk * KL, su);
            // BFS from the sources: a vertex can be in this round's frontier
            // for one lane while another lane's level of it is set in this
            // same round; pushing from that level would set the next level a
            // round early, and the pull rounds rely on round `it` setting
            // exactly level `it`.  So only levels set before this round push.
            if (levels) {
#pragma unroll
              for (int k = 0; k < KL; ++k)
                if (su[k] >= it) pm &= ~(1u << k);
            }
            if (pm && relax_lanes<Op, KL>(su, ew.y, pm, a.val + (size_t)x * KL, a.kinds) &&
                atomicExch(a.stamp + x, stamp_next) != stamp_next) {
              push = true;
              deg = __ldg(g.rp + x + 1) - __ldg(g.rp + x);
            }
          }
        }
        stage_push_units(push, x, deg, a.cshift, st, qout, qn_out, a.qcap, c, a.qerr, lane);
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
