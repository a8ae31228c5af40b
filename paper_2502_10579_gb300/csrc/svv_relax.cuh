// svv_relax.cuh -- Algorithm 2 (concurrent relaxation of every window
// snapshot) and the output scatter as team phases (see svv_relax.cu).
#pragma once

#include "svv_device.cuh"
#include "svv_push.cuh"
#include "svv_team.cuh"

namespace svv {

// query q's relaxation: the op's own, or (a mixed pair) query q's kind
template <class Op>
__device__ __forceinline__ uint32_t relax_q(const RelaxArgs& a, bool q1, uint32_t sv, uint32_t w) {
  if constexpr (is_mixed<Op>::value) return OpMixed::relax_kind(q1 ? a.kind1 : a.kind0, sv, w);
  else return Op::relax(sv, w);
}

template <class Op, int P, int K>
__device__ bool relax_team(const RelaxArgs& a, const Team& t, unsigned long long* stage) {
  const DevGraph& g = a.g;
  TeamCtl* c = a.ctl;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned nthreads = t.nthreads();
  const unsigned gtid = t.tid();
  const unsigned gwarp = gtid >> 5, nwarps = nthreads >> 5;
  if (cta_read(a.qerr) != 0u) return false;
  PushStage st{stage + (threadIdx.x >> 5) * kStageUnits, 0u};
  // rows [0, U0) are the first query's, [U0, U) a second query's (a.counts1)
  const uint32_t U0 = a.counts[0];
  const uint32_t U = U0 + (a.counts1 ? a.counts1[0] : 0u);
  const uint32_t LP = a.LP;
  const uint32_t lps = __ffs(LP) - 1;  // LP is a power of two

  // ---- round 0a: values and stamps.  A warp reads the starting values of
  // 32 rows at once (a lane per row), then writes those rows together (a
  // lane per column), so the dependent loads are paid once per 32 rows.
  for (uint32_t r0 = gwarp * 32u; r0 < U; r0 += nwarps * 32u) {
    const uint32_t r = r0 + lane;
    const uint32_t x = r < U ? ((r < U0 ? a.rI : a.rI1)[a.uv[r]] ^ ((a.flip >> (r < U0 ? 0 : 1)) & 1u ? ~0u : 0u))
                             : 0u;
    if (r < U) a.stamp[r] = 0u;
    const uint32_t nr = min(32u, U - r0);
    for (uint32_t k = 0; k < nr; ++k) {
      const uint32_t xv = __shfl_sync(kFullMask, x, k);
      uint32_t* row = a.val + ((size_t)(r0 + k) << lps);
      for (uint32_t i = lane; i < LP; i += 32u) row[i] = xv;
    }
  }
  if (!t.sync()) return false;
  if (a.trace && gtid == 0 && a.trace_cap) a.trace[0] = global_ns() & 0xFFFFFFFFFFull;

  // ---- round 0b: seed from addition edges with an unstable sink; four
  // qualifying edges per warp iteration, lanes over the slab's snapshots
  // each query's seeds (the second query's rows map to its own range)
  for (int qi = 0; qi < (a.counts1 ? 2 : 1); ++qi) {
    const uint32_t* srow = qi ? a.row1 : a.row;
    const uint32_t* srI = qi ? a.rI1 : a.rI;
    const Window swin = qi ? a.win1 : a.win;
    const uint32_t ssnap = swin.b + a.s0;
    const uint32_t sflip = ((a.flip >> qi) & 1u) ? ~0u : 0u;
    for (uint32_t k0 = gwarp * 32u; k0 < g.NF; k0 += nwarps * 32u) {
      const uint32_t k = k0 + lane;
      bool qual = false;
      uint32_t rx = kNone, cand = 0;
      if (k < g.NF) {
        const uint2 e = __ldg(g.nfcw + k);
        rx = srow[e.x];
        if (rx != kNone) {
          bool any, all;
          window_any_all(g.nfmask + (size_t)k * g.W, swin, any, all);
          qual = any && !all;
          if (qual) cand = relax_q<Op>(a, qi != 0, srI[__ldg(g.nfsrc + k)] ^ sflip, e.y);
        }
      }
      // the owner lane extracts the slab's presence bits once; the warp then
      // takes four qualifying edges at a time with the bits in registers
      uint64_t mlo = 0ull, mhi = 0ull;
      if (qual) {
        const uint64_t* mp = g.nfmask + (size_t)k * g.W;
        mlo = mask_extract(mp, g.W, ssnap);
        if (a.ls > 64u) mhi = mask_extract(mp, g.W, ssnap + 64u);
      }
      unsigned bq = __ballot_sync(kFullMask, qual);
      constexpr int HS = 4;
      while (bq) {
        int j[HS];
  #pragma unroll
        for (int h = 0; h < HS; ++h) {
          j[h] = bq ? __ffs(bq) - 1 : -1;
          if (bq) bq &= bq - 1u;
        }
        uint32_t ex[HS], ec[HS];
        uint64_t ml[HS], mh[HS];
  #pragma unroll
        for (int h = 0; h < HS; ++h) {
          const int src = j[h] < 0 ? j[0] : j[h];
          ex[h] = __shfl_sync(kFullMask, rx, src);
          ec[h] = __shfl_sync(kFullMask, cand, src);
          ml[h] = __shfl_sync(kFullMask, mlo, src);
          mh[h] = __shfl_sync(kFullMask, mhi, src);
        }
        bool imp[HS];
  #pragma unroll
        for (int h = 0; h < HS; ++h) imp[h] = false;
        for (uint32_t i = lane; i < a.ls; i += 32u) {
          bool want[HS];
          uint32_t curv[HS];
  #pragma unroll
          for (int h = 0; h < HS; ++h) {
            const uint64_t bit = i < 64u ? (ml[h] >> i) : (mh[h] >> (i - 64u));
            want[h] = j[h] >= 0 && (bit & 1ull);
            curv[h] = want[h] ? ld_val(a.val + ((size_t)ex[h] << lps) + i) : 0u;
          }
  #pragma unroll
          for (int h = 0; h < HS; ++h) {
            if (want[h] && Op::better(ec[h], curv[h])) {
              Op::red(a.val + ((size_t)ex[h] << lps) + i, ec[h]);
              imp[h] = true;
            }
          }
        }
        // lane h claims edge h's target (the HS stamp exchanges run side by
        // side) and one warp append queues every claimed row
        unsigned anyb = 0;
  #pragma unroll
        for (int h = 0; h < HS; ++h) anyb |= (__any_sync(kFullMask, imp[h]) ? 1u : 0u) << h;
        uint32_t px = 0;
        bool claim = false;
  #pragma unroll
        for (int h = 0; h < HS; ++h)
          if (lane == (unsigned)h) {
            px = ex[h];
            claim = (anyb >> h) & 1u;
          }
        bool push = false;
        uint32_t deg = 0;
        if (claim) {
          const uint4 d = a.qrow[px];
          if (atomicExch(a.stamp + px, 1u) != 1u) {
            push = true;
            deg = d.w - d.x;
          }
        }
        stage_push_units(push, px, deg, a.cshift, st, a.q1, &c->qn[1], a.qcap, c, a.qerr, lane);
      }
    }
  }
  stage_flush_cta(st, a.q1, &c->qn[1], a.qcap, c, a.qerr, lane);
  if (!t.sync()) return false;

  // ---- rounds >= 1: Algorithm 2 while-loop over the frontier
  constexpr int G = 32 / P;
  const unsigned grp = lane / P, gl = lane % P;
  const unsigned gmask = (P == 32) ? kFullMask : (((1u << P) - 1u) << (grp * P));
  unsigned long long relaxed = 0;
  uint32_t it = 1;
  for (;; ++it) {
    const uint32_t cur = it % 3u, nxt = (it + 1u) % 3u, clr = (it + 2u) % 3u;
    uint32_t n = cta_read(&c->qn[cur]);
    if (a.trace && gtid == 0 && it < a.trace_cap) a.trace[it] = ((unsigned long long)n << 40) | (global_ns() & 0xFFFFFFFFFFull);
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

    // G units (one per lane group) per batch
    const Batches bt{n, (uint32_t)G, nwarps, gwarp, &c->ticket[cur]};
    for (uint32_t t0 = bt.first(); t0 < n; t0 = bt.next(lane)) {
      const uint32_t ui = t0 + grp;
      uint32_t beg = 0, end = 0, fe = 0, nfb = 0;
      bool q1 = false;  // the unit's row belongs to the second query
      uint32_t sv[K];
#pragma unroll
      for (int kk = 0; kk < K; ++kk) sv[kk] = Op::kIdentity;
      if (ui < n) {
        const unsigned long long u = qin[ui];  // written before the last barrier
        const uint32_t r = (uint32_t)u, ch = (uint32_t)(u >> 32);
        q1 = r >= U0;
        const uint4 d = a.qrow[r];
        beg = d.x + (ch << a.cshift);
        end = min(d.w, beg + (1u << a.cshift));
        fe = d.y;
        nfb = d.z;
        const uint32_t* src = a.val + ((size_t)r << lps) + gl;
#pragma unroll
        for (int kk = 0; kk < K; ++kk) sv[kk] = ld_val(src + kk * P);
      }
      const uint32_t cnt = end > beg ? end - beg : 0u;
      const uint32_t maxcnt = __reduce_max_sync(kFullMask, cnt);
      if (gl == 0) relaxed += cnt;
      for (uint32_t j0 = 0; j0 < maxcnt; j0 += P) {
        const uint32_t e = beg + j0 + gl;
        uint32_t xr = 0, w = 0;
        uint64_t m0 = ~0ull, m1 = ~0ull;
        if (e < end) {
          const uint2 ew = a.qcw[e];
          xr = ew.x;
          w = ew.y;
          if (e >= fe) {
            const uint64_t* mp = a.qmask + (size_t)(nfb + (e - fe)) * a.QW;
            m0 = mask_extract(mp, a.QW, a.s0);
            if (P * K > 64) m1 = mask_extract(mp, a.QW, a.s0 + 64u);
          }
        }
        bool pend = false;
        uint32_t pend_x = 0;
        const uint32_t nj = min((uint32_t)P, maxcnt - j0);
        // H edges per iteration: every target row is loaded before any is
        // compared, so each lane keeps H load chains in flight
        constexpr int H = (K <= 2) ? 4 : 2;
        for (uint32_t jj = 0; jj < nj; jj += H) {
          uint32_t ex[H], ewt[H];
          uint64_t em0[H], em1[H];
          bool ev[H];
#pragma unroll
          for (int h = 0; h < H; ++h) {
            const uint32_t src = min(jj + h, (uint32_t)P - 1u);
            ex[h] = __shfl_sync(kFullMask, xr, src, P);
            ewt[h] = __shfl_sync(kFullMask, w, src, P);
            em0[h] = __shfl_sync(kFullMask, m0, src, P);
            em1[h] = ~0ull;
            if (P * K > 64) em1[h] = __shfl_sync(kFullMask, m1, src, P);
            ev[h] = (jj + h < nj) && (beg + j0 + jj + h) < end;
          }
          uint32_t curv[H][K];
          bool want[H][K];
#pragma unroll
          for (int h = 0; h < H; ++h) {
            uint32_t* row = a.val + ((size_t)ex[h] << lps) + gl;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
              const uint32_t i = gl + kk * P;
              const bool bit = (i < 64u) ? ((em0[h] >> i) & 1ull) : ((em1[h] >> (i - 64u)) & 1ull);
              want[h][kk] = ev[h] && i < a.ls && bit;
              curv[h][kk] = want[h][kk] ? ld_val(row + kk * P) : 0u;
            }
          }
          bool imp[H];
#pragma unroll
          for (int h = 0; h < H; ++h) {
            imp[h] = false;
            uint32_t* row = a.val + ((size_t)ex[h] << lps) + gl;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
              if (want[h][kk]) {
                const uint32_t cand = relax_q<Op>(a, q1, sv[kk], ewt[h]);
                if (Op::better(cand, curv[h][kk])) {
                  Op::red(row + kk * P, cand);
                  imp[h] = true;
                }
              }
            }
          }
#pragma unroll
          for (int h = 0; h < H; ++h) {
            const unsigned bi = __ballot_sync(kFullMask, imp[h]) & gmask;
            if (gl == jj + h && bi) {
              pend = true;
              pend_x = ex[h];
            }
          }
        }
        bool push = false;
        uint32_t deg = 0;
        if (pend) {
          const uint4 d = a.qrow[pend_x];  // issued alongside the stamp exchange
          if (atomicExch(a.stamp + pend_x, stamp_next) != stamp_next) {
            push = true;
            deg = d.w - d.x;
          }
        }
        stage_push_units(push, pend_x, deg, a.cshift, st, qout, qn_out, a.qcap, c, a.qerr, lane);
      }
    }
    stage_flush_cta(st, qout, qn_out, a.qcap, c, a.qerr, lane);
    if (!t.sync()) return false;
  }
  if (gl == 0 && relaxed) atomicAdd(&c->relaxed, relaxed);
  if (gtid == 0) c->iters = it - 1u;
  return true;
}

// Output scatter over a team: tiles of kScatterTV vertices x ls snapshots are
// staged in `tile` (ls * (kScatterTV + 1) words of shared memory) so the row
// reads and the snapshot-major writes both coalesce.
constexpr int kScatterTV = 64;

__device__ __forceinline__ void scatter_team(const ScatterArgs& a, const Team& t, uint32_t* tile) {
  const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t lps = __ffs(a.LP) - 1;
  const uint32_t ntiles = (a.V + kScatterTV - 1) / kScatterTV;
  for (uint32_t tl = t.rank; tl < ntiles; tl += t.nblocks) {
    const uint32_t v0 = tl * kScatterTV;
    for (uint32_t tv = wid; tv < (uint32_t)kScatterTV; tv += nw) {
      const uint32_t v = v0 + tv;
      if (v >= a.V) break;
      const uint32_t r = a.row[v];
      if (r == kNone) {
        const uint32_t x = a.rI[v];
        for (uint32_t i = lane; i < a.ls; i += 32u) tile[i * (kScatterTV + 1) + tv] = x;
      } else {
        const uint32_t* src = a.val + ((size_t)r << lps);
        for (uint32_t i = lane; i < a.ls; i += 32u) tile[i * (kScatterTV + 1) + tv] = __ldcg(src + i);
      }
    }
    __syncthreads();
    const uint32_t nv = min((uint32_t)kScatterTV, a.V - v0);
    for (uint32_t idx = threadIdx.x; idx < a.ls * (uint32_t)kScatterTV; idx += blockDim.x) {
      const uint32_t i = idx / kScatterTV, tv = idx % kScatterTV;
      if (tv < nv) a.out[(size_t)(a.s0 + i) * a.V + v0 + tv] = tile[i * (kScatterTV + 1) + tv];
    }
    __syncthreads();
  }
}

}  // namespace svv
