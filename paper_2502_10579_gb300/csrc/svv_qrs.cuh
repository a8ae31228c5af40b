// svv_qrs.cuh -- stable-vertex compaction and Q-relevant subgraph extraction
// as a team phase (see svv_qrs.cu for what it computes).
#pragma once

#include "svv_device.cuh"
#include "svv_team.cuh"

namespace svv {



// exclusive block scan of two counters; block totals in ta/tb
__device__ __forceinline__ void block_excl_scan2(uint32_t a, uint32_t b, uint32_t& ea, uint32_t& eb,
                                                 uint32_t& ta, uint32_t& tb) {
  __shared__ uint32_t s_a[33], s_b[33];
  const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t ia = warp_incl_scan(a, lane), ib = warp_incl_scan(b, lane);
  if (lane == 31) {
    s_a[wid] = ia;
    s_b[wid] = ib;
  }
  __syncthreads();
  if (wid == 0) {
    const uint32_t xa = lane < nw ? s_a[lane] : 0u, xb = lane < nw ? s_b[lane] : 0u;
    const uint32_t ya = warp_incl_scan(xa, lane), yb = warp_incl_scan(xb, lane);
    if (lane < nw) {
      s_a[lane] = ya - xa;
      s_b[lane] = yb - xb;
    }
    if (lane == 31) {
      s_a[32] = ya;
      s_b[32] = yb;
    }
  }
  __syncthreads();
  ea = s_a[wid] + ia - a;
  eb = s_b[wid] + ib - b;
  ta = s_a[32];
  tb = s_b[32];
  __syncthreads();
}

// sum of four counters over the block
__device__ __forceinline__ void block_sum4(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) {
  __shared__ uint32_t s[4][32];
  const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(kFullMask, a, o);
    b += __shfl_xor_sync(kFullMask, b, o);
    c += __shfl_xor_sync(kFullMask, c, o);
    d += __shfl_xor_sync(kFullMask, d, o);
  }
  if (lane == 0) {
    s[0][wid] = a;
    s[1][wid] = b;
    s[2][wid] = c;
    s[3][wid] = d;
  }
  __syncthreads();
  a = b = c = d = 0u;
  for (unsigned i = 0; i < nw; ++i) {
    a += s[0][i];
    b += s[1][i];
    c += s[2][i];
    d += s[3][i];
  }
  __syncthreads();
}

// Walk the edges of every unit in the queue (warp-balanced, as in the solve)
// and classify each edge: all-window (F) or masked (M) kept edge.
// FILL=false: add per-row counts; FILL=true: write the edges.
// With a second query (a.rI1), rows from U0 on are that query's: its edges
// are classified against its own row map and window.
template <bool FILL>
__device__ void qrs_walk(const QrsArgs& a, const Team& t, uint32_t NU, uint32_t U0, unsigned* ticket) {
  const DevGraph& g = a.g;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t nwarps = t.nthreads() >> 5;
  const uint32_t gwarp = t.tid() >> 5;
  const Batches bt{NU, batch_size(NU, nwarps, 32u), nwarps, gwarp, ticket};
  const uint32_t tk = bt.tk;
  for (uint32_t t0 = bt.first(); t0 < NU; t0 = bt.next(lane)) {
    const uint32_t ui = t0 + lane;
    uint32_t r = 0, beg = 0, cnt = 0, fe = 0, nfb = 0;
    if (lane < tk && ui < NU) {
      const unsigned long long u = a.units[ui];  // earlier phases: ordered by the barrier
      r = (uint32_t)u;
      const uint32_t ch = (uint32_t)(u >> 32);
      const uint32_t v = a.uv[r];
      const uint32_t r0 = __ldg(g.rp + v), r1 = __ldg(g.rp + v + 1);
      const uint32_t nf0 = __ldg(g.nfp + v), nf1 = __ldg(g.nfp + v + 1);
      fe = r1 - (nf1 - nf0);
      nfb = nf0;
      beg = r0 + (ch << a.cshift);
      const uint32_t end = min(r1, beg + (1u << a.cshift));
      cnt = end > beg ? end - beg : 0u;
    }
    const uint32_t incl = warp_incl_scan(cnt, lane);
    const uint32_t total = __shfl_sync(kFullMask, incl, 31);
    // two 32-edge steps per iteration: both steps' loads are issued before
    // either step's counts or writes
    for (uint32_t p0 = 0; p0 < total; p0 += 64u) {
      int kk[2];
      uint32_t rkk[2], rx[2], w[2];
      bool isF[2], isM[2];
      const uint64_t* m[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t p = p0 + 32u * h + lane;
        const int k = warp_owner(incl, p < total ? p : total - 1u);
        const uint32_t ik = __shfl_sync(kFullMask, incl, k);
        const uint32_t ck = __shfl_sync(kFullMask, cnt, k);
        const uint32_t bk = __shfl_sync(kFullMask, beg, k);
        const uint32_t fk = __shfl_sync(kFullMask, fe, k);
        const uint32_t nk = __shfl_sync(kFullMask, nfb, k);
        kk[h] = k;
        rkk[h] = __shfl_sync(kFullMask, r, k);
        isF[h] = isM[h] = false;
        rx[h] = kNone;
        w[h] = 0;
        m[h] = nullptr;
        if (p < total) {
          const uint32_t e = bk + (p - (ik - ck));
          const uint2 ew = __ldg(g.cw + e);
          const bool q1 = a.rI1 && rkk[h] >= U0;
          rx[h] = (q1 ? a.row1 : a.row)[ew.x];
          w[h] = ew.y;
          if (rx[h] != kNone) {
            if (e < fk) {
              isF[h] = true;
            } else {
              m[h] = g.nfmask + (size_t)(nk + (e - fk)) * g.W;
              bool any, all;
              window_any_all(m[h], q1 ? a.win1 : a.win, any, all);
              isF[h] = all;
              isM[h] = any && !all;
            }
          }
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t p = p0 + 32u * h + lane;
        const uint32_t rk = rkk[h];
        const unsigned grp = __match_any_sync(kFullMask, p < total ? (uint32_t)kk[h] : 64u + lane);
        const unsigned bF = __ballot_sync(kFullMask, isF[h]), bM = __ballot_sync(kFullMask, isM[h]);
        const int leader = __ffs(grp) - 1;
        const uint32_t nF = __popc(grp & bF), nM = __popc(grp & bM);
        if (!FILL) {
          if (lane == (unsigned)leader && p < total) {
            if (nF) atomicAdd(a.qcnt + 2u * rk, nF);
            if (nM) atomicAdd(a.qcnt + 2u * rk + 1u, nM);
          }
        } else {
          uint32_t baseF = 0, baseM = 0;
          if (lane == (unsigned)leader && p < total) {
            if (nF) baseF = atomicAdd(a.cur + 2u * rk, nF);
            if (nM) baseM = atomicAdd(a.cur + 2u * rk + 1u, nM);
          }
          baseF = __shfl_sync(kFullMask, baseF, leader);
          baseM = __shfl_sync(kFullMask, baseM, leader);
          if (isF[h]) {
            const uint32_t pos = baseF + __popc(grp & bF & lt);
            a.qcw[pos] = make_uint2(rx[h], w[h]);
          } else if (isM[h]) {
            const uint32_t pos = baseM + __popc(grp & bM & lt);
            a.qcw[pos] = make_uint2(rx[h], w[h]);
            const uint4 d = __ldcg(a.qrow + rk);
            uint64_t* out = a.qmask + (size_t)(d.z + (pos - d.y)) * a.QW;
            const uint32_t wb = (a.rI1 && rk >= U0) ? a.win1.b : a.win.b;
            for (uint32_t j = 0; j < a.QW; ++j) {
              uint64_t word = mask_extract(m[h], g.W, wb + 64u * j);
              const uint32_t left = a.win.l - 64u * j;
              if (left < 64u) word &= (1ull << left) - 1ull;
              out[j] = word;
            }
          }
        }
      }
    }
  }
}

__device__ inline bool qrs_team(const QrsArgs& a, const Team& t) {
  const DevGraph& g = a.g;
  TeamCtl* c = a.ctl;
  const unsigned nb = t.nblocks, b = t.rank, tid = threadIdx.x;
  if (cta_read(a.qerr) != 0u) return false;
  const uint32_t V = g.V;
  const uint32_t C = 1u << a.cshift;
  // A second query (a.rI1) is extracted in the same launch: its rows follow
  // the first query's, its units follow theirs, and the row scan and the
  // fill run over both ranges at once.
  const int nq = a.rI1 ? 2 : 1;

  // ---- P1: unstable vertices and their units, per CTA vertex range and query
  if (a.trace && b == 0 && tid == 0) a.trace[0] = global_ns();
  const unsigned long long per = (((unsigned long long)V + nb - 1) / nb + 31ull) & ~31ull;
  const uint32_t lo = (uint32_t)min((unsigned long long)V, per * b);
  const uint32_t hi = (uint32_t)min((unsigned long long)V, per * b + per);
  {
    uint32_t cnt = 0, nun = 0, cnt1 = 0, nun1 = 0;
    for (uint32_t v = lo + tid; v < hi; v += blockDim.x) {
      const uint32_t nv = (__ldg(g.rp + v + 1) - __ldg(g.rp + v) + C - 1u) >> a.cshift;
      if (!a.prune || a.rI[v] != a.rU[v]) {
        ++cnt;
        nun += nv;
      }
      if (nq > 1 && (!a.prune || a.rI1[v] != a.rU1[v])) {
        ++cnt1;
        nun1 += nv;
      }
    }
    block_sum4(cnt, nun, cnt1, nun1);
    if (tid == 0) {
      a.part[4 * b] = cnt;
      a.part[4 * b + 1] = nun;
      a.part[4 * b + 2] = cnt1;
      a.part[4 * b + 3] = nun1;
    }
  }
  if (!t.sync()) return false;

  // ---- P2: rows and units in vertex order, the first query's then the second's
  if (a.trace && b == 0 && tid == 0) a.trace[1] = global_ns();
  uint32_t U = 0, NU = 0, U0 = 0;
  for (int qi = 0; qi < nq; ++qi) {
    const uint32_t* qI = qi ? a.rI1 : a.rI;
    const uint32_t* qU = qi ? a.rU1 : a.rU;
    uint32_t* qrowmap = qi ? a.row1 : a.row;
    uint32_t o_r = 0, o_u = 0, t_r = 0, t_u = 0;
    for (uint32_t j = tid; j < nb; j += blockDim.x) {
      const uint32_t pr = ld_cg(a.part + 4 * j + 2 * qi), pu = ld_cg(a.part + 4 * j + 2 * qi + 1);
      t_r += pr;
      t_u += pu;
      if (j < b) {
        o_r += pr;
        o_u += pu;
      }
    }
    block_sum4(o_r, o_u, t_r, t_u);
    const uint32_t rbase = U, ubase = NU;  // after the first query's rows and units
    U += t_r;
    NU += t_u;
    if (qi == 0) U0 = t_r;
    if (b == 0 && tid == 0) {
      if (qi == 0) {
        c->aux[0] = t_r;
        c->aux[1] = t_u;
      } else {
        a.counts1_out[0] = t_r;
      }
    }
    if (NU > a.ucap || U > a.rowcap) {
      if (tid == 0) set_err(c, a.qerr, kErrInternal);
      return false;  // every CTA sees the same totals and leaves here
    }
    for (uint32_t base = lo; base < hi; base += blockDim.x) {
      const uint32_t v = base + tid;
      uint32_t flag = 0, nu = 0;
      if (v < hi && (!a.prune || qI[v] != qU[v])) {
        flag = 1;
        nu = (__ldg(g.rp + v + 1) - __ldg(g.rp + v) + C - 1u) >> a.cshift;
      }
      uint32_t ef, eu, tf, tu;
      block_excl_scan2(flag, nu, ef, eu, tf, tu);
      const uint32_t r = rbase + o_r + ef;
      if (v < hi) {
        qrowmap[v] = flag ? r : kNone;
        if (flag) {
          a.uv[r] = v;
          a.qcnt[2 * r] = 0u;
          a.qcnt[2 * r + 1] = 0u;
        }
      }
      // the warp writes its vertices' units together, so a hub's hundreds
      // of units do not serialise on one thread
      const unsigned lane = tid & 31u;
      const uint32_t incl = warp_incl_scan(nu, lane);
      const uint32_t wtot = __shfl_sync(kFullMask, incl, 31);
      for (uint32_t j0 = 0; j0 < wtot; j0 += 32u) {
        const uint32_t j = j0 + lane;
        const int k = warp_owner(incl, j < wtot ? j : wtot - 1u);
        const uint32_t ik = __shfl_sync(kFullMask, incl, k), nk = __shfl_sync(kFullMask, nu, k);
        const uint32_t rk = __shfl_sync(kFullMask, r, k), ek = __shfl_sync(kFullMask, eu, k);
        const uint32_t jj = j - (ik - nk);
        if (j < wtot) a.units[ubase + o_u + ek + jj] = (unsigned long long)rk | ((unsigned long long)jj << 32);
      }
      o_r += tf;
      o_u += tu;
    }
  }
  if (!t.sync()) return false;

  // ---- P3: per-row counts of kept edges
  if (a.trace && b == 0 && tid == 0) a.trace[2] = global_ns();
  qrs_walk<false>(a, t, NU, U0, &c->ticket[0]);
  if (!t.sync()) return false;

  // ---- P4: scan rows
  if (a.trace && b == 0 && tid == 0) a.trace[3] = global_ns();
  const unsigned long long rper = (((unsigned long long)U + nb - 1) / nb + 31ull) & ~31ull;
  const uint32_t rlo = (uint32_t)min((unsigned long long)U, rper * b);
  const uint32_t rhi = (uint32_t)min((unsigned long long)U, rper * b + rper);
  {
    uint32_t se = 0, sm = 0, z0 = 0, z1 = 0;
    for (uint32_t r = rlo + tid; r < rhi; r += blockDim.x) {
      const uint32_t f = ld_cg(a.qcnt + 2 * r), m = ld_cg(a.qcnt + 2 * r + 1);
      se += f + m;
      sm += m;
    }
    block_sum4(se, sm, z0, z1);
    if (tid == 0) {
      a.part[2 * nb + 2 * b] = se;
      a.part[2 * nb + 2 * b + 1] = sm;
    }
  }
  if (!t.sync()) return false;
  {
    uint32_t o_e = 0, o_m = 0, t_e = 0, t_m = 0;
    for (uint32_t j = tid; j < nb; j += blockDim.x) {
      const uint32_t pe = ld_cg(a.part + 2 * nb + 2 * j), pm = ld_cg(a.part + 2 * nb + 2 * j + 1);
      t_e += pe;
      t_m += pm;
      if (j < b) {
        o_e += pe;
        o_m += pm;
      }
    }
    block_sum4(o_e, o_m, t_e, t_m);
    if (b == 0 && tid == 0) {
      c->aux[2] = t_e;
      c->aux[3] = t_m;
    }
    if (t_e > a.ecap || (unsigned long long)t_m * a.QW > a.mcap) {
      if (tid == 0) set_err(c, a.qerr, kErrInternal);
      return false;
    }
    for (uint32_t base = rlo; base < rhi; base += blockDim.x) {
      const uint32_t r = base + tid;
      uint32_t f = 0, m = 0;
      if (r < rhi) {
        f = ld_cg(a.qcnt + 2 * r);
        m = ld_cg(a.qcnt + 2 * r + 1);
      }
      uint32_t ee, em, te, tm;
      block_excl_scan2(f + m, m, ee, em, te, tm);
      if (r < rhi) {
        const uint32_t start = o_e + ee;
        a.qrow[r] = make_uint4(start, start + f, o_m + em, start + f + m);
        a.cur[2 * r] = start;
        a.cur[2 * r + 1] = start + f;
      }
      o_e += te;
      o_m += tm;
    }
  }
  if (!t.sync()) return false;

  // ---- P5: fill
  if (a.trace && b == 0 && tid == 0) a.trace[4] = global_ns();
  qrs_walk<true>(a, t, NU, U0, &c->ticket[1]);
  if (a.trace && tid == 0) atomicMax(a.trace + 5, global_ns());  // the last CTA to finish
  return true;
}

}  // namespace svv
