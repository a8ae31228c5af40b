// svv_group_api.cu -- host side of query groups: their scratch, and the two
// group solves (svv_group.cuh) that give every member query its
// intersection- and union-graph values (Section 3 Step 1) from one set of
// frontier rounds.  Each member then runs its own stable compaction, subgraph
// extraction, relaxation and scatter (enqueue_tail) from its lane's planar
// copy of the bounds.
#include "svv_ctx.h"

namespace svv {

void free_group(svv_ctx* c) {
  c->last_rI = c->last_rU = c->last_row = nullptr;
  for (void* p : c->group_bufs) cudaFree(p);
  c->group_bufs.clear();
  c->gcap = c->gcup = c->gnfl = c->gipl = c->gerr = nullptr;
  for (int k = 0; k < kGroupMax; ++k) c->gI[k] = c->gU[k] = nullptr;
  c->group_ready = false;
}

svv_status ensure_group(svv_ctx* c) {
  if (c->group_ready) return SVV_OK;
  const uint64_t V = c->g.V, NF = std::max<uint32_t>(c->g.NF, 1);
  svv_status st;
  if ((st = alloc_n(c, c->group_bufs, V * kGroupMax, &c->gcap)) ||
      (st = alloc_n(c, c->group_bufs, V * kGroupMax, &c->gcup)) || (st = alloc_n(c, c->group_bufs, NF, &c->gnfl)) ||
      (st = alloc_n(c, c->group_bufs, NF, &c->gipl)) || (st = alloc_n(c, c->group_bufs, 1, &c->gerr))) {
    free_group(c);
    return st;
  }
  for (int k = 0; k < kGroupMax; ++k) {
    if ((st = alloc_n(c, c->group_bufs, V, &c->gI[k])) || (st = alloc_n(c, c->group_bufs, V, &c->gU[k]))) {
      free_group(c);
      return st;
    }
  }
  c->group_ready = true;
  return SVV_OK;
}

// The two bound solves of n (2..kGroupMax) same-type queries, lane k = inst[k],
// then the split into gI[k] (intersection values) and gU[k] (union values).
// The group's error word ends up in gerr: each member's phases start from it.
svv_status enqueue_group_bounds(svv_ctx* c, int t, const BatchInstance* inst, uint32_t n, cudaStream_t s) {
  if (n < 1 || n > (uint32_t)kGroupMax) return fail(c, SVV_EINTERNAL, "group size out of range");
  svv_status st = ensure_group(c);
  if (st) return st;
  const uint32_t KL = n <= 2 ? 2u : n <= 4 ? 4u : 8u;
  const Knobs kn = knobs_of(c, t, inst[0].wl);
  // several types: every lane in the min lattice with its own relaxation
  // kind, SSWP lanes complemented (undone by the split)
  bool mixed = false;
  for (uint32_t k = 1; k < n; ++k) mixed |= inst[k].type != inst[0].type;
  uint32_t kinds = 0, flip = 0;
  if (mixed) {
    for (uint32_t k = 0; k < n; ++k) {
      const int tk = inst[k].type;
      const uint32_t kind = tk == 0 ? kKindSum : tk == 1 ? kKindMaxNot : tk == 2 ? kKindHop : kKindMax;
      kinds |= kind << (2 * k);
      if (tk == 1) flip |= 1u << k;
    }
  }
  const int gt = mixed ? kTypeMixed : t;
  cudaError_t e = cudaMemsetAsync(c->ctl + 4, 0, sizeof(TeamCtl) * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->qerr, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");

  LanesArgs la{};
  la.g = c->g;
  la.nlanes = n;
  for (uint32_t k = 0; k < n; ++k) la.win[k] = Window{inst[k].wb, inst[k].wl};
  la.nflanes = c->gnfl;
  la.iplanes = c->g.ifd ? c->gipl : nullptr;
  if ((e = launch_group_lanes(la, s)) != cudaSuccess) return cuda_fail(c, e, "launch lane words");

  const SolveArgs base = solve_base(c, 0, 1, t, kn);
  GroupArgs a{};
  a.g = c->g;
  a.nlanes = n;
  for (uint32_t k = 0; k < n; ++k) a.source[k] = inst[k].source;
  a.init = kInitSource;
  a.val = c->gcap;
  a.nflanes = c->gnfl;
  a.iplanes = c->gipl;
  a.stamp = c->stamp;
  a.q0 = c->q0;
  a.q1 = c->q1;
  a.qcap = c->qcap;
  a.cshift = kn.solve_cs;
  a.ctl = c->ctl + 4;
  a.qerr = c->qerr;
  a.maxit = c->maxit ? c->maxit : c->g.V + 2u;
  a.spin_ns = base.spin_ns;
  // pull thresholds of the group solves (0 = push only)
  uint32_t pull_u[2] = {0, 0}, push_v[2] = {0, 0};
  for (int i = 0; i < 2; ++i) {
    const uint32_t pct = c->group_pull_pct[i];
    if (c->g.ifd && pct && pct < 100) {
      const uint64_t all_units = (uint64_t)c->g.V + (c->g.E >> kn.solve_cs);
      pull_u[i] = (uint32_t)std::max<uint64_t>(1, all_units * pct / 100);
      push_v[i] = (uint32_t)std::max<uint64_t>(1, (uint64_t)c->g.V * pct / 100);
    }
  }
  a.pull_units = pull_u[0];
  a.push_verts = push_v[0];
  a.kinds = kinds;
  if (c->round_trace) {  // phases 0 and 1 of the round trace: the group's two solves
    cudaMemsetAsync(c->trace, 0, 2 * kTraceCap * sizeof(unsigned long long), s);
    a.trace = c->trace;
    a.trace_cap = kTraceCap;
  }
  const LaunchCfg cfg = cfg_for(c, KL == 2 ? c->occ_group2 : c->occ_group, kn.bps);
  // phase timing of the group's two solves (read back after the batch)
  bool timed = c->phase_timing && !c->graph_mode && !c->serve.active;
  for (auto& ev : c->gev)
    if (timed && !ev && cudaEventCreate(&ev) != cudaSuccess) timed = false;
  if (timed) cudaEventRecord(c->gev[0], s);
  c->gev_pending = timed;
  if ((e = launch_group_solve(gt, KL, kPredAll, a, cfg, s)) != cudaSuccess)
    return cuda_fail(c, e, "launch group intersection solve");
  if (timed) cudaEventRecord(c->gev[1], s);
  SplitArgs sp{};
  sp.V = c->g.V;
  sp.nlanes = n;
  sp.KL = KL;
  sp.flip = flip;
  sp.cap = c->gcap;
  sp.cup = c->gcap;
  if (c->prune) {  // without pruning the union values are never read
    GroupArgs b = a;
    b.init = kInitSeed;
    b.base = c->gcap;
    b.val = c->gcup;
    b.ctl = c->ctl + 5;
    b.pull_units = pull_u[1];
    b.push_verts = push_v[1];
    if (c->round_trace) b.trace = c->trace + kTraceCap;
    if ((e = launch_group_solve(gt, KL, kPredAny, b, cfg, s)) != cudaSuccess)
      return cuda_fail(c, e, "launch group union solve");
    sp.cup = c->gcup;
  }
  if (timed) cudaEventRecord(c->gev[2], s);
  for (uint32_t k = 0; k < n; ++k) {
    sp.rI[k] = c->gI[k];
    sp.rU[k] = c->gU[k];
  }
  if ((e = launch_group_split(sp, s)) != cudaSuccess) return cuda_fail(c, e, "launch group split");
  if ((e = cudaMemcpyAsync(c->gerr, c->qerr, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return cuda_fail(c, e, "group status copy");
  return SVV_OK;
}

// ---------------------------------------------------------------------------
// Two-query tails.  One extraction launch compacts both queries' unstable
// vertices and builds both subgraphs into the pair arrays (the first query's
// rows [0, U0), the second's after them); one relaxation launch then runs
// Algorithm 2 over both queries' rows with one frontier, and each query's
// scatter reads its own rows.  A pair of different types relaxes in the min
// lattice (OpMixed), an SSWP query's rows on complemented widths.

void free_pair(svv_ctx* c) {
  if (c->p_row1 && c->last_row == c->p_row1) c->last_row = nullptr;
  for (void* p : c->pair_bufs) cudaFree(p);
  c->pair_bufs.clear();
  c->p_uv = c->p_qcnt = c->p_cur = c->p_stamp = c->p_row1 = nullptr;
  c->p_qrow = nullptr;
  c->p_qcw = nullptr;
  c->p_qmask = nullptr;
  c->p_val = nullptr;
  c->p_q0 = c->p_q1 = c->p_units = nullptr;
  c->p_valcap = c->p_qcap = c->p_mcap = 0;
}

svv_status ensure_pair_rows(svv_ctx* c, uint32_t LP) {
  const uint64_t V = c->g.V;
  const uint64_t need_v = 2 * V * LP;
  // the mask capacity follows the longest window seen (ensure_window)
  if (c->p_uv && need_v <= c->p_valcap && 2 * c->mcap <= c->p_mcap) return SVV_OK;
  free_pair(c);
  // every array holds two queries' worth of what the single-query scratch holds
  svv_status st;
  if ((st = alloc_n(c, c->pair_bufs, 2 * V, &c->p_uv)) || (st = alloc_n(c, c->pair_bufs, 4 * V, &c->p_qcnt)) ||
      (st = alloc_n(c, c->pair_bufs, 4 * V, &c->p_cur)) || (st = alloc_n(c, c->pair_bufs, 2 * V, &c->p_stamp)) ||
      (st = alloc_n(c, c->pair_bufs, V, &c->p_row1)) || (st = alloc_n(c, c->pair_bufs, 2 * V, &c->p_qrow)) ||
      (st = alloc_n(c, c->pair_bufs, 2 * (uint64_t)c->ecap, &c->p_qcw)) ||
      (st = alloc_n(c, c->pair_bufs, 2 * c->mcap, &c->p_qmask)) ||
      (st = alloc_n(c, c->pair_bufs, need_v, &c->p_val)) ||
      (st = alloc_n(c, c->pair_bufs, 2 * (uint64_t)c->ucap, &c->p_units)) ||
      (st = alloc_n(c, c->pair_bufs, 2 * (uint64_t)c->qcap, &c->p_q0)) ||
      (st = alloc_n(c, c->pair_bufs, 2 * (uint64_t)c->qcap, &c->p_q1))) {
    free_pair(c);
    return st;
  }
  c->p_valcap = need_v;
  c->p_mcap = 2 * c->mcap;
  c->p_qcap = 2 * (uint64_t)c->qcap;
  return SVV_OK;
}

svv_status enqueue_pair_tail(svv_ctx* c, const BatchInstance* inst, uint32_t* const* out, const uint32_t* const* rI,
                             const uint32_t* const* rU, cudaStream_t s, bool* done) {
  *done = false;
  const uint32_t wl = inst[0].wl;
  if (!c->pair_tails || inst[1].wl != wl || wl > kMaxSlab) return SVV_OK;
  const Knobs k0 = knobs_of(c, inst[0].type, wl), k1 = knobs_of(c, inst[1].type, wl);
  if (wl > std::max<uint32_t>(1, std::min(k0.slab_max, kMaxSlab)) ||
      wl > std::max<uint32_t>(1, std::min(k1.slab_max, kMaxSlab)) || k0.relax_lanes != k1.relax_lanes)
    return SVV_OK;
  uint32_t P, K;
  slab_shape_p(wl, k0.relax_lanes, P, K);
  svv_status st = ensure_pair_rows(c, P * K);
  if (st) return st;
  if (c->p_qcap > 0xFFFFFFFFull) return SVV_OK;
  cudaError_t e = cudaMemsetAsync(c->ctl + 2, 0, sizeof(TeamCtl) * 2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ctl + 6, 0, sizeof(TeamCtl), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  c->last_rI = rI[1];  // svv_get_bounds: the batch's last instance
  c->last_rU = rU[1];
  c->last_row = c->p_row1;
  const uint32_t QW = ceil_div(wl, 64);
  // both queries' stable compaction and subgraph in one launch
  QrsArgs q{};
  q.g = c->g;
  q.win = Window{inst[0].wb, wl};
  q.win1 = Window{inst[1].wb, wl};
  q.QW = QW;
  q.prune = c->prune ? 1 : 0;
  q.rI = rI[0];
  q.rU = rU[0];
  q.rI1 = rI[1];
  q.rU1 = rU[1];
  q.row = c->row;
  q.row1 = c->p_row1;
  q.counts1_out = &(c->ctl + 6)->aux[0];
  q.uv = c->p_uv;
  q.part = c->part;
  q.units = c->p_units;
  q.ucap = (uint32_t)std::min<uint64_t>(2 * (uint64_t)c->ucap, 0xFFFFFFFFull);
  q.cshift = c->qrs_cs;
  q.qcnt = c->p_qcnt;
  q.qrow = c->p_qrow;
  q.cur = c->p_cur;
  q.qcw = c->p_qcw;
  q.qmask = c->p_qmask;
  q.ecap = (uint32_t)std::min<uint64_t>(2 * (uint64_t)c->ecap, 0xFFFFFFFFull);
  q.mcap = c->p_mcap;  // what the pair mask array holds
  q.rowcap = 2 * c->g.V;
  q.ctl = c->ctl + 2;
  q.qerr = c->qerr;
  q.spin_ns = (unsigned long long)c->spin_ms * 1000000ull;
  LaunchCfg qc = cfg_for(c, c->occ_qrs, k0.bps);
  if ((int64_t)qc.blocks > (int64_t)c->num_sms * 4) qc.blocks = c->num_sms * 4;
  if ((e = launch_qrs(q, qc, s)) != cudaSuccess) return cuda_fail(c, e, "launch subgraph extraction");
  const bool mixed = inst[0].type != inst[1].type;
  auto kind_of = [](int t) { return t == 0 ? kKindSum : t == 1 ? kKindMaxNot : t == 2 ? kKindHop : kKindMax; };
  RelaxArgs r{};
  r.g = c->g;
  r.win = Window{inst[0].wb, wl};
  r.win1 = Window{inst[1].wb, wl};
  r.s0 = 0;
  r.ls = wl;
  r.QW = QW;
  r.rI = rI[0];
  r.rI1 = rI[1];
  r.row = c->row;
  r.row1 = c->p_row1;
  r.uv = c->p_uv;
  r.qrow = c->p_qrow;
  r.qcw = c->p_qcw;
  r.qmask = c->p_qmask;
  r.counts = &(c->ctl + 2)->aux[0];
  r.counts1 = &(c->ctl + 6)->aux[0];
  if (mixed) {
    r.kind0 = kind_of(inst[0].type);
    r.kind1 = kind_of(inst[1].type);
    r.flip = (inst[0].type == 1 ? 1u : 0u) | (inst[1].type == 1 ? 2u : 0u);
  }
  r.val = c->p_val;
  r.LP = P * K;
  r.stamp = c->p_stamp;
  r.q0 = c->p_q0;
  r.q1 = c->p_q1;
  r.qcap = (uint32_t)c->p_qcap;
  r.cshift = c->relax_cs;
  r.ctl = c->ctl + 3;
  r.qerr = c->qerr;
  r.maxit = c->maxit ? c->maxit : 2 * c->g.V + 2u;
  r.spin_ns = (unsigned long long)c->spin_ms * 1000000ull;
  if ((e = launch_relax(mixed ? kTypeMixed : inst[0].type, P, K, r, cfg_for(c, c->occ_relax, k0.bps), s)) !=
      cudaSuccess)
    return cuda_fail(c, e, "launch paired relaxation");
  for (int qi = 0; qi < 2; ++qi) {
    ScatterArgs sa{};
    sa.V = c->g.V;
    sa.s0 = 0;
    sa.ls = wl;
    sa.rI = rI[qi];
    sa.row = qi ? c->p_row1 : c->row;
    sa.val = c->p_val;
    sa.LP = P * K;
    sa.out = out[qi];
    sa.qerr = c->qerr;
    sa.rflip = ((r.flip >> qi) & 1u) ? 0xFFFFFFFFu : 0u;
    if ((e = launch_scatter(sa, s)) != cudaSuccess) return cuda_fail(c, e, "launch scatter");
  }
  *done = true;
  return SVV_OK;
}

}  // namespace svv
