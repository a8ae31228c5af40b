// svv_batch_api.cu -- host side of svv_query_batch: per-team scratch pool,
// per-instance arrays, one persistent launch of the batch kernel.
#include <cstring>

#include "svv_ctx.h"

namespace svv {

void free_batch(svv_ctx* c) {
  BatchPool& p = c->batch;
  for (void* b : p.bufs) cudaFree(b);
  for (void* b : p.ibufs) cudaFree(b);
  c->allocated -= std::min<uint64_t>(c->allocated, p.bytes + p.ibytes);
  p = BatchPool{};
}

// bytes one team needs for windows up to L (its share of query scratch)
static uint64_t team_bytes(const svv_ctx* c, uint32_t LP, uint32_t QW, uint32_t team_blocks) {
  const uint64_t V = c->g.V, E = std::max<uint32_t>(c->g.E, 1), NF = std::max<uint32_t>(c->g.NF, 1);
  const uint64_t qcap = V + E / (1u << std::min(c->solve_cs, c->relax_cs)) + 64;
  const uint64_t ucap = V + E / (1u << c->qrs_cs) + 64;
  uint64_t b = 0;
  b += 5 * round256(V * 4);                  // rI, rU, stamp, row, uv
  b += round256(4ull * team_blocks * 4);     // part
  b += 2 * round256(2 * V * 4);              // qcnt, cur
  b += round256(V * 16);                     // qrow
  b += round256(E * 8);                      // qcw
  b += round256(NF * QW * 8);                // qmask
  b += round256(V * LP * 4);                 // val
  b += 2 * round256(qcap * 8) + round256(ucap * 8);
  b += round256((V + (E >> 4) + 64) * 4);  // procv
  return b;
}

static svv_status alloc_team(svv_ctx* c, std::vector<void*>& owner, uint32_t LP, uint32_t QW, uint32_t team_blocks,
                      TeamScratch& t) {
  const uint64_t V = c->g.V, E = std::max<uint32_t>(c->g.E, 1), NF = std::max<uint32_t>(c->g.NF, 1);
  const uint64_t qcap = V + E / (1u << std::min(c->solve_cs, c->relax_cs)) + 64;
  const uint64_t ucap = V + E / (1u << c->qrs_cs) + 64;
  svv_status st;
  if ((st = alloc_n(c, owner, V, &t.rI)) || (st = alloc_n(c, owner, V, &t.rU)) ||
      (st = alloc_n(c, owner, V, &t.stamp)) || (st = alloc_n(c, owner, V, &t.row)) ||
      (st = alloc_n(c, owner, V, &t.uv)) || (st = alloc_n(c, owner, 4ull * team_blocks, &t.part)) ||
      (st = alloc_n(c, owner, 2 * V, &t.qcnt)) || (st = alloc_n(c, owner, 2 * V, &t.cur)) ||
      (st = alloc_n(c, owner, V, &t.qrow)) || (st = alloc_n(c, owner, E, &t.qcw)) ||
      (st = alloc_n(c, owner, NF * QW, &t.qmask)) || (st = alloc_n(c, owner, V * LP, &t.val)) ||
      (st = alloc_n(c, owner, qcap, &t.q0)) || (st = alloc_n(c, owner, qcap, &t.q1)) ||
      (st = alloc_n(c, owner, ucap, &t.units)) || (st = alloc_n(c, owner, V + (E >> 4) + 64, &t.procv)))
    return st;
  t.pcap = (uint32_t)(V + (E >> 4) + 64);
  t.qcap = (uint32_t)qcap;
  t.ucap = (uint32_t)ucap;
  t.ecap = (uint32_t)E;
  t.mcap = NF * QW;
  return SVV_OK;
}

// teams with scratch for windows up to L; fewer teams when the budget is short
svv_status ensure_pool(svv_ctx* c, int want_teams, uint32_t L) {
  BatchPool& p = c->batch;
  uint32_t P, K;
  slab_shape(std::min(L, kMaxSlab), P, K);
  const uint32_t LP = P * K, QW = ceil_div(L, 64);
  const int per_sm = std::max(1, std::min(c->occ_batch, 2));
  const int total_blocks = c->num_sms * per_sm;
  want_teams = std::max(1, std::min(want_teams, total_blocks));
  // the grid is split evenly, so a different team count needs a new pool
  if (p.teams && p.want == want_teams && p.LP >= LP && p.QW >= QW) return SVV_OK;
  // (re)build
  for (void* b : p.bufs) cudaFree(b);
  c->allocated -= std::min<uint64_t>(c->allocated, p.bytes);
  p.bufs.clear();
  p.bytes = 0;
  p.teams = 0;
  const uint64_t before = c->allocated;
  int teams = want_teams;
  if (c->budget) {
    const uint64_t per = team_bytes(c, LP, QW, total_blocks / teams + 1);
    const uint64_t room = c->budget > c->allocated ? c->budget - c->allocated : 0;
    teams = (int)std::min<uint64_t>(teams, room / (per + 4096));
    if (teams < 1) return fail(c, SVV_ENOMEM, "batch scratch of one team exceeds the device budget");
  }
  const uint32_t team_blocks = (uint32_t)(total_blocks / teams);
  std::vector<TeamScratch> host(teams);
  svv_status st;
  for (int i = 0; i < teams; ++i)
    if ((st = alloc_team(c, p.bufs, LP, QW, (uint32_t)total_blocks, host[i]))) return st;  // any team size
  if ((st = alloc_n(c, p.bufs, (uint64_t)teams, &p.d_sc)) ||
      (st = alloc_n(c, p.bufs, (uint64_t)teams * kBatchCtl, &p.d_ctl)))
    return st;
  cudaError_t e = cudaMemcpy(p.d_sc, host.data(), sizeof(TeamScratch) * teams, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "uploading team scratch");
  p.want = want_teams;
  p.teams = teams;
  p.team_blocks = team_blocks;
  p.LP = LP;
  p.QW = QW;
  p.bytes = c->allocated - before;
  return SVV_OK;
}

namespace {

svv_status ensure_instances(svv_ctx* c, uint32_t n) {
  BatchPool& p = c->batch;
  if (p.icap >= n && p.d_inst) return SVV_OK;
  for (void* b : p.ibufs) cudaFree(b);
  c->allocated -= std::min<uint64_t>(c->allocated, p.ibytes);
  p.ibufs.clear();
  p.ibytes = 0;
  p.icap = 0;
  const uint64_t before = c->allocated;
  const uint32_t cap = std::max<uint32_t>(n, 64);
  svv_status st;
  if ((st = alloc_n(c, p.ibufs, cap, &p.d_inst)) || (st = alloc_n(c, p.ibufs, cap, &p.d_qerr)) ||
      (st = alloc_n(c, p.ibufs, cap, &p.d_done)) || (st = alloc_n(c, p.ibufs, cap, &p.d_t0)) ||
      (st = alloc_n(c, p.ibufs, cap, &p.d_t1)) || (st = alloc_n(c, p.ibufs, 1, &p.d_next)))
    return st;
  p.icap = cap;
  p.ibytes = c->allocated - before;
  return SVV_OK;
}

}  // namespace

// Teams for batched work: the "batch_teams" knob, else by graph size.  A query
// on a graph of a few million vertices already fills the GPU in its big rounds,
// so splitting the grid only pays for smaller graphs (8 teams up to 1M
// vertices, 2 at 4M, 1 from 8M).
int default_teams(const svv_ctx* c) {
  if (c->batch_teams > 0) return c->batch_teams;
  const uint64_t t = (8ull << 20) / std::max<uint64_t>(c->g.V, 1);
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(8, t));
}

// One launch for the batch, or the instances in order (svv_query's kernels).
// From 2M vertices a query's big rounds already fill the GPU and the
// per-phase kernels run at higher occupancy than the all-phase batch kernel,
// so teams sharing the grid lose to queries in order.
bool batch_one_launch(const svv_ctx* c) {
  if (c->batch_mode) return c->batch_mode == 1;
  return c->g.V < (2u << 20);
}

BatchArgs batch_args(svv_ctx* c) {
  BatchPool& p = c->batch;
  BatchArgs b{};
  b.g = c->g;
  b.inst = p.d_inst;
  b.next = p.d_next;
  b.qerr = p.d_qerr;
  b.done = p.d_done;
  b.t_start = p.d_t0;
  b.t_end = p.d_t1;
  b.scratch = p.d_sc;
  b.ctl = p.d_ctl;
  b.team_blocks = p.team_blocks;
  b.solve_cs = c->solve_cs;
  b.relax_cs = c->relax_cs;
  b.qrs_cs = c->qrs_cs;
  b.delta[0] = c->delta[0];
  b.delta[1] = c->delta[1];
  b.maxit = c->maxit;
  b.spin_ns = (unsigned long long)c->spin_ms * 1000000ull;
  b.skip_same = c->skip_same ? 1u : 0u;
  if (c->g.ifd && c->pull_pct) {
    const uint64_t all_units = (uint64_t)c->g.V + (c->g.E >> c->solve_cs);
    b.pull_units = (uint32_t)std::max<uint64_t>(1, all_units * c->pull_pct / 100);
    b.push_verts = (uint32_t)std::max<uint64_t>(1, (uint64_t)c->g.V * c->pull_pct / 100);
  }
  return b;
}

svv_status check_spec(const svv_ctx* c, const svv_query_spec& q) {
  if ((int)q.type < 0 || (int)q.type > 3) return SVV_EINVAL;
  if (q.source >= c->g.V || q.win_len == 0 || (uint64_t)q.win_begin + q.win_len > c->g.S || !q.out)
    return SVV_EINVAL;
  return SVV_OK;
}

svv_status status_of(uint32_t qerr, uint32_t done) {
  if (!done) return SVV_ETIMEOUT;
  if (qerr == 0) return SVV_OK;
  if (qerr == kErrTimeout) return SVV_ETIMEOUT;
  if (qerr == SVV_ECUDA || qerr == SVV_ENOMEM) return (svv_status)qerr;  // the serving scheduler's failures
  return SVV_EINTERNAL;
}

}  // namespace svv

using namespace svv;

extern "C" svv_status svv_query_batch(svv_ctx* c, uint32_t n, svv_query_spec* specs, void* stream) {
  if (!c || (n && !specs)) return SVV_EINVAL;
  if (!c->loaded) return fail(c, SVV_ENOTLOADED, "no graph loaded");
  if (n == 0) return SVV_OK;
  DeviceGuard dg(c->device);
  std::vector<BatchInstance> inst;
  std::vector<uint32_t> idx;
  uint32_t Lmax = 1;
  svv_status first_bad = SVV_OK;
  for (uint32_t i = 0; i < n; ++i) {
    svv_status st = check_spec(c, specs[i]);
    specs[i].status = st;
    if (st) {
      if (!first_bad) first_bad = st;
      continue;
    }
    inst.push_back(BatchInstance{(int)specs[i].type, specs[i].source, specs[i].win_begin, specs[i].win_len,
                                 specs[i].out});
    idx.push_back(i);
    Lmax = std::max(Lmax, specs[i].win_len);
  }
  if (inst.empty()) return fail(c, first_bad, "no valid query in the batch");
  const uint32_t m = (uint32_t)inst.size();
  cudaStream_t s = (cudaStream_t)stream;
  svv_status st;
  // a failure of the whole call leaves no valid result: every spec says so
  auto fail_all = [&](svv_status why) {
    for (uint32_t k = 0; k < m; ++k) specs[idx[k]].status = why;
    return why;
  };
  // outputs in host memory (page-locked or not) run in order, staged
  std::vector<char> host_out(m, 0);
  bool any_host = false;
  for (uint32_t k = 0; k < m; ++k) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, inst[k].out) != cudaSuccess) {
      cudaGetLastError();
      at.type = cudaMemoryTypeUnregistered;
    }
    host_out[k] = at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
    any_host |= host_out[k] != 0;
  }
  if (any_host || !batch_one_launch(c)) {
    if ((st = ensure_instances(c, m))) return fail_all(st);
    std::vector<uint32_t> qerr(m);
    float ms = 0.f;
    {
      ServeFence fence(c, s);
      if ((st = batch_in_order(c, inst.data(), m, any_host ? host_out.data() : nullptr, c->batch.d_qerr,
                               qerr.data(), s, &ms)))
        return fail_all(st);
    }
    svv_status overall = first_bad;
    for (uint32_t k = 0; k < m; ++k) {
      const svv_status si = status_of(qerr[k], 1u);
      specs[idx[k]].status = si;
      if (si && !overall) overall = si;
    }
    c->stats = svv_stats{};
    c->stats.ms_batch = ms;
    c->stats.batch_teams = 0;
    if (c->gev_pending) {  // the stream was synchronised at the end of the batch
      cudaEventElapsedTime(&c->stats.ms_group_cap, c->gev[0], c->gev[1]);
      cudaEventElapsedTime(&c->stats.ms_group_cup, c->gev[1], c->gev[2]);
      c->stats.phase_timing = 1;
      c->gev_pending = false;
    }
    if (overall) return fail(c, overall, "some batched queries failed");
    c->err.clear();
    return SVV_OK;
  }
  if ((st = ensure_pool(c, default_teams(c), Lmax))) return fail_all(st);
  if ((st = ensure_instances(c, m))) return fail_all(st);
  BatchPool& p = c->batch;
  cudaError_t e = cudaMemcpyAsync(p.d_inst, inst.data(), sizeof(BatchInstance) * m, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.d_ctl, 0, sizeof(TeamCtl) * kBatchCtl * p.teams, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.d_next, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.d_qerr, 0, sizeof(uint32_t) * m, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.d_done, 0, sizeof(uint32_t) * m, s);
  if (e != cudaSuccess) return fail_all(cuda_fail(c, e, "batch setup"));
  BatchArgs b = batch_args(c);
  b.n_inst = m;
  // fewer instances than teams: fewer, larger teams over the same grid
  const int teams = std::min<int>(p.teams, (int)m);
  b.team_blocks = (uint32_t)(p.teams * (int)p.team_blocks / teams);
  if ((e = launch_batch(b, LaunchCfg{teams * (int)b.team_blocks, 512}, s)) != cudaSuccess)
    return fail_all(cuda_fail(c, e, "launch batch"));
  std::vector<uint32_t> qerr(m), done(m);
  std::vector<unsigned long long> t0(m), t1(m);
  e = cudaMemcpyAsync(qerr.data(), p.d_qerr, 4ull * m, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(done.data(), p.d_done, 4ull * m, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t0.data(), p.d_t0, 8ull * m, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t1.data(), p.d_t1, 8ull * m, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_all(cuda_fail(c, e, "batch"));
  svv_status overall = first_bad;
  unsigned long long lo = ~0ull, hi = 0;
  for (uint32_t k = 0; k < m; ++k) {
    const svv_status si = status_of(qerr[k], done[k]);
    specs[idx[k]].status = si;
    if (si && !overall) overall = si;
    if (done[k]) {
      lo = std::min(lo, t0[k]);
      hi = std::max(hi, t1[k]);
    }
  }
  c->stats = svv_stats{};
  c->stats.ms_batch = hi > lo ? (float)((hi - lo) / 1e6) : 0.f;
  c->stats.batch_teams = (uint32_t)teams;
  c->stats.batch_team_blocks = b.team_blocks;
  if (overall) return fail(c, overall, "some batched queries failed");
  c->err.clear();
  return SVV_OK;
}
