// svv_api.cu -- the C ABI declared in include/svv.h: context, resident graph,
// scratch sizing and the stream-ordered query pipelines.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "svv_ctx.h"

using namespace svv;

namespace svv {

void free_list(svv_ctx*, std::vector<void*>& bufs) {
  for (void* p : bufs) cudaFree(p);
  bufs.clear();
}

void free_graph(svv_ctx* c) {
  free_serve(c);
  free_batch(c);
  free_group(c);
  free_pair(c);
  free_list(c, c->graph_bufs);
  free_list(c, c->scratch_bufs);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  free_list(c, c->bstage_bufs);
  c->bstage[0] = c->bstage[1] = nullptr;
  c->bstage_cap = 0;
  c->allocated = 0;
  c->loaded = false;
  c->g = DevGraph{};
  c->qmask = nullptr;
  c->val = nullptr;
  c->staging = nullptr;
  c->mcap = c->valcap = c->staging_cap = 0;
}

Knobs default_knobs(const svv_ctx* c, int type) {
  const uint32_t delta = (type == 0 || type == 1) ? c->delta[type] : 0u;
  return Knobs{c->solve_cs, c->bps, c->relax_lanes, c->skip_same, c->pull_pct, delta, c->slab_max};
}

// the knobs the autotuner chose for this type and window length (the nearest
// tuned length bucket), else the defaults
Knobs knobs_of(const svv_ctx* c, int type, uint32_t L) {
  if (type < 0 || type > 3) return default_knobs(c, 0);
  const int b = len_bucket(L);
  for (int d = 0; d < kLenBuckets; ++d) {
    if (b - d >= 0 && c->has_tuned[type][b - d]) return c->tuned[type][b - d];
    if (b + d < kLenBuckets && c->has_tuned[type][b + d]) return c->tuned[type][b + d];
  }
  return default_knobs(c, type);
}

LaunchCfg cfg_for(const svv_ctx* c, int occ, int bps) {
  int per_sm = occ;
  if (bps > 0) per_sm = std::min(per_sm, bps);
  per_sm = std::max(1, std::min(per_sm, 4));
  return LaunchCfg{c->num_sms * per_sm, c->threads};
}

svv_status ensure_window(svv_ctx* c, uint32_t L) {
  const uint32_t QW = ceil_div(L, 64);
  const uint64_t need_m = (uint64_t)std::max<uint32_t>(c->g.NF, 1) * QW;
  uint32_t P, K;
  slab_shape(std::min(L, kMaxSlab), P, K);  // any slab width a query of L may use
  const uint64_t need_v = (uint64_t)std::max<uint32_t>(c->g.V, 1) * P * K;
  // an in-order server's queued requests, or stream-ordered queries, may
  // still read the old buffers
  if ((need_m > c->mcap || need_v > c->valcap) && c->serve.active && c->serve.stream)
    cudaStreamSynchronize(c->serve.stream);
  if ((need_m > c->mcap || need_v > c->valcap) && c->async_last) cudaEventSynchronize(c->async_last);
  if (need_m > c->mcap) {
    if (c->qmask) {
      auto it = std::find(c->scratch_bufs.begin(), c->scratch_bufs.end(), (void*)c->qmask);
      if (it != c->scratch_bufs.end()) c->scratch_bufs.erase(it);
      cudaFree(c->qmask);
      c->allocated -= ((c->mcap * 8 + 255) & ~uint64_t(255));
      c->qmask = nullptr;
      c->mcap = 0;
    }
    svv_status s = alloc_n(c, c->scratch_bufs, need_m, &c->qmask);
    if (s) return s;
    c->mcap = need_m;
  }
  if (need_v > c->valcap) {
    if (c->val) {
      auto it = std::find(c->scratch_bufs.begin(), c->scratch_bufs.end(), (void*)c->val);
      if (it != c->scratch_bufs.end()) c->scratch_bufs.erase(it);
      cudaFree(c->val);
      c->allocated -= ((c->valcap * 4 + 255) & ~uint64_t(255));
      c->val = nullptr;
      c->valcap = 0;
    }
    svv_status s = alloc_n(c, c->scratch_bufs, need_v, &c->val);
    if (s) return s;
    c->valcap = need_v;
  }
  return SVV_OK;
}

svv_status check_query(svv_ctx* c, int type, uint32_t source, uint32_t wb, uint32_t wl, const void* out) {
  if (!c) return SVV_EINVAL;
  if (!c->loaded) return fail(c, SVV_ENOTLOADED, "no graph loaded");
  if (type < 0 || type > 3) return fail(c, SVV_EINVAL, "unknown query type");
  if (source >= c->g.V) return fail(c, SVV_EINVAL, "source >= V");
  if (wl == 0) return fail(c, SVV_EINVAL, "win_len == 0");
  if ((uint64_t)wb + wl > c->g.S) return fail(c, SVV_EINVAL, "win_begin + win_len > S");
  if (!out) return fail(c, SVV_EINVAL, "out is NULL");
  return SVV_OK;
}

SolveArgs solve_base(svv_ctx* c, uint32_t wb, uint32_t wl, int type, const Knobs& kn) {
  SolveArgs a{};
  a.g = c->g;
  a.win = Window{wb, wl};
  a.stamp = c->stamp;
  a.q0 = c->q0;
  a.q1 = c->q1;
  a.qcap = c->qcap;
  a.cshift = kn.solve_cs;
  a.qerr = c->qerr;
  a.delta = (type == 0 || type == 1) ? kn.delta : 0u;
  // deferred rounds add to the round count, so the default cap is wider
  const uint64_t cap = a.delta ? 16ull * c->g.V + 64 : (uint64_t)c->g.V + 2;
  a.maxit = c->maxit ? c->maxit : (uint32_t)std::min<uint64_t>(cap, 0xFFFFFFF0ull);
  a.spin_ns = (unsigned long long)c->spin_ms * 1000000ull;
  if (c->g.ifd && kn.pull_pct) {
    const uint64_t all_units = (uint64_t)c->g.V + (c->g.E >> kn.solve_cs);
    a.pull_units = (uint32_t)std::max<uint64_t>(1, all_units * kn.pull_pct / 100);
    a.push_verts = (uint32_t)std::max<uint64_t>(1, (uint64_t)c->g.V * kn.pull_pct / 100);
  }
  if (kn.skip_same && c->procv) {
    a.procv = c->procv;
    a.pcap = c->g.V + (c->g.E >> kn.solve_cs) + 2u;  // chunk ids stay below this
  }
  return a;
}

svv_status finish(svv_ctx* c, cudaStream_t s, int nctl_copy) {
  cudaError_t e = cudaMemcpyAsync(c->hctl, c->ctl, sizeof(TeamCtl) * nctl_copy, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->hqerr, c->qerr, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "query");
  const uint32_t q = *c->hqerr;
  if (q == kErrTimeout) return fail(c, SVV_ETIMEOUT, "a device wait or the round cap expired");
  if (q == 2u) return fail(c, SVV_ENOMEM, "rows_out is smaller than U * win_len");
  if (q != 0) return fail(c, SVV_EINTERNAL, "device capacity check failed");
  c->err.clear();
  return SVV_OK;
}

}  // namespace svv

extern "C" {

const char* svv_status_str(svv_status s) {
  switch (s) {
    case SVV_OK: return "SVV_OK";
    case SVV_EINVAL: return "SVV_EINVAL";
    case SVV_ENOMEM: return "SVV_ENOMEM";
    case SVV_ECUDA: return "SVV_ECUDA";
    case SVV_ETIMEOUT: return "SVV_ETIMEOUT";
    case SVV_EBUSY: return "SVV_EBUSY";
    case SVV_ENOTLOADED: return "SVV_ENOTLOADED";
    case SVV_EINTERNAL: return "SVV_EINTERNAL";
  }
  return "SVV_UNKNOWN";
}

const char* svv_last_error(const svv_ctx* c) { return c ? c->err.c_str() : ""; }

uint64_t svv_device_bytes(const svv_ctx* c) { return c ? c->allocated : 0; }

svv_status svv_create(svv_ctx** out, int device, uint64_t budget) {
  if (!out) return SVV_EINVAL;
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SVV_ECUDA;
  }
  if (device < 0 || device >= n) return SVV_EINVAL;
  svv_ctx* c = new (std::nothrow) svv_ctx();
  if (!c) return SVV_ENOMEM;
  c->device = device;
  c->budget = budget;
  c->budget_auto = budget == 0;
  DeviceGuard dg(device);
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (!coop || c->num_sms <= 0) {
    delete c;
    return SVV_ECUDA;
  }
  c->occ_solve = occupancy_solve(c->threads);
  c->occ_qrs = occupancy_qrs(c->threads);
  c->occ_relax = occupancy_relax(c->threads);
  c->occ_batch = occupancy_batch(c->threads);
  c->occ_group = occupancy_group(c->threads, false);
  c->occ_group2 = occupancy_group(c->threads, true);
  if (c->occ_solve <= 0 || c->occ_qrs <= 0 || c->occ_relax <= 0 || c->occ_batch <= 0 || c->occ_group <= 0 ||
      c->occ_group2 <= 0) {
    delete c;
    return SVV_ECUDA;
  }
  e = cudaMallocHost((void**)&c->hctl, sizeof(TeamCtl) * kNumCtl);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->hqerr, sizeof(uint32_t));
  if (e != cudaSuccess) {
    if (c->hctl) cudaFreeHost(c->hctl);
    delete c;
    cudaGetLastError();
    return SVV_ENOMEM;
  }
  *out = c;
  return SVV_OK;
}

void svv_destroy(svv_ctx* c) {
  if (!c) return;
  {
    DeviceGuard dg(c->device);
    cudaDeviceSynchronize();
    free_graph(c);
    if (c->hctl) cudaFreeHost(c->hctl);
    if (c->hqerr) cudaFreeHost(c->hqerr);
    for (auto& e : c->ev)
      if (e) cudaEventDestroy(e);
    for (auto& e : c->bev)
      if (e) cudaEventDestroy(e);
    for (auto& e : c->gev)
      if (e) cudaEventDestroy(e);
    for (int i = 0; i < 2; ++i) {
      if (c->ev_done[i]) cudaEventDestroy(c->ev_done[i]);
      if (c->ev_copied[i]) cudaEventDestroy(c->ev_copied[i]);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    for (auto& e : c->aev)
      if (e) cudaEventDestroy(e);
    if (c->astatus) cudaFreeHost(c->astatus);
    if (c->trace) cudaFree(c->trace);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->bgexec) cudaGraphExecDestroy(c->bgexec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  }
  delete c;
}

svv_status svv_set_tuning(svv_ctx* c, const char* key, int64_t v) {
  if (!c || !key) return SVV_EINVAL;
  auto log2_ok = [](int64_t x, int lo, int hi, uint32_t& out) {
    for (int s = lo; s <= hi; ++s)
      if (x == (int64_t(1) << s)) {
        out = (uint32_t)s;
        return true;
      }
    return false;
  };
  std::string k(key);
  if (k == "max_iters") {
    if (v < 0 || v > 0xFFFFFFF0ll) return fail(c, SVV_EINVAL, "max_iters out of range");
    c->maxit = (uint32_t)v;
  } else if (k == "spin_limit_ms") {
    if (v < 1 || v > 600000) return fail(c, SVV_EINVAL, "spin_limit_ms out of range");
    c->spin_ms = (uint32_t)v;
  } else if (k == "solve_chunk") {
    if (!log2_ok(v, 4, 12, c->solve_cs)) return fail(c, SVV_EINVAL, "solve_chunk: power of two in [16, 4096]");
  } else if (k == "relax_chunk") {
    if (!log2_ok(v, 3, 12, c->relax_cs)) return fail(c, SVV_EINVAL, "relax_chunk: power of two in [8, 4096]");
  } else if (k == "qrs_chunk") {
    if (!log2_ok(v, 5, 14, c->qrs_cs)) return fail(c, SVV_EINVAL, "qrs_chunk: power of two in [32, 16384]");
  } else if (k == "phase_timing") {
    if (v != 0 && v != 1) return fail(c, SVV_EINVAL, "phase_timing is 0 or 1");
    if (v && !c->ev[0]) {
      DeviceGuard dg(c->device);
      for (auto& e : c->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "cudaEventCreate");
    }
    c->phase_timing = v != 0;
  } else if (k == "slab_max") {
    if (v < 1 || v > (int64_t)kMaxSlab) return fail(c, SVV_EINVAL, "slab_max in [1, 128]");
    c->slab_max = (uint32_t)v;
  } else if (k == "prune") {
    if (v != 0 && v != 1) return fail(c, SVV_EINVAL, "prune is 0 or 1");
    c->prune = v != 0;
  } else if (k == "pull") {
    if (v != 0 && v != 1) return fail(c, SVV_EINVAL, "pull is 0 or 1");
    c->pull = v != 0;  // takes effect at the next svv_load
  } else if (k == "pull_pct") {
    if (v < 0 || v > 100) return fail(c, SVV_EINVAL, "pull_pct in [0, 100]");
    c->pull_pct = (uint32_t)v;
  } else if (k == "graph") {
    if (v != 0 && v != 1) return fail(c, SVV_EINVAL, "graph is 0 or 1");
    c->graph_mode = v != 0;
  } else if (k == "relax_lanes") {
    if (v != 8 && v != 16 && v != 32) return fail(c, SVV_EINVAL, "relax_lanes is 8, 16 or 32");
    c->relax_lanes = (uint32_t)v;
  } else if (k == "skip_same") {
    if (v != 0 && v != 1) return fail(c, SVV_EINVAL, "skip_same is 0 or 1");
    c->skip_same = v != 0;
  } else if (k == "batch_mode") {
    if (v < 0 || v > 2) return fail(c, SVV_EINVAL, "batch_mode is 0 (by graph size), 1 (one launch) or 2 (in order)");
    c->batch_mode = (int)v;
  } else if (k == "pair_tails") {
    if (v < 0 || v > 1) return fail(c, SVV_EINVAL, "pair_tails: 0 or 1");
    c->pair_tails = v != 0;
  } else if (k == "group_mix") {
    if (v < 0 || v > 1) return fail(c, SVV_EINVAL, "group_mix: 0 or 1");
    c->group_mix = v != 0;
  } else if (k == "group_pull_pct" || k == "group_pull_pct_union") {
    if (v < 0 || v > 100) return fail(c, SVV_EINVAL, k + " in [0, 100]");
    c->group_pull_pct[k == "group_pull_pct" ? 0 : 1] = (uint32_t)v;
  } else if (k == "test_skip_arrival") {
    if (v < 0 || v > 0xFFFF) return fail(c, SVV_EINVAL, "test_skip_arrival in [0, 65535]");
    c->skip_arrival = (uint32_t)v;
  } else if (k == "isolated_fast") {
    if (v != 0 && v != 1) return fail(c, SVV_EINVAL, "isolated_fast is 0 or 1");
    c->isolated_fast = v != 0;
  } else if (k == "group_max") {
    if (v < 1 || v > kGroupMax) return fail(c, SVV_EINVAL, "group_max in [1, 8]");
    c->group_max = (uint32_t)v;
  } else if (k == "batch_teams") {
    if (v < 0 || v > 64) return fail(c, SVV_EINVAL, "batch_teams in [0, 64]");
    c->batch_teams = (int)v;
  } else if (k == "round_trace") {
    if (v != 0 && v != 1) return fail(c, SVV_EINVAL, "round_trace is 0 or 1");
    if (v && !c->trace) {
      DeviceGuard dg(c->device);
      if (cudaMalloc(&c->trace, 4 * kTraceCap * sizeof(unsigned long long)) != cudaSuccess) {
        c->trace = nullptr;
        return cuda_fail(c, cudaGetLastError(), "trace buffer");
      }
    }
    c->round_trace = v != 0;
  } else if (k == "delta_sssp" || k == "delta_sswp") {
    if (v < 0 || v > 0x7FFFFFFF) return fail(c, SVV_EINVAL, k + " out of range");
    c->delta[k == "delta_sssp" ? 0 : 1] = (uint32_t)v;
  } else if (k == "blocks_per_sm") {
    if (v < 0 || v > 4) return fail(c, SVV_EINVAL, "blocks_per_sm in [0, 4]");
    c->bps = (int)v;
  } else {
    return fail(c, SVV_EINVAL, "unknown tuning key: " + k);
  }
  // capacities depend on the chunk sizes: resize on the next load
  if (c->loaded && (k == "solve_chunk" || k == "relax_chunk" || k == "qrs_chunk")) {
    const uint64_t need_q = (uint64_t)c->g.V + c->g.E / (1u << std::min(c->solve_cs, c->relax_cs)) + 64;
    const uint64_t need_u = (uint64_t)c->g.V + c->g.E / (1u << c->qrs_cs) + 64;
    if (need_q > c->qcap || need_u > c->ucap) {
      return fail(c, SVV_EINVAL, "chunk smaller than the one the graph was loaded with; set it before svv_load");
    }
  }
  return SVV_OK;
}

svv_status svv_get_stats(svv_ctx* c, svv_stats* out) {
  if (!c || !out) return SVV_EINVAL;
  *out = c->stats;
  return SVV_OK;
}

svv_status svv_load(svv_ctx* c, uint32_t V, uint64_t E, uint32_t S, const uint64_t* row_ptr,
                    const uint32_t* col, const uint32_t* weight, const uint64_t* mask,
                    int inputs_on_device) {
  if (!c) return SVV_EINVAL;
  if (V == 0 || V >= 0xFFFFFFFFu) return fail(c, SVV_EINVAL, "V must be in [1, 2^32-2]");
  if (S == 0) return fail(c, SVV_EINVAL, "S must be >= 1");
  if (E >= 0xFFFFFFFFull) return fail(c, SVV_EINVAL, "E must be < 2^32-1");
  if (!row_ptr || (E && (!col || !weight || !mask))) return fail(c, SVV_EINVAL, "NULL input array");
  DeviceGuard dg(c->device);
  const uint32_t W = ceil_div(S, 64);

  // host copies of device inputs
  std::vector<uint64_t> h_rp, h_mask;
  std::vector<uint32_t> h_col, h_w;
  if (inputs_on_device) {
    h_rp.resize((size_t)V + 1);
    h_col.resize(E);
    h_w.resize(E);
    h_mask.resize((size_t)E * W);
    cudaError_t e = cudaMemcpy(h_rp.data(), row_ptr, h_rp.size() * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && E) e = cudaMemcpy(h_col.data(), col, E * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && E) e = cudaMemcpy(h_w.data(), weight, E * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && E) e = cudaMemcpy(h_mask.data(), mask, h_mask.size() * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "copying device inputs");
    row_ptr = h_rp.data();
    col = h_col.data();
    weight = h_w.data();
    mask = h_mask.data();
  }
  // validate
  if (row_ptr[0] != 0) return fail(c, SVV_EINVAL, "row_ptr[0] != 0");
  for (uint32_t v = 0; v < V; ++v)
    if (row_ptr[v + 1] < row_ptr[v]) return fail(c, SVV_EINVAL, "row_ptr not non-decreasing");
  if (row_ptr[V] != E) return fail(c, SVV_EINVAL, "row_ptr[V] != E");
  for (uint64_t e = 0; e < E; ++e)
    if (col[e] >= V) return fail(c, SVV_EINVAL, "col >= V");

  // classify against the history [0, S): full / partial / absent
  std::vector<uint64_t> hist(W);
  for (uint32_t j = 0; j < W; ++j) {
    const uint32_t n = std::min<uint32_t>(64, S - 64 * j);
    hist[j] = n == 64 ? ~0ull : ((1ull << n) - 1ull);
  }
  std::vector<uint32_t> rp((size_t)V + 1, 0), nfp((size_t)V + 1, 0);
  std::vector<uint8_t> kind(E);  // 0 absent, 1 full, 2 partial
  for (uint32_t v = 0; v < V; ++v) {
    uint32_t nfull = 0, npart = 0;
    for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      bool all = true, any = false;
      const uint64_t* m = mask + e * W;
      for (uint32_t j = 0; j < W; ++j) {
        const uint64_t x = m[j] & hist[j];
        all &= (x == hist[j]);
        any |= (x != 0);
      }
      kind[e] = all ? 1 : (any ? 2 : 0);
      nfull += all;
      npart += (!all && any);
    }
    rp[v + 1] = rp[v] + nfull + npart;
    nfp[v + 1] = nfp[v] + npart;
  }
  const uint32_t E2 = rp[V], NF = nfp[V];
  std::vector<uint2> cw(std::max<uint32_t>(E2, 1)), nfcw(std::max<uint32_t>(NF, 1));
  std::vector<uint32_t> nfsrc(std::max<uint32_t>(NF, 1));
  std::vector<uint64_t> nfm((size_t)std::max<uint32_t>(NF, 1) * W);
  for (uint32_t v = 0; v < V; ++v) {
    uint32_t pf = rp[v], pn = rp[v + 1] - (nfp[v + 1] - nfp[v]), k = nfp[v];
    for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      if (kind[e] == 1) {
        cw[pf++] = make_uint2(col[e], weight[e]);
      } else if (kind[e] == 2) {
        cw[pn++] = make_uint2(col[e], weight[e]);
        nfcw[k] = make_uint2(col[e], weight[e]);
        nfsrc[k] = v;
        for (uint32_t j = 0; j < W; ++j) nfm[(size_t)k * W + j] = mask[e * W + j] & hist[j];
        ++k;
      }
    }
  }

  // transposed graph, edge-flat: in-edges sorted by target (counting sort;
  // sources ascending within a target), all-snapshot ones and partial ones
  // (with their masks) in separate arrays
  const uint32_t EF = E2 - NF;
  std::vector<uint32_t> ifd, ipd;
  std::vector<uint2> ifcw, ipcw;
  std::vector<uint64_t> ipm;
  if (c->pull) {
    std::vector<uint32_t> pos_f((size_t)V + 1, 0), pos_p((size_t)V + 1, 0);
    for (uint32_t u = 0; u < V; ++u) {
      const uint32_t fe = rp[u + 1] - (nfp[u + 1] - nfp[u]);
      for (uint32_t e = rp[u]; e < rp[u + 1]; ++e) (e < fe ? pos_f : pos_p)[cw[e].x + 1]++;
    }
    for (uint32_t v = 0; v < V; ++v) {
      pos_f[v + 1] += pos_f[v];
      pos_p[v + 1] += pos_p[v];
    }
    ifd.assign(std::max<uint32_t>(EF, 1), 0u);
    ifcw.assign(std::max<uint32_t>(EF, 1), make_uint2(0, 0));
    ipd.assign(std::max<uint32_t>(NF, 1), 0u);
    ipcw.assign(std::max<uint32_t>(NF, 1), make_uint2(0, 0));
    ipm.assign((size_t)std::max<uint32_t>(NF, 1) * W, 0ull);
    for (uint32_t u = 0; u < V; ++u) {
      const uint32_t fe = rp[u + 1] - (nfp[u + 1] - nfp[u]);
      for (uint32_t e = rp[u]; e < rp[u + 1]; ++e) {
        const uint32_t x = cw[e].x;
        if (e < fe) {
          const uint32_t i2 = pos_f[x]++;
          ifd[i2] = x;
          ifcw[i2] = make_uint2(u, cw[e].y);
        } else {
          const uint32_t k = pos_p[x]++;
          ipd[k] = x;
          ipcw[k] = make_uint2(u, cw[e].y);
          for (uint32_t w = 0; w < W; ++w) ipm[(size_t)k * W + w] = nfm[(size_t)(nfp[u] + (e - fe)) * W + w];
        }
      }
    }
  }

  // replace the resident graph
  cudaDeviceSynchronize();
  free_graph(c);
  if (c->budget_auto) {
    // free memory less a margin and the local memory the driver reserves when
    // the batch kernel first runs (its stack frames)
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    const uint64_t keep = (512ull << 20) + batch_local_bytes(c->device);
    c->budget = fr > keep ? fr - keep : fr / 2;
  }
  DevGraph g{};
  g.V = V;
  g.S = S;
  g.W = W;
  g.E = E2;
  g.NF = NF;
  uint32_t *d_rp, *d_nfp, *d_nfsrc;
  uint2 *d_cw, *d_nfcw;
  uint64_t* d_nfm;
  svv_status st;
  if ((st = alloc_n(c, c->graph_bufs, (uint64_t)V + 1, &d_rp)) || (st = alloc_n(c, c->graph_bufs, (uint64_t)V + 1, &d_nfp)) ||
      (st = alloc_n(c, c->graph_bufs, std::max<uint32_t>(E2, 1), &d_cw)) ||
      (st = alloc_n(c, c->graph_bufs, (uint64_t)std::max<uint32_t>(NF, 1) * W, &d_nfm)) ||
      (st = alloc_n(c, c->graph_bufs, std::max<uint32_t>(NF, 1), &d_nfsrc)) ||
      (st = alloc_n(c, c->graph_bufs, std::max<uint32_t>(NF, 1), &d_nfcw))) {
    free_graph(c);
    return st;
  }
  cudaError_t e = cudaMemcpy(d_rp, rp.data(), rp.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_nfp, nfp.data(), nfp.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_cw, cw.data(), (size_t)E2 * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_nfm, nfm.data(), (size_t)NF * W * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_nfsrc, nfsrc.data(), (size_t)NF * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_nfcw, nfcw.data(), (size_t)NF * 8, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_graph(c);
    return cuda_fail(c, e, "uploading the graph");
  }
  g.rp = d_rp;
  g.nfp = d_nfp;
  g.cw = d_cw;
  g.nfmask = d_nfm;
  g.nfsrc = d_nfsrc;
  g.nfcw = d_nfcw;
  if (c->pull) {
    uint32_t *d_ifd, *d_ipd;
    uint2 *d_ifcw, *d_ipcw;
    uint64_t* d_ipm;
    if ((st = alloc_n(c, c->graph_bufs, std::max<uint32_t>(EF, 1), &d_ifd)) ||
        (st = alloc_n(c, c->graph_bufs, std::max<uint32_t>(EF, 1), &d_ifcw)) ||
        (st = alloc_n(c, c->graph_bufs, std::max<uint32_t>(NF, 1), &d_ipd)) ||
        (st = alloc_n(c, c->graph_bufs, std::max<uint32_t>(NF, 1), &d_ipcw)) ||
        (st = alloc_n(c, c->graph_bufs, (uint64_t)std::max<uint32_t>(NF, 1) * W, &d_ipm))) {
      free_graph(c);
      return st;
    }
    cudaError_t e2 = cudaMemcpy(d_ifd, ifd.data(), (size_t)EF * 4, cudaMemcpyHostToDevice);
    if (e2 == cudaSuccess) e2 = cudaMemcpy(d_ifcw, ifcw.data(), (size_t)EF * 8, cudaMemcpyHostToDevice);
    if (e2 == cudaSuccess) e2 = cudaMemcpy(d_ipd, ipd.data(), (size_t)NF * 4, cudaMemcpyHostToDevice);
    if (e2 == cudaSuccess) e2 = cudaMemcpy(d_ipcw, ipcw.data(), (size_t)NF * 8, cudaMemcpyHostToDevice);
    if (e2 == cudaSuccess) e2 = cudaMemcpy(d_ipm, ipm.data(), (size_t)NF * W * 8, cudaMemcpyHostToDevice);
    if (e2 != cudaSuccess) {
      free_graph(c);
      return cuda_fail(c, e2, "uploading the transposed graph");
    }
    g.ifd = d_ifd;
    g.ifcw = d_ifcw;
    g.ipd = d_ipd;
    g.ipcw = d_ipcw;
    g.ipmask = d_ipm;
  }

  // scratch sized from V and E
  const uint64_t qcap = (uint64_t)V + E2 / (1u << std::min(c->solve_cs, c->relax_cs)) + 64;
  const uint64_t ucap = (uint64_t)V + E2 / (1u << c->qrs_cs) + 64;
  if (qcap >= 0xFFFFFFFFull || ucap >= 0xFFFFFFFFull) {
    free_graph(c);
    return fail(c, SVV_EINVAL, "graph too large for 32-bit work queues");
  }
  const uint64_t nblk = (uint64_t)c->num_sms * 4;
  if ((st = alloc_n(c, c->scratch_bufs, V, &c->rI)) || (st = alloc_n(c, c->scratch_bufs, V, &c->rU)) ||
      (st = alloc_n(c, c->scratch_bufs, V, &c->stamp)) || (st = alloc_n(c, c->scratch_bufs, V, &c->row)) ||
      (st = alloc_n(c, c->scratch_bufs, V, &c->uv)) || (st = alloc_n(c, c->scratch_bufs, 4 * nblk, &c->part)) ||
      (st = alloc_n(c, c->scratch_bufs, 2ull * V, &c->qcnt)) || (st = alloc_n(c, c->scratch_bufs, 2ull * V, &c->cur)) ||
      (st = alloc_n(c, c->scratch_bufs, V, &c->qrow)) ||
      (st = alloc_n(c, c->scratch_bufs, std::max<uint32_t>(E2, 1), &c->qcw)) ||
      (st = alloc_n(c, c->scratch_bufs, qcap, &c->q0)) || (st = alloc_n(c, c->scratch_bufs, qcap, &c->q1)) ||
      (st = alloc_n(c, c->scratch_bufs, ucap, &c->units)) ||
      (st = alloc_n(c, c->scratch_bufs, kNumCtl, &c->ctl)) || (st = alloc_n(c, c->scratch_bufs, 1, &c->qerr)) ||
      (st = alloc_n(c, c->scratch_bufs, (uint64_t)V + (E2 >> 4) + 64, &c->procv))) {
    free_graph(c);
    return st;
  }
  c->qcap = (uint32_t)qcap;
  c->ucap = (uint32_t)ucap;
  c->pcap = (uint32_t)((uint64_t)V + (E2 >> 4) + 64);
  c->ecap = std::max<uint32_t>(E2, 1);
  c->g = g;
  // out-degree over the edges present in some snapshot: a source without any
  // reaches nothing in any window (the query's result is known without a solve)
  c->hdeg.resize(V);
  for (uint32_t v = 0; v < V; ++v) c->hdeg[v] = rp[v + 1] - rp[v];
  c->loaded = true;
  c->stats = svv_stats{};
  c->err.clear();
  return SVV_OK;
}

}  // extern "C"

namespace svv {

// Enqueue every step of one query on stream s (no host synchronisation, so a
// graph capture can record it).  With timing, CUDA events bracket the phases.
// With rows_out set, the scatter is replaced by a copy of the relaxed rows
// (compact output).

bool source_is_isolated(const svv_ctx* c, uint32_t source) {
  return source < c->hdeg.size() && c->hdeg[source] == 0 && c->isolated_fast;
}

// A source with no out-edge in any snapshot: both bounds (Section 3 Step 1)
// hold the source value at the source and the identity everywhere else, every
// vertex is stable (Theorem 2), and the result is that row in every window
// snapshot.  One kernel writes the result, the bounds and the row map.
svv_status enqueue_isolated(svv_ctx* c, int t, uint32_t source, uint32_t wl, uint32_t* out, cudaStream_t s,
                            bool timing, const CompactOut* co) {
  IsolatedArgs f{};
  f.V = c->g.V;
  f.L = co ? 0u : wl;
  f.source = source;
  f.ident = t == 1 ? 0u : kInf;
  f.src_val = t == 1 ? kInf : 0u;
  f.out = co ? nullptr : out;
  f.rI = c->rI;
  f.rU = c->rU;
  f.row = c->row;
  f.sms = (uint32_t)c->num_sms;
  cudaError_t e = launch_isolated(f, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "launch isolated-source fill");
  c->last_rI = c->rI;
  c->last_rU = c->rU;
  c->last_row = c->row;
  if (co) {
    const size_t n = (size_t)c->g.V * sizeof(uint32_t);
    if (co->cap_out && (e = cudaMemcpyAsync(co->cap_out, c->rI, n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return cuda_fail(c, e, "copy intersection values");
    if (co->row_out && (e = cudaMemcpyAsync(co->row_out, c->row, n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return cuda_fail(c, e, "copy row map");
  }
  if (timing)
    for (int i = 1; i <= 6; ++i) cudaEventRecord(c->ev[i], s);
  return SVV_OK;
}

svv_status enqueue_query(svv_ctx* c, int t, uint32_t source, uint32_t wb, uint32_t wl, uint32_t* out,
                         cudaStream_t s, bool timing, float* ms_relax_out, float* ms_scatter_out,
                         const CompactOut* co) {
  *ms_relax_out = *ms_scatter_out = 0.f;
  cudaError_t e = cudaMemsetAsync(c->ctl, 0, sizeof(TeamCtl) * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->qerr, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  if (timing) cudaEventRecord(c->ev[0], s);
  if (source_is_isolated(c, source)) return enqueue_isolated(c, t, source, wl, out, s, timing, co);

  // a1: intersection graph (edges present in every window snapshot)
  const Knobs kn = knobs_of(c, t, wl);
  SolveArgs a1 = solve_base(c, wb, wl, t, kn);
  a1.init = kInitSource;
  a1.source = source;
  a1.val = c->rI;
  a1.ctl = c->ctl + 0;
  a1.skip_nf = (wb == 0 && wl == c->g.S) ? 1 : 0;
  a1.skip_arrival = c->skip_arrival;
  if (c->round_trace) {
    cudaMemsetAsync(c->trace, 0, 4 * kTraceCap * sizeof(unsigned long long), s);
    a1.trace = c->trace;
    a1.trace_cap = kTraceCap;
  }
  if ((e = launch_solve(t, kPredAll, a1, cfg_for(c, c->occ_solve, kn.bps), s)) != cudaSuccess)
    return cuda_fail(c, e, "launch intersection solve");
  if (timing) cudaEventRecord(c->ev[1], s);
  // a2: union graph, incrementally from the intersection values
  SolveArgs a2 = solve_base(c, wb, wl, t, kn);
  a2.init = kInitSeed;
  a2.source = source;
  a2.base = c->rI;
  a2.val = c->rU;
  a2.ctl = c->ctl + 1;
  if (c->round_trace) {
    a2.trace = c->trace + kTraceCap;
    a2.trace_cap = kTraceCap;
  }
  if (c->prune && (e = launch_solve(t, kPredAny, a2, cfg_for(c, c->occ_solve, kn.bps), s)) != cudaSuccess)
    return cuda_fail(c, e, "launch union solve");
  if (timing) cudaEventRecord(c->ev[2], s);
  return enqueue_tail(c, t, wb, wl, out, c->rI, c->rU, s, timing, ms_relax_out, ms_scatter_out, co, false);
}

// a3-a6 of one query from its bound values rI (intersection graph) and rU
// (union graph): stable compaction and subgraph extraction, then relaxation
// and scatter per slab of at most 128 snapshots.  With `fresh` the phases'
// control blocks are cleared first (a query whose bounds came from a group).
svv_status enqueue_tail(svv_ctx* c, int t, uint32_t wb, uint32_t wl, uint32_t* out, const uint32_t* rI,
                        const uint32_t* rU, cudaStream_t s, bool timing, float* ms_relax_out, float* ms_scatter_out,
                        const CompactOut* co, bool fresh) {
  cudaError_t e = cudaSuccess;
  const Knobs kn = knobs_of(c, t, wl);
  if (fresh && (e = cudaMemsetAsync(c->ctl + 2, 0, sizeof(TeamCtl) * 2, s)) != cudaSuccess)
    return cuda_fail(c, e, "memset");
  c->last_rI = rI;
  c->last_rU = rU;
  c->last_row = c->row;
  // a3+a4: stable compaction and the Q-relevant subgraph
  QrsArgs q{};
  q.g = c->g;
  q.win = Window{wb, wl};
  q.QW = ceil_div(wl, 64);
  q.prune = c->prune ? 1 : 0;
  q.rI = rI;
  q.rU = rU;
  q.row = c->row;
  q.uv = c->uv;
  q.part = c->part;
  q.units = c->units;
  q.ucap = c->ucap;
  q.cshift = c->qrs_cs;
  q.qcnt = c->qcnt;
  q.qrow = c->qrow;
  q.cur = c->cur;
  q.qcw = c->qcw;
  q.qmask = c->qmask;
  q.ecap = c->ecap;
  q.mcap = c->mcap;
  q.rowcap = c->g.V;
  q.ctl = c->ctl + 2;
  q.qerr = c->qerr;
  q.spin_ns = (unsigned long long)c->spin_ms * 1000000ull;
  if (c->round_trace) q.trace = c->trace + 3 * kTraceCap;
  LaunchCfg qc = cfg_for(c, c->occ_qrs, kn.bps);
  if ((int64_t)qc.blocks > (int64_t)c->num_sms * 4) qc.blocks = c->num_sms * 4;
  if ((e = launch_qrs(q, qc, s)) != cudaSuccess) return cuda_fail(c, e, "launch subgraph extraction");
  if (timing) cudaEventRecord(c->ev[3], s);
  float ms_relax = 0.f, ms_scatter = 0.f;
  // a5+a6 per slab of at most 128 snapshots (a window longer than that is
  // relaxed slab by slab over the same subgraph; snapshots are independent)
  const uint32_t slab = std::max<uint32_t>(1, std::min(kn.slab_max, kMaxSlab));
  for (uint32_t s0 = 0; s0 < wl; s0 += slab) {
    const uint32_t ls = std::min(slab, wl - s0);
    uint32_t P, K;
    slab_shape_p(ls, kn.relax_lanes, P, K);
    if (s0 > 0 && (e = cudaMemsetAsync(c->ctl + 3, 0, sizeof(TeamCtl), s)) != cudaSuccess)
      return cuda_fail(c, e, "memset");
    if (timing) cudaEventRecord(c->ev[6], s);
    RelaxArgs r{};
    r.g = c->g;
    r.win = Window{wb, wl};
    r.s0 = s0;
    r.ls = ls;
    r.QW = q.QW;
    r.rI = rI;
    r.row = c->row;
    r.uv = c->uv;
    r.qrow = c->qrow;
    r.qcw = c->qcw;
    r.qmask = c->qmask;
    r.counts = &(c->ctl + 2)->aux[0];
    r.val = c->val;
    r.LP = P * K;
    r.stamp = c->stamp;
    r.q0 = c->q0;
    r.q1 = c->q1;
    r.qcap = c->qcap;
    r.cshift = c->relax_cs;
    r.ctl = c->ctl + 3;
    r.qerr = c->qerr;
    r.maxit = c->maxit ? c->maxit : c->g.V + 2u;
    r.spin_ns = (unsigned long long)c->spin_ms * 1000000ull;
    if (c->round_trace) {
      r.trace = c->trace + 2 * kTraceCap;
      r.trace_cap = kTraceCap;
    }
    if ((e = launch_relax(t, P, K, r, cfg_for(c, c->occ_relax, kn.bps), s)) != cudaSuccess)
      return cuda_fail(c, e, "launch relaxation");
    if (timing) cudaEventRecord(c->ev[4], s);
    if (co) {
      CompactArgs ca{};
      ca.counts = &(c->ctl + 2)->aux[0];
      ca.val = c->val;
      ca.LP = P * K;
      ca.s0 = s0;
      ca.ls = ls;
      ca.wl = wl;
      ca.rows_out = co->rows_out;
      ca.rows_cap = co->rows_cap;
      ca.qerr = c->qerr;
      if ((e = launch_compact(ca, s)) != cudaSuccess) return cuda_fail(c, e, "launch compact copy");
      if (timing) cudaEventRecord(c->ev[5], s);
      continue;
    }
    ScatterArgs sa{};
    sa.V = c->g.V;
    sa.s0 = s0;
    sa.ls = ls;
    sa.rI = rI;
    sa.row = c->row;
    sa.val = c->val;
    sa.LP = P * K;
    sa.out = out;
    sa.qerr = c->qerr;
    if ((e = launch_scatter(sa, s)) != cudaSuccess) return cuda_fail(c, e, "launch scatter");
    if (timing) {
      cudaEventRecord(c->ev[5], s);
      if (wl > slab) {  // several slabs: accumulate per slab
        float a = 0.f, b = 0.f;
        cudaEventSynchronize(c->ev[5]);
        cudaEventElapsedTime(&a, c->ev[6], c->ev[4]);
        cudaEventElapsedTime(&b, c->ev[4], c->ev[5]);
        ms_relax += a;
        ms_scatter += b;
      }
    }
  }
  if (co) {
    const size_t n = (size_t)c->g.V * sizeof(uint32_t);
    if (co->cap_out && (e = cudaMemcpyAsync(co->cap_out, rI, n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return cuda_fail(c, e, "copy intersection values");
    if (co->row_out && (e = cudaMemcpyAsync(co->row_out, c->row, n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return cuda_fail(c, e, "copy row map");
  }
  *ms_relax_out = ms_relax;
  *ms_scatter_out = ms_scatter;
  return SVV_OK;
}

// Graph mode: capture the query's launches, update the instantiated graph in
// place (same topology for the same window shape) or instantiate it, launch it.
svv_status graph_query(svv_ctx* c, int t, uint32_t source, uint32_t wb, uint32_t wl, uint32_t* out,
                       cudaStream_t s, bool* captured) {
  *captured = false;
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return SVV_ECUDA;
  }
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return SVV_ECUDA;
  }
  float a = 0.f, b = 0.f;
  svv_status st = enqueue_query(c, t, source, wb, wl, out, c->cap_stream, false, &a, &b);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (st || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st ? st : SVV_ECUDA;
  }
  bool ok = false;
  if (c->gexec) {
    cudaGraphExecUpdateResultInfo info;
    ok = cudaGraphExecUpdate(c->gexec, g, &info) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
  }
  if (!ok) {
    if (cudaGraphInstantiate(&c->gexec, g, 0) != cudaSuccess) {
      cudaGetLastError();
      c->gexec = nullptr;
      cudaGraphDestroy(g);
      return SVV_ECUDA;
    }
    c->graph_builds++;
  }
  cudaGraphDestroy(g);
  *captured = true;
  if ((e = cudaGraphLaunch(c->gexec, s)) != cudaSuccess) return cuda_fail(c, e, "graph launch");
  c->graph_launches++;
  return SVV_OK;
}

}  // namespace svv

namespace svv {

// In-order batch: the instances run one after another with the per-phase
// kernels on one stream.  Each instance's error word is copied to its own
// device slot, and all are read back once at the end, so nothing waits on the
// host between instances.
// Two device staging slots of L*V words for host outputs (grown on demand).
static svv_status ensure_bstage(svv_ctx* c, uint64_t words) {
  cudaError_t e = cudaSuccess;
  if (!c->copy_stream && (e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(c, e, "copy stream");
  for (int i = 0; i < 2; ++i) {
    if (!c->ev_done[i] && (e = cudaEventCreateWithFlags(&c->ev_done[i], cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(c, e, "cudaEventCreate");
    if (!c->ev_copied[i] && (e = cudaEventCreateWithFlags(&c->ev_copied[i], cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(c, e, "cudaEventCreate");
  }
  if (words <= c->bstage_cap) return SVV_OK;
  cudaStreamSynchronize(c->copy_stream);
  free_list(c, c->bstage_bufs);
  c->allocated -= std::min<uint64_t>(c->allocated, 2 * round256(c->bstage_cap * 4));
  c->bstage[0] = c->bstage[1] = nullptr;
  c->bstage_cap = 0;
  svv_status st;
  if ((st = alloc_n(c, c->bstage_bufs, words, &c->bstage[0])) || (st = alloc_n(c, c->bstage_bufs, words, &c->bstage[1])))
    return st;
  c->bstage_cap = words;
  return SVV_OK;
}

// Groups of at most gmax instances of one type, each in arrival order, the
// groups ordered by their first member.  An instance whose source has no
// out-edge is answered by one fill and gets a group of its own.
std::vector<std::vector<uint32_t>> form_groups(const svv_ctx* c, const BatchInstance* inst, uint32_t m,
                                               uint32_t gmax) {
  std::vector<std::vector<uint32_t>> groups;
  int open[4] = {-1, -1, -1, -1};  // the group still filling, per type
  for (uint32_t k = 0; k < m; ++k) {
    if (source_is_isolated(c, inst[k].source)) {
      groups.push_back({k});
      continue;
    }
    // with group_mix every type shares one group stream
    const int t = c->group_mix ? 0 : std::max(0, std::min(3, inst[k].type));
    if (open[t] < 0 || groups[open[t]].size() >= std::max<uint32_t>(1, gmax)) {
      open[t] = (int)groups.size();
      groups.emplace_back();
    }
    groups[open[t]].push_back(k);
  }
  return groups;
}

svv_status batch_in_order(svv_ctx* c, const BatchInstance* inst, uint32_t m, const char* host_out,
                          uint32_t* qerr_dev, uint32_t* qerr_host, cudaStream_t s, float* ms) {
  uint32_t Lmax = 1, Lhost = 0;
  for (uint32_t k = 0; k < m; ++k) {
    Lmax = std::max(Lmax, inst[k].wl);
    if (host_out && host_out[k]) Lhost = std::max(Lhost, inst[k].wl);
  }
  svv_status st = ensure_window(c, Lmax);
  if (st) return st;
  if (Lhost && (st = ensure_bstage(c, (uint64_t)Lhost * c->g.V))) return st;
  cudaError_t e = cudaSuccess;
  for (auto& ev : c->bev)
    if (!ev && (e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(c, e, "cudaEventCreate");
  cudaEventRecord(c->bev[0], s);
  // Instances run in groups of up to group_max of one type (in order of
  // their first member): one pair of group solves gives every member its
  // bounds, then each member runs its own phases.  A host output is computed
  // into a staging slot and copied back on the copy stream while the next
  // instance computes; a slot is reused only after its last copy has finished.
  const std::vector<std::vector<uint32_t>> groups = form_groups(c, inst, m, c->group_max);
  // graph mode (device outputs): the batch's launches are captured into one
  // CUDA graph, updated in place when the next batch has the same shape, and
  // launched on `s`; allocations happen before the capture
  cudaStream_t es = s;
  bool capture = c->graph_mode && !host_out && !c->round_trace;
  if (capture) {
    for (const auto& grp : groups) {
      if (grp.size() > 1 && (st = ensure_group(c))) return st;
      if (grp.size() == 2 && c->pair_tails && inst[grp[0]].wl == inst[grp[1]].wl && inst[grp[0]].wl <= kMaxSlab) {
        uint32_t P, K;
        slab_shape_p(inst[grp[0]].wl, knobs_of(c, inst[grp[0]].type, inst[grp[0]].wl).relax_lanes, P, K);
        if ((st = ensure_pair_rows(c, P * K))) return st;
      }
    }
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      capture = false;
    } else if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      capture = false;
    } else {
      es = c->cap_stream;
    }
  }
  auto end_capture = [&](svv_status why) -> svv_status {
    cudaGraph_t gr = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->cap_stream, &gr);
    if (why || ec != cudaSuccess || !gr) {
      if (gr) cudaGraphDestroy(gr);
      cudaGetLastError();
      return why ? why : fail(c, SVV_ECUDA, "batch capture failed");
    }
    bool ok = false;
    if (c->bgexec) {
      cudaGraphExecUpdateResultInfo info;
      ok = cudaGraphExecUpdate(c->bgexec, gr, &info) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        cudaGraphExecDestroy(c->bgexec);
        c->bgexec = nullptr;
      }
    }
    if (!ok && cudaGraphInstantiate(&c->bgexec, gr, 0) != cudaSuccess) {
      cudaGetLastError();
      c->bgexec = nullptr;
      cudaGraphDestroy(gr);
      return fail(c, SVV_ECUDA, "batch graph instantiation failed");
    }
    cudaGraphDestroy(gr);
    const cudaError_t el = cudaGraphLaunch(c->bgexec, s);
    if (el != cudaSuccess) return cuda_fail(c, el, "batch graph launch");
    c->graph_launches++;
    return SVV_OK;
  };
  bool used[2] = {false, false};
  uint32_t nh = 0;
  for (const auto& grp : groups) {
    const bool grouped = grp.size() > 1;
    if (grouped) {
      BatchInstance gi[kGroupMax];
      for (size_t j = 0; j < grp.size(); ++j) gi[j] = inst[grp[j]];
      if ((st = enqueue_group_bounds(c, gi[0].type, gi, (uint32_t)grp.size(), es)))
        return capture ? end_capture(st) : st;
      // a pair with device outputs: both tails with one relaxation launch
      if (grp.size() == 2 && !(host_out && (host_out[grp[0]] || host_out[grp[1]]))) {
        uint32_t* po[2] = {inst[grp[0]].out, inst[grp[1]].out};
        const uint32_t* pI[2] = {c->gI[0], c->gI[1]};
        const uint32_t* pU[2] = {c->gU[0], c->gU[1]};
        bool done = false;
        if ((e = cudaMemcpyAsync(c->qerr, c->gerr, sizeof(uint32_t), cudaMemcpyDeviceToDevice, es)) != cudaSuccess)
          st = cuda_fail(c, e, "group status copy");
        else
          st = enqueue_pair_tail(c, gi, po, pI, pU, es, &done);
        if (st) return capture ? end_capture(st) : st;
        if (done) {
          for (int j = 0; j < 2; ++j)
            if ((e = cudaMemcpyAsync(qerr_dev + grp[j], c->qerr, sizeof(uint32_t), cudaMemcpyDeviceToDevice, es)) !=
                cudaSuccess) {
              st = cuda_fail(c, e, "batch status copy");
              return capture ? end_capture(st) : st;
            }
          continue;
        }
      }
    }
    for (size_t j = 0; j < grp.size(); ++j) {
      const uint32_t k = grp[j];
      float a = 0.f, b = 0.f;
      uint32_t* out = inst[k].out;
      int slot = -1;
      if (host_out && host_out[k]) {
        slot = (int)(nh++ & 1u);
        if (used[slot] && (e = cudaStreamWaitEvent(s, c->ev_copied[slot], 0)) != cudaSuccess)
          return cuda_fail(c, e, "staging wait");
        out = c->bstage[slot];
      }
      if (grouped) {
        if ((e = cudaMemcpyAsync(c->qerr, c->gerr, sizeof(uint32_t), cudaMemcpyDeviceToDevice, es)) != cudaSuccess)
          st = cuda_fail(c, e, "group status copy");
        else
          st = enqueue_tail(c, inst[k].type, inst[k].wb, inst[k].wl, out, c->gI[j], c->gU[j], es, false, &a, &b,
                            nullptr, true);
      } else {
        st = enqueue_query(c, inst[k].type, inst[k].source, inst[k].wb, inst[k].wl, out, es, false, &a, &b);
      }
      if (!st && (e = cudaMemcpyAsync(qerr_dev + k, c->qerr, sizeof(uint32_t), cudaMemcpyDeviceToDevice, es)) !=
                     cudaSuccess)
        st = cuda_fail(c, e, "batch status copy");
      if (st) return capture ? end_capture(st) : st;
      if (slot >= 0) {
        const size_t bytes = (size_t)inst[k].wl * c->g.V * sizeof(uint32_t);
        e = cudaEventRecord(c->ev_done[slot], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy_stream, c->ev_done[slot], 0);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(inst[k].out, out, bytes, cudaMemcpyDeviceToHost, c->copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_copied[slot], c->copy_stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "copying a result to the host");
        used[slot] = true;
      }
    }
  }
  if (capture && (st = end_capture(SVV_OK))) return st;
  cudaEventRecord(c->bev[1], s);
  e = cudaMemcpyAsync(qerr_host, qerr_dev, sizeof(uint32_t) * m, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && nh) e = cudaStreamSynchronize(c->copy_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "batch");
  *ms = 0.f;
  cudaEventElapsedTime(ms, c->bev[0], c->bev[1]);
  return SVV_OK;
}

svv_status reserve_window(svv_ctx* c, uint32_t L) { return ensure_window(c, L); }

}  // namespace svv

extern "C" {

svv_status svv_query(svv_ctx* c, svv_type type, uint32_t source, uint32_t wb, uint32_t wl, uint32_t* out,
                     void* stream) {
  svv_status st = check_query(c, (int)type, source, wb, wl, out);
  if (st) return st;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  ServeFence fence(c, s);  // before any scratch is resized
  if ((st = ensure_window(c, wl))) return st;
  const int t = (int)type;
  bool timing = c->phase_timing;
  float ms_relax = 0.f, ms_scatter = 0.f;
  bool done = false;
  if (c->graph_mode && !c->round_trace) {
    bool captured = false;
    st = graph_query(c, t, source, wb, wl, out, s, &captured);
    if (captured && st) return st;
    done = captured;
    if (done) timing = false;
  }
  if (!done && (st = enqueue_query(c, t, source, wb, wl, out, s, timing, &ms_relax, &ms_scatter))) return st;
  st = finish(c, s, 4);
  svv_stats& S = c->stats;
  S = svv_stats{};
  S.unstable = c->hctl[2].aux[0];
  S.qrs_edges = c->hctl[2].aux[2];
  S.qrs_masked = c->hctl[2].aux[3];
  S.iters_cap = c->hctl[0].iters;
  S.iters_cup = c->hctl[1].iters;
  S.iters_relax = c->hctl[3].iters;  // last slab
  S.edges_relaxed_cap = c->hctl[0].relaxed;
  S.edges_relaxed_cup = c->hctl[1].relaxed;
  S.edges_relaxed_multi = c->hctl[3].relaxed;
  if (timing && st == SVV_OK) {
    S.phase_timing = 1;
    cudaEventElapsedTime(&S.ms_cap, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&S.ms_cup, c->ev[1], c->ev[2]);
    cudaEventElapsedTime(&S.ms_qrs, c->ev[2], c->ev[3]);
    if (wl > std::max<uint32_t>(1, std::min(knobs_of(c, t, wl).slab_max, kMaxSlab))) {
      S.ms_relax = ms_relax;
      S.ms_scatter = ms_scatter;
    } else {
      cudaEventElapsedTime(&S.ms_relax, c->ev[3], c->ev[4]);
      cudaEventElapsedTime(&S.ms_scatter, c->ev[4], c->ev[5]);
    }
  }
  return st;
}

svv_status svv_query_async(svv_ctx* c, svv_type type, uint32_t source, uint32_t wb, uint32_t wl, uint32_t* out,
                           void* stream, uint64_t* ticket) {
  svv_status st = check_query(c, (int)type, source, wb, wl, out);
  if (st) return st;
  if (!ticket) return fail(c, SVV_EINVAL, "ticket is NULL");
  DeviceGuard dg(c->device);
  cudaError_t e = cudaSuccess;
  if (!c->astatus) {
    if ((e = cudaMallocHost((void**)&c->astatus, sizeof(uint32_t) * kAsyncSlots)) != cudaSuccess) {
      c->astatus = nullptr;
      return cuda_fail(c, e, "status ring");
    }
    for (auto& ev : c->aev)
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(c, e, "cudaEventCreate");
  }
  const uint32_t slot = (uint32_t)(c->anext % kAsyncSlots);
  // the ring holds kAsyncSlots queries: the oldest must be done before its
  // slot is reused
  if (c->anext >= (uint64_t)kAsyncSlots && (e = cudaEventSynchronize(c->aev[slot])) != cudaSuccess)
    return cuda_fail(c, e, "waiting for the oldest query");
  cudaStream_t s = (cudaStream_t)stream;
  ServeFence fence(c, s);  // after the queries queued before, before any scratch is resized
  if ((st = ensure_window(c, wl))) return st;
  float a = 0.f, b = 0.f;
  if ((st = enqueue_query(c, (int)type, source, wb, wl, out, s, false, &a, &b))) return st;
  if ((e = cudaMemcpyAsync(c->astatus + slot, c->qerr, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaEventRecord(c->aev[slot], s)) != cudaSuccess)
    return cuda_fail(c, e, "queueing the query's status");
  c->async_last = c->aev[slot];
  *ticket = c->anext++;
  c->err.clear();
  return SVV_OK;
}

svv_status svv_query_wait(svv_ctx* c, uint64_t ticket, int wait) {
  if (!c) return SVV_EINVAL;
  if (ticket >= c->anext) return fail(c, SVV_EINVAL, "unknown ticket");
  if (c->anext - ticket > (uint64_t)kAsyncSlots)
    return fail(c, SVV_EINVAL, "ticket expired: more than 64 queries were queued after it");
  DeviceGuard dg(c->device);
  const uint32_t slot = (uint32_t)(ticket % kAsyncSlots);
  cudaError_t e = wait ? cudaEventSynchronize(c->aev[slot]) : cudaEventQuery(c->aev[slot]);
  if (e == cudaErrorNotReady) {
    cudaGetLastError();
    return SVV_EBUSY;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "query");
  const uint32_t q = reinterpret_cast<volatile uint32_t*>(c->astatus)[slot];
  if (q == kErrTimeout) return fail(c, SVV_ETIMEOUT, "a device wait or the round cap expired");
  if (q != 0) return fail(c, SVV_EINTERNAL, "device capacity check failed");
  return SVV_OK;
}

svv_status svv_query_compact(svv_ctx* c, svv_type type, uint32_t source, uint32_t wb, uint32_t wl,
                             uint32_t* cap_out, uint32_t* row_out, uint32_t* rows_out, uint64_t rows_cap,
                             uint32_t* unstable_out, void* stream) {
  svv_status st = check_query(c, (int)type, source, wb, wl, rows_out);
  if (st) return st;
  if (!cap_out || !row_out) return fail(c, SVV_EINVAL, "cap_out and row_out are required");
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  ServeFence fence(c, s);  // before any scratch is resized
  if ((st = ensure_window(c, wl))) return st;
  const CompactOut co{cap_out, row_out, rows_out, rows_cap};
  float a = 0.f, b = 0.f;
  if ((st = enqueue_query(c, (int)type, source, wb, wl, nullptr, s, false, &a, &b, &co))) return st;
  st = finish(c, s, 4);
  c->stats = svv_stats{};
  c->stats.unstable = c->hctl[2].aux[0];
  c->stats.qrs_edges = c->hctl[2].aux[2];
  c->stats.qrs_masked = c->hctl[2].aux[3];
  if (unstable_out) *unstable_out = c->hctl[2].aux[0];
  return st;
}

svv_status svv_query_plain(svv_ctx* c, svv_type type, uint32_t source, uint32_t wb, uint32_t wl,
                           uint32_t* out, void* stream) {
  svv_status st = check_query(c, (int)type, source, wb, wl, out);
  if (st) return st;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  ServeFence fence(c, s);
  const uint32_t nslot = std::min<uint32_t>(wl, kNumCtl - 8);
  cudaError_t e = cudaMemsetAsync(c->ctl + 8, 0, sizeof(TeamCtl) * nslot, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->qerr, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  const bool timing = c->phase_timing;
  if (timing) cudaEventRecord(c->ev[0], s);
  for (uint32_t i = 0; i < wl; ++i) {
    TeamCtl* slot = c->ctl + 8 + (i % (kNumCtl - 8));
    if (i >= (uint32_t)(kNumCtl - 8) && (e = cudaMemsetAsync(slot, 0, sizeof(TeamCtl), s)) != cudaSuccess)
      return cuda_fail(c, e, "memset");
    SolveArgs a = solve_base(c, wb, wl, (int)type, knobs_of(c, (int)type, wl));
    a.init = kInitSource;
    a.source = source;
    a.bit = wb + i;
    a.val = out + (size_t)i * c->g.V;
    a.ctl = slot;
    if ((e = launch_solve((int)type, kPredBit, a, cfg_for(c, c->occ_solve, knobs_of(c, (int)type, wl).bps), s)) !=
        cudaSuccess)
      return cuda_fail(c, e, "launch per-snapshot solve");
  }
  if (timing) cudaEventRecord(c->ev[1], s);
  st = finish(c, s, 8 + nslot);
  svv_stats& S = c->stats;
  S = svv_stats{};
  if (timing && st == SVV_OK) {
    S.phase_timing = 1;
    cudaEventElapsedTime(&S.ms_cap, c->ev[0], c->ev[1]);
  }
  for (uint32_t i = 0; i < nslot; ++i) {
    S.iters_plain_max = std::max(S.iters_plain_max, c->hctl[8 + i].iters);
    S.edges_relaxed_cap += c->hctl[8 + i].relaxed;
  }
  return st;
}

svv_status svv_get_bounds(svv_ctx* c, uint32_t* cap, uint32_t* cup, uint32_t* row, void* stream) {
  if (!c) return SVV_EINVAL;
  if (!c->loaded) return fail(c, SVV_ENOTLOADED, "no graph loaded");
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  ServeFence fence(c, s);
  const size_t n = (size_t)c->g.V * sizeof(uint32_t);
  cudaError_t e = cudaSuccess;
  const uint32_t* rI = c->last_rI ? c->last_rI : c->rI;
  const uint32_t* rU = c->last_rU ? c->last_rU : c->rU;
  if (cap) e = cudaMemcpyAsync(cap, rI, n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && cup) e = cudaMemcpyAsync(cup, rU, n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && row)
    e = cudaMemcpyAsync(row, c->last_row ? c->last_row : c->row, n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "copying bounds");
  return SVV_OK;
}

svv_status svv_get_round_trace(svv_ctx* c, uint32_t phase, uint64_t* out, uint32_t cap, uint32_t* n_out) {
  if (!c || !out || !n_out || phase > 3) return SVV_EINVAL;
  *n_out = 0;
  if (!c->trace) return fail(c, SVV_EINVAL, "round_trace was never enabled");
  DeviceGuard dg(c->device);
  const uint32_t n = std::min(cap, kTraceCap);
  cudaError_t e = cudaMemcpy(out, c->trace + phase * kTraceCap, n * sizeof(uint64_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "copying the round trace");
  *n_out = n;
  return SVV_OK;
}

svv_status svv_query_host(svv_ctx* c, svv_type type, uint32_t source, uint32_t wb, uint32_t wl,
                          uint32_t* out_host, void* stream) {
  svv_status st = check_query(c, (int)type, source, wb, wl, out_host);
  if (st) return st;
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  // page-locked and mapped: the scatter writes the host buffer directly
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, out_host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
      at.devicePointer != nullptr && at.device == c->device) {
    if ((st = svv_query(c, type, source, wb, wl, static_cast<uint32_t*>(at.devicePointer), stream))) return st;
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "query into host memory");
    return SVV_OK;
  }
  cudaGetLastError();  // not a registered pointer
  const uint64_t need = (uint64_t)wl * c->g.V;
  if (need > c->staging_cap) {
    if (c->staging) {
      auto it = std::find(c->scratch_bufs.begin(), c->scratch_bufs.end(), (void*)c->staging);
      if (it != c->scratch_bufs.end()) c->scratch_bufs.erase(it);
      cudaFree(c->staging);
      c->allocated -= ((c->staging_cap * 4 + 255) & ~uint64_t(255));
      c->staging = nullptr;
      c->staging_cap = 0;
    }
    if ((st = alloc_n(c, c->scratch_bufs, need, &c->staging))) return st;
    c->staging_cap = need;
  }
  st = svv_query(c, type, source, wb, wl, c->staging, stream);
  if (st) return st;
  cudaError_t e = cudaMemcpyAsync(out_host, c->staging, need * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "copying the result to the host");
  return SVV_OK;
}

}  // extern "C"
