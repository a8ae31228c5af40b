// svv_tune.cu -- the autotuner: picks the launch knobs of one query type by
// timing candidate configurations on a probe query of that type.
#include <cfloat>

#include "svv_ctx.h"

using namespace svv;

extern "C" svv_status svv_autotune(svv_ctx* c, svv_type type, uint32_t source, uint32_t win_begin,
                                   uint32_t win_len, uint32_t reps, svv_tune_result* out) {
  if (!c) return SVV_EINVAL;
  if (!c->loaded) return fail(c, SVV_ENOTLOADED, "no graph loaded");
  if ((int)type < 0 || (int)type > 3) return fail(c, SVV_EINVAL, "unknown query type");
  if (source >= c->g.V || win_len == 0 || (uint64_t)win_begin + win_len > c->g.S)
    return fail(c, SVV_EINVAL, "bad probe query");
  if (reps == 0) reps = 3;
  DeviceGuard dg(c->device);
  // probe output: the host-query staging buffer
  const uint64_t need = (uint64_t)win_len * c->g.V;
  if (need > c->staging_cap) {
    if (c->staging) {
      auto it = std::find(c->scratch_bufs.begin(), c->scratch_bufs.end(), (void*)c->staging);
      if (it != c->scratch_bufs.end()) c->scratch_bufs.erase(it);
      cudaFree(c->staging);
      c->allocated -= round256(c->staging_cap * 4);
      c->staging = nullptr;
      c->staging_cap = 0;
    }
    svv_status st = alloc_n(c, c->scratch_bufs, need, &c->staging);
    if (st) return st;
    c->staging_cap = need;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cuda_fail(c, cudaGetLastError(), "autotune events");
  const int t = (int)type;
  const bool had = c->has_tuned[t];
  const Knobs saved = c->tuned[t];
  const Knobs base{c->solve_cs, c->bps, c->relax_lanes, c->skip_same};
  // candidate grid; the chunk never goes below the one the queues were sized for
  const uint32_t cs_opts[2] = {std::max<uint32_t>(c->solve_cs, 5u), std::max<uint32_t>(c->solve_cs, 5u) + 1u};
  const int bps_opts[3] = {0, 2, 3};
  const uint32_t lane_opts[2] = {32u, 16u};
  const bool skip_opts[2] = {true, false};
  Knobs best = base;
  float best_ms = FLT_MAX, base_ms = FLT_MAX;
  uint32_t tried = 0;
  svv_status st = SVV_OK;
  auto time_one = [&](const Knobs& k, float* ms) -> svv_status {
    c->tuned[t] = k;
    c->has_tuned[t] = true;
    float sum = 0.f;
    for (uint32_t r = 0; r <= reps; ++r) {  // first run warms up
      cudaEventRecord(e0, 0);
      svv_status q = svv_query(c, type, source, win_begin, win_len, c->staging, nullptr);
      cudaEventRecord(e1, 0);
      if (q) return q;
      cudaEventSynchronize(e1);
      float m = 0.f;
      cudaEventElapsedTime(&m, e0, e1);
      if (r) sum += m;
    }
    *ms = sum / reps;
    return SVV_OK;
  };
  if ((st = time_one(base, &base_ms))) goto done;
  best_ms = base_ms;
  for (uint32_t cs : cs_opts)
    for (int bps : bps_opts)
      for (uint32_t lanes : lane_opts)
        for (bool skip : skip_opts) {
          const Knobs k{cs, bps, lanes, skip};
          float ms = 0.f;
          if ((st = time_one(k, &ms))) goto done;
          ++tried;
          if (ms < best_ms) {
            best_ms = ms;
            best = k;
          }
        }
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) {
    c->tuned[t] = saved;
    c->has_tuned[t] = had;
    return st;
  }
  c->tuned[t] = best;
  c->has_tuned[t] = true;
  if (out) {
    out->solve_chunk = 1u << best.solve_cs;
    out->blocks_per_sm = (uint32_t)best.bps;
    out->relax_lanes = best.relax_lanes;
    out->skip_same = best.skip_same ? 1u : 0u;
    out->best_ms = best_ms;
    out->default_ms = base_ms;
    out->candidates = tried + 1;
  }
  c->err.clear();
  return SVV_OK;
}
