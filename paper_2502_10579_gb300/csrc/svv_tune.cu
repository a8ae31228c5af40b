// svv_tune.cu -- the autotuner: picks the launch knobs of one query type and
// window-length bucket by timing a probe query of that type.
//
// Coordinate descent from the current defaults: for each knob in turn --
// the pull threshold of the solves' direction switch, the near-far width
// (SSSP, SSWP), edges per work unit, CTAs per SM, lanes per edge and chunk
// skipping of the relaxation and solves, the relaxation's slab width -- every
// candidate value is timed with the others fixed at the best found so far,
// and kept if it is faster by more than 2%.  Every candidate gives the same
// values: only the schedule changes.
#include <cfloat>
#include <vector>

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
  const int b = len_bucket(win_len);
  const bool had = c->has_tuned[t][b];
  const Knobs saved = c->tuned[t][b];
  Knobs cur = default_knobs(c, t);
  float best_ms = FLT_MAX, base_ms = FLT_MAX;
  uint32_t tried = 0;
  svv_status st = SVV_OK;
  auto time_one = [&](const Knobs& k, float* ms) -> svv_status {
    c->tuned[t][b] = k;
    c->has_tuned[t][b] = true;
    float sum = 0.f;
    for (uint32_t r = 0; r <= reps; ++r) {  // the first run warms up
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
    ++tried;
    return SVV_OK;
  };
  // one knob at a time: candidate values, and the field they set
  auto try_dim = [&](const std::vector<uint32_t>& vals, void (*set)(Knobs&, uint32_t)) -> svv_status {
    for (uint32_t v : vals) {
      Knobs k = cur;
      set(k, v);
      if (k.solve_cs == cur.solve_cs && k.bps == cur.bps && k.relax_lanes == cur.relax_lanes &&
          k.skip_same == cur.skip_same && k.pull_pct == cur.pull_pct && k.delta == cur.delta &&
          k.slab_max == cur.slab_max)
        continue;  // the current value
      float ms = 0.f;
      svv_status q = time_one(k, &ms);
      if (q) return q;
      if (ms < 0.98f * best_ms) {
        best_ms = ms;
        cur = k;
      }
    }
    return SVV_OK;
  };
  const uint32_t cs0 = std::max<uint32_t>(c->solve_cs, 5u);
  if ((st = time_one(cur, &base_ms))) goto done;
  best_ms = base_ms;
  if (c->g.ifd && (st = try_dim({0u, 5u, 10u, 15u, 25u, 40u}, [](Knobs& k, uint32_t v) { k.pull_pct = v; }))) goto done;
  if (t == 0 && (st = try_dim({0u, 250u, 1000u, 4000u}, [](Knobs& k, uint32_t v) { k.delta = v; }))) goto done;
  if (t == 1 && (st = try_dim({0u, 50u, 200u, 800u}, [](Knobs& k, uint32_t v) { k.delta = v; }))) goto done;
  if ((st = try_dim({cs0, cs0 + 1u}, [](Knobs& k, uint32_t v) { k.solve_cs = v; }))) goto done;
  if ((st = try_dim({0u, 2u, 3u}, [](Knobs& k, uint32_t v) { k.bps = (int)v; }))) goto done;
  if ((st = try_dim({32u, 16u}, [](Knobs& k, uint32_t v) { k.relax_lanes = v; }))) goto done;
  if ((st = try_dim({1u, 0u}, [](Knobs& k, uint32_t v) { k.skip_same = v != 0; }))) goto done;
  if (win_len > 32 && (st = try_dim({kMaxSlab, 64u, 32u}, [](Knobs& k, uint32_t v) { k.slab_max = v; }))) goto done;
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) {
    c->tuned[t][b] = saved;
    c->has_tuned[t][b] = had;
    return st;
  }
  c->tuned[t][b] = cur;
  c->has_tuned[t][b] = true;
  if (out) {
    out->solve_chunk = 1u << cur.solve_cs;
    out->blocks_per_sm = (uint32_t)cur.bps;
    out->relax_lanes = cur.relax_lanes;
    out->skip_same = cur.skip_same ? 1u : 0u;
    out->pull_pct = cur.pull_pct;
    out->delta = cur.delta;
    out->slab_max = cur.slab_max;
    out->best_ms = best_ms;
    out->default_ms = base_ms;
    out->candidates = tried;
  }
  c->err.clear();
  return SVV_OK;
}
