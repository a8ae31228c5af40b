// svv_device.cuh -- device helpers: coherent loads, the bounded team barrier,
// warp scans, the three edge functions and the window predicates.
#pragma once

#include <cstdint>
#include "svv_internal.h"

namespace svv {

constexpr unsigned kFullMask = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Loads of data that other CTAs of the same launch write (values, queues,
// counters) bypass L1 so a CTA never reads a stale line.
__device__ __forceinline__ uint32_t ld_cg(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long ld_cg(const unsigned long long* p) { return __ldcg(p); }

// Plain (L1-cacheable) load of a value another CTA may write in the same
// round.  Values only improve, so a stale read can only give a worse
// candidate, and the writer's change puts its vertex in the next frontier;
// across rounds the team barrier's acquire orders these loads after every
// write of the earlier rounds.
__device__ __forceinline__ uint32_t ld_val(const uint32_t* p) { return *p; }

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void set_err(TeamCtl* c, uint32_t* qerr, uint32_t code) {
  atomicCAS(&c->err, 0u, code);
  if (qerr) atomicCAS(qerr, 0u, code);
}

// ---------------------------------------------------------------------------
// Team barrier over `nblocks` co-resident CTAs (cooperative launch), with a
// bounded wait: a CTA that waits longer than `spin_ns`, or sees an error flag
// raised by another CTA, records the error and returns false; every caller
// then leaves the kernel.  Sense is a generation counter.
__device__ __forceinline__ bool team_sync(TeamCtl* c, uint32_t* qerr, unsigned nblocks,
                                          unsigned long long spin_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned gen = ld_acquire(&c->bar_gen);
    __threadfence();
    unsigned arrived = atomicAdd(&c->bar_count, 1u) + 1u;
    if (arrived == nblocks) {
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      unsigned long long t0 = global_ns();
      unsigned ns = 32;
      while (ld_acquire(&c->bar_gen) == gen) {
        if (ld_acquire(&c->err) != 0u || (qerr && ld_acquire(qerr) != 0u)) {
          ok = 0;
          break;
        }
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        if (global_ns() - t0 > spin_ns) {
          set_err(c, qerr, kErrTimeout);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (ok && (ld_acquire(&c->err) != 0u || (qerr && ld_acquire(qerr) != 0u))) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// One acquire load per CTA, broadcast through shared memory: a per-round
// counter read by every thread would send one uncached request per thread to
// the same L2 line.
__device__ __forceinline__ void cta_read2(const unsigned* p, const unsigned* q, uint32_t& x, uint32_t& y) {
  __shared__ uint32_t s_v[2];
  if (threadIdx.x == 0) {
    s_v[0] = ld_acquire(p);
    s_v[1] = q ? ld_acquire(q) : 0u;
  }
  __syncthreads();
  x = s_v[0];
  y = s_v[1];
  __syncthreads();
}

__device__ __forceinline__ uint32_t cta_read(const unsigned* p) {
  uint32_t x, y;
  cta_read2(p, nullptr, x, y);
  return x;
}

// Work distribution over n units, `tk` units per batch: a warp's first batch
// is static (batch gwarp), later ones come from `ticket`; no atomic at all when
// the static batches cover the round.
struct Batches {
  uint32_t n, tk, nwarps, gwarp;
  unsigned* ticket;
  __device__ __forceinline__ uint32_t first() const { return gwarp * tk; }
  __device__ __forceinline__ uint32_t next(unsigned lane) const {
    const unsigned long long stat = (unsigned long long)nwarps * tk;
    if (stat >= n) return n;
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(ticket, tk);
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    const unsigned long long r = stat + t;
    return r >= n ? n : (uint32_t)r;
  }
};

__device__ __forceinline__ uint32_t batch_size(uint32_t n, uint32_t nwarps, uint32_t cap) {
  const uint32_t t = (n + nwarps - 1) / nwarps;
  return t < 1u ? 1u : (t > cap ? cap : t);
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, unsigned lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(kFullMask, x, d);
    if (lane >= (unsigned)d) x += y;
  }
  return x;
}

// first lane k with incl[k] > p (incl non-decreasing across the warp, p <
// incl[31]); every lane takes part
__device__ __forceinline__ int warp_owner(uint32_t incl, uint32_t p) {
  int k = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    uint32_t v = __shfl_sync(kFullMask, incl, k + step - 1);
    if (v <= p) k += step;
  }
  return k;
}

// ---------------------------------------------------------------------------
// Edge functions, Table 2.
struct OpSSSP {  // CASMIN(Val(v), Val(u) + w), saturating
  static constexpr bool kLevels = false;
  static constexpr uint32_t kIdentity = kInf;
  static constexpr uint32_t kSource = 0;
  __device__ __forceinline__ static uint32_t relax(uint32_t sv, uint32_t w) {
    if (sv == kInf) return kInf;
    unsigned long long s = (unsigned long long)sv + w;
    return s > kSat ? kSat : (uint32_t)s;
  }
  __device__ __forceinline__ static bool better(uint32_t a, uint32_t b) { return a < b; }
  __device__ __forceinline__ static uint32_t atomic(uint32_t* p, uint32_t v) { return atomicMin(p, v); }
};

struct OpSSWP {  // CASMAX(Val(v), min(Val(u), w))
  static constexpr bool kLevels = false;
  static constexpr uint32_t kIdentity = 0;
  static constexpr uint32_t kSource = kInf;
  __device__ __forceinline__ static uint32_t relax(uint32_t sv, uint32_t w) { return sv < w ? sv : w; }
  __device__ __forceinline__ static bool better(uint32_t a, uint32_t b) { return a > b; }
  __device__ __forceinline__ static uint32_t atomic(uint32_t* p, uint32_t v) { return atomicMax(p, v); }
};

struct OpBFS {  // CASMIN(Val(v), Val(u) + 1)
  static constexpr bool kLevels = true;  // a round from the source sets exactly one level
  static constexpr uint32_t kIdentity = kInf;
  static constexpr uint32_t kSource = 0;
  __device__ __forceinline__ static uint32_t relax(uint32_t sv, uint32_t) { return sv == kInf ? kInf : sv + 1; }
  __device__ __forceinline__ static bool better(uint32_t a, uint32_t b) { return a < b; }
  __device__ __forceinline__ static uint32_t atomic(uint32_t* p, uint32_t v) { return atomicMin(p, v); }
};

struct OpSSNP {  // CASMIN(Val(v), max(Val(u), w))
  static constexpr bool kLevels = false;
  static constexpr uint32_t kIdentity = kInf;
  static constexpr uint32_t kSource = 0;
  __device__ __forceinline__ static uint32_t relax(uint32_t sv, uint32_t w) {
    return sv == kInf ? kInf : (sv > w ? sv : w);
  }
  __device__ __forceinline__ static bool better(uint32_t a, uint32_t b) { return a < b; }
  __device__ __forceinline__ static uint32_t atomic(uint32_t* p, uint32_t v) { return atomicMin(p, v); }
};

// ---------------------------------------------------------------------------
// Window predicates on a W-word presence mask (bit i = snapshot i).
__device__ __forceinline__ uint64_t window_word(Window w, uint32_t j) {
  uint32_t lo = max(w.b, j * 64u), hi = min(w.b + w.l, j * 64u + 64u);
  if (lo >= hi) return 0ull;
  uint32_t n = hi - lo;
  uint64_t m = (n == 64u) ? ~0ull : ((1ull << n) - 1ull);
  return m << (lo - j * 64u);
}

// bits [0,S) in word j
__device__ __forceinline__ uint64_t history_word(uint32_t S, uint32_t j) {
  return window_word(Window{0u, S}, j);
}

__device__ __forceinline__ bool window_all(const uint64_t* m, Window w) {
  uint32_t j0 = w.b >> 6, j1 = (w.b + w.l - 1) >> 6;
  for (uint32_t j = j0; j <= j1; ++j) {
    uint64_t wm = window_word(w, j);
    if ((__ldg(m + j) & wm) != wm) return false;
  }
  return true;
}

__device__ __forceinline__ bool window_any(const uint64_t* m, Window w) {
  uint32_t j0 = w.b >> 6, j1 = (w.b + w.l - 1) >> 6;
  for (uint32_t j = j0; j <= j1; ++j)
    if (__ldg(m + j) & window_word(w, j)) return true;
  return false;
}

// (any, all) in one pass
__device__ __forceinline__ void window_any_all(const uint64_t* m, Window w, bool& any, bool& all) {
  uint32_t j0 = w.b >> 6, j1 = (w.b + w.l - 1) >> 6;
  any = false;
  all = true;
  for (uint32_t j = j0; j <= j1; ++j) {
    uint64_t wm = window_word(w, j), x = __ldg(m + j) & wm;
    any |= (x != 0ull);
    all &= (x == wm);
  }
}

__device__ __forceinline__ bool mask_bit(const uint64_t* m, uint32_t i) {
  return (__ldg(m + (i >> 6)) >> (i & 63u)) & 1ull;
}

// bits [start, start+64) of a W-word mask, as one word (bits past the mask are 0)
__device__ __forceinline__ uint64_t mask_extract(const uint64_t* m, uint32_t W, uint32_t start) {
  uint32_t j = start >> 6, sh = start & 63u;
  uint64_t lo = j < W ? __ldg(m + j) : 0ull;
  if (sh == 0) return lo;
  uint64_t hi = (j + 1) < W ? __ldg(m + j + 1) : 0ull;
  return (lo >> sh) | (hi << (64u - sh));
}

}  // namespace svv
