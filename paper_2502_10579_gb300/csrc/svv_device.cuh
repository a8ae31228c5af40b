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

// Improvement tests.  A lane whose candidate beats the value it loaded
// updates with a reduction (no return) and counts the target as changed: if
// the reduction did not lower the value, another lane lowered it in the same
// round, so the target changed in this round either way.
//
// Plain (L1-cacheable) load of a value another CTA may write in the same
// round.  Values only improve, so a stale read can only give a worse
// candidate, and the writer's change puts its vertex in the next frontier;
// across rounds the team barrier's acquire orders these loads after every
// write of the earlier rounds.
__device__ __forceinline__ uint32_t ld_val(const uint32_t* p) { return *p; }

// Read-only loads of data streamed once per pass (the edge arrays of a pull
// round): no L1 allocation, so the pass leaves L1 to the value gathers.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ uint2 ld_stream(const uint2* p) {
  uint2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}

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

__device__ __forceinline__ unsigned long long atom_add_acq_rel(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Relaxed polls: an acquire load on every spin would also drop the SM's L1
// lines that co-resident CTAs are still reading; one acquire fence after the
// poll that sees the release gives the same ordering.
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" : : "l"(p), "l"(v) : "memory");
}

constexpr unsigned long long kGenErr = 1ull << 63;

// ---------------------------------------------------------------------------
// Team barrier over `nblocks` co-resident CTAs (cooperative launch), with a
// bounded wait.  Arrivals are counted for the whole launch and never reset:
// arrival number a belongs to barrier k = ceil(a / nblocks), and the CTA that
// makes the count k * nblocks publishes k in `bar_gen` with a release store.
// That last arriver also reads the team's error word (its acquire-release
// add orders the read after every arrival, and so after every error set
// before one) and publishes it in the same store, so every CTA learns of an
// error from the one word it polls and they all leave together.  A CTA that
// waits longer than `spin_ns`, or sees the error word set while waiting (a
// CTA that timed out leaves without arriving), records the error and returns
// false; every caller then leaves the kernel.
__device__ __forceinline__ bool team_sync(TeamCtl* c, uint32_t* qerr, unsigned nblocks,
                                          unsigned long long spin_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t* ef = qerr ? qerr : &c->err;
    const unsigned long long a = atom_add_acq_rel(&c->bar_count, 1ull) + 1ull;
    const unsigned long long k = (a + nblocks - 1ull) / nblocks;
    int ok = 1;
    if (a == k * nblocks) {
      const unsigned long long flag = ld_acquire(ef) != 0u ? kGenErr : 0ull;
      st_release(&c->bar_gen, k | flag);
      ok = flag == 0ull;
    } else {
      const unsigned long long t0 = global_ns();
      unsigned polls = 0;
      for (;;) {
        const unsigned long long g = ld_relaxed(&c->bar_gen);
        if ((g & ~kGenErr) >= k) {
          fence_acq_rel();
          ok = (g & kGenErr) == 0ull;
          break;
        }
        if ((++polls & 15u) == 0u) {
          if (ld_relaxed(ef) != 0u) {
            ok = 0;
            break;
          }
          if (global_ns() - t0 > spin_ns) {
            set_err(c, qerr, kErrTimeout);
            ok = 0;
            break;
          }
        }
        if (polls > 64u) __nanosleep(64);
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// One load per CTA, broadcast through shared memory: a per-round counter read
// by every thread would send one uncached request per thread to the same L2
// line.  The counters are read after a team barrier (or at kernel start), whose
// acquire already orders them, so the load is relaxed.
__device__ __forceinline__ void cta_read2(const unsigned* p, const unsigned* q, uint32_t& x, uint32_t& y) {
  __shared__ uint32_t s_v[2];
  if (threadIdx.x == 0) {
    s_v[0] = ld_relaxed(p);
    s_v[1] = q ? ld_relaxed(q) : 0u;
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
  __device__ __forceinline__ static void red(uint32_t* p, uint32_t v) { atomicMin(p, v); }  // no return: a reduction
};

struct OpSSWP {  // CASMAX(Val(v), min(Val(u), w))
  static constexpr bool kLevels = false;
  static constexpr uint32_t kIdentity = 0;
  static constexpr uint32_t kSource = kInf;
  __device__ __forceinline__ static uint32_t relax(uint32_t sv, uint32_t w) { return sv < w ? sv : w; }
  __device__ __forceinline__ static bool better(uint32_t a, uint32_t b) { return a > b; }
  __device__ __forceinline__ static uint32_t atomic(uint32_t* p, uint32_t v) { return atomicMax(p, v); }
  __device__ __forceinline__ static void red(uint32_t* p, uint32_t v) { atomicMax(p, v); }  // no return: a reduction
};

struct OpBFS {  // CASMIN(Val(v), Val(u) + 1)
  static constexpr bool kLevels = true;  // a round from the source sets exactly one level
  static constexpr uint32_t kIdentity = kInf;
  static constexpr uint32_t kSource = 0;
  __device__ __forceinline__ static uint32_t relax(uint32_t sv, uint32_t) { return sv == kInf ? kInf : sv + 1; }
  __device__ __forceinline__ static bool better(uint32_t a, uint32_t b) { return a < b; }
  __device__ __forceinline__ static uint32_t atomic(uint32_t* p, uint32_t v) { return atomicMin(p, v); }
  __device__ __forceinline__ static void red(uint32_t* p, uint32_t v) { atomicMin(p, v); }  // no return: a reduction
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
  __device__ __forceinline__ static void red(uint32_t* p, uint32_t v) { atomicMin(p, v); }  // no return: a reduction
};

// A query group may mix types.  Every type's values then live in the min
// lattice (identity kInf, source 0): SSSP, BFS and SSNP already do, and SSWP's
// widths are kept as complements, since the widest path (max over paths of
// the min weight) is the complement of the min over paths of the max
// complemented weight.  Each lane relaxes with its own kind (kKind*).

struct OpMixed {
  static constexpr bool kLevels = false;
  static constexpr uint32_t kIdentity = kInf;
  static constexpr uint32_t kSource = 0;
  __device__ __forceinline__ static uint32_t relax_kind(uint32_t kind, uint32_t sv, uint32_t w) {
    if (sv == kInf) return kInf;
    if (kind == kKindSum) {
      const unsigned long long s = (unsigned long long)sv + w;
      return s > kSat ? kSat : (uint32_t)s;
    }
    if (kind == kKindHop) return sv + 1u;
    const uint32_t x = kind == kKindMax ? w : ~w;
    return sv > x ? sv : x;
  }
  __device__ __forceinline__ static bool better(uint32_t a, uint32_t b) { return a < b; }
  __device__ __forceinline__ static void red(uint32_t* p, uint32_t v) { atomicMin(p, v); }
};

template <class Op>
struct is_mixed {
  static constexpr bool value = false;
};
template <>
struct is_mixed<OpMixed> {
  static constexpr bool value = true;
};

// lane k's relaxation: the op's own, or lane k's kind (2 bits of `kinds`)
template <class Op>
__device__ __forceinline__ uint32_t lane_relax(uint32_t kinds, int k, uint32_t sv, uint32_t w) {
  if constexpr (is_mixed<Op>::value) return OpMixed::relax_kind((kinds >> (2 * k)) & 3u, sv, w);
  else return Op::relax(sv, w);
}

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
