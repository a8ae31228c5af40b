// svv_push.cuh -- warp-cooperative frontier append.
#pragma once

#include "svv_device.cuh"

namespace svv {

// Every lane with `push` set appends the work units of vertex (or row) `x`:
// ceil(deg / 2^cshift) units "x | chunk << 32", none when deg == 0.  The warp
// reserves space with one atomic and writes the units cooperatively, so a hub
// with thousands of units costs its warp a few stores per lane, not one lane
// thousands.  All 32 lanes must call this.
__device__ __forceinline__ void warp_push_units(bool push, uint32_t x, uint32_t deg, uint32_t cshift,
                                                unsigned long long* q, unsigned* qn, uint32_t qcap,
                                                TeamCtl* c, uint32_t* qerr, unsigned lane) {
  if (__ballot_sync(kFullMask, push) == 0u) return;
  uint32_t nu = push ? ((deg + (1u << cshift) - 1u) >> cshift) : 0u;
  uint32_t incl = warp_incl_scan(nu, lane);
  uint32_t tot = __shfl_sync(kFullMask, incl, 31);
  if (tot == 0u) return;
  uint32_t base = 0;
  if (lane == 31) base = atomicAdd(qn, tot);
  base = __shfl_sync(kFullMask, base, 31);
  if ((unsigned long long)base + tot > qcap) {
    if (lane == 0) set_err(c, qerr, kErrInternal);
    return;
  }
  for (uint32_t j0 = 0; j0 < tot; j0 += 32u) {
    uint32_t j = j0 + lane;
    int k = warp_owner(incl, j < tot ? j : tot - 1u);
    uint32_t xk = __shfl_sync(kFullMask, x, k);
    uint32_t ik = __shfl_sync(kFullMask, incl, k);
    uint32_t nk = __shfl_sync(kFullMask, nu, k);
    if (j < tot) q[base + j] = (unsigned long long)xk | ((unsigned long long)(j - (ik - nk)) << 32);
  }
}

// ---------------------------------------------------------------------------
// Staged append.  Every warp appends into a private buffer of kStageUnits
// units in shared memory and copies it to the queue with one atomic when it
// fills; at the end of a round the CTA copies all leftovers with one atomic.
// One counter serves every warp of the grid, and same-address atomics
// serialise in L2, so an atomic per push would cap a round's throughput.
constexpr uint32_t kStageUnits = 64;

struct PushStage {
  unsigned long long* buf;  // this warp's slots in shared memory
  uint32_t fill;            // warp-uniform
};

__device__ __forceinline__ void stage_flush_warp(PushStage& st, unsigned long long* q, unsigned* qn,
                                                 uint32_t qcap, TeamCtl* c, uint32_t* qerr, unsigned lane) {
  if (st.fill == 0u) return;
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(qn, st.fill);
  base = __shfl_sync(kFullMask, base, 0);
  __syncwarp();
  if ((unsigned long long)base + st.fill > qcap) {
    if (lane == 0) set_err(c, qerr, kErrInternal);
  } else {
    for (uint32_t j = lane; j < st.fill; j += 32u) q[base + j] = st.buf[j];
  }
  __syncwarp();
  st.fill = 0;
}

// Same contract as warp_push_units, through the warp's stage.
__device__ __forceinline__ void stage_push_units(bool push, uint32_t x, uint32_t deg, uint32_t cshift,
                                                 PushStage& st, unsigned long long* q, unsigned* qn,
                                                 uint32_t qcap, TeamCtl* c, uint32_t* qerr, unsigned lane) {
  if (__ballot_sync(kFullMask, push) == 0u) return;
  const uint32_t nu = push ? ((deg + (1u << cshift) - 1u) >> cshift) : 0u;
  const uint32_t incl = warp_incl_scan(nu, lane);
  const uint32_t tot = __shfl_sync(kFullMask, incl, 31);
  if (tot == 0u) return;
  unsigned long long* dst;
  if (tot > kStageUnits) {  // a hub: straight to the queue
    uint32_t base = 0;
    if (lane == 31) base = atomicAdd(qn, tot);
    base = __shfl_sync(kFullMask, base, 31);
    if ((unsigned long long)base + tot > qcap) {
      if (lane == 0) set_err(c, qerr, kErrInternal);
      return;
    }
    dst = q + base;
  } else {
    if (st.fill + tot > kStageUnits) stage_flush_warp(st, q, qn, qcap, c, qerr, lane);
    dst = st.buf + st.fill;
    st.fill += tot;
  }
  for (uint32_t j0 = 0; j0 < tot; j0 += 32u) {
    const uint32_t j = j0 + lane;
    const int k = warp_owner(incl, j < tot ? j : tot - 1u);
    const uint32_t xk = __shfl_sync(kFullMask, x, k);
    const uint32_t ik = __shfl_sync(kFullMask, incl, k);
    const uint32_t nk = __shfl_sync(kFullMask, nu, k);
    if (j < tot) dst[j] = (unsigned long long)xk | ((unsigned long long)(j - (ik - nk)) << 32);
  }
  __syncwarp();
}

// End of a round: every warp's leftovers go to the queue with one atomic per
// CTA.  Every thread of the CTA must call it.
__device__ __forceinline__ void stage_flush_cta(PushStage& st, unsigned long long* q, unsigned* qn,
                                                uint32_t qcap, TeamCtl* c, uint32_t* qerr, unsigned lane) {
  __shared__ uint32_t s_off[33];
  const unsigned wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) s_off[wid] = st.fill;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (unsigned i = 0; i < nw; ++i) {
      const uint32_t f = s_off[i];
      s_off[i] = tot;
      tot += f;
    }
    uint32_t base = 0;
    if (tot) {
      base = atomicAdd(qn, tot);
      if ((unsigned long long)base + tot > qcap) {
        set_err(c, qerr, kErrInternal);
        base = 0xFFFFFFFFu;
      }
    }
    s_off[32] = base;
  }
  __syncthreads();
  const uint32_t base = s_off[32];
  if (base != 0xFFFFFFFFu)
    for (uint32_t j = lane; j < st.fill; j += 32u) q[base + s_off[wid] + j] = st.buf[j];
  st.fill = 0;
  __syncthreads();
}

// warp maximum of `x`; lane 0 folds it into *slot when any lane has `on` set
__device__ __forceinline__ void warp_fold_max(bool on, uint32_t x, unsigned* slot, unsigned lane) {
  if (__ballot_sync(kFullMask, on) == 0u) return;
  const uint32_t m = __reduce_max_sync(kFullMask, on ? x : 0u);
  if (lane == 0) atomicMax(slot, m);
}

}  // namespace svv
