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

}  // namespace svv
