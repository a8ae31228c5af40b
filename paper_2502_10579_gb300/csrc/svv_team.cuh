// svv_team.cuh -- a team of co-resident CTAs that runs one query phase.
//
// A single query uses the whole cooperative grid as one team; the batch kernel
// splits its grid into several teams that each run whole queries.  A team has
// its own barrier state and error flag (`bar`) and reports errors of the
// query it runs in `qerr`.
#pragma once

#include "svv_device.cuh"

namespace svv {

struct Team {
  TeamCtl* bar;
  uint32_t* qerr;
  unsigned nblocks, rank;
  unsigned long long spin_ns;
  __device__ __forceinline__ unsigned nthreads() const { return nblocks * blockDim.x; }
  __device__ __forceinline__ unsigned tid() const { return rank * blockDim.x + threadIdx.x; }
  __device__ __forceinline__ bool sync() const { return team_sync(bar, qerr, nblocks, spin_ns); }
};

}  // namespace svv
