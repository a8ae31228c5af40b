// svv_group.cu -- the intersection- and union-graph solves (Section 3 Step 1)
// of a group of same-type queries in one persistent cooperative launch each,
// with one query-oblivious frontier (Section 4.2) shared by the group; see
// svv_group.cuh.  Around the solves:
//   group_lanes_kernel: per partial edge, the lanes whose window holds it in
//     every snapshot / in some snapshot (read once per group instead of the
//     masks in every round);
//   group_split_kernel: each lane's bound values copied into planar arrays,
//     where the per-query phases (stable compaction, subgraph extraction,
//     relaxation, scatter) read them.
#include <algorithm>
#include <iterator>
#include <vector>

#include "svv_group.cuh"

namespace svv {

constexpr int kGroupThreads = 512;

__global__ void __launch_bounds__(256) group_lanes_kernel(LanesArgs a) {
  const DevGraph& g = a.g;
  const uint32_t n = g.NF;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint64_t* m = g.nfmask + (size_t)k * g.W;
    uint32_t w = 0;
    for (uint32_t l = 0; l < a.nlanes; ++l) {
      bool any, all;
      window_any_all(m, a.win[l], any, all);
      w |= (all ? 1u : 0u) << l;
      w |= (any ? 1u : 0u) << (16u + l);
    }
    a.nflanes[k] = w;
    if (a.iplanes) {
      const uint64_t* mi = g.ipmask + (size_t)k * g.W;
      uint32_t wi = 0;
      for (uint32_t l = 0; l < a.nlanes; ++l) {
        bool any, all;
        window_any_all(mi, a.win[l], any, all);
        wi |= (all ? 1u : 0u) << l;
        wi |= (any ? 1u : 0u) << (16u + l);
      }
      a.iplanes[k] = wi;
    }
  }
}

// two-lane groups fit 40 registers: 3 CTAs per SM, as the single solve
template <class Op, int KL, int PRED>
__global__ void __launch_bounds__(kGroupThreads, KL == 2 ? 3 : 2) group_solve_kernel(GroupArgs a) {
  __shared__ unsigned long long s_stage[(kGroupThreads / 32) * kStageUnits];
  const Team t{a.ctl, a.qerr, gridDim.x, blockIdx.x, a.spin_ns};
  group_solve_team<Op, KL, PRED>(a, t, s_stage);
}

// a thread per vertex: the lane rows of both bounds in, one word per lane and
// bound out (every lane's planar arrays are written by consecutive threads)
template <int KL>
__global__ void __launch_bounds__(256) group_split_kernel(SplitArgs a) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < a.V; v += gridDim.x * blockDim.x) {
    uint32_t ci[KL], cu[KL];
    if constexpr (KL == 2) {
      const uint2 x = __ldcs(reinterpret_cast<const uint2*>(a.cap + (size_t)v * KL));
      const uint2 y = __ldcs(reinterpret_cast<const uint2*>(a.cup + (size_t)v * KL));
      ci[0] = x.x, ci[1] = x.y;
      cu[0] = y.x, cu[1] = y.y;
    } else {
      const uint4* pi = reinterpret_cast<const uint4*>(a.cap + (size_t)v * KL);
      const uint4* pu = reinterpret_cast<const uint4*>(a.cup + (size_t)v * KL);
#pragma unroll
      for (int i = 0; i < KL / 4; ++i) {
        const uint4 x = __ldcs(pi + i), y = __ldcs(pu + i);
        ci[4 * i] = x.x, ci[4 * i + 1] = x.y, ci[4 * i + 2] = x.z, ci[4 * i + 3] = x.w;
        cu[4 * i] = y.x, cu[4 * i + 1] = y.y, cu[4 * i + 2] = y.z, cu[4 * i + 3] = y.w;
      }
    }
#pragma unroll
    for (int k = 0; k < KL; ++k) {
      if ((uint32_t)k < a.nlanes) {
        // a complemented lane (SSWP in a mixed group) gets its widths back
        const uint32_t f = ((a.flip >> k) & 1u) ? 0xFFFFFFFFu : 0u;
        a.rI[k][v] = ci[k] ^ f;
        a.rU[k][v] = cu[k] ^ f;
      }
    }
  }
}

cudaError_t launch_group_lanes(const LanesArgs& a, cudaStream_t s) {
  if (a.g.NF == 0) return cudaSuccess;
  const uint32_t blocks = std::min<uint32_t>((a.g.NF + 255u) / 256u, 152u * 8u);
  group_lanes_kernel<<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <class Op, int KL, int PRED>
static cudaError_t launch_g(const GroupArgs& a, LaunchCfg cfg, cudaStream_t s) {
  GroupArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)group_solve_kernel<Op, KL, PRED>, dim3(cfg.blocks),
                                     dim3(cfg.threads), args, 0, s);
}

template <class Op>
static cudaError_t launch_gk(uint32_t KL, int pred, const GroupArgs& a, LaunchCfg cfg, cudaStream_t s) {
  if (KL == 2) return pred == kPredAll ? launch_g<Op, 2, kPredAll>(a, cfg, s) : launch_g<Op, 2, kPredAny>(a, cfg, s);
  if (KL == 4) return pred == kPredAll ? launch_g<Op, 4, kPredAll>(a, cfg, s) : launch_g<Op, 4, kPredAny>(a, cfg, s);
  if (KL == 8) return pred == kPredAll ? launch_g<Op, 8, kPredAll>(a, cfg, s) : launch_g<Op, 8, kPredAny>(a, cfg, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_group_solve(int type, uint32_t KL, int pred, const GroupArgs& a, LaunchCfg cfg, cudaStream_t s) {
  switch (type) {
    case 0: return launch_gk<OpSSSP>(KL, pred, a, cfg, s);
    case 1: return launch_gk<OpSSWP>(KL, pred, a, cfg, s);
    case 3: return launch_gk<OpSSNP>(KL, pred, a, cfg, s);
    case kTypeMixed: return launch_gk<OpMixed>(KL, pred, a, cfg, s);
    default: return launch_gk<OpBFS>(KL, pred, a, cfg, s);
  }
}

cudaError_t launch_group_split(const SplitArgs& a, cudaStream_t s) {
  const uint32_t blocks = std::min<uint32_t>((a.V + 255u) / 256u, 152u * 16u);
  if (a.KL == 2) group_split_kernel<2><<<blocks, 256, 0, s>>>(a);
  else if (a.KL == 4) group_split_kernel<4><<<blocks, 256, 0, s>>>(a);
  else if (a.KL == 8) group_split_kernel<8><<<blocks, 256, 0, s>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <class Op>
static int occ_g(int threads, bool two) {
  const void* k2[] = {(const void*)group_solve_kernel<Op, 2, kPredAll>, (const void*)group_solve_kernel<Op, 2, kPredAny>};
  const void* k48[] = {(const void*)group_solve_kernel<Op, 4, kPredAll>, (const void*)group_solve_kernel<Op, 4, kPredAny>,
                       (const void*)group_solve_kernel<Op, 8, kPredAll>, (const void*)group_solve_kernel<Op, 8, kPredAny>};
  std::vector<const void*> ks;
  if (two) ks.assign(std::begin(k2), std::end(k2));
  else ks.assign(std::begin(k48), std::end(k48));
  int best = 1 << 30;
  for (const void* k : ks) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, 0) != cudaSuccess) return 0;
    best = n < best ? n : best;
  }
  return best;
}

// CTAs per SM of the group solves of four or eight lanes (two = false) or of
// two lanes (two = true)
int occupancy_group(int threads, bool two) {
  const int a = occ_g<OpSSSP>(threads, two), b = occ_g<OpSSWP>(threads, two), c = occ_g<OpBFS>(threads, two),
            d = occ_g<OpSSNP>(threads, two), e = occ_g<OpMixed>(threads, two);
  return std::min(std::min(std::min(a, b), std::min(c, d)), e);
}

}  // namespace svv
