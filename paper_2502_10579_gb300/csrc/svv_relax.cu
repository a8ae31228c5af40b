// svv_relax.cu -- concurrent relaxation of every window snapshot over the
// Q-relevant subgraph (Section 4.2, Algorithm 2), and the output scatter.
//
// Values are kept vertex-major: row r of `val` holds the LP values of unstable
// vertex uv[r], one per snapshot of the slab, so one out-edge of a frontier
// vertex touches one contiguous run of the target's values.  A group of P
// lanes owns one work unit (row, chunk of edges); lane gl of the group holds
// snapshots gl, gl+P, ... (K of them).  The group loads P edges at once, then
// broadcasts them one by one; each lane relaxes its snapshots whose bit is set
// in the edge's mask (edge ownership, Section 4.2).  The frontier is
// snapshot-oblivious: a row is queued once per round if any of its snapshots
// improved.
//
// Round 0 initialises every row to the intersection-graph value (Algorithm 2
// "R_i = R_QRS") and seeds from the addition edges whose sink is unstable
// (Algorithm 2 addition batches; Section 3 Step 4 drops those with a stable
// sink).  The seeding reads the resident list of edges that are not present in
// all snapshots; an edge present in every window snapshot belongs to the
// intersection graph, whose values are already a fixed point on it, so it is
// skipped.  Sources of seed edges hold their intersection-graph value in every
// snapshot at that point.
#include <algorithm>

#include "svv_relax.cuh"

namespace svv {

constexpr int kRelaxThreads = 512;

template <class Op, int P, int K>
__global__ void __launch_bounds__(kRelaxThreads, 2) relax_kernel(RelaxArgs a) {
  __shared__ unsigned long long s_stage[(kRelaxThreads / 32) * kStageUnits];
  const Team t{a.ctl, a.qerr, gridDim.x, blockIdx.x, a.spin_ns};
  relax_team<Op, P, K>(a, t, s_stage);
}

// ---------------------------------------------------------------------------
// Output scatter: out[(s0+i)*V + v] = intersection value if v is stable, else
// the relaxed value of its row.  A CTA stages a tile of kTV vertices x ls
// snapshots in shared memory so the row reads and the snapshot-major writes
// both coalesce.  The tile's row map is read first; then a warp takes four
// vertices at a time with a lane per snapshot, every load independent of the
// others.  Tile element (i, t) sits at i*kTV + (t ^ (i & 31)): the lanes of a
// fill store (consecutive i, one t) hit 32 different banks, and the four
// words of an aligned 16-byte group stay in one group, permuted by i & 3.
// When V is a multiple of 4 the writes are 16-byte streaming stores (the
// output is not read again by this query).
constexpr int kTV = 128;
constexpr int kScatterThreads = 256;

__device__ __forceinline__ uint32_t pick4(const uint4& w, uint32_t k) {
  return k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w;
}

__global__ void __launch_bounds__(kScatterThreads) scatter_kernel(ScatterArgs a) {
  extern __shared__ __align__(16) uint32_t tile[];  // [ls][kTV], swizzled
  __shared__ uint32_t s_row[kTV];
  __shared__ __align__(16) uint32_t s_x[kTV];
  if (*a.qerr != 0u) return;
  const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t lps = __ffs(a.LP) - 1;
  const bool vec = (a.V & 3u) == 0u && ((uintptr_t)a.out & 15u) == 0u;
  constexpr uint32_t kQ = kTV / 4, kRows = kScatterThreads / kQ;  // 16-byte stores: 32 per tile row
  const uint32_t q = threadIdx.x % kQ, r0 = threadIdx.x / kQ;
  {
    const uint32_t tl = blockIdx.x;  // one tile per CTA
    const uint32_t v0 = tl * kTV;
    const uint32_t nv = min((uint32_t)kTV, a.V - v0);
    bool mine = false;
    for (uint32_t t = threadIdx.x; t < (uint32_t)kTV; t += blockDim.x) {
      const bool in = t < nv;
      const uint32_t r = in ? a.row[v0 + t] : kNone;
      s_row[t] = r;
      s_x[t] = in ? a.rI[v0 + t] : 0u;
      mine |= r != kNone;
    }
    if (!__syncthreads_or(mine) && vec && nv == (uint32_t)kTV) {
      // every vertex of the tile is stable: each snapshot row is the tile's
      // intersection values, written straight from the row map's buffer
      const uint4 x = *reinterpret_cast<const uint4*>(s_x + 4u * q);
      for (uint32_t i = r0; i < a.ls; i += kRows)
        __stcs(reinterpret_cast<uint4*>(a.out + (size_t)(a.s0 + i) * a.V + v0) + q, x);
      return;
    }
    for (uint32_t t0 = 4u * wid; t0 < (uint32_t)kTV; t0 += 4u * nw) {
      uint32_t r[4], x[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        r[h] = s_row[t0 + h];
        x[h] = s_x[t0 + h];
      }
      for (uint32_t i = lane; i < a.ls; i += 32u) {
        uint32_t y[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) y[h] = r[h] == kNone ? x[h] : (a.val[((size_t)r[h] << lps) + i] ^ a.rflip);
#pragma unroll
        for (int h = 0; h < 4; ++h) tile[i * kTV + ((t0 + h) ^ (i & 31u))] = y[h];
      }
    }
    __syncthreads();
    if (vec && nv == (uint32_t)kTV) {
      // a warp per tile row: 32 threads x 16 bytes
      for (uint32_t i = r0; i < a.ls; i += kRows) {
        const uint32_t sw = i & 31u;
        const uint4 w = *reinterpret_cast<const uint4*>(tile + i * kTV + 4u * (q ^ (sw >> 2)));
        const uint32_t k = sw & 3u;
        const uint4 o = make_uint4(pick4(w, k), pick4(w, 1u ^ k), pick4(w, 2u ^ k), pick4(w, 3u ^ k));
        __stcs(reinterpret_cast<uint4*>(a.out + (size_t)(a.s0 + i) * a.V + v0) + q, o);
      }
    } else {
      for (uint32_t i = wid; i < a.ls; i += nw)
        for (uint32_t t = lane; t < nv; t += 32u)
          a.out[(size_t)(a.s0 + i) * a.V + v0 + t] = tile[i * kTV + (t ^ (i & 31u))];
    }
  }
}

// Compact output: copy slab columns [s0, s0+ls) of the U relaxed rows into the
// caller's U x wl array.
__global__ void __launch_bounds__(256) compact_kernel(CompactArgs a) {
  if (*a.qerr != 0u) return;
  const uint32_t U = a.counts[0];
  if ((unsigned long long)U * a.wl > a.rows_cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(a.qerr, 0u, 2u);  // 2 = SVV_ENOMEM
    return;
  }
  const uint32_t lps = __ffs(a.LP) - 1;
  const unsigned long long n = (unsigned long long)U * a.ls;
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t r = (uint32_t)(k / a.ls), i = (uint32_t)(k % a.ls);
    a.rows_out[(size_t)r * a.wl + a.s0 + i] = a.val[((size_t)r << lps) + i];
  }
}

// The result of a query from a source with no out-edge, written at the
// output's bandwidth: 16-byte streaming stores when V is a multiple of 4.
__global__ void __launch_bounds__(256) isolated_kernel(IsolatedArgs a) {
  const size_t nthreads = (size_t)gridDim.x * blockDim.x;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (size_t v = tid; v < a.V; v += nthreads) {
    const uint32_t x = v == a.source ? a.src_val : a.ident;
    a.rI[v] = x;
    a.rU[v] = x;
    a.row[v] = kNone;
  }
  if (!a.out) return;
  if ((a.V & 3u) == 0u && ((uintptr_t)a.out & 15u) == 0u) {
    const size_t per_row = a.V >> 2, n = per_row * a.L;
    for (size_t k = tid; k < n; k += nthreads) {
      const uint32_t v = (uint32_t)(k % per_row) * 4u;
      uint4 o = make_uint4(a.ident, a.ident, a.ident, a.ident);
      if (a.source - v < 4u) {
        const uint32_t j = a.source - v;
        if (j == 0) o.x = a.src_val;
        else if (j == 1) o.y = a.src_val;
        else if (j == 2) o.z = a.src_val;
        else o.w = a.src_val;
      }
      __stcs(reinterpret_cast<uint4*>(a.out) + k, o);
    }
  } else {
    const size_t n = (size_t)a.V * a.L;
    for (size_t k = tid; k < n; k += nthreads) a.out[k] = (k % a.V) == a.source ? a.src_val : a.ident;
  }
}

cudaError_t launch_isolated(const IsolatedArgs& a, cudaStream_t s) {
  isolated_kernel<<<std::max<uint32_t>(1, a.sms) * 8u, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_compact(const CompactArgs& a, cudaStream_t s) {
  compact_kernel<<<1216, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
template <class Op, int P, int K>
static cudaError_t launch_r(const RelaxArgs& a, LaunchCfg cfg, cudaStream_t s) {
  RelaxArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)relax_kernel<Op, P, K>, dim3(cfg.blocks),
                                     dim3(cfg.threads), args, 0, s);
}

template <class Op>
static cudaError_t launch_pk(uint32_t P, uint32_t K, const RelaxArgs& a, LaunchCfg cfg, cudaStream_t s) {
  switch (P * 100 + K) {
    case 801: return launch_r<Op, 8, 1>(a, cfg, s);
    case 802: return launch_r<Op, 8, 2>(a, cfg, s);
    case 804: return launch_r<Op, 8, 4>(a, cfg, s);
    case 808: return launch_r<Op, 8, 8>(a, cfg, s);
    case 1601: return launch_r<Op, 16, 1>(a, cfg, s);
    case 1602: return launch_r<Op, 16, 2>(a, cfg, s);
    case 1604: return launch_r<Op, 16, 4>(a, cfg, s);
    case 1608: return launch_r<Op, 16, 8>(a, cfg, s);
    case 3201: return launch_r<Op, 32, 1>(a, cfg, s);
    case 3202: return launch_r<Op, 32, 2>(a, cfg, s);
    case 3204: return launch_r<Op, 32, 4>(a, cfg, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_relax(int type, uint32_t P, uint32_t K, const RelaxArgs& a, LaunchCfg cfg,
                         cudaStream_t s) {
  switch (type) {
    case 0: return launch_pk<OpSSSP>(P, K, a, cfg, s);
    case 1: return launch_pk<OpSSWP>(P, K, a, cfg, s);
    case 3: return launch_pk<OpSSNP>(P, K, a, cfg, s);
    case kTypeMixed: return launch_pk<OpMixed>(P, K, a, cfg, s);
    default: return launch_pk<OpBFS>(P, K, a, cfg, s);
  }
}

cudaError_t launch_scatter(const ScatterArgs& a, cudaStream_t s) {
  const uint32_t blocks = (a.V + kTV - 1) / kTV;  // one tile per CTA
  const size_t smem = (size_t)a.ls * kTV * sizeof(uint32_t);  // up to 64 KB at 128 snapshots
  // the opt-in covers the dynamic tile plus the kernel's static row map
  if (smem + 2 * kTV * sizeof(uint32_t) > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute((const void*)scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  scatter_kernel<<<blocks, kScatterThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <class Op>
static int occ_op(int threads) {
  const void* ks[] = {(const void*)relax_kernel<Op, 8, 1>,  (const void*)relax_kernel<Op, 8, 2>,
                      (const void*)relax_kernel<Op, 8, 4>,  (const void*)relax_kernel<Op, 8, 8>,
                      (const void*)relax_kernel<Op, 16, 1>, (const void*)relax_kernel<Op, 16, 2>,
                      (const void*)relax_kernel<Op, 16, 4>, (const void*)relax_kernel<Op, 16, 8>,
                      (const void*)relax_kernel<Op, 32, 1>, (const void*)relax_kernel<Op, 32, 2>,
                      (const void*)relax_kernel<Op, 32, 4>};
  int best = 1 << 30;
  for (const void* k : ks) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, 0) != cudaSuccess) return 0;
    best = n < best ? n : best;
  }
  return best;
}

int occupancy_relax(int threads) {
  int a = occ_op<OpSSSP>(threads), b = occ_op<OpSSWP>(threads), c = occ_op<OpBFS>(threads);
  int d = occ_op<OpSSNP>(threads), e = occ_op<OpMixed>(threads);
  int m = a < b ? a : b;
  m = m < c ? m : c;
  m = m < d ? m : d;
  return m < e ? m : e;
}

}  // namespace svv
