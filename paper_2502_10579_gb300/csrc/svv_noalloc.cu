// svv_noalloc.cu -- svv_solve_snapshot_noalloc: one snapshot's full solve
// that allocates nothing.
//
// Some callers cannot allocate device memory at the time they call: code that
// runs inside a host or device memory pool that forbids cudaMalloc, plug-ins
// whose host application owns every allocation, or services that reserve all
// memory up front.  This entry point takes the caller's device CSR (the same
// layout svv_load takes) and the caller's output array, and keeps its own
// working memory (frontier queues, round stamps, control block) in a fixed
// file-scope device array of kNoAllocScratchBytes.  Every GPU that loads the
// library holds that array until the process exits.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the address is looked up once per device
// with cudaGetSymbolAddress, with that device current, and passed to the
// kernel.  Calls share the array: two calls that overlap on the GPU race.
#include <mutex>

#include "../../include/svv.h"
#include "svv_device.cuh"
#include "svv_push.cuh"

namespace svv {
namespace {

constexpr size_t kNoAllocScratchBytes = 32ull << 20;  // 32 MiB
constexpr int kNaThreads = 512;
constexpr uint32_t kNaChunkShift = 6;  // 64 edges per work unit
constexpr uint32_t kErrInput = 1;      // malformed CSR found by the kernel (SVV_EINVAL)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NaArgs {
  uint32_t V, W;
  unsigned long long E;
  const uint64_t* rp;
  const uint32_t* col;
  const uint32_t* wt;
  const uint64_t* mask;
  uint32_t snap, source;
  uint32_t* val;
  TeamCtl* ctl;
  uint32_t* qerr;
  uint32_t* stamp;
  unsigned long long* q0;
  unsigned long long* q1;
  uint32_t qcap;
  uint32_t maxit;
  unsigned long long spin_ns;
};

// Same round structure as the plain per-snapshot solve (persistent
// cooperative grid, bounded team barrier, chunked work units, warp-balanced
// edge walk), read straight from the svv_load layout: 64-bit row offsets,
// separate target and weight arrays, edge-major masks.  Rows or targets that
// break the CSR rules are skipped and reported, so no access leaves the arrays.
template <class Op>
__global__ void __launch_bounds__(kNaThreads) noalloc_solve_kernel(NaArgs a) {
  TeamCtl* c = a.ctl;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned nthreads = gridDim.x * blockDim.x;
  const unsigned gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t C = 1u << kNaChunkShift;

  // starting values, and the CSR rules the queue bound rests on: row_ptr[0]
  // = 0, rows never go backwards, row_ptr[V] = E (then every vertex's units
  // fit the V + E/64 + 64 queue in every round)
  for (uint32_t v = gtid; v < a.V; v += nthreads) {
    a.val[v] = Op::kIdentity;
    a.stamp[v] = 0u;
    const uint64_t r0 = __ldg(a.rp + v), r1 = __ldg(a.rp + v + 1);
    if (r1 < r0 || r1 > a.E || (v == 0 && r0 != 0) || (v + 1 == a.V && r1 != a.E)) set_err(c, a.qerr, kErrInput);
  }
  if (!team_sync(c, a.qerr, gridDim.x, a.spin_ns)) return;

  if (blockIdx.x == 0 && threadIdx.x < 32) {
    uint32_t deg = 0;
    if (lane == 0) {
      a.val[a.source] = Op::kSource;
      a.stamp[a.source] = 1u;
      const uint64_t r0 = a.rp[a.source], r1 = a.rp[a.source + 1];
      if (r1 >= r0 && r1 <= a.E) deg = (uint32_t)(r1 - r0);
      else set_err(c, a.qerr, kErrInput);
    }
    warp_push_units(lane == 0, a.source, deg, kNaChunkShift, a.q1, &c->qn[1], a.qcap, c, a.qerr, lane);
  }
  if (!team_sync(c, a.qerr, gridDim.x, a.spin_ns)) return;

  const uint32_t word = a.snap >> 6;
  const uint64_t bit = 1ull << (a.snap & 63u);
  uint32_t it = 1;
  for (;; ++it) {
    const uint32_t cur = it % 3u, nxt = (it + 1u) % 3u, clr = (it + 2u) % 3u;
    uint32_t n = ld_acquire(&c->qn[cur]);
    if (n == 0u) break;
    if (it > a.maxit) {
      if (gtid == 0) set_err(c, a.qerr, kErrTimeout);
      break;
    }
    n = min(n, a.qcap);
    if (gtid == 0) {
      atomicExch(&c->qn[clr], 0u);
      atomicExch(&c->ticket[clr], 0u);
    }
    const unsigned long long* qin = (it & 1u) ? a.q1 : a.q0;
    unsigned long long* qout = (it & 1u) ? a.q0 : a.q1;
    const uint32_t stamp_next = it + 1u;
    for (;;) {
      uint32_t t0 = 0;
      if (lane == 0) t0 = atomicAdd(&c->ticket[cur], 32u);
      t0 = __shfl_sync(kFullMask, t0, 0);
      if (t0 >= n) break;
      const uint32_t ui = t0 + lane;
      uint64_t beg = 0;
      uint32_t cnt = 0, sv = Op::kIdentity;
      if (ui < n) {
        const unsigned long long u = ld_cg(qin + ui);
        const uint32_t v = (uint32_t)u, ch = (uint32_t)(u >> 32);
        const uint64_t r0 = __ldg(a.rp + v), r1 = __ldg(a.rp + v + 1);
        if (r1 < r0 || r1 > a.E) {
          set_err(c, a.qerr, kErrInput);
        } else {
          beg = r0 + ((uint64_t)ch << kNaChunkShift);
          const uint64_t end = min(r1, beg + C);
          cnt = end > beg ? (uint32_t)(end - beg) : 0u;
          sv = ld_cg(a.val + v);
        }
      }
      const uint32_t incl = warp_incl_scan(cnt, lane);
      const uint32_t total = __shfl_sync(kFullMask, incl, 31);
      for (uint32_t p0 = 0; p0 < total; p0 += 32u) {
        const uint32_t p = p0 + lane;
        const int k = warp_owner(incl, p < total ? p : total - 1u);
        const uint32_t ik = __shfl_sync(kFullMask, incl, k);
        const uint32_t ck = __shfl_sync(kFullMask, cnt, k);
        const uint64_t bk = __shfl_sync(kFullMask, beg, k);
        const uint32_t sk = __shfl_sync(kFullMask, sv, k);
        bool push = false;
        uint32_t x = 0, deg = 0;
        if (p < total) {
          const uint64_t e = bk + (p - (ik - ck));
          if (__ldg(a.mask + e * a.W + word) & bit) {
            x = __ldg(a.col + e);
            if (x >= a.V) {
              set_err(c, a.qerr, kErrInput);
            } else {
              const uint32_t cand = Op::relax(sk, __ldg(a.wt + e));
              if (Op::better(cand, ld_cg(a.val + x))) {
                const uint32_t old = Op::atomic(a.val + x, cand);
                if (Op::better(cand, old) && atomicExch(a.stamp + x, stamp_next) != stamp_next) {
                  const uint64_t x0 = __ldg(a.rp + x), x1 = __ldg(a.rp + x + 1);
                  if (x1 >= x0 && x1 <= a.E) {
                    push = true;
                    deg = (uint32_t)(x1 - x0);
                  } else {
                    set_err(c, a.qerr, kErrInput);
                  }
                }
              }
            }
          }
        }
        warp_push_units(push, x, deg, kNaChunkShift, qout, &c->qn[nxt], a.qcap, c, a.qerr, lane);
      }
    }
    if (!team_sync(c, a.qerr, gridDim.x, a.spin_ns)) return;
  }
  if (gtid == 0) c->iters = it - 1u;
}

struct NaDevice {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch
  int blocks = 0;
};

std::mutex g_na_mu;
NaDevice g_na_dev[kMaxDevices];

int na_occupancy() {
  int best = 1 << 30;
  const void* ks[] = {(const void*)noalloc_solve_kernel<OpSSSP>, (const void*)noalloc_solve_kernel<OpSSWP>,
                      (const void*)noalloc_solve_kernel<OpBFS>};
  for (const void* k : ks) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kNaThreads, 0) != cudaSuccess) return 0;
    best = n < best ? n : best;
  }
  return best;
}

// Once per device, with that device current: look up the array's device
// address and the cooperative grid size.
svv_status na_setup(int dev, NaDevice** out) {
  std::lock_guard<std::mutex> lk(g_na_mu);
  NaDevice& d = g_na_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return SVV_ECUDA;
    }
    int coop = 0, sms = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || !coop || sms <= 0) {
      cudaGetLastError();
      return SVV_ECUDA;
    }
    const int occ = na_occupancy();
    if (occ <= 0) {
      cudaGetLastError();
      return SVV_ECUDA;
    }
    d.base = static_cast<unsigned char*>(p);
    d.blocks = sms * (occ < 2 ? occ : 2);
    d.ready = true;
  }
  *out = &d;
  return SVV_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace svv

using namespace svv;

extern "C" svv_status svv_solve_snapshot_noalloc(svv_type type, uint32_t V, uint64_t E, uint32_t S,
                                                 const uint64_t* row_ptr, const uint32_t* col,
                                                 const uint32_t* weight, const uint64_t* mask, uint32_t snapshot,
                                                 uint32_t source, uint32_t* out, void* cuda_stream) {
  if ((int)type < 0 || (int)type > 2) return SVV_EINVAL;
  if (V == 0 || V >= 0xFFFFFFFFu || S == 0 || snapshot >= S || source >= V) return SVV_EINVAL;
  if (E >= 0xFFFFFFFFull) return SVV_EINVAL;
  if (!row_ptr || !out || (E && (!col || !weight || !mask))) return SVV_EINVAL;
  // working memory: control block, error word, stamps[V], two queues of
  // V + E/64 + 64 units
  const uint64_t qcap = (uint64_t)V + (E >> kNaChunkShift) + 64;
  const size_t off_qerr = align256(sizeof(TeamCtl));
  const size_t off_stamp = off_qerr + 256;
  const size_t off_q0 = off_stamp + align256((size_t)V * 4);
  const size_t off_q1 = off_q0 + align256((size_t)qcap * 8);
  const size_t need = off_q1 + align256((size_t)qcap * 8);
  if (need > kNoAllocScratchBytes) return SVV_EINVAL;  // graph too large for the fixed scratch

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SVV_ECUDA;
  }
  NaDevice* d = nullptr;
  svv_status st = na_setup(dev, &d);
  if (st != SVV_OK) return st;

  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (cudaMemsetAsync(d->base, 0, off_stamp, s) != cudaSuccess) {  // control block + error word
    cudaGetLastError();
    return SVV_ECUDA;
  }
  NaArgs a{};
  a.V = V;
  a.W = (S + 63) / 64;
  a.E = E;
  a.rp = row_ptr;
  a.col = col;
  a.wt = weight;
  a.mask = mask;
  a.snap = snapshot;
  a.source = source;
  a.val = out;
  a.ctl = reinterpret_cast<TeamCtl*>(d->base);
  a.qerr = reinterpret_cast<uint32_t*>(d->base + off_qerr);
  a.stamp = reinterpret_cast<uint32_t*>(d->base + off_stamp);
  a.q0 = reinterpret_cast<unsigned long long*>(d->base + off_q0);
  a.q1 = reinterpret_cast<unsigned long long*>(d->base + off_q1);
  a.qcap = (uint32_t)qcap;
  a.maxit = V + 2u;
  a.spin_ns = 1000000000ull;
  void* args[] = {&a};
  const void* k = type == SVV_SSSP ? (const void*)noalloc_solve_kernel<OpSSSP>
                  : type == SVV_SSWP ? (const void*)noalloc_solve_kernel<OpSSWP>
                                     : (const void*)noalloc_solve_kernel<OpBFS>;
  cudaError_t e = cudaLaunchCooperativeKernel(k, dim3(d->blocks), dim3(kNaThreads), args, 0, s);
  uint32_t herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, a.qerr, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SVV_ECUDA;
  }
  if (herr == kErrTimeout) return SVV_ETIMEOUT;
  if (herr == kErrInput) return SVV_EINVAL;
  if (herr != 0) return SVV_EINTERNAL;
  return SVV_OK;
}
