// svv_ctx.h -- the library context and its host-side helpers (shared by the
// host translation units).
#pragma once

#include <algorithm>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/svv.h"
#include "svv_internal.h"

namespace svv {

constexpr int kNumCtl = 8 + 256;  // 0..3 query phases, 4..5 group solves, 8.. per-snapshot plain solves
constexpr int kAsyncSlots = 64;   // svv_query_async queries in flight
constexpr uint32_t kMaxSlab = 128;
constexpr uint32_t kTraceCap = 4096;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// scratch of the batch kernel's teams, sized for a window length
struct BatchPool {
  int want = 0;   // teams asked for when the pool was built
  int teams = 0;  // teams built (fewer when the budget is short)
  uint32_t team_blocks = 0;
  uint32_t LP = 0, QW = 0;
  TeamScratch* d_sc = nullptr;
  TeamCtl* d_ctl = nullptr;
  std::vector<void*> bufs;
  uint64_t bytes = 0;
  // per-instance arrays
  uint32_t icap = 0;
  BatchInstance* d_inst = nullptr;
  uint32_t *d_qerr = nullptr, *d_done = nullptr;
  unsigned long long *d_t0 = nullptr, *d_t1 = nullptr;
  unsigned* d_next = nullptr;
  std::vector<void*> ibufs;
  uint64_t ibytes = 0;
};

// launch knobs of one query type and window-length bucket (the autotuner
// picks them; the defaults come from svv_set_tuning)
struct Knobs {
  uint32_t solve_cs;
  int bps;
  uint32_t relax_lanes;
  bool skip_same;
  uint32_t pull_pct;  // pull when the frontier holds more than this % of all units (0 = push only)
  uint32_t delta;     // near-far width of the SSSP / SSWP solves (0 = off)
  uint32_t slab_max;  // snapshots relaxed per pass
};
constexpr int kLenBuckets = 5;  // windows of up to 8, 16, 32, 64, 128+ snapshots
inline int len_bucket(uint32_t L) {
  return L <= 8 ? 0 : L <= 16 ? 1 : L <= 32 ? 2 : L <= 64 ? 3 : 4;
}

// serving: instance ring in host-mapped memory, output arena, live kernel
struct ServeSlot {
  uint64_t ticket = 0;
  bool busy = false;     // submitted, not yet released
  bool arena = false;    // output lives in the arena
  uint64_t off = 0, size = 0;
  uint32_t* out = nullptr;
};

// Grouped serving (graphs from 2M vertices): a scheduler thread takes the
// submitted requests, forms query groups and queues them on the server's
// stream; `enq` serialises that with every other use of the query scratch.
struct ServeSched {
  std::thread th;
  std::mutex mu;                 // pending, stop
  std::condition_variable cv;
  std::deque<uint32_t> pending;  // ring slots submitted and not yet queued
  bool stop = false;             // drain the pending requests, then leave
  std::mutex enq;
  uint32_t *h_gflag = nullptr, *d_gflag = nullptr;  // per queued group: bounds done
  uint32_t gring = 256;
  uint64_t gcount = 0;           // groups queued
  uint64_t grouped = 0;          // requests that ran in a group of two or more
};

struct ServeState {
  bool active = false;
  uint32_t cap = 0, maxL = 0;
  BatchInstance* h_inst = nullptr;
  BatchInstance* d_inst = nullptr;
  uint32_t *h_ctrl = nullptr, *d_ctrl = nullptr;  // [0] tail, [1] stop
  uint32_t *h_done = nullptr, *d_done = nullptr;
  uint32_t *h_qerr = nullptr, *d_qerr = nullptr;
  unsigned long long *h_t0 = nullptr, *d_t0 = nullptr, *h_t1 = nullptr, *d_t1 = nullptr;
  unsigned* d_next = nullptr;
  uint64_t tail = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool launched = false;
  uint64_t launches = 0;
  // output arena: a ring of allocations released roughly in order
  struct Alloc {
    uint64_t off, size;
    bool freed;
  };
  unsigned char* arena = nullptr;
  uint64_t arena_bytes = 0, a_end = 0;  // a_end: end of the newest allocation
  std::deque<Alloc> allocs;             // in allocation order
  std::vector<ServeSlot> slots;
  std::vector<void*> bufs;
  uint64_t bytes = 0;
  unsigned long long idle_ns = 200000000ull;
  // grouped mode: requests run in query groups queued by the scheduler on
  // `stream`, with svv_query's scratch
  bool in_order = false;
  cudaEvent_t ord = nullptr;  // orders other streams' use of the query scratch
  std::unique_ptr<ServeSched> sched;
};

}  // namespace svv

struct svv_ctx {
  int device = 0;
  uint64_t budget = 0;      // 0 until a graph is loaded if the caller passed 0
  bool budget_auto = false;
  uint64_t allocated = 0;
  int num_sms = 0;
  std::string err;
  std::thread::id worker;  // the serving scheduler's thread, while it runs

  // tuning
  uint32_t maxit = 0;
  uint32_t spin_ms = 1000;
  uint32_t solve_cs = 5, relax_cs = 4, qrs_cs = 5;
  uint32_t delta[3] = {0, 0, 0};  // near-far width per query type (0 = off)
  int bps = 0;
  int threads = 512;
  int occ_solve = 0, occ_qrs = 0, occ_relax = 0;
  bool phase_timing = false;
  bool round_trace = false;
  unsigned long long* trace = nullptr;  // [3][kTraceCap]: intersection, union, relaxation
  bool skip_same = true;                // per-chunk last-relaxed value (procv)
  uint32_t relax_lanes = 32;            // lanes per edge in the relaxation (8, 16, 32)
  bool pull = true;                     // build the transposed graph at load; pull dense rounds
  uint32_t pull_pct = 15;               // pull when the frontier holds > pull_pct % of all units
  uint32_t* procv = nullptr;
  uint32_t pcap = 0;
  cudaEvent_t ev[7] = {};

  // resident graph
  bool loaded = false;
  svv::DevGraph g{};
  std::vector<void*> graph_bufs;

  // query scratch (sized at load from V and E; the L-dependent part on demand)
  std::vector<void*> scratch_bufs;
  uint32_t *rI = nullptr, *rU = nullptr, *stamp = nullptr, *row = nullptr, *uv = nullptr;
  uint32_t *part = nullptr, *qcnt = nullptr, *cur = nullptr, *qerr = nullptr;
  uint4* qrow = nullptr;
  uint2* qcw = nullptr;
  unsigned long long *q0 = nullptr, *q1 = nullptr, *units = nullptr;
  uint32_t qcap = 0, ucap = 0, ecap = 0;
  svv::TeamCtl* ctl = nullptr;
  svv::TeamCtl* hctl = nullptr;  // pinned mirror
  uint32_t* hqerr = nullptr;
  // window-dependent
  uint64_t* qmask = nullptr;
  uint64_t mcap = 0;
  uint32_t* val = nullptr;
  uint64_t valcap = 0;
  uint32_t* staging = nullptr;  // device output for svv_query_host
  uint64_t staging_cap = 0;
  // a two-query group's tails in one relaxation launch: both queries' rows,
  // subgraph edges and masks in one set of arrays (allocated on first use)
  std::vector<void*> pair_bufs;
  uint32_t *p_uv = nullptr, *p_qcnt = nullptr, *p_cur = nullptr, *p_stamp = nullptr, *p_row1 = nullptr;
  uint4* p_qrow = nullptr;
  uint2* p_qcw = nullptr;
  uint64_t* p_qmask = nullptr;
  uint32_t* p_val = nullptr;
  unsigned long long *p_q0 = nullptr, *p_q1 = nullptr, *p_units = nullptr;
  uint64_t p_valcap = 0, p_qcap = 0, p_mcap = 0;
  bool pair_tails = true;  // run a two-query group's relaxations in one launch
  // svv_query_batch with host outputs: two staging slots and a copy stream
  uint32_t* bstage[2] = {nullptr, nullptr};
  uint64_t bstage_cap = 0;      // words per slot
  std::vector<void*> bstage_bufs;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_done[2] = {}, ev_copied[2] = {};

  // paper's ablations (Table 3): snapshots per relaxation pass (1 = one
  // snapshot at a time, the non-concurrent mode) and stable-vertex pruning
  // (off = every vertex relaxed, the common-graph direct-hop evaluation)
  uint32_t slab_max = svv::kMaxSlab;
  bool prune = true;

  // graph mode: each query's launches captured and replayed as one graph
  bool graph_mode = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphExec_t bgexec = nullptr;  // the last in-order batch, captured
  uint64_t graph_builds = 0, graph_launches = 0;

  // per-type knobs chosen by svv_autotune
  svv::Knobs tuned[4][svv::kLenBuckets] = {};
  bool has_tuned[4][svv::kLenBuckets] = {};

  // batched queries
  svv::BatchPool batch;
  svv::ServeState serve;
  int batch_teams = 0;  // 0: from the graph size
  int batch_mode = 0;   // 0: by graph size, 1: one launch, 2: in order
  int occ_batch = 0;
  cudaEvent_t bev[2] = {};  // span of an in-order batch
  cudaEvent_t gev[3] = {};  // phase timing of the last query group: before, between and after its solves
  bool gev_pending = false;

  // query groups: lane rows of the two bounds, per-lane planar copies, lane
  // words of the partial edges, the group's error word
  uint32_t group_max = svv::kGroupMax;  // queries per group (1 = every query alone)
  // pull threshold of the group solves (intersection, union), % of all units:
  // a group pull round gathers a whole lane row per in-edge, so groups pull later
  uint32_t group_pull_pct[2] = {15, 100};
  bool group_mix = false;  // groups may hold queries of different types
  int occ_group = 0;   // group solves of 4 or 8 lanes
  int occ_group2 = 0;  // of 2 lanes
  bool group_ready = false;
  std::vector<void*> group_bufs;
  uint32_t *gcap = nullptr, *gcup = nullptr, *gnfl = nullptr, *gipl = nullptr, *gerr = nullptr;
  uint32_t* gI[svv::kGroupMax] = {};
  uint32_t* gU[svv::kGroupMax] = {};
  // stream-ordered queries (svv_query_async): a ring of completion events
  // and page-locked status words; the latest one orders later scratch users
  cudaEvent_t aev[svv::kAsyncSlots] = {};
  uint32_t* astatus = nullptr;
  uint64_t anext = 0;
  cudaEvent_t async_last = nullptr;
  // host copy of each vertex's out-degree over edges present in some snapshot
  std::vector<uint32_t> hdeg;
  bool isolated_fast = true;  // answer queries from a source without out-edges by one fill
  uint32_t skip_arrival = 0;  // test hook of the bounded barrier waits (see SolveArgs)
  // bounds the last query's phases read (svv_get_bounds)
  const uint32_t* last_rI = nullptr;
  const uint32_t* last_rU = nullptr;
  const uint32_t* last_row = nullptr;  // its vertex -> relaxation-row map (a pair's second query: the pair arrays')

  svv_stats stats{};
};

namespace svv {

inline svv_status fail(svv_ctx* c, svv_status s, const std::string& msg) {
  // the serving scheduler's failures reach the caller through the request's
  // status; only the caller's own thread writes the message
  if (c && std::this_thread::get_id() != c->worker) c->err = msg;
  return s;
}

inline svv_status cuda_fail(svv_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a launch error where possible
  return fail(c, e == cudaErrorMemoryAllocation ? SVV_ENOMEM : SVV_ECUDA, m);
}

inline uint64_t round256(uint64_t b) { return (b + 255) & ~uint64_t(255); }

inline svv_status dev_alloc(svv_ctx* c, std::vector<void*>& owner, size_t bytes, void** out) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = round256(bytes);
  if (c->budget && c->allocated + bytes > c->budget)
    return fail(c, SVV_ENOMEM,
                "device budget exceeded: need " + std::to_string(c->allocated + bytes) + " of " +
                    std::to_string(c->budget) + " bytes");
  cudaError_t e = cudaMalloc(out, bytes);
  if (e != cudaSuccess) {
    *out = nullptr;
    cudaGetLastError();
    return fail(c, SVV_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  owner.push_back(*out);
  c->allocated += bytes;
  return SVV_OK;
}

template <class T>
svv_status alloc_n(svv_ctx* c, std::vector<void*>& owner, uint64_t n, T** out) {
  return dev_alloc(c, owner, (size_t)n * sizeof(T), reinterpret_cast<void**>(out));
}

inline uint32_t ceil_div(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

// lanes per edge P and snapshots per lane K for a slab of ls snapshots, with
// at most max_p lanes per edge (P*K is the padded row length)
inline void slab_shape_p(uint32_t ls, uint32_t max_p, uint32_t& P, uint32_t& K) {
  uint32_t LP = 8;
  while (LP < ls) LP <<= 1;
  P = std::min(LP, max_p);
  if (LP / P > 8) P = LP / 8;
  K = LP / P;
}

inline void slab_shape(uint32_t ls, uint32_t& P, uint32_t& K) {
  if (ls <= 8) {
    P = 8;
    K = 1;
  } else if (ls <= 16) {
    P = 16;
    K = 1;
  } else if (ls <= 32) {
    P = 32;
    K = 1;
  } else if (ls <= 64) {
    P = 32;
    K = 2;
  } else {
    P = 32;
    K = 4;
  }
}

// host helpers of the query pipeline (svv_api.cu)
struct CompactOut {
  uint32_t* cap_out;
  uint32_t* row_out;
  uint32_t* rows_out;
  uint64_t rows_cap;
};
Knobs default_knobs(const svv_ctx* c, int type);
Knobs knobs_of(const svv_ctx* c, int type, uint32_t L);
LaunchCfg cfg_for(const svv_ctx* c, int occ, int bps);
SolveArgs solve_base(svv_ctx* c, uint32_t wb, uint32_t wl, int type, const Knobs& kn);
svv_status enqueue_query(svv_ctx* c, int t, uint32_t source, uint32_t wb, uint32_t wl, uint32_t* out,
                         cudaStream_t s, bool timing, float* ms_relax_out, float* ms_scatter_out,
                         const CompactOut* co = nullptr);
bool source_is_isolated(const svv_ctx* c, uint32_t source);
svv_status enqueue_isolated(svv_ctx* c, int t, uint32_t source, uint32_t wl, uint32_t* out, cudaStream_t s,
                            bool timing, const CompactOut* co);
svv_status enqueue_tail(svv_ctx* c, int t, uint32_t wb, uint32_t wl, uint32_t* out, const uint32_t* rI,
                        const uint32_t* rU, cudaStream_t s, bool timing, float* ms_relax_out, float* ms_scatter_out,
                        const CompactOut* co, bool fresh);
// the tails of a two-query group (same window length, one slab) with one
// relaxation launch; false in *done when the pair does not qualify
svv_status enqueue_pair_tail(svv_ctx* c, const svv::BatchInstance* inst, uint32_t* const* out,
                             const uint32_t* const* rI, const uint32_t* const* rU, cudaStream_t s, bool* done);
void free_pair(svv_ctx* c);
svv_status ensure_pair_rows(svv_ctx* c, uint32_t LP);  // the pair arrays for rows of LP values

// query groups (svv_group_api.cu): the bounds of up to group_max same-type
// queries from one pair of group solves, then each query's own phases
svv_status ensure_group(svv_ctx* c);
svv_status enqueue_group_bounds(svv_ctx* c, int type, const BatchInstance* inst, uint32_t n, cudaStream_t s);
void free_group(svv_ctx* c);

void free_batch(svv_ctx* c);
void free_serve(svv_ctx* c);
BatchArgs batch_args(svv_ctx* c);
int default_teams(const svv_ctx* c);
svv_status ensure_pool(svv_ctx* c, int want_teams, uint32_t L);
svv_status status_of(uint32_t qerr, uint32_t done);
svv_status check_spec(const svv_ctx* c, const svv_query_spec& q);
bool batch_one_launch(const svv_ctx* c);
svv_status reserve_window(svv_ctx* c, uint32_t L);

// While an in-order server is active it shares the single-query scratch: a
// call that uses that scratch on another stream is ordered after the requests
// already submitted, and the requests submitted later after the call.
struct ServeFence {
  svv_ctx* c;
  cudaStream_t s;
  bool on;
  std::unique_lock<std::mutex> lk;  // the scheduler's queueing lock while the call runs
  ServeFence(svv_ctx* c, cudaStream_t s);
  ~ServeFence();
};
svv_status batch_in_order(svv_ctx* c, const BatchInstance* inst, uint32_t m, const char* host_out,
                          uint32_t* qerr_dev, uint32_t* qerr_host, cudaStream_t s, float* ms);

}  // namespace svv
