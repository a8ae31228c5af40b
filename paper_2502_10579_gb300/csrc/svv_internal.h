// svv_internal.h -- structures shared by the host orchestration and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace svv {

constexpr uint32_t kNone = 0xFFFFFFFFu;  // "no row": the vertex is stable
constexpr uint32_t kInf = 0xFFFFFFFFu;
constexpr uint32_t kSat = 0xFFFFFFFEu;   // SSSP sums saturate here
constexpr int kTypeMixed = 4;            // a query group of several types (group solves only)
// relaxation kinds of a mixed group's lanes: Val(u)+w (SSSP), Val(u)+1 (BFS),
// max(Val(u), w) (SSNP), max(Val(u), ~w) (SSWP on complemented widths)
enum : uint32_t { kKindSum = 0, kKindHop = 1, kKindMax = 2, kKindMaxNot = 3 };

// error codes written by kernels; numerically equal to svv_status values
enum : uint32_t { kErrNone = 0, kErrTimeout = 4, kErrInternal = 7 };

enum Pred : int { kPredAll = 0, kPredAny = 1, kPredBit = 2 };
enum Init : int { kInitSource = 0, kInitSeed = 1 };

// Control block of one team of CTAs (one cooperative launch, or one slice of
// it).  Fields live on separate 128-byte lines so the barrier counter does not
// share a line with the counters that every warp hits.
struct alignas(128) TeamCtl {
  unsigned long long bar_count;  // arrivals since launch (never reset)
  unsigned int pad0[30];
  unsigned long long bar_gen;    // last released barrier | kGenErr
  unsigned int pad1[30];
  unsigned int qn[3];      // frontier sizes, a ring over rounds
  unsigned int pad2[29];
  unsigned int ticket[3];  // work tickets, a ring over rounds
  unsigned int pad3[29];
  unsigned int err;        // kErr* of this team
  unsigned int iters;      // rounds completed
  unsigned int aux[14];    // phase outputs (counts) / per-round best-value ring, see the kernels
  unsigned long long relaxed;  // edges examined (diagnostic)
  unsigned long long pad4[8];
};
static_assert(sizeof(TeamCtl) % 128 == 0, "TeamCtl must be cache-line sized");

// Resident versioned graph (Section 4.1 layout, reordered at load):
// row v holds edges [rp[v], rp[v+1]); the first (rp[v+1]-rp[v]) -
// (nfp[v+1]-nfp[v]) of them are present in all S snapshots and carry no
// mask; the rest ("non-full") have W mask words at nfmask[(nfp[v]+j)*W].
// The non-full edges are also kept as a coordinate list (nfsrc, nfcw) in the
// same order, for the seeding passes.
struct DevGraph {
  uint32_t V, S, W;
  uint32_t E, NF;
  const uint32_t* rp;       // [V+1]
  const uint32_t* nfp;      // [V+1]
  const uint2* cw;          // [E] (target, weight)
  const uint64_t* nfmask;   // [NF*W]
  const uint32_t* nfsrc;    // [NF]
  const uint2* nfcw;        // [NF]
  // Transposed graph for pull rounds, edge-flat (may be absent: ifd ==
  // nullptr).  The E-NF in-edges present in all S snapshots, sorted by
  // target: ifd[i] is the target, ifcw[i] (source, weight).  The NF partial
  // in-edges, sorted by target, in their own arrays with W mask words each
  // at ipmask[k*W].  A pull pass streams both with no row lookups.
  const uint32_t* ifd;      // [E-NF]
  const uint2* ifcw;        // [E-NF]
  const uint32_t* ipd;      // [NF]
  const uint2* ipcw;        // [NF]
  const uint64_t* ipmask;   // [NF*W]
};

struct Window {
  uint32_t b, l;  // snapshots [b, b+l)
};

struct SolveArgs {
  DevGraph g;
  Window win;
  uint32_t bit;      // kPredBit: the snapshot tested
  uint32_t source;
  int init;          // kInit*
  int skip_nf;       // kPredAll over [0,S): non-full edges can never pass
  const uint32_t* base;  // kInitSeed: starting values (the intersection-graph solve)
  uint32_t* val;     // [V] result
  uint32_t* stamp;   // [V] round in which a vertex was last queued
  unsigned long long* q0;  // work units: vertex | chunk << 32
  unsigned long long* q1;
  uint32_t qcap;
  uint32_t cshift;   // edges per unit = 1 << cshift
  TeamCtl* ctl;
  uint32_t* qerr;    // query-wide error word
  uint32_t maxit;
  unsigned long long spin_ns;
  uint32_t delta;    // near-far width: a round relaxes only units within delta
                     // of the frontier's best value (0 = relax every unit)
  unsigned long long* trace;  // optional: per round {frontier units, start ns}
  uint32_t trace_cap;
  // optional: per work chunk, the source value its edges were last relaxed
  // with; a chunk whose vertex still holds that value is skipped (relaxing it
  // again with the same value cannot improve anything).  pcap entries.
  uint32_t* procv;
  uint32_t pcap;
  // direction switch (needs the transposed graph): a round whose frontier
  // holds more than pull_units units runs as a pull pass over every vertex's
  // in-edges; after a pull round that changed more than push_verts vertices the
  // next round pulls again.  0 disables pulling.
  uint32_t pull_units, push_verts;
  // test hook (0 = off): CTA skip_arrival-1 leaves before its first barrier
  // arrival, so the other CTAs' bounded waits expire (SVV_ETIMEOUT)
  uint32_t skip_arrival;
};

struct QrsArgs {
  DevGraph g;
  Window win;
  uint32_t QW;            // mask words per relaxation edge: ceil(win.l / 64)
  int prune;              // 1: only vertices whose bounds differ get rows (the
                          // method); 0: every vertex does (no pruning)
  const uint32_t* rI;     // intersection-graph values
  const uint32_t* rU;     // union-graph values
  uint32_t* row;          // [V] vertex -> row, kNone if stable
  uint32_t* uv;           // [V] row -> vertex
  uint32_t* part;         // [4 * gridDim] per-CTA partial sums
  unsigned long long* units;  // row | chunk << 32 over unstable rows
  uint32_t ucap;
  uint32_t cshift;
  uint32_t* qcnt;         // [2V] per row: (#all-window edges, #other edges)
  uint4* qrow;            // [V] per row: {start, all-window end, mask base, end}
  uint32_t* cur;          // [2V] fill cursors
  uint2* qcw;             // [E] (target row, weight)
  uint64_t* qmask;        // [NF*QW] window-rebased masks
  uint32_t ecap;
  unsigned long long mcap;  // words
  TeamCtl* ctl;           // aux[0]=U, aux[1]=#units, aux[2]=E_Q, aux[3]=#masked
  uint32_t* qerr;
  unsigned long long spin_ns;
  unsigned long long* trace;  // optional: start ns of each of the five passes, then the end
  uint32_t rowcap;        // rows the row arrays hold (uv, qrow; qcnt and cur hold 2 per row)
  // a second query extracted in the same launch (rI1 null: none), same window
  // length: its rows, units, edges and masks follow the first query's; its
  // number of rows goes to counts1_out[0] (aux[0] holds the first query's)
  const uint32_t* rI1;
  const uint32_t* rU1;
  uint32_t* row1;
  Window win1;
  unsigned int* counts1_out;
};

struct RelaxArgs {
  DevGraph g;
  Window win;
  uint32_t s0, ls;        // snapshot slab [win.b+s0, win.b+s0+ls) of this pass
  uint32_t QW;
  const uint32_t* rI;
  const uint32_t* row;
  const uint32_t* uv;
  const uint4* qrow;
  const uint2* qcw;
  const uint64_t* qmask;
  const unsigned int* counts;  // qrs team aux: [0]=U
  // a second query relaxed in the same launch (counts1 null: none): its rows
  // follow the first query's, its subgraph edges point at rows of either
  // range only within its own; same window length and slab
  const unsigned int* counts1;
  const uint32_t* rI1;
  const uint32_t* row1;
  Window win1;
  // a pair of different types (OpMixed): each query's relaxation kind, and
  // bit q set when query q's rows hold complemented values (SSWP)
  uint32_t kind0, kind1, flip;
  uint32_t* val;          // [U * LP]
  uint32_t LP;            // row stride of val (>= ls)
  uint32_t* stamp;        // [V]
  unsigned long long* q0;
  unsigned long long* q1;
  uint32_t qcap;
  uint32_t cshift;
  TeamCtl* ctl;
  uint32_t* qerr;
  uint32_t maxit;
  unsigned long long spin_ns;
  unsigned long long* trace;
  uint32_t trace_cap;
};

// compact output: the relaxed rows of one slab copied to the caller's U x wl
// array (row-major, stride wl)
struct CompactArgs {
  const unsigned int* counts;  // U at [0]
  const uint32_t* val;
  uint32_t LP, s0, ls, wl;
  uint32_t* rows_out;
  unsigned long long rows_cap;  // entries
  uint32_t* qerr;
};

cudaError_t launch_compact(const CompactArgs& a, cudaStream_t s);

// result of a query whose source has no out-edge: out[i*V + v] = src_val if
// v == source else ident for i < L; the same row into rI and rU; row = kNone
struct IsolatedArgs {
  uint32_t V, L, source, ident, src_val;
  uint32_t* out;  // may be null (L = 0)
  uint32_t* rI;
  uint32_t* rU;
  uint32_t* row;
  uint32_t sms;
};

cudaError_t launch_isolated(const IsolatedArgs& a, cudaStream_t s);

struct ScatterArgs {
  uint32_t V;
  uint32_t s0, ls;
  const uint32_t* rI;
  const uint32_t* row;
  const uint32_t* val;
  uint32_t LP;
  uint32_t* out;          // [win.l * V]; rows s0.. of this pass
  const uint32_t* qerr;
  uint32_t rflip;         // XORed into every row value (complemented rows of a mixed pair)
};

// ---------------------------------------------------------------------------
// Batched queries: many (type, source, window) instances in one persistent
// launch whose grid is split into teams.

struct BatchInstance {
  int type;
  uint32_t source, wb, wl;
  uint32_t* out;  // device, wl * V
};

// per-team query scratch (same roles as the single-query scratch)
struct TeamScratch {
  uint32_t *rI, *rU, *stamp, *row, *uv, *part, *qcnt, *cur;
  uint4* qrow;
  uint2* qcw;
  uint64_t* qmask;
  uint32_t* val;
  unsigned long long *q0, *q1, *units;
  uint32_t qcap, ucap, ecap;
  unsigned long long mcap;
  uint32_t* procv;  // per-chunk last-relaxed values (pcap entries)
  uint32_t pcap;
};

constexpr int kBatchCtl = 5;  // per team: barrier, intersection, union, extraction, relaxation

struct BatchArgs {
  DevGraph g;
  const BatchInstance* inst;
  uint32_t n_inst;
  // serving: the host appends instances and raises *live_tail; the kernel
  // waits (bounded) for more work and leaves after idle_ns without any, or
  // when *live_stop is set.  NULL in one-shot batches.
  const volatile uint32_t* live_tail;
  const volatile uint32_t* live_stop;
  unsigned long long idle_ns;
  uint32_t ring;                    // serving: instance i lives in slot i % ring (0 = no ring)
  unsigned* next;                   // instance ticket
  uint32_t* qerr;                   // [capacity] per-instance error words
  volatile uint32_t* done;          // [capacity] 1 when an instance completed (any status)
  unsigned long long* t_start;      // [capacity] device ns
  unsigned long long* t_end;
  const TeamScratch* scratch;       // [teams]
  TeamCtl* ctl;                     // [teams * kBatchCtl]
  uint32_t team_blocks;
  uint32_t solve_cs, relax_cs, qrs_cs;
  uint32_t delta[2];
  uint32_t maxit;                   // 0 = per-instance default
  unsigned long long spin_ns;
  uint32_t pull_units, push_verts;  // direction switch of the solves (0 = push only)
  uint32_t skip_same;               // per-chunk last-relaxed value skip in the solves
};

// ---------------------------------------------------------------------------
// Query groups: the bound solves of up to kGroupMax same-type queries in one
// set of frontier rounds (svv_group.cuh).  Lane k of a group is query k; its
// values sit at val[v * KL + k] (KL = 4 or 8 lanes per row).
constexpr int kGroupMax = 8;

struct GroupArgs {
  DevGraph g;
  uint32_t nlanes;                 // queries in the group (lanes >= nlanes stay inert)
  uint32_t source[kGroupMax];
  int init;                        // kInitSource (intersection) or kInitSeed (union)
  const uint32_t* base;            // kInitSeed: the intersection rows [V * KL]
  uint32_t* val;                   // [V * KL] result rows
  const uint32_t* nflanes;         // [NF] lane word of each partial edge, row order
  const uint32_t* iplanes;         // [NF] lane word of each partial in-edge, transposed order
  uint32_t* stamp;                 // [V]
  unsigned long long* q0;
  unsigned long long* q1;
  uint32_t qcap;
  uint32_t cshift;
  TeamCtl* ctl;
  uint32_t* qerr;
  uint32_t maxit;
  unsigned long long spin_ns;
  uint32_t pull_units, push_verts;  // direction switch, as in SolveArgs
  uint32_t kinds;                   // mixed-type groups: lane k's relaxation kind in bits 2k..2k+1
  unsigned long long* trace;
  uint32_t trace_cap;
};

// lane words of the partial edges: bit k = lane k's window holds the edge in
// every snapshot, bit 16 + k = in at least one
struct LanesArgs {
  DevGraph g;
  uint32_t nlanes;
  Window win[kGroupMax];
  uint32_t* nflanes;
  uint32_t* iplanes;  // may be null (no transposed graph)
};

// per-lane planar copies of the group's bound rows, for the per-query phases
struct SplitArgs {
  uint32_t V, nlanes, KL;
  uint32_t flip;                    // bit k: lane k holds complemented values (SSWP in a mixed group)
  const uint32_t* cap;
  const uint32_t* cup;
  uint32_t* rI[kGroupMax];
  uint32_t* rU[kGroupMax];
};

// launch helpers (defined in the .cu files)
struct LaunchCfg {
  int blocks;     // cooperative grid size
  int threads;
};

cudaError_t launch_group_lanes(const LanesArgs& a, cudaStream_t s);
cudaError_t launch_group_solve(int type, uint32_t KL, int pred, const GroupArgs& a, LaunchCfg cfg, cudaStream_t s);
cudaError_t launch_group_split(const SplitArgs& a, cudaStream_t s);
int occupancy_group(int threads, bool two_lanes);

cudaError_t launch_batch(const BatchArgs& b, LaunchCfg cfg, cudaStream_t s);
int occupancy_batch(int threads);
uint64_t batch_local_bytes(int device);

cudaError_t launch_solve(int type, int pred, const SolveArgs& a, LaunchCfg cfg, cudaStream_t s);
cudaError_t launch_qrs(const QrsArgs& a, LaunchCfg cfg, cudaStream_t s);
cudaError_t launch_relax(int type, uint32_t P, uint32_t K, const RelaxArgs& a, LaunchCfg cfg,
                         cudaStream_t s);
cudaError_t launch_scatter(const ScatterArgs& a, cudaStream_t s);

// occupancy of each cooperative kernel: max resident CTAs per SM at `threads`
int occupancy_solve(int threads);
int occupancy_qrs(int threads);
int occupancy_relax(int threads);

}  // namespace svv
