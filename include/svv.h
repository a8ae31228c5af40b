/*
 * svv.h -- C ABI of libsvv: stable-vertex-value queries over the snapshots of an
 * evolving graph, on one GB300 GPU (sm_103a).
 *
 * The method (arXiv 2502.10579):
 *   Section 3, Step 1 / Algorithm 1: solve the query on the intersection graph
 *     (edges present in every snapshot of the window) and on the union graph
 *     (present in any), giving per-vertex bounds (Theorem 1, Table 1).
 *   Section 3, Step 2 / Theorem 2: a vertex whose two bounds agree is stable:
 *     its value is the same in every snapshot.
 *   Section 3, Step 3-4: drop the in-edges of stable vertices (the Q-relevant
 *     subgraph) and the additions whose sink is stable.
 *   Section 4 / Algorithm 2: relax every snapshot of the window concurrently
 *     over that subgraph, from the intersection-graph values, with one
 *     snapshot-oblivious frontier and a per-edge snapshot-presence bitmask
 *     (Section 4.1, versioned graph).
 * The result equals, bit for bit, a from-scratch solve of every snapshot.
 *
 * Conventions used by every call:
 *   - Vertices are 0..V-1 and exist in every snapshot (Section 2).  The graph is
 *     a multigraph of edge INSTANCES: a re-added edge is a new instance with its
 *     own weight and mask, which gives the minimum-weight reading of Section 3
 *     (maximum for SSWP) without merging.
 *   - Presence masks: W = ceil(S/64) uint64 words per edge, edge-major
 *     (mask[e*W + k]); bit b of word k says the edge is present in snapshot
 *     64k+b, so the least significant bit of word 0 is snapshot 0 (Section 4.1,
 *     version labels).  Bits >= S are ignored.
 *   - Values are uint32.  SSSP: distance, source 0, unreachable 0xFFFFFFFF,
 *     sums saturate at 0xFFFFFFFE.  BFS: hop count, source 0, unreachable
 *     0xFFFFFFFF.  SSWP: width, source 0xFFFFFFFF (+inf), unreachable 0.
 *     SSNP: the smallest possible largest weight on a path, source 0,
 *     unreachable 0xFFFFFFFF (Table 1: bounds as for SSSP).
 *     (Table 2 edge functions; the paper leaves the encodings unstated.)
 *   - Output layout: out[i*V + v] is the value of v in snapshot win_begin+i,
 *     for 0 <= i < win_len (snapshot-major, win_len x V).
 *   - Nothing throws or aborts across this ABI; every call returns a status.
 *     Every device spin-wait is bounded; an expired wait or the iteration cap
 *     returns SVV_ETIMEOUT and the context stays usable.
 *   - A context is not thread-safe: one host thread drives it at a time.
 */
#ifndef SVV_H
#define SVV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct svv_ctx svv_ctx; /* opaque, owned by the library */

typedef enum { SVV_SSSP = 0, SVV_SSWP = 1, SVV_BFS = 2, SVV_SSNP = 3 } svv_type;

typedef enum {
    SVV_OK = 0,
    SVV_EINVAL = 1,      /* bad argument (message via svv_last_error) */
    SVV_ENOMEM = 2,      /* device allocation failed or over the HBM budget */
    SVV_ECUDA = 3,       /* a CUDA call failed */
    SVV_ETIMEOUT = 4,    /* a bounded device wait expired or the iteration cap was hit */
    SVV_EBUSY = 5,       /* serving queue full */
    SVV_ENOTLOADED = 6,  /* no graph loaded */
    SVV_EINTERNAL = 7    /* internal capacity check failed (a library bug) */
} svv_status;

/* One instance of a batched query: the arguments of svv_query plus the status
 * the batch call writes back. */
typedef struct {
    svv_type type;
    uint32_t source, win_begin, win_len;
    uint32_t *out;          /* caller-owned buffer of win_len*V uint32: device memory,
                               or host memory in svv_query_batch (staged copy) */
    svv_status status;      /* written by svv_query_batch */
} svv_query_spec;

/* Per-query diagnostics of the last svv_query / svv_query_plain call. */
typedef struct {
    uint32_t unstable;        /* U: vertices whose bounds differ (Section 3, Step 2) */
    uint32_t qrs_edges;       /* edges of the Q-relevant subgraph kept for relaxation */
    uint32_t qrs_masked;      /* of those, edges not present in every window snapshot */
    uint32_t iters_cap;       /* frontier rounds of the intersection-graph solve */
    uint32_t iters_cup;       /* frontier rounds of the union-graph solve */
    uint32_t iters_relax;     /* frontier rounds of the multi-snapshot relaxation */
    uint32_t iters_plain_max; /* largest round count of a per-snapshot solve */
    uint32_t phase_timing;    /* 1 if the ms_* fields below were measured */
    uint64_t edges_relaxed_cap, edges_relaxed_cup, edges_relaxed_multi;
    /* device time of each phase (CUDA events on the query stream), when the
     * "phase_timing" tuning key is 1: intersection solve, union solve, stable
     * compaction + subgraph extraction, multi-snapshot relaxation, scatter;
     * for svv_query_plain, ms_cap holds the total of the per-snapshot solves */
    float ms_cap, ms_cup, ms_qrs, ms_relax, ms_scatter;
    float ms_batch;           /* device span of the last svv_query_batch (first start to last end) */
    uint32_t batch_teams;     /* teams the last batch ran with */
    uint32_t batch_team_blocks;
    /* device time of the last query group's intersection-graph and union-graph
     * solves in the last in-order svv_query_batch, when "phase_timing" is 1
     * (and "graph" is 0); 0 otherwise */
    float ms_group_cap, ms_group_cup;
} svv_stats;

/* Create a context on CUDA device `device`.  `hbm_budget_bytes` caps the bytes
 * the library allocates on the device (resident graph plus query scratch);
 * 0 means "free memory at load time".  No device memory is allocated here. */
svv_status svv_create(svv_ctx **ctx, int device, uint64_t hbm_budget_bytes);

/* Host-side builder of the versioned union graph (Section 4.1): one edge per
 * instance k with t_add[k] < t_del[k], grouped by source in instance order,
 * mask bit i set iff t_add[k] <= i < t_del[k] (instance live in snapshot i).
 * Inputs are host arrays of n_inst entries; outputs are caller-owned host
 * arrays: row_ptr[V+1], col[n_inst], weight[n_inst], mask[n_inst*ceil(S/64)].
 * *E_out receives the number of edges written.  SVV_EINVAL on src/dst >= V,
 * S == 0 or t_add/t_del > S. */
svv_status svv_build_versioned_csr(uint32_t V, uint32_t S, uint64_t n_inst, const uint32_t *src,
                                   const uint32_t *dst, const uint32_t *w, const uint32_t *t_add,
                                   const uint32_t *t_del, uint64_t *row_ptr, uint32_t *col,
                                   uint32_t *weight, uint64_t *mask, uint64_t *E_out);

/* Load the union CSR with per-edge presence masks (Section 4.1) and keep it
 * resident on the device.  Arrays: row_ptr[V+1] (row_ptr[0]=0, non-decreasing,
 * row_ptr[V]=E), col[E] (< V), weight[E], mask[E*ceil(S/64)] edge-major.  They
 * live on the host, or on the device when inputs_on_device != 0; the library
 * copies them and the caller keeps ownership.  Internally each row is reordered
 * so that edges present in all S snapshots come first (Section 4.1), and edges
 * present in no snapshot are dropped.  Unless the "pull" tuning key is 0, a
 * transposed copy (in-edges sorted by target, 12 bytes per edge plus the masks
 * of partial edges) is kept as well for the solves' pull rounds.  Replaces any
 * graph loaded before.
 * SVV_EINVAL on a malformed CSR, S == 0, V >= 2^32-1 or E >= 2^32;
 * SVV_ENOMEM if the resident graph does not fit the budget. */
svv_status svv_load(svv_ctx *ctx, uint32_t V, uint64_t E, uint32_t S, const uint64_t *row_ptr,
                    const uint32_t *col, const uint32_t *weight, const uint64_t *mask,
                    int inputs_on_device);

/* One query through the intersection-union path (Algorithms 1 and 2):
 * bounds on the window's intersection and union graphs, stable-vertex
 * compaction, Q-relevant subgraph extraction, concurrent relaxation of all
 * window snapshots, and the scatter into `out`.  `out` is a caller-owned
 * DEVICE buffer of win_len*V uint32 (e.g. a torch tensor).  Work is ordered on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream); the call
 * returns after the stream reaches the end of the query, with its status
 * (svv_query_async returns as soon as the work is queued).
 * On failure `out` holds no valid result (a window of more than 128 snapshots
 * is relaxed and written slab by slab, so earlier slabs may have been written).
 * SVV_EINVAL on type, source >= V, win_len == 0 or win_begin+win_len > S. */
svv_status svv_query(svv_ctx *ctx, svv_type type, uint32_t source, uint32_t win_begin,
                     uint32_t win_len, uint32_t *out, void *cuda_stream);

/* svv_query without the host wait: the arguments are checked, the query's
 * kernels are queued on `cuda_stream` and the call returns; *ticket
 * identifies the query.  `out` is written when the stream reaches the end of
 * the query (its status, which only the device knows -- a bounded wait that
 * expired or the round cap -- is read with svv_query_wait).  Queries of one
 * context share its scratch, so the library orders each one after those
 * queued before it (stream waits, no host wait), on any stream; every other
 * call that uses the scratch is ordered after them too.  At most 64 queries
 * are in flight: queuing a 65th first waits for the oldest.  Diagnostics
 * (svv_get_stats) are not recorded for these queries.  SVV_EINVAL as
 * svv_query. */
svv_status svv_query_async(svv_ctx *ctx, svv_type type, uint32_t source, uint32_t win_begin,
                           uint32_t win_len, uint32_t *out, void *cuda_stream, uint64_t *ticket);

/* Status of a query queued by svv_query_async: with wait != 0 the call waits
 * for the query; with wait == 0 it returns SVV_EBUSY while the query runs.
 * A ticket stays valid until 64 later queries have been queued (then
 * SVV_EINVAL). */
svv_status svv_query_wait(svv_ctx *ctx, uint64_t ticket, int wait);

/* Many queries in one call (the instances may mix types, sources and window
 * lengths).  On graphs below 2M vertices the batch runs as ONE persistent
 * launch: the cooperative grid is split into teams of CTAs; each team takes
 * instances from a device work queue and runs the whole intersection-union
 * pipeline of svv_query for each, with its own scratch, so instances overlap
 * on the GPU.  From 2M vertices, where one query's rounds already fill the
 * GPU, the instances run in QUERY GROUPS: up to "group_max" (default 8)
 * instances of one type (of any types with "group_mix"), in arrival order,
 * share one intersection-graph solve
 * and one union-graph solve -- one set of frontier rounds in which every
 * vertex holds one value per member query (a query-oblivious frontier, as
 * Section 4.2 shares one frontier between snapshots), so each round reads
 * each edge once and ends at one barrier for the whole group -- and each
 * member then runs its own stable compaction, subgraph extraction,
 * relaxation and scatter.  Each instance's status is kept on the device and
 * read back once at the end ("batch_mode" tuning key: 0 = by graph size,
 * 1 = one launch, 2 = in order, in groups).
 * A spec's `out` may also be HOST memory (win_len*V uint32): the batch then
 * runs in order, and each such result is computed into one of two device
 * staging slots and copied back on a second stream while the next instance
 * computes; the call returns after the last copy.
 * Each spec is checked as in svv_query; an invalid spec gets SVV_EINVAL and
 * is skipped.  Every valid spec's `out` is written as svv_query would write
 * it, and its status is set (SVV_OK, or SVV_ETIMEOUT for an instance that hit
 * a bounded wait or was not reached because its team stopped).  The call
 * returns after the stream reaches the end of the batch, with SVV_OK if every
 * spec succeeded, else the first failing status.  In one-launch mode the
 * number of teams ("batch_teams" tuning key) is reduced when their scratch
 * would exceed the HBM budget; SVV_ENOMEM if not even one team fits. */
svv_status svv_query_batch(svv_ctx *ctx, uint32_t n, svv_query_spec *specs, void *cuda_stream);

/* ---- Serving: requests that arrive while others run -------------------------
 * svv_serve_start keeps the batch kernel of svv_query_batch running on a
 * library stream as a live server: submitted requests enter a ring in
 * host-mapped memory, an idle team starts each one as soon as it is free, and
 * running requests overlap on the GPU.  The graph, the bitmasks and every
 * team's bound/value state stay resident.  Requests with out == NULL get their
 * output from a device arena of `arena_bytes` (0 = whatever the HBM budget
 * leaves); a request that does not fit is refused with SVV_EBUSY until earlier
 * results are released -- that is the admission control.  The kernel leaves
 * after an idle period and is relaunched by the next svv_submit or svv_poll.
 * That is the mode below 2M vertices.  From 2M vertices ("batch_mode" as set
 * when the server starts: 0 = by graph size, 1 = live kernel, 2 = groups),
 * where one request already fills the GPU, requests run in QUERY GROUPS
 * (continuous batching): a scheduler thread of the library takes the
 * submitted requests in arrival order and, each time the group queued last
 * has finished its bound solves, queues the next group on the library stream
 * -- up to "group_max" pending requests of the oldest request's type, whose
 * intersection- and union-graph solves share one set of frontier rounds
 * (svv_query_batch), then each member's own phases -- framed by one-thread
 * marker launches that write each request's times, status and completion
 * flag to the same mapped memory.  Requests that arrive while a group runs
 * join the next group, so their work overlaps on the device.  A request whose
 * source has no out-edge is answered alone by one fill.  In that mode the
 * server shares svv_query's scratch: svv_query, svv_query_compact,
 * svv_query_plain, svv_query_batch and svv_get_bounds on another stream wait
 * (without blocking the host) for the groups already queued, and the groups
 * queued later wait for them; a request still waiting for its group may run
 * after such a call.
 * max_window bounds win_len; capacity is the number of requests that may be
 * submitted and not yet released.  SVV_ENOMEM if the team scratch (or, in
 * order, the query scratch for max_window) or the arena does not fit the
 * budget. */
svv_status svv_serve_start(svv_ctx *ctx, uint32_t max_window, uint32_t capacity,
                           uint64_t arena_bytes);

/* Queue one request (spec->status is ignored).  *ticket identifies it.
 * SVV_EBUSY when the ring or the arena is full (nothing was queued);
 * SVV_EINVAL as svv_query for bad arguments or win_len > max_window. */
svv_status svv_submit(svv_ctx *ctx, const svv_query_spec *spec, uint64_t *ticket);

/* Completion of a request: returns SVV_OK and sets *result (the request's own
 * status, as svv_query would return it) once it is done; with wait == 0 returns
 * SVV_EBUSY while it is still queued or running; with wait != 0 blocks (bounded
 * by 60 s, then SVV_ETIMEOUT).  Reads host-mapped memory: no CUDA call unless
 * the server must be relaunched. */
svv_status svv_poll(svv_ctx *ctx, uint64_t ticket, int wait, svv_status *result);

/* The device buffer holding a request's output (its own or the arena's) and
 * the device times (ns, %globaltimer) at which it started and finished.
 * Valid until svv_release. */
svv_status svv_ticket_info(svv_ctx *ctx, uint64_t ticket, uint32_t **out,
                           uint64_t *device_start_ns, uint64_t *device_end_ns);

/* Free a finished request's slot and arena space (SVV_EBUSY while running). */
svv_status svv_release(svv_ctx *ctx, uint64_t ticket);

/* Load driver for measurement: serve n requests that arrive at arrival_s[k]
 * seconds after the call starts (non-decreasing), each submitted at its arrival
 * time or, if the server refuses it, as soon as room frees up (arrival order).
 * latency_ms[k] receives completion minus arrival, done_s[k] (may be NULL) the
 * completion time.  Returns when every request is done: SVV_OK, or the first
 * failing request status. */
svv_status svv_serve_replay(svv_ctx *ctx, uint32_t n, const svv_query_spec *specs,
                            const double *arrival_s, double *latency_ms, double *done_s);

/* Stop the server and free its memory (live mode abandons pending requests;
 * in groups, the call first runs the submitted ones and waits for them). */
svv_status svv_serve_stop(svv_ctx *ctx);

/* svv_query without the dense output (the paper keeps one result array per
 * snapshot; this returns what determines them): cap_out[v] = the value of v
 * on the window's intersection graph, row_out[v] = v's row or 0xFFFFFFFF if v
 * is stable, rows_out[r*win_len + i] = the value of the vertex of row r in
 * snapshot win_begin+i.  So value(v, i) = row_out[v] == 0xFFFFFFFF ?
 * cap_out[v] : rows_out[row_out[v]*win_len + i].  All three are caller DEVICE
 * buffers (V, V and rows_cap uint32); *unstable_out (host, may be NULL)
 * receives the number of rows U.  SVV_ENOMEM if rows_cap < U*win_len. */
svv_status svv_query_compact(svv_ctx *ctx, svv_type type, uint32_t source, uint32_t win_begin,
                             uint32_t win_len, uint32_t *cap_out, uint32_t *row_out,
                             uint32_t *rows_out, uint64_t rows_cap, uint32_t *unstable_out,
                             void *cuda_stream);

/* The same query answered the plain way (Fig. 2a): one full solve per window
 * snapshot, each written straight into its row of `out`.  Same arguments and
 * output as svv_query; on failure the rows of `out` are unspecified. */
svv_status svv_query_plain(svv_ctx *ctx, svv_type type, uint32_t source, uint32_t win_begin,
                           uint32_t win_len, uint32_t *out, void *cuda_stream);

/* svv_query with `out_host` a HOST buffer of win_len*V uint32, complete when
 * the call returns.  Page-locked memory the device can address (cudaHostAlloc,
 * cudaHostRegister, torch pin_memory) is written directly by the output
 * scatter over the host link, so the transfer overlaps the scatter; any other
 * host memory goes through a device staging buffer and one copy. */
svv_status svv_query_host(svv_ctx *ctx, svv_type type, uint32_t source, uint32_t win_begin,
                          uint32_t win_len, uint32_t *out_host, void *cuda_stream);

/* Step-level results of the last successful svv_query (or of the last
 * instance of an in-order svv_query_batch), for inspection: the
 * intersection-graph values (Section 3 Step 1, upper bound for SSSP/BFS, lower
 * for SSWP), the union-graph values, and the vertex -> relaxation-row map
 * (0xFFFFFFFF for a stable vertex, Theorem 2).  Each destination is a caller
 * DEVICE buffer of V uint32 and may be NULL.  The copies are ordered on
 * `cuda_stream` and complete before the call returns. */
svv_status svv_get_bounds(svv_ctx *ctx, uint32_t *cap, uint32_t *cup, uint32_t *row,
                          void *cuda_stream);

/* One snapshot's full solve that allocates no memory (the paper has no
 * counterpart: this serves callers that cannot allocate device memory when they
 * call -- code running under an allocator that forbids cudaMalloc, plug-ins
 * whose host owns every allocation, services that reserve all memory up front).
 * Inputs are the caller's DEVICE arrays in the svv_load layout (row_ptr[V+1],
 * col[E], weight[E], mask[E*ceil(S/64)]); `out` is a caller DEVICE array of V
 * uint32 that receives the value of every vertex in snapshot `snapshot` (the
 * same values as row snapshot-win_begin of svv_query_plain).  No context is
 * needed: the call runs on the calling thread's current CUDA device, ordered
 * on `cuda_stream`, and synchronises that stream before it returns, so the
 * result is in `out` when it returns.
 * Types SSSP, SSWP and BFS (SSNP gets SVV_EINVAL).
 * Working memory is a fixed 32 MiB device array inside the library, held by
 * every GPU that loads it until the process exits; a graph whose
 * 4*V + 16*(V + E/64 + 64) bytes (plus 1 KiB) exceed it is rejected with
 * SVV_EINVAL, as are bad arguments and a CSR the kernel finds malformed
 * (row_ptr[0] != 0, a row that goes backwards, row_ptr[V] != E, a target >= V;
 * the kernel checks each before it uses it).  The
 * first call on a device looks up that array's device address
 * (cudaGetSymbolAddress), so make it before any stream capture.  Every call
 * shares the array: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  No cudaMalloc,
 * cudaFree or other allocating call is made. */
svv_status svv_solve_snapshot_noalloc(svv_type type, uint32_t V, uint64_t E, uint32_t S,
                                      const uint64_t *row_ptr, const uint32_t *col,
                                      const uint32_t *weight, const uint64_t *mask,
                                      uint32_t snapshot, uint32_t source, uint32_t *out,
                                      void *cuda_stream);

/* Per-round trace of the last svv_query (needs the "round_trace" tuning key):
 * phase 0 = intersection solve, 1 = union solve, 2 = relaxation (last slab).
 * out[0] = device time (ns, low 40 bits) when round 1 began after
 * initialisation; out[r] for r >= 1 = (frontier units << 40) | start time of
 * round r (ns, low 40 bits); entries past the last round are 0.  `out` is a
 * HOST array of `cap` entries (at most 4096 are written); *n_out receives the
 * number written.  Phase 3 = subgraph extraction: out[0..4] = device time (ns,
 * %globaltimer) at which its five passes began (counts, rows, kept-edge
 * counts, scan, fill), out[5] = when the last CTA finished. */
svv_status svv_get_round_trace(svv_ctx *ctx, uint32_t phase, uint64_t *out, uint32_t cap,
                               uint32_t *n_out);

/* Result of svv_autotune: the knobs chosen for one query type and window-
 * length bucket. */
typedef struct {
    uint32_t solve_chunk, blocks_per_sm, relax_lanes, skip_same;
    uint32_t pull_pct;          /* direction switch of the solves (0 = push only) */
    uint32_t delta;             /* near-far width (SSSP, SSWP; 0 = off) */
    uint32_t slab_max;          /* snapshots relaxed per pass */
    float best_ms, default_ms;  /* probe query time with the chosen and the default knobs */
    uint32_t candidates;        /* configurations timed */
} svv_tune_result;

/* Autotuner: times a probe query (type, source, window), `reps` timed runs per
 * candidate after one warm-up (0 = 3), and keeps the fastest knobs for that
 * query type and window-length bucket (windows of up to 8, 16, 32, 64 and
 * more than 64 snapshots).  The search is coordinate descent from the
 * current defaults, one knob at a time with the others at the best found so
 * far: the pull threshold of the solves' direction switch (0, 5, 10, 15, 25,
 * 40 % of all work units), the near-far width (SSSP: 0, 250, 1000, 4000;
 * SSWP: 0, 50, 200, 800), edges per work unit of the solves (two sizes at or
 * above the loaded one), CTAs per SM (occupancy limit, 2, 3), lanes per edge in
 * the relaxation (32, 16), per-chunk skipping of already-relaxed work (on,
 * off), and for windows over 32 snapshots the slab width (128, 64, 32); a
 * value is kept when it is more than 2% faster.  Later svv_query,
 * svv_query_plain, batch and served queries of the type use the knobs of
 * their bucket (or of the nearest tuned one).  Results are identical for
 * every candidate.  The probe output goes to a library buffer of win_len*V
 * uint32.  `out` may be NULL. */
svv_status svv_autotune(svv_ctx *ctx, svv_type type, uint32_t source, uint32_t win_begin,
                        uint32_t win_len, uint32_t reps, svv_tune_result *out);

/* Tuning knobs, by name: "max_iters" (frontier-round cap per solve, 0 = V+2),
 * "spin_limit_ms" (bound on every device-side wait, default 1000),
 * "solve_chunk" / "relax_chunk" / "qrs_chunk" (edges per work unit, powers of
 * two; defaults 32 / 16 / 32; a chunk smaller than the one the graph was
 * loaded with must be set before svv_load), "blocks_per_sm" (0 = occupancy limit), "delta_sssp" / "delta_sswp"
 * (near-far width of the SSSP / SSWP solves: a frontier round relaxes only the
 * vertices within this distance of the round's best value and keeps the rest
 * queued; 0 relaxes every queued vertex; results are identical either way),
 * "slab_max" (1..128, default 128: snapshots relaxed per pass; 1 evaluates
 * the snapshots one after another over the subgraph, the paper's
 * non-concurrent mode), "prune" (1 default; 0 gives every vertex a row and
 * keeps every edge -- common-graph direct-hop evaluation without the
 * stable-vertex pruning; results are identical),
 * "graph" (1 = svv_query captures its launches into a CUDA graph, updates the
 * instantiated graph in place for the next query of the same shape and
 * replays it; falls back to direct launches where capture is refused; phase
 * timing is not recorded in this mode; an in-order svv_query_batch with
 * device outputs likewise captures all its launches into one graph),
 * "group_max" (1..8, default 8: queries per group of an in-order batch and of
 * the server from 2M vertices; 1 runs every query alone), "group_mix" (0
 * default: a group holds queries of one type; 1: queries of any types share a
 * group, every lane solved in the min lattice with its own relaxation --
 * SSWP lanes on complemented widths, converted back when the bounds are
 * split -- results identical), "pair_tails" (1 default: a two-query group
 * with device outputs whose windows have one length of at most 128 snapshots
 * relaxes both queries in one launch over both queries' rows; 0 relaxes them
 * one after the other; results identical), "group_pull_pct" /
 * "group_pull_pct_union" (0..100, defaults 15 / 100: a group's intersection /
 * union solve pulls when its frontier holds more than this % of all work
 * units; 0 or 100 = push only), "isolated_fast" (1 default: a query whose
 * source has no out-edge in any snapshot is answered by one fill -- the
 * source value at the source, unreachable everywhere else -- instead of the
 * full pipeline; 0 runs the pipeline; results are identical),
 * "test_skip_arrival" (test hook, 0 = off: k+1 makes CTA k of every
 * intersection-graph solve leave before its first barrier arrival, so the
 * other CTAs' bounded waits expire after "spin_limit_ms" and the query
 * returns SVV_ETIMEOUT -- the way to test failure detection without a fault),
 * "batch_teams" (teams of svv_query_batch and the server, 1..64; 0 = by graph
 * size: 8 up to 1M vertices, fewer above, 1 from 8M), "batch_mode" (0 = by
 * graph size, 1 = one launch, 2 = in order; see svv_query_batch), "relax_lanes" (8, 16, 32:
 * lanes per edge in the relaxation), "skip_same" (1 = skip work chunks already
 * relaxed with their vertex's current value), "round_trace" (1 = record, per frontier round of the intersection solve,
 * the union solve and the relaxation, the frontier size and a device
 * timestamp; read with svv_get_round_trace), "phase_timing" (1 = record
 * CUDA events between the phases of each query, reported by svv_get_stats).  SVV_EINVAL on an unknown key
 * or a value out of range. */
svv_status svv_set_tuning(svv_ctx *ctx, const char *key, int64_t value);

/* Diagnostics of the last completed query. */
svv_status svv_get_stats(svv_ctx *ctx, svv_stats *out);

/* Bytes currently allocated on the device by this context. */
uint64_t svv_device_bytes(const svv_ctx *ctx);

/* Human-readable name of a status. */
const char *svv_status_str(svv_status s);

/* Detail of the last error on this context ("" if none). */
const char *svv_last_error(const svv_ctx *ctx);

/* Free every device allocation and the context.  NULL is ignored. */
void svv_destroy(svv_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SVV_H */
