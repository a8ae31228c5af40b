// svv_serve.cu -- the serving loop: requests arrive while others run.
//
// Two modes, chosen like svv_query_batch's: below 2M vertices the batch
// kernel runs in live mode (below); from 2M vertices, where one request's
// rounds fill the GPU, requests run in QUERY GROUPS (continuous batching): a
// scheduler thread takes the submitted requests in arrival order and, each
// time the group queued last has finished its bound solves, queues the next
// group -- up to group_max pending requests of the oldest request's type (of
// any type with group_mix) --
// on the server's stream: one pair of group solves for the members' bounds
// (one value lane per request, one set of frontier rounds), then each
// member's own phases.  Requests that arrive while a group runs join the next
// one, so their work overlaps on the device in the shared rounds.  One-thread
// marker launches write each request's start time, status, end time and
// completion flag into mapped memory, so svv_poll and admission are the same
// in both modes.
//
// Live mode: the batch kernel runs on a library stream.  svv_submit writes
// the request into a ring of instances in host-mapped pinned memory and raises
// the tail; an idle team picks it up within microseconds, so requests that
// arrive while others are on the GPU start as soon as a team is free (teams
// are the slots) and overlap with the running ones.  Outputs are carved from a
// device arena sized by the HBM budget: a request that does not fit is refused
// with SVV_EBUSY until earlier results are released (admission by memory).
// The device writes each request's completion flag and timestamps into mapped
// memory, so svv_poll needs no CUDA call.  The kernel leaves after an idle
// period and is relaunched on the next submit or poll.
#include <atomic>
#include <chrono>
#include <cstring>
#include <thread>

#include "svv_ctx.h"
#include "svv_device.cuh"

namespace svv {

// In-order request marker: the start time, or (done != nullptr) the request's
// error word, end time and completion flag.  The flag is written last, after a
// system-scope fence, so a host that sees it sees the rest.
__global__ void serve_mark_kernel(const uint32_t* qerr, uint32_t* qerr_out, uint32_t* done,
                                  unsigned long long* t) {
  if (done) *qerr_out = *reinterpret_cast<const volatile uint32_t*>(qerr);
  *t = global_ns();
  if (done) {
    __threadfence_system();
    *reinterpret_cast<volatile uint32_t*>(done) = 1u;
  }
}

// Groups set this flag when their bound solves are done.
__global__ void serve_flag_kernel(uint32_t* flag) {
  __threadfence_system();
  *reinterpret_cast<volatile uint32_t*>(flag) = 1u;
}

ServeFence::ServeFence(svv_ctx* c_, cudaStream_t s_) : c(c_), s(s_), on(false) {
  // stream-ordered queries still in flight use the same scratch
  if (c->async_last) cudaStreamWaitEvent(s, c->async_last, 0);
  ServeState& v = c->serve;
  if (!v.active || !v.in_order || s == v.stream) return;
  if (v.sched) lk = std::unique_lock<std::mutex>(v.sched->enq);  // no group is queued meanwhile
  if (cudaEventRecord(v.ord, v.stream) == cudaSuccess && cudaStreamWaitEvent(s, v.ord, 0) == cudaSuccess) on = true;
  else cudaStreamSynchronize(v.stream);
}

ServeFence::~ServeFence() {
  if (!on) return;
  ServeState& v = c->serve;
  if (cudaEventRecord(v.ord, s) != cudaSuccess || cudaStreamWaitEvent(v.stream, v.ord, 0) != cudaSuccess)
    cudaStreamSynchronize(s);
}

void free_serve(svv_ctx* c) {
  ServeState& v = c->serve;
  if (v.sched) {
    if (v.sched->th.joinable()) {
      {
        std::lock_guard<std::mutex> g(v.sched->mu);
        v.sched->stop = true;
      }
      v.sched->cv.notify_all();
      v.sched->th.join();
    }
    c->worker = std::thread::id();
    if (v.sched->h_gflag) cudaFreeHost(v.sched->h_gflag);
  }
  if (v.stream) {
    if (v.h_ctrl) {
      reinterpret_cast<volatile uint32_t*>(v.h_ctrl)[1] = 1u;
      std::atomic_thread_fence(std::memory_order_seq_cst);
    }
    cudaStreamSynchronize(v.stream);
  }
  if (v.h_inst) cudaFreeHost(v.h_inst);
  if (v.h_ctrl) cudaFreeHost(v.h_ctrl);
  if (v.h_done) cudaFreeHost(v.h_done);
  if (v.h_qerr) cudaFreeHost(v.h_qerr);
  if (v.h_t0) cudaFreeHost(v.h_t0);
  if (v.h_t1) cudaFreeHost(v.h_t1);
  for (void* b : v.bufs) cudaFree(b);
  c->allocated -= std::min<uint64_t>(c->allocated, v.bytes);
  if (v.ev) cudaEventDestroy(v.ev);
  if (v.ord) cudaEventDestroy(v.ord);
  if (v.stream) cudaStreamDestroy(v.stream);
  v = ServeState{};
}

namespace {

template <class T>
svv_status host_mapped(svv_ctx* c, uint64_t n, T** h, T** d) {
  *h = nullptr;
  *d = nullptr;
  if (cudaHostAlloc((void**)h, n * sizeof(T), cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, SVV_ENOMEM, "cudaHostAlloc (mapped)");
  }
  std::memset(*h, 0, n * sizeof(T));
  if (cudaHostGetDevicePointer((void**)d, *h, 0) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "mapped pointer");
  return SVV_OK;
}

// Queue one group (or one request) on the server's stream.  Members that
// cannot be queued are completed at once with the failure as their status.
void queue_group(svv_ctx* c, const std::vector<uint32_t>& grp) {
  ServeState& v = c->serve;
  ServeSched& S = *v.sched;
  cudaStream_t st = v.stream;
  const uint32_t gslot = (uint32_t)(S.gcount % S.gring);
  reinterpret_cast<volatile uint32_t*>(S.h_gflag)[gslot] = 0u;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  S.gcount++;
  std::vector<bool> marked(grp.size(), false);
  svv_status bad = SVV_OK;
  for (uint32_t slot : grp) serve_mark_kernel<<<1, 1, 0, st>>>(nullptr, nullptr, nullptr, v.d_t0 + slot);
  if (cudaGetLastError() != cudaSuccess) bad = SVV_ECUDA;
  float a = 0.f, b = 0.f;
  if (!bad && grp.size() > 1) {
    BatchInstance gi[kGroupMax];
    for (size_t j = 0; j < grp.size(); ++j) gi[j] = v.h_inst[grp[j]];
    bad = enqueue_group_bounds(c, gi[0].type, gi, (uint32_t)grp.size(), st);
    if (!bad) {
      serve_flag_kernel<<<1, 1, 0, st>>>(S.d_gflag + gslot);
      if (cudaGetLastError() != cudaSuccess) bad = SVV_ECUDA;
    }
    for (size_t j = 0; j < grp.size() && !bad; ++j) {
      const BatchInstance& q = gi[j];
      const uint32_t slot = grp[j];
      if (cudaMemcpyAsync(c->qerr, c->gerr, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        bad = SVV_ECUDA;
        break;
      }
      if ((bad = enqueue_tail(c, q.type, q.wb, q.wl, q.out, c->gI[j], c->gU[j], st, false, &a, &b, nullptr, true)))
        break;
      serve_mark_kernel<<<1, 1, 0, st>>>(c->qerr, v.d_qerr + slot, v.d_done + slot, v.d_t1 + slot);
      if (cudaGetLastError() != cudaSuccess) bad = SVV_ECUDA;
      else marked[j] = true;
    }
    if (!bad) S.grouped += grp.size();
  } else if (!bad) {
    const uint32_t slot = grp[0];
    const BatchInstance& q = v.h_inst[slot];
    bad = enqueue_query(c, q.type, q.source, q.wb, q.wl, q.out, st, false, &a, &b);
    if (!bad) {
      serve_flag_kernel<<<1, 1, 0, st>>>(S.d_gflag + gslot);
      serve_mark_kernel<<<1, 1, 0, st>>>(c->qerr, v.d_qerr + slot, v.d_done + slot, v.d_t1 + slot);
      if (cudaGetLastError() != cudaSuccess) bad = SVV_ECUDA;
      else marked[0] = true;
    }
  }
  if (bad) {
    cudaGetLastError();
    cudaStreamSynchronize(st);  // what was queued has finished; then report the rest
    for (size_t j = 0; j < grp.size(); ++j) {
      if (marked[j]) continue;
      reinterpret_cast<volatile uint32_t*>(v.h_qerr)[grp[j]] = (uint32_t)bad;
      std::atomic_thread_fence(std::memory_order_seq_cst);
      reinterpret_cast<volatile uint32_t*>(v.h_done)[grp[j]] = 1u;
    }
    reinterpret_cast<volatile uint32_t*>(S.h_gflag)[gslot] = 1u;
  }
}

// The scheduler: forms a group whenever the previous one has its bounds.
void sched_loop(svv_ctx* c) {
  ServeState& v = c->serve;
  ServeSched& S = *v.sched;
  cudaSetDevice(c->device);
  std::unique_lock<std::mutex> lk(S.mu);
  for (;;) {
    if (S.pending.empty()) {
      if (S.stop) break;
      S.cv.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    if (S.gcount > 0 && !reinterpret_cast<volatile uint32_t*>(S.h_gflag)[(S.gcount - 1) % S.gring]) {
      // the last group is still solving its bounds: let requests gather
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(10));
      lk.lock();
      continue;
    }
    std::vector<uint32_t> grp;
    const uint32_t first = S.pending.front();
    const BatchInstance q0 = v.h_inst[first];
    if (c->group_max <= 1 || source_is_isolated(c, q0.source)) {
      grp.push_back(first);
      S.pending.pop_front();
    } else {
      for (auto it = S.pending.begin(); it != S.pending.end() && grp.size() < c->group_max;) {
        const BatchInstance& q = v.h_inst[*it];
        if ((c->group_mix || q.type == q0.type) && !source_is_isolated(c, q.source)) {
          grp.push_back(*it);
          it = S.pending.erase(it);
        } else {
          ++it;
        }
      }
    }
    lk.unlock();
    {
      std::lock_guard<std::mutex> g(S.enq);
      queue_group(c, grp);
    }
    lk.lock();
  }
}

svv_status launch_live(svv_ctx* c) {
  ServeState& v = c->serve;
  BatchPool& p = c->batch;
  cudaError_t e = cudaMemsetAsync(p.d_ctl, 0, sizeof(TeamCtl) * kBatchCtl * p.teams, v.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "serve setup");
  BatchArgs b = batch_args(c);
  b.inst = v.d_inst;
  b.n_inst = 0;
  b.ring = v.cap;
  b.live_tail = v.d_ctrl;
  b.live_stop = v.d_ctrl + 1;
  b.idle_ns = v.idle_ns;
  b.next = v.d_next;
  b.qerr = v.d_qerr;
  b.done = v.d_done;
  b.t_start = v.d_t0;
  b.t_end = v.d_t1;
  if ((e = launch_batch(b, LaunchCfg{p.teams * (int)p.team_blocks, 512}, v.stream)) != cudaSuccess)
    return cuda_fail(c, e, "launch serving kernel");
  if ((e = cudaEventRecord(v.ev, v.stream)) != cudaSuccess) return cuda_fail(c, e, "serve event");
  v.launched = true;
  v.launches++;
  return SVV_OK;
}

// relaunch the live kernel if it has left while requests are waiting
svv_status ensure_running(svv_ctx* c) {
  ServeState& v = c->serve;
  if (v.in_order) return SVV_OK;  // every request was queued when submitted
  if (!v.launched) return launch_live(c);
  const cudaError_t q = cudaEventQuery(v.ev);
  if (q == cudaErrorNotReady) return SVV_OK;
  if (q != cudaSuccess) return cuda_fail(c, q, "serving kernel");
  unsigned next = 0;
  cudaError_t e = cudaMemcpyAsync(&next, v.d_next, sizeof(unsigned), cudaMemcpyDeviceToHost, v.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "serving kernel state");
  if ((uint64_t)next < v.tail) return launch_live(c);
  return SVV_OK;
}

// Ring allocation in the arena.  Allocations are kept in order; the free
// space is after the newest one (up to the end, or up to the oldest live one
// once the ring has wrapped) and, before wrapping, at the start.
void arena_trim(ServeState& v) {
  while (!v.allocs.empty() && v.allocs.front().freed) v.allocs.pop_front();
  if (v.allocs.empty()) v.a_end = 0;
}

bool arena_alloc(ServeState& v, uint64_t size, uint64_t* off) {
  size = round256(size);
  arena_trim(v);
  uint64_t at;
  if (v.allocs.empty()) {
    if (size > v.arena_bytes) return false;
    at = 0;
  } else {
    const uint64_t head = v.allocs.front().off;
    if (v.a_end > head) {  // not wrapped: [a_end, end) then [0, head)
      if (v.a_end + size <= v.arena_bytes) at = v.a_end;
      else if (size <= head) at = 0;
      else return false;
    } else {  // wrapped: [a_end, head)
      if (v.a_end + size <= head) at = v.a_end;
      else return false;
    }
  }
  v.allocs.push_back(ServeState::Alloc{at, size, false});
  v.a_end = at + size;
  *off = at;
  return true;
}

void arena_free(ServeState& v, uint64_t off) {
  for (auto& a : v.allocs)
    if (a.off == off && !a.freed) {
      a.freed = true;
      break;
    }
  arena_trim(v);
}

ServeSlot* slot_of(svv_ctx* c, uint64_t ticket) {
  ServeState& v = c->serve;
  if (!v.active || ticket >= v.tail) return nullptr;
  ServeSlot& s = v.slots[ticket % v.cap];
  return (s.busy && s.ticket == ticket) ? &s : nullptr;
}

}  // namespace
}  // namespace svv

using namespace svv;

extern "C" {

svv_status svv_serve_start(svv_ctx* c, uint32_t max_window, uint32_t capacity, uint64_t arena_bytes) {
  if (!c) return SVV_EINVAL;
  if (!c->loaded) return fail(c, SVV_ENOTLOADED, "no graph loaded");
  if (c->serve.active) return fail(c, SVV_EINVAL, "serving already started");
  if (max_window == 0 || max_window > c->g.S) return fail(c, SVV_EINVAL, "max_window must be in [1, S]");
  if (capacity == 0 || capacity > (1u << 24)) return fail(c, SVV_EINVAL, "capacity must be in [1, 2^24]");
  DeviceGuard dg(c->device);
  ServeState& v = c->serve;
  v.in_order = !batch_one_launch(c);
  svv_status st = v.in_order ? reserve_window(c, max_window) : ensure_pool(c, default_teams(c), max_window);
  if (!st && v.in_order) st = ensure_group(c);
  if (st) return st;
  v.cap = capacity;
  v.maxL = max_window;
  if ((st = host_mapped(c, capacity, &v.h_inst, &v.d_inst)) || (st = host_mapped(c, 2, &v.h_ctrl, &v.d_ctrl)) ||
      (st = host_mapped(c, capacity, &v.h_done, &v.d_done)) || (st = host_mapped(c, capacity, &v.h_qerr, &v.d_qerr)) ||
      (st = host_mapped(c, capacity, &v.h_t0, &v.d_t0)) || (st = host_mapped(c, capacity, &v.h_t1, &v.d_t1))) {
    free_serve(c);
    return st;
  }
  const uint64_t before = c->allocated;
  if ((st = alloc_n(c, v.bufs, 1, &v.d_next))) {
    free_serve(c);
    return st;
  }
  if (arena_bytes == 0) {
    const uint64_t room = c->budget > c->allocated ? c->budget - c->allocated : 0;
    arena_bytes = room > (256ull << 20) ? room - (256ull << 20) : 0;
  }
  if (arena_bytes == 0 || (st = alloc_n(c, v.bufs, arena_bytes, &v.arena))) {
    free_serve(c);
    return st ? st : fail(c, SVV_ENOMEM, "no room for the serving output arena");
  }
  v.arena_bytes = arena_bytes;
  v.bytes = c->allocated - before;
  cudaError_t e = cudaMemset(v.d_next, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&v.stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v.ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v.ord, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_serve(c);
    return cuda_fail(c, e, "serve start");
  }
  v.slots.assign(capacity, ServeSlot{});
  if (v.in_order) {
    v.sched.reset(new (std::nothrow) ServeSched());
    if (!v.sched) {
      free_serve(c);
      return fail(c, SVV_ENOMEM, "serving scheduler");
    }
    if ((st = host_mapped(c, v.sched->gring, &v.sched->h_gflag, &v.sched->d_gflag))) {
      free_serve(c);
      return st;
    }
    v.active = true;
    try {
      v.sched->th = std::thread(sched_loop, c);
    } catch (...) {
      free_serve(c);
      return fail(c, SVV_ENOMEM, "could not start the serving scheduler");
    }
    c->worker = v.sched->th.get_id();
  }
  v.active = true;
  c->err.clear();
  return SVV_OK;
}

svv_status svv_submit(svv_ctx* c, const svv_query_spec* spec, uint64_t* ticket) {
  if (!c || !spec || !ticket) return SVV_EINVAL;
  ServeState& v = c->serve;
  if (!v.active) return fail(c, SVV_EINVAL, "serving not started");
  svv_query_spec q = *spec;
  const bool use_arena = q.out == nullptr;
  if (use_arena) q.out = reinterpret_cast<uint32_t*>(v.arena);  // placeholder for the check
  svv_status st = check_spec(c, q);
  if (st) return fail(c, st, "bad request");
  if (q.win_len > v.maxL) return fail(c, SVV_EINVAL, "window longer than the serving maximum");
  ServeSlot& s = v.slots[v.tail % v.cap];
  if (s.busy) return fail(c, SVV_EBUSY, "request ring full: release finished requests");
  uint64_t off = 0;
  if (use_arena) {
    if (!arena_alloc(v, (uint64_t)q.win_len * c->g.V * 4, &off))
      return fail(c, SVV_EBUSY, "output arena full: release finished requests");
    q.out = reinterpret_cast<uint32_t*>(v.arena + off);
  }
  DeviceGuard dg(c->device);
  const uint32_t slot = (uint32_t)(v.tail % v.cap);
  s = ServeSlot{v.tail, true, use_arena, off, (uint64_t)q.win_len * c->g.V * 4, q.out};
  v.h_inst[slot] = BatchInstance{(int)q.type, q.source, q.win_begin, q.win_len, q.out};
  reinterpret_cast<volatile uint32_t*>(v.h_qerr)[slot] = 0u;
  reinterpret_cast<volatile uint32_t*>(v.h_done)[slot] = 0u;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  if (v.in_order) {  // the scheduler queues it with the next group
    {
      std::lock_guard<std::mutex> g(v.sched->mu);
      v.sched->pending.push_back(slot);
    }
    v.sched->cv.notify_one();
    *ticket = v.tail++;
    c->err.clear();
    return SVV_OK;
  }
  *ticket = v.tail;
  v.tail++;
  reinterpret_cast<volatile uint32_t*>(v.h_ctrl)[0] = (uint32_t)v.tail;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  return ensure_running(c);
}

svv_status svv_poll(svv_ctx* c, uint64_t ticket, int wait, svv_status* result) {
  if (!c || !result) return SVV_EINVAL;
  ServeSlot* s = slot_of(c, ticket);
  if (!s) return fail(c, SVV_EINVAL, "unknown or released ticket");
  ServeState& v = c->serve;
  const uint32_t slot = (uint32_t)(ticket % v.cap);
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    if (reinterpret_cast<volatile uint32_t*>(v.h_done)[slot]) {
      std::atomic_thread_fence(std::memory_order_acquire);
      *result = status_of(reinterpret_cast<volatile uint32_t*>(v.h_qerr)[slot], 1u);
      return SVV_OK;
    }
    DeviceGuard dg(c->device);
    svv_status st = ensure_running(c);
    if (st) return st;
    if (!wait) return SVV_EBUSY;
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60))
      return fail(c, SVV_ETIMEOUT, "request did not complete within 60 s");
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

svv_status svv_ticket_info(svv_ctx* c, uint64_t ticket, uint32_t** out, uint64_t* device_start_ns,
                           uint64_t* device_end_ns) {
  if (!c) return SVV_EINVAL;
  ServeSlot* s = slot_of(c, ticket);
  if (!s) return fail(c, SVV_EINVAL, "unknown or released ticket");
  ServeState& v = c->serve;
  const uint32_t slot = (uint32_t)(ticket % v.cap);
  if (out) *out = s->out;
  if (device_start_ns) *device_start_ns = reinterpret_cast<volatile unsigned long long*>(v.h_t0)[slot];
  if (device_end_ns) *device_end_ns = reinterpret_cast<volatile unsigned long long*>(v.h_t1)[slot];
  return SVV_OK;
}

svv_status svv_release(svv_ctx* c, uint64_t ticket) {
  if (!c) return SVV_EINVAL;
  ServeSlot* s = slot_of(c, ticket);
  if (!s) return fail(c, SVV_EINVAL, "unknown or released ticket");
  ServeState& v = c->serve;
  if (!reinterpret_cast<volatile uint32_t*>(v.h_done)[ticket % v.cap])
    return fail(c, SVV_EBUSY, "request still running");
  if (s->arena) arena_free(v, s->off);
  *s = ServeSlot{};
  return SVV_OK;
}

svv_status svv_serve_replay(svv_ctx* c, uint32_t n, const svv_query_spec* specs, const double* arrival_s,
                            double* latency_ms, double* done_s) {
  if (!c || (n && (!specs || !arrival_s || !latency_ms))) return SVV_EINVAL;
  ServeState& v = c->serve;
  if (!v.active) return fail(c, SVV_EINVAL, "serving not started");
  using clk = std::chrono::steady_clock;
  std::vector<uint64_t> ticket(n, 0);
  std::vector<uint8_t> state(n, 0);  // 0 waiting, 1 submitted, 2 done
  std::deque<uint32_t> inflight;     // submitted, in submission order
  uint32_t next_arrival = 0, ndone = 0;
  svv_status worst = SVV_OK;
  const auto t0 = clk::now();
  auto now_s = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
  std::deque<uint32_t> arrived;  // arrived, not yet admitted
  while (ndone < n) {
    const double t = now_s();
    while (next_arrival < n && arrival_s[next_arrival] <= t) arrived.push_back(next_arrival++);
    // admit in arrival order while there is room
    while (!arrived.empty()) {
      const uint32_t k = arrived.front();
      uint64_t tk = 0;
      svv_status st = svv_submit(c, &specs[k], &tk);
      if (st == SVV_EBUSY) break;
      if (st) return st;
      ticket[k] = tk;
      state[k] = 1;
      inflight.push_back(k);
      arrived.pop_front();
    }
    // completions (device flags in mapped memory)
    bool any = false;
    for (auto it = inflight.begin(); it != inflight.end();) {
      const uint32_t k = *it;
      const uint32_t slot = (uint32_t)(ticket[k] % v.cap);
      if (reinterpret_cast<volatile uint32_t*>(v.h_done)[slot]) {
        std::atomic_thread_fence(std::memory_order_acquire);
        const double td = now_s();
        latency_ms[k] = 1e3 * (td - arrival_s[k]);
        if (done_s) done_s[k] = td;
        const svv_status rs = status_of(reinterpret_cast<volatile uint32_t*>(v.h_qerr)[slot], 1u);
        if (rs && !worst) worst = rs;
        svv_release(c, ticket[k]);
        state[k] = 2;
        ndone++;
        it = inflight.erase(it);
        any = true;
      } else {
        ++it;
      }
    }
    if (!any && !inflight.empty()) {
      DeviceGuard dg(c->device);
      svv_status st = ensure_running(c);
      if (st) return st;
    }
    if (now_s() > (n ? arrival_s[n - 1] : 0.0) + 600.0) return fail(c, SVV_ETIMEOUT, "replay did not finish");
  }
  return worst;
}

svv_status svv_serve_stop(svv_ctx* c) {
  if (!c) return SVV_EINVAL;
  if (!c->serve.active) return SVV_OK;
  DeviceGuard dg(c->device);
  free_serve(c);
  return SVV_OK;
}

}  // extern "C"
