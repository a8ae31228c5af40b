// svv_serve.cu -- the serving loop: requests arrive while others run.
//
// Two modes, chosen like svv_query_batch's: below 2M vertices the batch
// kernel runs in live mode (below); from 2M vertices, where one request's
// rounds fill the GPU, each request is queued on the library stream as
// svv_query's kernels between two one-thread marker launches that write its
// start time, and its status, end time and completion flag, into the same
// mapped memory the live kernel uses -- so svv_poll and admission are shared.
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

ServeFence::ServeFence(svv_ctx* c_, cudaStream_t s_) : c(c_), s(s_), on(false) {
  ServeState& v = c->serve;
  if (!v.active || !v.in_order || s == v.stream) return;
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
  if (v.in_order) {
    serve_mark_kernel<<<1, 1, 0, v.stream>>>(nullptr, nullptr, nullptr, v.d_t0 + slot);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && (st = enqueue_instance(c, v.h_inst[slot], v.stream)) == SVV_OK) {
      serve_mark_kernel<<<1, 1, 0, v.stream>>>(c->qerr, v.d_qerr + slot, v.d_done + slot, v.d_t1 + slot);
      e = cudaGetLastError();
    }
    if (st || e != cudaSuccess) {
      if (use_arena) arena_free(v, off);
      s = ServeSlot{};
      return st ? st : cuda_fail(c, e, "queueing a request");
    }
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
