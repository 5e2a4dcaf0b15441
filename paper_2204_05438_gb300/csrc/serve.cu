// Served form: a request loop that meshes a stream of independent meshes with
// continuous batching (no counterpart in the paper).
//
// A server owns a device-memory budget and a set of slots.  A slot is a handle
// with capacity for a size class (power-of-two triangle count c >= 4096, up to
// c / 2 + 2 vertices) whose device state -- inputs, labels, walk and repair
// buffers, output CSR -- stays allocated and is reused by the next request of
// that class.  One worker thread:
//   * admits pending requests in arrival order while a free slot of the right
//     class (or of a class up to 8x larger) exists; otherwise it reserves the
//     budget for a new slot (idle slots of other classes are released to make
//     room) and a second thread creates it, so that the allocations never hold up
//     the requests already on the device; a request whose class alone exceeds the
//     budget fails with POLYLLA_ERR_OOM, and one whose slot cannot be allocated
//     fails with POLYLLA_ERR_OOM when the creation does;
//   * keeps one idle slot ahead of demand: when a request takes the last idle slot
//     that could serve its class, a spare of that class is created in the
//     background if it fits the budget and leaves one slot of the slot limit free;
//   * runs each admitted request on its slot's stream -- host-to-device copy of
//     the inputs, the whole path (polylla_run), a copy of the output counts --
//     so the requests that are admitted together overlap on the device;
//   * when a slot's counts arrive, copies exactly the output CSR to the caller's
//     buffers, and when that lands, completes the request.
// Requests that arrive while others are on the GPU are admitted as soon as a
// slot and memory free up; each is meshed by its own handle, so its result does
// not depend on what else is running.
#include <algorithm>
#include <condition_variable>
#include <chrono>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <utility>
#include <vector>

#include <cuda_runtime.h>
#include <sys/prctl.h>

#include "polylla.h"

namespace {

using Clock = std::chrono::steady_clock;

struct SReq {
  int64_t id = 0;
  const int64_t* xy = nullptr;
  const int32_t* tri = nullptr;
  const int32_t* twin = nullptr;
  int64_t n = 0, m = 0;
  int64_t* off_out = nullptr;
  int32_t* vtx_out = nullptr;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Slot {
  polylla_mesh_t h = nullptr;
  int64_t cls = 0;  // triangle capacity
  int64_t bytes = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  int64_t* pin = nullptr;  // pinned: n_poly, n_vtx, error
  int stage = 0;           // 0 idle, 1 running, 2 copying the result
  SReq req;
  Clock::time_point idle_since;
};

int64_t class_of(int64_t n, int64_t m) {
  int64_t need = m > 2 * n ? m : 2 * n;
  int64_t c = 4096;
  while (c < need) c <<= 1;
  return c;
}

int64_t slot_bytes(int64_t cls) {
  const int64_t b = polylla_mesh_footprint(cls / 2 + 2, cls, 1);
  return b < 0 ? -1 : b + 4096;
}

}  // namespace

struct polylla_server {
  int device = 0;
  int64_t budget = 0;
  int max_slots = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<SReq> pending;
  std::vector<polylla_result> done;
  std::vector<Slot*> slots;
  // slot creation on the creator thread: queued and in-flight creations (size
  // class, the request that waits for it or -1 for a spare), and the requests
  // whose slot could not be allocated
  std::condition_variable cv_create;
  std::deque<std::pair<int64_t, int64_t>> to_create;
  std::vector<std::pair<int64_t, int64_t>> creating;
  std::vector<int64_t> create_failed;
  std::thread creator;
  bool creator_stop = false;  // set once the worker has finished
  int64_t used = 0;
  int64_t next_id = 1;
  int64_t completed = 0;
  int running = 0;
  int peak_running = 0;
  bool stop = false;
  Clock::time_point t0;
  std::thread worker;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void destroy_slot(Slot* s) {
  if (s->h) polylla_mesh_destroy(s->h);
  if (s->ev) cudaEventDestroy(s->ev);
  if (s->s) cudaStreamDestroy(s->s);
  if (s->pin) cudaFreeHost(s->pin);
  delete s;
}

Slot* create_slot(int64_t cls) {
  Slot* s = new (std::nothrow) Slot();
  if (!s) return nullptr;
  s->cls = cls;
  s->bytes = slot_bytes(cls);
  if (polylla_mesh_create_host(cls / 2 + 2, cls, &s->h) != POLYLLA_OK ||
      cudaStreamCreateWithFlags(&s->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&s->pin, 4 * sizeof(int64_t)) != cudaSuccess) {
    destroy_slot(s);
    return nullptr;
  }
  return s;
}

// Enqueue request r on slot s (inputs in, the path, the counts out).
polylla_status start(Slot* s, const SReq& r) {
  int64_t* xy;
  int32_t *tri, *twin;
  polylla_status st = polylla_mesh_set_size(s->h, r.n, r.m);
  if (st == POLYLLA_OK) st = polylla_mesh_inputs(s->h, &xy, &tri, &twin);
  if (st != POLYLLA_OK) return st;
  cudaError_t e = cudaMemcpyAsync(xy, r.xy, sizeof(int64_t) * 2 * r.n, cudaMemcpyHostToDevice, s->s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tri, r.tri, sizeof(int32_t) * 3 * r.m, cudaMemcpyHostToDevice, s->s);
  if (e == cudaSuccess && r.twin)
    e = cudaMemcpyAsync(twin, r.twin, sizeof(int32_t) * 3 * r.m, cudaMemcpyHostToDevice, s->s);
  if (e != cudaSuccess) return POLYLLA_ERR_CUDA;
  if (!r.twin && (st = polylla_mesh_build_twin(s->h, s->s)) != POLYLLA_OK) return st;
  st = polylla_run(s->h, s->s);
  if (st != POLYLLA_OK) return st;
  const int64_t* off;
  const int32_t* vtx;
  const int64_t* counts;
  const int32_t* err;
  st = polylla_get_polygons_async(s->h, &off, &vtx, &counts, &err);
  if (st != POLYLLA_OK) return st;
  s->pin[2] = 0;
  e = cudaMemcpyAsync(s->pin, counts, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s->s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->pin + 2, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s->s);
  if (e == cudaSuccess) e = cudaEventRecord(s->ev, s->s);
  return e == cudaSuccess ? POLYLLA_OK : POLYLLA_ERR_CUDA;
}

void finish(polylla_server* S, Slot* s, int32_t status) {
  polylla_result r{};
  r.id = s->req.id;
  r.status = status;
  r.n_poly = status == POLYLLA_OK ? s->pin[0] : 0;
  r.n_vtx = status == POLYLLA_OK ? s->pin[1] : 0;
  r.submit_s = s->req.t_submit;
  r.admit_s = s->req.t_admit;
  r.done_s = S->now();
  s->stage = 0;
  s->idle_since = Clock::now();
  --S->running;
  ++S->completed;
  S->done.push_back(r);
}

void fail_pending(polylla_server* S, const SReq& q, int32_t status) {
  polylla_result r{};
  r.id = q.id;
  r.status = status;
  r.submit_s = q.t_submit;
  r.admit_s = r.done_s = S->now();
  ++S->completed;
  S->done.push_back(r);
}

// An idle slot that can serve size class cls (its class up to 8x larger).
bool idle_slot_for(const polylla_server* S, int64_t cls) {
  for (const Slot* s : S->slots)
    if (s->stage == 0 && s->cls >= cls && s->cls <= 8 * cls) return true;
  return false;
}

// A queued or in-flight creation of a slot that can serve size class cls.
bool creation_for(const polylla_server* S, int64_t cls) {
  for (const auto& c : S->to_create)
    if (c.first >= cls && c.first <= 8 * cls) return true;
  for (const auto& c : S->creating)
    if (c.first >= cls && c.first <= 8 * cls) return true;
  return false;
}

// The requests on the device whose current stage has ended: the output copy
// started, or the request completed.  Returns whether any moved.
bool poll_running(polylla_server* S) {
  bool moved = false;
  for (Slot* s : S->slots) {
    if (s->stage == 0) continue;
    const cudaError_t q = cudaEventQuery(s->ev);
    if (q == cudaErrorNotReady) continue;
    moved = true;
    if (q != cudaSuccess) {
      finish(S, s, POLYLLA_ERR_CUDA);
      continue;
    }
    if (s->stage == 1) {
      const int32_t code = *reinterpret_cast<const int32_t*>(s->pin + 2);  // the error word
      if (code != 0) {
        finish(S, s, code);
        continue;
      }
      const int64_t* off;
      const int32_t* vtx;
      const int64_t* counts;
      const int32_t* perr;
      cudaError_t e = cudaErrorUnknown;
      if (polylla_get_polygons_async(s->h, &off, &vtx, &counts, &perr) == POLYLLA_OK &&
          s->pin[0] <= s->req.m && s->pin[1] <= 3 * s->req.m) {
        e = cudaMemcpyAsync(s->req.off_out, off, sizeof(int64_t) * (size_t)(s->pin[0] + 1),
                            cudaMemcpyDeviceToHost, s->s);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(s->req.vtx_out, vtx, sizeof(int32_t) * (size_t)s->pin[1],
                              cudaMemcpyDeviceToHost, s->s);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev, s->s);
      }
      if (e != cudaSuccess) {
        finish(S, s, POLYLLA_ERR_CUDA);
        continue;
      }
      s->stage = 2;
    } else {
      finish(S, s, POLYLLA_OK);
    }
  }
  if (moved) S->cv_done.notify_all();
  return moved;
}

// One pass over the slots and the queue; returns whether anything moved.
bool step(polylla_server* S) {
  bool moved = poll_running(S);
  // admissions, in arrival order; the running requests are checked again after
  // each one (enqueuing a request takes tens of microseconds of launches, and a
  // burst of admissions would otherwise hold up every completion behind it)
  while (!S->pending.empty()) {
    const SReq& q = S->pending.front();
    const int64_t cls = class_of(q.n, q.m);
    const int64_t need = slot_bytes(cls);
    if (need < 0 || need > S->budget) {
      fail_pending(S, q, POLYLLA_ERR_OOM);
      S->pending.pop_front();
      S->cv_done.notify_all();
      moved = true;
      continue;
    }
    // an idle slot of the class, else of the smallest larger class up to 8x (a
    // capacity handle serves any smaller mesh): a burst of one class then waits
    // for no slot creation, whose allocations stall the device
    Slot* pick = nullptr;
    for (Slot* s : S->slots)
      if (s->stage == 0 && s->cls >= cls && s->cls <= 8 * cls && (!pick || s->cls < pick->cls))
        pick = s;
    if (!pick) {
      // its slot could not be allocated
      auto failed = std::find(S->create_failed.begin(), S->create_failed.end(), q.id);
      if (failed != S->create_failed.end()) {
        S->create_failed.erase(failed);
        fail_pending(S, q, POLYLLA_ERR_OOM);
        S->pending.pop_front();
        S->cv_done.notify_all();
        moved = true;
        continue;
      }
      // a slot that can serve it is being created: wait for it
      if (creation_for(S, cls)) break;
      // make room: release idle slots of other classes, oldest first
      while ((S->used + need > S->budget ||
              (int)(S->slots.size() + S->creating.size() + S->to_create.size()) >=
                  S->max_slots)) {
        Slot* victim = nullptr;
        size_t vi = 0;
        for (size_t k = 0; k < S->slots.size(); ++k) {
          Slot* s = S->slots[k];
          if (s->stage == 0 && (!victim || s->idle_since < victim->idle_since)) {
            victim = s;
            vi = k;
          }
        }
        if (!victim) break;
        S->used -= victim->bytes;
        S->slots.erase(S->slots.begin() + (long)vi);
        destroy_slot(victim);
      }
      if (S->used + need > S->budget ||
          (int)(S->slots.size() + S->creating.size() + S->to_create.size()) >= S->max_slots)
        break;  // wait
      S->used += need;  // reserved for the slot the creator thread allocates
      S->to_create.emplace_back(cls, q.id);
      S->cv_create.notify_one();
      break;  // wait for it
    }
    pick->req = q;
    pick->req.t_admit = S->now();
    S->pending.pop_front();
    pick->stage = 1;
    ++S->running;
    if (S->running > S->peak_running) S->peak_running = S->running;
    const polylla_status st = start(pick, pick->req);
    if (st != POLYLLA_OK) finish(S, pick, st);
    moved = true;
    poll_running(S);
    // a spare ahead of the next burst of this class, if none is idle or coming
    if (!idle_slot_for(S, cls) && !creation_for(S, cls) && S->used + need <= S->budget &&
        (int)(S->slots.size() + S->creating.size() + S->to_create.size()) + 1 < S->max_slots) {
      S->used += need;
      S->to_create.emplace_back(cls, -1);
      S->cv_create.notify_one();
    }
  }
  return moved;
}

// While requests are on the device the worker checks their events every few
// microseconds: each request passes two device stages (the path, then the copy of
// its result), and the time until the worker notices a stage's end adds to the
// request's latency.  The thread's timer slack is set to 1 us (Linux's default of
// 50 us would stretch every such wait to about 70 us).  With nothing in flight it
// sleeps until a submission wakes it.
constexpr auto kPollBusy = std::chrono::microseconds(4);
constexpr auto kPollIdle = std::chrono::milliseconds(50);

void worker_main(polylla_server* S) {
  cudaSetDevice(S->device);
  prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    const bool moved = step(S);
    if (S->stop && S->pending.empty() && S->running == 0) break;
    if (!moved) S->cv_work.wait_for(lk, S->running > 0 ? kPollBusy : kPollIdle);
  }
  S->cv_done.notify_all();
}

// Creates the slots the worker asks for, outside the server's lock (a slot's
// device and pinned allocations take milliseconds), and hands them over idle.
void creator_main(polylla_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_create.wait(lk, [&] { return S->creator_stop || !S->to_create.empty(); });
    if (S->creator_stop) break;  // the worker is done: no request waits for a slot
    const std::pair<int64_t, int64_t> job = S->to_create.front();
    S->to_create.pop_front();
    S->creating.push_back(job);
    lk.unlock();
    Slot* s = create_slot(job.first);
    lk.lock();
    S->creating.erase(std::find(S->creating.begin(), S->creating.end(), job));
    if (s) {
      s->idle_since = Clock::now();
      S->slots.push_back(s);
    } else {
      S->used -= slot_bytes(job.first);
      if (job.second >= 0) S->create_failed.push_back(job.second);
    }
    S->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

polylla_status polylla_server_create(int64_t budget_bytes, int max_slots, polylla_server_t* out) {
  if (!out) return POLYLLA_ERR_INVALID_ARG;
  *out = nullptr;
  if (budget_bytes < (int64_t)1 << 20 || max_slots < 1 || max_slots > 1024)
    return POLYLLA_ERR_INVALID_ARG;
  polylla_server* S = new (std::nothrow) polylla_server();
  if (!S) return POLYLLA_ERR_OOM;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return POLYLLA_ERR_CUDA;
  }
  S->budget = budget_bytes;
  S->max_slots = max_slots;
  S->t0 = Clock::now();
  try {
    S->creator = std::thread(creator_main, S);
  } catch (...) {
    delete S;
    return POLYLLA_ERR_OOM;
  }
  try {
    S->worker = std::thread(worker_main, S);
  } catch (...) {
    {
      std::lock_guard<std::mutex> g(S->mu);
      S->creator_stop = true;
    }
    S->cv_create.notify_all();
    S->creator.join();
    delete S;
    return POLYLLA_ERR_OOM;
  }
  *out = S;
  return POLYLLA_OK;
}

polylla_status polylla_server_submit(polylla_server_t S, const int64_t* h_xy, int64_t n_vertices,
                                     const int32_t* h_tri, const int32_t* h_twin, int64_t n_tri,
                                     int64_t* h_off_out, int32_t* h_vtx_out, int64_t* id) {
  if (!S || !h_xy || !h_tri || !h_off_out || !h_vtx_out || !id) return POLYLLA_ERR_INVALID_ARG;
  if (n_vertices < 3 || n_tri < 1 || n_vertices >= ((int64_t)1 << 30) ||
      n_tri >= ((int64_t)1 << 29))
    return POLYLLA_ERR_INVALID_ARG;
  SReq r;
  r.xy = h_xy;
  r.tri = h_tri;
  r.twin = h_twin;
  r.n = n_vertices;
  r.m = n_tri;
  r.off_out = h_off_out;
  r.vtx_out = h_vtx_out;
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) return POLYLLA_ERR_STATE;
    r.id = S->next_id++;
    r.t_submit = S->now();
    S->pending.push_back(r);
  }
  S->cv_work.notify_one();
  *id = r.id;
  return POLYLLA_OK;
}

int64_t polylla_server_poll(polylla_server_t S, polylla_result* out, int64_t cap,
                            int64_t wait_us) {
  if (!S || !out || cap < 1) return -1;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->done.empty() && wait_us > 0)
    S->cv_done.wait_for(lk, std::chrono::microseconds(wait_us),
                        [&] { return !S->done.empty(); });
  const int64_t k = (int64_t)S->done.size() < cap ? (int64_t)S->done.size() : cap;
  for (int64_t i = 0; i < k; ++i) out[i] = S->done[(size_t)i];
  S->done.erase(S->done.begin(), S->done.begin() + (long)k);
  return k;
}

polylla_status polylla_server_cancel(polylla_server_t S, int64_t id) {
  if (!S) return POLYLLA_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->pending.begin();
    while (it != S->pending.end() && it->id != id) ++it;
    if (it == S->pending.end()) return POLYLLA_ERR_STATE;  // admitted, done or unknown
    fail_pending(S, *it, POLYLLA_ERR_CANCELLED);
    S->pending.erase(it);
  }
  S->cv_done.notify_all();
  return POLYLLA_OK;
}

polylla_status polylla_server_info(polylla_server_t S, polylla_server_stats* out) {
  if (!S || !out) return POLYLLA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(S->mu);
  out->slots = (int64_t)S->slots.size();
  out->bytes_in_use = S->used;
  out->budget_bytes = S->budget;
  out->pending = (int64_t)S->pending.size();
  out->running = S->running;
  out->peak_running = S->peak_running;
  out->completed = S->completed;
  out->now_s = S->now();
  return POLYLLA_OK;
}

polylla_status polylla_server_destroy(polylla_server_t S) {
  if (!S) return POLYLLA_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();  // every request completed
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->creator_stop = true;
  }
  S->cv_create.notify_all();
  if (S->creator.joinable()) S->creator.join();
  for (Slot* s : S->slots) destroy_slot(s);
  S->slots.clear();
  S->used = 0;
  delete S;
  return POLYLLA_OK;
}

}  // extern "C"
