// Serving runtime: time frames of different sizes arrive from host memory,
// are admitted when a slot (stream + tracking context) and room in the
// caller's device-memory budget are free, run concurrently on the device, and
// release their scratch the moment they finish, so frames that arrive while
// others run are admitted as resources free up (continuous batching).  The
// paper's source-side rate control (Section 3) throttles by the amount of data
// in flight; here the in-flight limit is the device-memory budget itself.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tpct_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over one device range, free blocks coalesced; offsets
// and sizes are multiples of 256 bytes.
class Arena {
 public:
  Arena(size_t bytes) : total_(bytes / 256 * 256) {
    if (total_) free_[0] = total_;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    if (bytes == 0) bytes = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        if (used_ > peak_) peak_ = used_;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    if (bytes == 0) bytes = 256;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t total() const { return total_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t total_ = 0, used_ = 0, peak_ = 0;
};

enum FrameState { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Frame {
  tpct_host_frame src{};
  FrameState state = kQueued;
  tpct_status status = TPCT_OK;
  int slot = -1;
  size_t off_scratch = 0, bytes_scratch = 0, off_out = 0, bytes_out = 0;
  int32_t cap_tracks = 0, cap_ids = 0;
  tpct_tracks_out out{};
  int32_t counts[2] = {0, 0};
  bool retried = false;
  Clock::time_point t_submit, t_start, t_done;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  tpct_ctx* ctx = nullptr;
  int32_t* counts = nullptr;   // pinned host [2]: n_tracks, n_ids of the running frame
  uint64_t ticket = 0;          // 0: idle
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

struct tpct_server {
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  char* base = nullptr;
  Arena arena{0};
  std::vector<Slot> slots;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Frame> frames;
  uint64_t next_ticket = 1;
  cudaStream_t copy_stream = nullptr;
  int device = 0;
  tpct_server_stats stats{};
  tpct_status fatal = TPCT_OK;
};

namespace {

// Device bytes a frame needs: its inputs and workspace (released when the
// frame finishes) and its outputs (released by tpct_server_release).
void frame_bytes(tpct_ctx* ctx, const tpct_host_frame& f, int32_t cap_tracks, int32_t cap_ids,
                 size_t* scratch, size_t* out) {
  const size_t n = (size_t)f.n;
  size_t in = align256(n * 4) * 3 + align256(n * 2) + align256(n) + align256(8 * (size_t)(f.n_instances + 1));
  *scratch = in + align256(tpct_workspace_bytes(ctx, f.n, f.n_instances));
  *out = align256(8) + 5 * align256(4 * (size_t)cap_tracks) + 2 * align256(8 * (size_t)cap_tracks) +
         align256(40 * (size_t)cap_tracks) + align256(120 * (size_t)cap_tracks) + align256(4 * (size_t)cap_ids);
}

// Enqueue one admitted frame on its slot: copies in, tracking, done event.
tpct_status launch_frame(tpct_server* S, uint64_t ticket, Frame& F) {
  Slot& sl = S->slots[F.slot];
  char* p = S->base + F.off_scratch;
  const tpct_host_frame& f = F.src;
  const size_t n = (size_t)f.n;
  auto take = [&](size_t b) { char* q = p; p += align256(b); return q; };
  float* x = (float*)take(n * 4);
  float* y = (float*)take(n * 4);
  float* z = (float*)take(n * 4);
  uint16_t* ch = (uint16_t*)take(n * 2);
  uint8_t* row = (uint8_t*)take(n);
  int64_t* offs = (int64_t*)take(8 * (size_t)(f.n_instances + 1));
  char* ws = p;
  const size_t ws_bytes = tpct_workspace_bytes(sl.ctx, f.n, f.n_instances);
  cudaStream_t s = sl.stream;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t b) {
    if (e == cudaSuccess && src && b) e = cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, s);
  };
  cp(x, f.x, n * 4);
  cp(y, f.y, n * 4);
  cp(z, f.z, n * 4);
  cp(ch, f.charge, n * 2);
  cp(row, f.row, n);
  cp(offs, f.sector_offsets, 8 * (size_t)(f.n_instances + 1));
  if (e != cudaSuccess) return TPCT_E_CUDA;
  tpct_status st = tpct_set_workspace(sl.ctx, ws, ws_bytes, f.n, f.n_instances);
  if (st != TPCT_OK) return st;
  // outputs
  char* o = S->base + F.off_out;
  auto takeo = [&](size_t b) { char* q = o; o += align256(b); return q; };
  tpct_tracks_out& out = F.out;
  out.capacity_tracks = F.cap_tracks;
  out.capacity_ids = F.cap_ids;
  out.n_tracks = (int32_t*)takeo(8);
  out.n_ids = out.n_tracks + 1;
  out.instance = (int32_t*)takeo(4 * (size_t)F.cap_tracks);
  out.n_cl = (int32_t*)takeo(4 * (size_t)F.cap_tracks);
  out.offset = (int32_t*)takeo(4 * (size_t)F.cap_tracks);
  out.ndf = (int32_t*)takeo(4 * (size_t)F.cap_tracks);
  out.status = (int32_t*)takeo(4 * (size_t)F.cap_tracks);
  out.x_ref = (double*)takeo(8 * (size_t)F.cap_tracks);
  out.chi2 = (double*)takeo(8 * (size_t)F.cap_tracks);
  out.param = (double*)takeo(40 * (size_t)F.cap_tracks);
  out.cov = (double*)takeo(120 * (size_t)F.cap_tracks);
  out.cluster_ids = (int32_t*)takeo(4 * (size_t)F.cap_ids);
  tpct_clusters cl{};
  cl.x = x; cl.y = y; cl.z = z; cl.charge = f.charge ? ch : nullptr; cl.row = f.row ? row : nullptr;
  cl.sector_offsets = offs;
  cl.n_instances = f.n_instances;
  st = tpct_track(sl.ctx, &cl, f.n, &out, (tpct_stream)s);
  if (st != TPCT_OK) return st;
  e = cudaMemcpyAsync(sl.counts, out.n_tracks, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, s);
  return e == cudaSuccess ? TPCT_OK : TPCT_E_CUDA;
}

// One scheduler pass (caller holds the lock): retire finished frames, then
// admit queued frames in arrival order while a slot and memory are free.
void schedule(tpct_server* S) {
  for (size_t i = 0; i < S->slots.size(); ++i) {
    Slot& sl = S->slots[i];
    if (!sl.ticket) continue;
    cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    Frame& F = S->frames[sl.ticket];
    F.t_done = Clock::now();
    F.counts[0] = sl.counts[0];
    F.counts[1] = sl.counts[1];
    S->arena.release(F.off_scratch, F.bytes_scratch);
    F.bytes_scratch = 0;
    if (q != cudaSuccess) {
      F.state = kFailed;
      F.status = TPCT_E_CUDA;
    } else if ((F.counts[0] > F.cap_tracks || F.counts[1] > F.cap_ids) && !F.retried) {
      // outputs overflowed the planned capacity: run again with the exact bound
      S->arena.release(F.off_out, F.bytes_out);
      F.retried = true;
      F.cap_tracks = (int32_t)(F.src.n / 3 + 1);
      F.cap_ids = (int32_t)F.src.n;
      F.state = kQueued;
      S->queue.push_front(sl.ticket);
      S->stats.retries++;
    } else {
      F.state = (F.counts[0] > F.cap_tracks || F.counts[1] > F.cap_ids) ? kFailed : kDone;
      F.status = F.state == kDone ? TPCT_OK : TPCT_E_CAPACITY;
      S->stats.completed++;
      S->stats.clusters_completed += F.src.n;
    }
    sl.ticket = 0;
  }
  while (!S->queue.empty()) {
    int free_slot = -1;
    for (size_t i = 0; i < S->slots.size(); ++i)
      if (!S->slots[i].ticket) { free_slot = (int)i; break; }
    if (free_slot < 0) break;
    const uint64_t tk = S->queue.front();
    Frame& F = S->frames[tk];
    size_t sb, ob;
    frame_bytes(S->slots[free_slot].ctx, F.src, F.cap_tracks, F.cap_ids, &sb, &ob);
    size_t so, oo;
    if (!S->arena.alloc(sb, &so)) break;   // FIFO: wait until memory frees up
    if (!S->arena.alloc(ob, &oo)) { S->arena.release(so, sb); break; }
    S->queue.pop_front();
    F.off_scratch = so; F.bytes_scratch = sb; F.off_out = oo; F.bytes_out = ob;
    F.slot = free_slot;
    F.state = kRunning;
    F.t_start = Clock::now();
    S->slots[free_slot].ticket = tk;
    const tpct_status st = launch_frame(S, tk, F);
    if (st != TPCT_OK) {
      // host-detected failure: free everything, report on the ticket
      S->arena.release(so, sb); S->arena.release(oo, ob);
      F.bytes_scratch = F.bytes_out = 0;
      F.state = kFailed;
      F.status = st;
      S->slots[free_slot].ticket = 0;
    }
    int running = 0;
    for (auto& s2 : S->slots) running += s2.ticket != 0;
    if (running > S->stats.peak_in_flight) S->stats.peak_in_flight = running;
  }
  S->stats.queued = (int32_t)S->queue.size();
  S->stats.bytes_in_use = S->arena.used();
  S->stats.peak_bytes = S->arena.peak();
}

void worker_loop(tpct_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lock(S->mu);
  while (!S->stop) {
    schedule(S);
    bool busy = false;
    for (auto& sl : S->slots) busy |= sl.ticket != 0;
    if (busy) S->cv.wait_for(lock, std::chrono::microseconds(50));
    else S->cv.wait_for(lock, std::chrono::milliseconds(5));
  }
}

}  // namespace

extern "C" {

tpct_status tpct_server_create(const tpct_geometry* g, double bz, const tpct_cuts* cuts, tpct_precision prec,
                               const tpct_server_config* cfg, tpct_server** out) {
  if (!g || !cuts || !cfg || !out || cfg->n_slots < 1 || cfg->n_slots > 64 || !cfg->arena ||
      ((uintptr_t)cfg->arena % 256) || cfg->arena_bytes < 4096)
    return TPCT_E_INVALID;
  tpct_server* S = new (std::nothrow) tpct_server();
  if (!S) return TPCT_E_NOMEM;
  S->base = (char*)cfg->arena;
  S->arena = Arena(cfg->arena_bytes);
  if (cudaGetDevice(&S->device) != cudaSuccess) { delete S; return TPCT_E_CUDA; }
  S->slots.resize(cfg->n_slots);
  tpct_status st = TPCT_OK;
  for (auto& sl : S->slots) {
    if (st == TPCT_OK) st = tpct_create(g, bz, cuts, prec, &sl.ctx);
    if (st == TPCT_OK && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) st = TPCT_E_CUDA;
    if (st == TPCT_OK && cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) st = TPCT_E_CUDA;
    if (st == TPCT_OK && cudaHostAlloc((void**)&sl.counts, 8, cudaHostAllocDefault) != cudaSuccess) st = TPCT_E_CUDA;
  }
  if (st == TPCT_OK && cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
    st = TPCT_E_CUDA;
  if (st != TPCT_OK) { tpct_server_destroy(S); return st; }
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return TPCT_OK;
}

void tpct_server_destroy(tpct_server* S) {
  if (!S) return;
  if (S->worker.joinable()) {
    { std::lock_guard<std::mutex> l(S->mu); S->stop = true; }
    S->cv.notify_all();
    S->worker.join();
  }
  for (auto& sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ctx) tpct_destroy(sl.ctx);
    if (sl.counts) cudaFreeHost(sl.counts);
  }
  if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
  delete S;
}

tpct_status tpct_server_submit(tpct_server* S, const tpct_host_frame* f, uint64_t* ticket) {
  if (!S || !f || !ticket || f->n < 0 || f->n_instances < 1 || !f->sector_offsets) return TPCT_E_INVALID;
  if (f->n > 0 && (!f->y || !f->z || (!f->row && !f->x))) return TPCT_E_INVALID;
  if (f->n > INT32_MAX / 4) return TPCT_E_BUDGET;
  Frame F;
  F.src = *f;
  F.cap_tracks = (int32_t)(f->n / 16 + 1024);
  F.cap_ids = (int32_t)f->n;
  size_t sb, ob, sb_max, ob_max;
  frame_bytes(S->slots[0].ctx, *f, F.cap_tracks, F.cap_ids, &sb, &ob);
  frame_bytes(S->slots[0].ctx, *f, (int32_t)(f->n / 3 + 1), (int32_t)f->n, &sb_max, &ob_max);
  if (sb_max + ob_max > S->arena.total()) return TPCT_E_BUDGET;   // can never be admitted
  F.t_submit = Clock::now();
  std::lock_guard<std::mutex> l(S->mu);
  const uint64_t tk = S->next_ticket++;
  S->frames.emplace(tk, F);
  S->queue.push_back(tk);
  S->stats.submitted++;
  *ticket = tk;
  S->cv.notify_all();
  return TPCT_OK;
}

tpct_status tpct_server_poll(tpct_server* S, uint64_t ticket, tpct_frame_info* info) {
  if (!S || !info) return TPCT_E_INVALID;
  std::lock_guard<std::mutex> l(S->mu);
  auto it = S->frames.find(ticket);
  if (it == S->frames.end()) return TPCT_E_INVALID;
  const Frame& F = it->second;
  info->state = (int32_t)F.state;
  info->status = F.status;
  info->n_tracks = F.counts[0];
  info->n_ids = F.counts[1];
  auto us = [&](Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::micro>(b - a).count();
  };
  info->queue_us = F.state >= kRunning || F.state == kFailed ? us(F.t_submit, F.t_start) : -1.0;
  info->latency_us = (F.state == kDone || F.state == kFailed) && F.t_done.time_since_epoch().count()
                         ? us(F.t_submit, F.t_done) : -1.0;
  return TPCT_OK;
}

tpct_status tpct_server_wait(tpct_server* S, uint64_t ticket, double timeout_s) {
  if (!S) return TPCT_E_INVALID;
  const auto t_end = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  while (true) {
    {
      std::lock_guard<std::mutex> l(S->mu);
      auto it = S->frames.find(ticket);
      if (it == S->frames.end()) return TPCT_E_INVALID;
      if (it->second.state == kDone) return TPCT_OK;
      if (it->second.state == kFailed) return it->second.status;
    }
    if (Clock::now() > t_end) return TPCT_E_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

tpct_status tpct_server_fetch(tpct_server* S, uint64_t ticket, tpct_host_tracks* h) {
  if (!S || !h) return TPCT_E_INVALID;
  tpct_tracks_out o;
  int32_t nt, ni;
  {
    std::lock_guard<std::mutex> l(S->mu);
    auto it = S->frames.find(ticket);
    if (it == S->frames.end() || it->second.state != kDone) return TPCT_E_STATE;
    o = it->second.out;
    nt = it->second.counts[0];
    ni = it->second.counts[1];
  }
  h->n_tracks = nt;
  h->n_ids = ni;
  if (nt > h->capacity_tracks || ni > h->capacity_ids) return TPCT_E_CAPACITY;
  cudaStream_t s = S->copy_stream;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t b) {
    if (e == cudaSuccess && dst && b) e = cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, s);
  };
  cp(h->instance, o.instance, 4 * (size_t)nt);
  cp(h->n_cl, o.n_cl, 4 * (size_t)nt);
  cp(h->offset, o.offset, 4 * (size_t)nt);
  cp(h->ndf, o.ndf, 4 * (size_t)nt);
  cp(h->status, o.status, 4 * (size_t)nt);
  cp(h->x_ref, o.x_ref, 8 * (size_t)nt);
  cp(h->param, o.param, 40 * (size_t)nt);
  cp(h->cov, o.cov, 120 * (size_t)nt);
  cp(h->chi2, o.chi2, 8 * (size_t)nt);
  cp(h->cluster_ids, o.cluster_ids, 4 * (size_t)ni);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? TPCT_OK : TPCT_E_CUDA;
}

tpct_status tpct_server_release(tpct_server* S, uint64_t ticket) {
  if (!S) return TPCT_E_INVALID;
  std::lock_guard<std::mutex> l(S->mu);
  auto it = S->frames.find(ticket);
  if (it == S->frames.end()) return TPCT_E_INVALID;
  if (it->second.state == kQueued || it->second.state == kRunning) return TPCT_E_STATE;
  if (it->second.bytes_out) S->arena.release(it->second.off_out, it->second.bytes_out);
  S->frames.erase(it);
  S->cv.notify_all();
  return TPCT_OK;
}

tpct_status tpct_server_get_stats(tpct_server* S, tpct_server_stats* out) {
  if (!S || !out) return TPCT_E_INVALID;
  std::lock_guard<std::mutex> l(S->mu);
  S->stats.bytes_in_use = S->arena.used();
  S->stats.peak_bytes = S->arena.peak();
  S->stats.budget_bytes = S->arena.total();
  int running = 0;
  for (auto& sl : S->slots) running += sl.ticket != 0;
  S->stats.in_flight = running;
  *out = S->stats;
  return TPCT_OK;
}

}  // extern "C"
