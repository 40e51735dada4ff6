// Served path of libdh: requests (one frame each) are admitted by their device
// memory footprint and run by continuous batching.
//
// The paper's engine (Sec. 3.3) feeds whole frames from a reader queue to
// worker processes.  Here one scheduler thread per context keeps the GPU busy
// with "waves": each wave is one launch of the persistent pair kernel over a
// slice of the work items of the admitted requests (a pair budget sized for a
// few milliseconds, given to the requests with the least work left first; see
// launch_wave).  A request that arrives while others
// run is admitted as soon as pool memory and a slot are free, and its items
// join the next wave next to the remaining items of the running requests, so
// small frames are not stuck behind large ones.  Each minimum-image variant
// (no box, orthorhombic, triclinic, triclinic with image search) has its own
// lane: a stream and a pipeline of waves, so the kernels of different lanes
// overlap on the device and fill each other's launch tails.  Completion is
// observed with CUDA events polled by the scheduler, so no kernel ever waits on
// the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dh_runtime.h"

namespace dh {

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kAlign = 256;
constexpr int kWaveSlots = 4;          // waves that may be in flight at once
// Histogram-width classes of a wave: one pair-kernel launch per class,
// ceil(log2 of the sweep width) up to 16 and one class above it.
constexpr int kWidthClasses = 8;
int width_class(int width) {
  int b = 0;
  while (b < 30 && (1 << b) < width) ++b;
  return b <= 9 ? 0 : (b >= 16 ? kWidthClasses - 1 : b - 9);
}
// Waves in flight per lane.  One: the next wave is built when the running one
// completes (the scheduler polls every 50 us), so a request that arrives waits
// for the running wave only, not also for one queued behind it; the idle gap
// per wave is a few tens of microseconds, and the other lanes fill it.
constexpr int kWavesAhead = 1;
constexpr double kWaveSecondsDefault = 0.006;  // target device time of one wave
// While requests wait for admission (the server is saturated), waves are this
// many times longer: a wave's tail (its last items finishing on part of the
// SMs) and the gap before the next wave are then a smaller share of the time,
// and a new request waits for the queue ahead of it anyway.
constexpr double kSaturatedWaveFactor = 4.0;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over an address range [0, cap) with coalescing.
class Arena {
 public:
  void init(size_t cap) {
    free_.clear();
    used_.clear();
    cap_ = cap;
    if (cap) free_[0] = cap;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(std::max<size_t>(bytes, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        size_t rest = it->second - bytes;
        size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_[*off] = bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off) {
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t size = u->second;
    used_.erase(u);
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + size == next->first) {
      size += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += size;
        return;
      }
    }
    free_[off] = size;
  }
  size_t capacity() const { return cap_; }

 private:
  size_t cap_ = 0;
  std::map<size_t, size_t> free_;
  std::unordered_map<size_t, size_t> used_;
};

enum ReqState { Q_QUEUED = 0, Q_ACTIVE = 1, Q_FINAL = 2 };

struct Request {
  uint64_t ticket = 0;
  dh_frame frame{};
  std::vector<int64_t> offs;
  PlannedFrame pf{};
  bool dev_ptrs = false;
  int stride = 3;
  size_t dev_bytes = 0, pin_bytes = 0;
  size_t dev_off = 0, pin_off = 0;
  bool has_dev = false, has_pin = false;
  FrameDev* fd = nullptr;        // device descriptor (pool)
  StageJob* job_dev = nullptr;   // device staging job (pool)
  float4* X = nullptr;
  float* raw = nullptr;          // device copy of host coordinates
  uint64_t* hist = nullptr;      // device histograms (caller's when DH_DEVICE_PTRS)
  FrameDev* fd_pin = nullptr;    // pinned: upload source, later the read-back
  StageJob* job_pin = nullptr;
  float* raw_pin = nullptr;      // pinned copy of host coordinates
  uint64_t* res_pin = nullptr;   // pinned histogram read-back
  size_t res_count = 0;
  double* T = nullptr;
  std::vector<Segment> segs;     // all segments, items numbered from 0
  // spatial order of the species (periodic frames): plan, device scratch, pinned upload
  std::vector<SortSeg> sorts;
  int64_t sort_keys = 0;
  int sort_chunks = 0;
  SortSeg* sort_dev = nullptr;
  SortSeg* sort_pin = nullptr;
  float4* sort_X = nullptr;
  int32_t* sort_K = nullptr;
  uint32_t* sort_C = nullptr;
  int64_t n_items = 0, next = 0;
  bool prepped = false, finalize_enqueued = false, cancel = false;
  bool timed_out = false;        // cancelled because it passed its deadline (dh_config.timeout_ns)
  uint64_t last_wave = 0;        // sequence number of the last wave carrying its work
  cudaEvent_t done_ev = nullptr;
  int state = Q_QUEUED;
  dh_status status = DH_PENDING;
  std::string error;
  Clock::time_point t_submit;
};

struct WaveSlot {
  DevBuf segs;
  HostBuf hsegs;
  DevBuf ctl;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  uint64_t seq = 0;
  bool busy = false;
  double pairs = 0;
};

// One minimum-image variant: its stream and its pipeline of waves.
struct Lane {
  cudaStream_t stream = nullptr;
  WaveSlot slots[kWaveSlots];
  std::deque<int> inflight;  // slot indices in launch order
  uint64_t wave_seq = 0, done_seq = 0;
  double rate = 1.0e12;      // measured pairs/s of recent waves
  DevBuf tstat;              // threshold build status
};

}  // namespace

class Server {
 public:
  explicit Server(dh_ctx* c) : ctx_(c) {}
  ~Server() { shutdown(); }

  dh_status start();
  void shutdown();
  dh_status submit(const dh_frame* f, uint64_t* ticket);
  dh_status poll(uint64_t ticket);
  dh_status wait(uint64_t ticket, uint64_t timeout_ns);
  dh_status cancel(uint64_t ticket);

 private:
  void loop();
  void expire();
  void admit();
  bool launch_wave(int v);
  void reap();
  dh_status prep(Request& r);
  dh_status finalize_enqueue(Request& r);
  void complete(Request& r, dh_status st, const char* msg);
  void release_resources(Request& r);

  dh_ctx* ctx_;
  int device_ = 0;
  void* pool_ = nullptr;
  void* pinned_ = nullptr;
  Arena dev_arena_, pin_arena_;
  int max_inflight_ = 64;
  double wave_seconds_ = kWaveSecondsDefault;
  uint64_t timeout_ns_ = 0;  // deadline of a request after its submission (0: none)
  Lane lanes_[kNumVariants];

  std::mutex mu_;
  std::condition_variable cv_work_, cv_done_;
  bool stop_ = false;
  std::thread th_;
  uint64_t next_ticket_ = 1;
  std::deque<Request*> queue_;
  std::vector<Request*> active_;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> all_;
  std::string thread_error_;
};

dh_status Server::start() {
  device_ = ctx_->device;
  DH_CUDA_TRY(cudaSetDevice(device_));
  size_t free_b = 0, total_b = 0;
  DH_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  size_t pool = ctx_->cfg.pool_bytes ? (size_t)ctx_->cfg.pool_bytes
                                     : std::min<size_t>(free_b / 2, (size_t)16 << 30);
  if (pool > free_b) return fail(DH_ERR_NOMEM, "pool of %zu bytes exceeds free device memory", pool);
  DH_CUDA_TRY(cudaMalloc(&pool_, pool));
  dev_arena_.init(pool);
  size_t pin = std::min<size_t>(std::max<size_t>(pool / 8, (size_t)64 << 20), (size_t)512 << 20);
  DH_CUDA_TRY(cudaMallocHost(&pinned_, pin));
  pin_arena_.init(pin);
  max_inflight_ = ctx_->cfg.max_inflight > 0 ? ctx_->cfg.max_inflight : 64;
  if (ctx_->cfg.wave_us) wave_seconds_ = 1e-6 * (double)ctx_->cfg.wave_us;
  timeout_ns_ = ctx_->cfg.timeout_ns;
  for (Lane& ln : lanes_) {
    DH_CUDA_TRY(cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking));
    DH_CUDA_TRY(ln.tstat.ensure(64));
    DH_CUDA_TRY(cudaMemsetAsync(ln.tstat.p, 0, 64, ln.stream));
    for (auto& w : ln.slots) {
      DH_CUDA_TRY(w.ctl.ensure(sizeof(Control) * kWidthClasses));
      DH_CUDA_TRY(cudaEventCreate(&w.ev0));
      DH_CUDA_TRY(cudaEventCreate(&w.ev1));
    }
  }
  th_ = std::thread([this] { loop(); });
  return DH_OK;
}

void Server::shutdown() {
  {
    std::lock_guard<std::mutex> g(mu_);
    if (stop_) return;
    stop_ = true;
    for (Request* r : queue_) complete(*r, DH_ERR_CANCELLED, "context destroyed");
    queue_.clear();
  }
  cv_work_.notify_all();
  if (th_.joinable()) th_.join();
  for (Lane& ln : lanes_)
    if (ln.stream) cudaStreamSynchronize(ln.stream);
  std::lock_guard<std::mutex> g(mu_);
  for (Request* r : active_) {
    release_resources(*r);
    if (r->state != Q_FINAL) complete(*r, DH_ERR_CANCELLED, "context destroyed");
  }
  active_.clear();
  for (auto& kv : all_)
    if (kv.second->done_ev) cudaEventDestroy(kv.second->done_ev);
  all_.clear();
  for (Lane& ln : lanes_) {
    for (auto& w : ln.slots) {
      w.segs.release();
      w.hsegs.release();
      w.ctl.release();
      if (w.ev0) cudaEventDestroy(w.ev0);
      if (w.ev1) cudaEventDestroy(w.ev1);
      w.ev0 = w.ev1 = nullptr;
    }
    ln.tstat.release();
    if (ln.stream) cudaStreamDestroy(ln.stream);
    ln.stream = nullptr;
  }
  if (pool_) cudaFree(pool_);
  if (pinned_) cudaFreeHost(pinned_);
  pool_ = pinned_ = nullptr;
  cv_done_.notify_all();
}

dh_status Server::submit(const dh_frame* f, uint64_t* ticket) {
  auto r = std::make_unique<Request>();
  if (f->n_species < 1) return fail(DH_ERR_INVALID, "n_species must be >= 1");
  if (!f->species_offsets) return fail(DH_ERR_INVALID, "species_offsets is NULL");
  r->frame = *f;
  r->offs.assign(f->species_offsets, f->species_offsets + f->n_species + 1);
  r->frame.species_offsets = r->offs.data();
  if (f->flags & DH_COORDS_F64)
    return fail(DH_ERR_INVALID, "the served path takes float32 coordinates (DH_COORDS_F64: use dh_histogram)");
  dh_status s = check_frame(&r->frame, r->pf, ctx_->max_width);
  if (s != DH_OK) return s;
  r->pf.src = &r->frame;
  r->dev_ptrs = (f->flags & DH_DEVICE_PTRS) != 0;
  r->stride = (f->flags & DH_COORDS_F4) ? 4 : 3;
  r->res_count = (size_t)r->pf.n_hist * (size_t)f->nbins;
  size_t n = (size_t)f->n;
  r->dev_bytes = align_up(sizeof(FrameDev)) + align_up(sizeof(StageJob)) + align_up(16 * std::max<size_t>(n, 1));
  r->pin_bytes = align_up(sizeof(FrameDev)) + align_up(sizeof(StageJob));
  r->sorts = plan_spatial_order(r->pf, nullptr, 0, 0, &r->sort_keys, &r->sort_chunks);
  if (!r->sorts.empty()) {
    r->dev_bytes += align_up(sizeof(SortSeg) * r->sorts.size()) + align_up(16 * n) + align_up(4 * n) +
                    align_up(4 * (size_t)r->sort_keys);
    r->pin_bytes += align_up(sizeof(SortSeg) * r->sorts.size());
  }
  if (!r->dev_ptrs) {
    r->dev_bytes += align_up(4 * (size_t)r->stride * n) + align_up(8 * r->res_count);
    r->pin_bytes += align_up(4 * (size_t)r->stride * n) + align_up(8 * r->res_count);
  }
  std::lock_guard<std::mutex> g(mu_);
  if (stop_) return fail(DH_ERR_CANCELLED, "server is shutting down");
  if (!thread_error_.empty()) return fail(DH_ERR_CUDA, "%s", thread_error_.c_str());
  if (r->dev_bytes > dev_arena_.capacity() || r->pin_bytes > pin_arena_.capacity())
    return fail(DH_ERR_NOMEM, "request needs %zu device / %zu pinned bytes, pool holds %zu / %zu",
                r->dev_bytes, r->pin_bytes, dev_arena_.capacity(), pin_arena_.capacity());
  r->ticket = next_ticket_++;
  r->t_submit = Clock::now();
  *ticket = r->ticket;
  queue_.push_back(r.get());
  all_[r->ticket] = std::move(r);
  cv_work_.notify_one();
  return DH_OK;
}

dh_status Server::poll(uint64_t ticket) {
  std::lock_guard<std::mutex> g(mu_);
  auto it = all_.find(ticket);
  if (it == all_.end()) return fail(DH_ERR_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  Request& r = *it->second;
  if (r.state != Q_FINAL) return DH_PENDING;
  dh_status st = r.status;
  if (st < 0) fail(st, "%s", r.error.c_str());
  if (r.done_ev) cudaEventDestroy(r.done_ev);
  all_.erase(it);
  return st;
}

dh_status Server::wait(uint64_t ticket, uint64_t timeout_ns) {
  {
    std::unique_lock<std::mutex> lk(mu_);
    auto deadline = Clock::now() + std::chrono::nanoseconds(timeout_ns);
    for (;;) {
      auto it = all_.find(ticket);
      if (it == all_.end()) return fail(DH_ERR_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
      if (it->second->state == Q_FINAL) break;
      if (cv_done_.wait_until(lk, deadline) == std::cv_status::timeout) {
        auto again = all_.find(ticket);
        if (again != all_.end() && again->second->state == Q_FINAL) break;
        return fail(DH_ERR_TIMEOUT, "request %llu still running", (unsigned long long)ticket);
      }
    }
  }
  return poll(ticket);
}

dh_status Server::cancel(uint64_t ticket) {
  std::lock_guard<std::mutex> g(mu_);
  auto it = all_.find(ticket);
  if (it == all_.end()) return fail(DH_ERR_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  Request& r = *it->second;
  if (r.state == Q_FINAL) return DH_OK;
  r.cancel = true;
  if (r.state == Q_QUEUED) {
    queue_.erase(std::remove(queue_.begin(), queue_.end(), &r), queue_.end());
    complete(r, DH_ERR_CANCELLED, "cancelled");
  }
  cv_work_.notify_one();
  return DH_OK;
}

void Server::complete(Request& r, dh_status st, const char* msg) {
  r.state = Q_FINAL;
  r.status = st;
  r.error = msg ? msg : "";
  cv_done_.notify_all();
}

void Server::release_resources(Request& r) {
  if (r.T) ctx_->tcache.release(r.T);
  r.T = nullptr;
  if (r.has_dev) dev_arena_.release(r.dev_off);
  if (r.has_pin) pin_arena_.release(r.pin_off);
  r.has_dev = r.has_pin = false;
}

// Admit queued requests in arrival order while slots, pool and pinned memory allow.
void Server::admit() {
  while (!queue_.empty() && (int)active_.size() < max_inflight_) {
    Request& r = *queue_.front();
    size_t doff = 0, poff = 0;
    if (!dev_arena_.alloc(r.dev_bytes, &doff)) break;
    if (!pin_arena_.alloc(r.pin_bytes, &poff)) {
      dev_arena_.release(doff);
      break;
    }
    r.dev_off = doff;
    r.pin_off = poff;
    r.has_dev = r.has_pin = true;
    char* d = (char*)pool_ + doff;
    char* p = (char*)pinned_ + poff;
    r.fd = (FrameDev*)d;
    d += align_up(sizeof(FrameDev));
    r.job_dev = (StageJob*)d;
    d += align_up(sizeof(StageJob));
    r.X = (float4*)d;
    d += align_up(16 * std::max<size_t>((size_t)r.frame.n, 1));
    r.fd_pin = (FrameDev*)p;
    p += align_up(sizeof(FrameDev));
    r.job_pin = (StageJob*)p;
    p += align_up(sizeof(StageJob));
    if (!r.sorts.empty()) {
      r.sort_dev = (SortSeg*)d;
      d += align_up(sizeof(SortSeg) * r.sorts.size());
      r.sort_X = (float4*)d;
      d += align_up(16 * (size_t)r.frame.n);
      r.sort_K = (int32_t*)d;
      d += align_up(4 * (size_t)r.frame.n);
      r.sort_C = (uint32_t*)d;
      d += align_up(4 * (size_t)r.sort_keys);
      r.sort_pin = (SortSeg*)p;
      p += align_up(sizeof(SortSeg) * r.sorts.size());
    }
    if (!r.dev_ptrs) {
      r.raw = (float*)d;
      d += align_up(4 * (size_t)r.stride * (size_t)r.frame.n);
      r.hist = (uint64_t*)d;
      r.raw_pin = (float*)p;
      p += align_up(4 * (size_t)r.stride * (size_t)r.frame.n);
      r.res_pin = (uint64_t*)p;
      // host coordinates are copied to pinned memory now so the upload is asynchronous
      if (r.frame.n > 0)
        std::memcpy(r.raw_pin, r.frame.coords, 4 * (size_t)r.stride * (size_t)r.frame.n);
    } else {
      r.hist = r.frame.out;
    }
    r.segs.clear();
    r.n_items = add_segments(r.pf, r.fd, 0, r.segs);
    r.next = 0;
    r.state = Q_ACTIVE;
    queue_.pop_front();
    active_.push_back(&r);
  }
}

// Enqueue the per-request preparation: uploads, thresholds, staging, window setup.
dh_status Server::prep(Request& r) {
  Lane& ln = lanes_[r.pf.variant];
  cudaStream_t st = ln.stream;
  dh_status s = ctx_->tcache.acquire(r.frame.r_max, r.frame.nbins, st, (int32_t*)ln.tstat.p, &r.T, nullptr);
  if (s != DH_OK) return s;
  fill_frame_dev(r.pf, *r.fd_pin, r.X, r.hist, r.T);
  std::memset(r.job_pin, 0, sizeof(StageJob));
  r.job_pin->src = r.dev_ptrs ? r.frame.coords : r.raw;
  r.job_pin->dst = r.X;
  r.job_pin->fd = r.fd;
  r.job_pin->n = r.frame.n;
  r.job_pin->stride = r.stride;
  r.job_pin->chunk0 = 0;
  DH_CUDA_TRY(cudaMemcpyAsync(r.fd, r.fd_pin, sizeof(FrameDev), cudaMemcpyHostToDevice, st));
  DH_CUDA_TRY(cudaMemcpyAsync(r.job_dev, r.job_pin, sizeof(StageJob), cudaMemcpyHostToDevice, st));
  if (!r.dev_ptrs && r.frame.n > 0)
    DH_CUDA_TRY(cudaMemcpyAsync(r.raw, r.raw_pin, 4 * (size_t)r.stride * (size_t)r.frame.n,
                                cudaMemcpyHostToDevice, st));
  if (!r.dev_ptrs || !(r.frame.flags & DH_ACCUMULATE))
    DH_CUDA_TRY(cudaMemsetAsync(r.hist, 0, 8 * r.res_count, st));
  int64_t chunks = (r.frame.n + kStageChunk - 1) / kStageChunk;
  if (chunks > 0) DH_CUDA_TRY(launch_stage(r.job_dev, 1, chunks, st));
  if (!r.sorts.empty()) {
    for (size_t q = 0; q < r.sorts.size(); ++q) {
      r.sort_pin[q] = r.sorts[q];
      r.sort_pin[q].fd = r.fd;
    }
    DH_CUDA_TRY(cudaMemcpyAsync(r.sort_dev, r.sort_pin, sizeof(SortSeg) * r.sorts.size(), cudaMemcpyHostToDevice,
                                st));
    DH_CUDA_TRY(cudaMemsetAsync(r.sort_C, 0, 4 * (size_t)r.sort_keys, st));
    DH_CUDA_TRY(launch_spatial_sort(r.sort_dev, (int)r.sorts.size(), r.sort_chunks, r.X, r.sort_X, nullptr, nullptr,
                                    r.sort_K, r.sort_C, st));
  }
  DH_CUDA_TRY(launch_frame_setup(r.fd, 1, 0, st));
  // marks the end of the preparation: a request cancelled before its first wave
  // keeps its pool memory until this work has finished
  if (!r.done_ev) DH_CUDA_TRY(cudaEventCreateWithFlags(&r.done_ev, cudaEventDisableTiming));
  DH_CUDA_TRY(cudaEventRecord(r.done_ev, st));
  r.prepped = true;
  return DH_OK;
}

// After the request's last wave: read back its flags and (host outputs) histograms.
dh_status Server::finalize_enqueue(Request& r) {
  cudaStream_t st = lanes_[r.pf.variant].stream;
  DH_CUDA_TRY(cudaMemcpyAsync(r.fd_pin, r.fd, sizeof(FrameDev), cudaMemcpyDeviceToHost, st));
  if (!r.dev_ptrs)
    DH_CUDA_TRY(cudaMemcpyAsync(r.res_pin, r.hist, 8 * r.res_count, cudaMemcpyDeviceToHost, st));
  if (!r.done_ev) DH_CUDA_TRY(cudaEventCreateWithFlags(&r.done_ev, cudaEventDisableTiming));
  DH_CUDA_TRY(cudaEventRecord(r.done_ev, st));
  r.finalize_enqueued = true;
  return DH_OK;
}

// One wave of lane v: the lane's pair budget over the running requests of that
// variant, the least work left first (the order is stated below), as one
// pair-kernel launch per histogram-width class.
bool Server::launch_wave(int v) {
  Lane& ln = lanes_[v];
  int slot = -1;
  for (int k = 0; k < kWaveSlots; ++k)
    if (!ln.slots[k].busy) {
      slot = k;
      break;
    }
  if (slot < 0) return false;
  std::vector<Request*> run;
  for (Request* r : active_) {
    if (r->pf.variant != v || r->cancel) continue;
    if (r->next < r->n_items) {
      run.push_back(r);
    } else if (!r->finalize_enqueued && r->n_items == 0) {
      // nothing to compute (no pairs): preparation and read-back only
      dh_status s = r->prepped ? DH_OK : prep(*r);
      if (s == DH_OK) s = finalize_enqueue(*r);
      if (s != DH_OK) {
        r->cancel = true;
        r->error = last_error_message();
      }
    }
  }
  if (run.empty()) return false;
  WaveSlot& W = ln.slots[slot];
  const double pairs_per_item = (double)kTile * (double)kTile;
  // The wave's pair budget goes to the requests with the least work left
  // first, so small requests finish in the wave they join.  While every
  // admitted request can run (no request waits for admission), the order is
  // shortest remaining work first: each request takes all it needs and the
  // rest of the budget goes to the next smallest (equal parts would let two
  // large requests that overlap each finish about as late as both together).
  // While requests wait for admission, each takes what it needs up to an equal
  // share of what remains: the queue, not the order, sets their latency then,
  // and equal shares keep the saturated throughput higher (measured).  Every
  // request takes at least one work item per wave.
  std::stable_sort(run.begin(), run.end(),
                   [](const Request* a, const Request* b) { return a->n_items - a->next < b->n_items - b->next; });
  const bool saturated = !queue_.empty();
  double budget_left = ln.rate * wave_seconds_ * (saturated ? kSaturatedWaveFactor : 1.0);
  // segments per histogram-width class: requests of very different widths run
  // in separate launches, each with the launch shape of its own width (one
  // wide request would otherwise give every request of the wave the shape of
  // the widest histogram: larger blocks and fewer of them per SM)
  std::vector<Segment> csegs[kWidthClasses];
  int64_t citems[kWidthClasses] = {};
  int cwidth[kWidthClasses], cmulti[kWidthClasses] = {};
  for (int q = 0; q < kWidthClasses; ++q) cwidth[q] = 1;
  int64_t witems = 0;
  double wpairs = 0;
  std::vector<Request*> finishing;
  for (size_t q = 0; q < run.size(); ++q) {
    Request* r = run[q];
    if (!r->prepped) {
      dh_status s = prep(*r);
      if (s != DH_OK) {
        r->cancel = true;
        r->error = last_error_message();
        continue;
      }
    }
    const double share = std::max(0.0, budget_left) / (saturated ? (double)(run.size() - q) : 1.0);
    int64_t take = std::max<int64_t>(1, (int64_t)(share / pairs_per_item));
    take = std::min(take, r->n_items - r->next);
    budget_left -= (double)take * pairs_per_item;
    int64_t lo = r->next, hi = r->next + take;
    const int cl = width_class(r->pf.sweep_width);
    for (const Segment& sg : r->segs) {
      int64_t count = sg.intra ? (int64_t)sg.n_ti * (sg.n_ti + 1) / 2 : (int64_t)sg.n_ti * sg.n_tj;
      int64_t a = std::max(lo, sg.item0), b = std::min(hi, sg.item0 + count);
      if (a >= b) continue;
      Segment w = sg;
      w.item0 = citems[cl];
      w.item_base = a - sg.item0;
      citems[cl] += b - a;
      witems += b - a;
      csegs[cl].push_back(w);
    }
    r->next = hi;
    r->last_wave = ln.wave_seq + 1;
    cwidth[cl] = std::max(cwidth[cl], r->pf.sweep_width);
    cmulti[cl] |= r->pf.sweeps > 1;
    wpairs += (double)std::min<uint64_t>(r->pf.pairs, (uint64_t)((double)take * pairs_per_item));
    if (r->next >= r->n_items) finishing.push_back(r);
  }
  if (witems == 0) return false;
  size_t nseg = 0;
  for (int q = 0; q < kWidthClasses; ++q) nseg += csegs[q].size();
  size_t bytes = sizeof(Segment) * nseg;
  if (W.segs.ensure(bytes) != cudaSuccess || W.hsegs.ensure(bytes) != cudaSuccess) {
    thread_error_ = "out of memory for wave descriptors";
    return false;
  }
  size_t at = 0;
  for (int q = 0; q < kWidthClasses; ++q) {
    if (!csegs[q].empty()) std::memcpy((Segment*)W.hsegs.p + at, csegs[q].data(), sizeof(Segment) * csegs[q].size());
    at += csegs[q].size();
  }
  cudaMemcpyAsync(W.segs.p, W.hsegs.p, bytes, cudaMemcpyHostToDevice, ln.stream);
  cudaMemsetAsync(W.ctl.p, 0, sizeof(Control) * kWidthClasses, ln.stream);
  cudaEventRecord(W.ev0, ln.stream);
  cudaError_t e = cudaSuccess;
  at = 0;
  for (int q = 0; q < kWidthClasses && e == cudaSuccess; ++q) {
    if (csegs[q].empty()) continue;
    PairLaunch L;
    std::memset(&L, 0, sizeof L);
    L.segs = (const Segment*)W.segs.p + at;
    L.n_segs = (int32_t)csegs[q].size();
    L.n_items = citems[q];
    L.hist_width = cwidth[q];
    L.multi = cmulti[q];
    L.block = default_block(v, cwidth[q]);
    L.ctl = (Control*)W.ctl.p + q;
    const int bps = pair_kernel_blocks_per_sm(v, cwidth[q], 1, L.block);
    e = launch_pairs(L, v, pair_grid(ctx_->num_sms, bps, citems[q]), pair_kernel_smem(cwidth[q], 1, L.block),
                     ln.stream);
    at += csegs[q].size();
  }
  cudaEventRecord(W.ev1, ln.stream);
  if (e != cudaSuccess) thread_error_ = cudaGetErrorString(e);
  W.busy = true;
  W.seq = ++ln.wave_seq;
  W.pairs = wpairs;
  ln.inflight.push_back(slot);
  for (Request* r : finishing)
    if (finalize_enqueue(*r) != DH_OK) {
      r->cancel = true;
      r->error = last_error_message();
    }
  return true;
}

void Server::reap() {
  for (Lane& ln : lanes_) {
    while (!ln.inflight.empty()) {
      WaveSlot& W = ln.slots[ln.inflight.front()];
      cudaError_t q = cudaEventQuery(W.ev1);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) thread_error_ = cudaGetErrorString(q);
      float ms = 0;
      if (cudaEventElapsedTime(&ms, W.ev0, W.ev1) == cudaSuccess && ms > 0.05f && W.pairs > 0)
        ln.rate = 0.7 * ln.rate + 0.3 * (W.pairs / (ms * 1e-3));
      ln.done_seq = W.seq;
      W.busy = false;
      ln.inflight.pop_front();
    }
  }
  for (size_t k = 0; k < active_.size();) {
    Request& r = *active_[k];
    bool finished = false;
    if (r.finalize_enqueued && r.done_ev) {
      cudaError_t q = cudaEventQuery(r.done_ev);
      if (q == cudaSuccess) {
        finished = true;
        if (r.cancel) {
          complete(r, r.timed_out ? DH_ERR_TIMEOUT : DH_ERR_CANCELLED,
                   r.timed_out ? "request passed its deadline (dh_config.timeout_ns)" : "cancelled");
        } else if (r.fd_pin->bad) {
          complete(r, DH_ERR_INVALID, "frame has non-finite coordinates");
        } else {
          if (!r.dev_ptrs) {
            uint64_t* out = r.frame.out;
            if (r.frame.flags & DH_ACCUMULATE)
              for (size_t i = 0; i < r.res_count; ++i) out[i] += r.res_pin[i];
            else
              std::memcpy(out, r.res_pin, 8 * r.res_count);
          }
          complete(r, DH_OK, nullptr);
        }
      } else if (q != cudaErrorNotReady) {
        finished = true;
        complete(r, DH_ERR_CUDA, cudaGetErrorString(q));
      }
    } else if (r.cancel && r.last_wave <= lanes_[r.pf.variant].done_seq &&
               (!r.prepped || !r.done_ev || cudaEventQuery(r.done_ev) != cudaErrorNotReady)) {
      finished = true;  // no work of it left on the device
      if (r.timed_out)
        complete(r, DH_ERR_TIMEOUT, "request passed its deadline (dh_config.timeout_ns)");
      else
        complete(r, r.error.empty() ? DH_ERR_CANCELLED : DH_ERR_CUDA,
                 r.error.empty() ? "cancelled" : r.error.c_str());
    }
    if (finished) {
      release_resources(r);
      active_.erase(active_.begin() + (long)k);
    } else {
      ++k;
    }
  }
}

// Requests past their deadline: queued ones end now, running ones are
// cancelled and end once none of their work is left on the device.
void Server::expire() {
  if (!timeout_ns_) return;
  const auto now = Clock::now();
  const auto limit = std::chrono::nanoseconds(timeout_ns_);
  for (size_t k = 0; k < queue_.size();) {
    Request& r = *queue_[k];
    if (now - r.t_submit > limit) {
      r.timed_out = r.cancel = true;
      complete(r, DH_ERR_TIMEOUT, "request passed its deadline (dh_config.timeout_ns) while queued");
      queue_.erase(queue_.begin() + (long)k);
    } else {
      ++k;
    }
  }
  for (Request* r : active_)
    if (!r->cancel && now - r->t_submit > limit) r->timed_out = r->cancel = true;
}

void Server::loop() {
  cudaSetDevice(device_);
  std::unique_lock<std::mutex> lk(mu_);
  while (!stop_) {
    expire();
    reap();
    admit();
    for (int v = 0; v < kNumVariants; ++v)
      while ((int)lanes_[v].inflight.size() < kWavesAhead && launch_wave(v)) {
      }
    reap();
    bool busy = false;
    for (Lane& ln : lanes_) busy |= !ln.inflight.empty();
    for (Request* r : active_)
      if (r->finalize_enqueued || r->cancel) busy = true;
    if (busy) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(50));
      lk.lock();
    } else {
      cv_work_.wait_for(lk, std::chrono::milliseconds(20));
    }
  }
}

Server* server_create(dh_ctx* c, dh_status* st) {
  auto s = std::make_unique<Server>(c);
  *st = s->start();
  if (*st != DH_OK) return nullptr;
  return s.release();
}

void server_destroy(Server* s) { delete s; }
dh_status server_submit(Server* s, const dh_frame* f, uint64_t* t) { return s->submit(f, t); }
dh_status server_poll(Server* s, uint64_t t) { return s->poll(t); }
dh_status server_wait(Server* s, uint64_t t, uint64_t ns) { return s->wait(t, ns); }
dh_status server_cancel(Server* s, uint64_t t) { return s->cancel(t); }

}  // namespace dh
