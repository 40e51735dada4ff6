// Host-runtime internals shared by the plain/batched path (dh_runtime.cpp) and
// the served path (dh_serve.cpp).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/dh.h"
#include "dh_internal.h"

namespace dh {

// Record a failure message for dh_last_error() on this thread and return s.
dh_status fail(dh_status s, const char* fmt, ...);
const char* last_error_message();

#define DH_CUDA_TRY(expr)                                                                        \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return ::dh::fail(e_ == cudaErrorMemoryAllocation ? DH_ERR_NOMEM : DH_ERR_CUDA, "%s: %s", \
                        #expr, cudaGetErrorString(e_));                                          \
  } while (0)

// Device buffer that only grows.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes);
  void release();
};

// Pinned host buffer that only grows.
struct HostBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes);
  void release();
};

// Binary64 bin-threshold tables per (r_max, nbins), shared by all paths of a
// context.  acquire() returns a table (building it on `st` if missing) and
// holds a reference; release() drops it.  A table built on one stream is made
// visible to work on another stream through an event wait.  Unreferenced tables
// beyond the cap are freed stream-ordered.
class ThresholdCache {
 public:
  dh_status acquire(double r_max, int32_t nbins, cudaStream_t st, int32_t* status_dev, double** T,
                    int* launched);
  void release(const double* T);
  void clear(cudaStream_t st);

 private:
  struct Key {
    uint64_t rbits;
    int32_t nbins;
    bool operator<(const Key& o) const { return rbits != o.rbits ? rbits < o.rbits : nbins < o.nbins; }
  };
  struct Entry {
    double* T;
    int refs;
    uint64_t last;
    cudaStream_t built_on;  // stream of the build kernel
    cudaEvent_t ready;      // recorded after it; other streams wait on it
  };
  std::mutex mu_;
  std::map<Key, Entry> map_;
  std::unordered_map<const double*, Key> rev_;
  uint64_t tick_ = 0;
  size_t cap_ = 64;
};

// A frame checked and planned on the host.
struct PlannedFrame {
  const dh_frame* src;
  int32_t variant;
  int32_t n_hist;
  int32_t sweeps;
  int32_t sweep_width;
  double margin;
  uint64_t pairs;
};

dh_status check_frame(const dh_frame* f, PlannedFrame& pf, int max_width);
void fill_frame_dev(const PlannedFrame& pf, FrameDev& F, const float4* X, uint64_t* out, const double* T);
int64_t add_segments(const PlannedFrame& pf, FrameDev* fd, int64_t item0, std::vector<Segment>& segs);
// Blocks for the pair kernel: `bps` per SM, at most one per item.
int pair_grid(int num_sms, int bps, int64_t n_items);

class Server;  // served path (dh_serve.cpp)
Server* server_create(dh_ctx* c, dh_status* st);
void server_destroy(Server* s);
dh_status server_submit(Server* s, const dh_frame* f, uint64_t* ticket);
dh_status server_poll(Server* s, uint64_t ticket);
dh_status server_wait(Server* s, uint64_t ticket, uint64_t timeout_ns);
dh_status server_cancel(Server* s, uint64_t ticket);

}  // namespace dh

struct dh_ctx {
  int device = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t user_stream = nullptr;
  bool has_user_stream = false;
  std::recursive_mutex mu;
  int num_sms = 0;
  int max_width = 0;
  dh_config cfg{};

  dh::DevBuf raw;      // caller coordinates copied from the host (n x stride floats)
  dh::DevBuf X;        // packed float4 coordinates
  dh::DevBuf hist;     // uint64 histograms (host-pointer outputs)
  dh::DevBuf meta;     // FrameDev | StageJob | Segment arrays
  dh::DevBuf ctl;      // Control
  dh::HostBuf hmeta;   // pinned staging for meta
  dh::HostBuf hout;    // pinned staging for accumulate-on-host
  dh::DevBuf tstat;    // threshold build status
  dh::ThresholdCache tcache;
  std::vector<const double*> held_tables;  // tables referenced by work not yet finished

  dh_stats stats{};
  cudaEvent_t ev_pair0 = nullptr, ev_pair1 = nullptr;  // pair-kernel timing (DH_CFG_TIMING)
  bool timed = false;
  bool pending_async = false;
  cudaGraphExec_t gexec = nullptr;  // batched path: executable graph, updated per call

  std::mutex server_mu;
  dh::Server* server = nullptr;

  cudaStream_t stream() const { return has_user_stream ? user_stream : own_stream; }
};
