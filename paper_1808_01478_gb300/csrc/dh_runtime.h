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
// jm: j tiles of kTile/jm particles per i tile of kTile.  fill_segments writes
// at most cap segments to out and the total to *n_out; add_segments appends all.
int64_t fill_segments(const PlannedFrame& pf, FrameDev* fd, int64_t item0, int jm, Segment* out, int cap,
                      int* n_out);
int64_t add_segments(const PlannedFrame& pf, FrameDev* fd, int64_t item0, std::vector<Segment>& segs, int jm = 1);

// Launch shape of one pair-kernel launch.
struct LaunchParams {
  int32_t jm = 1;                // j tiles per i tile: tile_j = kTile / jm
  int32_t depth = 1;             // private histogram copies per block
  int32_t bps = 0;               // blocks per SM (0: as many as fit)
  int32_t block = kBlockSmall;   // threads per block (kBlockSmall, kBlockLarge or kBlockHuge)
  int32_t agg = 0;               // 256-thread blocks, one sweep: warp-aggregated increments
};

// Autotuner key of a launch: variant, histogram width, frame size, frame count (all bucketed).
struct TuneKey {
  int32_t variant = 0, width_log2 = 0, n_log2 = 0, frames_log4 = 0;
  bool operator<(const TuneKey& o) const {
    if (variant != o.variant) return variant < o.variant;
    if (width_log2 != o.width_log2) return width_log2 < o.width_log2;
    if (n_log2 != o.n_log2) return n_log2 < o.n_log2;
    return frames_log4 < o.frames_log4;
  }
};
struct TuneEntry {
  LaunchParams p;
  double gpairs_s = 0.0;
};
TuneKey make_tune_key(int variant, int width, double mean_pairs_per_frame, int frames);

// Bytes of a frame's coordinate array (float32 or binary64, 3 or 4 per particle).
size_t coord_bytes(const dh_frame* f);

// Species of frames without the 27-image search are put in spatial (Morton)
// order before the pair kernel (no box: over the frame's bounding box), from this many particles on, with about 16
// particles per cell.  plan_spatial_order lists the species of one frame (its
// particles from x0 in the packed coordinates, its counters from key0) and
// returns the counters and most staging chunks they need.
constexpr int32_t kSortMinParticles = 2048;
int sort_grid_bits(int64_t n);
std::vector<SortSeg> plan_spatial_order(const PlannedFrame& pf, const FrameDev* fd, int64_t x0, int64_t key0,
                                        int64_t* keys, int* chunks);

// Threads per block for a launch without a measured shape: from 16,384 bins on,
// a 256-thread block's histogram leaves room for at most two blocks per SM, and
// one 1024-thread block sharing one histogram keeps more warps resident (512
// threads when the larger block's queues do not fit next to the histogram).
int default_block(int variant, int width);

// Measured launch shapes per key (dh_tune.cpp), optionally kept in a text file.
class Tuner {
 public:
  bool lookup(const TuneKey& k, LaunchParams* p);
  void store(const TuneKey& k, const TuneEntry& e);
  size_t size();
  int load(const std::string& path, int sms);   // entries read, -1 if the file cannot be read
  bool save(const std::string& path, int sms);

 private:
  std::mutex mu_;
  std::map<TuneKey, TuneEntry> map_;
};
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
  dh::DevBuf aux;      // small per-call arrays (g(r) pair densities)
  dh::DevBuf X64;      // binary64 input coordinates (double4), when a frame has them
  dh::DevBuf sortX64;  // spatial order: scratch copy of those,
  dh::DevBuf sortX;    // of the float32 coordinates,
  dh::DevBuf sortK;    //   cell keys,
  dh::DevBuf sortC;    //   and cell counters
  dh::ThresholdCache tcache;
  std::vector<const double*> held_tables;  // tables referenced by work not yet finished

  dh::Tuner tuner;
  std::string tune_path;           // autotuner cache file ("" for none)
  bool tune_forced = false;        // measurement in progress: every launch uses tune_force
  dh::LaunchParams tune_force;
  int32_t tune_runs = 0;           // measurement launches made for the current call
  double tune_cap_pairs = 0.0;     // measurement: stop each pair-kernel launch after about this many pairs

  dh_stats stats{};
  cudaEvent_t ev_pair0 = nullptr, ev_pair1 = nullptr;  // pair-kernel timing (DH_CFG_TIMING)
  bool timed = false;
  bool pending_async = false;
  cudaGraphExec_t gexec = nullptr;  // batched path: executable graph, updated per call

  std::mutex server_mu;
  dh::Server* server = nullptr;

  cudaStream_t stream() const { return has_user_stream ? user_stream : own_stream; }
};
