// Internal interface between the host runtime (dh_runtime.cpp) and the CUDA
// kernels (dh_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dh {

// Kernel variants of the minimum-image step (Eq. 5).
enum Variant : int32_t {
  V_NONE = 0,         // no periodic box
  V_ORTHO = 1,        // diagonal B: per-axis nearest image
  V_TRIC = 2,         // triclinic, r_max below half the smallest plane spacing: one wrap
  V_TRIC_SEARCH = 3,  // triclinic, larger r_max: Eq. 5 wrap plus the 27-image search
};

constexpr int kTile = 1024;          // i particles per work item (and the longest j tile)
constexpr int kSubJ = 256;           // j sub-chunk with its own tile image per warp
// Pair-kernel blocks: 256 threads with 4 i particles each, 512 with 2, or 1024 with 1.
constexpr int kBlockSmall = 256;
constexpr int kBlockLarge = 512;
constexpr int kBlockHuge = 1024;
constexpr int kQueueCap = 64;        // deferred pairs per warp queue
constexpr int kNumVariants = 4;

// One frame as seen by the device.  Host fills the first part; the staging and
// setup kernels fill the second.
struct FrameDev {
  const float4* X;   // packed coordinates (x,y,z,0), frame-local index
  const double4* X64;  // binary64 input coordinates (x,y,z,0), or null for float32 input
  uint64_t* out;     // S(S+1)/2 x nbins histograms of this frame
  const double* T;   // binary64 thresholds T[0..nbins]
  const float2* Tf;  // the same thresholds as float pairs (hi, lo), hi + lo = T to ~2^-48
  int32_t variant;
  int32_t nbins;
  int32_t n;         // particles
  int32_t sweep_width;  // bins per sweep (pass p covers [p*w, min(nbins,(p+1)*w)))
  double r_max;
  double B[9];       // row-major, columns a,b,c
  double Linv[3];    // orthorhombic: 1.0/L per axis, binary64
  float Bf[9];       // float32 copies of B
  float Bl[9];       // float32(B - Bf): B as double-float (Bf + Bl)
  float invf[3];     // float32 reciprocals: ortho 1/Lx,1/Ly,1/Lz; triclinic 1/ax,1/by,1/cz
  float S;           // float32(nbins / r_max)
  float dr_f;        // float32(r_max / nbins), the bin width
  float rmax_f;      // float32(r_max)
  float S2;          // float32((nbins / r_max)^2)
  float margin;      // triclinic: 1 - 2 r_max / h_min (no-search precondition margin)
  float tshift[27][3];  // triclinic tile images: -B k rounded once from binary64, k in {-1,0,1}^3
                        // (index 9 (kx+1) + 3 (ky+1) + (kz+1))
  float tserr[27][3];   // |tshift - (-B k)|, rounded up
  float convf[3];       // binary64 input: per-axis conversion error (conv), rounded up
  float kxdb;           // triclinic: largest |kx| times |ax32 - ax|, rounded up
  float dBf[9];         // |B32 - B| per entry, rounded up
  float tie_t[3];       // orthorhombic: t-space tie term of one wrapped axis (0: none), rounded up
  float tie_all;        // orthorhombic: the frame's tie term (all axes wrapped), rounded up
  float rr2;            // orthorhombic: (r_max (1 + 2/nbins))^2, rounded up
  double eps_S;      // |S - nbins/r_max| / (nbins/r_max)
  double eps_S2;     // |S2 - (nbins/r_max)^2| / (nbins/r_max)^2
  // ---- written on the device
  int32_t cmin[3];   // ordered-integer encodings of the per-axis coordinate min / max
  int32_t cmax[3];
  int32_t bad;       // a non-finite coordinate was seen
  int32_t all_defer; // float32 decisions are not safe for this frame: every pair is deferred
  int32_t in_range;  // no box, one sweep: every pair's root stays below nbins + 1 (the clamp is a no-op)
  int32_t cull_ok;   // no box: tiles can lie outside a sweep (several sweeps, or r_max below the extent)
  float beta_u;      // beta of tiles that take a uniform image (orthorhombic, triclinic)
  float beta_w[3];   // beta of tiles with a uniform image on all axes but a, wrapped per pair
  float tie_m[3];    // orthorhombic: margin of the uniform-image test (0: not needed)
  float mid2, mid1;  // double-float tier: |r2 - T[n]| <= mid2*r2 + mid1*s decides nothing
  float tie_eps;     // orthorhombic: | |d'_c| - L_c/2 | <= tie_eps is re-decided in binary64
  float delta;       // float32 window half-width in bin units at t = nbins (reported)
  float alpha_t, beta_t;  // the t-space bound alpha*t + beta behind the q-space test (per-pair images)
  float eps_s;       // search variant: fractional-coordinate ambiguity margin
  unsigned long long deferred;  // statistics: pairs queued for the double-float tier
  unsigned long long exact;     // pairs that also needed the binary64 replay
  unsigned long long uniform_pairs;  // pairs of (warp i run, j tile) blocks with one nearest image for all
  unsigned long long axis_pairs;     // pairs of such blocks whose image is uniform on all axes but one
  unsigned long long culled_pairs;   // pairs of blocks skipped: no pair of them has its bin in the sweep
};

// One species pair (a,b) of one frame and one bin sweep, cut into kTile x kTile
// work items numbered row by row over (ti, tj) (intra-species: tj >= ti only).
// A launch may carry only part of a segment's items: launch items
// [item0, item0 + count) are the segment's items [item_base, item_base + count).
struct Segment {
  FrameDev* fd;
  int32_t intra;     // a == b: only j tiles not below the i tile, pairs j > i
  int32_t h;         // histogram index within the frame
  int32_t pass;      // bin sweep: bins [pass*w, min(nbins, (pass+1)*w)), w = fd->sweep_width
  int32_t n_ti, n_tj;  // i tiles of kTile particles, j tiles of kTile/jm particles
  int32_t a0, na, b0, nb;  // frame-local particle ranges of species a and b
  int32_t jm;        // j tiles per i tile (1, 2 or 4; 0 means 1)
  int64_t item0;     // first launch item of this segment
  int64_t item_base; // segment-local index of that item
};

// Staging job: one frame's coordinates (n x stride floats) -> float4.
struct StageJob {
  const float* src;  // n x stride float32, or binary64 when dst64 is set
  float4* dst;
  double4* dst64;    // binary64 input: the values themselves (dst gets them rounded to float32)
  FrameDev* fd;
  int64_t n;
  int32_t stride;
  int32_t pad;
  int64_t chunk0;    // first staging chunk of this job
};
constexpr int kStageChunk = 8192;

// Spatial ordering of one species of one periodic frame: its particles are
// grouped by cell of a 2^g x 2^g x 2^g grid over the fractional coordinates, in
// Morton order, so that tiles of consecutive particles are compact in space.
// The histogram does not depend on the order of particles within a species.
struct SortSeg {
  const FrameDev* fd;
  int64_t x0;        // first particle (index into the packed coordinates)
  int32_t n;         // particles
  int32_t g;         // grid bits per axis
  int64_t key0;      // first counter of this segment (2^(3g) counters)
};
constexpr int kSortChunk = 4096;

struct Control {
  unsigned long long next_item;  // dynamic work counter (reset before each launch)
  int32_t status;                // 0 ok, else an error code
  int32_t pad;
};

struct PairLaunch {
  const Segment* segs;
  int32_t n_segs;
  int32_t hist_width;  // shared-memory bins per histogram copy (the widest sweep of the launch)
  int64_t n_items;
  Control* ctl;
  int32_t hist_depth;  // private histogram copies per block (warp w uses copy w mod depth); 0 means 1
  int32_t multi;       // nonzero when some sweep of the launch starts above bin 0
  int32_t block;       // threads per block: kBlockSmall (0 means it), kBlockLarge or kBlockHuge
  int32_t agg;         // 256-thread blocks, one sweep: warp-aggregated histogram increments (match.any)
};

// ---- launchers (dh_kernels.cu); all enqueue on `stream` and return the launch error
cudaError_t launch_stage(const StageJob* jobs, int n_jobs, int64_t n_chunks, cudaStream_t stream);
cudaError_t launch_frame_setup(FrameDev* frames, int n_frames, int pass_hi_max, cudaStream_t stream);
// counts: zeroed, sum of 2^(3g) over the segments; keys and Xs: one per particle
// X64 and Xs64 (binary64 copies, same indexing) may be null
cudaError_t launch_spatial_sort(const SortSeg* segs, int n_segs, int max_chunks, float4* X, float4* Xs,
                                double4* X64, double4* Xs64, int32_t* keys, uint32_t* counts,
                                cudaStream_t stream);
cudaError_t launch_thresholds(double r_max, int32_t nbins, double* T, int32_t* status,
                              cudaStream_t stream);
// One pair-kernel launch over segments whose frames all have minimum-image variant `variant`.
cudaError_t launch_pairs(const PairLaunch& p, int variant, int grid, size_t smem, cudaStream_t stream);
cudaError_t launch_check_sqrt(unsigned long long* out, cudaStream_t stream);
cudaError_t launch_check_tiles(const FrameDev* F, int variant, uint64_t n_tiles, uint64_t seed,
                               unsigned long long* out, cudaStream_t stream);
cudaError_t launch_check_window(const FrameDev* F, uint64_t n_samples, uint64_t seed, unsigned long long* out,
                                cudaStream_t stream);
cudaError_t launch_rdf(const uint64_t* counts, int32_t n_hist, int32_t nbins, double r_max,
                       const double* pair_density, uint64_t n_frames, double* g, cudaStream_t stream);
size_t pair_kernel_smem(int hist_width, int depth = 1, int block = kBlockSmall);
int pair_kernel_max_width();
int pair_kernel_blocks_per_sm(int variant, int hist_width, int depth = 1, int block = kBlockSmall);

// Host/device shared definition of the binary64 bin of Alg. 1 (used to build thresholds).
int64_t host_bin_of(double r2, double r_max, int32_t nbins);
int build_thresholds_host(double r_max, int32_t nbins, double* T);

}  // namespace dh
