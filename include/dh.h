/*
 * dh.h — C ABI of the GB300 particle-pair distance histogram library (libdh.so).
 *
 * What it computes (Reuter & Koefinger, "CADISHI", Sec. 2):
 *   For one trajectory frame of N particles split into S species (contiguous
 *   segments of the coordinate array), every unique pair is binned by its
 *   distance: intra-species pairs i < j (single-species variant of Alg. 1,
 *   Sec. 2.2) and inter-species pairs, all i in species a and j in species b
 *   (Alg. 1).  Periodic boxes apply the minimum image convention of Eq. 5
 *   (orthorhombic: diagonal B, Sec. 2.3; triclinic: general B plus the
 *   neighbouring-cell search of Sec. 2.3).  The bin of a pair is
 *   kappa = (int) nbins * r / r_max (Alg. 1), bins are half open
 *   [kappa dr, (kappa+1) dr) (Eq. 4), and pairs with kappa >= nbins are not
 *   counted.  Counts are exact unsigned 64-bit integers.
 *
 * Exactness: the result equals, bin for bin, the histogram obtained when every
 * step above is evaluated in IEEE binary64 in this order: d = xj - xi
 * (coordinates promoted exactly from float32); orthorhombic
 * k = nearbyint(d * (1/L)), d = fma(-k, L, d); triclinic s = B^-1 d by back
 * substitution, k = nearbyint(s), d -= B k, then the minimum of |d + B m|^2
 * over m in {-1,0,1}^3; r^2 = fma(dz,dz, fma(dy,dy, dx*dx));
 * kappa = floor((nbins * sqrt(r^2)) / r_max).  Most pairs are decided in
 * float32 arithmetic whose error is bounded; pairs whose float32 value lies
 * within that bound of a bin edge are re-decided with higher precision.
 *
 * Histogram order: the S(S+1)/2 histograms of species pairs (a,b), a <= b, are
 * stored one after another in the order (0,0),(0,1),...,(0,S-1),(1,1),...,
 * i.e. histogram h(a,b) = a*S - a*(a-1)/2 + (b-a) occupies
 * out[h*nbins .. h*nbins + nbins).
 *
 * Box matrix: 9 doubles, row-major 3x3 whose COLUMNS are the box vectors
 * a, b, c (the matrix B of Eq. 5).  DH_BOX_ORTHO requires a diagonal B with
 * positive entries.  DH_BOX_TRICLINIC requires an upper-triangular B
 * (a = (ax,0,0), b = (bx,by,0), c = (cx,cy,cz)) with positive diagonal, in
 * reduced form: |bx| <= ax/2, |cx| <= ax/2, |cy| <= by/2.
 *
 * Errors: every entry point returns a dh_status; nothing throws across the
 * ABI.  On DH_ERR_* the output buffer is unspecified (it may be partly
 * written) and dh_last_error() describes the failure.
 *
 * Threads: one dh_ctx may be used from several host threads; calls on one
 * context are serialised internally.
 */
#ifndef DH_H
#define DH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DH_OK = 0,
  DH_PENDING = 1,          /* dh_poll: the request has not finished yet */
  DH_ERR_INVALID = -1,     /* bad argument: offsets, nbins, r_max, box, non-finite coordinates */
  DH_ERR_NOMEM = -2,       /* device or pinned host memory could not be obtained */
  DH_ERR_CUDA = -3,        /* a CUDA call failed (message in dh_last_error) */
  DH_ERR_TIMEOUT = -4,     /* dh_wait ran out of time, or a served request passed its deadline */
  DH_ERR_CANCELLED = -5,   /* the request was cancelled before it finished */
  DH_ERR_NOTFOUND = -6     /* unknown ticket */
} dh_status;

typedef enum { DH_BOX_NONE = 0, DH_BOX_ORTHO = 1, DH_BOX_TRICLINIC = 2 } dh_box_type;

/* dh_frame.flags */
#define DH_DEVICE_PTRS 0x1u /* coords and out are device pointers (same device as the context) */
#define DH_ACCUMULATE 0x2u  /* add into out instead of overwriting it */
#define DH_COORDS_F4 0x4u   /* coords are n x 4 floats (x,y,z,ignored) instead of n x 3 */
#define DH_COORDS_F64 0x8u  /* coords point to binary64 values (cast the pointer): the distance vector
                               is then rounded once per component, as the binary64 definition does;
                               plain and batched paths only (dh_submit and dh_histogram_noalloc
                               return DH_ERR_INVALID) */

/* dh_config.flags */
#define DH_CFG_NO_GRAPH 0x1u /* batched path: launch directly instead of replaying a CUDA graph */
#define DH_CFG_TIMING 0x2u   /* record CUDA events around the pair-kernel launches (dh_stats.pair_kernel_ms) */
#define DH_CFG_AUTOTUNE 0x4u /* plain and batched paths: measure the launch shapes (j-tile length,
                                threads per block, private histogram copies per block, blocks per
                                SM) of every new launch key on a synthetic batch of its shape
                                before the first call that needs it, and use the fastest; see
                                dh_tune_cache_count */

typedef struct dh_ctx dh_ctx;

typedef struct {
  int32_t device;        /* CUDA device ordinal */
  uint64_t pool_bytes;   /* served path: device memory the admission control may use (0: 1/2 of free) */
  int32_t max_inflight;  /* served path: most requests resident on the device at once (0: 64) */
  uint64_t timeout_ns;   /* served path: deadline of a request, counted from its dh_submit; a request
                            not finished by then is cancelled and reports DH_ERR_TIMEOUT (0: none) */
  const char* tune_cache;/* autotuner cache file (read at dh_create, rewritten after each new
                            measurement), or NULL for in-memory only */
  uint32_t flags;        /* DH_CFG_* */
  uint32_t wave_us;      /* served path: target device time of one wave in microseconds (0: 6000) */
} dh_config;

typedef struct {
  const float* coords;             /* n x 3 (or n x 4 with DH_COORDS_F4) float32 (binary64 with
                                      DH_COORDS_F64), species contiguous */
  int64_t n;                       /* number of particles, >= 0 */
  const int64_t* species_offsets;  /* HOST array of n_species+1 entries: 0 = o[0] <= o[1] <= ... <= o[S] = n */
  int32_t n_species;               /* S >= 1 */
  int32_t box_type;                /* dh_box_type */
  double box[9];                   /* box matrix (ignored for DH_BOX_NONE) */
  double r_max;                    /* upper end of the histogram, > 0 and finite */
  int32_t nbins;                   /* number of bins, 1 <= nbins <= DH_MAX_BINS */
  uint64_t* out;                   /* S(S+1)/2 x nbins counts */
  uint32_t flags;                  /* DH_DEVICE_PTRS | DH_ACCUMULATE | DH_COORDS_F4 | DH_COORDS_F64 */
} dh_frame;

/* 2^22 - 64: the float32 bin coordinate, clamped a few bins beyond the last
   one, must stay below 2^22 for its nearest-integer step to be exact. */
#define DH_MAX_BINS 4194240

/* Per-context statistics of the most recent dh_histogram / dh_histogram_batch call. */
typedef struct {
  uint64_t pairs;          /* unique pairs evaluated */
  uint64_t deferred;       /* pairs whose float32 value fell within the error bound of an edge */
  uint64_t exact_fallback; /* deferred pairs that needed the binary64 replay */
  int32_t sweeps;          /* passes over the pairs (histogram wider than shared memory) */
  int32_t blocks;          /* CUDA blocks launched for the pair kernel */
  int32_t items;           /* work items (tile pairs) */
  int32_t kernel_launches; /* kernels launched by the call */
  int32_t graph_replays;   /* 1 when the call ran as a replayed CUDA graph */
  int32_t tune_runs;       /* autotuner measurement launches made before the call (DH_CFG_AUTOTUNE) */
  double pair_kernel_ms;   /* device time of the pair-kernel launches (needs DH_CFG_TIMING), else 0 */
  int32_t tile_j;          /* launch shape of the largest pair-kernel launch: j-tile length, */
  int32_t hist_depth;      /*   private histogram copies per block (warp w uses copy w mod depth), */
  int32_t blocks_per_sm;   /*   blocks per SM */
  int32_t block_threads;   /*   and threads per block */
  uint64_t uniform_pairs;  /* pairs evaluated with one nearest image for their whole tile (no per-pair rounding) */
  uint64_t axis_pairs;     /* pairs whose tile image is uniform on all axes but one (that axis wrapped per pair) */
  int32_t warp_agg;        /* 1 when the largest launch aggregated its increments per warp (tune cache agg) */
  int32_t reserved;
  uint64_t culled_pairs;   /* pairs (counted once per bin sweep) of tiles skipped because their distance
                              bounds put no pair in the sweep's bins (periodic frames) */
} dh_stats;

/* Create a context on config->device (NULL: device 0, defaults).  Owns a CUDA
 * stream, device workspace and pinned host staging buffers, all released by
 * dh_destroy.  *out receives the context. */
dh_status dh_create(const dh_config* config, dh_ctx** out);

/* Release everything the context owns.  Pending served requests are cancelled. */
dh_status dh_destroy(dh_ctx* ctx);

/* Use the given cudaStream_t (passed as void*) for subsequent device work of
 * dh_histogram / dh_histogram_batch; NULL restores the context's own stream. */
dh_status dh_set_stream(dh_ctx* ctx, void* stream);

/* Histograms of one frame: Alg. 1 (Sec. 2.2) over every species pair, with
 * the minimum image of Eq. 5 for periodic boxes and the bins of Eq. 4.
 * Synchronous: on return, out holds the result.  With DH_DEVICE_PTRS the work
 * runs on the context stream and the call waits for it. */
dh_status dh_histogram(dh_ctx* ctx, const dh_frame* frame);

/* Like dh_histogram, but with DH_DEVICE_PTRS it only enqueues the work on the
 * context stream and returns; errors found on the device are reported by the
 * next synchronous call (or dh_sync). */
dh_status dh_histogram_async(dh_ctx* ctx, const dh_frame* frame);

/* Wait for work enqueued by dh_histogram_async and report device-side errors. */
dh_status dh_sync(dh_ctx* ctx);

/* k frames of possibly different N, species, box and nbins (the frame-by-frame
 * workload of the paper's engine, Sec. 3.3) through one persistent pair-kernel
 * launch per minimum-image variant present, all bin sweeps included.  All
 * frames must use the same pointer kind (all DH_DEVICE_PTRS or none).  With
 * device pointers the launch sequence is captured as a CUDA graph and replayed
 * (unless DH_CFG_NO_GRAPH).  Synchronous. */
dh_status dh_histogram_batch(dh_ctx* ctx, const dh_frame* frames, int32_t k);

/* Served path: submit one frame as a request.  Coordinates and output stay on
 * the device (DH_DEVICE_PTRS) or are staged by the library (host pointers);
 * the caller's buffers must stay valid and unmodified until dh_poll/dh_wait
 * report a final status.  Admission is by device-memory footprint; requests
 * that do not fit wait in a queue.  *ticket identifies the request. */
dh_status dh_submit(dh_ctx* ctx, const dh_frame* frame, uint64_t* ticket);

/* DH_PENDING while the request runs, then its final status (once). */
dh_status dh_poll(dh_ctx* ctx, uint64_t ticket);

/* Block until the request finishes or timeout_ns passes (DH_ERR_TIMEOUT). */
dh_status dh_wait(dh_ctx* ctx, uint64_t ticket, uint64_t timeout_ns);

/* Cancel a queued or running request; its output is left unspecified. */
dh_status dh_cancel(dh_ctx* ctx, uint64_t ticket);

/* Radial distribution function g(r) of Eq. 1 from histograms summed over the
 * frames of a trajectory (Eqs. 2-4; sum the frames into one histogram with
 * DH_ACCUMULATE).  For each of n_hist histograms of nbins bins:
 *   g[h][k] = (counts[h][k] / n_frames) / (pair_density[h] * (4 pi / 3)(r_{k+1}^3 - r_k^3)),
 * r_k = k r_max / nbins: the mean pairs per frame in bin k over the pairs that a
 * uniform pair density puts in its spherical shell (the finite-bin form of the
 * 4 pi r^2 dr of Eq. 1).  pair_density is a host array of n_hist values N_pairs / V
 * (N_a (N_a - 1) / 2 / V within a species, N_a N_b / V between two; the caller
 * chooses V, e.g. the box volume, or its average over the frames).  counts
 * (uint64) and g (double) are device pointers on the context's device, n_hist x
 * nbins row-major.  Binary64 arithmetic on the GPU, on the context's stream; the
 * call returns when g is written.  DH_ERR_INVALID: NULL pointers, n_hist < 1,
 * nbins outside [1, DH_MAX_BINS], r_max not > 0 and finite, n_frames = 0, or a
 * pair density not > 0 and finite. */
dh_status dh_rdf(dh_ctx* ctx, const uint64_t* counts, int32_t n_hist, int32_t nbins, double r_max,
                 const double* pair_density, uint64_t n_frames, double* g);

/* Statistics of the last dh_histogram / dh_histogram_batch call on ctx. */
dh_status dh_get_stats(dh_ctx* ctx, dh_stats* stats);

/* Message describing the last error on this host thread (owned by the library). */
const char* dh_last_error(dh_ctx* ctx);

/* Host-only helper, no GPU needed: the binary64 bin thresholds used for exact
 * decisions.  thresholds[0] = 0 and, for 1 <= k <= nbins, thresholds[k] is the
 * smallest binary64 value q >= 0 with floor((nbins * sqrt(q)) / r_max) >= k;
 * a pair with r^2 = q lies in bin k iff thresholds[k] <= q < thresholds[k+1],
 * and is counted iff q < thresholds[nbins].  thresholds must hold nbins+1 doubles. */
dh_status dh_bin_thresholds(double r_max, int32_t nbins, double* thresholds);

/* Host-only helper, no GPU needed: reads an autotuner cache file, the text file
 * that dh_create reads and the autotuner rewrites (DH_CFG_AUTOTUNE with
 * dh_config.tune_cache): lines starting with '#' are comments, every other line
 * is one launch key and its measured shape,
 *   sms variant width_log2 n_log2 frames_log4 tile_j block depth bps gpairs_s [agg]
 * (variant: 0 none, 1 orthorhombic, 2 triclinic, 3 triclinic with the
 * 27-image search; width_log2 = ceil(log2 of the shared-memory histogram
 * width); n_log2 = round(log2 of the mean particles per frame); frames_log4 =
 * min(3, floor(log4 of the frames per launch)); tile_j in {256, 512, 1024};
 * block, the threads per block, in {256, 512, 1024}; depth in {1, 2, 4, 8}; bps, the
 * blocks per SM, >= 1 (at most what fits is used); gpairs_s > 0; agg, optional,
 * 1 for warp-aggregated histogram increments (match.any: the lanes of a warp
 * that hit one bin add their count once), only with 256-thread blocks and a
 * single bin sweep, else 0).  *n_entries receives the number
 * of distinct launch keys with a well-formed line for a GPU with sm_count SMs
 * (a later line replaces an earlier one of the same key); lines for other SM
 * counts and malformed lines are skipped.  DH_ERR_NOTFOUND if the file cannot
 * be read. */
dh_status dh_tune_cache_count(const char* path, int32_t sm_count, int32_t* n_entries);

/* Diagnostics of the float32 decision rule (not part of the histogram).
 *  what = DH_CHECK_SQRT: out[0] = largest relative error of the float32 square
 *    root of the fast path over every float in [1, 4), against the correctly
 *    rounded value; the window derivation assumes at most 2^-21.
 *  what = DH_CHECK_WINDOW: stages `frame` (as dh_histogram would) and evaluates
 *    n_samples pairs (i, j) drawn with splitmix64 from `seed`: out[0] = largest
 *    |t32 - t64| / delta, where t = nbins * r / r_max in float32 (fast path) and
 *    binary64 (definition) and delta is the frame's decision window (must be
 *    < 1); out[1] = sampled pairs the float32 path would decide whose bin differs
 *    from the binary64 bin (must be 0); out[2] = pairs compared; out[3] = delta.
 *  what = DH_CHECK_TILES (orthorhombic or triclinic frames without search):
 *    stages `frame` and draws n_samples tiles with splitmix64 from `seed`, each
 *    a run of 128 consecutive particles against a run of 256 (the pair kernel's
 *    warp tiles, in the staged order); every pair of a tile is evaluated in the
 *    tile's image mode with the tile's own window, as the pair kernel does:
 *    out[0] = largest |t32 - t64| / (alpha t64 + beta_tile) (must be < 1),
 *    out[1] = pairs decided in float32 with a bin other than the binary64 one
 *    (must be 0), out[2] = pairs compared, out[3] = tiles drawn that took a
 *    shifted (uniform or one-axis) mode.  DH_ERR_INVALID for other boxes.
 * out must hold 4 doubles.  Synchronous. */
#define DH_CHECK_SQRT 0
#define DH_CHECK_WINDOW 1
#define DH_CHECK_TILES 2
dh_status dh_selfcheck(dh_ctx* ctx, int32_t what, const dh_frame* frame, uint64_t n_samples, uint64_t seed,
                       double* out);

/* Diagnostics: throughput of one GPU pipe that the pair kernel runs on (the
 * paper sizes its kernels from measured occupancy and throughput, Sec. 3.2.4
 * and Sec. 4.2; these are the ceilings the pair kernel's rate is compared
 * with).  Runs one microbenchmark on `device`: a single wave of blocks keeping
 * every resident warp busy with independent instances of one instruction, after
 * a warm-up launch.  out (4 doubles): out[0] = operations per clock per SM (from
 * the SM cycle counter), out[1] = operations per second, out[2] = the SM clock
 * in MHz over the measured launch, out[3] = its duration in ms.  An operation
 * is one lane's result (a packed float32x2 instruction counts 2), one shared or
 * global atomic, one match.  width: histogram bins of the atomic benchmarks
 * (shared: 64..57,344 uint32 bins of one block-private histogram; cluster:
 * 64 c..57,344 c bins over a cluster of c blocks; global: 64..2^24 uint64
 * bins), ignored otherwise.  The call allocates and frees a few
 * small device buffers and its own stream.  DH_ERR_INVALID for an unknown pipe
 * or a width out of range. */
#define DH_PIPE_FFMA2 0                 /* fma.rn.f32x2 */
#define DH_PIPE_FADD2 1                 /* add.rn.f32x2 */
#define DH_PIPE_FMUL2 2                 /* mul.rn.f32x2 */
#define DH_PIPE_FFMA 3                  /* fma.rn.f32 */
#define DH_PIPE_SQRT 4                  /* sqrt.approx.ftz.f32 (MUFU) */
#define DH_PIPE_FRND 5                  /* cvt.rni.f32.f32 */
#define DH_PIPE_F2I 6                   /* cvt.rni.s32.f32 */
#define DH_PIPE_LOP3 7                  /* lop3.b32 */
#define DH_PIPE_IADD 8                  /* add.u32 */
#define DH_PIPE_IMAD 9                  /* mad.lo.u32 */
#define DH_PIPE_DFMA 10                 /* fma.rn.f64 */
#define DH_PIPE_MATCH 11                /* match.any.sync.b32 */
#define DH_PIPE_SMEM_ATOMIC_RANDOM 12   /* red.shared.add.u32, uniform random bins */
#define DH_PIPE_SMEM_ATOMIC_CLUSTERED 13 /* the same, the 32 lanes of a warp on 4 neighbouring bins */
#define DH_PIPE_SMEM_ATOMIC_SAME 14     /* the same, all lanes of a warp on one bin */
#define DH_PIPE_SMEM_ATOMIC_SEQUENTIAL 15 /* the same, lane l on bin base + l (no bank conflict) */
#define DH_PIPE_GLOBAL_ATOMIC64 16      /* atom.global.add.u64, uniform random bins */
#define DH_PIPE_DSMEM_ATOMIC_C2 17      /* red.shared::cluster.add.u32: one histogram split over a cluster of 2, */
#define DH_PIPE_DSMEM_ATOMIC_C4 18      /*   4 or 8 blocks (width = the whole histogram), uniform random bins, */
#define DH_PIPE_DSMEM_ATOMIC_C8 19      /*   most of them in another block's shared memory */
dh_status dh_pipe_rate(int32_t device, int32_t pipe, int32_t width, double* out);

/* Allocation-free histogram (the paper has no counterpart of this entry point).
 *
 * For callers that must not allocate device memory: frameworks whose device
 * memory belongs to their own caching allocator (a cudaMalloc behind its back
 * fragments or overcommits the pool it manages), and processes that run under
 * a fixed device-memory budget.  Every other entry point keeps its workspace in
 * memory the context obtains with cudaMalloc; this one needs no context and
 * calls no cudaMalloc, cudaFree or other allocating routine.  It computes
 * exactly what dh_histogram computes.
 *
 * frame->flags must contain DH_DEVICE_PTRS: coords and out are device
 * pointers on the current device (species_offsets stays a host array); the
 * work runs on `stream` (a cudaStream_t, NULL for the default stream) and the
 * call returns when it has finished.  Scratch memory is one file-scope device
 * array of DH_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds
 * until the process exits; limits: n <= DH_NOALLOC_MAX_N, nbins <=
 * DH_NOALLOC_MAX_BINS, at most 256 species-pair work segments (n_species <= 15
 * when one bin sweep suffices).  Larger frames return DH_ERR_INVALID before
 * any work is enqueued (out and the scratch are then left untouched).
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the array: each call clears what must start at
 * zero, and calls whose GPU work overlaps (other streams, host threads) race
 * on it and must be serialised by the caller. */
#define DH_NOALLOC_MAX_N 131072
#define DH_NOALLOC_MAX_BINS 65536
#define DH_NOALLOC_SCRATCH_BYTES 3164928
dh_status dh_histogram_noalloc(const dh_frame* frame, void* stream);

/* Library version string. */
const char* dh_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DH_H */
