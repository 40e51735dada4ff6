// dh_histogram_noalloc: the histogram of one frame without allocating memory.
//
// The regular entry points keep their workspace (packed coordinates, the
// binary64 threshold table, frame and work descriptors, the work counter) in
// device memory that the context allocates with cudaMalloc on first use.  Some
// callers cannot allow that: code inside a framework whose device memory is
// owned by its own allocator (a cudaMalloc behind its back fragments or
// overcommits the pool it manages), or a process that runs under a fixed
// device-memory budget, must not trigger new device allocations.  This variant
// takes device input and output from the
// caller and keeps all of its scratch in one file-scope __device__ array of a
// fixed size, so it never calls cudaMalloc, cudaFree or any other allocating
// routine.  The paper has no counterpart of it.
//
// The array is reserved on every GPU that loads the library and is kept until
// the process exits.  All calls share it: a call clears what must start at
// zero, and calls whose GPU work overlaps (different streams, host threads or
// processes sharing one context) race on it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "dh_runtime.h"

namespace dh {
namespace {

// Scratch layout (bytes, each part 256-byte aligned).
constexpr size_t kNaCtl = 256;                                  // Control
constexpr size_t kNaFrame = 2048;                               // FrameDev
constexpr size_t kNaJob = 256;                                  // StageJob
constexpr size_t kNaSegs = 16 * 1024;                           // Segment[] (256 of them)
constexpr size_t kNaT = ((size_t)DH_NOALLOC_MAX_BINS + 1) * 16; // thresholds + float-pair copy
constexpr size_t kNaTPad = (kNaT + 255) & ~(size_t)255;
constexpr size_t kNaX = (size_t)DH_NOALLOC_MAX_N * 16;          // float4 coordinates
constexpr size_t kNaOffFrame = kNaCtl;
constexpr size_t kNaOffJob = kNaOffFrame + kNaFrame;
constexpr size_t kNaOffSegs = kNaOffJob + kNaJob;
constexpr size_t kNaOffT = kNaOffSegs + kNaSegs;
constexpr size_t kNaOffX = kNaOffT + kNaTPad;
constexpr size_t kNaBytes = kNaOffX + kNaX;
static_assert(kNaBytes == DH_NOALLOC_SCRATCH_BYTES, "scratch size must match the value published in dh.h");
static_assert(sizeof(FrameDev) <= kNaFrame && sizeof(StageJob) <= kNaJob && sizeof(Control) <= kNaCtl,
              "scratch slots too small");
constexpr int kNaMaxSegs = (int)(kNaSegs / sizeof(Segment));
constexpr int kNaMaxDevices = 64;

// The scratch itself.  Host code must not pass this name to a kernel: on the
// host it is only a stand-in; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

std::mutex g_na_mu;
unsigned char* g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.
dh_status scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  DH_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) return fail(DH_ERR_INVALID, "device %d out of range", dev);
  std::lock_guard<std::mutex> g(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(DH_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_na_ptr[dev] = (unsigned char*)p;
  }
  *out = g_na_ptr[dev];
  return DH_OK;
}

}  // namespace
}  // namespace dh

using namespace dh;

extern "C" dh_status dh_histogram_noalloc(const dh_frame* frame, void* stream_ptr) {
  if (!frame) return fail(DH_ERR_INVALID, "frame is NULL");
  if (!(frame->flags & DH_DEVICE_PTRS))
    return fail(DH_ERR_INVALID, "dh_histogram_noalloc needs DH_DEVICE_PTRS (device coords and out)");
  if (frame->flags & DH_COORDS_F64)
    return fail(DH_ERR_INVALID, "dh_histogram_noalloc takes float32 coordinates");
  if (frame->n > DH_NOALLOC_MAX_N)
    return fail(DH_ERR_INVALID, "n = %lld exceeds the allocation-free limit of %d particles",
                (long long)frame->n, DH_NOALLOC_MAX_N);
  if (frame->nbins > DH_NOALLOC_MAX_BINS)
    return fail(DH_ERR_INVALID, "nbins = %d exceeds the allocation-free limit of %d bins", frame->nbins,
                DH_NOALLOC_MAX_BINS);
  int dev = -1;
  DH_CUDA_TRY(cudaGetDevice(&dev));
  int num_sms = 0, max_width = 0;
  DH_CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  max_width = pair_kernel_max_width();
  if (max_width < 1024) return fail(DH_ERR_CUDA, "not enough shared memory per block");
  PlannedFrame pf;
  dh_status s = check_frame(frame, pf, max_width);
  if (s != DH_OK) return s;
  unsigned char* base = nullptr;
  s = scratch_for_current_device(&base);
  if (s != DH_OK) return s;
  cudaStream_t st = (cudaStream_t)stream_ptr;

  Control* ctl = (Control*)(base);
  FrameDev* fd = (FrameDev*)(base + kNaOffFrame);
  StageJob* job = (StageJob*)(base + kNaOffJob);
  Segment* segs = (Segment*)(base + kNaOffSegs);
  double* T = (double*)(base + kNaOffT);
  float4* X = (float4*)(base + kNaOffX);

  // Every host-side check comes before the first enqueued operation, so that a
  // call that fails leaves the caller's output and the shared scratch untouched.
  Segment hS[kNaMaxSegs];
  int n_segs = 0;
  const int64_t n_items = fill_segments(pf, fd, 0, 1, hS, kNaMaxSegs, &n_segs);
  if (n_segs > kNaMaxSegs)
    return fail(DH_ERR_INVALID, "%d species x %d sweeps need %d work segments, beyond the allocation-free limit of %d",
                frame->n_species, pf.sweeps, n_segs, kNaMaxSegs);
  const int block = default_block(pf.variant, pf.sweep_width);
  const int bps = n_items > 0 ? pair_kernel_blocks_per_sm(pf.variant, pf.sweep_width, 1, block) : 1;
  if (bps < 1) return fail(DH_ERR_INVALID, "histogram of %d bins does not fit in shared memory", pf.sweep_width);

  // Host-side descriptors live on the stack; the copies below read them before returning.
  FrameDev hF;
  fill_frame_dev(pf, hF, X, frame->out, T);
  StageJob hJ;
  std::memset(&hJ, 0, sizeof hJ);
  hJ.src = frame->coords;
  hJ.dst = X;
  hJ.fd = fd;
  hJ.n = frame->n;
  hJ.stride = (frame->flags & DH_COORDS_F4) ? 4 : 3;
  hJ.chunk0 = 0;
  size_t out_bytes = sizeof(uint64_t) * (size_t)pf.n_hist * (size_t)frame->nbins;

  // Clear what must start at zero, upload descriptors, build the table, stage, run.
  DH_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(Control), st));
  DH_CUDA_TRY(cudaMemcpyAsync(fd, &hF, sizeof(FrameDev), cudaMemcpyHostToDevice, st));
  DH_CUDA_TRY(cudaMemcpyAsync(job, &hJ, sizeof(StageJob), cudaMemcpyHostToDevice, st));
  if (n_segs > 0) DH_CUDA_TRY(cudaMemcpyAsync(segs, hS, sizeof(Segment) * n_segs, cudaMemcpyHostToDevice, st));
  if (!(frame->flags & DH_ACCUMULATE)) DH_CUDA_TRY(cudaMemsetAsync(frame->out, 0, out_bytes, st));
  DH_CUDA_TRY(launch_thresholds(frame->r_max, frame->nbins, T, &ctl->status, st));
  int64_t chunks = (frame->n + kStageChunk - 1) / kStageChunk;
  if (chunks > 0) DH_CUDA_TRY(launch_stage(job, 1, chunks, st));
  DH_CUDA_TRY(launch_frame_setup(fd, 1, 0, st));
  if (n_items > 0) {
    PairLaunch L;
    std::memset(&L, 0, sizeof L);
    L.block = block;
    L.segs = segs;
    L.n_segs = n_segs;
    L.n_items = n_items;
    L.hist_width = pf.sweep_width;
    L.multi = pf.sweeps > 1;
    L.ctl = ctl;
    DH_CUDA_TRY(launch_pairs(L, pf.variant, pair_grid(num_sms, bps, n_items),
                             pair_kernel_smem(pf.sweep_width, 1, block), st));
  }
  // Read back the flags into stack memory and wait.
  int32_t status = 0, bad = 0;
  DH_CUDA_TRY(cudaMemcpyAsync(&status, &ctl->status, sizeof status, cudaMemcpyDeviceToHost, st));
  DH_CUDA_TRY(cudaMemcpyAsync(&bad, &fd->bad, sizeof bad, cudaMemcpyDeviceToHost, st));
  DH_CUDA_TRY(cudaStreamSynchronize(st));
  if (status != 0) return fail(DH_ERR_CUDA, "bin threshold table did not converge");
  if (bad) return fail(DH_ERR_INVALID, "frame has non-finite coordinates");
  return DH_OK;
}
