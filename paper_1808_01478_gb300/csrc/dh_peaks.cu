// Throughput of the GPU pipes the pair kernel runs on (diagnostics).
//
// The paper tunes its kernels against occupancy and throughput measurements of
// the GPUs it targets (Sec. 3.2.4, Sec. 4.2); this file measures the same kind
// of ceilings on the GPU at hand, so that the pair kernel's rate can be stated
// as a fraction of measured per-pipe peaks rather than of nominal unit counts.
// Each microbenchmark keeps every warp slot of every SM busy with long runs of
// independent instances of one instruction and reports operations per clock
// per SM (from clock64 on each SM) and per second (from CUDA events), so that
// the rate can be scaled to the clock observed under any other load.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "dh_runtime.h"

namespace dh {
namespace {

constexpr int kPeakBlock = 256;

__device__ __forceinline__ uint64_t clk64() {
  uint64_t c;
  asm volatile("mov.u64 %0, %%clock64;" : "=l"(c));
  return c;
}

__device__ __forceinline__ uint64_t gtimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Per block: the SM cycles and the nanoseconds of the global timer between
// its first and last instruction, summed over the blocks (cycles[0], cycles[1]):
// their ratio is the SM clock over the launch, whether its blocks ran in one
// wave or several.
__device__ __forceinline__ void record_cycles(uint64_t t0, uint64_t g0, unsigned long long* cycles) {
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(cycles, (unsigned long long)(clk64() - t0));
    atomicAdd(cycles + 1, (unsigned long long)(gtimer_ns() - g0));
  }
}

// A result the compiler cannot drop: stored only when it takes a value that the
// compiler cannot rule out but the inputs never produce.
__device__ __forceinline__ void keep(float v, float* sink) {
  if (v == -1.2345e-30f) sink[threadIdx.x] = v;
}
__device__ __forceinline__ void keep_u(uint32_t v, float* sink) {
  if (v == 0x9E3779B9u) sink[threadIdx.x] = 1.0f;
}

// Packed float32: `iters` x 8 independent FFMA2 / FADD2 / FMUL2 per thread (2 lane operations each).
template <int OP>
__global__ void __launch_bounds__(kPeakBlock, 8) packed_kernel(int iters, float* sink, unsigned long long* cycles) {
  float2 a[8];
  for (int k = 0; k < 8; ++k) a[k] = make_float2(1.0f + 1e-3f * k + 1e-6f * threadIdx.x, 0.5f + 1e-3f * k);
  const float2 b = make_float2(0.99999f, 0.99998f), c = make_float2(1e-6f, -1e-6f);
  __syncthreads();
  const uint64_t g0 = gtimer_ns(), t0 = clk64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (OP == 0) a[k] = __ffma2_rn(a[k], b, c);
      else if (OP == 1) a[k] = __fadd2_rn(a[k], c);
      else a[k] = __fmul2_rn(a[k], b);
    }
  }
  record_cycles(t0, g0, cycles);
  float s = 0.f;
  for (int k = 0; k < 8; ++k) s += a[k].x + a[k].y;
  keep(s, sink);
}

// Scalar float32 FFMA: `iters` x 16 independent per thread.
__global__ void __launch_bounds__(kPeakBlock, 8) ffma_kernel(int iters, float* sink, unsigned long long* cycles) {
  float a[16];
  for (int k = 0; k < 16; ++k) a[k] = 1.0f + 1e-3f * k + 1e-6f * threadIdx.x;
  const float b = 0.99999f, c = 1e-6f;
  __syncthreads();
  const uint64_t g0 = gtimer_ns(), t0 = clk64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = __fmaf_rn(a[k], b, c);
  }
  record_cycles(t0, g0, cycles);
  float s = 0.f;
  for (int k = 0; k < 16; ++k) s += a[k];
  keep(s, sink);
}

// Special-function and conversion units: `iters` x 8 independent instructions per thread.
//  OP 0: sqrt.approx.ftz.f32 (the fast path's square root)
//  OP 1: cvt.rni.f32.f32 (round to integral, FRND)
//  OP 2: cvt.rni.s32.f32 (float to int, F2I), folded into the next input with one LOP3
template <int OP>
__global__ void __launch_bounds__(kPeakBlock, 8) xu_kernel(int iters, float* sink, unsigned long long* cycles) {
  float a[8];
  uint32_t acc = 0;
  for (int k = 0; k < 8; ++k) a[k] = 2.0f + 0.37f * k + 1e-3f * threadIdx.x;
  __syncthreads();
  const uint64_t g0 = gtimer_ns(), t0 = clk64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (OP == 0) {
        asm volatile("sqrt.approx.ftz.f32 %0, %0;" : "+f"(a[k]));
      } else if (OP == 1) {
        asm volatile("cvt.rni.f32.f32 %0, %0;" : "+f"(a[k]));
      } else {
        int v;
        asm volatile("cvt.rni.s32.f32 %0, %1;" : "=r"(v) : "f"(a[k]));
        acc ^= (uint32_t)v;
      }
    }
  }
  record_cycles(t0, g0, cycles);
  float s = 0.f;
  for (int k = 0; k < 8; ++k) s += a[k];
  keep(s, sink);
  keep_u(acc, sink);
}

// Integer ALU / IMAD: `iters` x 8 independent instructions per thread.
//  OP 0: lop3 (x = x ^ y ^ z), OP 1: iadd3, OP 2: imad
template <int OP>
__global__ void __launch_bounds__(kPeakBlock, 8) int_kernel(int iters, float* sink, unsigned long long* cycles) {
  uint32_t a[8];
  const uint32_t y = 0x9E3779B9u ^ threadIdx.x, z = 0x7F4A7C15u + blockIdx.x;
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 2654435761u + k;
  __syncthreads();
  const uint64_t g0 = gtimer_ns(), t0 = clk64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (OP == 0) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[k]) : "r"(y), "r"(z));
      else if (OP == 1) asm volatile("add.u32 %0, %0, %1;\n\tadd.u32 %0, %0, %2;" : "+r"(a[k]) : "r"(y), "r"(z));
      else asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(y), "r"(z));
    }
  }
  record_cycles(t0, g0, cycles);
  uint32_t s = 0;
  for (int k = 0; k < 8; ++k) s ^= a[k];
  keep_u(s, sink);
}

// Binary64 FMA: `iters` x 8 independent DFMA per thread.
__global__ void __launch_bounds__(kPeakBlock, 8) dfma_kernel(int iters, float* sink, unsigned long long* cycles) {
  double a[8];
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * k + 1e-6 * threadIdx.x;
  const double b = 0.9999999, c = 1e-9;
  __syncthreads();
  const uint64_t g0 = gtimer_ns(), t0 = clk64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = __fma_rn(a[k], b, c);
  }
  record_cycles(t0, g0, cycles);
  double s = 0.0;
  for (int k = 0; k < 8; ++k) s += a[k];
  keep((float)s, sink);
}

// Warp match: `iters` x 4 independent __match_any_sync per thread on values
// that take 8 distinct values per warp.
__global__ void __launch_bounds__(kPeakBlock, 8) match_kernel(int iters, float* sink, unsigned long long* cycles) {
  uint32_t v[4];
  for (int k = 0; k < 4; ++k) v[k] = (threadIdx.x & 7) + 8 * k;
  uint32_t acc = 0;
  __syncthreads();
  const uint64_t g0 = gtimer_ns(), t0 = clk64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 4; ++k) acc += __match_any_sync(0xffffffffu, v[k] + (uint32_t)it);
  }
  record_cycles(t0, g0, cycles);
  keep_u(acc, sink);
}

// Bins of the shared-atomic benchmark, 16 per lane, drawn once before the timed
// loop so that the loop issues nothing but the increments:
//  MODE 0: uniform random over the width
//  MODE 1: clustered: the 32 lanes of a warp on 4 neighbouring bins
//  MODE 2: all lanes of a warp on one bin
//  MODE 3: conflict free: lane l on bin base + l
__device__ __forceinline__ uint32_t mixh(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

template <int MODE>
__device__ __forceinline__ uint32_t bench_bin(int k, uint32_t width) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (MODE == 0) return __umulhi(mixh(threadIdx.x * 0x9E3779B9u + blockIdx.x * 0x85EBCA6Bu + (uint32_t)k * 0x27D4EB2Fu),
                                 width);
  const uint32_t base = __umulhi(mixh(warp * 0x9E3779B9u + blockIdx.x * 0x85EBCA6Bu + (uint32_t)k * 0x27D4EB2Fu),
                                 width - 32u);
  if (MODE == 1) return base + (lane & 3u);
  if (MODE == 2) return base;
  return base + lane;
}

// Shared-memory histogram increments (red.shared.add.u32), `iters` x 16 per
// thread, into a block-private histogram of `width` bins (the pair kernel's A7
// update).  Each lane cycles through its 16 precomputed bins.
template <int MODE>
__global__ void __launch_bounds__(kPeakBlock) smem_atomic_kernel(int iters, uint32_t width, float* sink,
                                                                 unsigned long long* cycles) {
  extern __shared__ uint32_t hist[];
  for (uint32_t k = threadIdx.x; k < width; k += blockDim.x) hist[k] = 0u;
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(hist);
  uint32_t addr[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) addr[k] = base + 4u * bench_bin<MODE>(k, width);
  __syncthreads();
  const uint64_t g0 = gtimer_ns(), t0 = clk64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 16; ++k) asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr[k]) : "memory");
  }
  record_cycles(t0, g0, cycles);
  __syncthreads();
  uint32_t s = 0;
  for (uint32_t k = threadIdx.x; k < width; k += blockDim.x) s += hist[k];
  keep_u(s, sink);
}

// Cluster-distributed histogram increments (red.shared::cluster.add.u32): a
// cluster of `csize` blocks holds one histogram of `width` bins, block r the
// bins [r w, (r + 1) w), w = width / csize; every lane increments uniform random
// bins of the whole histogram, (csize - 1) / csize of them in another block's
// shared memory.  16 cluster addresses per lane are formed before the timed
// loop (mapa).  The cluster waits for all its blocks before the first and after
// the last increment, so that no block leaves while others still write to it.
constexpr int kClusterBlock = 1024;  // one block per SM holds a large slice: all 32 warps of the SM in it
__global__ void __launch_bounds__(kClusterBlock) dsmem_atomic_kernel(int iters, uint32_t width, float* sink,
                                                                  unsigned long long* cycles) {
  extern __shared__ uint32_t hist[];
  uint32_t csize, crank;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(csize));
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(crank));
  const uint32_t w = width / csize;
  for (uint32_t k = threadIdx.x; k < w; k += blockDim.x) hist[k] = 0u;
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(hist);
  uint32_t addr[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint32_t b = __umulhi(mixh(threadIdx.x * 0x9E3779B9u + blockIdx.x * 0x85EBCA6Bu + (uint32_t)k * 0x27D4EB2Fu),
                                w * csize);
    const uint32_t owner = b / w, local = base + 4u * (b - owner * w);
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(addr[k]) : "r"(local), "r"(owner));
  }
  asm volatile("barrier.cluster.arrive.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
  const uint64_t g0 = gtimer_ns(), t0 = clk64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 16; ++k) asm volatile("red.shared::cluster.add.u32 [%0], 1;" ::"r"(addr[k]) : "memory");
  }
  record_cycles(t0, g0, cycles);
  asm volatile("barrier.cluster.arrive.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
  uint32_t sum = 0;
  for (uint32_t k = threadIdx.x; k < w; k += blockDim.x) sum += hist[k];
  keep_u(sum, sink);
}

// 64-bit global atomics (the A8 merge): `iters` x 4 atomicAdd per thread on
// uniform random bins of a uint64 array of `width` entries (L2 resident).
__global__ void __launch_bounds__(kPeakBlock, 8) global_atomic_kernel(int iters, uint32_t width, uint64_t* g,
                                                                   unsigned long long* cycles) {
  uint32_t h = mixh(threadIdx.x * 0x9E3779B9u + blockIdx.x * 0x85EBCA6Bu);
  __syncthreads();
  const uint64_t g0 = gtimer_ns(), t0 = clk64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      h = h * 0x2C1B3C6Du + 0x297A2D39u;
      atomicAdd((unsigned long long*)(g + __umulhi(h ^ (h >> 15), width)), 1ull);
    }
  }
  record_cycles(t0, g0, cycles);
}

// What each microbenchmark counts per thread and iteration.
struct PeakSpec {
  double ops_per_iter;  // operations counted per thread per loop iteration
  int iters;
};

PeakSpec spec_of(int pipe) {
  switch (pipe) {
    case DH_PIPE_FFMA2: case DH_PIPE_FADD2: case DH_PIPE_FMUL2: return {16.0, 16384};  // 8 x 2 lanes
    case DH_PIPE_FFMA: return {16.0, 16384};
    case DH_PIPE_SQRT: case DH_PIPE_FRND: case DH_PIPE_F2I: return {8.0, 8192};
    case DH_PIPE_LOP3: case DH_PIPE_IMAD: return {8.0, 16384};
    case DH_PIPE_IADD: return {16.0, 8192};  // two adds per instance
    case DH_PIPE_DFMA: return {8.0, 256};
    case DH_PIPE_MATCH: return {4.0, 2048};
    case DH_PIPE_SMEM_ATOMIC_RANDOM: case DH_PIPE_SMEM_ATOMIC_CLUSTERED:
    case DH_PIPE_SMEM_ATOMIC_SAME: case DH_PIPE_SMEM_ATOMIC_SEQUENTIAL: return {16.0, 1024};
    case DH_PIPE_GLOBAL_ATOMIC64: return {4.0, 256};
    case DH_PIPE_DSMEM_ATOMIC_C2: case DH_PIPE_DSMEM_ATOMIC_C4: case DH_PIPE_DSMEM_ATOMIC_C8: return {16.0, 256};
    default: return {0.0, 0};
  }
}

const void* kernel_of(int pipe) {
  switch (pipe) {
    case DH_PIPE_FFMA2: return (const void*)packed_kernel<0>;
    case DH_PIPE_FADD2: return (const void*)packed_kernel<1>;
    case DH_PIPE_FMUL2: return (const void*)packed_kernel<2>;
    case DH_PIPE_FFMA: return (const void*)ffma_kernel;
    case DH_PIPE_SQRT: return (const void*)xu_kernel<0>;
    case DH_PIPE_FRND: return (const void*)xu_kernel<1>;
    case DH_PIPE_F2I: return (const void*)xu_kernel<2>;
    case DH_PIPE_LOP3: return (const void*)int_kernel<0>;
    case DH_PIPE_IADD: return (const void*)int_kernel<1>;
    case DH_PIPE_IMAD: return (const void*)int_kernel<2>;
    case DH_PIPE_DFMA: return (const void*)dfma_kernel;
    case DH_PIPE_MATCH: return (const void*)match_kernel;
    case DH_PIPE_SMEM_ATOMIC_RANDOM: return (const void*)smem_atomic_kernel<0>;
    case DH_PIPE_SMEM_ATOMIC_CLUSTERED: return (const void*)smem_atomic_kernel<1>;
    case DH_PIPE_SMEM_ATOMIC_SAME: return (const void*)smem_atomic_kernel<2>;
    case DH_PIPE_SMEM_ATOMIC_SEQUENTIAL: return (const void*)smem_atomic_kernel<3>;
    case DH_PIPE_DSMEM_ATOMIC_C2: case DH_PIPE_DSMEM_ATOMIC_C4: case DH_PIPE_DSMEM_ATOMIC_C8:
      return (const void*)dsmem_atomic_kernel;
    default: return (const void*)global_atomic_kernel;
  }
}

int cluster_of(int pipe) {
  return pipe == DH_PIPE_DSMEM_ATOMIC_C2 ? 2 : pipe == DH_PIPE_DSMEM_ATOMIC_C4 ? 4 : pipe == DH_PIPE_DSMEM_ATOMIC_C8 ? 8 : 1;
}

}  // namespace
}  // namespace dh

using namespace dh;

extern "C" dh_status dh_pipe_rate(int32_t device, int32_t pipe, int32_t width, double* out) {
  if (!out) return fail(DH_ERR_INVALID, "out is NULL");
  const PeakSpec sp = spec_of(pipe);
  if (sp.iters == 0) return fail(DH_ERR_INVALID, "unknown pipe %d", pipe);
  const int csize = cluster_of(pipe);
  const bool smem = (pipe >= DH_PIPE_SMEM_ATOMIC_RANDOM && pipe <= DH_PIPE_SMEM_ATOMIC_SEQUENTIAL) || csize > 1;
  const bool glob = pipe == DH_PIPE_GLOBAL_ATOMIC64;
  const int wmax = smem ? 56 * 1024 * csize : 1 << 24;
  if ((smem || glob) && (width < 64 * csize || width > wmax))
    return fail(DH_ERR_INVALID, "width %d outside [%d, %d]", width, 64 * csize, wmax);
  DH_CUDA_TRY(cudaSetDevice(device));
  int sms = 0;
  DH_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  cudaStream_t st = nullptr;
  DH_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float* sink = nullptr;
  unsigned long long* cyc = nullptr;
  uint64_t* g = nullptr;
  dh_status result = DH_OK;
  const size_t smem_bytes = smem ? 4 * (size_t)(width / csize) : 0;
  auto run = [&](int iters, int grid) -> cudaError_t {
    switch (pipe) {
      case DH_PIPE_FFMA2: packed_kernel<0><<<grid, kPeakBlock, 0, st>>>(iters, sink, cyc); break;
      case DH_PIPE_FADD2: packed_kernel<1><<<grid, kPeakBlock, 0, st>>>(iters, sink, cyc); break;
      case DH_PIPE_FMUL2: packed_kernel<2><<<grid, kPeakBlock, 0, st>>>(iters, sink, cyc); break;
      case DH_PIPE_FFMA: ffma_kernel<<<grid, kPeakBlock, 0, st>>>(iters, sink, cyc); break;
      case DH_PIPE_SQRT: xu_kernel<0><<<grid, kPeakBlock, 0, st>>>(iters, sink, cyc); break;
      case DH_PIPE_FRND: xu_kernel<1><<<grid, kPeakBlock, 0, st>>>(iters, sink, cyc); break;
      case DH_PIPE_F2I: xu_kernel<2><<<grid, kPeakBlock, 0, st>>>(iters, sink, cyc); break;
      case DH_PIPE_LOP3: int_kernel<0><<<grid, kPeakBlock, 0, st>>>(iters, sink, cyc); break;
      case DH_PIPE_IADD: int_kernel<1><<<grid, kPeakBlock, 0, st>>>(iters, sink, cyc); break;
      case DH_PIPE_IMAD: int_kernel<2><<<grid, kPeakBlock, 0, st>>>(iters, sink, cyc); break;
      case DH_PIPE_DFMA: dfma_kernel<<<grid, kPeakBlock, 0, st>>>(iters, sink, cyc); break;
      case DH_PIPE_MATCH: match_kernel<<<grid, kPeakBlock, 0, st>>>(iters, sink, cyc); break;
      case DH_PIPE_SMEM_ATOMIC_RANDOM:
        smem_atomic_kernel<0><<<grid, kPeakBlock, smem_bytes, st>>>(iters, (uint32_t)width, sink, cyc); break;
      case DH_PIPE_SMEM_ATOMIC_CLUSTERED:
        smem_atomic_kernel<1><<<grid, kPeakBlock, smem_bytes, st>>>(iters, (uint32_t)width, sink, cyc); break;
      case DH_PIPE_SMEM_ATOMIC_SAME:
        smem_atomic_kernel<2><<<grid, kPeakBlock, smem_bytes, st>>>(iters, (uint32_t)width, sink, cyc); break;
      case DH_PIPE_SMEM_ATOMIC_SEQUENTIAL:
        smem_atomic_kernel<3><<<grid, kPeakBlock, smem_bytes, st>>>(iters, (uint32_t)width, sink, cyc); break;
      case DH_PIPE_DSMEM_ATOMIC_C2: case DH_PIPE_DSMEM_ATOMIC_C4: case DH_PIPE_DSMEM_ATOMIC_C8: {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)csize;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(kClusterBlock);
        cfg.dynamicSmemBytes = smem_bytes;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, dsmem_atomic_kernel, iters, (uint32_t)width, sink, cyc);
      }
      default: global_atomic_kernel<<<grid, kPeakBlock, 0, st>>>(iters, (uint32_t)width, g, cyc); break;
    }
    return cudaGetLastError();
  };
  do {
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess ||
        (e = cudaMalloc(&sink, sizeof(float) * kClusterBlock)) != cudaSuccess ||
        (e = cudaMalloc(&cyc, 2 * sizeof(unsigned long long))) != cudaSuccess ||
        (glob && (e = cudaMalloc(&g, 8 * (size_t)width)) != cudaSuccess)) {
      result = fail(DH_ERR_CUDA, "dh_pipe_rate setup: %s", cudaGetErrorString(e));
      break;
    }
    if (glob && (e = cudaMemsetAsync(g, 0, 8 * (size_t)width, st)) != cudaSuccess) {
      result = fail(DH_ERR_CUDA, "dh_pipe_rate: %s", cudaGetErrorString(e));
      break;
    }
    // blocks per SM: as many as are resident at once (one wave, every warp slot
    // busy where registers and shared memory allow)
    int bps = 0;
    const void* fn = kernel_of(pipe);
    if (smem && ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes)) !=
                     cudaSuccess ||
                 (e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                           (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)) {
      result = fail(DH_ERR_CUDA, "dh_pipe_rate: %s", cudaGetErrorString(e));
      break;
    }
    const int threads = csize > 1 ? kClusterBlock : kPeakBlock;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, threads, smem_bytes)) != cudaSuccess ||
        bps < 1) {
      result = fail(DH_ERR_CUDA, "dh_pipe_rate: no block fits");
      break;
    }
    int grid = sms * bps;
    if (csize > 1) {  // whole clusters, as many as are resident at once
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)csize;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)(csize * 64));
      cfg.blockDim = dim3(kClusterBlock);
      cfg.dynamicSmemBytes = smem_bytes;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      if ((e = cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg)) != cudaSuccess || clusters < 1) {
        result = fail(DH_ERR_CUDA, "dh_pipe_rate: no cluster of %d fits", csize);
        break;
      }
      grid = clusters * csize;
    }
    // warm-up (clocks up, code loaded), then the measured launch
    if ((e = run(sp.iters / 8 > 0 ? sp.iters / 8 : 1, grid)) != cudaSuccess ||
        (e = cudaMemsetAsync(cyc, 0, 2 * sizeof(unsigned long long), st)) != cudaSuccess ||
        (e = cudaEventRecord(e0, st)) != cudaSuccess || (e = run(sp.iters, grid)) != cudaSuccess ||
        (e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      result = fail(DH_ERR_CUDA, "dh_pipe_rate run: %s", cudaGetErrorString(e));
      break;
    }
    float ms = 0.f;
    unsigned long long cg[2] = {0, 0};
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess ||
        (e = cudaMemcpy(cg, cyc, sizeof cg, cudaMemcpyDeviceToHost)) != cudaSuccess) {
      result = fail(DH_ERR_CUDA, "dh_pipe_rate: %s", cudaGetErrorString(e));
      break;
    }
    const double ops = sp.ops_per_iter * (double)sp.iters * (double)threads * (double)grid;
    const double mhz = cg[1] > 0 ? 1e3 * (double)cg[0] / (double)cg[1] : 0.0;
    out[1] = ops / (ms * 1e-3);                                   // per second
    out[0] = mhz > 0.0 ? out[1] / ((double)sms * mhz * 1e6) : 0.0;  // per clock per SM at that clock
    out[2] = mhz;                                                 // SM clock over the launch
    out[3] = ms;
  } while (0);
  if (sink) cudaFree(sink);
  if (cyc) cudaFree(cyc);
  if (g) cudaFree(g);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  return result;
}
