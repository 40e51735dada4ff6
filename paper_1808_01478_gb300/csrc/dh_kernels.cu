// CUDA kernels of the particle-pair distance histogram (sm_103a).
//
// Hot path (Reuter & Koefinger, Sec. 2 and 3.2): for every unique pair the
// distance vector, the minimum image of Eq. 5, the Euclidean distance and the
// bin kappa = (int) nbins r / r_max of Alg. 1 are computed, and the bin of a
// block-private shared-memory histogram is incremented (the hybrid strategy of
// Sec. 2.4: groups of threads share a private histogram, merged into the
// global one at the end, Sec. 3.2.3).  Private counts are uint32 and are
// flushed into the uint64 global histogram before they can overflow
// (Sec. 3.1, also applied on the GPU).
//
// Precision design (not in the paper, which computes in float32 only): the
// result must equal the binary64 definition bin for bin.  Each pair is first
// evaluated in float32 with an error bound delta (in bin units) derived for the
// exact operation sequence below; a pair whose float32 bin coordinate t lies
// farther than delta from every integer is decided in float32.  The others are
// pushed into a per-warp queue and re-decided by replaying the binary64
// definition (same operations, same order, explicit round-to-nearest
// intrinsics, no contraction) and comparing r^2 with a table of binary64
// thresholds T[k] = smallest r^2 whose bin is >= k.
#include <float.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "dh_internal.h"

namespace dh {

// ------------------------------------------------------------------ helpers

// Every launcher reports the error of its own launch: a non-sticky error that an
// earlier, unrelated API call on this thread left behind (this library's or
// another's) is cleared first.  Errors of kernels already running are sticky
// and still surface at the next synchronisation.
static inline void clear_stale_error() { (void)cudaGetLastError(); }

// Order-preserving map float -> int32 (for atomicMin/atomicMax on floats).
__device__ __forceinline__ int32_t ord_of(float f) {
  int32_t i = __float_as_int(f);
  return i >= 0 ? i : (i ^ 0x7FFFFFFF);
}
__device__ __forceinline__ float float_of_ord(int32_t k) {
  return __int_as_float(k >= 0 ? k : (k ^ 0x7FFFFFFF));
}

constexpr float kMagicRound = 12582912.0f;  // 1.5 * 2^23: fma(x, s, M) - M = nint_even(x*s), |x*s| < 2^22
constexpr float kMagicFloor = 8388608.0f;   // 2^23: fadd.rd(t, 2^23) - 2^23 = floor(t), 0 <= t < 2^23
constexpr unsigned kFull = 0xffffffffu;

// Relative error bound assumed for sqrt.approx.ftz.f32 (checked exhaustively
// over two binades by the GPU test suite).
constexpr double kSqrtRelErr = 8.0 / 16777216.0;  // 8 * 2^-24

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// IEEE minimum that propagates NaN (masked pairs carry NaN and must stay NaN).
__device__ __forceinline__ float min_nan(float a, float b) {
  float y;
  asm("min.NaN.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
  return y;
}
__device__ __forceinline__ float nint_scaled(float x, float s) {
  return __fadd_rn(__fmaf_rn(x, s, kMagicRound), -kMagicRound);
}
__device__ __forceinline__ float nint_f(float x) {
  return __fadd_rn(__fadd_rn(x, kMagicRound), -kMagicRound);
}

// ------------------------------------------------------------------ binary64 bin of Alg. 1

// kappa = floor((nbins * sqrt(r2)) / r_max), evaluated left to right in
// binary64; nbins when the pair is beyond the histogram.
__host__ __device__ inline int64_t bin_of_b64(double r2, double r_max, int32_t nbins) {
#ifdef __CUDA_ARCH__
  double r = __dsqrt_rn(r2);
  double t = __dmul_rn((double)nbins, r);
  t = __ddiv_rn(t, r_max);
#else
  double r = std::sqrt(r2);
  double t = (double)nbins * r;
  t = t / r_max;
#endif
  if (!(t < (double)nbins)) return nbins;
  return (int64_t)floor(t);
}

// Smallest binary64 q >= 0 with bin(q) >= k (k >= 1), found by stepping ulp by
// ulp from the rounded edge (k r_max / nbins)^2.  *ok is cleared if the walk
// does not settle within 4096 steps.
__host__ __device__ inline double threshold_of(int32_t k, double r_max, int32_t nbins, int* ok) {
  if (k <= 0) return 0.0;
  double e = ((double)k * r_max) / (double)nbins;
  double q = e * e;
  int it = 0;
  if (bin_of_b64(q, r_max, nbins) >= k) {
    for (; it < 4096; ++it) {
      double p = nextafter(q, 0.0);
      if (!(p < q) || bin_of_b64(p, r_max, nbins) < k) break;
      q = p;
    }
  } else {
    for (; it < 4096; ++it) {
      q = nextafter(q, (double)INFINITY);
      if (bin_of_b64(q, r_max, nbins) >= k) break;
    }
  }
  if (it >= 4096) *ok = 0;
  return q;
}

int64_t host_bin_of(double r2, double r_max, int32_t nbins) { return bin_of_b64(r2, r_max, nbins); }

int build_thresholds_host(double r_max, int32_t nbins, double* T) {
  int ok = 1;
  for (int32_t k = 0; k <= nbins; ++k) T[k] = threshold_of(k, r_max, nbins, &ok);
  return ok;
}

// T[k] for k = 0..nbins, followed by the same values as float pairs (hi, lo)
// at (float2*)(T + nbins + 1) for the double-float tier.
__global__ void thresholds_kernel(double r_max, int32_t nbins, double* T, int32_t* status) {
  int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > nbins) return;
  int ok = 1;
  double t = threshold_of(k, r_max, nbins, &ok);
  T[k] = t;
  float hi = __double2float_rn(t);
  float lo = __double2float_rn(t - (double)hi);
  reinterpret_cast<float2*>(T + nbins + 1)[k] = make_float2(hi, lo);
  if (!ok) atomicExch(status, 7);
}

// ------------------------------------------------------------------ A1: staging

// Staging of several frames at once: block b handles chunk b of the job whose
// chunk range contains it; coords (n x stride floats, or doubles) -> float4
// (and double4 for binary64 input), per-axis min/max of the float32 values (for
// the error window) and finiteness.
__global__ void stage_kernel(const StageJob* __restrict__ jobs, int n_jobs) {
  const long long chunk = blockIdx.x;
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].chunk0 <= chunk) lo = mid; else hi = mid - 1;
  }
  const StageJob J = jobs[lo];
  const int64_t i0 = (chunk - J.chunk0) * (int64_t)kStageChunk;
  const int64_t i1 = min(J.n, i0 + (int64_t)kStageChunk);
  float mn0 = INFINITY, mn1 = INFINITY, mn2 = INFINITY;
  float mx0 = -INFINITY, mx1 = -INFINITY, mx2 = -INFINITY;
  int bad = 0;
  const float* __restrict__ src = J.src;
  const int stride = J.stride;
  const double* __restrict__ src64 = reinterpret_cast<const double*>(src);
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    float x, y, z;
    if (J.dst64) {  // binary64 input: kept as given, and rounded to float32 for the fast path
      double a = src64[i * stride], b = src64[i * stride + 1], c = src64[i * stride + 2];
      J.dst64[i] = make_double4(a, b, c, 0.0);
      x = __double2float_rn(a);
      y = __double2float_rn(b);
      z = __double2float_rn(c);
    } else {
      x = src[i * stride];
      y = src[i * stride + 1];
      z = src[i * stride + 2];
    }
    bad |= !(isfinite(x) && isfinite(y) && isfinite(z));
    J.dst[i] = make_float4(x, y, z, 0.0f);
    mn0 = fminf(mn0, x); mn1 = fminf(mn1, y); mn2 = fminf(mn2, z);
    mx0 = fmaxf(mx0, x); mx1 = fmaxf(mx1, y); mx2 = fmaxf(mx2, z);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn0 = fminf(mn0, __shfl_xor_sync(kFull, mn0, o));
    mn1 = fminf(mn1, __shfl_xor_sync(kFull, mn1, o));
    mn2 = fminf(mn2, __shfl_xor_sync(kFull, mn2, o));
    mx0 = fmaxf(mx0, __shfl_xor_sync(kFull, mx0, o));
    mx1 = fmaxf(mx1, __shfl_xor_sync(kFull, mx1, o));
    mx2 = fmaxf(mx2, __shfl_xor_sync(kFull, mx2, o));
    bad |= __shfl_xor_sync(kFull, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    FrameDev* F = J.fd;
    if (mn0 <= mx0) {
      atomicMin(&F->cmin[0], ord_of(mn0)); atomicMin(&F->cmin[1], ord_of(mn1));
      atomicMin(&F->cmin[2], ord_of(mn2));
      atomicMax(&F->cmax[0], ord_of(mx0)); atomicMax(&F->cmax[1], ord_of(mx1));
      atomicMax(&F->cmax[2], ord_of(mx2));
    }
    if (bad) atomicExch(&F->bad, 1);
  }
}

// ------------------------------------------------------------------ spatial order (staging)

__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // bit k of v -> bit 3k
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Morton cell of a particle from its fractional coordinates in the box, or in
// the frame's bounding box without one (approximate float32; only the order
// depends on it).
__device__ __forceinline__ uint32_t cell_key(const FrameDev& F, float4 p, int g) {
  float s[3];
  if (F.variant == V_NONE) {
    const float q[3] = {p.x, p.y, p.z};
    for (int c = 0; c < 3; ++c) {
      const float lo = float_of_ord(F.cmin[c]), hi = float_of_ord(F.cmax[c]);
      s[c] = (hi > lo) ? fminf((q[c] - lo) / (hi - lo), 0.999999f) : 0.0f;
    }
  } else if (F.variant == V_ORTHO) {
    s[0] = p.x * F.invf[0];
    s[1] = p.y * F.invf[1];
    s[2] = p.z * F.invf[2];
  } else {
    s[2] = p.z * F.invf[2];
    s[1] = (p.y - F.Bf[5] * s[2]) * F.invf[1];
    s[0] = (p.x - F.Bf[1] * s[1] - F.Bf[2] * s[2]) * F.invf[0];
  }
  const float G = (float)(1 << g);
  uint32_t c[3];
  for (int a = 0; a < 3; ++a) {
    float f = s[a] - floorf(s[a]);
    int ci = (int)(f * G);
    c[a] = (uint32_t)min(max(ci, 0), (1 << g) - 1);
  }
  return spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
}

__global__ void sort_count_kernel(const SortSeg* segs, const float4* __restrict__ X, int32_t* keys,
                                  uint32_t* counts) {
  const SortSeg S = segs[blockIdx.y];
  const int64_t i0 = (int64_t)blockIdx.x * kSortChunk;
  const int64_t i1 = min((int64_t)S.n, i0 + kSortChunk);
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    uint32_t k = cell_key(*S.fd, X[S.x0 + i], S.g);
    keys[S.x0 + i] = (int32_t)k;
    atomicAdd(counts + S.key0 + k, 1u);
  }
}

// Exclusive prefix sum of each segment's counters, in place (one block per segment).
__global__ void sort_scan_kernel(const SortSeg* segs, uint32_t* counts) {
  const SortSeg S = segs[blockIdx.x];
  const int64_t m = (int64_t)1 << (3 * S.g);
  uint32_t* c = counts + S.key0;
  const int64_t per = (m + blockDim.x - 1) / blockDim.x;
  const int64_t b = min(m, (int64_t)threadIdx.x * per), e = min(m, b + per);
  uint32_t local = 0;
  for (int64_t k = b; k < e; ++k) local += c[k];
  __shared__ uint32_t warp_sum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = local;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t v = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x / 32;
    uint32_t v = lane < nw ? warp_sum[lane] : 0u, inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane < nw) warp_sum[lane] = inc - v;  // exclusive over warps
  }
  __syncthreads();
  uint32_t run = warp_sum[warp] + incl - local;  // exclusive start of this thread's chunk
  for (int64_t k = b; k < e; ++k) {
    uint32_t v = c[k];
    c[k] = run;
    run += v;
  }
}

__global__ void sort_scatter_kernel(const SortSeg* segs, const float4* __restrict__ X,
                                    const double4* __restrict__ X64, const int32_t* __restrict__ keys,
                                    uint32_t* cursors, float4* Xs, double4* Xs64) {
  const SortSeg S = segs[blockIdx.y];
  const int64_t i0 = (int64_t)blockIdx.x * kSortChunk;
  const int64_t i1 = min((int64_t)S.n, i0 + kSortChunk);
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    uint32_t pos = atomicAdd(cursors + S.key0 + (uint32_t)keys[S.x0 + i], 1u);
    Xs[S.x0 + pos] = X[S.x0 + i];
    if (X64) Xs64[S.x0 + pos] = X64[S.x0 + i];
  }
}

__global__ void sort_copy_kernel(const SortSeg* segs, const float4* __restrict__ Xs, float4* X,
                                 const double4* __restrict__ Xs64, double4* X64) {
  const SortSeg S = segs[blockIdx.y];
  const int64_t i0 = (int64_t)blockIdx.x * kSortChunk;
  const int64_t i1 = min((int64_t)S.n, i0 + kSortChunk);
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    X[S.x0 + i] = Xs[S.x0 + i];
    if (X64) X64[S.x0 + i] = Xs64[S.x0 + i];
  }
}

// ------------------------------------------------------------------ per-frame error window

// Largest rounding error (half an ulp) of a float32 result whose exact value
// has magnitude at most D.
__device__ inline double half_ulp_below(double D) {
  if (!(D > 0.0)) return 0.0;
  int E;
  frexp(D, &E);  // D = m 2^E, m in [1/2, 1): |x| <= D < 2^E
  return ldexp(1.0, E - 25);
}

// Derives, for one frame, the bound of the float32 decision and of the
// double-float tier from its box, r_max, nbins and the coordinate ranges found
// by stage_kernel.  Every float32 operation rounds to nearest (relative error
// <= u = 2^-24); S = nbins/r_max, t = S r, q = t^2, R_c = coordinate range.
//  t-space bound |t' - t| <= alpha*t + beta for t' = sqrt(q32) (the exact root
//  of the computed q):
//   alpha: rounding of d (none) or of the final wrapped d' (u), the
//          r^2 = fma(dz,dz,fma(dy,dy,dx*dx)) chain (3u on r^2 -> 1.5u),
//          float32 S^2 and the product q = r^2 S^2 ((eps_S2 + u)/2);
//   beta:  S*|a|, a_c the absolute error of d'_c: rounding of xj - xi (half an
//          ulp of the largest |d_c| <= R_c), of each wrap intermediate (half an
//          ulp of its largest magnitude) and the float32 box entries
//          (|k| |B32 - B|, |k| at most the nearest integer of the largest
//          |d|/L); for orthorhombic boxes, where float32 and binary64 may round
//          d/L to different images within eta of a half integer (both images
//          then have |d'_c| within eta L of L_c/2), S*2 eta L for as many
//          components as can reach L_c/2 below r_max (1 + 2/nbins).
//  q-space test: with n the integer nearest to sqrt(q32), floor(t) is decided
//  when |q32 - n^2| > (alpha t' + beta)(2 t' + 1) = 2 alpha q + (alpha + 2 beta) t' + beta;
//  load_fast_params turns it into one FMA in q (t' <= (q/tau + tau)/2 for any
//  tau > 0).
//  Tiles with a uniform image (tile_image) take beta_u: the same with their
//  own absolute errors (the image subtracted exactly, orthorhombic; the i's
//  moved by a rounded B k, triclinic).
//  double-float tier: |r2_df - r2_64| <= 2^-38 r2 + 2 r |a_mid| with |a_mid|
//  from 2^-40 times the wrap magnitudes (binary64 oracle rounding and the
//  float pair arithmetic, both far below it).
// beta also carries 2^-28 for the binary64 rounding of t itself (< 2^-29 for t < 2^22).
// If a precondition of the float32 path fails (nearest-integer range,
// triclinic margin) or the t-space bound reaches 1/4, every pair is deferred.
__global__ void frame_setup_kernel(FrameDev* frames, int n_frames) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_frames) return;
  FrameDev& F = frames[f];
  const double u = 1.0 / 16777216.0;
  double R[3] = {0, 0, 0};
  // binary64 input: the float32 path starts from coordinates rounded to float32,
  // each within half an ulp of the largest magnitude on its axis
  double conv[3] = {0, 0, 0};
  double Xm[3] = {0, 0, 0};  // largest coordinate magnitude per axis
  if (F.n > 0 && F.cmin[0] <= F.cmax[0]) {
    for (int c = 0; c < 3; ++c) {
      double lo = float_of_ord(F.cmin[c]), hi = float_of_ord(F.cmax[c]);
      R[c] = hi - lo;
      Xm[c] = fmax(fabs(lo), fabs(hi));
      if (F.X64) conv[c] = 2.0 * half_ulp_below(Xm[c]);
    }
  }
  double S = (double)F.nbins / F.r_max;
  double alpha = 3.0 * u + 0.5 * F.eps_S2;
  double a[3] = {0, 0, 0};
  double I[3] = {R[0], R[1], R[2]};  // magnitudes of the wrap intermediates (for the double-float tier)
  double tie = 0.0, tie_eps = 0.0;
  double au[3] = {0, 0, 0};  // absolute error of d'_c in tiles with a uniform image
  double aw[3][3] = {};      // the same, axis a wrapped per pair (M_AXIS + a); tie term tie_w[a]
  double tie_w[3] = {0, 0, 0};
  for (int c = 0; c < 3; ++c) {
    F.tie_m[c] = 0.0f;
    F.tie_t[c] = 0.0f;
    F.convf[c] = __double2float_ru(conv[c]);
  }
  F.kxdb = 0.0f;
  F.tie_all = 0.0f;
  F.rr2 = 0.0f;
  int all_defer = 0;
  float eps_s = 0.0f;
  const double* B = F.B;
  double dB[9];
  for (int q = 0; q < 9; ++q) {
    dB[q] = fabs((double)F.Bf[q] - B[q]);
    F.dBf[q] = __double2float_ru(dB[q]);
  }
  if (F.variant == V_ORTHO) {
    double Lmin = INFINITY, tie_c[3];
    for (int c = 0; c < 3; ++c) {
      double L = B[4 * c];
      double K = floor(R[c] / L * (1.0 + 1e-9) + 0.5);  // largest |k| = nint(d/L) over |d| <= R_c
      a[c] = half_ulp_below(R[c]) + K * dB[4 * c] + conv[c];
      I[c] = R[c] + K * L;
      if (R[c] / L > 1048576.0) all_defer = 1;  // nearest integer via the 1.5*2^23 trick needs |d/L| < 2^22
      Lmin = fmin(Lmin, L);
      // float32 and binary64 can round d/L to different images only within eta of a
      // half integer; both images then have |d'_c| within eta L of L/2
      double eta = (half_ulp_below(R[c]) + conv[c] + R[c] * fabs((double)F.invf[c] - 1.0 / L)) / L +
                   1e-15 * (R[c] / L + 1.0);
      tie_c[c] = 2.0 * eta * L;
    }
    // components that can sit at L_c/2 while t <= nbins + 1 (r <= r_max (1 + 1/nbins))
    double rr = F.r_max * (1.0 + 2.0 / (double)F.nbins);
    int m = (int)fmin(3.0, floor(4.0 * rr * rr / (Lmin * Lmin)));
    if (m >= 1) {
      double t1 = fmax(tie_c[0], fmax(tie_c[1], tie_c[2]));
      double t3 = sqrt(tie_c[0] * tie_c[0] + tie_c[1] * tie_c[1] + tie_c[2] * tie_c[2]);
      tie = S * (m >= 3 ? t3 : (m == 2 ? fmin(t3, 1.4142135623730951 * t1) : t1)) * 1.01;
    }
    tie_eps = 2.0 * fmax(tie_c[0], fmax(tie_c[1], tie_c[2])) + 1e-12 * Lmin;
    // uniform-image tiles: the image is subtracted exactly (|k| <= 1), so d'_c
    // errs only by the float32 box entry; the tie term is not needed where the
    // tile's difference range, widened by tie_m = 4 eta L, keeps one image
    for (int c = 0; c < 3; ++c) {
      au[c] = dB[4 * c] + conv[c];
      F.tie_m[c] = tie > 0.0 ? (float)(2.0 * tie_c[c]) : 0.0f;
    }
    // one axis wrapped per pair: its own error and, alone, its tie term
    for (int w = 0; w < 3; ++w) {
      for (int c = 0; c < 3; ++c) aw[w][c] = c == w ? a[c] : au[c];
      tie_w[w] = tie > 0.0 ? S * tie_c[w] * 1.01 : 0.0;
      F.tie_t[w] = __double2float_ru(tie_w[w]);
    }
    F.tie_all = __double2float_ru(tie);
    F.rr2 = __double2float_ru(rr * rr);
  } else if (F.variant == V_TRIC) {
    // sequential wrap along c, then b, then a (Eq. 5 below half the plane spacing);
    // D are the largest magnitudes of the intermediates, K the largest |k|
    double ax = B[0], bx = B[1], cx = B[2], by = B[4], cy = B[5], cz = B[8];
    double Kz = floor(R[2] / cz * (1.0 + 1e-9) + 0.5);
    double D1x = R[0] + Kz * fabs(cx), D1y = R[1] + Kz * fabs(cy);
    double Ky = floor(D1y / by * (1.0 + 1e-9) + 0.5);
    double D2x = D1x + Ky * fabs(bx);
    double Kx = floor(D2x / ax * (1.0 + 1e-9) + 0.5);
    a[0] = half_ulp_below(R[0]) + half_ulp_below(D1x) + half_ulp_below(D2x) + Kz * dB[2] + Ky * dB[1] + Kx * dB[0] +
           conv[0];
    a[1] = half_ulp_below(R[1]) + half_ulp_below(D1y) + Kz * dB[5] + Ky * dB[4] + conv[1];
    a[2] = half_ulp_below(R[2]) + Kz * dB[8] + conv[2];
    // tile images (|k| <= 1): the i's move by B k, rounded to float32 from
    // binary64 (half an ulp of the row sum), then added (half an ulp of the
    // largest |x + B k|); d = xj - x'i itself rounds relative to |d| (alpha)
    const double Sx = ax + fabs(bx) + fabs(cx), Sy = by + fabs(cy), Sz = cz;
    au[0] = half_ulp_below(Xm[0] + Sx) + half_ulp_below(Sx) + conv[0];
    au[1] = half_ulp_below(Xm[1] + Sy) + half_ulp_below(Sy) + conv[1];
    au[2] = half_ulp_below(Xm[2] + Sz) + half_ulp_below(Sz) + conv[2];
    // x wrapped per pair after the uniform c and b images (M_AXIS): d_x before
    // its wrap rounds at up to R_x + |bx| + |cx|, and the wrap adds |kx| |ax32 - ax|
    const double Dxw = R[0] + fabs(bx) + fabs(cx);
    aw[0][0] = au[0] + half_ulp_below(Dxw) + Kx * dB[0];
    aw[0][1] = au[1];
    aw[0][2] = au[2];
    for (int m = 0; m < 27; ++m) {
      const double kx = m / 9 - 1, ky = (m / 3) % 3 - 1, kz = m % 3 - 1;
      const double v[3] = {-((kx * ax + ky * bx) + kz * cx), -(ky * by + kz * cy), -(kz * cz)};
      for (int c = 0; c < 3; ++c) {
        F.tshift[m][c] = (float)v[c];
        // the binary64 sum itself errs by at most 2^-52 of the row sum
        F.tserr[m][c] = __double2float_ru(fabs((double)F.tshift[m][c] - v[c]) + fmax(Sx, fmax(Sy, Sz)) * 0x1p-51);
      }
    }
    F.kxdb = __double2float_ru(Kx * dB[0]);
    I[0] = D2x + Kx * ax;
    I[1] = D1y + Ky * by;
    I[2] = R[2] + Kz * cz;
    // the three nearest-integer decisions must be exact for every pair closer
    // than r_max: their float32 errors must stay below a quarter of the margin
    double ez = (2.0 * u * R[2] + conv[2] + R[2] * fabs((double)F.invf[2] * cz - 1.0)) / cz;
    double ey = (2.0 * (fmax(a[1], au[1]) + u * D1y) + D1y * fabs((double)F.invf[1] * by - 1.0)) / by;
    double ex = (2.0 * (fmax(a[0], au[0]) + u * D2x) + D2x * fabs((double)F.invf[0] * ax - 1.0)) / ax;
    double exw = (2.0 * (aw[0][0] + u * Dxw) + Dxw * fabs((double)F.invf[0] * ax - 1.0)) / ax;
    double emax = fmax(fmax(ex, exw), fmax(ey, ez));
    if (!(emax < 0.25 * (double)F.margin) || D2x / ax > 1048576.0 || D1y / by > 1048576.0 ||
        R[2] / cz > 1048576.0)
      all_defer = 1;
  } else if (F.variant == V_TRIC_SEARCH) {
    double ax = B[0], bx = B[1], cx = B[2], by = B[4], cy = B[5], cz = B[8];
    double Sz = R[2] / cz + 1.0;
    double Sy = (R[1] + fabs(cy) * Sz) / by + 1.0;
    double Sx = (R[0] + fabs(bx) * Sy + fabs(cx) * Sz) / ax + 1.0;
    double ez = 3.0 * u * (R[2] / cz + Sz);
    double ey = (3.0 * u * (R[1] + fabs(cy) * Sz) + fabs(cy) * ez) / by + 2.0 * u * Sy;
    double ex = (3.0 * u * (R[0] + fabs(bx) * Sy + fabs(cx) * Sz) + fabs(bx) * ey + fabs(cx) * ez) / ax +
                2.0 * u * Sx;
    // binary64 input: the converted coordinates move every fractional coordinate by
    // at most the sum of the conversion errors over the plane spacings
    eps_s = (float)(2.0 * fmax(ex, fmax(ey, ez)) + 4.0 * (conv[0] / ax + conv[1] / by + conv[2] / cz) + 1e-12);
    double Kx = floor(Sx + 0.5) + 1.0, Ky = floor(Sy + 0.5) + 1.0, Kz = floor(Sz + 0.5) + 1.0;
    double Ix = R[0] + Kx * ax + Ky * fabs(bx) + Kz * fabs(cx) + ax + fabs(bx) + fabs(cx);
    double Iy = R[1] + Ky * by + Kz * fabs(cy) + by + fabs(cy);
    double Iz = R[2] + Kz * cz + cz;
    a[0] = u * (R[0] + 7.0 * Ix) + (Kx + 1) * dB[0] + (Ky + 1) * dB[1] + (Kz + 1) * dB[2] + conv[0];
    a[1] = u * (R[1] + 6.0 * Iy) + (Ky + 1) * dB[4] + (Kz + 1) * dB[5] + conv[1];
    a[2] = u * (R[2] + 3.0 * Iz) + (Kz + 1) * dB[8] + conv[2];
    I[0] = Ix; I[1] = Iy; I[2] = Iz;
    if (Sx > 1048576.0 || Sy > 1048576.0 || Sz > 1048576.0 || eps_s > 0.05f) all_defer = 1;
  }
  if (F.variant == V_NONE)
    for (int c = 0; c < 3; ++c) a[c] = conv[c];  // d = xj - xi itself rounds relative to |d| (alpha)
  const double abs_u = sqrt(au[0] * au[0] + au[1] * au[1] + au[2] * au[2]);
  double beta = S * sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]) * (1.0 + 64.0 * u) + tie + 1.0 / 268435456.0;
  double beta_u = (F.variant == V_ORTHO || F.variant == V_TRIC) ? S * abs_u * (1.0 + 64.0 * u) + 1.0 / 268435456.0
                                                                 : beta;
  double beta_w[3] = {beta, beta, beta};
  for (int w = 0; w < 3; ++w)
    if (F.variant == V_ORTHO || (F.variant == V_TRIC && w == 0))
      beta_w[w] = S * sqrt(aw[w][0] * aw[w][0] + aw[w][1] * aw[w][1] + aw[w][2] * aw[w][2]) * (1.0 + 64.0 * u) +
                  tie_w[w] + 1.0 / 268435456.0;
  alpha = alpha * (1.0 + 1.0 / 1024.0) + 1e-12;
  double delta = alpha * ((double)F.nbins + 1.0) + beta;
  const double beta_max = fmax(fmax(beta, beta_u), fmax(beta_w[0], fmax(beta_w[1], beta_w[2])));
  if (!(delta < 0.25) || !(alpha * ((double)F.nbins + 1.0) + beta_max < 0.25)) all_defer = 1;
  // the q-space test itself is formed per sweep (load_fast_params)
  double Imax = fmax(I[0], fmax(I[1], I[2]));
  double amid = 1.7320508075688772 * (R[0] + R[1] + R[2] + 4.0 * Imax) / 1099511627776.0;  // 2^-40
  if (F.X64)  // binary64 input: the split coordinates (2^-48 of the magnitude each) and d rounded in binary64
    amid += 1.7320508075688772 * 4.0 * fmax(conv[0], fmax(conv[1], conv[2])) / 16777216.0 +
            1.7320508075688772 * (R[0] + R[1] + R[2]) / 4503599627370496.0;
  F.mid2 = (float)(1.0 / 274877906944.0);                                                   // 2^-38
  F.mid1 = (float)(2.0 * amid / S * 1.01);
  F.tie_eps = (float)tie_eps;
  F.delta = (float)fmin(delta, 1.0);
  F.alpha_t = (float)alpha;
  F.beta_t = (float)beta;
  F.beta_u = (float)beta_u;
  for (int w = 0; w < 3; ++w) F.beta_w[w] = (float)beta_w[w];
  F.eps_s = eps_s;
  F.all_defer = all_defer;
  // No box, one sweep: the largest possible distance, sqrt(sum R_c^2), maps below
  // nbins + 1 even after the float32 roundings of q and of its square root
  // (relative 2^-18 covers them), so no pair's root reaches the clamp.
  {
    const double D = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
    F.in_range = F.variant == V_NONE && F.sweep_width >= F.nbins && !all_defer &&
                 S * D * (1.0 + 1.0 / 262144.0) < (double)F.nbins + 1.0;
    // no box: bounding tiles pays only when some tile can miss a sweep
    F.cull_ok = F.variant == V_NONE && (F.sweep_width < F.nbins || F.r_max < D);
  }
}

// ------------------------------------------------------------------ A2-A8: pair kernel

// j particles per deferral-mask group: 32 pairs per lane and group without a box
// and 16 for the periodic variants (whose larger loop bodies, one per tile mode,
// outgrow the instruction cache when doubled), whatever the i particles per
// thread (mask bit = u * RI + r); the j tile is padded to kJUMax
template <int V, int RI>
constexpr int ju_of() { return (V == V_NONE ? 32 : 16) / RI; }
constexpr int kJUMax = 32;

// Tile modes of the periodic variants (tile_image): per-pair images, one
// uniform image, or a uniform image on all axes but one (M_AXIS + a:
// orthorhombic axis a; triclinic only a = 0, x), which is wrapped per pair.
// No box: M_UNI marks a tile of an in-range frame without padding, whose
// roots need no clamp.
constexpr int M_PAIR = 0, M_UNI = 1, M_AXIS = 2;
constexpr int M_SKIP = -1;  // a tile none of whose pairs has its bin in the current sweep
constexpr bool shifted_mode(int mode) { return mode >= M_UNI; }

struct FastParams {
  float S2;
  float qb1, qb0;       // near-edge bound |n^2 - q| <= qb1 q + qb0 (set_bound)
  int32_t kb1;          // bits(kMagicRound) + lo + 1
  uint32_t width;       // hi - lo
  int32_t lo, hi;       // bins [lo, hi) of this sweep
  float b[9];
  float inv[3];
  float amb_thr;        // search variant: 0.5 - eps_s
};

// The q-space test of the sweep [P.lo, P.hi) as one FMA in q.  The bound
// 2 alpha q + gamma t' + beta (gamma = alpha + 2 beta; beta of the tile mode:
// beta_t, beta_u, beta_w[a]) with t' <= (q/tau + tau)/2, true for any tau > 0,
// becomes (2 alpha + gamma/(2 tau)) q + (gamma tau/2 + beta), exact at t' = tau;
// tau = (hi + 2)/sqrt(2) (at least lo + 1) minimises the mean window over the
// sweep for pair counts growing like t^2.  The float32 evaluation (a few
// roundings, and alpha_t, beta_t rounded) is covered by the factor 1 + 2^-10.
__device__ __forceinline__ void set_bound_beta(const FrameDev& F, FastParams& P, float beta) {
  if (F.all_defer) {
    P.qb1 = P.qb0 = 1e30f;
    return;
  }
  const float tau = fmaxf((float)(P.hi + 2) * 0.70710678f, (float)(P.lo + 1));
  const float slack = 1.0f + 1.0f / 1024.0f;
  const float g = F.alpha_t + 2.0f * beta;
  P.qb1 = (2.0f * F.alpha_t + g / (2.0f * tau)) * slack;
  P.qb0 = (0.5f * g * tau + beta) * slack;
}
__device__ __forceinline__ void set_bound(const FrameDev& F, FastParams& P, int mode) {
  set_bound_beta(F, P, mode == M_PAIR ? F.beta_t : (mode == M_UNI ? F.beta_u : F.beta_w[mode - M_AXIS]));
}

// Half an ulp of the largest float32 of magnitude at most X (X >= 0, finite):
// the rounding error of any result whose magnitude X bounds.
__device__ __forceinline__ float half_ulp_f(float X) {
  return __uint_as_float(__float_as_uint(X) & 0x7f800000u) * 0x1p-24f;
}

// Largest |k| = |nint(d/L)| over |d| <= D, with room for the float32 roundings.
__device__ __forceinline__ float k_bound(float D, float inv) {
  return floorf(__fmaf_ru(D, inv * (1.0f + 0x1p-16f), 0.5f + 0x1p-16f));
}

// beta of one tile (img = (kx, ky, kz, mode) from tile_image) from the tile's
// own magnitudes instead of the frame's largest: the terms of frame_setup_kernel
// with each coordinate range, intermediate and image bound taken over the warp
// run and the j sub-chunk (imin..jmax).  Every float32 value of the tile lies
// between the rounded extreme differences (rounding is monotone), so half an ulp
// of the larger bound covers each rounding.  Orthorhombic: uniform axes err by
// |k| |L32 - L|, wrapped axes by the rounding of d = xj - xi and |k| |L32 - L|;
// the tie term of a wrapped axis a is kept only when some pair of the tile
// could lie within r_max (1 + 2/nbins) with |d'_a| near L_a/2, judged from the
// smallest displacements on the uniform axes.  Triclinic, shifted modes:
// x'_i = fl(x_i - tshift) rounds at half an ulp of the run's largest |x'|,
// tshift errs by tserr; in M_AXIS the x difference before its wrap rounds at
// half an ulp of its largest magnitude and the wrap adds |kx| |ax32 - ax|.
// Triclinic, per-pair images: the sequential wrap's intermediates.  Each is
// bounded by the frame's counterpart, so the result never exceeds the frame's
// beta of the mode; the outer factors are the same.
template <int V>
__device__ float tile_beta(const FrameDev& F, const float* imin, const float* imax, const float* jmin,
                           const float* jmax, float4 img) {
  const int mode = (int)img.w;
  const float kk[3] = {img.x, img.y, img.z};
  float a[3], tie = 0.0f;
  if (V == V_ORTHO) {
    if (mode == M_UNI) return F.beta_u;
    float mn2 = 0.0f;  // smallest squared displacement over the uniform axes (rounded down)
    for (int c = 0; c < 3; ++c) {
      if (mode == M_PAIR || mode == M_AXIS + c) {
        const float D = fmaxf(fabsf(__fsub_rn(jmin[c], imax[c])), fabsf(__fsub_rn(jmax[c], imin[c])));
        a[c] = half_ulp_f(D) + k_bound(D, F.invf[c]) * F.dBf[4 * c] + F.convf[c];
      } else {
        a[c] = fabsf(kk[c]) * F.dBf[4 * c] + F.convf[c];
        // exact displacements lie in [jmin - imax, jmax - imin] - k L, L within dBf of L32
        const float kL = kk[c] * F.Bf[4 * c];
        const float lo = __fsub_rd(__fsub_rd(jmin[c], imax[c]), kL) - F.dBf[4 * c];
        const float hi = __fsub_ru(__fsub_ru(jmax[c], imin[c]), kL) + F.dBf[4 * c];
        const float m = (lo > 0.0f) ? lo : (hi < 0.0f ? -hi : 0.0f);
        mn2 = __fmaf_rd(m, m, mn2);
      }
    }
    if (mode == M_PAIR) {
      tie = F.tie_all;
    } else {
      const int w = mode - M_AXIS;
      const float h = __fmul_rd(0.5f * F.Bf[4 * w], 1.0f - 0x1p-10f);
      if (__fmaf_rd(h, h, mn2) <= F.rr2) tie = F.tie_t[w];
    }
  } else {
    if (mode >= M_UNI) {
      const int m = 9 * (int)(kk[0] + 1.0f) + 3 * (int)(kk[1] + 1.0f) + (int)(kk[2] + 1.0f);
      for (int c = 0; c < 3; ++c) {
        const float lo = __fsub_rn(imin[c], F.tshift[m][c]), hi = __fsub_rn(imax[c], F.tshift[m][c]);
        a[c] = half_ulp_f(fmaxf(fabsf(lo), fabsf(hi))) + F.tserr[m][c] + F.convf[c];
        if (c == 0 && mode >= M_AXIS) {
          const float D = fmaxf(fabsf(__fsub_rn(jmax[0], lo)), fabsf(__fsub_rn(jmin[0], hi)));
          a[0] += half_ulp_f(D) + F.kxdb;
        }
      }
    } else {
      float D[3];
      for (int c = 0; c < 3; ++c)
        D[c] = fmaxf(fabsf(__fsub_rn(jmin[c], imax[c])), fabsf(__fsub_rn(jmax[c], imin[c])));
      const float* b = F.Bf;
      const float Kz = k_bound(D[2], F.invf[2]);
      const float D1x = __fmaf_ru(Kz, fabsf(b[2]), D[0]), D1y = __fmaf_ru(Kz, fabsf(b[5]), D[1]);
      const float Ky = k_bound(D1y, F.invf[1]);
      const float D2x = __fmaf_ru(Ky, fabsf(b[1]), D1x);
      const float Kx = k_bound(D2x, F.invf[0]);
      a[0] = half_ulp_f(D[0]) + half_ulp_f(D1x) + half_ulp_f(D2x) + Kz * F.dBf[2] + Ky * F.dBf[1] +
             Kx * F.dBf[0] + F.convf[0];
      a[1] = half_ulp_f(D[1]) + half_ulp_f(D1y) + Kz * F.dBf[5] + Ky * F.dBf[4] + F.convf[1];
      a[2] = half_ulp_f(D[2]) + Kz * F.dBf[8] + F.convf[2];
    }
  }
  const float a2 = __fmaf_ru(a[2], a[2], __fmaf_ru(a[1], a[1], __fmul_ru(a[0], a[0])));
  return __fadd_ru(__fmul_ru(__fmul_ru(F.S, __fsqrt_ru(a2)), 1.0f + 0x1p-12f), tie) + 0x1p-28f;
}

// Guard words on each side of a shared-memory histogram copy: the increments
// of pairs outside [lo, hi) land there (see count_or_defer).
constexpr int kGuard = 36;

struct ItemDesc {
  FrameDev* fd;
  int32_t valid;   // 0: no more work
  int32_t h;
  int32_t pass;
  int32_t i0, ni, j0, nj;
  int32_t masked;
  int32_t skip;    // frame has no bins in this pass
};

// float32 |d'|^2 after the minimum image of the variant (NaN in, NaN out).
template <int V>
__device__ __forceinline__ float wrap_r2(float dx, float dy, float dz, const FastParams& P, bool& amb) {
  if (V == V_ORTHO) {
    dx = __fmaf_rn(-nint_scaled(dx, P.inv[0]), P.b[0], dx);
    dy = __fmaf_rn(-nint_scaled(dy, P.inv[1]), P.b[4], dy);
    dz = __fmaf_rn(-nint_scaled(dz, P.inv[2]), P.b[8], dz);
  } else if (V == V_TRIC) {
    // sequential wrap along c, b, a: the unique image inside the box-aligned brick
    float kz = nint_scaled(dz, P.inv[2]);
    dx = __fmaf_rn(-kz, P.b[2], dx);
    dy = __fmaf_rn(-kz, P.b[5], dy);
    dz = __fmaf_rn(-kz, P.b[8], dz);
    float ky = nint_scaled(dy, P.inv[1]);
    dx = __fmaf_rn(-ky, P.b[1], dx);
    dy = __fmaf_rn(-ky, P.b[4], dy);
    float kx = nint_scaled(dx, P.inv[0]);
    dx = __fmaf_rn(-kx, P.b[0], dx);
  } else if (V == V_TRIC_SEARCH) {
    // Eq. 5 wrap via back substitution, then the 27 neighbouring shifts
    float sz = __fmul_rn(dz, P.inv[2]);
    float sy = __fmul_rn(__fmaf_rn(-P.b[5], sz, dy), P.inv[1]);
    float sx = __fmul_rn(__fmaf_rn(-P.b[2], sz, __fmaf_rn(-P.b[1], sy, dx)), P.inv[0]);
    float kx = nint_f(sx), ky = nint_f(sy), kz = nint_f(sz);
    amb = (fabsf(__fsub_rn(sx, kx)) > P.amb_thr) || (fabsf(__fsub_rn(sy, ky)) > P.amb_thr) ||
          (fabsf(__fsub_rn(sz, kz)) > P.amb_thr);
    dx = __fmaf_rn(-kz, P.b[2], __fmaf_rn(-ky, P.b[1], __fmaf_rn(-kx, P.b[0], dx)));
    dy = __fmaf_rn(-kz, P.b[5], __fmaf_rn(-ky, P.b[4], dy));
    dz = __fmaf_rn(-kz, P.b[8], dz);
    float best = INFINITY;
#pragma unroll
    for (int mx = -1; mx <= 1; ++mx) {
      float ex1 = __fmaf_rn((float)mx, P.b[0], dx);
#pragma unroll
      for (int my = -1; my <= 1; ++my) {
        float ex2 = __fmaf_rn((float)my, P.b[1], ex1);
        float ey2 = __fmaf_rn((float)my, P.b[4], dy);
#pragma unroll
        for (int mz = -1; mz <= 1; ++mz) {
          float ex = __fmaf_rn((float)mz, P.b[2], ex2);
          float ey = __fmaf_rn((float)mz, P.b[5], ey2);
          float ez = __fmaf_rn((float)mz, P.b[8], dz);
          best = min_nan(best, __fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex))));
        }
      }
    }
    return best;
  }
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// ---- packed float32 arithmetic: two pairs per instruction (FFMA2/FADD2/FMUL2)

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// float32 |d'|^2 of two pairs after the minimum image of the variant; each
// component is rounded exactly as the scalar sequence of wrap_r2.  In the
// shifted modes the caller has already subtracted the tile's images from the
// coordinates, so d is the image vector itself, but for the one axis of an
// M_AXIS mode, wrapped here as wrap_r2 does.
template <int V, int MODE = M_PAIR>
__device__ __forceinline__ float2 wrap_r2_2(float2 dx, float2 dy, float2 dz, const FastParams& P, bool& amb_a,
                                            bool& amb_b) {
  const float2 M = bc2(kMagicRound), NM = bc2(-kMagicRound);
  if (shifted_mode(MODE) && (V == V_ORTHO || V == V_TRIC)) {
    if (MODE == M_AXIS + 0) {
      float2 kx = add2(fma2(dx, bc2(P.inv[0]), M), NM);
      dx = fma2(kx, bc2(-P.b[0]), dx);
    } else if (V == V_ORTHO && MODE == M_AXIS + 1) {
      float2 ky = add2(fma2(dy, bc2(P.inv[1]), M), NM);
      dy = fma2(ky, bc2(-P.b[4]), dy);
    } else if (V == V_ORTHO && MODE == M_AXIS + 2) {
      float2 kz = add2(fma2(dz, bc2(P.inv[2]), M), NM);
      dz = fma2(kz, bc2(-P.b[8]), dz);
    }
  } else if (V == V_ORTHO) {
    float2 kx = add2(fma2(dx, bc2(P.inv[0]), M), NM);
    float2 ky = add2(fma2(dy, bc2(P.inv[1]), M), NM);
    float2 kz = add2(fma2(dz, bc2(P.inv[2]), M), NM);
    dx = fma2(kx, bc2(-P.b[0]), dx);
    dy = fma2(ky, bc2(-P.b[4]), dy);
    dz = fma2(kz, bc2(-P.b[8]), dz);
  } else if (V == V_TRIC) {
    float2 kz = add2(fma2(dz, bc2(P.inv[2]), M), NM);
    dx = fma2(kz, bc2(-P.b[2]), dx);
    dy = fma2(kz, bc2(-P.b[5]), dy);
    dz = fma2(kz, bc2(-P.b[8]), dz);
    float2 ky = add2(fma2(dy, bc2(P.inv[1]), M), NM);
    dx = fma2(ky, bc2(-P.b[1]), dx);
    dy = fma2(ky, bc2(-P.b[4]), dy);
    float2 kx = add2(fma2(dx, bc2(P.inv[0]), M), NM);
    dx = fma2(kx, bc2(-P.b[0]), dx);
  } else if (V == V_TRIC_SEARCH) {
    return make_float2(wrap_r2<V>(dx.x, dy.x, dz.x, P, amb_a), wrap_r2<V>(dx.y, dy.y, dz.y, P, amb_b));
  }
  return fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
}

// Count one pair, branch free.  With sm = s_c + 1.5*2^23 (s_c the clamped root,
// bits(sm) - bits(1.5*2^23) = its nearest integer n) and the residual
// e = n^2 - q (e > 0: t < n, so floor(t) = n - 1; e < 0: floor(t) = n), the
// bin relative to the sweep is v - kb1 with v = bits(sm) + signbit(e), and the
// shared-memory address is 4 v + hbase (a shift and an add, which stay off the
// FMA pipe that the packed float32 arithmetic keeps busy; a multiply-add by 4
// measured 1-2 % slower).  Every pair increments that word.  The
// clamp of s_c to [lo - lane, hi + 1 + lane] (integers below 2^22) keeps the
// relative bin in [-1 - lane, width + 1 + lane]: pairs outside the sweep, and
// NaN pairs (s_c = hi + 1 + lane, e NaN with a clear sign bit: bin width + lane),
// land in the guard words, spread over the lanes.  A clamped pair that is
// decided is decided right: e > bound means t lies within the clamp's integer
// and the one below, e < -bound that t lies above it, out of the sweep (and
// the converse at the lower clamp).  A pair with |e| <= bound (false for NaN)
// also sets the bit `bit` of dmask: it is counted provisionally and re-decided
// by the drain, which moves its count to the exact bin when the two differ.
__device__ __forceinline__ void count_or_defer(float sm, float e, float bound, uint32_t hbase, uint32_t bit,
                                               uint32_t& dmask) {
  asm volatile(
      "{\n\t.reg .pred pn;\n\t.reg .u32 eb, sg, v, addr;\n\t.reg .f32 ae;\n\t"
      "mov.b32 eb, %2;\n\t"
      "shr.u32 sg, eb, 31;\n\t"
      "add.u32 v, %1, sg;\n\t"
      "shl.b32 addr, v, 2;\n\t"
      "add.u32 addr, addr, %4;\n\t"
      "abs.f32 ae, %2;\n\t"
      "setp.gtu.f32 pn, ae, %3;\n\t"
      "@!pn or.b32 %0, %0, %5;\n\t"
      "red.shared.add.u32 [addr], 1;\n\t"
      "}"
      : "+r"(dmask)
      : "r"(__float_as_uint(sm)), "f"(e), "f"(bound), "r"(hbase), "r"(bit));
}

// The same with the increments of the warp aggregated in software (the hybrid
// strategy of Sec. 2.4 taken to the warp: lanes that hit one word add their
// count once): the lanes with equal addresses are found with match.any, and the
// lowest of them adds their number.  Called by all 32 lanes together.  The
// address is formed in the same instructions as count_or_defer.
__device__ __forceinline__ void count_or_defer_agg(float sm, float e, float bound, uint32_t hbase, uint32_t bit,
                                                   uint32_t& dmask) {
  asm volatile(
      "{\n\t.reg .pred pn, pl;\n\t.reg .u32 eb, sg, v, addr, peers, lm, cnt;\n\t.reg .f32 ae;\n\t"
      "mov.b32 eb, %2;\n\t"
      "shr.u32 sg, eb, 31;\n\t"
      "add.u32 v, %1, sg;\n\t"
      "shl.b32 addr, v, 2;\n\t"
      "add.u32 addr, addr, %4;\n\t"
      "abs.f32 ae, %2;\n\t"
      "setp.gtu.f32 pn, ae, %3;\n\t"
      "@!pn or.b32 %0, %0, %5;\n\t"
      "match.any.sync.b32 peers, addr, 0xffffffff;\n\t"
      "mov.u32 lm, %%lanemask_lt;\n\t"
      "and.b32 lm, lm, peers;\n\t"
      "setp.eq.u32 pl, lm, 0;\n\t"
      "popc.b32 cnt, peers;\n\t"
      "@pl red.shared.add.u32 [addr], cnt;\n\t"
      "}"
      : "+r"(dmask)
      : "r"(__float_as_uint(sm)), "f"(e), "f"(bound), "r"(hbase), "r"(bit)
      : "memory");
}

// The float32 decision of two pairs (j, j+1 against one i).  With q = r^2 S^2
// (= t^2) and n the integer nearest to the clamped root s_c, the residual
// e = n^2 - q is rounded once (fma), so its sign gives floor(t) = n or n-1, and
// |e| is compared with the bound derived in frame_setup_kernel; within it the
// pair is deferred.  The clamp (chi = hi + 1 + lane, and clo = lo - lane for
// sweeps that start above bin 0) sends far pairs to guard words with a large
// |e|, so they are not deferred; NaN pairs are never deferred.
// decide_arith2 returns sm = s_c + 1.5*2^23, e and the bound as float pairs
// (search variant: ambiguous images force the bound to +inf so the pair is
// deferred); count_or_defer acts on them.
template <int V, bool MULTI, int MODE = M_PAIR>
__device__ __forceinline__ void decide_arith2(float2 dx, float2 dy, float2 dz, const FastParams& P, float chi,
                                              float clo, float2& sm, float2& e, float2& bound) {
  bool amb_a = false, amb_b = false;
  float2 r2 = wrap_r2_2<V, MODE>(dx, dy, dz, P, amb_a, amb_b);
  float2 nq = mul2(r2, bc2(-P.S2));  // -q
  float2 sq = make_float2(sqrt_approx(-nq.x), sqrt_approx(-nq.y));
  // NaN -> chi; a no-box tile of an in-range frame (M_UNI) has neither NaN nor
  // roots near the clamp
  float2 sc = (V == V_NONE && MODE == M_UNI) ? sq : make_float2(fminf(sq.x, chi), fminf(sq.y, chi));
  if (MULTI) sc = make_float2(fmaxf(sc.x, clo), fmaxf(sc.y, clo));
  sm = add2(sc, bc2(kMagicRound));
  float2 n = add2(sm, bc2(-kMagicRound));
  e = fma2(n, n, nq);  // n^2 - q
  bound = fma2(nq, bc2(-P.qb1), bc2(P.qb0));
  if (V == V_TRIC_SEARCH) {
    if (amb_a) bound.x = INFINITY;
    if (amb_b) bound.y = INFINITY;
  }
}

// The same decision as count_or_defer, as values (used by the self check;
// single sweep, lane 0's clamp).
template <int V>
__device__ __forceinline__ void fast_decide2(float2 dx, float2 dy, float2 dz, const FastParams& P, bool& near_a,
                                             bool& near_b, uint32_t& rel_a, uint32_t& rel_b) {
  float2 sm, e, bound;
  decide_arith2<V, false>(dx, dy, dz, P, (float)(P.hi + 1), 0.0f, sm, e, bound);
  near_a = fabsf(e.x) <= bound.x;
  near_b = fabsf(e.y) <= bound.y;
  rel_a = __float_as_uint(sm.x) + (__float_as_uint(e.x) >> 31) - (uint32_t)P.kb1;
  rel_b = __float_as_uint(sm.y) + (__float_as_uint(e.y) >> 31) - (uint32_t)P.kb1;
}

// The relative bin at which the float32 path counted a pair (provisionally,
// if it deferred it): the scalar replay of decide_arith2 and count_or_defer,
// operation for operation, for the lane `src_lane` that evaluated the pair.
template <int V, bool MULTI, int MODE = M_PAIR>
__device__ __forceinline__ int provisional_rel(const FastParams& P, float4 pi, float4 pj, int src_lane,
                                               float3 ti = make_float3(0.f, 0.f, 0.f),
                                               float3 sj = make_float3(0.f, 0.f, 0.f)) {
  bool amb = false;
  float r2;
  if ((V == V_ORTHO || V == V_TRIC) && shifted_mode(MODE)) {  // the coordinates shifted by the tile's images
    float dx = __fsub_rn(__fsub_rn(pj.x, sj.x), __fsub_rn(pi.x, ti.x));
    float dy = __fsub_rn(__fsub_rn(pj.y, sj.y), __fsub_rn(pi.y, ti.y));
    float dz = __fsub_rn(__fsub_rn(pj.z, sj.z), __fsub_rn(pi.z, ti.z));
    if (MODE == M_AXIS + 0) dx = __fmaf_rn(-nint_scaled(dx, P.inv[0]), P.b[0], dx);
    if (V == V_ORTHO && MODE == M_AXIS + 1) dy = __fmaf_rn(-nint_scaled(dy, P.inv[1]), P.b[4], dy);
    if (V == V_ORTHO && MODE == M_AXIS + 2) dz = __fmaf_rn(-nint_scaled(dz, P.inv[2]), P.b[8], dz);
    r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
  } else {
    r2 = wrap_r2<V>(__fadd_rn(pj.x, -pi.x), __fadd_rn(pj.y, -pi.y), __fadd_rn(pj.z, -pi.z), P, amb);
  }
  float nq = __fmul_rn(r2, -P.S2);
  float sc = fminf(sqrt_approx(-nq), (float)(P.hi + 1 + src_lane));
  if (MULTI) sc = fmaxf(sc, (float)(P.lo - src_lane));
  float sm = __fadd_rn(sc, kMagicRound);
  float n = __fadd_rn(sm, -kMagicRound);
  float e = __fmaf_rn(n, n, nq);
  return (int)(__float_as_uint(sm) + (__float_as_uint(e) >> 31) - (uint32_t)P.kb1);
}

// ---- double-float middle tier

struct DF {
  float h, l;  // unevaluated sum h + l
};

__device__ __forceinline__ DF two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
// v - k (bh + bl) for an integer k, renormalised: after a large image is
// taken off, the low part of v (the rounding error of a difference of large
// coordinates) can be far above an ulp of the small result, and the products
// of df_norm2 are accurate only for a normalised pair (|l| <= ulp(h) / 2)
__device__ __forceinline__ DF df_sub_kb(DF v, float k, float bh, float bl) {
  DF p = two_prod(k, bh);
  DF s = two_sum(v.h, -p.h);
  float low = __fmaf_rn(-k, bl, __fsub_rn(__fadd_rn(v.l, s.l), p.l));
  return two_sum(s.h, low);
}
__device__ __forceinline__ DF df_norm2(DF x, DF y, DF z) {
  DF ax = two_prod(x.h, x.h), ay = two_prod(y.h, y.h), az = two_prod(z.h, z.h);
  DF s1 = two_sum(ax.h, ay.h);
  DF s2 = two_sum(s1.h, az.h);
  float low = __fadd_rn(__fadd_rn(__fadd_rn(ax.l, ay.l), __fadd_rn(az.l, s1.l)), s2.l);
  low = __fmaf_rn(__fadd_rn(x.h, x.h), x.l, low);
  low = __fmaf_rn(__fadd_rn(y.h, y.h), y.l, low);
  low = __fmaf_rn(__fadd_rn(z.h, z.h), z.l, low);
  low = __fmaf_rn(x.l, x.l, __fmaf_rn(y.l, y.l, __fmaf_rn(z.l, z.l, low)));
  return {s2.h, low};
}

// xj - xi for binary64 values, as a double-float: each value split into float32
// high and low parts (x = h + l to about 2^-48 |x|), the high parts subtracted
// exactly and the low parts added to the error term.
__device__ __forceinline__ DF df_diff64(double xj, double xi) {
  const float hj = __double2float_rn(xj), hi = __double2float_rn(xi);
  const float lj = __double2float_rn(__dsub_rn(xj, (double)hj)), li = __double2float_rn(__dsub_rn(xi, (double)hi));
  DF s = two_sum(hj, -hi);
  return two_sum(s.h, __fadd_rn(s.l, __fsub_rn(lj, li)));  // renormalised (see df_sub_kb)
}

// Bin of a deferred pair from r^2 evaluated in double-float arithmetic (about
// 44 bits, with the exact coordinate differences (float32 input; binary64
// input to about 2^-47 of the coordinate magnitude) and the same nearest images
// as the float32 path), compared with the split binary64 threshold of the
// nearest edge.  Returns -1 when even this is too close to call.  i, j:
// frame-local indices; pi, pj: the float32 coordinates.
template <int V>
__device__ int mid_bin(const FrameDev& F, int i, int j, float4 pi, float4 pj) {
  if (V == V_TRIC_SEARCH) return -1;
  DF dx, dy, dz;
  if (F.X64) {
    const double4 a = F.X64[i], b = F.X64[j];
    dx = df_diff64(b.x, a.x);
    dy = df_diff64(b.y, a.y);
    dz = df_diff64(b.z, a.z);
  } else {
    dx = two_sum(pj.x, -pi.x);
    dy = two_sum(pj.y, -pi.y);
    dz = two_sum(pj.z, -pi.z);
  }
  if (V == V_ORTHO) {
    float kx = nint_scaled(dx.h, F.invf[0]), ky = nint_scaled(dy.h, F.invf[1]), kz = nint_scaled(dz.h, F.invf[2]);
    dx = df_sub_kb(dx, kx, F.Bf[0], F.Bl[0]);
    dy = df_sub_kb(dy, ky, F.Bf[4], F.Bl[4]);
    dz = df_sub_kb(dz, kz, F.Bf[8], F.Bl[8]);
    // float32 and binary64 may pick different images near |d'_c| = L_c/2; and the
    // images must be nearest at all (the nearest integer via 1.5 2^23 is exact
    // only below 2^22 cells): the wrapped components strictly inside L_c/2
    if (fabsf(fabsf(dx.h) - 0.5f * F.Bf[0]) <= F.tie_eps || fabsf(fabsf(dy.h) - 0.5f * F.Bf[4]) <= F.tie_eps ||
        fabsf(fabsf(dz.h) - 0.5f * F.Bf[8]) <= F.tie_eps)
      return -1;
    const float lim = 0.5f - 0x1p-20f;
    if (!(fabsf(dx.h * F.invf[0]) < lim && fabsf(dy.h * F.invf[1]) < lim && fabsf(dz.h * F.invf[2]) < lim)) return -1;
  } else if (V == V_TRIC) {
    // the nearest-image integers of the float32 path, replayed exactly
    float kz = nint_scaled(dz.h, F.invf[2]);
    float fx1 = __fmaf_rn(-kz, F.Bf[2], dx.h);
    float fy1 = __fmaf_rn(-kz, F.Bf[5], dy.h);
    float ky = nint_scaled(fy1, F.invf[1]);
    float fx2 = __fmaf_rn(-ky, F.Bf[1], fx1);
    float kx = nint_scaled(fx2, F.invf[0]);
    dx = df_sub_kb(df_sub_kb(df_sub_kb(dx, kz, F.Bf[2], F.Bl[2]), ky, F.Bf[1], F.Bl[1]), kx, F.Bf[0], F.Bl[0]);
    dy = df_sub_kb(df_sub_kb(dy, kz, F.Bf[5], F.Bl[5]), ky, F.Bf[4], F.Bl[4]);
    dz = df_sub_kb(dz, kz, F.Bf[8], F.Bl[8]);
    // The images are the float32 path's; they are the exact sequential nearest
    // planes along c, b, a (Babai's step, whose vector is the minimum image of
    // every pair closer than half the smallest plane spacing) when the wrapped
    // components lie strictly inside half the periods cz, by, ax: checked here on
    // the accurate values (the frame's float32 errors may be too large for the
    // images of its float32 path, e.g. far-unwrapped coordinates).  Otherwise the
    // binary64 replay decides.
    const float lim = 0.5f - 0x1p-20f;
    if (!(fabsf(dz.h * F.invf[2]) < lim && fabsf(dy.h * F.invf[1]) < lim && fabsf(dx.h * F.invf[0]) < lim))
      return -1;
  }
  DF r2 = df_norm2(dx, dy, dz);
  float s = sqrt_approx(__fmul_rn(r2.h, F.S2));
  float n = nint_f(s);
  if (!(n >= 0.5f)) return 0;  // t below 1/2: bin 0
  if (n > (float)F.nbins) return F.nbins;
  int ni = (int)n;
  float2 T = __ldg(F.Tf + ni);
  float diff = __fadd_rn(__fsub_rn(r2.h, T.x), __fsub_rn(r2.l, T.y));
  float bound = __fmaf_rn(F.mid2, r2.h, __fmul_rn(F.mid1, s));
  if (!(fabsf(diff) > bound)) return -1;
  return diff >= 0.0f ? ni : ni - 1;
}

// ---- binary64 last resort

// Squared minimum-image distance in binary64, the same operations in the same
// order as the definition (Alg. 1, Eq. 5, 27 neighbouring shifts); the
// coordinates are the caller's (float32 promoted exactly, or binary64).
template <int V>
__device__ double exact_r2(const FrameDev& F, double3 pi, double3 pj) {
  double dx = __dsub_rn(pj.x, pi.x);
  double dy = __dsub_rn(pj.y, pi.y);
  double dz = __dsub_rn(pj.z, pi.z);
  const double* B = F.B;
  if (V == V_ORTHO) {
    double kx = rint(__dmul_rn(dx, F.Linv[0]));
    double ky = rint(__dmul_rn(dy, F.Linv[1]));
    double kz = rint(__dmul_rn(dz, F.Linv[2]));
    dx = __fma_rn(-kx, B[0], dx);
    dy = __fma_rn(-ky, B[4], dy);
    dz = __fma_rn(-kz, B[8], dz);
  } else if (V == V_TRIC || V == V_TRIC_SEARCH) {
    const double ax = B[0], bx = B[1], cx = B[2], by = B[4], cy = B[5], cz = B[8];
    double sz = __ddiv_rn(dz, cz);
    double sy = __ddiv_rn(__dsub_rn(dy, __dmul_rn(cy, sz)), by);
    double sx = __ddiv_rn(__dsub_rn(__dsub_rn(dx, __dmul_rn(bx, sy)), __dmul_rn(cx, sz)), ax);
    double kx = rint(sx), ky = rint(sy), kz = rint(sz);
    dx = __dsub_rn(__dsub_rn(__dsub_rn(dx, __dmul_rn(ax, kx)), __dmul_rn(bx, ky)), __dmul_rn(cx, kz));
    dy = __dsub_rn(__dsub_rn(dy, __dmul_rn(by, ky)), __dmul_rn(cy, kz));
    dz = __dsub_rn(dz, __dmul_rn(cz, kz));
    // Below half the plane spacing (V_TRIC: r_max <= (1 - 2^-8) h_min / 2) the
    // shift m = 0 is the minimum of the 27 for every pair inside r_max: the
    // sequential rounding is Babai's nearest plane in the upper-triangular
    // basis, exact for vectors shorter than half its smallest Gram-Schmidt
    // length (cz, by, ax >= h_min), and every other shift is longer than
    // h_min - r_max > r_max.  Its value is the m = 0 term of the loop, bit for
    // bit (adding the zero products changes nothing); a pair beyond r_max stays
    // beyond it under any shift.  So the binary64 bin is the definition's.
    if (V == V_TRIC) return __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
    double best = INFINITY;
#pragma unroll 1
    for (int mx = -1; mx <= 1; ++mx)
#pragma unroll 1
      for (int my = -1; my <= 1; ++my)
#pragma unroll 1
        for (int mz = -1; mz <= 1; ++mz) {
          double ex = __dadd_rn(__dadd_rn(__dadd_rn(dx, __dmul_rn(ax, (double)mx)), __dmul_rn(bx, (double)my)),
                                __dmul_rn(cx, (double)mz));
          double ey = __dadd_rn(__dadd_rn(dy, __dmul_rn(by, (double)my)), __dmul_rn(cy, (double)mz));
          double ez = __dadd_rn(dz, __dmul_rn(cz, (double)mz));
          double r2 = __fma_rn(ez, ez, __fma_rn(ey, ey, __dmul_rn(ex, ex)));
          if (r2 < best) best = r2;
        }
    return best;
  }
  return __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
}

// Bin of a binary64 r^2 from the threshold table: the largest k with T[k] <= r2
// (T[0] = 0, T nondecreasing; 0 for NaN).  The float32 estimate S sqrt(r2) is
// within a bin or two of it; the two walks make the result exact whatever the
// estimate, with one or two dependent loads instead of a binary search's
// log2(nbins).
__device__ __forceinline__ int bin_from_thresholds(const double* __restrict__ T, float S, int nbins, double r2) {
  if (!(r2 >= 0.0)) return 0;
  int k = (int)fminf(__fmul_rn(sqrtf(__double2float_rn(r2)), S), (float)nbins);
  while (k > 0 && __ldg(T + k) > r2) --k;
  while (k < nbins && __ldg(T + k + 1) <= r2) ++k;
  return k;
}

// The caller's coordinates of particle i of a frame, in binary64.
__device__ __forceinline__ double3 coords64(const FrameDev& F, int i) {
  if (F.X64) {
    double4 p = F.X64[i];
    return make_double3(p.x, p.y, p.z);
  }
  float4 p = __ldg(F.X + i);
  return make_double3((double)p.x, (double)p.y, (double)p.z);
}

// The binary64 replay of one pair (about one deferred pair in 10^4): out of
// line, so that its code and registers stay out of the pair loop.
template <int V>
__device__ __noinline__ int exact_bin(const FrameDev& F, int i, int j) {
  return bin_from_thresholds(F.T, F.S, F.nbins, exact_r2<V>(F, coords64(F, i), coords64(F, j)));
}

// Exact bin of one deferred pair (frame-local indices i, j; float32 copies pi,
// pj): the double-float tier, then the binary64 replay.
template <int V>
__device__ __forceinline__ int deferred_bin(const FrameDev& F, int i, int j, float4 pi, float4 pj,
                                            unsigned& nexact) {
  int k = mid_bin<V>(F, i, j, pi, pj);
  if (k < 0) {
    k = exact_bin<V>(F, i, j);
    ++nexact;
  }
  return k;
}
// The no-box variant's drain is faster with the double-float tier out of line too.
template <int V>
__device__ __noinline__ int deferred_bin_call(const FrameDev& F, int i, int j, float4 pi, float4 pj,
                                              unsigned& nexact) {
  return deferred_bin<V>(F, i, j, pi, pj, nexact);
}

__device__ void load_fast_params(const FrameDev& F, int pass, FastParams& P);

// Decide the first `count` (<= 32) queued pairs, one per lane, move the
// provisional count of each to its exact bin where they differ, and shift the
// rest of the queue down.  A queue entry is (i - i0) | (j - j0) << 16 for the
// tile's first i and j; lane (i - i0) mod 32 evaluated the pair.
template <int V, bool MULTI, int MODE = M_PAIR>
__device__ __forceinline__ int drain_queue_body(const FrameDev* F, int pass, int i0, int j0, uint32_t* q, int qcount,
                                                uint32_t* sh, int lane, float3 ti = make_float3(0.f, 0.f, 0.f),
                                                float3 sj = make_float3(0.f, 0.f, 0.f)) {
  const int count = qcount < 32 ? qcount : 32;
  unsigned nexact = 0;
  if (lane < count) {
    const uint32_t e = q[lane];
    const int il = (int)(e & 0xFFFFu), jl = (int)(e >> 16);
    float4 pi = __ldg(F->X + i0 + il);
    float4 pj = __ldg(F->X + j0 + jl);
    FastParams P;
    load_fast_params(*F, pass, P);
    int relp = provisional_rel<V, MULTI, MODE>(P, pi, pj, il & 31, ti, sj);
    int relx = (V == V_NONE ? deferred_bin_call<V>(*F, i0 + il, j0 + jl, pi, pj, nexact)
                            : deferred_bin<V>(*F, i0 + il, j0 + jl, pi, pj, nexact)) - P.lo;
    if (relx != relp) {
      atomicAdd(sh + relp, 0xFFFFFFFFu);  // relp lies in the histogram or its guard words
      if ((uint32_t)relx < P.width) atomicAdd(sh + relx, 1u);
    }
  }
  __syncwarp();
  int rest = qcount - count;
  if (lane < rest) q[lane] = q[32 + lane];
  __syncwarp();
  for (int o = 16; o > 0; o >>= 1) nexact += __shfl_xor_sync(kFull, nexact, o);
  if (lane == 0 && nexact) atomicAdd(&const_cast<FrameDev*>(F)->exact, (unsigned long long)nexact);
  return rest;
}

template <int V, bool MULTI, int MODE = M_PAIR>
__device__ __noinline__ int drain_queue_call(const FrameDev* F, int pass, int i0, int j0, uint32_t* q, int qcount,
                                             uint32_t* sh, int lane, float3 ti = make_float3(0.f, 0.f, 0.f),
                                             float3 sj = make_float3(0.f, 0.f, 0.f)) {
  return drain_queue_body<V, MULTI, MODE>(F, pass, i0, j0, q, qcount, sh, lane, ti, sj);
}

// The register allocation of the hot loop and the size of its code decide which
// form is faster (measured): the triclinic variant keeps fewer live values across
// an inlined drain than across a call; the no-box variant is faster with the
// call, and so is the orthorhombic one, whose seven pair-loop instances (one per
// tile mode) otherwise outgrow the instruction cache (one out-of-line copy per
// mode: +0.4 % on the headline frame, +4 % on C2).
template <int V, bool MULTI, int MODE>
__device__ __forceinline__ int drain_queue(const FrameDev* F, int pass, int i0, int j0, uint32_t* q, int qcount,
                                           uint32_t* sh, int lane, float3 ti, float3 sj) {
  if constexpr (V == V_TRIC)
    return drain_queue_body<V, MULTI, MODE>(F, pass, i0, j0, q, qcount, sh, lane, ti, sj);
  else if constexpr (V == V_ORTHO)
    return drain_queue_call<V, MULTI, MODE>(F, pass, i0, j0, q, qcount, sh, lane, ti, sj);
  else
    return drain_queue_call<V, MULTI>(F, pass, i0, j0, q, qcount, sh, lane);
}

// j tile in shared memory as pairs of particles: A[p] = {x_2p, x_2p+1, y_2p, y_2p+1},
// Z[p] = {z_2p, z_2p+1}, so one LDS.128 + one LDS.64 feed two j particles.
// The i run `run` of the item (32 * RI consecutive i particles, lane + 32 r of
// it in this lane) against j particles [jb, je) of the staged tile (jb a
// multiple of kSubJ).
template <int V, bool MASKED, bool MULTI, int RI, int MODE, bool AGG>
__device__ __forceinline__ void run_tile(const FrameDev* F, const FastParams& P, const ItemDesc& it,
                                         const float4* __restrict__ sjA, const float2* __restrict__ sjZ,
                                         uint32_t* sh, uint32_t* q, int run, int lane, unsigned& ndeferred,
                                         float3 kt, int jb, int je) {
  const int ib = run * (32 * RI) + lane;
  // tile images: the image is subtracted from the coordinates, ti from the i's and
  // sj from the j's.  Orthorhombic (exact, see tile_image): k = -1 takes L from
  // the i's, k = +1 from the j's.  Triclinic: the i's move by the image vector
  // B k, rounded once (|k| <= 1, so the products are exact).
  constexpr bool SH = (V == V_ORTHO || V == V_TRIC) && shifted_mode(MODE);
  float3 ti = make_float3(0.f, 0.f, 0.f), sj = make_float3(0.f, 0.f, 0.f);
  if (V == V_ORTHO && SH) {
    ti = make_float3(kt.x < 0.f ? P.b[0] : 0.f, kt.y < 0.f ? P.b[4] : 0.f, kt.z < 0.f ? P.b[8] : 0.f);
    sj = make_float3(kt.x > 0.f ? P.b[0] : 0.f, kt.y > 0.f ? P.b[4] : 0.f, kt.z > 0.f ? P.b[8] : 0.f);
  } else if (V == V_TRIC && SH) {
    const float* v = F->tshift[9 * (int)(kt.x + 1.0f) + 3 * (int)(kt.y + 1.0f) + (int)(kt.z + 1.0f)];
    ti = make_float3(v[0], v[1], v[2]);
  }
  float2 xi[RI], yi[RI], zi[RI];  // i coordinates broadcast to both halves
#pragma unroll
  for (int r = 0; r < RI; ++r) {
    int li = ib + 32 * r;
    float x = __int_as_float(0x7fffffff), y = x, z = x;
    if (li < it.ni) {
      float4 p = __ldg(F->X + it.i0 + li);
      x = p.x; y = p.y; z = p.z;
      if (SH) {
        x = __fsub_rn(x, ti.x);
        y = __fsub_rn(y, ti.y);
        z = __fsub_rn(z, ti.z);
      }
    }
    xi[r] = bc2(-x); yi[r] = bc2(-y); zi[r] = bc2(-z);  // negated: d = xj + (-xi)
  }
  const unsigned lt_mask = (1u << lane) - 1u;
  const float qnan = __int_as_float(0x7fffffff);
  // address of bin rel = 4 (rel + kb1) + hbase (mod 2^32); clamp of the root per lane
  const uint32_t hbase = (uint32_t)__cvta_generic_to_shared(sh) - 4u * (uint32_t)P.kb1;
  const float chi = (float)(P.hi + 1 + lane);
  const float clo = (float)(P.lo - lane);
  constexpr int kJU = ju_of<V, RI>();
  const int nj4 = (je + kJU - 1) & ~(kJU - 1);  // the j tile is padded with NaN particles
  int qcount = 0;
  for (int jj0 = jb; jj0 < nj4; jj0 += kJU) {
    uint32_t dmask = 0u;
    // (u, r) are compile-time constants after unrolling: they name the mask bit
#pragma unroll
    for (int u = 0; u < kJU; u += 2) {
      const float4 A = sjA[(jj0 + u) >> 1];
      float2 Z = sjZ[(jj0 + u) >> 1];
      float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
      if (V == V_ORTHO && SH) {  // (the wrapped axis of an M_AXIS mode has no shift)
        if (MODE != M_AXIS + 0) xj = add2(xj, bc2(-sj.x));
        if (MODE != M_AXIS + 1) yj = add2(yj, bc2(-sj.y));
        if (MODE != M_AXIS + 2) Z = add2(Z, bc2(-sj.z));
      }
#pragma unroll
      for (int r = 0; r < RI; ++r) {
        float2 dx = add2(xj, xi[r]);
        float2 dy = add2(yj, yi[r]);
        float2 dz = add2(Z, zi[r]);
        if (MASKED) {
          // intra-species: only j > i; all three components so no later test sees a number
          const int ig = it.i0 + ib + 32 * r, jg = it.j0 + jj0 + u;
          if (!(jg > ig)) { dx.x = qnan; dy.x = qnan; dz.x = qnan; }
          if (!(jg + 1 > ig)) { dx.y = qnan; dy.y = qnan; dz.y = qnan; }
        }
        float2 sm, e, bound;
        decide_arith2<V, MULTI, MODE>(dx, dy, dz, P, chi, clo, sm, e, bound);
        if (AGG) {
          count_or_defer_agg(sm.x, e.x, bound.x, hbase, 1u << (u * RI + r), dmask);
          count_or_defer_agg(sm.y, e.y, bound.y, hbase, 1u << ((u + 1) * RI + r), dmask);
        } else {
          count_or_defer(sm.x, e.x, bound.x, hbase, 1u << (u * RI + r), dmask);
          count_or_defer(sm.y, e.y, bound.y, hbase, 1u << ((u + 1) * RI + r), dmask);
        }
      }
    }
    // queue the deferred pairs: one per lane per round, compacted with a ballot
    unsigned bal = __ballot_sync(kFull, dmask != 0u);
    while (bal) {
      if (dmask) {
        int b = __ffs(dmask) - 1;
        dmask &= dmask - 1u;
        int pos = qcount + __popc(bal & lt_mask);
        q[pos] = (uint32_t)(ib + 32 * (b % RI)) | ((uint32_t)(jj0 + b / RI) << 16);
      }
      int added = __popc(bal);
      qcount += added;
      ndeferred += added;
      if (qcount >= 32) {
        __syncwarp();
        qcount = drain_queue<V, MULTI, MODE>(F, it.pass, it.i0, it.j0, q, qcount, sh, lane, ti, sj);
      }
      bal = __ballot_sync(kFull, dmask != 0u);
    }
  }
  __syncwarp();
  if (qcount > 0) drain_queue<V, MULTI, MODE>(F, it.pass, it.i0, it.j0, q, qcount, sh, lane, ti, sj);
  __syncwarp();
}

// Tiles of an item claimed dynamically: the warps take (i run, j sub-chunk)
// tiles from lists per cost class, costliest first, so that a block's warps
// reach the barrier at the end of the item within about one tile of each other
// whatever mix of tile modes and culled tiles the item holds.
constexpr int kSubPerTile = kTile / kSubJ;  // j sub-chunks per item
constexpr int kCostClasses = 3;             // per-pair images, one axis per pair, uniform image
struct TileLists {
  unsigned char* list;  // kCostClasses lists of tile indices run * kSubPerTile + c, each `cap` long
  int* count;           // per class, then the claim counter
  int cap;
};

// The cost class of a tile that runs in `mode` (after the demotion of masked tiles).
__device__ __forceinline__ int cost_class(int mode) { return mode == M_PAIR ? 0 : (mode == M_UNI ? 2 : 1); }

// The decision parameters are reloaded per item (from the L1-cached frame
// descriptor) so that only the fields of this variant are live in the loop.
// MULTI: some sweep of the launch starts above bin 0, so the root is also
// clamped from below (valid for every sweep, a separate kernel for registers).
// For the periodic variants (and no-box frames that bound their tiles) the j
// tile is taken in sub-chunks of kSubJ particles; img[t] and tbeta[t] are the
// image, mode (w) and beta of tile t = run * kSubPerTile + c, listed in `tl`.
// Masked items (the diagonal of a species block) run every tile with
// per-pair images (fewer instances).
template <int V, bool MULTI, int RI, bool AGG>
__device__ void run_item(const FrameDev* F, const ItemDesc& it, const float4* sjA, const float2* sjZ, uint32_t* sh,
                         uint32_t* q, int warp, int lane, unsigned& ndeferred, const float4* img, const float* tbeta,
                         TileLists tl, bool bounds) {
  FastParams P;
  load_fast_params(*F, it.pass, P);
  if (V == V_ORTHO || V == V_TRIC || (V == V_NONE && bounds)) {
    const int n0 = tl.count[0], n1 = n0 + tl.count[1], n = n1 + tl.count[2];
    for (;;) {
      int g = 0;
      if (lane == 0) g = atomicAdd(tl.count + kCostClasses, 1);
      g = __shfl_sync(kFull, g, 0);
      if (g >= n) break;
      const int k = g < n0 ? (int)tl.list[g] : (g < n1 ? (int)tl.list[tl.cap + g - n0] : (int)tl.list[2 * tl.cap + g - n1]);
      const int run = k / kSubPerTile, c = k - run * kSubPerTile;
      const int jb = c * kSubJ, je = min(it.nj, jb + kSubJ);
      const float3 k0 = make_float3(0.f, 0.f, 0.f);
      if (V == V_NONE) {
        if (it.masked) run_tile<V, true, MULTI, RI, M_PAIR, AGG>(F, P, it, sjA, sjZ, sh, q, run, lane, ndeferred, k0, jb, je);
        else run_tile<V, false, MULTI, RI, M_PAIR, AGG>(F, P, it, sjA, sjZ, sh, q, run, lane, ndeferred, k0, jb, je);
        continue;
      }
      const float4 im = img[k];
      const float3 kt = make_float3(im.x, im.y, im.z);
      const int mode = it.masked ? M_PAIR : (int)im.w;
      // the tile's own beta; masked tiles demoted to per-pair images take the frame's
      if (mode == (int)im.w) set_bound_beta(*F, P, tbeta[k]);
      else set_bound(*F, P, mode);
#define DH_TILE(M_, K_) run_tile<V, M_, MULTI, RI, K_, AGG>(F, P, it, sjA, sjZ, sh, q, run, lane, ndeferred, kt, jb, je)
      if (it.masked) {
        DH_TILE(true, M_PAIR);
      } else {
        switch (mode) {
          case M_UNI: DH_TILE(false, M_UNI); break;
          case M_AXIS + 0: DH_TILE(false, M_AXIS + 0); break;
          case M_AXIS + 1: if (V == V_ORTHO) DH_TILE(false, M_AXIS + 1); break;
          case M_AXIS + 2: if (V == V_ORTHO) DH_TILE(false, M_AXIS + 2); break;
          default: DH_TILE(false, M_PAIR); break;
        }
      }
#undef DH_TILE
    }
    return;
  }
  const float3 k0 = make_float3(0.f, 0.f, 0.f);
  if (it.masked) {
    run_tile<V, true, MULTI, RI, M_PAIR, AGG>(F, P, it, sjA, sjZ, sh, q, warp, lane, ndeferred, k0, 0, it.nj);
  } else if (V == V_NONE && F->in_range && it.ni == kTile && (it.nj % kJUMax) == 0) {
    // every pair real (no NaN padding) and in range: the root needs no clamp
    run_tile<V, false, MULTI, RI, M_UNI, AGG>(F, P, it, sjA, sjZ, sh, q, warp, lane, ndeferred, k0, 0, it.nj);
  } else {
    run_tile<V, false, MULTI, RI, M_PAIR, AGG>(F, P, it, sjA, sjZ, sh, q, warp, lane, ndeferred, k0, 0, it.nj);
  }
}

// The nearest-image integers of a tile pair, when the float32 per-pair path
// would compute the same ones for every pair of it.  lo/hi bound the i and j
// coordinates per axis.  The per-pair path rounds d = xj - xi, then k =
// nint(d / L) (triclinic: along c, b, a, each after the previous images are
// subtracted); every step is a correctly rounded monotone function of d, so
// the tile's extreme differences fl(jmin - imax) and fl(jmax - imin) bound the
// value of every pair at every step, and equal integers at both ends are the
// integers of every pair.  Returns (kx, ky, kz, mode): M_UNI in that case;
// M_AXIS + a when that holds for every axis but a (orthorhombic; triclinic:
// for c and b, a = 0), whose k is then 0 and wrapped per pair; M_PAIR else.
template <int V>
__device__ float4 tile_image(const FrameDev& F, const float* imin, const float* imax, const float* jmin,
                             const float* jmax) {
  float lo[3], hi[3];
  for (int c = 0; c < 3; ++c) {
    lo[c] = __fsub_rn(jmin[c], imax[c]);
    hi[c] = __fsub_rn(jmax[c], imin[c]);
  }
  const float* b = F.Bf;
  if (V == V_ORTHO) {
    // and each image must be exactly subtractable from the coordinates it moves:
    // k = +1 from the j's, k = -1 from the i's, which Sterbenz's lemma grants when
    // they lie in [L/2, 2L]
    // (widened by tie_m, so that no pair lies where float32 and binary64 may
    // round d/L to different images); an axis that fails is wrapped per pair
    float k[3];
    int nw = 0, wa = 0;
    for (int c = 0; c < 3; ++c) {
      k[c] = nint_scaled(__fsub_rn(lo[c], F.tie_m[c]), F.invf[c]);
      const float L = b[4 * c];
      bool ok = nint_scaled(__fadd_rn(hi[c], F.tie_m[c]), F.invf[c]) == k[c] &&
                ((k[c] == 0.0f) || (k[c] == 1.0f && jmin[c] >= 0.5f * L && jmax[c] <= 2.0f * L) ||
                 (k[c] == -1.0f && imin[c] >= 0.5f * L && imax[c] <= 2.0f * L));
      if (!ok) {
        ++nw;
        wa = c;
        k[c] = 0.0f;
      }
    }
    if (nw > 1) return make_float4(0.f, 0.f, 0.f, (float)M_PAIR);
    return make_float4(k[0], k[1], k[2], nw == 0 ? (float)M_UNI : (float)(M_AXIS + wa));
  } else {
    // z, then y and x after the c image, then x after the b image
    const float kz = nint_scaled(lo[2], F.invf[2]);
    if (!(nint_scaled(hi[2], F.invf[2]) == kz)) return make_float4(0.f, 0.f, 0.f, 0.f);
    float ylo = __fmaf_rn(kz, -b[5], lo[1]), yhi = __fmaf_rn(kz, -b[5], hi[1]);
    float xlo = __fmaf_rn(kz, -b[2], lo[0]), xhi = __fmaf_rn(kz, -b[2], hi[0]);
    const float ky = nint_scaled(ylo, F.invf[1]);
    if (!(nint_scaled(yhi, F.invf[1]) == ky)) return make_float4(0.f, 0.f, 0.f, 0.f);
    xlo = __fmaf_rn(ky, -b[1], xlo);
    xhi = __fmaf_rn(ky, -b[1], xhi);
    if (fabsf(ky) > 1.0f || fabsf(kz) > 1.0f) return make_float4(0.f, 0.f, 0.f, (float)M_PAIR);
    const float kx = nint_scaled(xlo, F.invf[0]);
    if (!(nint_scaled(xhi, F.invf[0]) == kx) || fabsf(kx) > 1.0f) return make_float4(0.f, ky, kz, (float)M_AXIS);
    return make_float4(kx, ky, kz, (float)M_UNI);
  }
}

// Range [lo, hi] of a real value (outward-rounded float32 bounds) and its
// distance from zero, its largest magnitude, and its distance from the lattice
// L Z for a period known to lie in [L - dL, L + dL] (all rounded so as to stay
// bounds: distances down, magnitudes up).
__device__ __forceinline__ float iv_dist0(float lo, float hi) { return lo > 0.0f ? lo : (hi < 0.0f ? -hi : 0.0f); }
__device__ __forceinline__ float iv_absmax(float lo, float hi) { return fmaxf(fabsf(lo), fabsf(hi)); }
__device__ __forceinline__ float iv_dist_lattice(float lo, float hi, float L, float dL, float invL) {
  // the nearest multiples of the period lie among m - 1 .. m + 2, m = floor(hi / L)
  // taken with the rounded reciprocal invL (within one of the exact floor)
  const float m = floorf(hi * invL);
  float d = INFINITY;
#pragma unroll
  for (int q = -1; q <= 2; ++q) {
    const float k = m + (float)q, ak = fabsf(k);
    const float x_hi = __fadd_ru(__fmul_ru(k, L), __fmul_ru(ak, dL));  // k * (true period), bounds
    const float x_lo = __fsub_rd(__fmul_rd(k, L), __fmul_ru(ak, dL));
    d = fminf(d, fmaxf(0.0f, fmaxf(__fsub_rd(lo, x_hi), __fsub_rd(x_lo, hi))));
  }
  return d;
}

// Whether no pair of a warp tile (i run bounds imin..imax, j sub-chunk bounds
// jmin..jmax, tile image img from tile_image) can have its binary64 bin in
// [lo_bin, hi_bin): then the tile contributes nothing to this sweep and is
// skipped (the tile analogue of a cell list).  Bounds on the exact minimum-image
// distance r of every pair, in float32 with directed rounding: per axis, the
// displacement range [jmin - imax, jmax - imin] (widened by the binary64-input
// conversion error), minus the tile's uniform image where it has one (the box
// vectors within their float32 rounding error dBf of binary64), or, on an axis
// wrapped per pair, at least its distance from the lattice and at most half the
// period.  Pairs with r below r_max have the same nearest images in float32 and
// binary64 (the frame's precondition), and a translate shorter than
// r_max <= h_min/2 is the minimum image, so a tile whose image-based distances all
// lie outside the sweep's distances has no pair in the sweep.  The sweep's edges
// are widened by 2^-16 (relative) for the float32 roundings here and the
// binary64 roundings of r and of floor(nbins r / r_max).  Orthorhombic: every
// mode; triclinic: uniform tiles and tiles uniform on all axes but x, and
// per-pair tiles by their z and y components alone (below).
template <int V>
__device__ bool tile_outside_sweep(const FrameDev& F, const float* imin, const float* imax, const float* jmin,
                                   const float* jmax, float4 img, int lo_bin, int hi_bin) {
  const int mode = (int)img.w;
  if (V != V_NONE && F.all_defer) return false;  // (the no-box bound needs no images)
  float lo[3], hi[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float cv = 2.0f * F.convf[c];
    lo[c] = __fsub_rd(__fsub_rd(jmin[c], imax[c]), cv);
    hi[c] = __fadd_ru(__fsub_ru(jmax[c], imin[c]), cv);
  }
  float l[3], u[3];
  const float* b = F.Bf;
  const float* db = F.dBf;
  if (V == V_TRIC && mode == M_PAIR) {
    // Per-pair images: every image vector d - B k has z component d_z - kz cz and
    // y component d_y - ky by - kz cy, so |d - B k|^2 is at least, for its kz,
    // the z residual squared plus the distance of the y range shifted by kz cy
    // from the lattice by Z, squared.  When the z range is shorter than cz, only
    // the kz nearest to it can give less than cz^2 > r_max^2: the lower bound is
    // the minimum over those; only pairs beyond the sweep are skipped this way.
    if (!(__fsub_ru(hi[2], lo[2]) < b[8] - db[8])) return false;
    // (m is within one of the exact floor M; M - 1 .. M + 1 are the kz that matter)
    const float m = floorf(hi[2] * F.invf[2]);
    float best = INFINITY;
#pragma unroll
    for (int q = -2; q <= 2; ++q) {
      const float kz = m + (float)q, ak = fabsf(kz);
      const float sz_hi = __fadd_ru(__fmul_ru(kz, b[8]), __fmul_ru(ak, db[8]));
      const float sz_lo = __fsub_rd(__fmul_rd(kz, b[8]), __fmul_ru(ak, db[8]));
      const float sy_hi = __fadd_ru(__fmul_ru(kz, b[5]), __fmul_ru(ak, db[5]));
      const float sy_lo = __fsub_rd(__fmul_rd(kz, b[5]), __fmul_ru(ak, db[5]));
      const float dz = iv_dist0(__fsub_rd(lo[2], sz_hi), __fsub_ru(hi[2], sz_lo));
      const float dy = iv_dist_lattice(__fsub_rd(lo[1], sy_hi), __fsub_ru(hi[1], sy_lo), b[4], db[4], F.invf[1]);
      best = fminf(best, __fmaf_rd(dz, dz, __fmul_rd(dy, dy)));
    }
    const float r_hi = (hi_bin >= F.nbins) ? F.rmax_f : (float)hi_bin * F.dr_f;
    return best >= r_hi * r_hi * (1.0f + 0x1p-16f);
  }
  if (V == V_NONE) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      l[c] = iv_dist0(lo[c], hi[c]);
      u[c] = iv_absmax(lo[c], hi[c]);
    }
  } else if (V == V_ORTHO) {
    const float kk[3] = {img.x, img.y, img.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float L = b[4 * c], dL = db[4 * c];
      if (mode == M_PAIR || mode == M_AXIS + c) {  // wrapped per pair
        l[c] = iv_dist_lattice(lo[c], hi[c], L, dL, F.invf[c]);
        u[c] = __fmul_ru(__fadd_ru(L, dL), 0.5f);
      } else {  // |k| <= 1: the true shift lies in [k L32 - |k| dL, k L32 + |k| dL]
        const float s = kk[c] * L, e = fabsf(kk[c]) * dL;
        const float a = __fsub_rd(lo[c], __fadd_ru(s, e)), z = __fsub_ru(hi[c], __fsub_rd(s, e));
        l[c] = iv_dist0(a, z);
        u[c] = iv_absmax(a, z);
      }
    }
  } else {  // V_TRIC: the image vector B k (kx = 0 in the M_AXIS mode), each term |k| <= 1
    const float kx = img.x, ky = img.y, kz = img.z;
    const float ex = fabsf(kx) * db[0] + fabsf(ky) * db[1] + fabsf(kz) * db[2];
    const float ey = fabsf(ky) * db[4] + fabsf(kz) * db[5], ez = fabsf(kz) * db[8];
    const float sx_hi = __fadd_ru(__fadd_ru(__fadd_ru(kx * b[0], ky * b[1]), kz * b[2]), __fmul_ru(ex, 1.0f + 0x1p-20f));
    const float sx_lo = __fsub_rd(__fadd_rd(__fadd_rd(kx * b[0], ky * b[1]), kz * b[2]), __fmul_ru(ex, 1.0f + 0x1p-20f));
    const float sy_hi = __fadd_ru(__fadd_ru(ky * b[4], kz * b[5]), __fmul_ru(ey, 1.0f + 0x1p-20f));
    const float sy_lo = __fsub_rd(__fadd_rd(ky * b[4], kz * b[5]), __fmul_ru(ey, 1.0f + 0x1p-20f));
    const float sz_hi = __fadd_ru(kz * b[8], ez), sz_lo = __fsub_rd(kz * b[8], ez);
    const float ax = __fsub_rd(lo[0], sx_hi), bx = __fsub_ru(hi[0], sx_lo);
    const float ay = __fsub_rd(lo[1], sy_hi), by = __fsub_ru(hi[1], sy_lo);
    const float az = __fsub_rd(lo[2], sz_hi), bz = __fsub_ru(hi[2], sz_lo);
    if (mode == M_UNI) {
      l[0] = iv_dist0(ax, bx);
      u[0] = iv_absmax(ax, bx);
    } else {  // x wrapped per pair along a
      l[0] = iv_dist_lattice(ax, bx, b[0], db[0], F.invf[0]);
      u[0] = __fmul_ru(__fadd_ru(b[0], db[0]), 0.5f);
    }
    l[1] = iv_dist0(ay, by); u[1] = iv_absmax(ay, by);
    l[2] = iv_dist0(az, bz); u[2] = iv_absmax(az, bz);
  }
  const float lb2 = __fmaf_rd(l[2], l[2], __fmaf_rd(l[1], l[1], __fmul_rd(l[0], l[0])));
  const float ub2 = __fmaf_ru(u[2], u[2], __fmaf_ru(u[1], u[1], __fmul_ru(u[0], u[0])));
  // the sweep's edges in distance (squared), widened (bin width and r_max in
  // float32 from the frame descriptor: no binary64 arithmetic per tile)
  const float r_lo = (float)lo_bin * F.dr_f, r_hi = (hi_bin >= F.nbins) ? F.rmax_f : (float)hi_bin * F.dr_f;
  return (lo_bin > 0 && ub2 < r_lo * r_lo * (1.0f - 0x1p-16f)) || lb2 >= r_hi * r_hi * (1.0f + 0x1p-16f);
}

// Adds the `depth` private copies (stride words apart) bin by bin into the
// global uint64 histogram and clears them, with their guard words.
__device__ void flush_hist(uint32_t* sh, int width, int depth, int stride, uint64_t* dst, int tid) {
  const int nthreads = blockDim.x;
  for (int k = tid; k < width; k += nthreads) {
    uint32_t v = 0u;
    for (int c = 0; c < depth; ++c) {
      v += sh[c * stride + k];
      sh[c * stride + k] = 0u;
    }
    if (v) atomicAdd((unsigned long long*)(dst + k), (unsigned long long)v);
  }
  for (int k = tid; k < depth * 2 * kGuard; k += nthreads) {
    int c = k / (2 * kGuard), g = k - c * 2 * kGuard;
    sh[c * stride + (g < kGuard ? g - kGuard : width + g - kGuard)] = 0u;
  }
}

// Work item -> tile pair.  Items of a segment are numbered row by row over
// (ti, tj), i tiles of kTile particles and j tiles of kTile/jm; intra-species
// segments keep only j tiles that do not end before the i tile starts
// (tj >= jm ti), and mask pairs j <= i in those that overlap it (tj < jm (ti + 1)).
__device__ void decode_item(const PairLaunch& L, long long item, ItemDesc& it) {
  int lo = 0, hi = L.n_segs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (L.segs[mid].item0 <= item) lo = mid; else hi = mid - 1;
  }
  const Segment& s = L.segs[lo];
  const int jm = s.jm > 1 ? s.jm : 1;
  const int tile_j = kTile / jm;
  long long lid = item - s.item0 + s.item_base;
  int ti, tj;
  if (s.intra) {
    // row ti holds tj in [jm ti, n_tj) and starts at ti n_tj - jm ti (ti - 1) / 2
    long long n = s.n_tj;
    int a = 0, b = s.n_ti - 1;
    while (a < b) {
      int m = (a + b + 1) >> 1;
      long long start = (long long)m * n - (long long)jm * m * (m - 1) / 2;
      if (start <= lid) a = m; else b = m - 1;
    }
    ti = a;
    long long start = (long long)ti * n - (long long)jm * ti * (ti - 1) / 2;
    tj = jm * ti + (int)(lid - start);
  } else {
    ti = (int)(lid / s.n_tj);
    tj = (int)(lid - (long long)ti * s.n_tj);
  }
  it.valid = 1;
  it.fd = s.fd;
  it.h = s.h;
  it.pass = s.pass;
  it.i0 = s.a0 + ti * kTile;
  it.ni = min(kTile, s.na - ti * kTile);
  it.j0 = s.b0 + tj * tile_j;
  it.nj = min(tile_j, s.nb - tj * tile_j);
  it.masked = (s.intra && tj < jm * (ti + 1)) ? 1 : 0;
  int lo_bin = s.pass * s.fd->sweep_width;
  it.skip = (lo_bin >= s.fd->nbins) ? 1 : 0;
}

__device__ void load_fast_params(const FrameDev& F, int pass, FastParams& P) {
  int lo_bin = pass * F.sweep_width;
  int hi_bin = min(F.nbins, lo_bin + F.sweep_width);
  P.S2 = F.S2;
  P.kb1 = __float_as_int(kMagicRound) + lo_bin + 1;
  P.width = (uint32_t)(hi_bin - lo_bin);
  P.lo = lo_bin;
  P.hi = hi_bin;
#pragma unroll
  for (int c = 0; c < 9; ++c) P.b[c] = F.Bf[c];
#pragma unroll
  for (int c = 0; c < 3; ++c) P.inv[c] = F.invf[c];
  P.amb_thr = 0.5f - F.eps_s;
  set_bound(F, P, M_PAIR);
}

// One instance per minimum-image variant V (every segment of the launch has a
// frame of that variant) and per MULTI.
// Register budgets: 256-thread blocks keep three blocks per SM (80 registers)
// for the no-box and orthorhombic variants, two (128 registers: the triclinic
// loop spills at 80, which costs more than the third block gains); 512- and
// 1024-thread blocks, meant for wide histograms, one.
template <int V, int RI>
constexpr int min_blocks_per_sm() {
  return RI < 4 ? 1 : ((V == V_NONE || V == V_ORTHO) ? 3 : 2);
}

// AGG: the increments of a warp aggregated in software (count_or_defer_agg).
template <int V, bool MULTI, int RI, bool AGG = false>
__global__ void __launch_bounds__(kTile / RI, min_blocks_per_sm<V, RI>()) pair_kernel(PairLaunch L) {
  constexpr int BLOCK = kTile / RI;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // `depth` private histogram copies, each [kGuard guard words | bins | kGuard
  // guard words] (stride words), then the j tile and the per-warp queues
  const int depth = L.hist_depth > 1 ? L.hist_depth : 1;
  const int stride = ((L.hist_width + 3) & ~3) + 2 * kGuard;
  uint32_t* hist0 = reinterpret_cast<uint32_t*>(smem_raw) + kGuard;
  float4* sjA = reinterpret_cast<float4*>(reinterpret_cast<uint32_t*>(smem_raw) + depth * stride);
  float2* sjZ = reinterpret_cast<float2*>(sjA + kTile / 2);
  uint32_t* sq = reinterpret_cast<uint32_t*>(sjZ + kTile / 2);
  __shared__ ItemDesc s_it;
  constexpr bool kTileImage = (V == V_ORTHO || V == V_TRIC);
  // tile bounds: always with tile images; without a box for frames whose tiles
  // can miss a sweep (FrameDev::cull_ok), for culling only
  constexpr bool kTileBounds = kTileImage || V == V_NONE;
  // per j sub-chunk: j min xyz, j max xyz; per warp and sub-chunk: the tile image
  __shared__ float s_bnd[kTileBounds ? kTile / kSubJ : 1][6];
  __shared__ float4 s_img[kTileBounds ? BLOCK / 32 : 1][kTileBounds ? kTile / kSubJ : 1];
  __shared__ float s_beta[kTileImage ? BLOCK / 32 : 1][kTileImage ? kTile / kSubJ : 1];  // per-tile beta
  static_assert(!kTileBounds || BLOCK / 32 >= kTile / kSubJ, "one warp per j sub-chunk");
  // the item's tiles to run, per cost class, and the counters of run_item
  constexpr int kListCap = kTileBounds ? (BLOCK / 32) * kSubPerTile : 1;
  static_assert(kListCap <= 256, "tile indices fit a byte");
  __shared__ unsigned char s_list[kTileBounds ? kCostClasses : 1][kListCap];
  __shared__ int s_cnt[kCostClasses + 1];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t* q = sq + warp * kQueueCap;
  uint32_t* sh = hist0 + (warp % depth) * stride;  // this warp's copy
  for (int k = tid; k < depth * stride; k += BLOCK) reinterpret_cast<uint32_t*>(smem_raw)[k] = 0u;

  const FrameDev* cur_fd = nullptr;
  int cur_h = -1, cur_pass = -1;
  unsigned long long since = 0;  // pairs accumulated in sh since the last flush
  uint64_t* cur_dst = nullptr;
  int cur_width = 0;

  // Guided self-scheduling: thread 0 claims runs of consecutive items whose
  // length shrinks with the work left (at most 64, at least 1), so a block
  // mostly stays on one segment (few histogram flushes) and the tail stays fine.
  long long run_next = 0, run_end = 0;
  for (;;) {
    if (tid == 0) {
      if (run_next >= run_end) {
        long long cur = (long long)*(volatile unsigned long long*)&L.ctl->next_item;
        long long ch = (L.n_items - cur) / (4LL * gridDim.x);
        ch = ch < 1 ? 1 : (ch > 64 ? 64 : ch);
        run_next = (long long)atomicAdd(&L.ctl->next_item, (unsigned long long)ch);
        run_end = run_next + ch < (long long)L.n_items ? run_next + ch : (long long)L.n_items;
      }
      long long item = run_next++;
      if (item >= L.n_items) s_it.valid = 0;
      else decode_item(L, item, s_it);
      for (int k = 0; k <= kCostClasses; ++k) s_cnt[k] = 0;
    }
    __syncthreads();
    const ItemDesc it = s_it;
    if (!it.valid) break;
    if (!it.skip) {
      const FrameDev& F = *it.fd;
      const unsigned long long pairs = (unsigned long long)it.ni * (unsigned long long)it.nj;
      if (it.fd != cur_fd || it.h != cur_h || it.pass != cur_pass || since + pairs > 0xFFFFFFFFull) {
        if (cur_fd) {
          __syncthreads();
          flush_hist(hist0, cur_width, depth, stride, cur_dst, tid);
          __syncthreads();
        }
        int lo_bin = it.pass * F.sweep_width;
        cur_fd = it.fd;
        cur_h = it.h;
        cur_pass = it.pass;
        cur_width = min(F.nbins, lo_bin + F.sweep_width) - lo_bin;
        cur_dst = F.out + (size_t)it.h * F.nbins + lo_bin;
        since = 0;
      }
      since += pairs;
      // stage the j tile in pair layout, padded with NaN particles to a multiple of kJUMax
      const int nj4 = (it.nj + kJUMax - 1) & ~(kJUMax - 1);
      for (int k = tid; k < nj4; k += BLOCK) {
        float4 v = k < it.nj ? __ldg(F.X + it.j0 + k)
                             : make_float4(__int_as_float(0x7fffffff), __int_as_float(0x7fffffff),
                                           __int_as_float(0x7fffffff), 0.f);
        float* a = reinterpret_cast<float*>(sjA + (k >> 1));
        a[k & 1] = v.x;
        a[2 + (k & 1)] = v.y;
        reinterpret_cast<float*>(sjZ + (k >> 1))[k & 1] = v.z;
      }
      // tile images: the bounds of this warp's i run against those of each
      // j sub-chunk of kSubJ particles (warp c reduces sub-chunk c)
      float ib_[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
      const bool bounds = kTileImage || (V == V_NONE && F.cull_ok);  // the same for the whole block
      if (bounds) {
        const int ib = warp * (32 * RI) + lane;  // this warp's i run (the particles run_tile gives it)
        for (int r = 0; r < RI; ++r) {
          const int li = ib + 32 * r;
          if (li < it.ni) {
            float4 v = __ldg(F.X + it.i0 + li);
            ib_[0] = fminf(ib_[0], v.x); ib_[1] = fminf(ib_[1], v.y); ib_[2] = fminf(ib_[2], v.z);
            ib_[3] = fmaxf(ib_[3], v.x); ib_[4] = fmaxf(ib_[4], v.y); ib_[5] = fmaxf(ib_[5], v.z);
          }
        }
        for (int o = 16; o > 0; o >>= 1)
          for (int a = 0; a < 6; ++a) {
            float other = __shfl_xor_sync(kFull, ib_[a], o);
            ib_[a] = a < 3 ? fminf(ib_[a], other) : fmaxf(ib_[a], other);
          }
      }
      __syncthreads();
      if (bounds) {
        if (warp * kSubJ < it.nj) {
          float jm[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
          const int ke = min(it.nj, (warp + 1) * kSubJ);
          for (int k = warp * kSubJ + lane; k < ke; k += 32) {
            const float* a = reinterpret_cast<const float*>(sjA + (k >> 1));
            const float x = a[k & 1], y = a[2 + (k & 1)];
            const float z = reinterpret_cast<const float*>(sjZ + (k >> 1))[k & 1];
            jm[0] = fminf(jm[0], x); jm[1] = fminf(jm[1], y); jm[2] = fminf(jm[2], z);
            jm[3] = fmaxf(jm[3], x); jm[4] = fmaxf(jm[4], y); jm[5] = fmaxf(jm[5], z);
          }
          for (int o = 16; o > 0; o >>= 1)
            for (int a = 0; a < 6; ++a) {
              float other = __shfl_xor_sync(kFull, jm[a], o);
              jm[a] = a < 3 ? fminf(jm[a], other) : fmaxf(jm[a], other);
            }
          if (lane == 0)
            for (int a = 0; a < 6; ++a) s_bnd[warp][a] = jm[a];
        }
        __syncthreads();
        const int ni_w = min(32 * RI, it.ni - warp * 32 * RI);  // i particles of this warp
        const int lo_bin = it.pass * F.sweep_width, hi_bin = min(F.nbins, lo_bin + F.sweep_width);
        for (int c = 0; c * kSubJ < it.nj; ++c) {
          float4 img = make_float4(0.f, 0.f, 0.f, 0.f);
          float tb = 0.0f;
          if (kTileImage) {
            if (ni_w > 0) img = tile_image<V>(F, ib_, ib_ + 3, s_bnd[c], s_bnd[c] + 3);
            tb = tile_beta<V>(F, ib_, ib_ + 3, s_bnd[c], s_bnd[c] + 3, img);
          }
          const unsigned long long np =
              (unsigned long long)max(ni_w, 0) * (unsigned long long)(min(it.nj, (c + 1) * kSubJ) - c * kSubJ);
          const bool skip = ni_w > 0 && tile_outside_sweep<V>(F, ib_, ib_ + 3, s_bnd[c], s_bnd[c] + 3, img, lo_bin,
                                                             hi_bin);
          if (lane == 0) {
            if (skip) {
              img.w = (float)M_SKIP;
              atomicAdd(&it.fd->culled_pairs, np);
            } else if (img.w == (float)M_UNI) {
              atomicAdd(&it.fd->uniform_pairs, np);
            } else if (img.w >= (float)M_AXIS) {
              atomicAdd(&it.fd->axis_pairs, np);
            }
            s_img[warp][c] = img;
            if (kTileImage) s_beta[warp][c] = tb;
            if (!skip && ni_w > 0) {
              const int cls = cost_class(it.masked ? M_PAIR : (int)img.w);
              s_list[cls][atomicAdd(&s_cnt[cls], 1)] = (unsigned char)(warp * kSubPerTile + c);
            }
          }
        }
        __syncthreads();  // every tile listed
      }
      unsigned ndef = 0;
      run_item<V, MULTI, RI, AGG>(it.fd, it, sjA, sjZ, sh, q, warp, lane, ndef, &s_img[0][0], &s_beta[0][0],
                                  TileLists{&s_list[0][0], s_cnt, kListCap}, bounds);
      if (lane == 0 && ndef) atomicAdd(&it.fd->deferred, (unsigned long long)ndef);
    }
    __syncthreads();
  }
  if (cur_fd) {
    __syncthreads();
    flush_hist(hist0, cur_width, depth, stride, cur_dst, tid);
  }
}

// ------------------------------------------------------------------ self checks

// Largest relative error of sqrt.approx.ftz.f32 over every float in [1, 4)
// (two binades: the relative error pattern repeats with the exponent's parity),
// against the correctly rounded binary64 square root.
__global__ void check_sqrt_kernel(unsigned long long* max_err_bits) {
  const uint32_t base = 0x3F800000u;  // 1.0f
  const uint32_t count = 2u << 23;    // [1, 4)
  double worst = 0.0;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    float x = __uint_as_float(base + k);
    double ref = __dsqrt_rn((double)x);
    double e = fabs((double)sqrt_approx(x) - ref) / ref;
    worst = fmax(worst, e);
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(kFull, worst, o));
  if ((threadIdx.x & 31) == 0) atomicMax(max_err_bits, (unsigned long long)__double_as_longlong(worst));
}

// splitmix64: a counter-based generator for the sampled pairs
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// For sampled pairs of one frame, the decision rule against the binary64
// definition: out[0] = max |sqrt(q32) - t64| / (alpha t64 + beta) over pairs
// inside the histogram (bits of a double; the analysis says < 1); out[1] =
// pairs whose float32 or double-float decision differs from the binary64 bin
// (must be 0); out[2] = pairs compared.
template <int V>
__device__ void check_window_pair(const FrameDev& F, const FastParams& P, int i, int j, double* worst,
                                  unsigned long long* viol, unsigned long long* checked) {
  float4 pi = F.X[i], pj = F.X[j];
  bool nearedge, nb_unused;
  uint32_t rel, rb_unused;
  const float2 dx = bc2(__fsub_rn(pj.x, pi.x)), dy = bc2(__fsub_rn(pj.y, pi.y)), dz = bc2(__fsub_rn(pj.z, pi.z));
  fast_decide2<V>(dx, dy, dz, P, nearedge, nb_unused, rel, rb_unused);
  bool amb0 = false, amb1 = false;
  float q = __fmul_rn(wrap_r2_2<V>(dx, dy, dz, P, amb0, amb1).x, P.S2);
  double r2 = exact_r2<V>(F, coords64(F, i), coords64(F, j));
  int k64 = bin_from_thresholds(F.T, F.S, F.nbins, r2);
  double t64 = __dmul_rn(__dsqrt_rn(r2), (double)F.nbins / F.r_max);
  if (t64 < (double)F.nbins + 1.0 && isfinite(q)) {
    double tq = __dsqrt_rn((double)q);
    *worst = fmax(*worst, fabs(tq - t64) / ((double)F.alpha_t * t64 + (double)F.beta_t));
    ++*checked;
  }
  if (!nearedge) {
    int k32 = (int)rel;  // lo = 0 here
    if (rel > (uint32_t)F.nbins) k32 = F.nbins;
    if (k32 != k64) ++*viol;
  } else {
    int km = mid_bin<V>(F, i, j, pi, pj);
    if (km >= 0 && km != k64) ++*viol;
  }
}

__global__ void check_window_kernel(const FrameDev* Fp, uint64_t n_samples, uint64_t seed,
                                    unsigned long long* out) {
  const FrameDev& F = *Fp;
  FastParams P;
  load_fast_params(F, 0, P);
  P.width = (uint32_t)F.nbins;  // decide over the whole histogram
  P.hi = F.nbins;
  double worst = 0.0;
  unsigned long long viol = 0, checked = 0;
  if (F.n >= 2) {
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n_samples;
         s += (uint64_t)gridDim.x * blockDim.x) {
      uint64_t h = mix64(seed ^ mix64(s));
      int i = (int)(h % (uint64_t)F.n);
      int j = (int)((h >> 32) % (uint64_t)F.n);
      if (i == j) continue;
      switch (F.variant) {
        case V_NONE: check_window_pair<V_NONE>(F, P, i, j, &worst, &viol, &checked); break;
        case V_ORTHO: check_window_pair<V_ORTHO>(F, P, i, j, &worst, &viol, &checked); break;
        case V_TRIC: check_window_pair<V_TRIC>(F, P, i, j, &worst, &viol, &checked); break;
        default: check_window_pair<V_TRIC_SEARCH>(F, P, i, j, &worst, &viol, &checked); break;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    worst = fmax(worst, __shfl_xor_sync(kFull, worst, o));
    viol += __shfl_xor_sync(kFull, viol, o);
    checked += __shfl_xor_sync(kFull, checked, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(worst));
    atomicAdd(out + 1, viol);
    atomicAdd(out + 2, checked);
  }
}

cudaError_t launch_check_sqrt(unsigned long long* out, cudaStream_t stream) {
  clear_stale_error();
  check_sqrt_kernel<<<1024, 256, 0, stream>>>(out);
  return cudaGetLastError();
}

cudaError_t launch_check_window(const FrameDev* F, uint64_t n_samples, uint64_t seed, unsigned long long* out,
                                cudaStream_t stream) {
  clear_stale_error();
  check_window_kernel<<<1024, 256, 0, stream>>>(F, n_samples, seed, out);
  return cudaGetLastError();
}

// The tile modes against their own bounds: one pair of a tile evaluated with the
// arithmetic of run_tile in mode MODE (coordinates shifted by the tile's images,
// then decide_arith2 with the tile's bound), against the binary64 bin.
template <int V, int MODE>
__device__ void check_tile_pair(const FrameDev& F, const FastParams& P, float beta, float3 kt, int i, int j,
                                double* worst, unsigned long long* viol, unsigned long long* checked) {
  const float4 pi = F.X[i], pj = F.X[j];
  float3 ti = make_float3(0.f, 0.f, 0.f), sj = make_float3(0.f, 0.f, 0.f);
  if (V == V_ORTHO && MODE >= M_UNI) {
    ti = make_float3(kt.x < 0.f ? P.b[0] : 0.f, kt.y < 0.f ? P.b[4] : 0.f, kt.z < 0.f ? P.b[8] : 0.f);
    sj = make_float3(kt.x > 0.f ? P.b[0] : 0.f, kt.y > 0.f ? P.b[4] : 0.f, kt.z > 0.f ? P.b[8] : 0.f);
  } else if (V == V_TRIC && MODE >= M_UNI) {
    const float* v = F.tshift[9 * (int)(kt.x + 1.0f) + 3 * (int)(kt.y + 1.0f) + (int)(kt.z + 1.0f)];
    ti = make_float3(v[0], v[1], v[2]);
  }
  const float2 dx = bc2(__fsub_rn(__fsub_rn(pj.x, sj.x), __fsub_rn(pi.x, ti.x)));
  const float2 dy = bc2(__fsub_rn(__fsub_rn(pj.y, sj.y), __fsub_rn(pi.y, ti.y)));
  const float2 dz = bc2(__fsub_rn(__fsub_rn(pj.z, sj.z), __fsub_rn(pi.z, ti.z)));
  float2 sm, e, bound;
  decide_arith2<V, false, MODE>(dx, dy, dz, P, (float)(P.hi + 1), 0.0f, sm, e, bound);
  bool amb0 = false, amb1 = false;
  const float q = __fmul_rn(wrap_r2_2<V, MODE>(dx, dy, dz, P, amb0, amb1).x, P.S2);
  const double r2 = exact_r2<V>(F, coords64(F, i), coords64(F, j));
  const int k64 = bin_from_thresholds(F.T, F.S, F.nbins, r2);
  const double t64 = __dmul_rn(__dsqrt_rn(r2), (double)F.nbins / F.r_max);
  if (t64 < (double)F.nbins + 1.0 && isfinite(q)) {
    *worst = fmax(*worst, fabs(__dsqrt_rn((double)q) - t64) / ((double)F.alpha_t * t64 + (double)beta));
    ++*checked;
  }
  if (!(fabsf(e.x) <= bound.x)) {
    const uint32_t rel = __float_as_uint(sm.x) + (__float_as_uint(e.x) >> 31) - (uint32_t)P.kb1;
    const int k32 = rel > (uint32_t)F.nbins ? F.nbins : (int)rel;
    if (k32 != k64) ++*viol;
  }
}

// One block per sampled tile: a run of 128 consecutive particles (the i's of one
// warp of a 256-thread block) and a j sub-chunk of kSubJ, at random aligned
// starts.  out[0] = largest |t32 - t64| / (alpha t64 + beta_tile) (must be < 1),
// out[1] = pairs decided in float32 with a bin other than the binary64 one (must
// be 0), out[2] = pairs compared, out[3] = sampled tiles in a shifted mode.
template <int V>
__global__ void check_tiles_kernel(const FrameDev* Fp, uint64_t n_tiles, uint64_t seed, unsigned long long* out) {
  const FrameDev& F = *Fp;
  FastParams P;
  load_fast_params(F, 0, P);
  P.width = (uint32_t)F.nbins;
  P.hi = F.nbins;
  __shared__ float s_b[8][6];
  __shared__ float s_bnd[12];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double worst = 0.0;
  unsigned long long viol = 0, checked = 0, shifted = 0;
  const int ni = min(128, F.n), nj = min(kSubJ, F.n);
  for (uint64_t s = blockIdx.x; s < n_tiles; s += gridDim.x) {
    const uint64_t h = mix64(seed ^ mix64(s));
    const int i0 = (int)((h % (uint64_t)((F.n - ni) / 128 + 1)) * 128);
    const int j0 = (int)(((h >> 32) % (uint64_t)((F.n - nj) / kSubJ + 1)) * kSubJ);
    for (int part = 0; part < 2; ++part) {  // bounds of the i run, then of the j chunk
      const int b0 = part ? j0 : i0, nb = part ? nj : ni;
      float m[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
      for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const float4 v = F.X[b0 + k];
        m[0] = fminf(m[0], v.x); m[1] = fminf(m[1], v.y); m[2] = fminf(m[2], v.z);
        m[3] = fmaxf(m[3], v.x); m[4] = fmaxf(m[4], v.y); m[5] = fmaxf(m[5], v.z);
      }
      for (int o = 16; o > 0; o >>= 1)
        for (int a = 0; a < 6; ++a) {
          const float other = __shfl_xor_sync(kFull, m[a], o);
          m[a] = a < 3 ? fminf(m[a], other) : fmaxf(m[a], other);
        }
      if (lane == 0)
        for (int a = 0; a < 6; ++a) s_b[warp][a] = m[a];
      __syncthreads();
      if (threadIdx.x < 6) {
        float v = s_b[0][threadIdx.x];
        for (int w = 1; w < 8; ++w)
          v = threadIdx.x < 3 ? fminf(v, s_b[w][threadIdx.x]) : fmaxf(v, s_b[w][threadIdx.x]);
        s_bnd[6 * part + threadIdx.x] = v;
      }
      __syncthreads();
    }
    const float4 img = tile_image<V>(F, s_bnd, s_bnd + 3, s_bnd + 6, s_bnd + 9);
    const float beta = tile_beta<V>(F, s_bnd, s_bnd + 3, s_bnd + 6, s_bnd + 9, img);
    FastParams Q = P;
    set_bound_beta(F, Q, beta);
    const float3 kt = make_float3(img.x, img.y, img.z);
    if (threadIdx.x == 0 && img.w >= (float)M_UNI) ++shifted;
    for (int k = threadIdx.x; k < ni * nj; k += blockDim.x) {
      const int i = i0 + k % ni, j = j0 + k / ni;
      if (i == j) continue;
      switch ((int)img.w) {
        case M_UNI: check_tile_pair<V, M_UNI>(F, Q, beta, kt, i, j, &worst, &viol, &checked); break;
        case M_AXIS + 0: check_tile_pair<V, M_AXIS + 0>(F, Q, beta, kt, i, j, &worst, &viol, &checked); break;
        case M_AXIS + 1:
          if (V == V_ORTHO) check_tile_pair<V, M_AXIS + 1>(F, Q, beta, kt, i, j, &worst, &viol, &checked);
          break;
        case M_AXIS + 2:
          if (V == V_ORTHO) check_tile_pair<V, M_AXIS + 2>(F, Q, beta, kt, i, j, &worst, &viol, &checked);
          break;
        default: check_tile_pair<V, M_PAIR>(F, Q, beta, kt, i, j, &worst, &viol, &checked); break;
      }
    }
    __syncthreads();  // s_b, s_bnd are rewritten by the next tile
  }
  for (int o = 16; o > 0; o >>= 1) {
    worst = fmax(worst, __shfl_xor_sync(kFull, worst, o));
    viol += __shfl_xor_sync(kFull, viol, o);
    checked += __shfl_xor_sync(kFull, checked, o);
    shifted += __shfl_xor_sync(kFull, shifted, o);
  }
  if (lane == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(worst));
    atomicAdd(out + 1, viol);
    atomicAdd(out + 2, checked);
    atomicAdd(out + 3, shifted);
  }
}

cudaError_t launch_check_tiles(const FrameDev* F, int variant, uint64_t n_tiles, uint64_t seed,
                               unsigned long long* out, cudaStream_t stream) {
  clear_stale_error();
  if (variant == V_ORTHO) check_tiles_kernel<V_ORTHO><<<456, 256, 0, stream>>>(F, n_tiles, seed, out);
  else if (variant == V_TRIC) check_tiles_kernel<V_TRIC><<<456, 256, 0, stream>>>(F, n_tiles, seed, out);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}


// ------------------------------------------------------------------ g(r), Eq. 1

// g = (counts / n_frames) / (pair density x shell volume) per bin, binary64.
// The shell of bin k, (4 pi / 3)(r_{k+1}^3 - r_k^3) with r_k = k dr, is
// evaluated as (4 pi / 3) dr^3 (3k(k+1) + 1): the integer factor is exact for
// k < 2^25, so no cancellation between the two cubes.
__global__ void rdf_kernel(const uint64_t* __restrict__ counts, int32_t n_hist, int32_t nbins, double r_max,
                           const double* __restrict__ dens, uint64_t n_frames, double* __restrict__ g) {
  const int64_t total = (int64_t)n_hist * nbins;
  const double dr = __ddiv_rn(r_max, (double)nbins);
  const double c = __dmul_rn(__dmul_rn(4.0 * 3.14159265358979323846 / 3.0, dr), __dmul_rn(dr, dr));
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int32_t h = (int32_t)(idx / nbins);
    const double k = (double)(idx - (int64_t)h * nbins);
    const double poly = __fma_rn(__dmul_rn(3.0, k), __dadd_rn(k, 1.0), 1.0);
    const double per_frame = __ddiv_rn((double)counts[idx], (double)n_frames);
    g[idx] = __ddiv_rn(per_frame, __dmul_rn(dens[h], __dmul_rn(c, poly)));
  }
}

cudaError_t launch_rdf(const uint64_t* counts, int32_t n_hist, int32_t nbins, double r_max,
                       const double* pair_density, uint64_t n_frames, double* g, cudaStream_t stream) {
  clear_stale_error();
  int64_t total = (int64_t)n_hist * nbins;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  rdf_kernel<<<blocks, 256, 0, stream>>>(counts, n_hist, nbins, r_max, pair_density, n_frames, g);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers


size_t pair_kernel_smem(int hist_width, int depth, int block) {
  size_t stride = (size_t)((hist_width + 3) & ~3) + 2 * kGuard;
  size_t warps = (size_t)(block == kBlockHuge ? kBlockHuge : block == kBlockLarge ? kBlockLarge : kBlockSmall) / 32;
  return (size_t)(depth > 1 ? depth : 1) * stride * 4 + (size_t)kTile * 12 + warps * kQueueCap * 4;
}

int pair_kernel_max_width() {
  int dev = 0;
  cudaGetDevice(&dev);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  size_t fixed = pair_kernel_smem(0) + sizeof(ItemDesc) + 64;
  if ((size_t)optin <= fixed) return 0;
  return (int)(((size_t)optin - fixed) / 4) & ~3;
}

// Blocks of both instances that fit on one SM with `smem` bytes of dynamic
// shared memory; 0 (and no error left behind) when the request cannot be met.
template <int V, int RI>
int blocks_per_sm_vr(size_t smem) {
  int nb0 = 0, nb1 = 0;
  if (cudaFuncSetAttribute(pair_kernel<V, false, RI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb0, pair_kernel<V, false, RI>, kTile / RI, smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(pair_kernel<V, true, RI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb1, pair_kernel<V, true, RI>, kTile / RI, smem) !=
          cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return nb0 < nb1 ? nb0 : nb1;
}

template <int V>
int blocks_per_sm_v(int hist_width, int depth, int block) {
  size_t smem = pair_kernel_smem(hist_width, depth, block);
  if (block == kBlockSmall) {  // the aggregated-increment instance must fit as well
    int na = 0;
    if (cudaFuncSetAttribute(pair_kernel<V, false, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&na, pair_kernel<V, false, 4, true>, kBlockSmall, smem) !=
            cudaSuccess) {
      (void)cudaGetLastError();
      return 0;
    }
    const int nb = blocks_per_sm_vr<V, 4>(smem);
    return na < nb ? na : nb;
  }
  return block == kBlockHuge ? blocks_per_sm_vr<V, 1>(smem)
         : block == kBlockLarge ? blocks_per_sm_vr<V, 2>(smem) : blocks_per_sm_vr<V, 4>(smem);
}

int pair_kernel_blocks_per_sm(int variant, int hist_width, int depth, int block) {
  switch (variant) {
    case V_NONE: return blocks_per_sm_v<V_NONE>(hist_width, depth, block);
    case V_ORTHO: return blocks_per_sm_v<V_ORTHO>(hist_width, depth, block);
    case V_TRIC: return blocks_per_sm_v<V_TRIC>(hist_width, depth, block);
    default: return blocks_per_sm_v<V_TRIC_SEARCH>(hist_width, depth, block);
  }
}

cudaError_t launch_stage(const StageJob* jobs, int n_jobs, int64_t n_chunks, cudaStream_t stream) {
  clear_stale_error();
  if (n_jobs <= 0 || n_chunks <= 0) return cudaSuccess;
  stage_kernel<<<(unsigned)n_chunks, 256, 0, stream>>>(jobs, n_jobs);
  return cudaGetLastError();
}

cudaError_t launch_spatial_sort(const SortSeg* segs, int n_segs, int max_chunks, float4* X, float4* Xs,
                                double4* X64, double4* Xs64, int32_t* keys, uint32_t* counts,
                                cudaStream_t stream) {
  clear_stale_error();
  if (n_segs <= 0 || max_chunks <= 0) return cudaSuccess;
  dim3 grid((unsigned)max_chunks, (unsigned)n_segs);
  sort_count_kernel<<<grid, 256, 0, stream>>>(segs, X, keys, counts);
  sort_scan_kernel<<<n_segs, 1024, 0, stream>>>(segs, counts);
  sort_scatter_kernel<<<grid, 256, 0, stream>>>(segs, X, X64, keys, counts, Xs, Xs64);
  sort_copy_kernel<<<grid, 256, 0, stream>>>(segs, Xs, X, Xs64, X64);
  return cudaGetLastError();
}

cudaError_t launch_frame_setup(FrameDev* frames, int n_frames, int, cudaStream_t stream) {
  clear_stale_error();
  if (n_frames <= 0) return cudaSuccess;
  frame_setup_kernel<<<(n_frames + 63) / 64, 64, 0, stream>>>(frames, n_frames);
  return cudaGetLastError();
}

cudaError_t launch_thresholds(double r_max, int32_t nbins, double* T, int32_t* status,
                              cudaStream_t stream) {
  clear_stale_error();
  int threads = 128;
  int blocks = (nbins + 1 + threads - 1) / threads;
  thresholds_kernel<<<blocks, threads, 0, stream>>>(r_max, nbins, T, status);
  return cudaGetLastError();
}

template <int V, bool MULTI, int RI, bool AGG = false>
cudaError_t launch_pairs_vmr(const PairLaunch& p, int grid, size_t smem, cudaStream_t stream) {
  clear_stale_error();
  cudaError_t e =
      cudaFuncSetAttribute(pair_kernel<V, MULTI, RI, AGG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  pair_kernel<V, MULTI, RI, AGG><<<grid, kTile / RI, smem, stream>>>(p);
  return cudaGetLastError();
}

template <int V, bool MULTI>
cudaError_t launch_pairs_vm(const PairLaunch& p, int grid, size_t smem, cudaStream_t stream) {
  if constexpr (!MULTI)  // aggregated increments: 256-thread blocks, one sweep
    if (p.agg && (p.block == kBlockSmall || p.block == 0)) return launch_pairs_vmr<V, false, 4, true>(p, grid, smem, stream);
  return p.block == kBlockHuge    ? launch_pairs_vmr<V, MULTI, 1>(p, grid, smem, stream)
         : p.block == kBlockLarge ? launch_pairs_vmr<V, MULTI, 2>(p, grid, smem, stream)
                                  : launch_pairs_vmr<V, MULTI, 4>(p, grid, smem, stream);
}

template <int V>
cudaError_t launch_pairs_v(const PairLaunch& p, int grid, size_t smem, cudaStream_t stream) {
  return p.multi ? launch_pairs_vm<V, true>(p, grid, smem, stream) : launch_pairs_vm<V, false>(p, grid, smem, stream);
}

cudaError_t launch_pairs(const PairLaunch& p, int variant, int grid, size_t smem, cudaStream_t stream) {
  switch (variant) {
    case V_NONE: return launch_pairs_v<V_NONE>(p, grid, smem, stream);
    case V_ORTHO: return launch_pairs_v<V_ORTHO>(p, grid, smem, stream);
    case V_TRIC: return launch_pairs_v<V_TRIC>(p, grid, smem, stream);
    default: return launch_pairs_v<V_TRIC_SEARCH>(p, grid, smem, stream);
  }
}

}  // namespace dh
