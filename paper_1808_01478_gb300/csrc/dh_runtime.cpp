// Host runtime of libdh: argument checks, work planning, device workspace,
// threshold-table cache and the launch sequence behind the C ABI of dh.h.
//
// Transfer scheme (Reuter & Koefinger, Sec. 3.2): the coordinates of all
// species of a frame are one contiguous array copied to the device in one
// operation, all histograms of the frame come back in one copy, and device
// memory is allocated on first use and reused by later calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "dh_runtime.h"

namespace dh {

namespace {
thread_local std::string g_last_error;
bool is_finite(double v) { return std::isfinite(v); }

// Smallest distance between opposite faces of the cell spanned by the columns of B.
double min_plane_spacing(const double* B) {
  double a[3] = {B[0], B[3], B[6]}, b[3] = {B[1], B[4], B[7]}, c[3] = {B[2], B[5], B[8]};
  auto cross = [](const double* u, const double* v, double* w) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
  };
  auto norm = [](const double* w) { return std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]); };
  double bc[3], ca[3], ab[3];
  cross(b, c, bc);
  cross(c, a, ca);
  cross(a, b, ab);
  double vol = std::fabs(a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2]);
  return std::min(vol / norm(bc), std::min(vol / norm(ca), vol / norm(ab)));
}

}  // namespace

dh_status fail(dh_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

const char* last_error_message() { return g_last_error.c_str(); }

cudaError_t DevBuf::ensure(size_t bytes) {
  if (bytes <= cap) return cudaSuccess;
  size_t want = std::max(bytes, cap + cap / 2);
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  cap = want;
  return cudaSuccess;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
}

cudaError_t HostBuf::ensure(size_t bytes) {
  if (bytes <= cap) return cudaSuccess;
  size_t want = std::max(bytes, cap + cap / 2);
  if (p) cudaFreeHost(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = cudaMallocHost(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  cap = want;
  return cudaSuccess;
}

void HostBuf::release() {
  if (p) cudaFreeHost(p);
  p = nullptr;
  cap = 0;
}

dh_status ThresholdCache::acquire(double r_max, int32_t nbins, cudaStream_t st, int32_t* status_dev,
                                  double** T, int* launched) {
  std::lock_guard<std::mutex> g(mu_);
  Key key;
  std::memcpy(&key.rbits, &r_max, 8);
  key.nbins = nbins;
  auto it = map_.find(key);
  if (it != map_.end()) {
    it->second.refs++;
    it->second.last = ++tick_;
    if (it->second.built_on != st) DH_CUDA_TRY(cudaStreamWaitEvent(st, it->second.ready, 0));
    *T = it->second.T;
    return DH_OK;
  }
  // evict least recently used tables nobody holds (stream-ordered free)
  while (map_.size() >= cap_) {
    auto victim = map_.end();
    for (auto e = map_.begin(); e != map_.end(); ++e)
      if (e->second.refs == 0 && (victim == map_.end() || e->second.last < victim->second.last)) victim = e;
    if (victim == map_.end()) break;
    cudaStreamWaitEvent(st, victim->second.ready, 0);
    cudaFreeAsync(victim->second.T, st);
    cudaEventDestroy(victim->second.ready);
    rev_.erase(victim->second.T);
    map_.erase(victim);
  }
  double* t = nullptr;
  cudaEvent_t ev = nullptr;
  // binary64 thresholds followed by their float-pair copy
  DH_CUDA_TRY(cudaMallocAsync((void**)&t, 2 * sizeof(double) * (size_t)(nbins + 1), st));
  DH_CUDA_TRY(launch_thresholds(r_max, nbins, t, status_dev, st));
  DH_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  DH_CUDA_TRY(cudaEventRecord(ev, st));
  if (launched) ++*launched;
  map_[key] = Entry{t, 1, ++tick_, st, ev};
  rev_[t] = key;
  *T = t;
  return DH_OK;
}

void ThresholdCache::release(const double* T) {
  std::lock_guard<std::mutex> g(mu_);
  auto r = rev_.find(T);
  if (r == rev_.end()) return;
  auto it = map_.find(r->second);
  if (it != map_.end() && it->second.refs > 0) it->second.refs--;
}

void ThresholdCache::clear(cudaStream_t st) {
  std::lock_guard<std::mutex> g(mu_);
  for (auto& kv : map_) {
    cudaStreamWaitEvent(st, kv.second.ready, 0);
    cudaFreeAsync(kv.second.T, st);
    cudaEventDestroy(kv.second.ready);
  }
  map_.clear();
  rev_.clear();
}

int pair_grid(int num_sms, int bps, int64_t n_items) {
  int64_t g = (int64_t)std::max(bps, 1) * num_sms;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, n_items));
}

dh_status check_frame(const dh_frame* f, PlannedFrame& pf, int max_width) {
  if (!f) return fail(DH_ERR_INVALID, "frame is NULL");
  if (f->n < 0 || f->n > (int64_t)0x7FFFFFFF - 2 * kTile)
    return fail(DH_ERR_INVALID, "n = %lld out of range", (long long)f->n);
  if (f->n_species < 1) return fail(DH_ERR_INVALID, "n_species must be >= 1");
  if (!f->species_offsets) return fail(DH_ERR_INVALID, "species_offsets is NULL");
  const int64_t* o = f->species_offsets;
  if (o[0] != 0 || o[f->n_species] != f->n)
    return fail(DH_ERR_INVALID, "species offsets must start at 0 and end at n");
  for (int s = 0; s < f->n_species; ++s)
    if (o[s + 1] < o[s]) return fail(DH_ERR_INVALID, "species offsets must be nondecreasing");
  if (f->nbins < 1 || f->nbins > DH_MAX_BINS)
    return fail(DH_ERR_INVALID, "nbins = %d out of range [1, %d]", f->nbins, DH_MAX_BINS);
  if (!(f->r_max > 0.0) || !is_finite(f->r_max)) return fail(DH_ERR_INVALID, "r_max must be > 0 and finite");
  if (f->n > 0 && !f->coords) return fail(DH_ERR_INVALID, "coords is NULL");
  if (!f->out) return fail(DH_ERR_INVALID, "out is NULL");
  const double* B = f->box;
  pf.margin = 1.0;
  switch (f->box_type) {
    case DH_BOX_NONE:
      pf.variant = V_NONE;
      break;
    case DH_BOX_ORTHO:
      for (int q = 0; q < 9; ++q) {
        bool diag = (q == 0 || q == 4 || q == 8);
        if (!is_finite(B[q])) return fail(DH_ERR_INVALID, "box entry %d is not finite", q);
        if (diag && !(B[q] > 0.0)) return fail(DH_ERR_INVALID, "orthorhombic box lengths must be > 0");
        if (!diag && B[q] != 0.0) return fail(DH_ERR_INVALID, "orthorhombic box must be diagonal");
      }
      pf.variant = V_ORTHO;
      break;
    case DH_BOX_TRICLINIC: {
      for (int q = 0; q < 9; ++q)
        if (!is_finite(B[q])) return fail(DH_ERR_INVALID, "box entry %d is not finite", q);
      if (B[3] != 0.0 || B[6] != 0.0 || B[7] != 0.0)
        return fail(DH_ERR_INVALID, "triclinic box must be upper triangular (a along x, b in the xy plane)");
      if (!(B[0] > 0.0 && B[4] > 0.0 && B[8] > 0.0))
        return fail(DH_ERR_INVALID, "triclinic box diagonal must be > 0");
      if (std::fabs(B[1]) > 0.5 * B[0] || std::fabs(B[2]) > 0.5 * B[0] || std::fabs(B[5]) > 0.5 * B[4])
        return fail(DH_ERR_INVALID, "triclinic box must be reduced: |bx|,|cx| <= ax/2, |cy| <= by/2");
      double hmin = min_plane_spacing(B);
      double margin = 1.0 - 2.0 * f->r_max / hmin;
      pf.margin = margin;
      pf.variant = (margin >= 1.0 / 256.0) ? V_TRIC : V_TRIC_SEARCH;
      break;
    }
    default:
      return fail(DH_ERR_INVALID, "unknown box_type %d", f->box_type);
  }
  int64_t S = f->n_species;
  pf.src = f;
  pf.n_hist = (int32_t)(S * (S + 1) / 2);
  pf.sweeps = (f->nbins + max_width - 1) / max_width;
  pf.sweep_width = (f->nbins + pf.sweeps - 1) / pf.sweeps;
  uint64_t pairs = 0;
  for (int a = 0; a < S; ++a) {
    uint64_t na = (uint64_t)(o[a + 1] - o[a]);
    pairs += na * (na ? na - 1 : 0) / 2;
    for (int b = a + 1; b < S; ++b) pairs += na * (uint64_t)(o[b + 1] - o[b]);
  }
  pf.pairs = pairs;
  return DH_OK;
}

void fill_frame_dev(const PlannedFrame& pf, FrameDev& F, const float4* X, uint64_t* out, const double* T) {
  const dh_frame* f = pf.src;
  std::memset(&F, 0, sizeof F);
  F.X = X;
  F.out = out;
  F.T = T;
  F.Tf = reinterpret_cast<const float2*>(T + f->nbins + 1);
  F.variant = pf.variant;
  F.nbins = f->nbins;
  F.n = (int32_t)f->n;
  F.sweep_width = pf.sweep_width;
  F.r_max = f->r_max;
  for (int q = 0; q < 9; ++q) {
    F.B[q] = (f->box_type == DH_BOX_NONE) ? 0.0 : f->box[q];
    F.Bf[q] = (float)F.B[q];
    F.Bl[q] = (float)(F.B[q] - (double)F.Bf[q]);
  }
  if (pf.variant == V_ORTHO) {
    F.Linv[0] = 1.0 / F.B[0];
    F.Linv[1] = 1.0 / F.B[4];
    F.Linv[2] = 1.0 / F.B[8];
    F.invf[0] = (float)F.Linv[0];
    F.invf[1] = (float)F.Linv[1];
    F.invf[2] = (float)F.Linv[2];
  } else if (pf.variant == V_TRIC || pf.variant == V_TRIC_SEARCH) {
    F.invf[0] = (float)(1.0 / F.B[0]);
    F.invf[1] = (float)(1.0 / F.B[4]);
    F.invf[2] = (float)(1.0 / F.B[8]);
  }
  double S = (double)f->nbins / f->r_max;
  F.S = (float)S;
  F.dr_f = (float)(f->r_max / (double)f->nbins);
  F.rmax_f = (float)f->r_max;
  F.eps_S = std::fabs((double)F.S - S) / S;
  F.S2 = (float)(S * S);
  F.eps_S2 = std::fabs((double)F.S2 - S * S) / (S * S) + 1e-15;
  F.margin = (float)pf.margin;
  for (int c = 0; c < 3; ++c) {
    F.cmin[c] = 0x7FFFFFFF;                // ordered encoding of +huge: min starts high
    F.cmax[c] = (int32_t)0x80000000;       // and max starts low
  }
}

int sort_grid_bits(int64_t n) {
  int g = (int)std::floor(std::log2(std::cbrt((double)n / 16.0)));
  return std::min(6, std::max(1, g));
}

std::vector<SortSeg> plan_spatial_order(const PlannedFrame& pf, const FrameDev* fd, int64_t x0, int64_t key0,
                                        int64_t* keys, int* chunks) {
  std::vector<SortSeg> out;
  *keys = 0;
  *chunks = 0;
  if (pf.variant == V_TRIC_SEARCH) return out;
  const int64_t* o = pf.src->species_offsets;
  for (int a = 0; a < pf.src->n_species; ++a) {
    const int64_t na = o[a + 1] - o[a];
    if (na < kSortMinParticles) continue;
    SortSeg g;
    std::memset(&g, 0, sizeof g);
    g.fd = fd;
    g.x0 = x0 + o[a];
    g.n = (int32_t)na;
    g.g = sort_grid_bits(na);
    g.key0 = key0 + *keys;
    *keys += (int64_t)1 << (3 * g.g);
    *chunks = std::max<int>(*chunks, (int)((na + kSortChunk - 1) / kSortChunk));
    out.push_back(g);
  }
  return out;
}

size_t coord_bytes(const dh_frame* f) {
  const size_t elem = (f->flags & DH_COORDS_F64) ? sizeof(double) : sizeof(float);
  return elem * (size_t)f->n * ((f->flags & DH_COORDS_F4) ? 4 : 3);
}

int default_block(int variant, int width) {
  if (width < 16384) return kBlockSmall;
  for (int block = kBlockHuge; block > kBlockSmall; block /= 2)
    if (pair_kernel_blocks_per_sm(variant, width, 1, block) >= 1) return block;
  return kBlockSmall;
}

// Tiles of one frame's species pairs for every bin sweep (fd: the frame's
// device descriptor; items numbered from item0): the first min(cap, total)
// segments are written to out, *n_out receives the total, and the item count
// is returned.
int64_t fill_segments(const PlannedFrame& pf, FrameDev* fd, int64_t item0, int jm, Segment* out, int cap,
                      int* n_out) {
  const dh_frame* f = pf.src;
  jm = (jm == 2 || jm == 4) ? jm : 1;
  const int tile_j = kTile / jm;
  const int64_t* o = f->species_offsets;
  int S = f->n_species;
  int64_t items = 0;
  int n = 0;
  for (int pass = 0; pass < pf.sweeps; ++pass) {
    int h = 0;
    for (int a = 0; a < S; ++a)
      for (int b = a; b < S; ++b, ++h) {
        int32_t na = (int32_t)(o[a + 1] - o[a]), nb = (int32_t)(o[b + 1] - o[b]);
        bool intra = (a == b);
        if (na == 0 || nb == 0 || (intra && na < 2)) continue;
        Segment s;
        std::memset(&s, 0, sizeof s);
        s.fd = fd;
        s.intra = intra ? 1 : 0;
        s.h = h;
        s.pass = pass;
        s.a0 = (int32_t)o[a];
        s.na = na;
        s.b0 = (int32_t)o[b];
        s.nb = nb;
        s.n_ti = (na + kTile - 1) / kTile;
        s.n_tj = (nb + tile_j - 1) / tile_j;
        s.jm = jm;
        s.item0 = item0 + items;
        s.item_base = 0;
        // intra: row ti keeps the j tiles tj >= jm ti (at least one, since na > (n_ti - 1) kTile)
        items += intra ? (int64_t)s.n_ti * s.n_tj - (int64_t)jm * s.n_ti * (s.n_ti - 1) / 2
                       : (int64_t)s.n_ti * s.n_tj;
        if (n < cap) out[n] = s;
        ++n;
      }
  }
  *n_out = n;
  return items;
}

int64_t add_segments(const PlannedFrame& pf, FrameDev* fd, int64_t item0, std::vector<Segment>& segs, int jm) {
  int n = 0;
  fill_segments(pf, fd, item0, jm, nullptr, 0, &n);
  const size_t at = segs.size();
  segs.resize(at + (size_t)n);
  return fill_segments(pf, fd, item0, jm, segs.data() + at, n, &n);
}

namespace {

void release_held(dh_ctx* c) {
  for (const double* T : c->held_tables) c->tcache.release(T);
  c->held_tables.clear();
}

// The frames of one minimum-image variant in a call, as the autotuner keys them.
struct VariantSummary {
  int frames = 0, width = 1, multi = 0;
  double pairs = 0.0;
  TuneKey key() const { return make_tune_key(0, width, frames ? pairs / frames : 0.0, frames); }
};

VariantSummary summarize(const std::vector<PlannedFrame>& pfs, int v) {
  VariantSummary s;
  for (const auto& pf : pfs)
    if (pf.variant == v) {
      ++s.frames;
      s.width = std::max(s.width, pf.sweep_width);
      s.multi |= pf.sweeps > 1;
      s.pairs += (double)pf.pairs;
    }
  return s;
}

TuneKey variant_key(const VariantSummary& s, int v) {
  TuneKey k = s.key();
  k.variant = v;
  return k;
}

// Launch shape for a variant: forced during a measurement, else the tuned
// shape of its key, else one j tile per i tile, one histogram copy and as
// many blocks per SM as fit.
LaunchParams launch_params(dh_ctx* c, const VariantSummary& s, int v) {
  if (c->tune_forced) return c->tune_force;
  LaunchParams p;
  if (c->tuner.lookup(variant_key(s, v), &p)) return p;
  p.block = default_block(v, s.width);
  return p;
}

// Host-side plan of one call: buffers sized, threshold tables referenced,
// descriptors written to the pinned staging buffer, launch shapes chosen.
// Nothing in it enqueues work except threshold tables that are not cached yet.
struct CallPlan {
  int k = 0;
  bool host_coords = false, with_pairs = true;
  size_t meta_bytes = 0;
  int n_jobs = 0;
  int64_t n_chunks = 0;
  int64_t n_items = 0;
  int64_t vitems[kNumVariants] = {0, 0, 0, 0};
  size_t vseg0[kNumVariants + 1] = {0, 0, 0, 0, 0};
  int vwidth[kNumVariants] = {1, 1, 1, 1};
  int vmulti[kNumVariants] = {0, 0, 0, 0};
  LaunchParams vparams[kNumVariants];
  int vgrid[kNumVariants] = {0, 0, 0, 0};
  std::vector<size_t> raw_off;  // per frame, byte offset in c->raw (host coordinates)
  bool any_f64 = false;         // some frame has binary64 coordinates
  int max_pass = 1;
  int launched = 0;
  size_t seg_bytes = 0;          // Segment array in the metadata
  int n_sort = 0;                // spatial-order segments (after the Segments in the metadata)
  int sort_chunks = 0;           // most staging chunks of one of them
  int64_t sort_keys = 0;         // counters over all of them
  int64_t sort_particles = 0;    // particles of the frames (index space of keys and the scratch copy)
};



dh_status prepare_frames(dh_ctx* c, const std::vector<PlannedFrame>& pfs, const std::vector<uint64_t*>& dev_out,
                         bool host_coords, bool with_pairs, CallPlan& P) {
  cudaStream_t st = c->stream();
  int k = (int)pfs.size();
  P.k = k;
  P.host_coords = host_coords;
  P.with_pairs = with_pairs;
  std::vector<int64_t> xoff(k + 1, 0);
  size_t raw_bytes = 0;
  P.raw_off.assign((size_t)k, 0);
  P.any_f64 = false;
  for (int f = 0; f < k; ++f) {
    const dh_frame* fr = pfs[f].src;
    xoff[f + 1] = xoff[f] + fr->n;
    P.raw_off[f] = raw_bytes;
    P.any_f64 |= (fr->flags & DH_COORDS_F64) != 0;
    if (host_coords) raw_bytes += (coord_bytes(fr) + 15) & ~(size_t)15;
  }
  DH_CUDA_TRY(c->X.ensure(sizeof(float4) * (size_t)std::max<int64_t>(xoff[k], 1)));
  if (P.any_f64) DH_CUDA_TRY(c->X64.ensure(sizeof(double4) * (size_t)std::max<int64_t>(xoff[k], 1)));
  if (host_coords) DH_CUDA_TRY(c->raw.ensure(std::max<size_t>(raw_bytes, 16)));
  DH_CUDA_TRY(c->ctl.ensure(sizeof(Control) * kNumVariants));
  // device metadata: FrameDev[k] | StageJob[k] | Segment[m], uploaded in one copy;
  // segments are grouped by minimum-image variant (one pair-kernel launch each)
  std::vector<Segment> segs;
  VariantSummary vsum[kNumVariants];
  for (int v = 0; v < kNumVariants; ++v) {
    vsum[v] = summarize(pfs, v);
    P.vparams[v] = launch_params(c, vsum[v], v);
  }
  auto plan_segments = [&](FrameDev* dF) {
    segs.clear();
    P.n_items = 0;
    for (int v = 0; v < kNumVariants; ++v) {
      P.vseg0[v] = segs.size();
      P.vitems[v] = 0;
      for (int f = 0; f < k; ++f)
        if (pfs[f].variant == v)
          P.vitems[v] += add_segments(pfs[f], dF + f, P.vitems[v], segs, P.vparams[v].jm);
      P.n_items += P.vitems[v];
    }
    P.vseg0[kNumVariants] = segs.size();
  };
  // spatial order of the species of periodic frames without the 27-image search
  std::vector<SortSeg> sorts;
  auto plan_sorts = [&](FrameDev* dF) {
    sorts.clear();
    P.sort_keys = 0;
    P.sort_chunks = 0;
    for (int f = 0; f < k; ++f) {
      int64_t keys = 0;
      int chunks = 0;
      std::vector<SortSeg> fs = plan_spatial_order(pfs[f], dF + f, xoff[f], P.sort_keys, &keys, &chunks);
      sorts.insert(sorts.end(), fs.begin(), fs.end());
      P.sort_keys += keys;
      P.sort_chunks = std::max(P.sort_chunks, chunks);
    }
    P.n_sort = (int)sorts.size();
    P.sort_particles = xoff[k];
  };
  DH_CUDA_TRY(c->meta.ensure(sizeof(FrameDev) * (size_t)k + sizeof(StageJob) * (size_t)k));
  plan_segments((FrameDev*)c->meta.p);
  plan_sorts((FrameDev*)c->meta.p);
  P.seg_bytes = sizeof(Segment) * std::max<size_t>(segs.size(), 1);
  P.meta_bytes = sizeof(FrameDev) * (size_t)k + sizeof(StageJob) * (size_t)k + P.seg_bytes +
                 sizeof(SortSeg) * sorts.size();
  void* before = c->meta.p;
  DH_CUDA_TRY(c->meta.ensure(P.meta_bytes));
  DH_CUDA_TRY(c->hmeta.ensure(P.meta_bytes));
  if (c->meta.p != before) {  // buffer moved
    plan_segments((FrameDev*)c->meta.p);
    plan_sorts((FrameDev*)c->meta.p);
  }
  if (P.n_sort > 0) {
    DH_CUDA_TRY(c->sortX.ensure(sizeof(float4) * (size_t)P.sort_particles));
    if (P.any_f64) DH_CUDA_TRY(c->sortX64.ensure(sizeof(double4) * (size_t)P.sort_particles));
    DH_CUDA_TRY(c->sortK.ensure(sizeof(int32_t) * (size_t)P.sort_particles));
    DH_CUDA_TRY(c->sortC.ensure(sizeof(uint32_t) * (size_t)P.sort_keys));
  }
  FrameDev* dF = (FrameDev*)c->meta.p;
  FrameDev* hF = (FrameDev*)c->hmeta.p;
  StageJob* hJ = (StageJob*)(hF + k);
  Segment* hS = (Segment*)(hJ + k);
  for (int f = 0; f < k; ++f) {
    double* T = nullptr;
    dh_status s = c->tcache.acquire(pfs[f].src->r_max, pfs[f].src->nbins, st, (int32_t*)c->tstat.p, &T, &P.launched);
    if (s != DH_OK) return s;
    c->held_tables.push_back(T);
    fill_frame_dev(pfs[f], hF[f], (const float4*)c->X.p + xoff[f], dev_out[f], T);
    if (pfs[f].src->flags & DH_COORDS_F64) hF[f].X64 = (const double4*)c->X64.p + xoff[f];
    P.max_pass = std::max(P.max_pass, pfs[f].sweeps);
  }
  // A1 staging jobs
  P.n_jobs = 0;
  P.n_chunks = 0;
  for (int f = 0; f < k; ++f) {
    const dh_frame* fr = pfs[f].src;
    if (fr->n == 0) continue;
    StageJob& J = hJ[P.n_jobs++];
    std::memset(&J, 0, sizeof J);
    J.stride = (fr->flags & DH_COORDS_F4) ? 4 : 3;
    J.src = host_coords ? (const float*)((const unsigned char*)c->raw.p + P.raw_off[f]) : fr->coords;
    J.dst = (float4*)c->X.p + xoff[f];
    J.dst64 = (fr->flags & DH_COORDS_F64) ? (double4*)c->X64.p + xoff[f] : nullptr;
    J.fd = dF + f;
    J.n = fr->n;
    J.chunk0 = P.n_chunks;
    P.n_chunks += (fr->n + kStageChunk - 1) / kStageChunk;
  }
  if (!segs.empty()) std::memcpy(hS, segs.data(), sizeof(Segment) * segs.size());
  if (!sorts.empty())
    std::memcpy((unsigned char*)hS + P.seg_bytes, sorts.data(), sizeof(SortSeg) * sorts.size());
  // launch shapes (occupancy queries and kernel attributes stay outside any stream capture)
  for (int v = 0; v < kNumVariants; ++v) {
    P.vgrid[v] = 0;
    if (P.vitems[v] == 0 || !with_pairs) continue;
    const int width = vsum[v].width;
    P.vmulti[v] = vsum[v].multi;
    LaunchParams& lp = P.vparams[v];
    int bps_max = pair_kernel_blocks_per_sm(v, width, lp.depth, lp.block);
    if (bps_max < 1 && lp.depth > 1) {
      lp.depth = 1;  // the copies do not fit: one copy
      bps_max = pair_kernel_blocks_per_sm(v, width, 1, lp.block);
    }
    if (bps_max < 1 && lp.block != kBlockSmall) {
      lp.block = kBlockSmall;  // the larger block's queues do not fit either
      bps_max = pair_kernel_blocks_per_sm(v, width, 1, kBlockSmall);
    }
    if (bps_max < 1) return fail(DH_ERR_INVALID, "histogram of %d bins does not fit in shared memory", width);
    lp.bps = lp.bps > 0 ? std::min(lp.bps, bps_max) : bps_max;
    P.vwidth[v] = width;
    P.vgrid[v] = pair_grid(c->num_sms, lp.bps, P.vitems[v]);
  }
  return DH_OK;
}

// The stream operations of a planned call (capturable into a CUDA graph when
// the coordinates are device pointers).
dh_status record_frames(dh_ctx* c, const std::vector<PlannedFrame>& pfs, CallPlan& P) {
  cudaStream_t st = c->stream();
  int k = P.k;
  FrameDev* dF = (FrameDev*)c->meta.p;
  StageJob* dJ = (StageJob*)(dF + k);
  Segment* dS = (Segment*)(dJ + k);
  int launched = 0;
  if (P.host_coords)
    for (int f = 0; f < k; ++f) {
      const dh_frame* fr = pfs[f].src;
      if (fr->n == 0) continue;
      DH_CUDA_TRY(cudaMemcpyAsync((unsigned char*)c->raw.p + P.raw_off[f], fr->coords, coord_bytes(fr),
                                  cudaMemcpyHostToDevice, st));
    }
  DH_CUDA_TRY(cudaMemcpyAsync(dF, c->hmeta.p, P.meta_bytes, cudaMemcpyHostToDevice, st));
  if (P.n_jobs > 0) {
    DH_CUDA_TRY(launch_stage(dJ, P.n_jobs, P.n_chunks, st));
    ++launched;
  }
  if (P.n_sort > 0) {
    const SortSeg* dSort = (const SortSeg*)((unsigned char*)dS + P.seg_bytes);
    DH_CUDA_TRY(cudaMemsetAsync(c->sortC.p, 0, sizeof(uint32_t) * (size_t)P.sort_keys, st));
    DH_CUDA_TRY(launch_spatial_sort(dSort, P.n_sort, P.sort_chunks, (float4*)c->X.p, (float4*)c->sortX.p,
                                    P.any_f64 ? (double4*)c->X64.p : nullptr,
                                    P.any_f64 ? (double4*)c->sortX64.p : nullptr, (int32_t*)c->sortK.p,
                                    (uint32_t*)c->sortC.p, st));
    launched += 4;
  }
  DH_CUDA_TRY(launch_frame_setup(dF, k, 0, st));
  ++launched;
  // A2-A8: per variant, one persistent launch over its frames, species pairs and bin sweeps
  int grid = 0, top = -1;
  int64_t top_items = 0;
  bool any = false;
  for (int v = 0; v < kNumVariants; ++v) any |= P.vgrid[v] > 0;
  // timing events: inside a stream capture they must become event-record nodes
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DH_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
  const unsigned ev_flags = (cs == cudaStreamCaptureStatusActive) ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (any) {
    DH_CUDA_TRY(cudaMemsetAsync(c->ctl.p, 0, sizeof(Control) * kNumVariants, st));
    if (c->ev_pair0) DH_CUDA_TRY(cudaEventRecordWithFlags(c->ev_pair0, st, ev_flags));
    for (int v = 0; v < kNumVariants; ++v) {
      if (P.vgrid[v] == 0) continue;
      PairLaunch L;
      std::memset(&L, 0, sizeof L);
      L.segs = dS + P.vseg0[v];
      L.n_segs = (int32_t)(P.vseg0[v + 1] - P.vseg0[v]);
      L.n_items = P.vitems[v];
      if (c->tune_forced && c->tune_cap_pairs > 0.0) {  // a measurement: the first items only
        const double per_item = (double)kTile * (double)(kTile / P.vparams[v].jm);
        L.n_items = std::min<int64_t>(L.n_items, (int64_t)std::ceil(c->tune_cap_pairs / per_item));
      }
      L.hist_width = P.vwidth[v];
      L.hist_depth = P.vparams[v].depth;
      L.multi = P.vmulti[v];
      L.block = P.vparams[v].block;
      L.agg = (P.vparams[v].agg && L.block == kBlockSmall && !L.multi) ? 1 : 0;
      L.ctl = (Control*)c->ctl.p + v;
      DH_CUDA_TRY(launch_pairs(L, v, P.vgrid[v],
                               pair_kernel_smem(P.vwidth[v], P.vparams[v].depth, P.vparams[v].block), st));
      ++launched;
      grid = std::max(grid, P.vgrid[v]);
      if (P.vitems[v] > top_items) {
        top_items = P.vitems[v];
        top = v;
      }
    }
    if (c->ev_pair1) DH_CUDA_TRY(cudaEventRecordWithFlags(c->ev_pair1, st, ev_flags));
  }
  c->timed = (c->ev_pair0 != nullptr) && any;
  dh_stats& S = c->stats;
  std::memset(&S, 0, sizeof S);
  for (auto& pf : pfs) S.pairs += pf.pairs;
  S.sweeps = P.max_pass;
  S.blocks = grid;
  S.items = (int32_t)std::min<int64_t>(P.n_items, 0x7FFFFFFF);
  S.kernel_launches = launched + P.launched;
  S.tune_runs = c->tune_runs;
  if (top >= 0) {
    S.tile_j = kTile / P.vparams[top].jm;
    S.hist_depth = P.vparams[top].depth;
    S.blocks_per_sm = P.vparams[top].bps;
    S.block_threads = P.vparams[top].block;
    S.warp_agg = (P.vparams[top].agg && P.vparams[top].block == kBlockSmall && !P.vmulti[top]) ? 1 : 0;
  }
  return DH_OK;
}

dh_status enqueue_frames(dh_ctx* c, const std::vector<PlannedFrame>& pfs, const std::vector<uint64_t*>& dev_out,
                         bool host_coords, bool with_pairs = true) {
  CallPlan P;
  dh_status s = prepare_frames(c, pfs, dev_out, host_coords, with_pairs, P);
  if (s != DH_OK) return s;
  return record_frames(c, pfs, P);
}

// After the stream has drained: read back per-frame flags and statistics.
dh_status finish_frames(dh_ctx* c, int k) {
  FrameDev* hF = (FrameDev*)c->hmeta.p;
  DH_CUDA_TRY(cudaMemcpyAsync(hF, c->meta.p, sizeof(FrameDev) * (size_t)k, cudaMemcpyDeviceToHost, c->stream()));
  int32_t tstat = 0;
  DH_CUDA_TRY(cudaMemcpyAsync(&tstat, c->tstat.p, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream()));
  cudaError_t e = cudaStreamSynchronize(c->stream());
  release_held(c);
  DH_CUDA_TRY(e);
  if (tstat != 0) return fail(DH_ERR_CUDA, "bin threshold table did not converge");
  if (c->timed) {
    float ms = 0.0f;
    DH_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev_pair0, c->ev_pair1));
    c->stats.pair_kernel_ms = ms;
  }
  for (int f = 0; f < k; ++f) {
    c->stats.deferred += hF[f].deferred;
    c->stats.exact_fallback += hF[f].exact;
    c->stats.uniform_pairs += hF[f].uniform_pairs;
    c->stats.axis_pairs += hF[f].axis_pairs;
    c->stats.culled_pairs += hF[f].culled_pairs;
    if (hF[f].bad) return fail(DH_ERR_INVALID, "frame %d has non-finite coordinates", f);
  }
  return DH_OK;
}

dh_status autotune_call(dh_ctx* c, const std::vector<PlannedFrame>& pfs);

// One call: check, plan, then enqueue directly or (batched device-pointer
// calls) as a CUDA graph that is captured per call and replayed through an
// updated executable graph.
dh_status run_frames(dh_ctx* c, const dh_frame* frames, int k, bool wait, bool use_graph = false) {
  if (k < 0) return fail(DH_ERR_INVALID, "negative frame count");
  if (k == 0) return DH_OK;
  std::vector<PlannedFrame> pfs((size_t)k);
  bool dev = (frames[0].flags & DH_DEVICE_PTRS) != 0;
  for (int f = 0; f < k; ++f) {
    dh_status s = check_frame(&frames[f], pfs[f], c->max_width);
    if (s != DH_OK) return s;
    if (((frames[f].flags & DH_DEVICE_PTRS) != 0) != dev)
      return fail(DH_ERR_INVALID, "all frames of a batch must use the same pointer kind");
  }
  if (!c->tune_forced) {
    c->tune_runs = 0;
    dh_status ts = autotune_call(c, pfs);
    if (ts != DH_OK) return ts;
  }
  const bool graph = use_graph && dev && !(c->cfg.flags & DH_CFG_NO_GRAPH);
  cudaStream_t st = c->stream();
  std::vector<uint64_t*> dev_out((size_t)k);
  std::vector<size_t> hoff((size_t)k + 1, 0);
  for (int f = 0; f < k; ++f) hoff[f + 1] = hoff[f] + (size_t)pfs[f].n_hist * frames[f].nbins;
  if (dev) {
    for (int f = 0; f < k; ++f) dev_out[f] = frames[f].out;
  } else {
    DH_CUDA_TRY(c->hist.ensure(sizeof(uint64_t) * std::max<size_t>(hoff[k], 1)));
    for (int f = 0; f < k; ++f) dev_out[f] = (uint64_t*)c->hist.p + hoff[f];
  }
  DH_CUDA_TRY(cudaMemsetAsync(c->tstat.p, 0, sizeof(int32_t), st));
  CallPlan P;
  dh_status s = prepare_frames(c, pfs, dev_out, !dev, true, P);
  if (s == DH_OK && graph) {
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) s = fail(DH_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
  }
  if (s == DH_OK) {
    cudaError_t e = cudaSuccess;
    if (dev) {
      for (int f = 0; f < k && e == cudaSuccess; ++f)
        if (!(frames[f].flags & DH_ACCUMULATE))
          e = cudaMemsetAsync(frames[f].out, 0, sizeof(uint64_t) * (hoff[f + 1] - hoff[f]), st);
    } else {
      e = cudaMemsetAsync(c->hist.p, 0, sizeof(uint64_t) * hoff[k], st);
    }
    if (e != cudaSuccess) s = fail(DH_ERR_CUDA, "output memset: %s", cudaGetErrorString(e));
    if (s == DH_OK) s = record_frames(c, pfs, P);
  }
  if (graph && P.k > 0) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(st, &g);
      if (s == DH_OK && e != cudaSuccess) s = fail(DH_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
      if (s == DH_OK) {
        if (c->gexec) {
          cudaGraphExecUpdateResultInfo info;
          if (cudaGraphExecUpdate(c->gexec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
          }
        }
        if (!c->gexec) {
          e = cudaGraphInstantiate(&c->gexec, g, 0);
          if (e != cudaSuccess) {
            c->gexec = nullptr;
            s = fail(DH_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
          }
        }
        if (s == DH_OK) {
          e = cudaGraphLaunch(c->gexec, st);
          if (e != cudaSuccess) s = fail(DH_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
        }
      }
      if (g) cudaGraphDestroy(g);
      c->stats.graph_replays = (s == DH_OK) ? 1 : 0;
    }
  }
  if (s != DH_OK) {
    cudaStreamSynchronize(st);
    release_held(c);
    return s;
  }
  if (!dev) {
    bool any_acc = false;
    for (int f = 0; f < k; ++f) any_acc |= (frames[f].flags & DH_ACCUMULATE) != 0;
    if (any_acc) DH_CUDA_TRY(c->hout.ensure(sizeof(uint64_t) * std::max<size_t>(hoff[k], 1)));
    for (int f = 0; f < k; ++f) {
      size_t cnt = hoff[f + 1] - hoff[f];
      if (frames[f].flags & DH_ACCUMULATE)
        DH_CUDA_TRY(cudaMemcpyAsync((uint64_t*)c->hout.p + hoff[f], dev_out[f], sizeof(uint64_t) * cnt,
                                 cudaMemcpyDeviceToHost, st));
      else
        DH_CUDA_TRY(cudaMemcpyAsync(frames[f].out, dev_out[f], sizeof(uint64_t) * cnt, cudaMemcpyDeviceToHost, st));
    }
  }
  if (!wait && dev) {
    c->pending_async = true;
    return DH_OK;
  }
  s = finish_frames(c, k);
  if (s != DH_OK) return s;
  if (!dev) {
    for (int f = 0; f < k; ++f)
      if (frames[f].flags & DH_ACCUMULATE) {
        const uint64_t* src = (const uint64_t*)c->hout.p + hoff[f];
        for (size_t q = 0; q < hoff[f + 1] - hoff[f]; ++q) frames[f].out[q] += src[q];
      }
  }
  return DH_OK;
}

// ---- autotuner measurements

uint64_t splitmix64(uint64_t& z) {
  uint64_t x = (z += 0x9E3779B97F4A7C15ull);
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Measures every launch shape on a synthetic batch shaped like the frames of
// variant v in the call (same histogram width and sweeps, the mean frame size
// up to 2^21 particles, up to 64 frames): uniform particles at density 0.1 in a
// cube (none: every pair in range; orthorhombic: r_max = L/2) or in the
// 70/80/100-degree cell (r_max = 0.95 h_min/2, or 0.75 h_min for the 27-image
// search).  Each measurement covers about 6e9 pairs: whole frames, or the
// first work items of a larger one (the same tile geometry as the whole).  The
// fastest shape is stored under the variant's launch key.
dh_status tune_variant(dh_ctx* c, int v, const VariantSummary& vs) {
  const double mean_pairs = vs.pairs / std::max(vs.frames, 1);
  int64_t n = (int64_t)std::llround(std::sqrt(2.0 * std::max(mean_pairs, 1.0)));
  n = std::min<int64_t>(std::max<int64_t>(n, 64), (int64_t)1 << 21);
  const double pairs_one = 0.5 * (double)n * (double)(n - 1);
  const double target = 6e9;
  const int nf = (int)std::min<int64_t>(std::max<int64_t>(std::llround(target / pairs_one), 1),
                                        std::min(vs.frames, 64));
  c->tune_cap_pairs = (nf * pairs_one > 1.5 * target) ? target : 0.0;
  const int nbins = vs.multi ? 2 * vs.width : vs.width;
  const double vol = (double)n / 0.1;
  double box[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double r_max = 0.0;
  int32_t box_type = DH_BOX_NONE;
  if (v == V_NONE || v == V_ORTHO) {
    double L = std::cbrt(vol);
    box[0] = box[4] = box[8] = L;
    box_type = (v == V_NONE) ? DH_BOX_NONE : DH_BOX_ORTHO;
    r_max = (v == V_NONE) ? L * std::sqrt(3.0) * 1.0001 : 0.5 * L;
  } else {
    const double d2r = 3.14159265358979323846 / 180.0, ca = std::cos(70 * d2r), cb = std::cos(80 * d2r), cg = std::cos(100 * d2r),
                 sg = std::sin(100 * d2r);
    const double cy = (ca - cb * cg) / sg, cz = std::sqrt(1.0 - cb * cb - cy * cy);
    const double l = std::cbrt(vol / (sg * cz));
    box[0] = l; box[1] = l * cg; box[2] = l * cb;
    box[4] = l * sg; box[5] = l * cy;
    box[8] = l * cz;
    // plane spacings: V / |b x c|, V / |c x a|, V / |a x b|
    const double a[3] = {box[0], 0, 0}, b[3] = {box[1], box[4], 0}, cc[3] = {box[2], box[5], box[8]};
    auto cross_norm = [](const double* x, const double* y) {
      double u = x[1] * y[2] - x[2] * y[1], w = x[2] * y[0] - x[0] * y[2], z = x[0] * y[1] - x[1] * y[0];
      return std::sqrt(u * u + w * w + z * z);
    };
    const double V = box[0] * box[4] * box[8];
    const double h_min = std::min(V / cross_norm(b, cc), std::min(V / cross_norm(cc, a), V / cross_norm(a, b)));
    box_type = DH_BOX_TRICLINIC;
    r_max = (v == V_TRIC) ? 0.95 * 0.5 * h_min : 0.75 * h_min;
  }
  std::vector<float> hx((size_t)nf * n * 3);
  uint64_t z = 0x5eedull + (uint64_t)v;
  for (size_t q = 0; q < hx.size(); q += 3) {
    double s0 = (double)(splitmix64(z) >> 11) * 0x1.0p-53, s1 = (double)(splitmix64(z) >> 11) * 0x1.0p-53,
           s2 = (double)(splitmix64(z) >> 11) * 0x1.0p-53;
    hx[q] = (float)(box[0] * s0 + box[1] * s1 + box[2] * s2);
    hx[q + 1] = (float)(box[4] * s1 + box[5] * s2);
    hx[q + 2] = (float)(box[8] * s2);
    if (v == V_NONE) {  // the cube as a non-periodic region
      double L = box[0];
      hx[q] = (float)(L * s0); hx[q + 1] = (float)(L * s1); hx[q + 2] = (float)(L * s2);
    }
  }
  if (v == V_NONE) std::fill(box, box + 9, 0.0);
  DevBuf dx, dout;
  DH_CUDA_TRY(dx.ensure(sizeof(float) * hx.size()));
  DH_CUDA_TRY(dout.ensure(sizeof(uint64_t) * (size_t)nf * nbins));
  DH_CUDA_TRY(cudaMemcpy(dx.p, hx.data(), sizeof(float) * hx.size(), cudaMemcpyHostToDevice));
  int64_t offs[2] = {0, n};
  std::vector<dh_frame> fr((size_t)nf);
  for (int f = 0; f < nf; ++f) {
    dh_frame& d = fr[f];
    std::memset(&d, 0, sizeof d);
    d.coords = (const float*)dx.p + (size_t)f * n * 3;
    d.n = n;
    d.species_offsets = offs;
    d.n_species = 1;
    d.box_type = box_type;
    std::memcpy(d.box, box, sizeof box);
    d.r_max = r_max;
    d.nbins = nbins;
    d.out = (uint64_t*)dout.p + (size_t)f * nbins;
    d.flags = DH_DEVICE_PTRS;
  }
  const bool own_events = (c->ev_pair0 == nullptr);
  if (own_events) {
    DH_CUDA_TRY(cudaEventCreate(&c->ev_pair0));
    DH_CUDA_TRY(cudaEventCreate(&c->ev_pair1));
  }
  c->tune_forced = true;
  TuneEntry best;
  dh_status s = DH_OK;
  auto measure = [&](const LaunchParams& p, double* gps) {
    c->tune_force = p;
    dh_status r = run_frames(c, fr.data(), nf, true, false);
    if (r != DH_OK) return r;
    ++c->tune_runs;
    double ms = c->stats.pair_kernel_ms;
    double pairs = pairs_one * nf;
    if (c->tune_cap_pairs > 0.0) {  // whole items of the capped launch
      const double per_item = (double)kTile * (double)(kTile / p.jm);
      pairs = std::min(pairs, std::ceil(c->tune_cap_pairs / per_item) * per_item);
    }
    *gps = ms > 0.0 ? pairs / (ms * 1e6) : 0.0;
    return DH_OK;
  };
  // the shape used without a measurement is the reference; another shape must
  // beat it by 2 % (single measurements of nearby shapes differ by about 1 %)
  LaunchParams def;
  def.block = default_block(v, vs.width);
  def.bps = pair_kernel_blocks_per_sm(v, vs.width, 1, def.block);
  double g = 0.0;
  s = measure(def, &g);  // warm-up (first launches of a shape)
  if (s == DH_OK) s = measure(def, &g);
  best.p = def;
  best.gpairs_s = g;
  const double g_def = g;
  for (int block : {kBlockSmall, kBlockLarge, kBlockHuge})
    for (int jm = 1; jm <= 4 && s == DH_OK; jm *= 2)
      for (int depth = 1; depth <= 8 && s == DH_OK; depth *= 2) {
        int bmax = pair_kernel_blocks_per_sm(v, vs.width, depth, block);
        for (int bps = bmax; bps >= 1 && bps >= bmax - 1 && s == DH_OK; --bps) {
          LaunchParams p;
          p.jm = jm;
          p.depth = depth;
          p.bps = bps;
          p.block = block;
          s = measure(p, &g);
          if (s == DH_OK && g > best.gpairs_s && g > 1.02 * g_def) {
            best.p = p;
            best.gpairs_s = g;
          }
        }
      }
  // warp-aggregated increments (256-thread blocks, one sweep): the default
  // shape's copies and blocks with the aggregation
  if (s == DH_OK && !vs.multi && def.block == kBlockSmall) {
    LaunchParams p = def;
    p.agg = 1;
    s = measure(p, &g);
    if (s == DH_OK && g > best.gpairs_s && g > 1.02 * g_def) {
      best.p = p;
      best.gpairs_s = g;
    }
  }
  c->tune_forced = false;
  c->tune_cap_pairs = 0.0;
  if (own_events) {
    cudaEventDestroy(c->ev_pair0);
    cudaEventDestroy(c->ev_pair1);
    c->ev_pair0 = c->ev_pair1 = nullptr;
  }
  if (s != DH_OK) return s;
  if (best.gpairs_s > 0.0) {
    c->tuner.store(variant_key(vs, v), best);
    if (!c->tune_path.empty()) c->tuner.save(c->tune_path, c->num_sms);
  }
  return DH_OK;
}

// Before a call (DH_CFG_AUTOTUNE, outside any stream capture): measure the
// launch keys of its variants that have no tuned shape yet.
dh_status autotune_call(dh_ctx* c, const std::vector<PlannedFrame>& pfs) {
  if (!(c->cfg.flags & DH_CFG_AUTOTUNE)) return DH_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DH_CUDA_TRY(cudaStreamIsCapturing(c->stream(), &cs));
  if (cs != cudaStreamCaptureStatusNone) return DH_OK;
  for (int v = 0; v < kNumVariants; ++v) {
    VariantSummary vs = summarize(pfs, v);
    if (vs.frames == 0 || vs.pairs <= 0.0) continue;
    LaunchParams p;
    if (c->tuner.lookup(variant_key(vs, v), &p)) continue;
    dh_status s = tune_variant(c, v, vs);
    if (s != DH_OK) return s;
  }
  return DH_OK;
}

dh_status selfcheck(dh_ctx* c, int32_t what, const dh_frame* frame, uint64_t n_samples, uint64_t seed, double* out) {
  cudaStream_t st = c->stream();
  DevBuf res;
  DH_CUDA_TRY(res.ensure(4 * sizeof(unsigned long long)));
  DH_CUDA_TRY(cudaMemsetAsync(res.p, 0, 4 * sizeof(unsigned long long), st));
  unsigned long long h[4] = {0, 0, 0, 0};
  for (int q = 0; q < 4; ++q) out[q] = 0.0;
  if (what == DH_CHECK_SQRT) {
    DH_CUDA_TRY(launch_check_sqrt((unsigned long long*)res.p, st));
    DH_CUDA_TRY(cudaMemcpyAsync(h, res.p, sizeof h, cudaMemcpyDeviceToHost, st));
    DH_CUDA_TRY(cudaStreamSynchronize(st));
    res.release();
    std::memcpy(&out[0], &h[0], 8);
    return DH_OK;
  }
  if ((what != DH_CHECK_WINDOW && what != DH_CHECK_TILES) || !frame)
    return fail(DH_ERR_INVALID, "unknown self check %d", what);
  std::vector<PlannedFrame> pfs(1);
  dh_status s = check_frame(frame, pfs[0], c->max_width);
  if (s != DH_OK) return s;
  if (what == DH_CHECK_TILES && ((pfs[0].variant != V_ORTHO && pfs[0].variant != V_TRIC) || frame->n < 2))
    return fail(DH_ERR_INVALID, "the tile check needs an orthorhombic or triclinic frame without search");
  bool dev = (frame->flags & DH_DEVICE_PTRS) != 0;
  std::vector<uint64_t*> dev_out(1);
  DH_CUDA_TRY(c->hist.ensure(sizeof(uint64_t) * (size_t)pfs[0].n_hist * frame->nbins));
  dev_out[0] = (uint64_t*)c->hist.p;
  DH_CUDA_TRY(cudaMemsetAsync(c->tstat.p, 0, sizeof(int32_t), st));
  s = enqueue_frames(c, pfs, dev_out, !dev, false);
  if (s == DH_OK) {
    cudaError_t e =
        what == DH_CHECK_TILES
            ? launch_check_tiles((const FrameDev*)c->meta.p, pfs[0].variant, n_samples, seed,
                                 (unsigned long long*)res.p, st)
            : launch_check_window((const FrameDev*)c->meta.p, n_samples, seed, (unsigned long long*)res.p, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, res.p, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) s = fail(DH_ERR_CUDA, "self check: %s", cudaGetErrorString(e));
  }
  if (s == DH_OK) {
    s = finish_frames(c, 1);
  } else {
    cudaStreamSynchronize(st);
    release_held(c);
  }
  res.release();
  if (s != DH_OK) return s;
  double worst;
  std::memcpy(&worst, &h[0], 8);
  out[0] = worst;
  out[1] = (double)h[1];
  out[2] = (double)h[2];
  out[3] = what == DH_CHECK_TILES ? (double)h[3] : (double)((FrameDev*)c->hmeta.p)->delta;
  return DH_OK;
}

}  // namespace
}  // namespace dh

using namespace dh;

extern "C" {

const char* dh_version(void) { return "dh 0.1 (sm_103a)"; }

const char* dh_last_error(dh_ctx*) { return last_error_message(); }

dh_status dh_bin_thresholds(double r_max, int32_t nbins, double* thresholds) {
  if (!thresholds) return fail(DH_ERR_INVALID, "thresholds is NULL");
  if (nbins < 1 || nbins > DH_MAX_BINS) return fail(DH_ERR_INVALID, "nbins out of range");
  if (!(r_max > 0.0) || !std::isfinite(r_max)) return fail(DH_ERR_INVALID, "r_max must be > 0 and finite");
  if (!build_thresholds_host(r_max, nbins, thresholds))
    return fail(DH_ERR_INVALID, "threshold search did not converge");
  return DH_OK;
}

dh_status dh_rdf(dh_ctx* c, const uint64_t* counts, int32_t n_hist, int32_t nbins, double r_max,
                 const double* pair_density, uint64_t n_frames, double* g) {
  if (!c || !counts || !pair_density || !g) return fail(DH_ERR_INVALID, "NULL argument");
  if (n_hist < 1) return fail(DH_ERR_INVALID, "n_hist must be >= 1");
  if (nbins < 1 || nbins > DH_MAX_BINS) return fail(DH_ERR_INVALID, "nbins out of range");
  if (!(r_max > 0.0) || !std::isfinite(r_max)) return fail(DH_ERR_INVALID, "r_max must be > 0 and finite");
  if (n_frames == 0) return fail(DH_ERR_INVALID, "n_frames must be >= 1");
  for (int32_t h = 0; h < n_hist; ++h)
    if (!(pair_density[h] > 0.0) || !std::isfinite(pair_density[h]))
      return fail(DH_ERR_INVALID, "pair density %d must be > 0 and finite", h);
  std::lock_guard<std::recursive_mutex> g_(c->mu);
  DH_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t st = c->stream();
  DH_CUDA_TRY(c->aux.ensure(sizeof(double) * (size_t)n_hist));
  DH_CUDA_TRY(cudaMemcpyAsync(c->aux.p, pair_density, sizeof(double) * (size_t)n_hist, cudaMemcpyHostToDevice, st));
  DH_CUDA_TRY(launch_rdf(counts, n_hist, nbins, r_max, (const double*)c->aux.p, n_frames, g, st));
  DH_CUDA_TRY(cudaStreamSynchronize(st));
  return DH_OK;
}

dh_status dh_create(const dh_config* config, dh_ctx** out) {
  if (!out) return fail(DH_ERR_INVALID, "out is NULL");
  *out = nullptr;
  std::unique_ptr<dh_ctx> c(new dh_ctx());
  if (config) c->cfg = *config;
  c->device = c->cfg.device;
  int ndev = 0;
  DH_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (c->device < 0 || c->device >= ndev) return fail(DH_ERR_INVALID, "device %d not present", c->device);
  DH_CUDA_TRY(cudaSetDevice(c->device));
  DH_CUDA_TRY(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
  DH_CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  c->max_width = pair_kernel_max_width();
  if (c->max_width < 1024) return fail(DH_ERR_CUDA, "not enough shared memory per block");
  DH_CUDA_TRY(c->ctl.ensure(sizeof(Control) * kNumVariants));
  DH_CUDA_TRY(c->tstat.ensure(64));
  if (c->cfg.flags & DH_CFG_TIMING) {
    DH_CUDA_TRY(cudaEventCreate(&c->ev_pair0));
    DH_CUDA_TRY(cudaEventCreate(&c->ev_pair1));
  }
  if (c->cfg.tune_cache && c->cfg.tune_cache[0]) {
    c->tune_path = c->cfg.tune_cache;
    c->tuner.load(c->tune_path, c->num_sms);  // a missing file is an empty table
  }
  c->cfg.tune_cache = nullptr;  // the caller's string is not kept
  *out = c.release();
  return DH_OK;
}

dh_status dh_destroy(dh_ctx* c) {
  if (!c) return DH_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream());
  {
    std::lock_guard<std::mutex> g(c->server_mu);
    if (c->server) server_destroy(c->server);
    c->server = nullptr;
  }
  c->tcache.clear(c->stream());
  cudaStreamSynchronize(c->stream());
  c->raw.release();
  c->X.release();
  c->hist.release();
  c->meta.release();
  c->ctl.release();
  c->tstat.release();
  c->aux.release();
  c->sortX.release();
  c->sortX64.release();
  c->X64.release();
  c->sortK.release();
  c->sortC.release();
  c->hmeta.release();
  c->hout.release();
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->ev_pair0) cudaEventDestroy(c->ev_pair0);
  if (c->ev_pair1) cudaEventDestroy(c->ev_pair1);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
  return DH_OK;
}

dh_status dh_set_stream(dh_ctx* c, void* stream) {
  if (!c) return fail(DH_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> g(c->mu);
  c->user_stream = (cudaStream_t)stream;
  c->has_user_stream = stream != nullptr;
  return DH_OK;
}

dh_status dh_histogram(dh_ctx* c, const dh_frame* frame) {
  if (!c || !frame) return fail(DH_ERR_INVALID, "NULL argument");
  std::lock_guard<std::recursive_mutex> g(c->mu);
  cudaSetDevice(c->device);
  return run_frames(c, frame, 1, true);
}

dh_status dh_histogram_async(dh_ctx* c, const dh_frame* frame) {
  if (!c || !frame) return fail(DH_ERR_INVALID, "NULL argument");
  std::lock_guard<std::recursive_mutex> g(c->mu);
  cudaSetDevice(c->device);
  return run_frames(c, frame, 1, false);
}

dh_status dh_sync(dh_ctx* c) {
  if (!c) return fail(DH_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> g(c->mu);
  cudaSetDevice(c->device);
  if (!c->pending_async) {
    DH_CUDA_TRY(cudaStreamSynchronize(c->stream()));
    return DH_OK;
  }
  c->pending_async = false;
  return finish_frames(c, 1);
}

dh_status dh_histogram_batch(dh_ctx* c, const dh_frame* frames, int32_t k) {
  if (!c || (k > 0 && !frames)) return fail(DH_ERR_INVALID, "NULL argument");
  std::lock_guard<std::recursive_mutex> g(c->mu);
  cudaSetDevice(c->device);
  return run_frames(c, frames, k, true, true);
}

dh_status dh_selfcheck(dh_ctx* c, int32_t what, const dh_frame* frame, uint64_t n_samples, uint64_t seed,
                       double* out) {
  if (!c || !out) return fail(DH_ERR_INVALID, "NULL argument");
  std::lock_guard<std::recursive_mutex> g(c->mu);
  cudaSetDevice(c->device);
  return selfcheck(c, what, frame, n_samples, seed, out);
}

dh_status dh_get_stats(dh_ctx* c, dh_stats* s) {
  if (!c || !s) return fail(DH_ERR_INVALID, "NULL argument");
  std::lock_guard<std::recursive_mutex> g(c->mu);
  *s = c->stats;
  return DH_OK;
}

namespace {
dh::Server* get_server(dh_ctx* c, dh_status* st) {
  std::lock_guard<std::mutex> g(c->server_mu);
  *st = DH_OK;
  if (!c->server) c->server = server_create(c, st);
  return c->server;
}
}  // namespace

dh_status dh_submit(dh_ctx* c, const dh_frame* frame, uint64_t* ticket) {
  if (!c || !frame || !ticket) return fail(DH_ERR_INVALID, "NULL argument");
  dh_status st;
  dh::Server* s = get_server(c, &st);
  if (!s) return st;
  return server_submit(s, frame, ticket);
}

dh_status dh_poll(dh_ctx* c, uint64_t ticket) {
  if (!c) return fail(DH_ERR_INVALID, "ctx is NULL");
  dh_status st;
  dh::Server* s = get_server(c, &st);
  if (!s) return st;
  return server_poll(s, ticket);
}

dh_status dh_wait(dh_ctx* c, uint64_t ticket, uint64_t timeout_ns) {
  if (!c) return fail(DH_ERR_INVALID, "ctx is NULL");
  dh_status st;
  dh::Server* s = get_server(c, &st);
  if (!s) return st;
  return server_wait(s, ticket, timeout_ns);
}

dh_status dh_cancel(dh_ctx* c, uint64_t ticket) {
  if (!c) return fail(DH_ERR_INVALID, "ctx is NULL");
  dh_status st;
  dh::Server* s = get_server(c, &st);
  if (!s) return st;
  return server_cancel(s, ticket);
}

}  // extern "C"
