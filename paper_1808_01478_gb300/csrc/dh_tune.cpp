// Autotuner bookkeeping: launch keys, the table of measured launch shapes and
// its text file.  The measurements themselves run in dh_runtime.cpp.
//
// The paper picks its kernel and launch parameters per GPU model from fixed
// heuristics (block size, Sec. 3.2.4; kernel choice by problem size, Sec. 4);
// here they are measured per launch key on the GPU that runs the work.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "dh_runtime.h"

namespace dh {

namespace {

int ceil_log2(int64_t v) {
  int b = 0;
  while (b < 62 && ((int64_t)1 << b) < v) ++b;
  return b;
}

bool valid_shape(const LaunchParams& p) {
  return (p.jm == 1 || p.jm == 2 || p.jm == 4) && (p.depth == 1 || p.depth == 2 || p.depth == 4 || p.depth == 8) &&
         p.bps >= 1 && p.bps <= 32 && (p.block == kBlockSmall || p.block == kBlockLarge || p.block == kBlockHuge) &&
         (p.agg == 0 || (p.agg == 1 && p.block == kBlockSmall));
}

// One cache line -> (sms, key, entry); false if malformed.
bool parse_line(const char* line, int* sms, TuneKey* k, TuneEntry* e) {
  int tile_j = 0, agg = 0;
  double g = 0.0;
  int n = std::sscanf(line, "%d %d %d %d %d %d %d %d %d %lf %d", sms, &k->variant, &k->width_log2, &k->n_log2,
                      &k->frames_log4, &tile_j, &e->p.block, &e->p.depth, &e->p.bps, &g, &agg);
  if (n != 10 && n != 11) return false;
  e->p.agg = agg;
  if (tile_j != 256 && tile_j != 512 && tile_j != 1024) return false;
  e->p.jm = kTile / tile_j;
  e->gpairs_s = g;
  if (*sms < 1 || k->variant < 0 || k->variant >= kNumVariants || k->width_log2 < 0 || k->width_log2 > 23 ||
      k->n_log2 < 0 || k->n_log2 > 40 || k->frames_log4 < 0 || k->frames_log4 > 3 || !(g > 0.0) ||
      !std::isfinite(g))
    return false;
  return valid_shape(e->p);
}

}  // namespace

TuneKey make_tune_key(int variant, int width, double mean_pairs_per_frame, int frames) {
  TuneKey k;
  k.variant = variant;
  k.width_log2 = ceil_log2(width < 1 ? 1 : width);
  double n_mean = std::sqrt(2.0 * (mean_pairs_per_frame > 1.0 ? mean_pairs_per_frame : 1.0));
  k.n_log2 = (int)std::lround(std::log2(n_mean));
  int f4 = 0;
  while (f4 < 3 && ((int64_t)1 << (2 * (f4 + 1))) <= frames) ++f4;
  k.frames_log4 = f4;
  return k;
}

bool Tuner::lookup(const TuneKey& k, LaunchParams* p) {
  std::lock_guard<std::mutex> g(mu_);
  auto it = map_.find(k);
  if (it == map_.end()) return false;
  *p = it->second.p;
  return true;
}

void Tuner::store(const TuneKey& k, const TuneEntry& e) {
  std::lock_guard<std::mutex> g(mu_);
  map_[k] = e;
}

size_t Tuner::size() {
  std::lock_guard<std::mutex> g(mu_);
  return map_.size();
}

int Tuner::load(const std::string& path, int sms) {
  FILE* fp = std::fopen(path.c_str(), "r");
  if (!fp) return -1;
  char line[512];
  int n = 0;
  std::lock_guard<std::mutex> g(mu_);
  while (std::fgets(line, sizeof line, fp)) {
    if (line[0] == '#') continue;
    int s = 0;
    TuneKey k;
    TuneEntry e;
    if (!parse_line(line, &s, &k, &e) || s != sms) continue;
    map_[k] = e;
    ++n;
  }
  std::fclose(fp);
  return n;
}

// Rewrites the file: entries of other SM counts already in it are kept.
bool Tuner::save(const std::string& path, int sms) {
  std::string keep;
  if (FILE* fp = std::fopen(path.c_str(), "r")) {
    char line[512];
    while (std::fgets(line, sizeof line, fp)) {
      int s = 0;
      TuneKey k;
      TuneEntry e;
      if (line[0] != '#' && parse_line(line, &s, &k, &e) && s != sms) keep += line;
    }
    std::fclose(fp);
  }
  std::string tmp = path + ".tmp";
  FILE* fp = std::fopen(tmp.c_str(), "w");
  if (!fp) return false;
  std::fprintf(fp, "# dh autotune cache: sms variant width_log2 n_log2 frames_log4 tile_j block depth bps gpairs_s agg\n");
  std::fputs(keep.c_str(), fp);
  {
    std::lock_guard<std::mutex> g(mu_);
    for (const auto& kv : map_)
      std::fprintf(fp, "%d %d %d %d %d %d %d %d %d %.3f %d\n", sms, kv.first.variant, kv.first.width_log2,
                   kv.first.n_log2, kv.first.frames_log4, kTile / kv.second.p.jm, kv.second.p.block,
                   kv.second.p.depth, kv.second.p.bps, kv.second.gpairs_s, kv.second.p.agg);
  }
  bool ok = std::fclose(fp) == 0;
  return ok && std::rename(tmp.c_str(), path.c_str()) == 0;
}

}  // namespace dh

extern "C" dh_status dh_tune_cache_count(const char* path, int32_t sm_count, int32_t* n_entries) {
  if (!path || !n_entries) return dh::fail(DH_ERR_INVALID, "path and n_entries must not be NULL");
  *n_entries = 0;
  dh::Tuner t;
  int n = t.load(path, sm_count);
  if (n < 0) return dh::fail(DH_ERR_NOTFOUND, "cannot read %s", path);
  *n_entries = (int32_t)t.size();
  return DH_OK;
}
