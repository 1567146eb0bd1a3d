// Autotuner: picks the launch shapes that never change results (clusters per
// grid bin, tracklet and refit block sizes) for a workload's size class by
// timing the tracking chain on it, and caches the choice in a text file.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tpct_internal.cuh"

namespace {

std::string tuning_key(const tpct_ctx* ctx, int64_t n, int32_t n_inst, int prec, int n_rows) {
  int dev = 0;
  cudaDeviceProp prop{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    std::strcpy(prop.name, "unknown");
  std::string name(prop.name);
  for (auto& ch : name) if (ch == ' ' || ch == '|') ch = '_';
  const int cls = n_inst > 0 && n > 0 ? (int)std::lround(std::log2((double)n / n_inst)) : 0;
  const int icls = n_inst > 0 ? (int)std::lround(std::log2((double)n_inst)) : 0;
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s|prec=%d|rows=%d|clusters_per_instance=2^%d|instances=2^%d", name.c_str(), prec,
                n_rows, cls, icls);
  (void)ctx;
  return buf;
}

bool cache_lookup(const char* path, const std::string& key, tpct_tuning* t) {
  if (!path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    char k[300];
    int a, b, c;
    float ms;
    if (std::sscanf(line, "%299s %d %d %d %f", k, &a, &b, &c, &ms) == 5 && key == k) {
      t->clusters_per_bin = a; t->tracklet_block = b; t->refit_block = c; t->ms = ms;
      found = true;   // the last entry for a key wins
    }
  }
  std::fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, const tpct_tuning& t) {
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %.4f\n", key.c_str(), t.clusters_per_bin, t.tracklet_block, t.refit_block, t.ms);
  std::fclose(f);
}

}  // namespace

extern "C" tpct_status tpct_autotune(tpct_ctx* ctx, const tpct_clusters* cl, int64_t n, tpct_tracks_out* out,
                                     tpct_stream stream, const char* cache_path, tpct_tuning* result) {
  if (!ctx || !cl || !out || !result) return TPCT_E_INVALID;
  tpct_tuning cur{};
  tpct_get_tuning(ctx, &cur);
  const std::string key = tuning_key(ctx, n, cl->n_instances, cur.precision, cur.n_rows);
  tpct_tuning cached = cur;
  if (cache_lookup(cache_path, key, &cached)) {
    tpct_status st = tpct_set_tuning(ctx, cached.clusters_per_bin, cached.tracklet_block, cached.refit_block);
    if (st != TPCT_OK) return st;
    tpct_get_tuning(ctx, result);
    result->ms = cached.ms;
    result->from_cache = 1;
    return TPCT_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return TPCT_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return TPCT_E_CUDA; }
  tpct_status st = TPCT_OK;
  // median of three timed runs after one warm-up
  auto time_cfg = [&](int cpb, int tlb, int rfb, float* ms) -> tpct_status {
    tpct_status r = tpct_set_tuning(ctx, cpb, tlb, rfb);
    if (r != TPCT_OK) return r;
    r = tpct_track(ctx, cl, n, out, stream);
    if (r != TPCT_OK) return r;
    float t[3];
    for (int i = 0; i < 3; ++i) {
      cudaEventRecord(e0, s);
      r = tpct_track(ctx, cl, n, out, stream);
      if (r != TPCT_OK) return r;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t[i], e0, e1) != cudaSuccess)
        return TPCT_E_CUDA;
    }
    std::sort(t, t + 3);
    *ms = t[1];
    return TPCT_OK;
  };
  int best_cpb = cur.clusters_per_bin, best_tlb = cur.tracklet_block, best_rfb = cur.refit_block;
  float best = 0.f;
  st = time_cfg(best_cpb, best_tlb, best_rfb, &best);
  // coordinate descent, one knob at a time
  const int cpbs[] = {1, 2, 4, 8};
  const int blocks[] = {64, 128, 256};
  for (int c : cpbs) {
    if (st != TPCT_OK) break;
    float ms;
    if (c == best_cpb) continue;
    st = time_cfg(c, best_tlb, best_rfb, &ms);
    if (st == TPCT_OK && ms < best) { best = ms; best_cpb = c; }
  }
  for (int b : blocks) {
    if (st != TPCT_OK) break;
    float ms;
    if (b == best_tlb) continue;
    st = time_cfg(best_cpb, b, best_rfb, &ms);
    if (st == TPCT_OK && ms < best) { best = ms; best_tlb = b; }
  }
  for (int b : blocks) {
    if (st != TPCT_OK) break;
    float ms;
    if (b == best_rfb) continue;
    st = time_cfg(best_cpb, best_tlb, b, &ms);
    if (st == TPCT_OK && ms < best) { best = ms; best_rfb = b; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != TPCT_OK) return st;
  st = tpct_set_tuning(ctx, best_cpb, best_tlb, best_rfb);
  if (st != TPCT_OK) return st;
  tpct_get_tuning(ctx, result);
  result->ms = best;
  result->from_cache = 0;
  cache_store(cache_path, key, *result);
  return TPCT_OK;
}
