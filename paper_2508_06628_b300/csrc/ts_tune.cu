// ts_tune.cu -- launch-shape autotuner for the pair kernel: times each
// candidate CTA size on the live state with CUDA events and keeps the
// fastest, caching the choice in a text file keyed by (potential kinds,
// atom-count class, precision), one "key threads" line per entry.
#include <cstdio>
#include <fstream>
#include <map>
#include <sstream>

#include "ts_kernels.cuh"

namespace ts {

static std::string tune_key(const ts_batch* b) {
  std::ostringstream k;
  k << "pots=";
  for (int q = 0; q < b->n_pots; q++) k << b->pots[q].kind;
  int cls = 0;
  for (int64_t n = b->N; n > 1; n >>= 1) cls++;
  k << ";log2N=" << cls << ";fp64=" << (b->f64 ? 1 : 0);
  return k.str();
}

static std::map<std::string, int> read_cache(const std::string& path) {
  std::map<std::string, int> m;
  std::ifstream f(path);
  std::string key;
  int t;
  while (f >> key >> t) m[key] = t;
  return m;
}

void autotune_load(ts_batch* b) {
  b->pair_threads = 128;
}

}  // namespace ts

using namespace ts;

extern "C" ts_status ts_autotune(ts_batch* b, ts_state* s, void* stream) {
  ts_status r = check_state(b, s, false);
  if (r != TS_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  r = prologue(b, s, st, false);
  if (r != TS_OK) return r;
  ensure_forces(b, st);
  std::string key = tune_key(b);
  if (!b->cache_path.empty()) {
    auto m = read_cache(b->cache_path);
    auto it = m.find(key);
    if (it != m.end() && (it->second == 64 || it->second == 128 || it->second == 256)) {
      if (b->pair_threads != it->second) { b->pair_threads = it->second; b->graphs_valid = false; }
      return TS_OK;
    }
  }
  cudaEvent_t e0, e1;
  if (!cuda_ok(b, cudaEventCreate(&e0), "event") || !cuda_ok(b, cudaEventCreate(&e1), "event")) return TS_ERR_CUDA;
  const int cands[3] = {64, 128, 256};
  int best = b->pair_threads;
  float best_ms = 1e30f;
  for (int c : cands) {
    b->pair_threads = c;
    pair(b, st, false, false);   // warm
    cudaEventRecord(e0, st);
    for (int k = 0; k < 10; k++) pair(b, st, false, false);
    cudaEventRecord(e1, st);
    if (!cuda_ok(b, cudaEventSynchronize(e1), "event sync")) return TS_ERR_CUDA;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) { best_ms = ms; best = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->pair_threads = best;
  b->graphs_valid = false;
  if (!b->cache_path.empty()) {
    FILE* f = fopen(b->cache_path.c_str(), "a");
    if (f) { fprintf(f, "%s %d\n", key.c_str(), best); fclose(f); }
  }
  return cuda_ok(b, cudaGetLastError(), "ts_autotune") ? TS_OK : TS_ERR_CUDA;
}
