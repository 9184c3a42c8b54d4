// Autotuner of the batched persistent trace (host code): times candidate
// launch configurations on the caller's batch and caches the winner.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"

namespace sd {
namespace {

std::string tune_key(int n_req, long long total_elems, const sd_trace_opts* o, int n_lenses) {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return std::string();
  std::string name(prop.name);
  std::replace(name.begin(), name.end(), ' ', '_');
  std::ostringstream k;
  k << name << "|sm" << prop.multiProcessorCount << "|req" << n_req << "|elems" << total_elems
    << "|ks" << o->max_ks << "|n" << o->max_n_grid << "|lens" << n_lenses << "|norm" << o->norm
    << "|dt" << o->out_dtype;
  return k.str();
}

bool cache_lookup(const char* path, const std::string& key, sd_batch_config* c) {
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string k;
    sd_batch_config v{};
    if (is >> k >> v.threads >> v.rays_per_item >> v.blocks_per_sm && k == key) {
      *c = v;  // the last entry for a key wins
      found = true;
    }
  }
  return found;
}

void cache_store(const char* path, const std::string& key, const sd_batch_config& c, float ms) {
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << " " << c.threads << " " << c.rays_per_item << " " << c.blocks_per_sm << " " << ms
    << "\n";
}

}  // namespace
}  // namespace sd

extern "C" sd_status sd_dp_psf_trace_batched_tune(
    const sd_lens* const* lenses, int n_lenses, const sd_dp_sensor* sensor,
    const sd_psf_request* req, int n_req, const sd_trace_opts* opts, void* out,
    long long total_elems, int64_t* stats, void* workspace, size_t workspace_bytes,
    void* stream, const char* cache_path, sd_batch_config* best) {
  SD_API_RANGE("sd_dp_psf_trace_batched_tune");
  using namespace sd;
  if (!opts || !best) return SD_ERR_ARG;
  const std::string key = tune_key(n_req, total_elems, opts, n_lenses);
  if (!key.empty() && cache_lookup(cache_path, key, best)) return SD_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int max_n = opts->max_n_grid > 0 ? opts->max_n_grid : 512;
  size_t smem = (((size_t)(2 * max_n + 1) * 4) + 15 & ~(size_t)15) +
                (size_t)2 * opts->max_ks * opts->max_ks * 4;
  const int threads_c[] = {256, 512, 1024};
  const int rays_c[] = {4096, 8192, 16384, 32768, 65536};
  cudaEvent_t e0, e1;
  SD_CUDA_TRY(cudaEventCreate(&e0));
  SD_CUDA_TRY(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  sd_batch_config bc{};
  sd_status st = SD_OK;
  for (int bps = 1; bps <= 2 && st == SD_OK; ++bps) {
    if (smem * bps > 227 * 1024) break;
    for (int t : threads_c) {
      if (t * bps > 2048) continue;
      for (int rays : rays_c) {
        sd_batch_config c{t, rays, bps, 0};
        st = sd_dp_psf_trace_batched(lenses, n_lenses, sensor, req, n_req, opts, &c, out,
                                     total_elems, stats, workspace, workspace_bytes, stream);
        if (st != SD_OK) break;
        float times[3];
        for (int rep = 0; rep < 3 && st == SD_OK; ++rep) {
          cudaEventRecord(e0, s);
          st = sd_dp_psf_trace_batched(lenses, n_lenses, sensor, req, n_req, opts, &c, out,
                                       total_elems, stats, workspace, workspace_bytes, stream);
          cudaEventRecord(e1, s);
          if (cudaEventSynchronize(e1) != cudaSuccess) st = SD_ERR_CUDA;
          cudaEventElapsedTime(&times[rep], e0, e1);
        }
        if (st != SD_OK) break;
        std::sort(times, times + 3);
        if (times[1] < best_ms) {
          best_ms = times[1];
          bc = c;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SD_OK) return st;
  *best = bc;
  if (!key.empty()) cache_store(cache_path, key, bc, best_ms);
  return SD_OK;
}
