// Runtime autotuner for the split-precision step.
//
// For every tunable kernel a handful of variants is timed at setup on the handle's own
// buffers (CUDA events, median of 3 after one warm launch), and the fastest is kept.
// Choices are keyed by the kernel and the problem shape and can be persisted in a small
// JSON object file so that later setups of the same shape skip the timing.
#include <algorithm>
#include <cstdio>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"

namespace afq {
namespace {

std::mutex g_tune_mu;

std::string key_of(const Ctx& c, const char* kernel) {
  std::ostringstream k;
  k << kernel << ":M" << c.M << "X" << c.X << "u" << c.n_up << "d" << c.n_dn << "w" << c.Nw;
  return k.str();
}

// minimal flat JSON object {"key": int, ...}
std::map<std::string, int> load(const char* path) {
  std::map<std::string, int> m;
  if (!path) return m;
  std::ifstream f(path);
  if (!f) return m;
  std::string s((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
  size_t i = 0;
  while ((i = s.find('"', i)) != std::string::npos) {
    const size_t j = s.find('"', i + 1);
    if (j == std::string::npos) break;
    const std::string key = s.substr(i + 1, j - i - 1);
    const size_t colon = s.find(':', j);
    if (colon == std::string::npos) break;
    m[key] = std::atoi(s.c_str() + colon + 1);
    i = s.find_first_of(",}", colon);
    if (i == std::string::npos) break;
  }
  return m;
}

void save(const char* path, const std::map<std::string, int>& m) {
  if (!path) return;
  std::ofstream f(path);
  if (!f) return;
  f << "{";
  bool first = true;
  for (const auto& kv : m) {
    f << (first ? "" : ",") << "\n  \"" << kv.first << "\": " << kv.second;
    first = false;
  }
  f << "\n}\n";
}

// Median of three timed launches after a warm one; a variant whose first timed launch takes
// more than twice the best median so far cannot win and is not timed further.
template <class F>
float time_variant(F launch, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float best) {
  if (launch() != cudaSuccess) return 1e30f;
  std::vector<float> t;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0, s);
    if (launch() != cudaSuccess) return 1e30f;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r == 0 && ms > 2.f * best) return ms;
    t.push_back(ms);
  }
  std::sort(t.begin(), t.end());
  return t[1];
}

}  // namespace

cudaError_t autotune_mixed(Ctx& c, const char* cache_path, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto cache = load(cache_path);
  const std::string ke = key_of(c, "energy_v2"), kt = key_of(c, "propagate_v3"),
                    km = key_of(c, "orthonormalise_v1");
  bool dirty = false;
  cudaEvent_t e0, e1;
  cudaError_t err = cudaEventCreate(&e0);
  if (err != cudaSuccess) return err;
  err = cudaEventCreate(&e1);
  if (err != cudaSuccess) {
    cudaEventDestroy(e0);
    return err;
  }
  if (cache.count(ke) && (cache[ke] == 0 ? c.etc != nullptr : energy_variant_ok(c, cache[ke]))) {
    c.tune_energy_wb = cache[ke];
  } else {
    float best = 1e30f;
    for (int wb : {0, 2, 4, 8}) {   // 0: tensor-core kernel
      if (wb == 0 ? c.etc == nullptr : !energy_variant_ok(c, wb)) continue;
      const float t = time_variant(
          [&]() {
            return wb == 0 ? launch_energy_tc(c, s) : launch_energy_tiled(c, c.theta32, c.LtT, s, -1, wb);
          },
          s, e0, e1, best);
      if (t < best) { best = t; c.tune_energy_wb = wb; }
    }
    cache[ke] = c.tune_energy_wb;
    dirty = true;
  }
  if (cache.count(kt) && taylor_variant_ok(c, cache[kt])) {
    c.tune_taylor_smem = cache[kt];
  } else {
    float best = 1e30f;
    // the whole one-body + Taylor propagation: tensor-core (3, 4) or fused FP32 kernel (2), or
    // GEMM, Taylor (1, 0), GEMM;
    // every variant writes only scratch (phi32, the FP64 theta buffer)
    for (int v : {3, 4, 2, 1, 0}) {
      if (!taylor_variant_ok(c, v)) continue;
      const float t = time_variant([&]() { return launch_propagation(c, v, c.theta, c.phi32, s); },
                                   s, e0, e1, best);
      if (t < best) { best = t; c.tune_taylor_smem = v; }
    }
    cache[kt] = c.tune_taylor_smem;
    dirty = true;
  }
  if (cache.count(km) && (cache[km] == 0 || mgs_chol_ok(c))) {
    c.tune_mgs = cache[km];
  } else {
    // Cholesky QR (1) against the Gram-Schmidt kernels (0), on walkers that are orthonormal
    // already (the trial at setup), so the timing changes them only by rounding; log O is not
    // touched
    float best = 1e30f;
    for (int v : {1, 0}) {
      if (v == 1 && !mgs_chol_ok(c)) continue;
      c.tune_mgs = v;
      const float t = time_variant([&]() { return launch_mgs_warp(c, s, false); }, s, e0, e1, best);
      if (t < best) { best = t; cache[km] = v; }
    }
    c.tune_mgs = cache[km];
    dirty = true;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (dirty) save(cache_path, cache);
  return cudaGetLastError();
}

}  // namespace afq
