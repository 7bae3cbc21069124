// Autotuner: picks a plan's kernel variant (block size / TMA-fed pipeline
// for single-edge plans; one mixed-edge launch or one launch per edge for
// mixed plans) by timing the candidates on the device, and remembers the
// choice in a JSON file keyed by device name, SM count and problem.
//
// The selection and cache logic (fft3d_tune_select) takes the timer as a
// callback, so it can be exercised without a GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "fft3d.h"
#include "internal.h"

namespace fft3d {
namespace {

std::mutex g_tune_mu;

std::string sanitize(const std::string& s) {
  std::string o = s;
  for (char& c : o)
    if (c == '"' || c == '\\' || (unsigned char)c < 32) c = '_';
  return o;
}

// {"key": int, ...}; anything unreadable is skipped.
std::map<std::string, int> read_cache(const char* path) {
  std::map<std::string, int> m;
  if (!path || !*path) return m;
  std::ifstream f(path);
  if (!f) return m;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string t = ss.str();
  size_t i = 0;
  while ((i = t.find('"', i)) != std::string::npos) {
    const size_t j = t.find('"', i + 1);
    if (j == std::string::npos) break;
    const std::string key = t.substr(i + 1, j - i - 1);
    size_t k = t.find_first_not_of(" \t\r\n", j + 1);
    if (k == std::string::npos || t[k] != ':') {
      i = j + 1;
      continue;
    }
    k = t.find_first_not_of(" \t\r\n", k + 1);
    if (k == std::string::npos) break;
    char* end = nullptr;
    const long v = std::strtol(t.c_str() + k, &end, 10);
    if (end != t.c_str() + k && v >= 0 && v < 1000) m[key] = (int)v;
    i = (end && end > t.c_str() + k) ? (size_t)(end - t.c_str()) : j + 1;
  }
  return m;
}

int write_cache(const char* path, const std::map<std::string, int>& m) {
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream f(tmp, std::ios::trunc);
    if (!f) return FFT3D_ERR_INVALID_ARG;
    f << "{\n";
    size_t i = 0;
    for (const auto& kv : m)
      f << "  \"" << sanitize(kv.first) << "\": " << kv.second << (++i < m.size() ? ",\n" : "\n");
    f << "}\n";
    if (!f) return FFT3D_ERR_INVALID_ARG;
  }
  if (std::rename(tmp.c_str(), path) != 0) return FFT3D_ERR_INVALID_ARG;
  return FFT3D_SUCCESS;
}

std::string device_tag() {
  int dev = 0;
  cudaDeviceProp prop{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return "nodevice";
  }
  return sanitize(prop.name) + "|sm" + std::to_string(prop.multiProcessorCount);
}

// FNV-1a of the edge list of a mixed plan.
unsigned long long dims_hash(const int* dims, int count) {
  unsigned long long h = 1469598103934665603ull;
  for (int i = 0; i < count; ++i) {
    h ^= (unsigned long long)(unsigned)dims[i];
    h *= 1099511628211ull;
  }
  return h;
}

std::string problem_key(bool mixed, int n, int batch, int precision, int direction,
                        const int* dims, int count) {
  std::string k = device_tag() + "|";
  if (mixed) {
    char buf[64];
    std::snprintf(buf, sizeof(buf), "%016llx", dims_hash(dims, count));
    k += "mixed|c" + std::to_string(count) + "|h" + buf;
  } else {
    k += "n" + std::to_string(n) + "|b" + std::to_string(batch) + "|p" + std::to_string(precision);
  }
  return k + "|d" + std::to_string(direction);
}

struct TimerCtx {
  bool mixed;
  int n, batch, precision, direction;
  const int* dims;
  int count;
  void* in;
  void* out;
};

// Milliseconds per execute of a plan with the given variant (5 timed after
// 2 warm-up), or -1 when the variant cannot be planned or run.
double cuda_timer(int variant, void* vctx) {
  TimerCtx* c = static_cast<TimerCtx*>(vctx);
  fft3d_plan p = nullptr;
  if (fft3d_internal_create_variant(c->mixed, c->n, c->batch, c->precision, c->direction, c->dims,
                                    c->count, variant, &p) != FFT3D_SUCCESS)
    return -1.0;
  double ms = -1.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    bool ok = true;
    for (int i = 0; i < 2 && ok; ++i) ok = fft3d_execute(p, c->in, c->out, nullptr) == 0;
    cudaEventRecord(e0, nullptr);
    for (int i = 0; i < 5 && ok; ++i) ok = fft3d_execute(p, c->in, c->out, nullptr) == 0;
    cudaEventRecord(e1, nullptr);
    float t = 0.0f;
    if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess &&
        fft3d_get_device_status(p, nullptr) == FFT3D_SUCCESS)
      ms = t / 5.0;
  }
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  fft3d_plan_destroy(p);
  return ms;
}

int run_autotune(bool mixed, int n, int batch, int precision, int direction, const int* dims,
                 int count, const char* cache_path, int* best) {
  long long pts = 0;
  if (mixed)
    for (int g = 0; g < count; ++g) pts += (long long)dims[g] * dims[g] * dims[g];
  else
    pts = (long long)n * n * n * batch;
  void *in = nullptr, *out = nullptr;
  if (cudaMalloc(&in, 8 * (size_t)pts) != cudaSuccess ||
      cudaMalloc(&out, 8 * (size_t)pts) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(in);
    return FFT3D_ERR_ALLOC;
  }
  cudaMemset(in, 0, 8 * (size_t)pts);
  TimerCtx ctx{mixed, n, batch, precision, direction, dims, count, in, out};
  const std::vector<int> cand = variant_candidates(mixed, n, precision);
  const std::string key = problem_key(mixed, n, batch, precision, direction, dims, count);
  int from_cache = 0;
  const int rc = fft3d_tune_select(key.c_str(), (int)cand.size(), cand.data(), &cuda_timer, &ctx,
                                   cache_path, best, &from_cache);
  cudaFree(in);
  cudaFree(out);
  return rc;
}

}  // namespace

int pick_variant(bool mixed, int n, int batch, int precision, int direction, const int* dims,
                 int count) {
  const std::vector<int> cand = variant_candidates(mixed, n, precision);
  auto allowed = [&](int v) { return std::find(cand.begin(), cand.end(), v) != cand.end(); };
  const char* ov = std::getenv(mixed ? "FFT3D_MIXED_VARIANT" : "FFT3D_VARIANT");
  if (ov && *ov) {
    char* end = nullptr;
    const long v = std::strtol(ov, &end, 10);
    if (end && *end == 0 && v >= 0 && v < 100 && allowed((int)v)) return (int)v;
  }
  const char* path = std::getenv("FFT3D_TUNE_CACHE");
  if (path && *path) {
    const std::string key = problem_key(mixed, n, batch, precision, direction, dims, count);
    int v = -1;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      const auto m = read_cache(path);
      const auto it = m.find(key);
      if (it != m.end() && allowed(it->second)) v = it->second;
    }
    if (v >= 0) return v;
    const char* tune = std::getenv("FFT3D_TUNE");
    if (tune && tune[0] == '1' &&
        run_autotune(mixed, n, batch, precision, direction, dims, count, path, &v) ==
            FFT3D_SUCCESS &&
        allowed(v))
      return v;
  }
  return builtin_default_variant(mixed, n, batch, precision);
}

}  // namespace fft3d

using namespace fft3d;

extern "C" {

int fft3d_tune_select(const char* key, int ncand, const int* candidates, fft3d_tune_timer timer,
                      void* ctx, const char* cache_path, int* best_variant, int* from_cache) {
  if (!key || !candidates || !timer || !best_variant) return FFT3D_ERR_NULL_PTR;
  if (ncand < 1 || ncand > 64 || !*key) return FFT3D_ERR_INVALID_ARG;
  if (from_cache) *from_cache = 0;
  const std::string k = sanitize(key);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  std::map<std::string, int> cache = read_cache(cache_path);
  const auto it = cache.find(k);
  if (it != cache.end())
    for (int i = 0; i < ncand; ++i)
      if (candidates[i] == it->second) {
        *best_variant = it->second;
        if (from_cache) *from_cache = 1;
        return FFT3D_SUCCESS;
      }
  int best = -1;
  double best_ms = 0.0;
  for (int i = 0; i < ncand; ++i) {
    const double ms = timer(candidates[i], ctx);
    if (!(ms >= 0.0) || !std::isfinite(ms)) continue;  // failed candidate
    if (best < 0 || ms < best_ms) {
      best = candidates[i];
      best_ms = ms;
    }
  }
  if (best < 0) return FFT3D_ERR_CUDA;
  *best_variant = best;
  if (cache_path && *cache_path) {
    cache[k] = best;
    return write_cache(cache_path, cache);
  }
  return FFT3D_SUCCESS;
}

int fft3d_autotune(int n, int batch, int precision, int direction, const char* cache_path,
                   int* best_variant) {
  if (!best_variant) return FFT3D_ERR_NULL_PTR;
  if (n < 1 || batch < 1) return FFT3D_ERR_INVALID_ARG;
  if (fft3d_size_supported(n) != 1) return FFT3D_ERR_UNSUPPORTED_SIZE;
  if (precision < FFT3D_FP32 || precision > FFT3D_FP8) return FFT3D_ERR_INVALID_ARG;
  if (direction != FFT3D_FORWARD && direction != FFT3D_INVERSE) return FFT3D_ERR_INVALID_ARG;
  return run_autotune(false, n, batch, precision, direction, nullptr, 0, cache_path, best_variant);
}

int fft3d_autotune_mixed(int count, const int* dims, int direction, const char* cache_path,
                         int* best_variant) {
  if (!dims || !best_variant) return FFT3D_ERR_NULL_PTR;
  if (count < 1 || count > FFT3D_MAX_MIXED_GRIDS) return FFT3D_ERR_INVALID_ARG;
  for (int g = 0; g < count; ++g)
    if (fft3d_size_supported(dims[g]) != 1) return FFT3D_ERR_UNSUPPORTED_SIZE;
  if (direction != FFT3D_FORWARD && direction != FFT3D_INVERSE) return FFT3D_ERR_INVALID_ARG;
  return run_autotune(true, 0, count, FFT3D_FP32, direction, dims, count, cache_path, best_variant);
}

}  // extern "C"
