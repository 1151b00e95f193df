// Host-side store of the per-launch timing records (see profile.cuh).
#include <mutex>
#include <vector>

#include "profile.cuh"
#include "radsplat.h"

namespace rs {
namespace prof {

struct Record {
  const char* name;
  cudaEvent_t start, stop;
};

static std::mutex g_mu;
static bool g_on = false;
static std::vector<Record> g_records;
static std::vector<cudaEvent_t> g_pool;
static size_t g_open = (size_t)-1;

static cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

bool enabled() { return g_on; }

static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return true;
  return cs != cudaStreamCaptureStatusNone;
}

void begin(const char* name, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || capturing(s)) return;
  Record r{name, take_event(), take_event()};
  cudaEventRecord(r.start, s);
  g_records.push_back(r);
  g_open = g_records.size() - 1;
}

void end(cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_open == (size_t)-1 || g_open >= g_records.size()) return;
  cudaEventRecord(g_records[g_open].stop, s);
  g_open = (size_t)-1;
}

static void clear_locked() {
  for (auto& r : g_records) {
    g_pool.push_back(r.start);
    g_pool.push_back(r.stop);
  }
  g_records.clear();
  g_open = (size_t)-1;
}

}  // namespace prof
}  // namespace rs

using namespace rs::prof;

extern "C" rs_status rs_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_mu);
  clear_locked();
  g_on = on != 0;
  return RS_OK;
}

extern "C" int32_t rs_profile_count(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  return (int32_t)g_records.size();
}

extern "C" rs_status rs_profile_read(int32_t i, const char** name, float* ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (i < 0 || (size_t)i >= g_records.size() || !name || !ms) return RS_ERR_INVALID_ARG;
  const Record& r = g_records[(size_t)i];
  *name = r.name;
  if (cudaEventSynchronize(r.stop) != cudaSuccess) return RS_ERR_CUDA;
  return cudaEventElapsedTime(ms, r.start, r.stop) == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}
