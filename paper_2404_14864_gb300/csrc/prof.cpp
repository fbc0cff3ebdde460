// Kernel-class timing with CUDA events (kfbi_profile_*).  Each timed launch
// records an event pair on its stream; reading synchronises and sums them.
#include <cstdlib>
#include <mutex>
#include <vector>

#include "internal.h"

namespace kfbi {

bool g_prof_on = false;
bool g_pdl = [] {
  const char* e = std::getenv("KFBI_PDL");
  return !(e && e[0] == '0');
}();

void throw_launch_error(cudaError_t e) { throw CudaError{e, "kernel launch"}; }
unsigned g_prof_mask = 0;

namespace {
struct Rec {
  int cls;
  cudaEvent_t a, b;
  double work;   // floating-point operations the launch issues (0 if not counted)
  double bytes;  // algorithmic bytes the launch moves (0 if not counted)
};
std::mutex mu;
std::vector<Rec> recs;
std::vector<cudaEvent_t> pool;

cudaEvent_t take() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

void* prof_begin(int cls, cudaStream_t st) {
  if (!((g_prof_mask >> cls) & 1u)) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  Rec r{cls, take(), take(), 0.0, 0.0};
  if (!r.a || !r.b) return nullptr;
  cudaEventRecord(r.a, st);
  recs.push_back(r);
  return (void*)(recs.size());
}

void prof_end(void* tok, cudaStream_t st) {
  if (!tok) return;
  std::lock_guard<std::mutex> lk(mu);
  size_t i = (size_t)tok - 1;
  if (i < recs.size()) cudaEventRecord(recs[i].b, st);
}

void prof_add_work(void* tok, double work) {
  if (!tok) return;
  std::lock_guard<std::mutex> lk(mu);
  size_t i = (size_t)tok - 1;
  if (i < recs.size()) recs[i].work += work;
}

void prof_add_bytes(void* tok, double bytes) {
  if (!tok) return;
  std::lock_guard<std::mutex> lk(mu);
  size_t i = (size_t)tok - 1;
  if (i < recs.size()) recs[i].bytes += bytes;
}

}  // namespace kfbi

using namespace kfbi;

extern "C" {

void kfbi_profile_enable(int mask) {
  g_prof_mask = (unsigned)mask;
  g_prof_on = mask != 0;
}

void kfbi_profile_reset(void) {
  std::lock_guard<std::mutex> lk(mu);
  for (auto& r : recs) {
    cudaEventSynchronize(r.b);
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  recs.clear();
}

kfbi_status kfbi_profile_read(int cls, long long* launches, double* total_ms) {
  if (!launches || !total_ms || cls < 0 || cls >= KFBI_PROF_NCLASS) return KFBI_ERR_ARG;
  std::lock_guard<std::mutex> lk(mu);
  long long n = 0;
  double ms = 0.0;
  for (auto& r : recs) {
    if (r.cls != cls) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return KFBI_ERR_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return KFBI_ERR_CUDA;
    ms += t;
    ++n;
  }
  *launches = n;
  *total_ms = ms;
  return KFBI_OK;
}

kfbi_status kfbi_profile_work(int cls, double* flops) {
  if (!flops || cls < 0 || cls >= KFBI_PROF_NCLASS) return KFBI_ERR_ARG;
  std::lock_guard<std::mutex> lk(mu);
  double w = 0.0;
  for (auto& r : recs)
    if (r.cls == cls) w += r.work;
  *flops = w;
  return KFBI_OK;
}

kfbi_status kfbi_profile_bytes(int cls, double* bytes) {
  if (!bytes || cls < 0 || cls >= KFBI_PROF_NCLASS) return KFBI_ERR_ARG;
  std::lock_guard<std::mutex> lk(mu);
  double b = 0.0;
  for (auto& r : recs)
    if (r.cls == cls) b += r.bytes;
  *bytes = b;
  return KFBI_OK;
}

}  // extern "C"
