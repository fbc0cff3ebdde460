// Shared DST-I tables.  The matrix S[a][i] = sin(pi a i / M) of the box
// solve's sine transform and the eigenvalues lambda_a = -(4/h^2)
// sin^2(pi a / 2M) of the 1-D second difference (Sec. 3.2.6; fast Cartesian
// solve of the interface problem, Eq. 3.30) depend only on the grid, so
// every domain on the same grid (M, h) borrows one device copy.  A mixed
// domain also needs the TF32 pair (hi = tf32(S), lo = tf32(S - hi)), an
// FP32 copy of S for the CUDA-core sparse passes and FP32 eigenvalues;
// these are added the first time a mixed domain asks for them.
#include "internal.h"

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

namespace kfbi {

namespace {

std::mutex g_tab_mu;
std::map<std::pair<int, uint64_t>, std::weak_ptr<DstTables>> g_tabs;
long long g_tab_bytes = 0;  // device bytes of live tables (under g_tab_mu)

void free_tables(DstTables* t) {
  void* ptrs[] = {t->S, t->lam, t->S_hi, t->S_lo, t->S32, t->lam32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    g_tab_bytes -= t->bytes;
  }
  delete t;
}

template <class T>
T* upload(DstTables* t, const std::vector<T>& v) {
  T* p = nullptr;
  KFBI_CUDA(cudaMalloc(&p, v.size() * sizeof(T)));
  t->bytes += (long long)(v.size() * sizeof(T));
  KFBI_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return p;
}

// S zero padded to Mp x Mp, with a*i reduced mod 2M before the sine so the
// argument stays in [0, 2 pi).
std::vector<double> host_S(int M, int Mp) {
  const int n1 = M - 1;
  const double pi = 3.14159265358979323846264338327950288;
  std::vector<double> S((size_t)Mp * Mp, 0.0);
  for (int a = 1; a <= n1; ++a)
    for (int i = 1; i <= n1; ++i) {
      const long long ai = ((long long)a * i) % (2LL * M);
      S[(size_t)(a - 1) * Mp + (i - 1)] = std::sin(pi * (double)ai / (double)M);
    }
  return S;
}

}  // namespace

std::shared_ptr<DstTables> dst_tables(int M, int Mp, double h, bool mixed) {
  std::lock_guard<std::mutex> lk(g_tab_mu);
  uint64_t hb = 0;
  std::memcpy(&hb, &h, sizeof(hb));
  std::weak_ptr<DstTables>& slot = g_tabs[std::make_pair(M, hb)];
  std::shared_ptr<DstTables> t = slot.lock();
  std::vector<double> S;
  if (!t) {
    DstTables* raw = new DstTables();
    raw->M = M;
    raw->Mp = Mp;
    raw->h = h;
    t = std::shared_ptr<DstTables>(raw, free_tables);
    S = host_S(M, Mp);
    std::vector<double> lam(Mp, 0.0);
    const double pi = 3.14159265358979323846264338327950288;
    for (int a = 1; a <= M - 1; ++a) {
      const double s = std::sin(pi * (double)a / (2.0 * M));
      lam[a - 1] = -(4.0 / (h * h)) * s * s;
    }
    const long long before = t->bytes;
    t->S = upload(raw, S);
    t->lam = upload(raw, lam);
    g_tab_bytes += t->bytes - before;
    slot = t;
  }
  if (mixed && !t->S_hi) {
    if (S.empty()) S = host_S(M, Mp);
    const size_t plane = (size_t)Mp * Mp;
    std::vector<float> sh(plane), sl(plane), s32(plane), l32(Mp);
    for (size_t q = 0; q < plane; ++q) {
      sh[q] = tf32_round((float)S[q]);
      sl[q] = tf32_round((float)(S[q] - (double)sh[q]));
      s32[q] = (float)S[q];
    }
    std::vector<double> lam(Mp);
    KFBI_CUDA(cudaMemcpy(lam.data(), t->lam, Mp * sizeof(double), cudaMemcpyDeviceToHost));
    for (int q = 0; q < Mp; ++q) l32[q] = (float)lam[q];
    const long long before = t->bytes;
    t->S_hi = upload(t.get(), sh);
    t->S_lo = upload(t.get(), sl);
    t->S32 = upload(t.get(), s32);
    t->lam32 = upload(t.get(), l32);
    g_tab_bytes += t->bytes - before;
  }
  return t;
}

long long dst_tables_bytes() {
  std::lock_guard<std::mutex> lk(g_tab_mu);
  return g_tab_bytes;
}

}  // namespace kfbi

extern "C" long long kfbi_table_cache_bytes(void) { return kfbi::dst_tables_bytes(); }
