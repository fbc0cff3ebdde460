// Allocation-free box solve: kfbi_box_solve_noalloc.
//
// For callers that cannot allocate device memory at all -- code running
// where cudaMalloc is not allowed (inside a CUDA-graph capture owned by
// someone else, under a host allocator that forbids it, or in a plugin
// whose host application owns every device allocation).  It solves the
// five-point modified-Helmholtz system on the box with the same float64
// DST-I passes as the domain path, but its work space is a fixed static
// device array instead of buffers from kfbi_create_domain.  The paper has
// no counterpart to this entry point.
//
// The scratch array is file-scope device memory: every GPU that loads the
// library holds it (about 2.5 MiB) until the process exits.  Host code
// cannot use the array's name as a device address, so the address is
// looked up with cudaGetSymbolAddress the first time a call runs in a
// device's context (so that first call should come before any stream
// capture).  The cached address is keyed on the current CUDA context: after
// cudaDeviceReset, or in another context on the same device, the module is
// loaded again, the array may sit elsewhere, and the next call looks the
// address up again.  All calls share the one array and it keeps the last call's
// contents; every region the solve reads is rewritten by each call, and
// calls that overlap on the GPU (two streams at once) race on it.
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "internal.h"

namespace kfbi {
namespace na {

constexpr int kMaxMp = 256;  // largest padded transform size: M - 1 <= 256
constexpr size_t kPlane = (size_t)kMaxMp * kMaxMp;
// S (1 plane) + eigenvalues (kMaxMp) + two work buffers of two planes each
constexpr size_t kScratchDoubles = kPlane + kMaxMp + 4 * kPlane;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
static std::mutex g_mu;
// per device: the context the address was looked up in, and the address
static CUcontext g_ctx[kMaxDevices] = {nullptr};
static double* g_addr[kMaxDevices] = {nullptr};

// S[a][i] = sin(pi a i / M) (a*i reduced mod 2M), zero padded; lambda_a.
__global__ void k_na_tables(double* S, double* lam, int M, int Mp, double h) {
  KFBI_PDL_ENTRY();
  const size_t plane = (size_t)Mp * Mp;
  const double pi = 3.14159265358979323846264338327950288;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < plane;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / Mp), i = (int)(idx % Mp);
    double v = 0.0;
    if (a < M - 1 && i < M - 1) {
      const long long ai = ((long long)(a + 1) * (i + 1)) % (2LL * M);
      v = sin(pi * (double)ai / (double)M);
    }
    S[idx] = v;
    if (i == 0) {
      double l = 0.0;
      if (a < M - 1) {
        const double s = sin(pi * (double)(a + 1) / (2.0 * M));
        l = -(4.0 / (h * h)) * s * s;
      }
      lam[a] = l;
    }
  }
}

// caller layout (n1 x n1, interleaved if C) -> padded planes, zero padding
__global__ void k_na_pad(const double* src, double* dst, int n1, int Mp, int C) {
  KFBI_PDL_ENTRY();
  const size_t plane = (size_t)Mp * Mp;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < plane;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / Mp), c = (int)(idx % Mp);
    double re = 0.0, im = 0.0;
    if (r < n1 && c < n1) {
      const size_t s = (size_t)r * n1 + c;
      re = C ? src[2 * s] : src[s];
      im = C ? src[2 * s + 1] : 0.0;
    }
    dst[idx] = re;
    if (C) dst[plane + idx] = im;
  }
}

__global__ void k_na_unpad(const double* src, double* dst, int n1, int Mp, int C) {
  KFBI_PDL_ENTRY();
  const size_t plane = (size_t)Mp * Mp;
  const size_t n = (size_t)n1 * n1;
  for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n;
       s += (size_t)gridDim.x * blockDim.x) {
    const size_t p = (s / n1) * Mp + (s % n1);
    if (C) {
      dst[2 * s] = src[p];
      dst[2 * s + 1] = src[plane + p];
    } else {
      dst[s] = src[p];
    }
  }
}

// cuCtxGetCurrent through the runtime's driver entry point (the library
// does not link the driver library directly).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
static CtxGetCurrentFn ctx_get_current() {
  static std::once_flag once;
  static CtxGetCurrentFn fn = nullptr;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)p;
  });
  return fn;
}

// Device address of the scratch array in the current context (looked up on
// the first call in each context of a device).
static double* scratch_address(std::string& err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return nullptr;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    err = "device ordinal out of range";
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  // a context that differs from the cached one means the module (and the
  // array) may have been loaded again; with no context current yet, the
  // runtime lookup below makes the device's primary context current
  CtxGetCurrentFn get = ctx_get_current();
  if (!get) {
    err = "cuCtxGetCurrent is not available";
    return nullptr;
  }
  CUcontext ctx = nullptr;
  if (get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  if (!ctx || !g_addr[dev] || g_ctx[dev] != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return nullptr;
    }
    if (!ctx && (get(&ctx) != CUDA_SUCCESS || !ctx)) {
      err = "no current CUDA context";
      return nullptr;
    }
    g_addr[dev] = (double*)p;
    g_ctx[dev] = ctx;
  }
  return g_addr[dev];
}

}  // namespace na
}  // namespace kfbi

using namespace kfbi;
using namespace kfbi::na;

extern "C" kfbi_status kfbi_box_solve_noalloc(int M, double box_lo, double box_hi,
                                              double kappa_re, double kappa_im,
                                              const void* rhs_dev, void* u_dev, void* stream) {
  if (M < 2 || M - 1 > kMaxMp) {
    set_global_error("kfbi_box_solve_noalloc: M must satisfy 2 <= M <= 257 (the static "
                     "scratch holds transforms up to 256 x 256)");
    return KFBI_ERR_ARG;
  }
  if (!(box_hi > box_lo) || !rhs_dev || !u_dev) {
    set_global_error("kfbi_box_solve_noalloc: need box_lo < box_hi and device pointers");
    return KFBI_ERR_ARG;
  }
  std::string err;
  double* base = scratch_address(err);
  if (!base) {
    set_global_error("kfbi_box_solve_noalloc: " + err);
    return KFBI_ERR_CUDA;
  }
  return guarded(nullptr, [&]() -> kfbi_status {
    cudaStream_t st = (cudaStream_t)stream;
    const int n1 = M - 1;
    const int Mp = ((n1 + 127) / 128) * 128;
    const size_t plane = (size_t)Mp * Mp;
    const int C = kappa_im != 0.0 ? 1 : 0;
    const double h = (box_hi - box_lo) / M;
    double* S = base;
    double* lam = S + plane;
    double* A = lam + Mp;
    double* B = A + 2 * plane;
    KFBI_LAUNCH(k_na_tables, grid_for(plane, 256), 256, 0, st, S, lam, M, Mp, h);
    KFBI_LAUNCH(k_na_pad, grid_for(plane, 256), 256, 0, st, (const double*)rhs_dev, A, n1, Mp, C);
    dim3 gg(Mp / 64, Mp / 64, C ? 2 : 1);
    KFBI_LAUNCH(k_dgemm_t, gg, 256, 0, st, A, S, B, Mp);
    KFBI_LAUNCH(k_dgemm_t, gg, 256, 0, st, B, S, A, Mp);
    KFBI_LAUNCH(k_eigscale, grid_for(plane, 256), 256, 0, st, A, plane, Mp, n1, lam, kappa_re,
                kappa_im, (2.0 / M) * (2.0 / M), C);
    KFBI_LAUNCH(k_dgemm_t, gg, 256, 0, st, A, S, B, Mp);
    KFBI_LAUNCH(k_dgemm_t, gg, 256, 0, st, B, S, A, Mp);
    KFBI_LAUNCH(k_na_unpad, grid_for((size_t)n1 * n1, 256), 256, 0, st, A, (double*)u_dev, n1, Mp,
                C);
    KFBI_CHECK_LAUNCH();
    return KFBI_OK;
  });
}
