// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <new>
#include <stdexcept>
#include <memory>
#include <string>
#include <utility>

#include "kfbi.h"
#include "plan.h"

namespace kfbi {

// Count of kernel launches issued by the library (kfbi_launch_count).
extern std::atomic<long long> g_launches;
// Message of the last failure not tied to a domain.
void set_global_error(const std::string& s);

// Optional per-class event timing (prof.cpp).
extern bool g_prof_on;
extern unsigned g_prof_mask;
void* prof_begin(int cls, cudaStream_t st);
void prof_end(void* tok, cudaStream_t st);
void prof_add_work(void* tok, double work);
void prof_add_bytes(void* tok, double bytes);

// Programmatic dependent launch.  Every library kernel is launched with
// programmatic stream serialization (unless KFBI_PDL=0), so it can be
// scheduled while the previous kernel of its stream drains; its first
// statement, KFBI_PDL_ENTRY, waits for that kernel's completion and memory
// before any global access.  Stream order is kept; what overlaps is the
// launch and block scheduling.  No kernel triggers its dependents early:
// blocks of the next kernel launched at the start of the current one sat
// waiting on its SMs and slowed it (a float64 DGEMM pass by a third, the
// FFT passes by a quarter), so the dependents launch as its blocks exit.
// For a kernel not launched as a dependent the wait returns at once.
extern bool g_pdl;
#define KFBI_PDL_ENTRY() asm volatile("griddepcontrol.wait;" ::: "memory")

// Early exit of a kernel of a speculatively queued GMRES iteration: stop
// points at the solver's convergence flag (nonzero once an earlier
// iteration converged or failed); nullptr never stops.  Read after
// KFBI_PDL_ENTRY, so the flag written by the previous kernel is visible.
#define KFBI_STOP_RETURN(stop) \
  do {                         \
    if ((stop) && *(stop) != 0.0) return; \
  } while (0)

// Sets the programmatic-serialization attribute on a launch configuration
// whose attrs array has room for one more entry.
inline void add_pdl_attr(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* at) {
  if (!g_pdl) return;
  at[cfg.numAttrs].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[cfg.numAttrs].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  ++cfg.numAttrs;
}

struct CudaError;
[[noreturn]] void throw_launch_error(cudaError_t e);

// Precisions that run the mixed engine (FP32 correction and extraction,
// FP32 box solves with FP64 refinement).
inline bool is_mixed(int precision) {
  return precision == KFBI_MIXED_TF32 || precision == KFBI_MIXED_FFT32;
}

template <typename... P, typename... A>
inline void launch_kernel(void (*kern)(P...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  add_pdl_attr(cfg, at);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
  if (e != cudaSuccess) throw_launch_error(e);
}

// Launch a kernel of a profiling class, count it and (if enabled) time it.
#define KFBI_LAUNCH_P(cls, kern, grid, block, smem, stream, ...)                       \
  do {                                                                                  \
    void* tok_ = ::kfbi::g_prof_on ? ::kfbi::prof_begin((cls), (stream)) : nullptr;     \
    ::kfbi::launch_kernel(kern, (grid), (block), (smem), (stream), __VA_ARGS__);        \
    if (tok_) ::kfbi::prof_end(tok_, (stream));                                         \
    ::kfbi::g_launches.fetch_add(1, std::memory_order_relaxed);                         \
  } while (0)

// Launch a kernel and count it.
// As KFBI_LAUNCH_P, and the launch's floating-point work (flops) is added to
// its record for kfbi_profile_work.
#define KFBI_LAUNCH_PW(cls, flops, kern, grid, block, smem, stream, ...)               \
  do {                                                                                  \
    void* tok_ = ::kfbi::g_prof_on ? ::kfbi::prof_begin((cls), (stream)) : nullptr;     \
    ::kfbi::launch_kernel(kern, (grid), (block), (smem), (stream), __VA_ARGS__);        \
    if (tok_) {                                                                         \
      ::kfbi::prof_end(tok_, (stream));                                                 \
      ::kfbi::prof_add_work(tok_, (flops));                                             \
    }                                                                                   \
    ::kfbi::g_launches.fetch_add(1, std::memory_order_relaxed);                         \
  } while (0)

#define KFBI_LAUNCH(kern, grid, block, smem, stream, ...)                              \
  do {                                                                                  \
    ::kfbi::launch_kernel(kern, (grid), (block), (smem), (stream), __VA_ARGS__);        \
    ::kfbi::g_launches.fetch_add(1, std::memory_order_relaxed);                         \
  } while (0)

struct CudaError {
  cudaError_t code;
  std::string where;
};

#define KFBI_CUDA(call)                                                                 \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) throw ::kfbi::CudaError{e_, std::string(#call)};              \
  } while (0)

#define KFBI_CHECK_LAUNCH() KFBI_CUDA(cudaGetLastError())

struct Status {
  kfbi_status code;
  std::string msg;
};

// Round to the nearest TF32 value (10 explicit mantissa bits), ties to even.
__host__ __device__ inline float tf32_round(float x) {
#ifdef __CUDA_ARCH__
  uint32_t u = __float_as_uint(x);
#else
  uint32_t u;
  __builtin_memcpy(&u, &x, 4);
#endif
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0xfffu + ((u >> 13) & 1u);
    u &= 0xffffe000u;
  }
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float r;
  __builtin_memcpy(&r, &u, 4);
  return r;
#endif
}

#ifdef __CUDACC__
// FP32 <-> FP64 conversions on the integer and FP32 pipes.  GB300 runs FP64
// conversions on its narrow FP64 pipe (about two operations per clock per
// SM), which bounds the plane kernels of the refinement.  Both functions
// return exactly what the hardware conversions return (round to nearest,
// ties to even); inputs outside the exponent ranges they handle (zeros and
// tiny, huge or non-finite values) take the hardware conversion.

// The hardware split, out of line: inlined, the compiler predicates it into
// the fast path, where it still occupies the FP64 pipe.
static __device__ __noinline__ float2 split_f64_hw(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// float -> double, exact for every finite x (a NaN gives a NaN): the
// exponent rebiased from 127 to 1023, a subnormal normalised by its leading
// zeros, infinities and NaNs mapped to exponent 2047.
__device__ __forceinline__ double f32_to_f64(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  uint32_t de = e + 896u;
  unsigned long long dm = (unsigned long long)m << 29;
  if (e == 0u) {
    // 0 or m 2^-149: the top bit of m at position p = 31 - clz(m) gives
    // exponent p - 149 (biased p + 874), the bits below it the fraction
    const int p = 31 - __clz((int)m);
    de = m ? (uint32_t)(p + 874) : 0u;
    dm = m ? (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull) : 0ull;
  } else if (e == 0xffu) {
    de = 0x7ffu;
  }
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)de << 52) | dm;
  return __longlong_as_double((long long)b);
}

// x = hi + lo + O(2^-48 |x|): hi = (float)x, lo = (float)(x - (double)hi).
// For 949 <= biased exponent <= 1149 (2^-74 <= |x| < 2^127): hi keeps the
// top 24 significand bits, rounded on the 29 bits below them; x - hi is that
// remainder r (|r| <= 2^28) times 2^(e - 1075), converted to FP32 in one
// rounding as two exact 14-bit halves joined by an FMA.
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t w = (uint32_t)(b >> 32);
  const int e = (int)((w >> 20) & 0x7ffu);
  if (e < 949 || e > 1149) {
    if ((b << 1) == 0ull) {  // +-0 (the plane padding)
      hi = __uint_as_float(w);
      lo = 0.f;
      return;
    }
    const float2 v = split_f64_hw(x);
    hi = v.x;
    lo = v.y;
    return;
  }
  const uint32_t s = w & 0x80000000u;
  uint32_t f = s | ((uint32_t)(e - 896) << 23) | (uint32_t)((b >> 29) & 0x7fffffu);
  int r = (int)(b & 0x1fffffffu);
  if (r > 0x10000000 || (r == 0x10000000 && (f & 1u))) {
    f += 1u;  // a carry out of the significand raises the exponent: still exact
    r -= 0x20000000;
  }
  hi = __uint_as_float(f);
  const uint32_t ar = (uint32_t)(r < 0 ? -r : r);
  const float fh = __uint_as_float(0x4b000000u | (ar >> 14)) - 8388608.f;
  const float fl = __uint_as_float(0x4b000000u | (ar & 0x3fffu)) - 8388608.f;
  const float v = fmaf(fh, 16384.f, fl) * __uint_as_float((uint32_t)(e - 948) << 23);
  // sign of x - hi: sign of x, flipped where hi rounded away from zero (an
  // exact split leaves +0, as the hardware subtraction does)
  lo = (ar != 0u && (s != 0) != (r < 0)) ? -v : v;
}

// Complex eigenvalue division of a box solve in FP32:
// (x + i y) scale / (d - i kim) = (x + i y)(d + i kim) scale / (d^2 + kim^2).
__device__ __forceinline__ void eig_div_cplx32(float x, float y, float d, float kim, float scale,
                                               float& zr, float& zi) {
  const float sc = __fdividef(scale, fmaf(d, d, kim * kim));
  zr = (x * d - y * kim) * sc;
  zi = (x * kim + y * d) * sc;
}
#endif

struct TcDst;  // tensor-core DST engine (tc_dst.cu)

// DST-I tables shared by every domain on the same grid (M, h), tables.cu:
// S (Mp x Mp, zero padded) and the eigenvalues in FP64; for mixed domains
// also the TF32 pair of S, an FP32 copy of S and FP32 eigenvalues.
struct DstTables {
  int M = 0, Mp = 0;
  double h = 0;
  double* S = nullptr;
  double* lam = nullptr;
  float* S_hi = nullptr;
  float* S_lo = nullptr;
  float* S32 = nullptr;
  float* lam32 = nullptr;
  long long bytes = 0;
};
std::shared_ptr<DstTables> dst_tables(int M, int Mp, double h, bool mixed);
long long dst_tables_bytes();

}  // namespace kfbi

// Device-resident domain: tables from the plan and work buffers.
struct kfbi_domain {
  kfbi_domain_desc desc{};
  int M = 0, nb = 0, n1 = 0, Mp = 0;  // Mp: padded transform size (multiple of 128)
  double h = 0, lo = 0;
  int device = 0;
  std::string err;
  long long bytes = 0;

  // tables (padded grid offsets row*Mp + col)
  uint8_t* d_mask = nullptr;  // Mp*Mp, 1 = interior node inside Omega
  int n_irr = 0, n_arms = 0;
  int* d_irr_off = nullptr;
  int* d_arm_start = nullptr;
  int* d_arm_k0 = nullptr;
  double* d_arm_alpha = nullptr;  // [m * n_arms + a]
  double* d_arm_beta = nullptr;
  int* d_arm_fidx = nullptr;      // [q * n_arms + a]
  double* d_arm_fcoef = nullptr;
  int* d_node_gidx = nullptr;     // [m * nb + k]
  double* d_node_w = nullptr;
  double* d_node_a = nullptr;
  double* d_node_b = nullptr;
  int* d_node_fidx = nullptr;
  double* d_node_fcoef = nullptr;
  // Neumann tables (float64 domains): psi weights per arm, normal-derivative
  // extraction weights, their psi and f terms
  double* d_arm_delta = nullptr;
  double* d_node_wn = nullptr;
  double* d_node_e = nullptr;
  double* d_node_fcoef_n = nullptr;
  // their FP32 copies on mixed domains, and zero tables standing in for the
  // kappa weights (the psi terms have none)
  float* d_arm_delta32 = nullptr;
  float* d_node_wn32 = nullptr;
  float* d_node_e32 = nullptr;
  float* d_node_fcoef_n32 = nullptr;
  float* d_zero_arm32 = nullptr;
  float* d_zero_node32 = nullptr;
  // set while a Neumann entry point runs: the operator of apply_internal is
  // then psi -> d_n u+ (Phi = 0, Psi = psi) instead of phi -> u+
  bool neumann = false;
  float* d_arm_alpha32 = nullptr;  // FP32 copies for the mixed path
  float* d_arm_beta32 = nullptr;
  float* d_arm_fcoef32 = nullptr;
  float* d_node_w32 = nullptr;
  float* d_node_a32 = nullptr;
  float* d_node_b32 = nullptr;
  float* d_node_fcoef32 = nullptr;
  std::shared_ptr<kfbi::DstTables> tables;  // shared per grid
  double* d_S = nullptr;    // Mp*Mp DST-I matrix, zero padded (borrowed from tables)
  double* d_lam = nullptr;  // Mp eigenvalues, 0 beyond n1 (borrowed from tables)

  // FP64 work buffers, two planes each (complex = re plane, im plane)
  double* d_R = nullptr;
  double* d_T = nullptr;      // float64 domains only
  double* d_U = nullptr;
  double* d_fpad = nullptr;  // caller's f converted to the padded masked layout
  double* d_zero_nb = nullptr;  // 2*nb zeros (phi = 0)
  int rhs_sparse_planes = 0; // planes of d_R known to be zero off the irregular nodes

  // GMRES workspace (complex-interleaved vectors of length nb)
  int restart = 0;
  double* d_V = nullptr;    // (restart+1) * 2nb
  double* d_W = nullptr;    // 2nb
  double* d_X = nullptr;    // 2nb
  double* d_B = nullptr;    // 2nb
  double* d_H = nullptr;    // (restart+1)*restart complex, column-major
  double* d_cs = nullptr;   // restart
  double* d_sn = nullptr;   // restart complex
  double* d_g = nullptr;    // restart+1 complex
  double* d_part = nullptr; // per-CTA partial inner products (2 x (restart+1) x 64 complex)
  double* d_hcol = nullptr; // Hessenberg column being built (restart+1 complex)
  double* d_Rv = nullptr;   // refinement residual (2nb)
  double* d_Dv = nullptr;   // refinement correction (2nb)
  double* d_Ax = nullptr;   // accurate operator output (2nb)
  double* d_scal = nullptr; // device scalars: [0] ||b||, [1] residual estimate, ...
  double* h_scal = nullptr; // pinned mirror
  // GMRES lookahead: pinned snapshots of d_scal (two slots, in stream
  // order) and the events that mark them
  // scalar mailbox: host-mapped memory the GMRES kernels post their scalars
  // to (2 slots of 16 doubles: 8 scalars, then the sequence number), polled
  // by the host instead of a copy in the stream
  double* h_mbox = nullptr;
  double* d_mbox = nullptr;
  long long mbox_seq = 0;
  // residual reduction per Richardson step seen at kappa = (rich_kre,
  // rich_kim) in the last solve (0: none yet); sizes the first run of steps
  double rich_rate = 0.0, rich_kre = 0.0, rich_kim = 0.0;
  cudaEvent_t ev_scal = nullptr;

  kfbi::TcDst* tc = nullptr;  // mixed-precision engine (KFBI_MIXED_TF32 or KFBI_MIXED_FFT32)
};

struct kfbi_state {
  kfbi_domain* dom = nullptr;
  int eq = 0;
  int planes = 1;
  double dt = 0, theta = 0.25, kre = 0, kim = 0;
  bool initialised = false;
  bool phi_zero = true;
  bool neumann = false;  // boundary data are d_n u (Eq. 3.19), the density is psi
  double w = 0.0;        // nonlinear Schroedinger coefficient of batched steps
  double* d_u = nullptr;      // current field, padded planes
  double* d_F = nullptr;      // F^{n+1} (heat, wave) or u* (Schroedinger)
  double* d_Fprev = nullptr;  // F^n (wave)
  double* d_ft = nullptr;     // masked f-tilde of the current solve
  double* d_aux = nullptr;    // u** (Schroedinger)
  double* d_phi = nullptr;    // density, complex interleaved 2nb
  double* d_b = nullptr;      // BIE right-hand side, complex interleaved 2nb
  double* d_ub = nullptr;     // u+ of the volume part
  // mixed domains: superposition caches of the refined solve
  double* d_uf = nullptr;     // grid of the volume part, Y f-tilde (planes x Mp^2)
  double* d_ax = nullptr;     // A phi at the current phi (complex interleaved 2nb)
  bool ax_valid = false;
  // the previous step's density (and, mixed, its A phi) for the linear
  // extrapolation of the initial density in time
  double* d_phi_prev = nullptr;
  double* d_ax_prev = nullptr;
  bool hist = false;           // d_phi_prev holds the previous converged density
  bool ax_prev_valid = false;  // d_ax_prev holds A of it
  long long bytes = 0;
};

namespace kfbi {

// domain.cu
// The operator of the hot path: float64 on a KFBI_FP64 domain, the fast
// TF32x3 tensor-core path on a KFBI_MIXED_TF32 domain.
void apply_internal(kfbi_domain* D, double kre, double kim, const double* phi, int phi_stride,
                    const double* ft, double* out, int out_stride, bool want_grid,
                    cudaStream_t st);
// The operator to FP64-level accuracy (identical to apply_internal on a
// float64 domain; refined box solve on a mixed domain).  Grid left in d_U.
void apply_accurate(kfbi_domain* D, double kre, double kim, const double* phi, int phi_stride,
                    const double* ft, double* out, int out_stride, cudaStream_t st);
void correct_fp64(kfbi_domain* D, double kre, double kim, const double* phi, int ps,
                  const double* ft, cudaStream_t st);
void extract_fp64(kfbi_domain* D, double kre, double kim, const double* phi, int ps,
                  const double* ft, double* out, int os, cudaStream_t st);
// Switches a domain's operator to psi -> d_n u+ (the Neumann BIE of
// Eq. 3.19) for its lifetime when `on`.
struct NeumannScope {
  kfbi_domain* D;
  bool on;
  explicit NeumannScope(kfbi_domain* d, bool o = true) : D(d), on(o) {
    if (on) D->neumann = true;
  }
  ~NeumannScope() {
    if (on) D->neumann = false;
  }
};

// Run f (returning kfbi_status); convert exceptions into a status and keep
// the message on the domain (or globally when D is null).
template <class F>
kfbi_status guarded(kfbi_domain* D, F&& f) {
  std::string msg;
  kfbi_status code;
  try {
    return f();
  } catch (const CudaError& e) {
    msg = e.where + ": " + cudaGetErrorString(e.code);
    code = (e.code == cudaErrorMemoryAllocation) ? KFBI_ERR_OOM : KFBI_ERR_CUDA;
  } catch (const Status& s) {
    msg = s.msg;
    code = s.code;
  } catch (const std::bad_alloc&) {
    msg = "host allocation failed";
    code = KFBI_ERR_OOM;
  } catch (const std::exception& e) {
    msg = e.what();
    code = KFBI_ERR_ARG;
  }
  if (D)
    D->err = msg;
  else
    set_global_error(msg);
  return code;
}

// Kernels of the float64 box solve (domain.cu), also launched by the
// allocation-free variant (noalloc.cu).
__global__ void k_dgemm_t(const double* __restrict__ A, const double* __restrict__ S,
                          double* __restrict__ out, int Mp);
__global__ void k_eigscale(double* __restrict__ T, size_t plane, int Mp, int n1,
                           const double* __restrict__ lam, double kre, double kim, double scale,
                           int cplx);

// Caller layout <-> padded planes (domain.cu).
void pad_mask(kfbi_domain* D, const double* src, double* dst, bool C, cudaStream_t st);
void unpad(kfbi_domain* D, const double* src, double* dst, bool C, cudaStream_t st);
int grid_for(size_t n, int block);

// gmres.cu
// GMRES for A x = b (refined on a mixed domain).  ax0 (optional, mixed
// only): A x for the incoming x, reused for the first residual instead of an
// application.  ax_out (optional): receives A x at the returned x when the
// last residual was a fresh accurate application at it; *grid_wx is then
// true and D->d_U holds that application's grid, W x (no volume source).
kfbi_status gmres_solve(kfbi_domain* D, double kre, double kim, const double* b, double* x,
                        bool x_zero, kfbi_solve_info* info, cudaStream_t st,
                        const double* ax0 = nullptr, double* ax_out = nullptr,
                        bool* grid_wx = nullptr);
void gmres_alloc(kfbi_domain* D);
// Throws KFBI_ERR_TIMEOUT if a device kernel recorded a failed bounded wait
// (flags read back into h_scal by the last scalar read).
void check_device_flags(kfbi_domain* D);
void gmres_free(kfbi_domain* D);

// tc_dst.cu (mixed path)
TcDst* tc_create(kfbi_domain* D, const Plan& P);
void tc_destroy(TcDst* tc);
void tc_apply(kfbi_domain* D, double kre, double kim, const double* phi, int phi_stride,
              const double* ft, double* out, int out_stride, bool want_grid, cudaStream_t st);
void tc_apply_accurate(kfbi_domain* D, double kre, double kim, const double* phi, int phi_stride,
                       const double* ft, double* out, int out_stride, cudaStream_t st);
// Accurate application at phi = phi_prev + d from the grid of an accurate
// application at phi_prev (in D->d_U, no volume source) and one FP32 box
// solve of the correction d; the result's error is that of a box solve
// without refinement, relative to |A d|.
void tc_apply_correction(kfbi_domain* D, double kre, double kim, const double* d, const double* phi,
                         int phi_stride, double* out, int out_stride, cudaStream_t st);
long long tc_bytes(const TcDst* tc);
// Exact device bytes of what the allocation routines take for a plan: the
// tensor-core buffers, the GMRES workspace, a whole domain (not counting the
// shared DST tables) and one time-level state.
long long tc_bytes_for(const Plan& P, int Mp);
long long gmres_bytes(int m, int nb);
long long domain_bytes_for(const Plan& P);
long long state_bytes_for(int Mp, int nb, int equation, bool mixed);
// A device domain from a built plan (throws Status); kfbi_create_domain
// is build_plan followed by this.
kfbi_domain* domain_from_plan(const Plan& plan, cudaStream_t st);

// batch.cu, for the request server: a batch with no domains, (re)binding
// it to a set of domains (keeps allocations that fit, drops the captured
// graph; the autotuner's choice is kept), and a step whose heat source of
// instance i is src_scale[i] * src[i] (src_scale NULL: 1).
kfbi_batch* batch_new();
void batch_bind(kfbi_batch* B, kfbi_domain* const* domains, int n);
kfbi_status batch_step(kfbi_batch* B, kfbi_state* const* states, const void* const* g_next,
                       const double* const* src_or_v, const double* src_scale,
                       kfbi_solve_info* infos, cudaStream_t st);

}  // namespace kfbi
