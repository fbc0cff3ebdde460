// Domain setup upload and the float64 operator application (Procedure 2 of
// Sec. 3.3, arXiv 2404.14864) on the GPU.
//
//   (a) k_correct: one thread per irregular node sums its cut arms' jump
//       corrections (decoupled strategy of Sec. 3.4.2: the node owns its
//       arms, no atomics) from the precomputed arm tables;
//   (b) four passes of k_dgemm_t (out = (A S)^T, so two passes give S A S)
//       with k_eigscale between forward and inverse transforms: the box
//       solve of Eq. 3.31 by DST-I and the eigenvalue division;
//   (c) k_extract: one thread per boundary node, Eq. 3.36 with the
//       precomputed extraction weights and jump coefficients.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace kfbi {

std::atomic<long long> g_launches{0};
static std::mutex g_err_mu;
static std::string g_err;

void set_global_error(const std::string& s) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = s;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// Caller layout (n1 x n1, complex interleaved if C) -> padded planes, masked
// to Omega (f-tilde of Eq. 3.25).  Padding is zero.
template <bool C>
__global__ void k_pad_mask(const double* __restrict__ src, const uint8_t* __restrict__ mask,
                           double* __restrict__ dst, int n1, int Mp) {
  KFBI_PDL_ENTRY();
  const size_t plane = (size_t)Mp * Mp;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < plane;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / Mp), c = (int)(idx % Mp);
    double re = 0.0, im = 0.0;
    if (r < n1 && c < n1 && mask[idx]) {
      const size_t s = (size_t)r * n1 + c;
      if (C) {
        re = src[2 * s];
        im = src[2 * s + 1];
      } else {
        re = src[s];
      }
    }
    dst[idx] = re;
    if (C) dst[plane + idx] = im;
  }
}

// Padded planes -> caller layout (complex interleaved if C).
template <bool C>
__global__ void k_unpad(const double* __restrict__ src, double* __restrict__ dst, int n1, int Mp) {
  KFBI_PDL_ENTRY();
  const size_t plane = (size_t)Mp * Mp;
  const size_t n = (size_t)n1 * n1;
  for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n;
       s += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(s / n1), c = (int)(s % n1);
    const size_t p = (size_t)r * Mp + c;
    if (C) {
      dst[2 * s] = src[p];
      dst[2 * s + 1] = src[plane + p];
    } else {
      dst[s] = src[p];
    }
  }
}

// (a) corrected right-hand side at the irregular nodes:
// R(p) = f-tilde(p) + sum over arms of the jump correction (Sec. 3.2.4).
// Arm a contributes sum_m (alpha_m + kappa beta_m) phi[k0+m] + sum_q c_q f[idx_q]
// (weights already carry the sign and 1/h^2).
template <bool C>
__global__ void k_correct(double* __restrict__ R, size_t plane, const double* __restrict__ ft,
                          const int* __restrict__ irr_off, const int* __restrict__ arm_start,
                          const int* __restrict__ arm_k0, const double* __restrict__ alpha,
                          const double* __restrict__ beta, const int* __restrict__ fidx,
                          const double* __restrict__ fcoef, int n_irr, int n_arms, int nb,
                          const double* __restrict__ phi, int ps, double kre, double kim) {
  KFBI_PDL_ENTRY();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_irr) return;
  const int off = irr_off[n];
  double sr = ft ? ft[off] : 0.0;
  double si = (C && ft) ? ft[plane + off] : 0.0;
  const int a1 = arm_start[n + 1];
  for (int a = arm_start[n]; a < a1; ++a) {
    int k = arm_k0[a];
    double ar = 0.0, ai = 0.0, br = 0.0, bi = 0.0;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      const double al = alpha[m * n_arms + a], be = beta ? beta[m * n_arms + a] : 0.0;
      const double pr = phi[(size_t)k * ps];
      ar = fma(al, pr, ar);
      br = fma(be, pr, br);
      if (C) {
        const double pi = phi[(size_t)k * ps + 1];
        ai = fma(al, pi, ai);
        bi = fma(be, pi, bi);
      }
      k = (k + 1 == nb) ? 0 : k + 1;
    }
    sr += ar + kre * br;
    if (C) {
      sr -= kim * bi;
      si += ai + kre * bi + kim * br;
    }
    if (ft) {
      const int f0 = fidx[a], f1 = fidx[n_arms + a];
      const double c0 = fcoef[a], c1 = fcoef[n_arms + a];
      sr += c0 * ft[f0] + c1 * ft[f1];
      if (C) si += c0 * ft[plane + f0] + c1 * ft[plane + f1];
    }
  }
  R[off] = sr;
  if (C) R[plane + off] = si;
}

// (b) one DST-I pass in float64: out[p][c][r] = sum_k A[p][r][k] S[k][c].
// 64x64 output tile per block, 256 threads with 4x4 outputs each; the
// transposed store is coalesced along r.
__global__ void __launch_bounds__(256) k_dgemm_t(const double* __restrict__ A,
                                                 const double* __restrict__ S,
                                                 double* __restrict__ out, int Mp) {
  KFBI_PDL_ENTRY();
  __shared__ double As[16][65];
  __shared__ double Bs[16][64];
  const size_t plane = (size_t)Mp * Mp;
  const double* Ap = A + blockIdx.z * plane;
  double* Op = out + blockIdx.z * plane;
  const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  const int tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < Mp; k0 += 16) {
#pragma unroll
    for (int e = tid; e < 1024; e += 256) {
      const int r = e >> 4, k = e & 15;
      As[k][r] = Ap[(size_t)(r0 + r) * Mp + k0 + k];
      const int kk = e >> 6, c = e & 63;
      Bs[kk][c] = S[(size_t)(k0 + kk) * Mp + c0 + c];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][tr + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) Op[(size_t)(c0 + tc + 16 * j) * Mp + r0 + tr + 16 * i] = acc[i][j];
}

// (b) eigenvalue division of the transformed right-hand side:
// U^_ab = R^_ab * (2/M)^2 / (lambda_a + lambda_b - kappa).
__global__ void k_eigscale(double* __restrict__ T, size_t plane, int Mp, int n1,
                           const double* __restrict__ lam, double kre, double kim, double scale,
                           int cplx) {
  KFBI_PDL_ENTRY();
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < plane;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / Mp), b = (int)(idx % Mp);
    if (a >= n1 || b >= n1) continue;
    const double dr = lam[a] + lam[b] - kre;
    if (!cplx) {
      T[idx] *= scale / dr;
    } else {
      // (x + i y) * scale / (dr - i kim)
      const double den = scale / (dr * dr + kim * kim);
      const double x = T[idx], y = T[plane + idx];
      T[idx] = (x * dr - y * kim) * den;
      T[plane + idx] = (x * kim + y * dr) * den;
    }
  }
}

// (c) u+ at boundary node k (Eq. 3.36): sum_m w_m U(p_m) + jump terms.
template <bool C>
__global__ void k_extract(const double* __restrict__ U, size_t plane, const double* __restrict__ ft,
                          const int* __restrict__ gidx, const double* __restrict__ w,
                          const double* __restrict__ A, const double* __restrict__ B,
                          const int* __restrict__ fidx, const double* __restrict__ fcoef, int nb,
                          const double* __restrict__ phi, int ps, double kre, double kim,
                          double* __restrict__ out, int os) {
  KFBI_PDL_ENTRY();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  double sr = 0.0, si = 0.0;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const int g = gidx[m * nb + k];
    const double wm = w[m * nb + k];
    sr = fma(wm, U[g], sr);
    if (C) si = fma(wm, U[plane + g], si);
  }
  double ar = 0.0, ai = 0.0, br = 0.0, bi = 0.0;
  int kk = k - 2;
  if (kk < 0) kk += nb;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const double a = A[j * nb + k], b = B ? B[j * nb + k] : 0.0;
    const double pr = phi[(size_t)kk * ps];
    ar = fma(a, pr, ar);
    br = fma(b, pr, br);
    if (C) {
      const double pi = phi[(size_t)kk * ps + 1];
      ai = fma(a, pi, ai);
      bi = fma(b, pi, bi);
    }
    kk = (kk + 1 == nb) ? 0 : kk + 1;
  }
  sr += ar + kre * br;
  if (C) {
    sr -= kim * bi;
    si += ai + kre * bi + kim * br;
  }
  if (ft) {
    const int g = fidx[k];
    const double c = fcoef[k];
    sr += c * ft[g];
    if (C) si += c * ft[plane + g];
  }
  out[(size_t)k * os] = sr;
  if (C)
    out[(size_t)k * os + 1] = si;
  else if (os == 2)
    out[(size_t)k * os + 1] = 0.0;
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------

int grid_for(size_t n, int block) {
  size_t g = (n + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

template <class T>
static T* dev_upload(kfbi_domain* D, const std::vector<T>& v) {
  T* p = nullptr;
  const size_t bytes = std::max<size_t>(1, v.size()) * sizeof(T);
  KFBI_CUDA(cudaMalloc(&p, bytes));
  D->bytes += (long long)bytes;
  if (!v.empty()) KFBI_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return p;
}

template <class T>
static T* dev_alloc(kfbi_domain* D, size_t n) {
  T* p = nullptr;
  KFBI_CUDA(cudaMalloc(&p, std::max<size_t>(1, n) * sizeof(T)));
  D->bytes += (long long)(std::max<size_t>(1, n) * sizeof(T));
  return p;
}

static void free_domain(kfbi_domain* D) {
  if (!D) return;
  if (D->tc) tc_destroy(D->tc);
  gmres_free(D);
  void* ptrs[] = {D->d_mask, D->d_irr_off, D->d_arm_start, D->d_arm_k0, D->d_arm_alpha,
                  D->d_arm_beta, D->d_arm_fidx, D->d_arm_fcoef, D->d_node_gidx, D->d_node_w,
                  D->d_node_a, D->d_node_b, D->d_node_fidx, D->d_node_fcoef, D->d_arm_alpha32,
                  D->d_arm_beta32, D->d_arm_fcoef32, D->d_node_w32, D->d_node_a32,
                  D->d_node_b32, D->d_node_fcoef32, D->d_R, D->d_T, D->d_U,
                  D->d_fpad, D->d_zero_nb, D->d_arm_delta, D->d_node_wn, D->d_node_e,
                  D->d_node_fcoef_n, D->d_arm_delta32, D->d_node_wn32, D->d_node_e32,
                  D->d_node_fcoef_n32, D->d_zero_arm32, D->d_zero_node32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete D;
}

static std::vector<int> to_padded(const std::vector<int>& idx, int n1, int Mp) {
  std::vector<int> o(idx.size());
  for (size_t q = 0; q < idx.size(); ++q) o[q] = (idx[q] / n1) * Mp + (idx[q] % n1);
  return o;
}

// [rows][cols] host table -> [cols][rows] device layout (SoA per column).
template <class T>
static std::vector<T> transpose(const std::vector<T>& v, int rows, int cols) {
  std::vector<T> o(v.size());
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) o[(size_t)c * rows + r] = v[(size_t)r * cols + c];
  return o;
}

static std::vector<float> to_f32(const std::vector<double>& v) {
  std::vector<float> o(v.size());
  for (size_t q = 0; q < v.size(); ++q) o[q] = (float)v[q];
  return o;
}

static void upload_domain(kfbi_domain* D, const Plan& P) {
  const int n1 = D->n1, Mp = D->Mp, nb = D->nb, M = D->M;
  const size_t plane = (size_t)Mp * Mp;
  std::vector<uint8_t> mask(plane, 0);
  for (int j = 1; j < M; ++j)
    for (int i = 1; i < M; ++i) mask[(size_t)(j - 1) * Mp + (i - 1)] = P.in(i, j) ? 1 : 0;
  D->d_mask = dev_upload(D, mask);
  D->n_irr = P.n_irr();
  D->n_arms = P.n_arms();
  const int na = D->n_arms;
  D->d_irr_off = dev_upload(D, to_padded(P.irr, n1, Mp));
  D->d_arm_start = dev_upload(D, P.arm_start);
  D->d_arm_k0 = dev_upload(D, P.arm_k0);
  std::vector<double> alpha = transpose(P.arm_alpha, na, 6), beta = transpose(P.arm_beta, na, 6);
  std::vector<double> fcoef = transpose(P.arm_fcoef, na, 2);
  D->d_arm_alpha = dev_upload(D, alpha);
  D->d_arm_beta = dev_upload(D, beta);
  D->d_arm_fidx = dev_upload(D, transpose(to_padded(P.arm_fidx, n1, Mp), na, 2));
  D->d_arm_fcoef = dev_upload(D, fcoef);
  std::vector<double> nw = transpose(P.node_w, nb, 6), na_ = transpose(P.node_a, nb, 6),
                      nb_ = transpose(P.node_b, nb, 6);
  D->d_node_gidx = dev_upload(D, transpose(to_padded(P.node_gidx, n1, Mp), nb, 6));
  D->d_node_w = dev_upload(D, nw);
  D->d_node_a = dev_upload(D, na_);
  D->d_node_b = dev_upload(D, nb_);
  D->d_node_fidx = dev_upload(D, to_padded(P.node_fidx, n1, Mp));
  D->d_node_fcoef = dev_upload(D, P.node_fcoef);
  // Neumann tables (the refined applications of mixed domains use the FP64
  // ones too)
  std::vector<double> delta = transpose(P.arm_delta, na, 6), nwn = transpose(P.node_wn, nb, 6),
                      ne = transpose(P.node_e, nb, 6);
  D->d_arm_delta = dev_upload(D, delta);
  D->d_node_wn = dev_upload(D, nwn);
  D->d_node_e = dev_upload(D, ne);
  D->d_node_fcoef_n = dev_upload(D, P.node_fcoef_n);
  if (is_mixed(D->desc.precision)) {
    D->d_arm_delta32 = dev_upload(D, to_f32(delta));
    D->d_node_wn32 = dev_upload(D, to_f32(nwn));
    D->d_node_e32 = dev_upload(D, to_f32(ne));
    D->d_node_fcoef_n32 = dev_upload(D, to_f32(P.node_fcoef_n));
    D->d_zero_arm32 = dev_upload(D, std::vector<float>(delta.size(), 0.f));
    D->d_zero_node32 = dev_upload(D, std::vector<float>(ne.size(), 0.f));
  }
  if (is_mixed(D->desc.precision)) {
    D->d_arm_alpha32 = dev_upload(D, to_f32(alpha));
    D->d_arm_beta32 = dev_upload(D, to_f32(beta));
    D->d_arm_fcoef32 = dev_upload(D, to_f32(fcoef));
    D->d_node_w32 = dev_upload(D, to_f32(nw));
    D->d_node_a32 = dev_upload(D, to_f32(na_));
    D->d_node_b32 = dev_upload(D, to_f32(nb_));
    D->d_node_fcoef32 = dev_upload(D, to_f32(P.node_fcoef));
  }
  // DST-I matrix and eigenvalues, shared with every domain on this grid
  D->tables = dst_tables(M, Mp, D->h, is_mixed(D->desc.precision));
  D->d_S = D->tables->S;
  D->d_lam = D->tables->lam;
  D->d_R = dev_alloc<double>(D, 2 * plane);
  if (D->desc.precision == KFBI_FP64) D->d_T = dev_alloc<double>(D, 2 * plane);
  D->d_U = dev_alloc<double>(D, 2 * plane);
  D->d_fpad = dev_alloc<double>(D, 2 * plane);
  D->d_zero_nb = dev_alloc<double>(D, 2 * (size_t)nb);
  KFBI_CUDA(cudaMemset(D->d_R, 0, 2 * plane * sizeof(double)));
  KFBI_CUDA(cudaMemset(D->d_U, 0, 2 * plane * sizeof(double)));
  KFBI_CUDA(cudaMemset(D->d_zero_nb, 0, 2 * (size_t)nb * sizeof(double)));
  D->rhs_sparse_planes = 2;
}

// FP64 corrected right-hand side in D->d_R (f-tilde plus the jump
// corrections at the irregular nodes).
void correct_fp64(kfbi_domain* D, double kre, double kim, const double* phi, int ps,
                  const double* ft, cudaStream_t st) {
  const bool C = kim != 0.0;
  const int P = C ? 2 : 1;
  const size_t plane = (size_t)D->Mp * D->Mp;
  // base right-hand side: f-tilde everywhere, or zero off the irregular nodes
  if (ft) {
    KFBI_CUDA(cudaMemcpyAsync(D->d_R, ft, P * plane * sizeof(double), cudaMemcpyDeviceToDevice, st));
    D->rhs_sparse_planes = 0;
  } else if (D->rhs_sparse_planes < P) {
    KFBI_CUDA(cudaMemsetAsync(D->d_R, 0, 2 * plane * sizeof(double), st));
    D->rhs_sparse_planes = 2;
  }
  // Neumann: the density is psi, weighted by arm_delta, with no kappa term
  const double* al = D->neumann ? D->d_arm_delta : D->d_arm_alpha;
  const double* be = D->neumann ? nullptr : D->d_arm_beta;
  if (D->n_irr > 0) {
    if (C)
      KFBI_LAUNCH_P(KFBI_PROF_CORRECT, k_correct<true>, (D->n_irr + 127) / 128, 128, 0, st, D->d_R, plane, ft,
                  D->d_irr_off, D->d_arm_start, D->d_arm_k0, al, be,
                  D->d_arm_fidx, D->d_arm_fcoef, D->n_irr, D->n_arms, D->nb, phi, ps, kre, kim);
    else
      KFBI_LAUNCH_P(KFBI_PROF_CORRECT, k_correct<false>, (D->n_irr + 127) / 128, 128, 0, st, D->d_R, plane, ft,
                  D->d_irr_off, D->d_arm_start, D->d_arm_k0, al, be,
                  D->d_arm_fidx, D->d_arm_fcoef, D->n_irr, D->n_arms, D->nb, phi, ps, kre, kim);
  }
  KFBI_CHECK_LAUNCH();
}

// FP64 extraction of u+ (Neumann: d_n u+) from the grid solution in D->d_U.
void extract_fp64(kfbi_domain* D, double kre, double kim, const double* phi, int ps,
                  const double* ft, double* out, int os, cudaStream_t st) {
  const size_t plane = (size_t)D->Mp * D->Mp;
  const bool nm = D->neumann;
  const double* w = nm ? D->d_node_wn : D->d_node_w;
  const double* a = nm ? D->d_node_e : D->d_node_a;
  const double* b = nm ? nullptr : D->d_node_b;
  const double* fc = nm ? D->d_node_fcoef_n : D->d_node_fcoef;
  if (kim != 0.0)
    KFBI_LAUNCH_P(KFBI_PROF_EXTRACT, k_extract<true>, (D->nb + 127) / 128, 128, 0, st, D->d_U, plane, ft,
                D->d_node_gidx, w, a, b, D->d_node_fidx, fc, D->nb, phi, ps, kre, kim, out, os);
  else
    KFBI_LAUNCH_P(KFBI_PROF_EXTRACT, k_extract<false>, (D->nb + 127) / 128, 128, 0, st, D->d_U, plane, ft,
                D->d_node_gidx, w, a, b, D->d_node_fidx, fc, D->nb, phi, ps, kre, kim, out, os);
  KFBI_CHECK_LAUNCH();
}

void apply_internal(kfbi_domain* D, double kre, double kim, const double* phi, int ps,
                    const double* ft, double* out, int os, bool want_grid, cudaStream_t st) {
  if (D->tc) {
    tc_apply(D, kre, kim, phi, ps, ft, out, os, want_grid, st);
    return;
  }
  const bool C = kim != 0.0;
  const int P = C ? 2 : 1;
  const int Mp = D->Mp, n1 = D->n1;
  const size_t plane = (size_t)Mp * Mp;
  correct_fp64(D, kre, kim, phi, ps, ft, st);
  dim3 gg(Mp / 64, Mp / 64, P);
  // one float64 pass: P planes of an (n1 x n1) by (n1 x n1) product
  const double pass_fl = 2.0 * P * (double)n1 * n1 * n1;
  KFBI_LAUNCH_PW(KFBI_PROF_DST, pass_fl, k_dgemm_t, gg, 256, 0, st, D->d_R, D->d_S, D->d_T, Mp);
  KFBI_LAUNCH_PW(KFBI_PROF_DST, pass_fl, k_dgemm_t, gg, 256, 0, st, D->d_T, D->d_S, D->d_U, Mp);
  const double scale = (2.0 / D->M) * (2.0 / D->M);
  KFBI_LAUNCH_P(KFBI_PROF_GRID, k_eigscale, grid_for(plane, 256), 256, 0, st, D->d_U, plane, Mp, n1, D->d_lam, kre,
              kim, scale, C ? 1 : 0);
  KFBI_LAUNCH_PW(KFBI_PROF_DST, pass_fl, k_dgemm_t, gg, 256, 0, st, D->d_U, D->d_S, D->d_T, Mp);
  KFBI_LAUNCH_PW(KFBI_PROF_DST, pass_fl, k_dgemm_t, gg, 256, 0, st, D->d_T, D->d_S, D->d_U, Mp);
  if (out) extract_fp64(D, kre, kim, phi, ps, ft, out, os, st);
  KFBI_CHECK_LAUNCH();
}

void apply_accurate(kfbi_domain* D, double kre, double kim, const double* phi, int ps,
                    const double* ft, double* out, int os, cudaStream_t st) {
  if (D->tc)
    tc_apply_accurate(D, kre, kim, phi, ps, ft, out, os, st);
  else
    apply_internal(D, kre, kim, phi, ps, ft, out, os, true, st);
}

void pad_mask(kfbi_domain* D, const double* src, double* dst, bool C, cudaStream_t st) {
  const size_t plane = (size_t)D->Mp * D->Mp;
  if (C)
    KFBI_LAUNCH(k_pad_mask<true>, grid_for(plane, 256), 256, 0, st, src, D->d_mask, dst, D->n1, D->Mp);
  else
    KFBI_LAUNCH(k_pad_mask<false>, grid_for(plane, 256), 256, 0, st, src, D->d_mask, dst, D->n1, D->Mp);
  KFBI_CHECK_LAUNCH();
}

void unpad(kfbi_domain* D, const double* src, double* dst, bool C, cudaStream_t st) {
  const size_t n = (size_t)D->n1 * D->n1;
  if (C)
    KFBI_LAUNCH(k_unpad<true>, grid_for(n, 256), 256, 0, st, src, dst, D->n1, D->Mp);
  else
    KFBI_LAUNCH(k_unpad<false>, grid_for(n, 256), 256, 0, st, src, dst, D->n1, D->Mp);
  KFBI_CHECK_LAUNCH();
}

kfbi_domain* domain_from_plan(const Plan& plan, cudaStream_t st) {
  kfbi_domain* D = new kfbi_domain();
  D->desc = plan.desc;
  D->M = plan.M;
  D->nb = plan.nb;
  D->n1 = plan.n1;
  D->Mp = ((plan.n1 + 127) / 128) * 128;
  D->h = plan.h;
  D->lo = plan.lo;
  try {
    KFBI_CUDA(cudaGetDevice(&D->device));
    upload_domain(D, plan);
    gmres_alloc(D);
    if (is_mixed(plan.desc.precision)) D->tc = tc_create(D, plan);
    KFBI_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    free_domain(D);
    throw;
  }
  return D;
}

// Mirrors upload_domain + gmres_alloc + tc_create (every table allocation
// takes at least one element).
long long domain_bytes_for(const Plan& P) {
  auto n1 = [](size_t n) { return std::max<size_t>(1, n); };
  const int Mp = ((P.n1 + 127) / 128) * 128;
  const size_t plane = (size_t)Mp * Mp;
  const bool mixed = is_mixed(P.desc.precision);
  size_t b = n1(plane);                                                       // mask
  b += sizeof(int) * (n1(P.irr.size()) + n1(P.arm_start.size()) + n1(P.arm_k0.size()) +
                      n1(P.arm_fidx.size()) + n1(P.node_gidx.size()) + n1(P.node_fidx.size()));
  const size_t dtab = 2 * n1(P.arm_alpha.size()) + n1(P.arm_fcoef.size()) +
                      3 * n1(P.node_w.size()) + n1(P.node_fcoef.size());
  b += sizeof(double) * dtab;
  if (mixed) b += sizeof(float) * dtab;
  // Neumann tables: FP64 always; FP32 copies and two zero tables if mixed
  const size_t ntab = n1(P.arm_delta.size()) + 2 * n1(P.node_wn.size()) +
                      n1(P.node_fcoef_n.size());
  b += sizeof(double) * ntab;
  if (mixed) b += sizeof(float) * (ntab + n1(P.arm_delta.size()) + n1(P.node_wn.size()));
  b += sizeof(double) * (2 * plane * (mixed ? 3 : 4) + 2 * (size_t)P.nb);   // R, (T), U, fpad, zero_nb
  long long total = (long long)b + gmres_bytes(P.desc.gmres_restart, P.nb);
  if (mixed) total += tc_bytes_for(P, Mp);
  return total;
}

}  // namespace kfbi

using namespace kfbi;

extern "C" {

kfbi_status kfbi_create_domain(const kfbi_domain_desc* desc, void* stream, kfbi_domain** out) {
  if (!out) return KFBI_ERR_ARG;
  *out = nullptr;
  if (!desc) {
    set_global_error("desc is NULL");
    return KFBI_ERR_ARG;
  }
  if (desc->precision != KFBI_FP64 && !is_mixed(desc->precision)) {
    set_global_error("unknown precision");
    return KFBI_ERR_ARG;
  }
  if (desc->gmres_restart < 1 || desc->gmres_restart > 64 || desc->gmres_maxit < 1 ||
      !(desc->gmres_tol > 0.0)) {
    set_global_error("GMRES parameters out of range (1 <= restart <= 64, maxit >= 1, tol > 0)");
    return KFBI_ERR_ARG;
  }
  if (desc->solver != KFBI_GMRES && desc->solver != KFBI_RICHARDSON) {
    set_global_error("unknown solver");
    return KFBI_ERR_ARG;
  }
  if (desc->solver == KFBI_RICHARDSON &&
      !(desc->richardson_gamma > 0.0 && desc->richardson_gamma < 2.0)) {
    set_global_error("Richardson step gamma must lie in (0, 2)");
    return KFBI_ERR_ARG;
  }
  Plan plan;
  std::string err;
  kfbi_status s = build_plan(*desc, plan, err);
  if (s != KFBI_OK) {
    set_global_error(err);
    return s;
  }
  kfbi_domain* D = nullptr;
  s = guarded(nullptr, [&]() -> kfbi_status {
    D = domain_from_plan(plan, (cudaStream_t)stream);
    return KFBI_OK;
  });
  if (s != KFBI_OK) return s;
  *out = D;
  return KFBI_OK;
}

void kfbi_destroy_domain(kfbi_domain* dom) {
  if (!dom) return;
  cudaDeviceSynchronize();
  free_domain(dom);
}

kfbi_status kfbi_apply_operator(kfbi_domain* dom, double kappa_re, double kappa_im,
                                const void* phi_dev, const void* f_dev, void* out_dev,
                                void* stream) {
  if (!dom) return KFBI_ERR_ARG;
  if (!phi_dev || !out_dev) {
    dom->err = "phi_dev and out_dev must be device pointers";
    return KFBI_ERR_ARG;
  }
  return guarded(dom, [&]() -> kfbi_status {
    cudaStream_t st = (cudaStream_t)stream;
    const bool C = kappa_im != 0.0;
    const double* ft = nullptr;
    if (f_dev) {
      pad_mask(dom, (const double*)f_dev, dom->d_fpad, C, st);
      ft = dom->d_fpad;
    }
    apply_internal(dom, kappa_re, kappa_im, (const double*)phi_dev, C ? 2 : 1, ft,
                   (double*)out_dev, C ? 2 : 1, false, st);
    return KFBI_OK;
  });
}

kfbi_status kfbi_interface_solve(kfbi_domain* dom, double kappa_re, double kappa_im,
                                 const void* phi_dev, const void* f_dev, void* u_grid_dev,
                                 void* u_plus_dev, void* stream) {
  if (!dom) return KFBI_ERR_ARG;
  if (!phi_dev || !u_grid_dev) {
    dom->err = "phi_dev and u_grid_dev must be device pointers";
    return KFBI_ERR_ARG;
  }
  return guarded(dom, [&]() -> kfbi_status {
    cudaStream_t st = (cudaStream_t)stream;
    const bool C = kappa_im != 0.0;
    const double* ft = nullptr;
    if (f_dev) {
      pad_mask(dom, (const double*)f_dev, dom->d_fpad, C, st);
      ft = dom->d_fpad;
    }
    apply_internal(dom, kappa_re, kappa_im, (const double*)phi_dev, C ? 2 : 1, ft,
                   (double*)u_plus_dev, C ? 2 : 1, true, st);
    unpad(dom, dom->d_U, (double*)u_grid_dev, C, st);
    return KFBI_OK;
  });
}

const char* kfbi_last_error(const kfbi_domain* dom) { return dom ? dom->err.c_str() : ""; }

const char* kfbi_last_global_error(void) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  static thread_local std::string copy;
  copy = g_err;
  return copy.c_str();
}

long long kfbi_launch_count(void) { return g_launches.load(); }

long long kfbi_domain_device_bytes(const kfbi_domain* dom) {
  if (!dom) return 0;
  return dom->bytes + (dom->tc ? tc_bytes(dom->tc) : 0);
}

// ---- host-only plan ---------------------------------------------------------

struct kfbi_plan {
  Plan p;
};

kfbi_status kfbi_plan_create(const kfbi_domain_desc* desc, kfbi_plan** out) {
  if (!out || !desc) return KFBI_ERR_ARG;
  *out = nullptr;
  kfbi_plan* pl = new (std::nothrow) kfbi_plan();
  if (!pl) return KFBI_ERR_OOM;
  std::string err;
  kfbi_status s = build_plan(*desc, pl->p, err);
  if (s != KFBI_OK) {
    set_global_error(err);
    delete pl;
    return s;
  }
  *out = pl;
  return KFBI_OK;
}

void kfbi_plan_destroy(kfbi_plan* plan) { delete plan; }

long long kfbi_plan_device_bytes(const kfbi_plan* plan, int equation) {
  if (!plan || equation < KFBI_HEAT || equation > KFBI_SCHRODINGER) return -1;
  const Plan& P = plan->p;
  const int Mp = ((P.n1 + 127) / 128) * 128;
  return domain_bytes_for(P) +
         state_bytes_for(Mp, P.nb, equation, is_mixed(P.desc.precision));
}

long long kfbi_plan_size(const kfbi_plan* plan, int field) {
  if (!plan) return -1;
  const Plan& P = plan->p;
  switch (field) {
    case KFBI_PLAN_N_EDGES: return P.n_edges();
    case KFBI_PLAN_EDGE_I: case KFBI_PLAN_EDGE_J: case KFBI_PLAN_EDGE_DIR:
    case KFBI_PLAN_EDGE_COORD: case KFBI_PLAN_EDGE_THETA: return P.n_edges();
    case KFBI_PLAN_INSIDE: return (long long)P.inside.size();
    case KFBI_PLAN_N_IRREGULAR: return P.n_irr();
    case KFBI_PLAN_IRREGULAR: return P.n_irr();
    case KFBI_PLAN_N_ARMS: return P.n_arms();
    case KFBI_PLAN_ARM_NODE: case KFBI_PLAN_ARM_K0: return P.n_arms();
    case KFBI_PLAN_ARM_ALPHA: case KFBI_PLAN_ARM_BETA: case KFBI_PLAN_ARM_DELTA:
      return (long long)P.n_arms() * 6;
    case KFBI_PLAN_ARM_FIDX: case KFBI_PLAN_ARM_FCOEF: return (long long)P.n_arms() * 2;
    case KFBI_PLAN_NODE_GIDX: case KFBI_PLAN_NODE_W: case KFBI_PLAN_NODE_A:
    case KFBI_PLAN_NODE_B: case KFBI_PLAN_NODE_WN: case KFBI_PLAN_NODE_E:
      return (long long)P.nb * 6;
    case KFBI_PLAN_NODE_FIDX: case KFBI_PLAN_NODE_FCOEF: case KFBI_PLAN_NODE_FCOEF_N:
      return P.nb;
    default: return -1;
  }
}

kfbi_status kfbi_plan_export(const kfbi_plan* plan, int field, void* dst) {
  if (!plan || !dst) return KFBI_ERR_ARG;
  const Plan& P = plan->p;
  auto cp = [&](const auto& v) {
    std::memcpy(dst, v.data(), v.size() * sizeof(v[0]));
    return KFBI_OK;
  };
  switch (field) {
    case KFBI_PLAN_EDGE_I: return cp(P.e_i);
    case KFBI_PLAN_EDGE_J: return cp(P.e_j);
    case KFBI_PLAN_EDGE_DIR: return cp(P.e_dir);
    case KFBI_PLAN_EDGE_COORD: return cp(P.e_coord);
    case KFBI_PLAN_EDGE_THETA: return cp(P.e_theta);
    case KFBI_PLAN_INSIDE: return cp(P.inside);
    case KFBI_PLAN_IRREGULAR: return cp(P.irr);
    case KFBI_PLAN_ARM_NODE: return cp(P.arm_node);
    case KFBI_PLAN_ARM_K0: return cp(P.arm_k0);
    case KFBI_PLAN_ARM_ALPHA: return cp(P.arm_alpha);
    case KFBI_PLAN_ARM_BETA: return cp(P.arm_beta);
    case KFBI_PLAN_ARM_FIDX: return cp(P.arm_fidx);
    case KFBI_PLAN_ARM_FCOEF: return cp(P.arm_fcoef);
    case KFBI_PLAN_NODE_GIDX: return cp(P.node_gidx);
    case KFBI_PLAN_NODE_W: return cp(P.node_w);
    case KFBI_PLAN_NODE_A: return cp(P.node_a);
    case KFBI_PLAN_NODE_B: return cp(P.node_b);
    case KFBI_PLAN_NODE_FIDX: return cp(P.node_fidx);
    case KFBI_PLAN_NODE_FCOEF: return cp(P.node_fcoef);
    case KFBI_PLAN_ARM_DELTA: return cp(P.arm_delta);
    case KFBI_PLAN_NODE_WN: return cp(P.node_wn);
    case KFBI_PLAN_NODE_E: return cp(P.node_e);
    case KFBI_PLAN_NODE_FCOEF_N: return cp(P.node_fcoef_n);
    default: return KFBI_ERR_ARG;
  }
}

}  // extern "C"
