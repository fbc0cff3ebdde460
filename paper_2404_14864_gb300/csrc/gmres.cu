// GMRES(m) on the device for the Dirichlet BIE (Eq. 3.17, arXiv 2404.14864);
// the paper iterates with Richardson (Eq. 3.21) and names GMRES as the
// Krylov alternative (Sec. 5).
//
// Vectors are complex interleaved (re, im) of length nb; a real operator
// keeps every imaginary part exactly zero, so one code path serves the
// heat/wave (real kappa) and Schroedinger (complex kappa) solves.  Arnoldi
// orthogonalisation is classical Gram-Schmidt applied twice (CGS2: all
// inner products of a pass in parallel, one warp per basis vector), in
// float64, with complex Givens rotations on the Hessenberg column and the
// rotated residual |g_{j+1}| as the convergence estimate.  All of it runs
// in one CTA per kernel: the vectors are a few thousand entries.
#include <cmath>

#include "internal.h"

namespace kfbi {

namespace gm {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < kWarps) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) red[0] = v;
  }
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

// scal: [0] ||b||, [1] residual estimate, [2] status (0 running, 1 converged,
// 2 non-finite), [3] tol
__global__ void __launch_bounds__(kThreads) k_bnorm(const double2* __restrict__ b, int nb,
                                                     double* scal, double tol) {
  __shared__ double red[32];
  double s = 0.0;
  for (int e = threadIdx.x; e < nb; e += kThreads) s += b[e].x * b[e].x + b[e].y * b[e].y;
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    scal[0] = sqrt(s);
    scal[3] = tol;
  }
}

// r = b - Ax (Ax may be null for x = 0); V0 = r / beta; g = (beta, 0, ...).
__global__ void __launch_bounds__(kThreads) k_restart(const double2* __restrict__ b,
                                                       const double2* __restrict__ Ax,
                                                       double2* __restrict__ V0, double2* g,
                                                       int m, int nb, double* scal) {
  __shared__ double red[32];
  double s = 0.0;
  for (int e = threadIdx.x; e < nb; e += kThreads) {
    double2 r = b[e];
    if (Ax) {
      r.x -= Ax[e].x;
      r.y -= Ax[e].y;
    }
    V0[e] = r;
    s += r.x * r.x + r.y * r.y;
  }
  s = block_sum(s, red);
  const double beta = sqrt(s);
  const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  for (int e = threadIdx.x; e < nb; e += kThreads) {
    V0[e].x *= inv;
    V0[e].y *= inv;
  }
  if (threadIdx.x <= m) g[threadIdx.x] = make_double2(threadIdx.x == 0 ? beta : 0.0, 0.0);
  if (threadIdx.x == 0) {
    scal[1] = beta;
    scal[2] = !isfinite(beta) ? 2.0 : (beta <= scal[3] * scal[0] ? 1.0 : 0.0);
  }
}

// One Arnoldi step: w = A v_j on entry; CGS2 against v_0..v_j, v_{j+1} =
// w / ||w||, Hessenberg column j rotated by the previous Givens rotations,
// new rotation, g updated, residual estimate |g_{j+1}|.
__global__ void __launch_bounds__(kThreads) k_arnoldi(double2* __restrict__ V, int nb, int j,
                                                       const double2* __restrict__ w_in,
                                                       double2* H, double* cs, double2* sn,
                                                       double2* g, int m, double* scal) {
  __shared__ double red[32];
  __shared__ double2 hp[65], hacc[65];
  double2* w = V + (size_t)(j + 1) * nb;  // build the new basis vector in place
  for (int e = threadIdx.x; e < nb; e += kThreads) w[e] = w_in[e];
  if (threadIdx.x <= j) hacc[threadIdx.x] = make_double2(0.0, 0.0);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = warp; i <= j; i += kWarps) {
      const double2* vi = V + (size_t)i * nb;
      double2 s = make_double2(0.0, 0.0);
      for (int e = lane; e < nb; e += 32) {
        const double2 t = cconjmul(vi[e], w[e]);
        s.x += t.x;
        s.y += t.y;
      }
      for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      }
      if (lane == 0) hp[i] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb; e += kThreads) {
      double2 acc = w[e];
      for (int i = 0; i <= j; ++i) {
        const double2 t = cmul(hp[i], V[(size_t)i * nb + e]);
        acc.x -= t.x;
        acc.y -= t.y;
      }
      w[e] = acc;
    }
    if (threadIdx.x <= j) {
      hacc[threadIdx.x].x += hp[threadIdx.x].x;
      hacc[threadIdx.x].y += hp[threadIdx.x].y;
    }
    __syncthreads();
  }
  double s = 0.0;
  for (int e = threadIdx.x; e < nb; e += kThreads) s += w[e].x * w[e].x + w[e].y * w[e].y;
  s = block_sum(s, red);
  const double hn = sqrt(s);
  const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  for (int e = threadIdx.x; e < nb; e += kThreads) {
    w[e].x *= inv;
    w[e].y *= inv;
  }
  if (threadIdx.x == 0) {
    double2* col = H + (size_t)j * (m + 1);
    for (int i = 0; i <= j; ++i) col[i] = hacc[i];
    col[j + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < j; ++i) {  // previous rotations
      const double c = cs[i];
      const double2 sv = sn[i], a = col[i], bb = col[i + 1];
      const double2 t = cmul(sv, bb);
      const double2 csv = make_double2(sv.x, -sv.y);
      const double2 u = cmul(csv, a);
      col[i] = make_double2(c * a.x + t.x, c * a.y + t.y);
      col[i + 1] = make_double2(-u.x + c * bb.x, -u.y + c * bb.y);
    }
    const double2 a = col[j];
    const double bre = col[j + 1].x;  // real, >= 0
    double c;
    double2 sv;
    const double aa = hypot(a.x, a.y);
    if (bre == 0.0) {
      c = 1.0;
      sv = make_double2(0.0, 0.0);
    } else if (aa == 0.0) {
      c = 0.0;
      sv = make_double2(1.0, 0.0);
    } else {
      const double den = hypot(aa, bre);
      c = aa / den;
      sv = make_double2(a.x / aa * bre / den, a.y / aa * bre / den);
    }
    cs[j] = c;
    sn[j] = sv;
    col[j] = make_double2(c * a.x + sv.x * bre, c * a.y + sv.y * bre);
    col[j + 1] = make_double2(0.0, 0.0);
    const double2 gj = g[j];
    const double2 csv = make_double2(sv.x, -sv.y);
    const double2 u = cmul(csv, gj);
    g[j + 1] = make_double2(-u.x, -u.y);
    g[j] = make_double2(c * gj.x, c * gj.y);
    const double res = hypot(g[j + 1].x, g[j + 1].y);
    scal[1] = res;
    scal[2] = !isfinite(res) ? 2.0 : ((res <= scal[3] * scal[0] || hn == 0.0) ? 1.0 : 0.0);
  }
}

// x += V[:, :k] y with R y = g (k x k upper triangle of the rotated H).
__global__ void __launch_bounds__(kThreads) k_update(const double2* __restrict__ V, int nb, int k,
                                                      const double2* H, const double2* g, int m,
                                                      double2* __restrict__ x) {
  __shared__ double2 y[64];
  if (threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double2 s = g[i];
      for (int l = i + 1; l < k; ++l) {
        const double2 t = cmul(H[(size_t)l * (m + 1) + i], y[l]);
        s.x -= t.x;
        s.y -= t.y;
      }
      const double2 d = H[(size_t)i * (m + 1) + i];
      const double dd = d.x * d.x + d.y * d.y;
      y[i] = make_double2((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nb; e += kThreads) {
    double2 acc = x[e];
    for (int i = 0; i < k; ++i) {
      const double2 t = cmul(y[i], V[(size_t)i * nb + e]);
      acc.x += t.x;
      acc.y += t.y;
    }
    x[e] = acc;
  }
}

}  // namespace gm

using namespace gm;

void gmres_alloc(kfbi_domain* D) {
  const int m = D->desc.gmres_restart, nb = D->nb;
  D->restart = m;
  auto alloc = [&](double** p, size_t n) {
    KFBI_CUDA(cudaMalloc(p, n * sizeof(double)));
    D->bytes += (long long)(n * sizeof(double));
  };
  alloc(&D->d_V, (size_t)(m + 1) * 2 * nb);
  alloc(&D->d_W, 2 * (size_t)nb);
  alloc(&D->d_X, 2 * (size_t)nb);
  alloc(&D->d_B, 2 * (size_t)nb);
  alloc(&D->d_H, (size_t)(m + 1) * m * 2);
  alloc(&D->d_cs, m);
  alloc(&D->d_sn, 2 * (size_t)m);
  alloc(&D->d_g, 2 * (size_t)(m + 1));
  alloc(&D->d_scal, 8);
  KFBI_CUDA(cudaMallocHost(&D->h_scal, 8 * sizeof(double)));
}

void gmres_free(kfbi_domain* D) {
  double* ptrs[] = {D->d_V, D->d_W, D->d_X, D->d_B, D->d_H, D->d_cs, D->d_sn, D->d_g, D->d_scal};
  for (double* p : ptrs)
    if (p) cudaFree(p);
  if (D->h_scal) cudaFreeHost(D->h_scal);
  D->h_scal = nullptr;
}

static void read_scalars(kfbi_domain* D, cudaStream_t st) {
  KFBI_CUDA(cudaMemcpyAsync(D->h_scal, D->d_scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  KFBI_CUDA(cudaStreamSynchronize(st));
}

kfbi_status gmres_solve(kfbi_domain* D, double kre, double kim, const double* b, double* x,
                        bool x_zero, kfbi_solve_info* info, cudaStream_t st) {
  const int m = D->restart, nb = D->nb, maxit = D->desc.gmres_maxit;
  const double tol = D->desc.gmres_tol;
  double2* V = (double2*)D->d_V;
  double2* W = (double2*)D->d_W;
  double2* H = (double2*)D->d_H;
  double2* g = (double2*)D->d_g;
  double2* sn = (double2*)D->d_sn;
  KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_bnorm, 1, kThreads, 0, st, (const double2*)b, nb, D->d_scal, tol);
  int it = 0;
  bool first = true;
  kfbi_status status = KFBI_OK;
  if (info) *info = kfbi_solve_info{0, 0.0, 0, 0};
  for (;;) {
    const bool skip_ax = first && x_zero;
    if (!skip_ax) apply_internal(D, kre, kim, x, 2, nullptr, D->d_W, 2, false, st);
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_restart, 1, kThreads, 0, st, (const double2*)b, skip_ax ? nullptr : W, V, g, m,
                nb, D->d_scal);
    KFBI_CHECK_LAUNCH();
    read_scalars(D, st);
    if (info) info->applications += skip_ax ? 0 : 1;
    if (D->h_scal[0] == 0.0) {  // b = 0 -> x = 0
      KFBI_CUDA(cudaMemsetAsync(x, 0, 2 * (size_t)nb * sizeof(double), st));
      D->h_scal[1] = 0.0;
      D->h_scal[2] = 1.0;
      break;
    }
    if (D->h_scal[2] != 0.0 || it >= maxit) break;
    first = false;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      apply_internal(D, kre, kim, (const double*)(V + (size_t)j * nb), 2, nullptr, D->d_W, 2,
                     false, st);
      KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_arnoldi, 1, kThreads, 0, st, V, nb, j, (const double2*)W, H, D->d_cs, sn, g, m,
                  D->d_scal);
      KFBI_CHECK_LAUNCH();
      ++it;
      k = j + 1;
      read_scalars(D, st);
      if (D->h_scal[2] != 0.0 || it >= maxit) break;
    }
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_update, 1, kThreads, 0, st, V, nb, k, H, g, m, (double2*)x);
    KFBI_CHECK_LAUNCH();
    if (D->h_scal[2] != 0.0 || it >= maxit) break;
  }
  KFBI_CUDA(cudaStreamSynchronize(st));
  const double bn = D->h_scal[0] > 0.0 ? D->h_scal[0] : 1.0;
  if (info) {
    info->iters = it;
    info->applications += it;
    info->rel_residual = D->h_scal[1] / bn;
    info->converged = D->h_scal[2] == 1.0;
  }
  if (D->h_scal[2] == 2.0) {
    D->err = "non-finite GMRES residual";
    status = KFBI_ERR_NONFINITE;
  } else if (D->h_scal[2] != 1.0) {
    D->err = "GMRES reached gmres_maxit";
    status = KFBI_ERR_NOT_CONVERGED;
  }
  return status;
}

}  // namespace kfbi

using namespace kfbi;

namespace kfbi_cv {
__global__ void k_to_cplx(const double* __restrict__ src, double* __restrict__ dst, int n, int C) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  dst[2 * k] = C ? src[2 * k] : src[k];
  dst[2 * k + 1] = C ? src[2 * k + 1] : 0.0;
}
__global__ void k_from_cplx(const double* __restrict__ src, double* __restrict__ dst, int n, int C) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  if (C) {
    dst[2 * k] = src[2 * k];
    dst[2 * k + 1] = src[2 * k + 1];
  } else {
    dst[k] = src[2 * k];
  }
}
}  // namespace kfbi_cv

using namespace kfbi_cv;

extern "C" kfbi_status kfbi_solve_density(kfbi_domain* dom, double kappa_re, double kappa_im,
                                          const void* b_dev, void* phi_dev, kfbi_solve_info* info,
                                          void* stream) {
  if (!dom) return KFBI_ERR_ARG;
  if (!b_dev || !phi_dev) {
    dom->err = "b_dev and phi_dev must be device pointers";
    return KFBI_ERR_ARG;
  }
  return guarded(dom, [&]() -> kfbi_status {
    cudaStream_t st = (cudaStream_t)stream;
    const int C = kappa_im != 0.0, nb = dom->nb;
    KFBI_LAUNCH(k_to_cplx, (nb + 255) / 256, 256, 0, st, (const double*)b_dev, dom->d_B, nb, C);
    KFBI_LAUNCH(k_to_cplx, (nb + 255) / 256, 256, 0, st, (const double*)phi_dev, dom->d_X, nb, C);
    KFBI_CHECK_LAUNCH();
    kfbi_status s = gmres_solve(dom, kappa_re, kappa_im, dom->d_B, dom->d_X, false, info, st);
    KFBI_LAUNCH(k_from_cplx, (nb + 255) / 256, 256, 0, st, dom->d_X, (double*)phi_dev, nb, C);
    KFBI_CHECK_LAUNCH();
    KFBI_CUDA(cudaStreamSynchronize(st));
    return s;
  });
}
