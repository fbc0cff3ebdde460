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
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include <cooperative_groups.h>

#include "internal.h"
#include "tc_internal.h"

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
  KFBI_PDL_ENTRY();
  __shared__ double red[32];
  double s = 0.0;
  for (int e = threadIdx.x; e < nb; e += kThreads) s += b[e].x * b[e].x + b[e].y * b[e].y;
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    scal[0] = sqrt(s);
    scal[3] = tol;
    scal[7] = scal[0];  // kept for the refinement (inner solves reuse scal[0])
  }
}

// r = b - Ax (Ax may be null for x = 0); V0 = r / beta; g = (beta, 0, ...).
// The eight scalars and then, after a system-scope fence, their sequence
// number, written to host-mapped memory (slot seq & 1 of mbox) that the host
// polls: no copy or event in the stream, whose kernels would otherwise lose
// the programmatic-launch overlap at every scalar read.  One thread; mbox
// null: nothing.
__device__ __forceinline__ void mbox_post(const double* scal, double* mbox, long long seq) {
  if (!mbox) return;
  volatile double* slot = mbox + 16 * (seq & 1);
#pragma unroll
  for (int i = 0; i < 8; ++i) slot[i] = scal[i];
  __threadfence_system();
  reinterpret_cast<volatile long long*>(slot)[8] = seq;
}

// kRegPT elements of r per thread stay in registers between the norm and the
// scaling (nb <= kRegPT * kThreads); larger nb reads V0 back.
constexpr int kRegPT = 4;

__global__ void __launch_bounds__(kThreads) k_restart(const double2* __restrict__ b,
                                                       const double2* __restrict__ Ax,
                                                       double2* __restrict__ V0, double2* g,
                                                       int m, int nb, double* scal, double* mbox,
                                                       long long seq, double tol_x0) {
  KFBI_PDL_ENTRY();
  __shared__ double red[32];
  // x = 0 (Ax null) with tol_x0 >= 0: beta is ||b|| itself, so the start of
  // the solve writes scal[0] = ||b|| and scal[3] = tol here (no k_bnorm)
  const bool own_norm = !Ax && tol_x0 >= 0.0;
  const double s0 = own_norm ? 0.0 : scal[0], s3 = own_norm ? tol_x0 : scal[3];
  double s = 0.0;
  double2 rr[kRegPT];
  const bool in_regs = nb <= kRegPT * kThreads;
  if (in_regs) {
#pragma unroll
    for (int k = 0; k < kRegPT; ++k) {
      const int e = threadIdx.x + k * kThreads;
      double2 r = make_double2(0.0, 0.0);
      if (e < nb) {
        r = b[e];
        if (Ax) {
          const double2 a = Ax[e];
          r.x -= a.x;
          r.y -= a.y;
        }
      }
      rr[k] = r;
      s += r.x * r.x + r.y * r.y;
    }
  } else {
    for (int e = threadIdx.x; e < nb; e += kThreads) {
      double2 r = b[e];
      if (Ax) {
        r.x -= Ax[e].x;
        r.y -= Ax[e].y;
      }
      V0[e] = r;
      s += r.x * r.x + r.y * r.y;
    }
  }
  s = block_sum(s, red);
  // the square root and the reciprocal once (FP64 sequences every thread
  // would otherwise run on GB300's narrow FP64 pipe)
  __shared__ double s_beta, s_inv;
  if (threadIdx.x == 0) {
    s_beta = sqrt(s);
    s_inv = s_beta > 0.0 ? 1.0 / s_beta : 0.0;
  }
  __syncthreads();
  const double beta = s_beta, inv = s_inv;
  if (in_regs) {
#pragma unroll
    for (int k = 0; k < kRegPT; ++k) {
      const int e = threadIdx.x + k * kThreads;
      if (e < nb) V0[e] = make_double2(rr[k].x * inv, rr[k].y * inv);
    }
  } else {
    for (int e = threadIdx.x; e < nb; e += kThreads) {
      V0[e].x *= inv;
      V0[e].y *= inv;
    }
  }
  if (threadIdx.x <= m) g[threadIdx.x] = make_double2(threadIdx.x == 0 ? beta : 0.0, 0.0);
  if (threadIdx.x == 0) {
    const double bn = own_norm ? beta : s0;
    if (own_norm) {
      scal[0] = bn;
      scal[3] = s3;
    }
    scal[1] = beta;
    scal[2] = !isfinite(beta) ? 2.0 : (beta <= s3 * bn ? 1.0 : 0.0);
    mbox_post(scal, mbox, seq);
  }
}

// The refinement's residual check and the start of its inner solve in one
// kernel: r = b - Ax into Rv, ||r|| into scal[1], and (as k_restart from
// x = 0 on Rv) V0 = r / ||r||, g = (||r||, 0, ...), with the inner tolerance
// max(0.5 tol ||b|| / ||r||, floor) formed here from ||b|| in scal[7].
// When ||r|| <= tol ||b|| (or is not finite) the GMRES status scal[2] is set
// (1, 2), so an iteration queued behind this kernel returns at once.
__global__ void __launch_bounds__(kThreads) k_residual_restart(const double2* __restrict__ b,
                                                                const double2* __restrict__ Ax,
                                                                double2* __restrict__ Rv,
                                                                double2* __restrict__ V0,
                                                                double2* g, int m, int nb,
                                                                double* scal, double* mbox,
                                                                long long seq, double tol,
                                                                double floor_) {
  KFBI_PDL_ENTRY();
  __shared__ double red[32];
  double s = 0.0;
  double2 rr[kRegPT];
  const bool in_regs = nb <= kRegPT * kThreads;
  if (in_regs) {
#pragma unroll
    for (int k = 0; k < kRegPT; ++k) {
      const int e = threadIdx.x + k * kThreads;
      double2 r = make_double2(0.0, 0.0);
      if (e < nb) {
        r = b[e];
        if (Ax) {
          const double2 a = Ax[e];
          r.x -= a.x;
          r.y -= a.y;
        }
        Rv[e] = r;
      }
      rr[k] = r;
      s += r.x * r.x + r.y * r.y;
    }
  } else {
    for (int e = threadIdx.x; e < nb; e += kThreads) {
      double2 r = b[e];
      if (Ax) {
        r.x -= Ax[e].x;
        r.y -= Ax[e].y;
      }
      Rv[e] = r;
      s += r.x * r.x + r.y * r.y;
    }
  }
  s = block_sum(s, red);
  // the square root and the reciprocal once (FP64 sequences every thread
  // would otherwise run on GB300's narrow FP64 pipe)
  __shared__ double s_beta, s_inv;
  if (threadIdx.x == 0) {
    s_beta = sqrt(s);
    s_inv = s_beta > 0.0 ? 1.0 / s_beta : 0.0;
  }
  __syncthreads();
  const double beta = s_beta, inv = s_inv;
  if (in_regs) {
#pragma unroll
    for (int k = 0; k < kRegPT; ++k) {
      const int e = threadIdx.x + k * kThreads;
      if (e < nb) V0[e] = make_double2(rr[k].x * inv, rr[k].y * inv);
    }
  } else {
    for (int e = threadIdx.x; e < nb; e += kThreads)
      V0[e] = make_double2(Rv[e].x * inv, Rv[e].y * inv);
  }
  if (threadIdx.x <= m) g[threadIdx.x] = make_double2(threadIdx.x == 0 ? beta : 0.0, 0.0);
  if (threadIdx.x == 0) {
    const double bn = scal[7];
    const double st = !isfinite(beta) ? 2.0 : (beta <= tol * bn ? 1.0 : 0.0);
    scal[0] = beta;
    scal[1] = beta;
    scal[2] = st;
    scal[3] = st == 0.0 ? fmax(0.5 * tol * bn / beta, floor_) : 1.0;
    mbox_post(scal, mbox, seq);
  }
}

// ---- multi-CTA CGS2 Arnoldi ------------------------------------------------
// GB300 keeps a small fraction of FP64 throughput per SM, so one Arnoldi
// step is spread over up to 64 CTAs: each owns a slice of the vectors, the
// inner products of a pass are per-CTA partial sums (one warp per basis
// vector) reduced redundantly by every CTA in the next kernel.  Real
// problems touch only the real parts (C = false).
constexpr int GT = 256;  // threads per CTA of the grid kernels
constexpr int GMAX = 64; // maximum CTAs

template <bool C>
__device__ __forceinline__ double2 dotpart(const double2* __restrict__ a,
                                           const double2* __restrict__ b, int e0, int e1,
                                           int lane) {
  double2 s = make_double2(0.0, 0.0);
  for (int e = e0 + lane; e < e1; e += 32) {
    const double2 x = a[e], y = b[e];
    if (C) {
      s.x += x.x * y.x + x.y * y.y;
      s.y += x.x * y.y - x.y * y.x;
    } else {
      s.x += x.x * y.x;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
    if (C) s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
  }
  return s;
}

// Sum the G partials of entries 0..n-1 into sh[] (warp per entry).
template <bool C>
__device__ void reduce_parts(const double2* __restrict__ part, int n, int G, double2* sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < n; i += GT / 32) {
    double2 s = make_double2(0.0, 0.0);
    for (int b = lane; b < G; b += 32) {
      const double2 v = part[(size_t)i * GMAX + b];
      s.x += v.x;
      if (C) s.y += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      if (C) s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (lane == 0) sh[i] = s;
  }
}

// Pass-1 inner products <v_i, w>, i = 0..j, per CTA slice.
template <bool C>
__global__ void __launch_bounds__(GT) k_cgs_dots(const double2* __restrict__ V, int nb, int j,
                                                 const double2* __restrict__ w,
                                                 double2* __restrict__ part, int slice) {
  KFBI_PDL_ENTRY();
  const int b = blockIdx.x, G = gridDim.x;
  const int e0 = b * slice, e1 = min(nb, e0 + slice);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  (void)G;
  for (int i = warp; i <= j; i += GT / 32) {
    const double2 s = dotpart<C>(V + (size_t)i * nb, w, e0, e1, lane);
    if (lane == 0) part[(size_t)i * GMAX + b] = s;
  }
}

// Reduce the pass's inner products h, w -= V h on the slice, accumulate h
// into the Hessenberg column (CTA 0), then either the next pass's partial
// inner products (mode 0) or the partial squared norm (mode 1).
template <bool C>
__global__ void __launch_bounds__(GT) k_cgs_update(const double2* __restrict__ V, int nb, int j,
                                                   double2* __restrict__ w,
                                                   const double2* __restrict__ part_in,
                                                   double2* __restrict__ part_out,
                                                   double2* __restrict__ hcol, int first,
                                                   int mode, int slice) {
  KFBI_PDL_ENTRY();
  __shared__ double2 h[65];
  const int b = blockIdx.x, G = gridDim.x;
  const int e0 = b * slice, e1 = min(nb, e0 + slice);
  reduce_parts<C>(part_in, j + 1, G, h);
  __syncthreads();
  if (b == 0)
    for (int i = threadIdx.x; i <= j; i += GT) {
      if (first) {
        hcol[i] = h[i];
      } else {
        hcol[i].x += h[i].x;
        hcol[i].y += h[i].y;
      }
    }
  for (int e = e0 + threadIdx.x; e < e1; e += GT) {
    double2 acc = w[e];
    for (int i = 0; i <= j; ++i) {
      const double2 v = V[(size_t)i * nb + e], hi = h[i];
      if (C) {
        acc.x -= hi.x * v.x - hi.y * v.y;
        acc.y -= hi.x * v.y + hi.y * v.x;
      } else {
        acc.x -= hi.x * v.x;
      }
    }
    w[e] = acc;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (mode == 0) {
    for (int i = warp; i <= j; i += GT / 32) {
      const double2 s = dotpart<C>(V + (size_t)i * nb, w, e0, e1, lane);
      if (lane == 0) part_out[(size_t)i * GMAX + b] = s;
    }
  } else if (warp == 0) {
    const double2 s = dotpart<C>(w, w, e0, e1, lane);
    if (lane == 0) part_out[b] = make_double2(s.x, 0.0);
  }
}

// Hessenberg column j (col[0..j] = h, col[j+1] = ||w||) through the previous
// Givens rotations, the new rotation, g and the convergence scalars
// (scal[1] residual estimate, scal[2] 1 converged / 2 non-finite).  One
// thread.
__device__ void givens_column(double2* col, int j, double hn, double* cs, double2* sn, double2* g,
                              double* scal) {
  col[j + 1] = make_double2(hn, 0.0);
  // rotation i mixes the carried entry with the original col[i + 1]; the
  // operands of rotation i + 1 are loaded during rotation i, so the chain
  // is the arithmetic alone
  double2 carry = col[0];
  double c_n = 0.0;
  double2 s_n = make_double2(0.0, 0.0), b_n = make_double2(0.0, 0.0);
  if (j > 0) {
    c_n = cs[0];
    s_n = sn[0];
    b_n = col[1];
  }
  for (int i = 0; i < j; ++i) {
    const double c = c_n;
    const double2 sv = s_n, bb = b_n, a = carry;
    if (i + 1 < j) {
      c_n = cs[i + 1];
      s_n = sn[i + 1];
      b_n = col[i + 2];
    }
    const double2 t = cmul(sv, bb);
    const double2 u = cmul(make_double2(sv.x, -sv.y), a);
    col[i] = make_double2(c * a.x + t.x, c * a.y + t.y);
    carry = make_double2(-u.x + c * bb.x, -u.y + c * bb.y);
  }
  col[j] = carry;
  const double2 a = col[j];
  const double bre = col[j + 1].x;
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
  const double2 u = cmul(make_double2(sv.x, -sv.y), gj);
  g[j + 1] = make_double2(-u.x, -u.y);
  g[j] = make_double2(c * gj.x, c * gj.y);
  const double res = hypot(g[j + 1].x, g[j + 1].y);
  scal[1] = res;
  scal[2] = !isfinite(res) ? 2.0 : ((res <= scal[3] * scal[0] || hn == 0.0) ? 1.0 : 0.0);
}

// The same for a real problem (every h, sn and g real): real arithmetic
// only, which halves the dependent FP64 chain of each rotation.
__device__ void givens_column_real(double2* col, int j, double hn, double* cs, double2* sn,
                                   double2* g, double* scal) {
  // operands of rotation i + 1 are loaded during rotation i (see givens_column)
  double carry = col[0].x;
  double c_n = 0.0, s_n = 0.0, b_n = 0.0;
  if (j > 0) {
    c_n = cs[0];
    s_n = sn[0].x;
    b_n = col[1].x;
  }
  for (int i = 0; i < j; ++i) {
    const double c = c_n, sv = s_n, b = b_n;
    if (i + 1 < j) {
      c_n = cs[i + 1];
      s_n = sn[i + 1].x;
      b_n = col[i + 2].x;
    }
    col[i] = make_double2(c * carry + sv * b, 0.0);
    carry = -sv * carry + c * b;
  }
  const double a = carry, bre = hn;
  double c, sv;
  const double aa = fabs(a);
  if (bre == 0.0) {
    c = 1.0;
    sv = 0.0;
  } else if (aa == 0.0) {
    c = 0.0;
    sv = 1.0;
  } else {
    const double den = hypot(aa, bre);
    c = aa / den;
    sv = (a < 0.0 ? -1.0 : 1.0) * bre / den;
  }
  cs[j] = c;
  sn[j] = make_double2(sv, 0.0);
  col[j] = make_double2(c * a + sv * bre, 0.0);
  col[j + 1] = make_double2(0.0, 0.0);
  const double gj = g[j].x;
  g[j + 1] = make_double2(-sv * gj, 0.0);
  g[j] = make_double2(c * gj, 0.0);
  const double res = fabs(sv * gj);
  scal[1] = res;
  scal[2] = !isfinite(res) ? 2.0 : ((res <= scal[3] * scal[0] || hn == 0.0) ? 1.0 : 0.0);
}

// ||w|| from the partials, v_{j+1} = w / ||w||, then (CTA 0, one thread)
// the Hessenberg column with the previous Givens rotations, the new
// rotation, g and the convergence scalars.
__global__ void __launch_bounds__(GT) k_cgs_finalize(double2* __restrict__ V, int nb, int j,
                                                     const double2* __restrict__ w,
                                                     const double2* __restrict__ part,
                                                     const double2* __restrict__ hcol, double2* H,
                                                     double* cs, double2* sn, double2* g, int m,
                                                     double* scal, int slice) {
  KFBI_PDL_ENTRY();
  __shared__ double2 nrm[1];
  const int b = blockIdx.x, G = gridDim.x;
  const int e0 = b * slice, e1 = min(nb, e0 + slice);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double s = 0.0;
    for (int q = lane; q < G; q += 32) s += part[q].x;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const double h = sqrt(s);
      nrm[0] = make_double2(h, h > 0.0 ? 1.0 / h : 0.0);
    }
  }
  __syncthreads();
  const double hn = nrm[0].x;
  const double inv = nrm[0].y;
  double2* vn = V + (size_t)(j + 1) * nb;
  for (int e = e0 + threadIdx.x; e < e1; e += GT) vn[e] = make_double2(w[e].x * inv, w[e].y * inv);
  if (b == 0 && threadIdx.x == 0) {
    double2* col = H + (size_t)j * (m + 1);
    for (int i = 0; i <= j; ++i) col[i] = hcol[i];
    givens_column(col, j, hn, cs, sn, g, scal);
  }
}

// Rotations 0 .. j-1 of the Givens sequence applied to a new Hessenberg
// column col[0 .. j] by one warp (j <= 64).  Rotation i maps the carried
// entry x (col[i] after rotation i-1) and the untouched col[i+1] to
// col[i] = c_i x + s_i col[i+1] and the next carry -conj(s_i) x +
// c_i col[i+1]: the carries follow x_{i+1} = al_i x_i + be_i with al_i =
// -conj(s_i), be_i = c_i col[i+1], a first-order linear recurrence, so they
// are a prefix composition of affine maps.  Each lane composes the maps of
// rotations 2 lane and 2 lane + 1, a five-level scan over the lanes gives
// every lane the composition of all earlier maps, and each lane then forms
// its two outputs.  The chain is about ten dependent float64 operations
// instead of j (a float64 operation waits ~100+ cycles on this part).
// Leaves the rotated entries in col[0 .. j-1] and the last carry in col[j].
template <bool C>
__device__ void rotate_column_warp(double2* col, int j, const double* cs, const double2* sn,
                                   int lane) {
  auto mul = [](double2 a, double2 b) {
    return C ? make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x)
             : make_double2(a.x * b.x, 0.0);
  };
  auto add = [](double2 a, double2 b) { return make_double2(a.x + b.x, C ? a.y + b.y : 0.0); };
  const int i0 = 2 * lane, i1 = 2 * lane + 1;
  double2 al[2], be[2], sv[2], bv[2];
  double cv[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int i = 2 * lane + q;
    if (i < j) {
      cv[q] = cs[i];
      sv[q] = sn[i];
      bv[q] = col[i + 1];
      al[q] = make_double2(-sv[q].x, C ? sv[q].y : 0.0);
      be[q] = make_double2(cv[q] * bv[q].x, C ? cv[q] * bv[q].y : 0.0);
    } else {  // identity map
      cv[q] = 1.0;
      sv[q] = make_double2(0.0, 0.0);
      bv[q] = make_double2(0.0, 0.0);
      al[q] = make_double2(1.0, 0.0);
      be[q] = make_double2(0.0, 0.0);
    }
  }
  const double2 x0 = col[0];
  // this lane's composition f_i1 o f_i0, then the inclusive scan
  double2 A = mul(al[1], al[0]), B = add(mul(al[1], be[0]), be[1]);
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    double2 Ap, Bp;
    Ap.x = __shfl_up_sync(0xffffffffu, A.x, d);
    Ap.y = __shfl_up_sync(0xffffffffu, A.y, d);
    Bp.x = __shfl_up_sync(0xffffffffu, B.x, d);
    Bp.y = __shfl_up_sync(0xffffffffu, B.y, d);
    if (lane >= d) {
      B = add(mul(A, Bp), B);
      A = mul(A, Ap);
    }
  }
  // composition of the maps of all earlier lanes applied to col[0]
  double2 Ae, Be;
  Ae.x = __shfl_up_sync(0xffffffffu, A.x, 1);
  Ae.y = __shfl_up_sync(0xffffffffu, A.y, 1);
  Be.x = __shfl_up_sync(0xffffffffu, B.x, 1);
  Be.y = __shfl_up_sync(0xffffffffu, B.y, 1);
  if (lane == 0) {
    Ae = make_double2(1.0, 0.0);
    Be = make_double2(0.0, 0.0);
  }
  const double2 x_0 = add(mul(Ae, x0), Be);          // carry entering rotation i0
  const double2 x_1 = add(mul(al[0], x_0), be[0]);   // carry entering rotation i1
  const double2 x_2 = add(mul(al[1], x_1), be[1]);   // carry after rotation i1
  __syncwarp();  // every lane has read its inputs before the column is overwritten
  if (i0 < j) col[i0] = add(make_double2(cv[0] * x_0.x, C ? cv[0] * x_0.y : 0.0), mul(sv[0], bv[0]));
  if (i1 < j) col[i1] = add(make_double2(cv[1] * x_1.x, C ? cv[1] * x_1.y : 0.0), mul(sv[1], bv[1]));
  if (i0 == j - 1) col[j] = x_1;
  if (i1 == j - 1) col[j] = x_2;
  __syncwarp();
}

// The new rotation of an Arnoldi step: zeroes hn below the rotated entry
// a = col[j], stores (c, s), updates col and g and the residual estimate
// (scal[1]) and convergence flag (scal[2]).
template <bool C>
__device__ void givens_new(double2* col, int j, double hn, double* cs, double2* sn, double2* g,
                           double* scal) {
  const double2 a = col[j];
  const double bre = hn;
  double c;
  double2 sv;
  // one reciprocal square root per quantity (Hessenberg entries are far
  // from the overflow range); division and hypot are long chains of
  // dependent float64 operations on this part
  const double a2 = C ? a.x * a.x + a.y * a.y : a.x * a.x;
  if (bre == 0.0) {
    c = 1.0;
    sv = make_double2(0.0, 0.0);
  } else if (a2 == 0.0) {
    c = 0.0;
    sv = make_double2(1.0, 0.0);
  } else {
    const double inv_den = rsqrt(a2 + bre * bre);
    const double inv_aa = rsqrt(a2);
    const double aa = a2 * inv_aa;
    c = aa * inv_den;
    const double sb = bre * inv_den;
    if (C)
      sv = make_double2(a.x * inv_aa * sb, a.y * inv_aa * sb);
    else
      sv = make_double2((a.x < 0.0 ? -1.0 : 1.0) * sb, 0.0);
  }
  cs[j] = c;
  sn[j] = sv;
  col[j] = make_double2(c * a.x + sv.x * bre, C ? c * a.y + sv.y * bre : 0.0);
  col[j + 1] = make_double2(0.0, 0.0);
  const double2 gj = g[j];
  const double2 u = C ? cmul(make_double2(sv.x, -sv.y), gj) : make_double2(sv.x * gj.x, 0.0);
  g[j + 1] = make_double2(-u.x, -u.y);
  g[j] = make_double2(c * gj.x, C ? c * gj.y : 0.0);
  const double res = C ? hypot(g[j + 1].x, g[j + 1].y) : fabs(sv.x * gj.x);
  scal[1] = res;
  scal[2] = !isfinite(res) ? 2.0 : ((res <= scal[3] * scal[0] || hn == 0.0) ? 1.0 : 0.0);
}

// ---- one Arnoldi step in one launch: a thread-block cluster ----------------
// The CTAs of one cluster each own a slice of the basis vectors, staged once
// into shared memory (when it fits) because every phase reads it.  Every
// pass's partial inner products (and the partial squared norm) sit in each
// CTA's shared memory; after a cluster barrier every CTA sums all ranks'
// partials through distributed shared memory in rank order, so all CTAs
// hold bitwise identical coefficients.  CGS2: two projection passes, then
// normalisation and (rank 0, one thread) the Givens update.  Replaces the
// four launches of the grid version with one; the barriers are the
// cluster's hardware barrier, reached by every thread of every CTA.
constexpr int CLT = 256;                 // threads per CTA of the cluster kernel
constexpr int CL_MAX = 16;               // largest cluster
constexpr int VS_CAP = 200 * 1024;       // shared-memory cap of the staged basis slice

// Partial inner products <v_i, w>, i = 0..j, on a slice.  GB300 issues
// few FP64 instructions per clock, so the layout minimises them: groups of
// 8 lanes own one inner product (four per warp), each lane sums every 8th
// element with two accumulators, and three shuffle steps finish the group.
template <bool C>
__device__ __forceinline__ void slice_dots(const double2* __restrict__ Vb, int ld,
                                           const double2* __restrict__ ws, int ns, int j,
                                           double2* out, int warp, int lane) {
  constexpr int NWARP = CLT / 32;
  const int grp = lane >> 3, sub = lane & 7;
  for (int base = warp * 4; base <= j; base += NWARP * 4) {
    const int i = base + grp;
    const bool live = i <= j;
    double2 s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);
    if (live) {
      const double2* vr = Vb + (size_t)i * ld;
      int q = sub;
      for (; q + 8 < ns; q += 16) {
        const double2 x0 = vr[q], y0 = ws[q], x1 = vr[q + 8], y1 = ws[q + 8];
        if (C) {
          s0.x += x0.x * y0.x + x0.y * y0.y;
          s0.y += x0.x * y0.y - x0.y * y0.x;
          s1.x += x1.x * y1.x + x1.y * y1.y;
          s1.y += x1.x * y1.y - x1.y * y1.x;
        } else {
          s0.x += x0.x * y0.x;
          s1.x += x1.x * y1.x;
        }
      }
      if (q < ns) {
        const double2 x0 = vr[q], y0 = ws[q];
        if (C) {
          s0.x += x0.x * y0.x + x0.y * y0.y;
          s0.y += x0.x * y0.y - x0.y * y0.x;
        } else {
          s0.x += x0.x * y0.x;
        }
      }
      s0.x += s1.x;
      if (C) s0.y += s1.y;
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      s0.x += __shfl_xor_sync(0xffffffffu, s0.x, o);
      if (C) s0.y += __shfl_xor_sync(0xffffffffu, s0.y, o);
    }
    if (live && sub == 0) out[i] = s0;
  }
}

// Sum of entry i over the cluster's ranks, as a fixed pairwise tree (the
// same value in every CTA).
template <bool C>
__device__ __forceinline__ double2 cl_sum(cooperative_groups::cluster_group& cl, double2* buf,
                                          int i, int CL) {
  double2 v[CL_MAX];
#pragma unroll
  for (int r = 0; r < CL_MAX; ++r)
    v[r] = r < CL ? cl.map_shared_rank(buf, r)[i] : make_double2(0.0, 0.0);
#pragma unroll
  for (int w = 1; w < CL_MAX; w <<= 1)
#pragma unroll
    for (int r = 0; r + w < CL_MAX; r += 2 * w) {
      v[r].x += v[r + w].x;
      if (C) v[r].y += v[r + w].y;
    }
  return v[0];
}

// Sum over i in {i0, i0 + step, ...} <= j of h_i V[i][e] with two
// accumulators (i0, i0 + 2 step, ... and i0 + step, i0 + 3 step, ...)
// added at the end.
template <bool C>
__device__ __forceinline__ double2 hv_sum(const double2* __restrict__ Vb, int ld, int e, int j,
                                          const double2* h, int i0, int step) {
  double2 a0 = make_double2(0.0, 0.0), a1 = make_double2(0.0, 0.0);
  int i = i0;
  for (; i + step <= j; i += 2 * step) {
    const double2 v0 = Vb[(size_t)i * ld + e], g0 = h[i];
    const double2 v1 = Vb[(size_t)(i + step) * ld + e], g1 = h[i + step];
    if (C) {
      a0.x += g0.x * v0.x - g0.y * v0.y;
      a0.y += g0.x * v0.y + g0.y * v0.x;
      a1.x += g1.x * v1.x - g1.y * v1.y;
      a1.y += g1.x * v1.y + g1.y * v1.x;
    } else {
      a0.x += g0.x * v0.x;
      a1.x += g1.x * v1.x;
    }
  }
  if (i <= j) {
    const double2 v0 = Vb[(size_t)i * ld + e], g0 = h[i];
    if (C) {
      a0.x += g0.x * v0.x - g0.y * v0.y;
      a0.y += g0.x * v0.y + g0.y * v0.x;
    } else {
      a0.x += g0.x * v0.x;
    }
  }
  return make_double2(a0.x + a1.x, a0.y + a1.y);
}

// w -= V h on a slice.  When the slice has at most CLT / 2 elements two
// threads share an element (even and odd i), combined in a fixed order;
// every thread of the CTA reaches both barriers.
template <bool C>
__device__ __forceinline__ void slice_update(const double2* __restrict__ Vb, int ld,
                                             double2* __restrict__ ws, int ns, int j,
                                             const double2* h, double2* tmp) {
  const int t = threadIdx.x;
  if (2 * ns <= CLT) {
    const int par = t < ns ? 0 : 1;
    const int e = par ? t - ns : t;
    const bool mine = t < 2 * ns;
    double2 a = make_double2(0.0, 0.0);
    if (mine) a = hv_sum<C>(Vb, ld, e, j, h, par, 2);
    if (mine && par == 1) tmp[e] = a;
    __syncthreads();
    if (mine && par == 0) {
      const double2 o = tmp[e];
      ws[e] = make_double2(ws[e].x - (a.x + o.x), ws[e].y - (a.y + o.y));
    }
    __syncthreads();
  } else {
    for (int e = t; e < ns; e += CLT) {
      const double2 a = hv_sum<C>(Vb, ld, e, j, h, 0, 1);
      ws[e] = make_double2(ws[e].x - a.x, ws[e].y - a.y);
    }
    __syncthreads();
  }
}

template <bool C>
__global__ void __launch_bounds__(CLT) k_arnoldi_cl(double2* __restrict__ V, int nb, int j,
                                                    double2* __restrict__ w, double2* H, double* cs,
                                                    double2* sn, double2* g, int m, double* scal,
                                                    int cached, double* mbox, long long seq) {
  KFBI_PDL_ENTRY();
  // a step queued ahead of an earlier step that converged does nothing
  // (every CTA of the cluster reads the same flag and returns together)
  KFBI_STOP_RETURN(scal + 2);
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double2 vs[];  // staged basis slice, [i][e - e0]
  const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  __shared__ double2 pa[65], pb[65], h1[65], h2[65], tmp[CLT], gcol[66], gsn[65], gg[66];
  __shared__ double gcs[65];
  __shared__ double pn[CLT / 32];
  __shared__ double pnorm, s_hn, s_inv;
  const int slice = (nb + CL - 1) / CL;
  const int e0 = min(nb, rank * slice), e1 = min(nb, e0 + slice), ns = e1 - e0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double2* Vb;  // row i of this slice at Vb + i * ld
  int ld;
  if (cached) {
    for (int q = threadIdx.x; q < (j + 1) * ns; q += CLT) {
      const int i = q / ns, e = q - i * ns;
      vs[i * slice + e] = V[(size_t)i * nb + e0 + e];
    }
    __syncthreads();
    Vb = vs;
    ld = slice;
  } else {
    Vb = V + e0;
    ld = nb;
  }
  double2* ws = w + e0;
  if (rank == 0) {
    // the stored rotations and g: written by earlier steps, read only at the
    // end; loading them now overlaps their latency with the inner products
    for (int i = threadIdx.x; i <= j + 1; i += CLT) {
      if (i < j) {
        gcs[i] = cs[i];
        gsn[i] = sn[i];
      }
      gg[i] = g[i];
    }
  }
  // pass 1: <v_i, w> on this slice
  slice_dots<C>(Vb, ld, ws, ns, j, pa, warp, lane);
  cl.sync();
  for (int i = threadIdx.x; i <= j; i += CLT) h1[i] = cl_sum<C>(cl, pa, i, CL);
  __syncthreads();
  slice_update<C>(Vb, ld, ws, ns, j, h1, tmp);
  __syncthreads();
  // pass 2 (reorthogonalisation)
  slice_dots<C>(Vb, ld, ws, ns, j, pb, warp, lane);
  cl.sync();
  for (int i = threadIdx.x; i <= j; i += CLT) h2[i] = cl_sum<C>(cl, pb, i, CL);
  __syncthreads();
  slice_update<C>(Vb, ld, ws, ns, j, h2, tmp);
  __syncthreads();
  double ss = 0.0;
  for (int e = threadIdx.x; e < ns; e += CLT) ss += ws[e].x * ws[e].x + ws[e].y * ws[e].y;
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane == 0) pn[warp] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[CLT / 32];
#pragma unroll
    for (int q = 0; q < CLT / 32; ++q) t[q] = pn[q];
#pragma unroll
    for (int w2 = 1; w2 < CLT / 32; w2 <<= 1)
#pragma unroll
      for (int q = 0; q + w2 < CLT / 32; q += 2 * w2) t[q] += t[q + w2];
    pnorm = t[0];
  }
  cl.sync();
  if (threadIdx.x < 32) {
    // lane r < CL reads rank r's partial norm (every thread of the cluster
    // reading them all piled 4096 remote loads per CTA on 16 words); the
    // pairwise tree by shuffles adds in the same fixed order on every CTA
    double v = lane < CL ? *cl.map_shared_rank(&pnorm, lane) : 0.0;
#pragma unroll
    for (int w2 = 1; w2 < CL_MAX; w2 <<= 1) {
      const double o = __shfl_down_sync(0xffffffffu, v, w2);
      if ((lane & (2 * w2 - 1)) == 0) v += o;
    }
    if (lane == 0) {
      s_hn = sqrt(v);
      s_inv = s_hn > 0.0 ? 1.0 / s_hn : 0.0;
    }
  }
  __syncthreads();
  // that was the last read of a peer's shared memory: arrive on the
  // cluster barrier now, wait for the peers only before leaving
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  const double hn = s_hn;
  const double inv = s_inv;
  double2* vn = V + (size_t)(j + 1) * nb + e0;
  for (int e = threadIdx.x; e < ns; e += CLT) vn[e] = make_double2(ws[e].x * inv, ws[e].y * inv);
  if (rank == 0) {
    // the new column joins the rotations and g staged at the start, so the
    // sequential rotation chain waits on no global loads
    for (int i = threadIdx.x; i <= j; i += CLT)
      gcol[i] = make_double2(h1[i].x + h2[i].x, h1[i].y + h2[i].y);
    __syncthreads();
    if (threadIdx.x < 32) rotate_column_warp<C>(gcol, j, gcs, gsn, threadIdx.x);
    if (threadIdx.x == 0) {
      givens_new<C>(gcol, j, hn, gcs, gsn, gg, scal);
      mbox_post(scal, mbox, seq);
    }
    __syncthreads();
    double2* col = H + (size_t)j * (m + 1);
    for (int i = threadIdx.x; i <= j + 1; i += CLT) {
      col[i] = gcol[i];
      g[i] = gg[i];
    }
    if (threadIdx.x == 0) {
      cs[j] = gcs[j];
      sn[j] = gsn[j];
    }
  }
  // no CTA leaves while a peer may still read its shared memory
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// x += V[:, :k] y with R y = g: the CTA stages the triangle of R in shared
// memory, one warp solves it (row sums across lanes), then the CTA updates
// its slice.
__global__ void __launch_bounds__(GT) k_update_grid(const double2* __restrict__ V, int nb, int k,
                                                    const double2* H, const double2* g, int m,
                                                    double2* __restrict__ x, int slice) {
  KFBI_PDL_ENTRY();
  __shared__ double2 y[64], gs[64];
  __shared__ double2 R[64 * 65 / 2];  // R[l (l + 1) / 2 + i] = H(i, l), i <= l < k <= 64
  const int b = blockIdx.x;
  const int e0 = b * slice, e1 = min(nb, e0 + slice);
  // the triangle and g in one round of independent loads (the solve below
  // is a serial chain and must not wait on global memory)
  for (int t = threadIdx.x; t < k * (k + 1) / 2; t += GT) {
    int l = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while (l * (l + 1) / 2 > t) --l;
    while ((l + 1) * (l + 2) / 2 <= t) ++l;
    R[t] = H[(size_t)l * (m + 1) + (t - l * (l + 1) / 2)];
  }
  for (int i = threadIdx.x; i < k; i += GT) gs[i] = g[i];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = k - 1; i >= 0; --i) {
      double2 s = make_double2(0.0, 0.0);
      for (int l = i + 1 + lane; l < k; l += 32) {
        const double2 t = cmul(R[l * (l + 1) / 2 + i], y[l]);
        s.x += t.x;
        s.y += t.y;
      }
      for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      }
      if (lane == 0) {
        const double2 r = make_double2(gs[i].x - s.x, gs[i].y - s.y);
        const double2 d = R[i * (i + 1) / 2 + i];
        const double inv = 1.0 / (d.x * d.x + d.y * d.y);
        y[i] = make_double2((r.x * d.x + r.y * d.y) * inv, (r.y * d.x - r.x * d.y) * inv);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = e0 + threadIdx.x; e < e1; e += GT) {
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

void check_device_flags(kfbi_domain* D) {
  int flags = 0;
  std::memcpy(&flags, D->h_scal + 6, sizeof(int));
  if (flags != 0)
    throw Status{KFBI_ERR_TIMEOUT,
                 "a tensor-core DST pass gave up waiting on its pipeline (flags " +
                     std::to_string(flags) + ")"};
}

// Device bytes gmres_alloc takes for restart m and nb boundary nodes.
long long gmres_bytes(int m, int nb) {
  const size_t n = (size_t)(m + 1) * 2 * nb + 3 * 2 * (size_t)nb + (size_t)(m + 1) * m * 2 + m +
                   2 * (size_t)m + 2 * (size_t)(m + 1) + 2 * 2 * (size_t)(m + 1) * GMAX +
                   2 * (size_t)(m + 1) + 3 * 2 * (size_t)nb + 8;
  return (long long)(n * sizeof(double));
}

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
  alloc(&D->d_part, 2 * 2 * (size_t)(m + 1) * GMAX);
  alloc(&D->d_hcol, 2 * (size_t)(m + 1));
  alloc(&D->d_Rv, 2 * (size_t)nb);
  alloc(&D->d_Dv, 2 * (size_t)nb);
  alloc(&D->d_Ax, 2 * (size_t)nb);
  alloc(&D->d_scal, 8);
  KFBI_CUDA(cudaMemset(D->d_scal, 0, 8 * sizeof(double)));
  KFBI_CUDA(cudaMallocHost(&D->h_scal, 8 * sizeof(double)));
  std::memset(D->h_scal, 0, 8 * sizeof(double));
  KFBI_CUDA(cudaHostAlloc(&D->h_mbox, 32 * sizeof(double), cudaHostAllocMapped));
  std::memset(D->h_mbox, 0, 32 * sizeof(double));
  KFBI_CUDA(cudaHostGetDevicePointer((void**)&D->d_mbox, D->h_mbox, 0));
  D->mbox_seq = 0;
}

void gmres_free(kfbi_domain* D) {
  double* ptrs[] = {D->d_V,  D->d_W,  D->d_X,  D->d_B,  D->d_H,    D->d_cs,   D->d_sn,
                    D->d_g,  D->d_Rv, D->d_Dv, D->d_Ax, D->d_part, D->d_hcol, D->d_scal};
  for (double* p : ptrs)
    if (p) cudaFree(p);
  if (D->h_scal) cudaFreeHost(D->h_scal);
  D->h_scal = nullptr;
  if (D->h_mbox) cudaFreeHost(D->h_mbox);
  D->h_mbox = nullptr;
  D->d_mbox = nullptr;
}

static void read_scalars(kfbi_domain* D, cudaStream_t st) {
  KFBI_CUDA(cudaMemcpyAsync(D->h_scal, D->d_scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
  KFBI_CUDA(cudaStreamSynchronize(st));
  check_device_flags(D);
}

// Next sequence number of the scalar mailbox (never 0, the initial content).
static long long next_post(kfbi_domain* D) { return ++D->mbox_seq; }

// The scalars a kernel posted with sequence number q (mbox_post): poll the
// mapped slot; should the stream drain without that post (a kernel that
// returned early), fall back to copying the scalars after the stream.
static void wait_post(kfbi_domain* D, long long q, cudaStream_t st) {
  volatile double* slot = D->h_mbox + 16 * (q & 1);
  volatile long long* seq = reinterpret_cast<volatile long long*>(slot + 8);
  const auto t0 = std::chrono::steady_clock::now();
  for (long long spins = 1; *seq != q; ++spins) {
    if ((spins & 255) != 0) continue;
    const cudaError_t e = cudaStreamQuery(st);
    if (e == cudaSuccess) {
      if (*seq == q) break;
      read_scalars(D, st);
      return;
    }
    if (e != cudaErrorNotReady) KFBI_CUDA(e);
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60))
      throw Status{KFBI_ERR_TIMEOUT, "no GMRES scalars within 60 s"};
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  for (int i = 0; i < 8; ++i) D->h_scal[i] = slot[i];
  check_device_flags(D);
}

static void grid_shape(int nb, int& G, int& slice) {
  G = (nb + 31) / 32;
  if (G > GMAX) G = GMAX;
  slice = ((nb + G - 1) / G + 31) / 32 * 32;
  G = (nb + slice - 1) / slice;
}

// One Arnoldi step on w = A v_j (in D->d_W): CGS2 over the grid kernels.
// Cluster size of the one-launch Arnoldi step: 16 CTAs where the device
// runs such clusters (a non-portable size), else 8; 0 if clusters cannot be
// launched at all (the grid version is used then).
static int probe_cluster_size() {
  int cl = 0;
  for (int want : {16, 8}) {
    if (cudaFuncSetAttribute(k_arnoldi_cl<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, VS_CAP) != cudaSuccess ||
        cudaFuncSetAttribute(k_arnoldi_cl<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, VS_CAP) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    if (want > 8) {
      if (cudaFuncSetAttribute(k_arnoldi_cl<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
          cudaFuncSetAttribute(k_arnoldi_cl<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(want, 1, 1);
    cfg.blockDim = dim3(CLT, 1, 1);
    cfg.dynamicSmemBytes = VS_CAP;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = want;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n1 = 0, n2 = 0;
    if (cudaOccupancyMaxActiveClusters(&n1, k_arnoldi_cl<true>, &cfg) == cudaSuccess &&
        cudaOccupancyMaxActiveClusters(&n2, k_arnoldi_cl<false>, &cfg) == cudaSuccess && n1 > 0 &&
        n2 > 0) {
      cl = want;
      break;
    }
    cudaGetLastError();
  }
  return cl;
}

static int arnoldi_cluster_size() {
  static const int cl = probe_cluster_size();  // thread-safe one-time probe
  return cl;
}

static void arnoldi_step_cluster(kfbi_domain* D, bool C, int j, int CL, cudaStream_t st,
                                 long long post = 0) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, 1, 1);
  cfg.blockDim = dim3(CLT, 1, 1);
  cfg.stream = st;
  const int slice = (D->nb + CL - 1) / CL;
  const size_t vbytes = (size_t)(j + 1) * slice * sizeof(double2);
  const int cached = vbytes <= (size_t)VS_CAP ? 1 : 0;
  cfg.dynamicSmemBytes = cached ? vbytes : 0;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  add_pdl_attr(cfg, at);
  double2* V = (double2*)D->d_V;
  double2* w = (double2*)D->d_W;
  void* tok = g_prof_on ? prof_begin(KFBI_PROF_KRYLOV, st) : nullptr;
  double* mbox = post > 0 ? D->d_mbox : nullptr;
  if (C)
    KFBI_CUDA(cudaLaunchKernelEx(&cfg, k_arnoldi_cl<true>, V, D->nb, j, w, (double2*)D->d_H, D->d_cs,
                                 (double2*)D->d_sn, (double2*)D->d_g, D->restart, D->d_scal,
                                 cached, mbox, post));
  else
    KFBI_CUDA(cudaLaunchKernelEx(&cfg, k_arnoldi_cl<false>, V, D->nb, j, w, (double2*)D->d_H,
                                 D->d_cs, (double2*)D->d_sn, (double2*)D->d_g, D->restart,
                                 D->d_scal, cached, mbox, post));
  if (tok) prof_end(tok, st);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

static void arnoldi_step(kfbi_domain* D, bool C, int j, cudaStream_t st, long long post = 0) {
  const int CL = arnoldi_cluster_size();
  if (CL > 0) {
    arnoldi_step_cluster(D, C, j, CL, st, post);
    return;
  }
  const int nb = D->nb, m = D->restart;
  int G, slice;
  grid_shape(nb, G, slice);
  double2* V = (double2*)D->d_V;
  double2* w = (double2*)D->d_W;
  double2* p1 = (double2*)D->d_part;
  double2* p2 = p1 + (size_t)(m + 1) * GMAX;
  double2* hcol = (double2*)D->d_hcol;
  if (C) {
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_cgs_dots<true>, G, GT, 0, st, V, nb, j, w, p1, slice);
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_cgs_update<true>, G, GT, 0, st, V, nb, j, w, p1, p2, hcol, 1,
                  0, slice);
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_cgs_update<true>, G, GT, 0, st, V, nb, j, w, p2, p1, hcol, 0,
                  1, slice);
  } else {
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_cgs_dots<false>, G, GT, 0, st, V, nb, j, w, p1, slice);
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_cgs_update<false>, G, GT, 0, st, V, nb, j, w, p1, p2, hcol,
                  1, 0, slice);
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_cgs_update<false>, G, GT, 0, st, V, nb, j, w, p2, p1, hcol,
                  0, 1, slice);
  }
  KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_cgs_finalize, G, GT, 0, st, V, nb, j, w, p1, hcol,
                (double2*)D->d_H, D->d_cs, (double2*)D->d_sn, (double2*)D->d_g, m, D->d_scal,
                slice);
  KFBI_CHECK_LAUNCH();
}

// Sets the sparse-route stop flag of a mixed domain for the lifetime of a
// GMRES call that queues iterations ahead, and clears it on every exit.
struct StopScope {
  TcDst* T;
  StopScope(kfbi_domain* D, bool on) : T(on ? D->tc : nullptr) {
    if (T) T->stop = D->d_scal + 2;
  }
  ~StopScope() {
    if (T) T->stop = nullptr;
  }
};

// GMRES(m) with the domain's hot-path operator (apply_internal), relative
// tolerance tol, at most maxit iterations.
//
// Mixed domains with the cluster Arnoldi step queue one iteration ahead:
// iteration j + 1 (and iteration 0, ahead of the restart's check) is in the
// stream before the host reads iteration j's residual, so the GPU does not
// wait for the host between iterations; the exception is an iteration that
// the residual history predicts to be the last one (the previous residual
// times the previous reduction ratio within 3x of the target).  The restart
// and Arnoldi kernels post their scalars to a two-slot host-mapped mailbox
// (mbox_post), so no copy or event sits between the kernels of consecutive
// iterations; the host polls post q before it queues the kernel that posts
// q + 2 into the same slot.  When iteration j converged, the queued
// iteration j + 1 finds the convergence flag set and its kernels return at
// once; it would only have written H column j + 1, g[j + 1 .. j + 2] and
// V[j + 2], none of which the update with k = j + 1 reads.
// A first cycle already in the stream (the refinement queues it behind its
// residual check, k_residual_restart): the restart's post and iteration 0's.
struct Prestart {
  long long q0;
  long long qj0;
};

static kfbi_status gmres_core(kfbi_domain* D, double kre, double kim, const double* b, double* x,
                              bool x_zero, double tol, int maxit, kfbi_solve_info* info,
                              cudaStream_t st, const Prestart* pre = nullptr) {
  const int m = D->restart, nb = D->nb;
  const bool C = kim != 0.0;
  double2* V = (double2*)D->d_V;
  double2* W = (double2*)D->d_W;
  double2* H = (double2*)D->d_H;
  double2* g = (double2*)D->d_g;
  const bool ahead = D->tc && D->n_irr > 0 && arnoldi_cluster_size() > 0;
  StopScope scope(D, ahead);
  // with lookahead the restart and Arnoldi kernels post their scalars to the
  // mapped mailbox (sequence numbers qj[j] for iteration j)
  std::vector<long long> qj(m + 1, 0);
  auto iterate = [&](int j) {
    apply_internal(D, kre, kim, (const double*)(V + (size_t)j * nb), 2, nullptr, D->d_W, 2,
                   false, st);
    qj[j] = ahead ? next_post(D) : 0;
    arnoldi_step(D, C, j, st, qj[j]);
  };
  // from x = 0 the first restart takes ||b|| itself
  if (!x_zero && !pre)
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_bnorm, 1, kThreads, 0, st, (const double2*)b, nb, D->d_scal, tol);
  int it = 0;
  bool first = true;
  kfbi_status status = KFBI_OK;
  if (info) *info = kfbi_solve_info{0, 0.0, 0, 0};
  for (;;) {
    const bool skip_ax = first && x_zero;
    const bool queued_first = first && pre && ahead;
    long long q0 = 0;
    if (queued_first) {
      q0 = pre->q0;
      qj[0] = pre->qj0;
    } else {
      if (!skip_ax) apply_internal(D, kre, kim, x, 2, nullptr, D->d_W, 2, false, st);
      q0 = ahead ? next_post(D) : 0;
      KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_restart, 1, kThreads, 0, st, (const double2*)b, skip_ax ? nullptr : W, V, g, m,
                  nb, D->d_scal, ahead ? D->d_mbox : nullptr, q0, skip_ax ? tol : -1.0);
      KFBI_CHECK_LAUNCH();
    }
    if (ahead) {
      if (it < maxit && !queued_first) iterate(0);
      wait_post(D, q0, st);
    } else {
      read_scalars(D, st);
    }
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
    int queued = ahead && it < maxit ? 0 : -1;  // last iteration of this cycle in the stream
    double res1 = D->h_scal[1], res2 = 0.0;      // residual estimates after j - 1 and j - 2
    for (int j = 0; j < m; ++j) {
      if (ahead) {
        if (queued < j) {
          iterate(j);
          queued = j;
        }
        // queue j + 1 before reading j, unless j is expected to converge:
        // GMRES residuals fall at a fairly steady rate, and a queued
        // iteration after convergence still costs its (early-exiting)
        // launches
        const double target = D->h_scal[3] * D->h_scal[0];
        const bool likely_last = res2 > 0.0 && res1 * (res1 / res2) <= 3.0 * target;
        if (j + 1 < m && it + 2 <= maxit && !likely_last) {
          iterate(j + 1);
          queued = j + 1;
        }
        wait_post(D, qj[j], st);
        res2 = res1;
        res1 = D->h_scal[1];
      } else {
        iterate(j);
        read_scalars(D, st);
      }
      ++it;
      k = j + 1;
      if (D->h_scal[2] != 0.0 || it >= maxit) break;
    }
    {
      int G, slice;
      grid_shape(nb, G, slice);
      KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_update_grid, G, GT, 0, st, V, nb, k, H, g, m,
                    (double2*)x, slice);
      KFBI_CHECK_LAUNCH();
    }
    if (D->h_scal[2] != 0.0 || it >= maxit) break;
  }
  // the scalars already came from the mailbox; without it, the last read
  // is still in flight behind the update
  if (!ahead) KFBI_CUDA(cudaStreamSynchronize(st));
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

namespace gm {
// r = b - Ax (Ax null: r = b) and scal[1] = ||r||.
__global__ void __launch_bounds__(kThreads) k_residual(const double2* __restrict__ b,
                                                        const double2* __restrict__ Ax,
                                                        double2* __restrict__ r, int nb,
                                                        double* scal, double* mbox, long long seq) {
  KFBI_PDL_ENTRY();
  __shared__ double red[32];
  double s = 0.0;
  for (int e = threadIdx.x; e < nb; e += kThreads) {
    double2 v = b[e];
    if (Ax) {
      v.x -= Ax[e].x;
      v.y -= Ax[e].y;
    }
    r[e] = v;
    s += v.x * v.x + v.y * v.y;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    scal[1] = sqrt(s);
    mbox_post(scal, mbox, seq);
  }
}

__global__ void k_axpy(double2* __restrict__ x, const double2* __restrict__ d, int nb) {
  KFBI_PDL_ENTRY();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nb) {
    x[e].x += d[e].x;
    x[e].y += d[e].y;
  }
}
}  // namespace gm

namespace gm {
// Richardson scalars (scal): [0] ||b||, [1] ||r|| of the last step, [2] status
// (0 running, 1 converged, 2 non-finite, 3 maxit updates made), [3] tol,
// [4] updates made, [5] ||r|| of the step before the last.
__global__ void __launch_bounds__(kThreads) k_richardson_init(const double2* __restrict__ b,
                                                              int nb, double* scal, double tol) {
  KFBI_PDL_ENTRY();
  __shared__ double red[32];
  double s = 0.0;
  for (int e = threadIdx.x; e < nb; e += kThreads) s += b[e].x * b[e].x + b[e].y * b[e].y;
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    scal[0] = sqrt(s);
    scal[1] = 0.0;
    scal[2] = 0.0;
    scal[3] = tol;
    scal[4] = 0.0;
    scal[5] = 0.0;
  }
}

// One step of Eq. 3.21 after the application Ax = A x (Ax null: x = 0):
// r = b - Ax and its 2-norm, then, in this order,
//   ||b|| = 0                 -> x = 0, converged;
//   ||r|| <= tol ||b||        -> converged, x kept;
//   ||r|| not finite          -> status 2;
//   maxit updates already made -> status 3, x kept;
//   otherwise x += gamma r and one more update counted.
// A step queued behind one that set the status returns at once, so steps
// may be queued ahead of the host's convergence check.
__global__ void __launch_bounds__(kThreads) k_richardson_step(const double2* __restrict__ b,
                                                              const double2* __restrict__ Ax,
                                                              double2* __restrict__ x, int nb,
                                                              double gamma, int maxit,
                                                              double* scal) {
  KFBI_PDL_ENTRY();
  KFBI_STOP_RETURN(scal + 2);
  __shared__ double red[32];
  // every thread reads the scalars before the block_sum barriers; thread 0
  // writes them only after
  const double bn = scal[0], tol = scal[3], made = scal[4], last = scal[1];
  double s = 0.0;
  for (int e = threadIdx.x; e < nb; e += kThreads) {
    double2 r = b[e];
    if (Ax) {
      r.x -= Ax[e].x;
      r.y -= Ax[e].y;
    }
    s += r.x * r.x + r.y * r.y;
  }
  s = block_sum(s, red);
  const double rn = sqrt(s);
  int status = 0;
  if (bn == 0.0)
    status = 1;
  else if (rn <= tol * bn)
    status = 1;
  else if (!isfinite(rn))
    status = 2;
  else if (made >= (double)maxit)
    status = 3;
  if (status == 0 || bn == 0.0) {
    for (int e = threadIdx.x; e < nb; e += kThreads) {
      double2 v = make_double2(0.0, 0.0);
      if (bn != 0.0) {
        double2 r = b[e];
        if (Ax) {
          r.x -= Ax[e].x;
          r.y -= Ax[e].y;
        }
        v = x[e];
        v.x += gamma * r.x;
        v.y += gamma * r.y;
      }
      x[e] = v;
    }
  }
  if (threadIdx.x == 0) {
    scal[5] = last;
    scal[1] = bn == 0.0 ? 0.0 : rn;
    scal[2] = (double)status;
    if (status == 0) scal[4] = made + 1.0;
  }
}
}  // namespace gm

// The Richardson iteration of Eq. 3.21, phi <- phi + gamma (b - A phi), with
// the domain's hot-path operator (apply_internal), relative tolerance tol and
// at most maxit updates.  Each step is one application and one
// k_richardson_step; steps are queued in runs whose length the host
// predicts from the residual reduction it has seen (the residual of a
// Richardson iteration falls by a nearly constant factor, the spectral
// radius of I - gamma A), and the host reads the scalars once per run.  Steps
// queued past convergence do nothing: the step kernel returns at once and,
// on a mixed domain with irregular nodes, so do the kernels of the
// application (the sparse route's stop flag).
static kfbi_status richardson_core(kfbi_domain* D, double kre, double kim, const double* b,
                                   double* x, bool x_zero, double tol, int maxit,
                                   kfbi_solve_info* info, cudaStream_t st) {
  const int nb = D->nb;
  const double gamma = D->desc.richardson_gamma;
  const bool cheap_tail = D->tc && D->n_irr > 0;
  StopScope scope(D, cheap_tail);
  KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_richardson_init, 1, kThreads, 0, st, (const double2*)b, nb,
                D->d_scal, tol);
  KFBI_CHECK_LAUNCH();
  if (info) *info = kfbi_solve_info{0, 0.0, 0, 0};
  const long long cap = (long long)maxit + 1;  // steps that can still act
  long long queued = 0;
  // first run: on x = 0 (r_0 = b) with the rate of an earlier solve at the
  // same kappa, the steps until rate^k <= tol plus the step that sees it;
  // otherwise a short run to measure the rate on
  int run = cheap_tail ? 8 : 2;
  const bool known = D->rich_rate > 0.0 && D->rich_rate < 0.999 && D->rich_kre == kre &&
                     D->rich_kim == kim;
  if (x_zero && known) {
    const double k = std::ceil(std::log(tol) / std::log(D->rich_rate));
    run = (int)std::min(std::max(k + 1.0 + (cheap_tail ? 1.0 : 0.0), 1.0), 256.0);
  }
  double res_prev = 0.0, rate = 0.0;
  long long q_prev = 0;
  for (;;) {
    const long long n = std::min<long long>(run, cap - queued);
    for (long long i = 0; i < n; ++i, ++queued) {
      const bool skip = queued == 0 && x_zero;
      if (!skip) apply_internal(D, kre, kim, x, 2, nullptr, D->d_W, 2, false, st);
      KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_richardson_step, 1, kThreads, 0, st, (const double2*)b,
                    skip ? nullptr : (const double2*)D->d_W, (double2*)x, nb, gamma, maxit,
                    D->d_scal);
      KFBI_CHECK_LAUNCH();
    }
    read_scalars(D, st);
    if (D->h_scal[2] != 0.0 || queued >= cap) break;
    // reduction per step: over the steps since the last read, else over the
    // last step alone
    const double res = D->h_scal[1];
    rate = 0.0;
    if (res_prev > 0.0 && queued > q_prev)
      rate = std::pow(res / res_prev, 1.0 / (double)(queued - q_prev));
    else if (D->h_scal[5] > 0.0)
      rate = res / D->h_scal[5];
    res_prev = res;
    q_prev = queued;
    const double target = tol * D->h_scal[0];
    if (rate > 0.0 && rate < 0.999 && res > target) {
      // steps until the residual of a step falls below the target: the
      // last one read is r_(queued-1), the next step computes r_queued
      const double need = std::ceil(std::log(target / res) / std::log(rate));
      run = (int)std::min(std::max(need + (cheap_tail ? 1.0 : 0.0), 1.0), 256.0);
    } else {
      run = std::min(2 * run, 256);
    }
  }
  const int made = (int)D->h_scal[4];
  const int status = (int)D->h_scal[2];
  if (status == 1 && x_zero && made >= 2 && D->h_scal[0] > 0.0 && D->h_scal[1] > 0.0)
    rate = std::pow(D->h_scal[1] / D->h_scal[0], 1.0 / made);  // r_0 = b
  if (status == 1 && rate > 0.0 && rate < 0.999) {
    D->rich_rate = rate;
    D->rich_kre = kre;
    D->rich_kim = kim;
  }
  if (info) {
    info->iters = made;
    // applications whose residual the iteration used: every step that did
    // not return at once, less a first step on x = 0 (steps queued past
    // the stop are not counted)
    const int active = made + (status != 0 ? 1 : 0);
    info->applications = active - (x_zero && active > 0 ? 1 : 0);
    info->rel_residual = D->h_scal[0] > 0.0 ? D->h_scal[1] / D->h_scal[0] : 0.0;
    info->converged = status == 1;
  }
  if (status == 2) {
    D->err = "non-finite Richardson residual";
    return KFBI_ERR_NONFINITE;
  }
  if (status != 1) {
    D->err = "Richardson iteration reached gmres_maxit";
    return KFBI_ERR_NOT_CONVERGED;
  }
  return KFBI_OK;
}

// Inner solver of the domain (kfbi_solver).
static kfbi_status inner_solve(kfbi_domain* D, double kre, double kim, const double* b, double* x,
                               bool x_zero, double tol, int maxit, kfbi_solve_info* info,
                               cudaStream_t st, const Prestart* pre = nullptr) {
  if (D->desc.solver == KFBI_RICHARDSON)
    return richardson_core(D, kre, kim, b, x, x_zero, tol, maxit, info, st);
  return gmres_core(D, kre, kim, b, x, x_zero, tol, maxit, info, st, pre);
}

// Relative tolerance below which the inner solves of the refinement do not
// go: the TF32x3 operator is accurate to ~2e-6, so tighter inner solves
// only add iterations.
static const double kInnerFloor = 1e-6;

// Relative L-infinity error bound of a fast (unrefined) application, as the
// mixed and FFT operator tests state it.  In the 2-norm of an nb-vector the
// relative error is at most sqrt(nb) times that.
static const double kFastRelLinf = 2e-5;

kfbi_status gmres_solve(kfbi_domain* D, double kre, double kim, const double* b, double* x,
                        bool x_zero, kfbi_solve_info* info, cudaStream_t st, const double* ax0,
                        double* ax_out, bool* grid_wx) {
  const double tol = D->desc.gmres_tol;
  const int maxit = D->desc.gmres_maxit;
  if (grid_wx) *grid_wx = false;
  if (!D->tc) return inner_solve(D, kre, kim, b, x, x_zero, tol, maxit, info, st);
  // Mixed domain: iterative refinement.  The residual of the density,
  // r = b - A phi, uses the accurate operator (apply_accurate, FP64 vector
  // arithmetic); the corrections solve A_mixed d = r with the fast TF32x3
  // operator inside GMRES.
  const int nb = D->nb;
  const dim3 vb((nb + 255) / 256);
  // ||b|| goes to scal[0]; it is read with the first residual (one host
  // round trip instead of two), before the inner solves reuse the slot
  KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_bnorm, 1, kThreads, 0, st, (const double2*)b, nb, D->d_scal,
                tol);
  double bnorm = 0.0;
  int it = 0, apps = 0;
  double rn = 0.0;
  bool conv = false;
  kfbi_status status = KFBI_OK;
  bool fresh = false;  // D->d_Ax and D->d_U come from an application at the current x
  // A correction d from an inner solve satisfies |A d| <= 2 |r| (r the
  // residual it was solved for).  Once |r| is so small that the unrefined
  // error of A d, 2 sqrt(nb) kFastRelLinf |r|, is below a tenth of the
  // tolerance, the check at x + d reuses the last accurate grid and applies
  // only d (tc_apply_correction); the residual test then subtracts that
  // bound, so the refined result still meets the tolerance.
  const double fast_rel = kFastRelLinf * std::sqrt((double)nb);
  // the inner solver queues ahead through the mailbox (gmres_core's lookahead)
  const bool lookahead = D->desc.solver != KFBI_RICHARDSON && D->n_irr > 0 &&
                         arnoldi_cluster_size() > 0;
  double r_prev = 0.0;     // residual the last correction was solved for
  double err_bound = 0.0;  // bound on |A x - d_Ax| (corrections since the last full application)
  for (int sweep = 0; sweep < 8; ++sweep) {
    const bool skip = sweep == 0 && x_zero;
    const double* ax = skip ? nullptr : D->d_Ax;
    const bool grid_at_prev = fresh;
    fresh = false;
    if (!skip) {
      const double e = err_bound + 2.0 * fast_rel * r_prev;
      if (sweep == 0 && ax0) {
        ax = ax0;  // A x of the incoming x, kept by the caller (superposition)
        err_bound = 0.0;
      } else if (sweep > 0 && grid_at_prev && !D->neumann && e <= 0.1 * tol * bnorm) {
        tc_apply_correction(D, kre, kim, D->d_Dv, x, 2, D->d_Ax, 2, st);
        ++apps;
        fresh = true;
        err_bound = e;
      } else {
        apply_accurate(D, kre, kim, x, 2, nullptr, D->d_Ax, 2, st);
        ++apps;
        fresh = true;
        err_bound = 0.0;
      }
    }
    // With the GMRES inner solver on the mailbox path, the residual check
    // also starts the inner solve (k_residual_restart) and its first
    // iteration is queued before the host reads the residual: if the check
    // converged, that iteration finds the GMRES status set and returns.
    const bool spec = lookahead && it < maxit;
    Prestart pre{};
    long long q = 0;
    if (spec) {
      KFBI_CUDA(cudaMemsetAsync(D->d_Dv, 0, 2 * (size_t)nb * sizeof(double), st));
      q = next_post(D);
      KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_residual_restart, 1, kThreads, 0, st, (const double2*)b,
                    (const double2*)ax, (double2*)D->d_Rv, (double2*)D->d_V, (double2*)D->d_g,
                    D->restart, nb, D->d_scal, D->d_mbox, q, tol, kInnerFloor);
      KFBI_CHECK_LAUNCH();
      StopScope scope(D, true);
      apply_internal(D, kre, kim, D->d_V, 2, nullptr, D->d_W, 2, false, st);
      pre.q0 = q;
      pre.qj0 = next_post(D);
      arnoldi_step(D, kim != 0.0, 0, st, pre.qj0);
    } else {
      q = next_post(D);
      KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_residual, 1, kThreads, 0, st, (const double2*)b,
                    (const double2*)ax, (double2*)D->d_Rv, nb, D->d_scal, D->d_mbox, q);
      KFBI_CHECK_LAUNCH();
    }
    wait_post(D, q, st);
    if (sweep == 0) bnorm = D->h_scal[spec ? 7 : 0];
    rn = D->h_scal[1];
    if (!std::isfinite(rn)) {
      D->err = "non-finite density residual";
      status = KFBI_ERR_NONFINITE;
      break;
    }
    if (bnorm == 0.0) {  // b = 0: x = 0, whatever the initial guess
      KFBI_CUDA(cudaMemsetAsync(x, 0, 2 * (size_t)nb * sizeof(double), st));
      fresh = false;
      rn = 0.0;
      conv = true;
      break;
    }
    if (rn + err_bound <= tol * bnorm) {
      conv = true;
      break;
    }
    if (it >= maxit) break;
    r_prev = rn;
    const double inner_tol = std::max(0.5 * tol * bnorm / rn, kInnerFloor);
    if (!spec) KFBI_CUDA(cudaMemsetAsync(D->d_Dv, 0, 2 * (size_t)nb * sizeof(double), st));
    kfbi_solve_info in{};
    kfbi_status s = inner_solve(D, kre, kim, D->d_Rv, D->d_Dv, true, inner_tol, maxit - it, &in,
                                st, spec ? &pre : nullptr);
    it += in.iters;
    apps += in.applications;
    if (s == KFBI_ERR_NONFINITE) {
      status = s;
      break;
    }
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_axpy, vb, 256, 0, st, (double2*)x, (const double2*)D->d_Dv,
                  nb);
    KFBI_CHECK_LAUNCH();
  }
  if (conv && fresh && ax_out) {
    KFBI_CUDA(cudaMemcpyAsync(ax_out, D->d_Ax, 2 * (size_t)nb * sizeof(double),
                              cudaMemcpyDeviceToDevice, st));
    if (grid_wx) *grid_wx = true;
  }
  if (info) {
    info->iters = it;
    info->applications = apps;
    info->rel_residual = bnorm > 0.0 ? rn / bnorm : 0.0;
    info->converged = conv ? 1 : 0;
  }
  if (status == KFBI_OK && !conv) {
    D->err = "GMRES with refinement reached gmres_maxit";
    status = KFBI_ERR_NOT_CONVERGED;
  }
  // every scalar the host needed came through the mailbox; on success the
  // caller's remaining kernels queue behind the solve and the caller
  // synchronises once at its end, on failure the stream is drained here
  if (status != KFBI_OK) KFBI_CUDA(cudaStreamSynchronize(st));
  return status;
}

}  // namespace kfbi

using namespace kfbi;

namespace kfbi_cv {
__global__ void k_to_cplx(const double* __restrict__ src, double* __restrict__ dst, int n, int C) {
  KFBI_PDL_ENTRY();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  dst[2 * k] = C ? src[2 * k] : src[k];
  dst[2 * k + 1] = C ? src[2 * k + 1] : 0.0;
}
__global__ void k_from_cplx(const double* __restrict__ src, double* __restrict__ dst, int n, int C) {
  KFBI_PDL_ENTRY();
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

// ---- Neumann BVP (Eqs. 3.19, 3.20) ------------------------------------------


extern "C" kfbi_status kfbi_apply_neumann(kfbi_domain* dom, double kappa_re, double kappa_im,
                                          const void* psi_dev, const void* f_dev, void* out_dev,
                                          void* stream) {
  if (!dom) return KFBI_ERR_ARG;
  if (!psi_dev || !out_dev) {
    dom->err = "psi_dev and out_dev must be device pointers";
    return KFBI_ERR_ARG;
  }
  return guarded(dom, [&]() -> kfbi_status {
    NeumannScope ns(dom);
    cudaStream_t st = (cudaStream_t)stream;
    const bool C = kappa_im != 0.0;
    const double* ft = nullptr;
    if (f_dev) {
      pad_mask(dom, (const double*)f_dev, dom->d_fpad, C, st);
      ft = dom->d_fpad;
    }
    apply_internal(dom, kappa_re, kappa_im, (const double*)psi_dev, C ? 2 : 1, ft,
                   (double*)out_dev, C ? 2 : 1, false, st);
    return KFBI_OK;
  });
}

extern "C" kfbi_status kfbi_solve_neumann(kfbi_domain* dom, double kappa_re, double kappa_im,
                                          const void* gn_dev, const void* f_dev, void* psi_dev,
                                          void* u_grid_dev, kfbi_solve_info* info,
                                          void* stream) {
  if (!dom) return KFBI_ERR_ARG;
  if (!gn_dev || !psi_dev) {
    dom->err = "gn_dev and psi_dev must be device pointers";
    return KFBI_ERR_ARG;
  }
  return guarded(dom, [&]() -> kfbi_status {
    NeumannScope ns(dom);
    cudaStream_t st = (cudaStream_t)stream;
    const int C = kappa_im != 0.0, nb = dom->nb;
    const double* ft = nullptr;
    if (f_dev) {
      pad_mask(dom, (const double*)f_dev, dom->d_fpad, C, st);
      ft = dom->d_fpad;
    }
    KFBI_LAUNCH(k_to_cplx, (nb + 255) / 256, 256, 0, st, (const double*)gn_dev, dom->d_B, nb, C);
    KFBI_LAUNCH(k_to_cplx, (nb + 255) / 256, 256, 0, st, (const double*)psi_dev, dom->d_X, nb, C);
    KFBI_CHECK_LAUNCH();
    // b = g_N - d_n (Y f)+ : the known term of Eq. 3.19, left in d_B (the
    // refinement of mixed domains uses d_Rv and d_Dv as work space)
    if (ft) {
      apply_accurate(dom, kappa_re, kappa_im, dom->d_zero_nb, 2, ft, dom->d_Dv, 2, st);
      KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, k_residual, 1, kThreads, 0, st, (const double2*)dom->d_B,
                    (const double2*)dom->d_Dv, (double2*)dom->d_Rv, nb, dom->d_scal,
                    (double*)nullptr, 0LL);
      KFBI_CHECK_LAUNCH();
      KFBI_CUDA(cudaMemcpyAsync(dom->d_B, dom->d_Rv, 2 * (size_t)nb * sizeof(double),
                                cudaMemcpyDeviceToDevice, st));
    }
    kfbi_status s = gmres_solve(dom, kappa_re, kappa_im, dom->d_B, dom->d_X, false, info, st);
    if (u_grid_dev && s == KFBI_OK) {
      // u = Y f - V psi (Eq. 3.20): the interface solution with Psi = psi
      apply_accurate(dom, kappa_re, kappa_im, dom->d_X, 2, ft, nullptr, 2, st);
      unpad(dom, dom->d_U, (double*)u_grid_dev, C, st);
    }
    KFBI_LAUNCH(k_from_cplx, (nb + 255) / 256, 256, 0, st, dom->d_X, (double*)psi_dev, nb, C);
    KFBI_CHECK_LAUNCH();
    KFBI_CUDA(cudaStreamSynchronize(st));
    return s;
  });
}
