// Batched time steps over many KFBI instances of uneven size (mixed
// precision domains): every kernel of a step -- the volume-source and
// final applications, the refinement residuals, the GMRES iterations with
// their fast operator applications and CGS2 Arnoldi steps, and the F
// updates -- is one launch for the whole batch.  Small kernels take the
// instance from blockIdx.y; the tcgen05 DST passes are one persistent
// launch over the tiles of all instances (k_tc_pass with descriptor
// arrays).  Instances advance in lockstep; one that has converged is
// switched off by a device flag that every kernel checks, so the others keep
// iterating.  The per-iteration kernel sequence is captured once into a
// CUDA graph (the iteration index lives in device memory) and replayed.
//
// An instance's arithmetic does not depend on the other instances of the
// batch (each tile, reduction and GMRES decision is its own), so a domain
// gives the same bits whatever it is batched with.  Against the
// single-instance path the kernels differ in reduction order, and results
// agree to the GMRES tolerance.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "tc_internal.h"

namespace kfbi {
namespace bt {

using tc::GroupArgs;
using tc::PassDesc;

// Everything a grouped kernel needs about one instance.
struct GInst {
  int Mp, n1, nb, n_irr, n_arms, M, m, C, eq;
  int fft;  // KFBI_MIXED_FFT32 instance: FFT passes on single FP32 planes (Rh, T1h, T2h, U32)
  // FP32 pairs of 1/h^2, Re kappa, Im kappa (the double-float residual of
  // FFT instances; split on the host)
  float ih_hi, ih_lo, kr_hi, kr_lo, ki_hi, ki_lo;
  // FFT instances: the FP32 pair of f-tilde, split once per step (held in
  // the TF32 low planes, which the FFT passes leave unused)
  float* fth;
  float* ftl;
  int rmin, nrows;
  double h, kre, kim, scale, dt, theta;
  double w;  // Schroedinger: nonlinear coefficient of the B step (Eq. 3.10)
  // FP64 domain tables
  const uint8_t* mask;
  const int* irr_off;
  const int* arm_start;
  const int* arm_k0;
  const double* alpha;
  const double* beta;
  const int* arm_fidx;
  const double* arm_fcoef;
  const int* node_gidx;
  const double* node_w;
  const double* node_a;
  const double* node_b;
  const int* node_fidx;
  const double* node_fcoef;
  const double* lam64;
  const float* lam32;
  // FP32 tables of the mixed path
  const float* alpha32;
  const float* beta32;
  const float* arm_fcoef32;
  const float* node_w32;
  const float* node_a32;
  const float* node_b32;
  const float* S32;
  const int* row_start;
  const int* node_col;
  // work planes
  double* R64;
  double* U64;
  float* Rh;
  float* Rl;
  float* T1h;
  float* T2h;
  float* T2l;
  float* U32;
  float* T1sh;
  float* T1sl;
  float* rv;
  // GMRES workspace (complex interleaved)
  double2* V;
  double2* W;
  double2* H;
  double* cs;
  double2* sn;
  double2* g;
  double2* hcol;
  double2* part;
  double2* Rv;
  double2* Dv;
  double2* Ax;
  double* scal;  // [0] ||b||, [1] residual, [2] status, [3] tol
  // state
  double* u;
  double* F;
  double* Fprev;
  double* ft;
  double* aux;
  double2* x;    // density phi
  double2* b;
  double2* ub;
  double* uf;             // Y f-tilde grid kept from the b computation (superposition)
  double2* axc;           // A phi at the state's phi (superposition cache)
  const double* g_next;   // per step (caller layout)
  const double* src;      // heat source sum or Schroedinger potential (caller layout)
  double src_scale;       // heat: the source sum of this step is src_scale * src
  int* flags;             // [0] active, [1] k (iterations of the current cycle), [2] x_zero
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Grid-stride over the padded plane of the instance in blockIdx.y.
#define INST_PLANE_LOOP(I)                                                                 \
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;                         \
       idx < (size_t)(I).Mp * (I).Mp; idx += (size_t)gridDim.x * blockDim.x)

// Grid-stride over the padded plane in quads: four consecutive points of one
// grid row (Mp is a multiple of 128), moved with 16-byte vector accesses so
// that each thread keeps four points' loads in flight (one point per
// iteration left these kernels waiting on memory latency at a third of the
// HBM bandwidth).
#define INST_QUAD_LOOP(I)                                                                  \
  for (size_t idx = 4 * (blockIdx.x * (size_t)blockDim.x + threadIdx.x);                   \
       idx < (size_t)(I).Mp * (I).Mp; idx += 4 * (size_t)gridDim.x * blockDim.x)

struct Quad {
  double v[4];
};
__device__ __forceinline__ Quad ldq(const double* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  return Quad{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void stq(double* p, const Quad& q) {
  reinterpret_cast<double2*>(p)[0] = make_double2(q.v[0], q.v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(q.v[2], q.v[3]);
}
__device__ __forceinline__ float4 ldf4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void stf4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float f4at(const float4& v, int k) {
  return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

#define ACTIVE_OR_RETURN(I) \
  if ((I).flags[0] == 0) return;

// ---- volume source and base right-hand side --------------------------------

// heat/wave: f-tilde = -F on Omega; Schroedinger: u** = B(u*), f-tilde = -kappa u**
__global__ void gk_make_ft(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  const size_t plane = (size_t)I.Mp * I.Mp;
  if (I.eq != KFBI_SCHRODINGER) {
    INST_QUAD_LOOP(I) {
      const uchar4 mk = *reinterpret_cast<const uchar4*>(I.mask + idx);
      const Quad f = ldq(I.F + idx);
      const Quad v{{mk.x ? -f.v[0] : 0.0, mk.y ? -f.v[1] : 0.0, mk.z ? -f.v[2] : 0.0,
                    mk.w ? -f.v[3] : 0.0}};
      stq(I.ft + idx, v);
      if (I.fft) {
        float4 h, l;
        split_f64(v.v[0], h.x, l.x);
        split_f64(v.v[1], h.y, l.y);
        split_f64(v.v[2], h.z, l.z);
        split_f64(v.v[3], h.w, l.w);
        stf4(I.fth + idx, h);
        stf4(I.ftl + idx, l);
      }
    }
    return;
  }
  const double half_dt = 0.5 * I.dt, kim = I.kim;
  INST_PLANE_LOOP(I) {
    const int r = (int)((unsigned)idx / (unsigned)I.Mp), c = (int)idx - r * I.Mp;
    double xr = 0, xi = 0;
    if (r < I.n1 && c < I.n1) {
      // the modulus-preserving root of Eq. 3.10 (as k_schr_bstep)
      const double sr = I.F[idx], si = I.F[plane + idx];
      const double a = half_dt * (I.src[(size_t)r * I.n1 + c] + I.w * (sr * sr + si * si));
      const double den = 1.0 / (1.0 + a * a);
      const double pr = (1.0 - a * a) * den, pi = -2.0 * a * den;
      xr = pr * sr - pi * si;
      xi = pr * si + pi * sr;
    }
    I.aux[idx] = xr;
    I.aux[plane + idx] = xi;
    const bool in = I.mask[idx] != 0;
    const double vr = in ? kim * xi : 0.0, vi = in ? -kim * xr : 0.0;
    I.ft[idx] = vr;
    I.ft[plane + idx] = vi;
    if (I.fft) {
      split_f64(vr, I.fth[idx], I.ftl[idx]);
      split_f64(vi, I.fth[plane + idx], I.ftl[plane + idx]);
    }
  }
}

// R64 = f-tilde (with_ft) or 0 over the instance's planes; FFT instances
// take the FP32 pair (Rh, Rl) straight from the split of f-tilde.
__global__ void gk_base_rhs(const GInst* gi, int with_ft) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  const size_t plane = (size_t)I.Mp * I.Mp;
  const int P = I.C ? 2 : 1;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (I.fft) {
    INST_QUAD_LOOP(I) {
      for (int p = 0; p < P; ++p) {
        const size_t i = p * plane + idx;
        stf4(I.Rh + i, with_ft ? ldf4(I.fth + i) : z4);
        stf4(I.Rl + i, with_ft ? ldf4(I.ftl + i) : z4);
      }
    }
    return;
  }
  INST_QUAD_LOOP(I) {
    for (int p = 0; p < P; ++p) {
      const size_t i = p * plane + idx;
      stq(I.R64 + i, with_ft ? ldq(I.ft + i) : Quad{{0.0, 0.0, 0.0, 0.0}});
    }
  }
}

// FP64 corrected RHS at the irregular nodes (as k_correct); phi complex
// interleaved (stride 2).  which: 0 = zero density, 1 = x, 2 = V[j]
__device__ __forceinline__ const double* density_of(const GInst& I, int which, int j) {
  if (which == 0) return nullptr;
  if (which == 1) return (const double*)I.x;
  if (which == 3) return (const double*)I.Dv;
  return (const double*)(I.V + (size_t)j * I.nb);
}

__global__ void gk_correct64(const GInst* gi, int which, int with_ft, const int* dj) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= I.n_irr) return;
  const double* phi = density_of(I, which, dj ? *dj : 0);
  const double* ft = with_ft ? I.ft : nullptr;
  const bool C = I.C != 0;
  const size_t plane = (size_t)I.Mp * I.Mp;
  const int off = I.irr_off[n];
  double sr = ft ? ft[off] : 0.0;
  double si = (C && ft) ? ft[plane + off] : 0.0;
  const int a1 = I.arm_start[n + 1];
  const int na = I.n_arms, nb = I.nb;
  for (int a = I.arm_start[n]; a < a1; ++a) {
    int k = I.arm_k0[a];
    double ar = 0.0, ai = 0.0, br = 0.0, bi = 0.0;
    if (phi) {
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        const double al = I.alpha[m * na + a], be = I.beta[m * na + a];
        const double pr = phi[(size_t)k * 2];
        ar = fma(al, pr, ar);
        br = fma(be, pr, br);
        if (C) {
          const double pi = phi[(size_t)k * 2 + 1];
          ai = fma(al, pi, ai);
          bi = fma(be, pi, bi);
        }
        k = (k + 1 == nb) ? 0 : k + 1;
      }
    }
    sr += ar + I.kre * br;
    if (C) {
      sr -= I.kim * bi;
      si += ai + I.kre * bi + I.kim * br;
    }
    if (ft) {
      const int f0 = I.arm_fidx[a], f1 = I.arm_fidx[na + a];
      const double c0 = I.arm_fcoef[a], c1 = I.arm_fcoef[na + a];
      sr += c0 * ft[f0] + c1 * ft[f1];
      if (C) si += c0 * ft[plane + f0] + c1 * ft[plane + f1];
    }
  }
  if (I.fft) {  // the FP32 pair the FFT passes and the residual read
    split_f64(sr, I.Rh[off], I.Rl[off]);
    if (C) split_f64(si, I.Rh[plane + off], I.Rl[plane + off]);
    return;
  }
  I.R64[off] = sr;
  if (C) I.R64[plane + off] = si;
}

__device__ __forceinline__ float tf32r(float x) { return tf32_round(x); }

// TF32 pair of R64 (FFT instances have their pair from gk_base_rhs and
// gk_correct64)
__global__ void gk_split64(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  if (I.fft) return;
  const size_t plane = (size_t)I.Mp * I.Mp;
  const int P = I.C ? 2 : 1;
  INST_PLANE_LOOP(I) {
    for (int p = 0; p < P; ++p) {
      const size_t i = p * plane + idx;
      const double x = I.R64[i];
      const float h = tf32r((float)x);
      I.Rh[i] = h;
      I.Rl[i] = tf32r((float)(x - (double)h));
    }
  }
}

// Complex eigenvalue division on the TF32 pairs, in FP32 (k_eig_cplx32's
// arithmetic): a pair holds 22 significant bits, which FP32 keeps.
__global__ void gk_eig_cplx(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  if (!I.C || I.fft) return;  // the FFT solve pass divides by the eigenvalues itself
  const size_t plane = (size_t)I.Mp * I.Mp;
  const float kre = (float)I.kre, kim = (float)I.kim, scale = (float)I.scale;
  INST_PLANE_LOOP(I) {
    const int a = (int)((unsigned)idx / (unsigned)I.Mp), bcol = (int)idx - a * I.Mp;
    if (a >= I.n1 || bcol >= I.n1) continue;
    float zr, zi;
    eig_div_cplx32(I.T2h[idx] + I.T2l[idx], I.T2h[plane + idx] + I.T2l[plane + idx],
                   (I.lam32[a] - kre) + I.lam32[bcol], kim, scale, zr, zi);
    float h = tf32r(zr);
    I.T2h[idx] = h;
    I.T2l[idx] = tf32r(zr - h);
    h = tf32r(zi);
    I.T2h[plane + idx] = h;
    I.T2l[plane + idx] = tf32r(zi - h);
  }
}

__global__ void gk_f32_to_f64(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  if (I.fft) return;  // gk_resid_u32 starts the FP64 grid of FFT instances
  const size_t plane = (size_t)I.Mp * I.Mp;
  const int P = I.C ? 2 : 1;
  INST_PLANE_LOOP(I) {
    for (int p = 0; p < P; ++p) I.U64[p * plane + idx] = f32_to_f64(I.U32[p * plane + idx]);
  }
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// r = R - L u at one point, in double-float arithmetic from FP32 values:
// u and its four neighbours, uo the other plane's u (complex: L couples the
// planes through +-Im kappa, sg = +1 for the real plane, -1 for the
// imaginary one), (R_hi, R_lo) the FP32 pair of R.
template <bool C>
__device__ __forceinline__ float resid_df(const GInst& I, float u, float e, float w, float nn,
                                          float so, float uo, float sg, float R_hi, float R_lo) {
  float sh = -4.f * u, sl = 0.f, t;
  two_sum(sh, e, sh, t);
  sl += t;
  two_sum(sh, w, sh, t);
  sl += t;
  two_sum(sh, nn, sh, t);
  sl += t;
  two_sum(sh, so, sh, t);
  sl += t;
  float p1, e1, p2, e2;
  two_prod(sh, I.ih_hi, p1, e1);
  two_prod(I.kr_hi, u, p2, e2);
  float tail = e1 + fmaf(sh, I.ih_lo, sl * I.ih_hi) - e2 - I.kr_lo * u;
  float lu_hi, t2;
  two_sum(p1, -p2, lu_hi, t2);
  tail += t2;
  if (C) {
    float p3, e3;
    two_prod(I.ki_hi, uo, p3, e3);
    float t3;
    two_sum(lu_hi, sg * p3, lu_hi, t3);
    tail += t3 + sg * (e3 + I.ki_lo * uo);
  }
  float d, t4;
  two_sum(R_hi, -lu_hi, d, t4);
  return d + ((t4 + R_lo) - tail);
}

template <bool C>
__device__ __forceinline__ void resid_u32_quads(const GInst& I) {
  const size_t plane = (size_t)I.Mp * I.Mp;
  const int Mp = I.Mp, n1 = I.n1;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  INST_QUAD_LOOP(I) {
    const int r = (int)((unsigned)idx / (unsigned)Mp), c0 = (int)idx - r * Mp;
    const bool live = r < n1 && c0 < n1;
#pragma unroll
    for (int p = 0; p < (C ? 2 : 1); ++p) {
      const float* Up = I.U32 + p * plane;
      float4 res = z4, uq = z4;
      if (live) {
        uq = ldf4(Up + idx);
        const float4 un = r + 1 < n1 ? ldf4(Up + idx + Mp) : z4;
        const float4 us = r > 0 ? ldf4(Up + idx - Mp) : z4;
        const float uw = c0 > 0 ? Up[idx - 1] : 0.f;
        const float ue = c0 + 4 < n1 ? Up[idx + 4] : 0.f;
        const float4 uo = C ? ldf4(I.U32 + (1 - p) * plane + idx) : z4;
        const float4 rh = ldf4(I.Rh + p * plane + idx), rl = ldf4(I.Rl + p * plane + idx);
        float o[4], uu[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = c0 + k;
          const float u = c < n1 ? f4at(uq, k) : 0.f;
          const float e = c + 1 < n1 ? (k < 3 ? f4at(uq, k + 1) : ue) : 0.f;
          const float w = c > 0 ? (k > 0 ? f4at(uq, k - 1) : uw) : 0.f;
          uu[k] = u;
          o[k] = c < n1 ? resid_df<C>(I, u, e, w, f4at(un, k), f4at(us, k), f4at(uo, k),
                                      p == 0 ? 1.f : -1.f, f4at(rh, k), f4at(rl, k))
                        : 0.f;
        }
        res = make_float4(o[0], o[1], o[2], o[3]);
        uq = make_float4(uu[0], uu[1], uu[2], uu[3]);
      }
      stq(I.U64 + p * plane + idx, Quad{{f32_to_f64(uq.x), f32_to_f64(uq.y), f32_to_f64(uq.z),
                                         f32_to_f64(uq.w)}});
      stf4(I.Rh + p * plane + idx, res);
    }
  }
}

// Residual of the refinement for FFT instances (as k_resid_u32): from the
// FP32 grid U32 and the FP32 pair (Rh, Rl) of R in double-float arithmetic,
// r into Rh, and U64 = U32 (0 outside the n1 x n1 block).
__global__ void gk_resid_u32(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  if (!I.fft) return;
  if (I.C) resid_u32_quads<true>(I);
  else resid_u32_quads<false>(I);
}

__global__ void gk_resid_split(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  if (I.fft) return;  // gk_resid_u32
  const size_t plane = (size_t)I.Mp * I.Mp;
  const int Mp = I.Mp, n1 = I.n1;
  const double inv_h2 = 1.0 / (I.h * I.h);
  const bool C = I.C != 0;
  INST_PLANE_LOOP(I) {
    const int r = (int)((unsigned)idx / (unsigned)Mp), c = (int)idx - r * Mp;
    for (int p = 0; p < (C ? 2 : 1); ++p) {
      double res = 0.0;
      if (r < n1 && c < n1) {
        const double* Up = I.U64 + p * plane;
        const double u = Up[idx];
        const double e = c + 1 < n1 ? Up[idx + 1] : 0.0;
        const double w = c > 0 ? Up[idx - 1] : 0.0;
        const double nn = r + 1 < n1 ? Up[idx + Mp] : 0.0;
        const double s = r > 0 ? Up[idx - Mp] : 0.0;
        double Lu = (e + w + nn + s - 4.0 * u) * inv_h2 - I.kre * u;
        if (C) {
          const double uo = I.U64[(1 - p) * plane + idx];
          Lu += (p == 0) ? I.kim * uo : -I.kim * uo;
        }
        res = I.R64[p * plane + idx] - Lu;
      }
      if (I.fft) {
        I.Rh[p * plane + idx] = (float)res;
        continue;
      }
      const float h = tf32r((float)res);
      I.Rh[p * plane + idx] = h;
      I.Rl[p * plane + idx] = tf32r((float)(res - (double)h));
    }
  }
}

__global__ void gk_add_f32(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  const size_t plane = (size_t)I.Mp * I.Mp;
  const int P = I.C ? 2 : 1;
  INST_QUAD_LOOP(I) {
    for (int p = 0; p < P; ++p) {
      const size_t i = p * plane + idx;
      const float4 d = ldf4(I.U32 + i);
      Quad u = ldq(I.U64 + i);
      u.v[0] += f32_to_f64(d.x);
      u.v[1] += f32_to_f64(d.y);
      u.v[2] += f32_to_f64(d.z);
      u.v[3] += f32_to_f64(d.w);
      stq(I.U64 + i, u);
    }
  }
}

// FP64 extraction (as k_extract) into out (ub or Ax), complex interleaved.
__global__ void gk_extract64(const GInst* gi, int which, int with_ft, int target) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int nb = I.nb;
  if (k >= nb) return;
  const double* phi = density_of(I, which, 0);
  const double* ft = with_ft ? I.ft : nullptr;
  double* out = target == 0 ? (double*)I.ub : (double*)I.Ax;
  const bool C = I.C != 0;
  const size_t plane = (size_t)I.Mp * I.Mp;
  double sr = 0.0, si = 0.0;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const int gg = I.node_gidx[m * nb + k];
    const double wm = I.node_w[m * nb + k];
    sr = fma(wm, I.U64[gg], sr);
    if (C) si = fma(wm, I.U64[plane + gg], si);
  }
  double ar = 0.0, ai = 0.0, br = 0.0, bi = 0.0;
  if (phi) {
    int kk = k - 2;
    if (kk < 0) kk += nb;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const double a = I.node_a[j * nb + k], b = I.node_b[j * nb + k];
      const double pr = phi[(size_t)kk * 2];
      ar = fma(a, pr, ar);
      br = fma(b, pr, br);
      if (C) {
        const double pi = phi[(size_t)kk * 2 + 1];
        ai = fma(a, pi, ai);
        bi = fma(b, pi, bi);
      }
      kk = (kk + 1 == nb) ? 0 : kk + 1;
    }
  }
  sr += ar + I.kre * br;
  if (C) {
    sr -= I.kim * bi;
    si += ai + I.kre * bi + I.kim * br;
  }
  if (ft) {
    const int gg = I.node_fidx[k];
    const double c = I.node_fcoef[k];
    sr += c * ft[gg];
    if (C) si += c * ft[plane + gg];
  }
  out[(size_t)k * 2] = sr;
  out[(size_t)k * 2 + 1] = C ? si : 0.0;
}

// ---- fast (sparse) application with the density V[j] ----------------------

__global__ void gk_correct32_rv(const GInst* gi, const int* dj) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  if (I.fft) return;  // FFT instances build these rows inside their first pass
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= I.n_irr) return;
  const double* phi = (const double*)(I.V + (size_t)(*dj) * I.nb);
  const bool C = I.C != 0;
  const int na = I.n_arms, nb = I.nb;
  const float kre = (float)I.kre, kim = (float)I.kim;
  float sr = 0.f, si = 0.f;
  const int a1 = I.arm_start[n + 1];
  for (int a = I.arm_start[n]; a < a1; ++a) {
    int k = I.arm_k0[a];
    float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      const float al = I.alpha32[m * na + a], be = I.beta32[m * na + a];
      const float pr = (float)phi[(size_t)k * 2];
      ar = fmaf(al, pr, ar);
      br = fmaf(be, pr, br);
      if (C) {
        const float pi = (float)phi[(size_t)k * 2 + 1];
        ai = fmaf(al, pi, ai);
        bi = fmaf(be, pi, bi);
      }
      k = (k + 1 == nb) ? 0 : k + 1;
    }
    sr += ar + kre * br;
    if (C) {
      sr -= kim * bi;
      si += ai + kre * bi + kim * br;
    }
  }
  I.rv[n] = sr;
  if (C) I.rv[I.n_irr + n] = si;
}

// blockIdx.z = instance; (x, y) = 32 x 32 output tile as in k_sparse_p1
__global__ void __launch_bounds__(256) gk_sparse_p1(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.z];
  ACTIVE_OR_RETURN(I);
  if (I.fft) return;
  const int Mp = I.Mp;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  if (c0 >= Mp || r0 >= I.nrows) return;
  __shared__ float tile[2][32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int P = I.C ? 2 : 1;
  for (int rr = ty; rr < 32; rr += 8) {
    const int rl = r0 + rr;
    float a0 = 0.f, a1 = 0.f;
    if (rl < I.nrows) {
      const int ne = I.row_start[rl + 1];
      for (int n = I.row_start[rl]; n < ne; ++n) {
        const float sv = I.S32[(size_t)I.node_col[n] * Mp + c0 + tx];
        a0 = fmaf(I.rv[n], sv, a0);
        if (P == 2) a1 = fmaf(I.rv[I.n_irr + n], sv, a1);
      }
    }
    tile[0][rr][tx] = a0;
    tile[1][rr][tx] = a1;
  }
  __syncthreads();
  const size_t plane = (size_t)Mp * Mp;
  for (int cc = ty; cc < 32; cc += 8) {
    const int rl = r0 + tx;
    if (rl >= I.nrows) continue;
    const size_t o = (size_t)(c0 + cc) * Mp + (size_t)(I.rmin + rl);
    for (int p = 0; p < P; ++p) {
      const float x = tile[p][tx][cc];
      const float h = tf32r(x);
      I.T1sh[p * plane + o] = h;
      I.T1sl[p * plane + o] = tf32r(x - h);
    }
  }
}

// Gather of the stencil values and extraction (as k_gather_extract) into W.
// TF32 instances leave the last pass's input with rows = x indices; FFT
// instances (solve pass written transposed) with rows = y indices.  The six
// stencil points of a node lie in a 3 x 3 window of grid rows and columns:
// the node's warp streams the window's three grid rows and three S rows
// (float4) and forms the nine window sums.  One warp per node: a batch holds
// tens of thousands of nodes, and a block per node (as the single-domain
// kernel, where a grid has about a thousand) kept too few nodes in flight.
constexpr int GB_NODES = 4;  // nodes (warps) per block

template <bool C, bool TY>
__device__ __forceinline__ void gather_window(const GInst& I, int lane, int jlo, int ilo,
                                              float* win) {
  constexpr int NP = C ? 2 : 1;
  const int Mp = I.Mp;
  const size_t plane = (size_t)Mp * Mp;
  const float4* tr[NP][3];
  const float4* srow[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    // rows past the plane are clamped; their sums are never picked
    const int ii = min(ilo + d, Mp - 1), jj = min(jlo + d, Mp - 1);
    const int tt = TY ? jj : ii, ss = TY ? ii : jj;
#pragma unroll
    for (int q = 0; q < NP; ++q)
      tr[q][d] = reinterpret_cast<const float4*>(I.U32 + q * plane + (size_t)tt * Mp);
    srow[d] = reinterpret_cast<const float4*>(I.S32 + (size_t)ss * Mp);
  }
  float acc[NP][3][3];
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int dj = 0; dj < 3; ++dj)
#pragma unroll
      for (int di = 0; di < 3; ++di) acc[q][dj][di] = 0.f;
#pragma unroll 1
  for (int a4 = lane; a4 < Mp / 4; a4 += 32) {
    float4 t[NP][3], sv[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int q = 0; q < NP; ++q) t[q][d] = tr[q][d][a4];
      sv[d] = srow[d][a4];
    }
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
      for (int dj = 0; dj < 3; ++dj)
#pragma unroll
        for (int di = 0; di < 3; ++di) {
          // window point (row jlo + dj, column ilo + di)
          const float4 tv = t[q][TY ? dj : di], s4 = sv[TY ? di : dj];
          float x = acc[q][dj][di];
          x = fmaf(tv.x, s4.x, x);
          x = fmaf(tv.y, s4.y, x);
          x = fmaf(tv.z, s4.z, x);
          x = fmaf(tv.w, s4.w, x);
          acc[q][dj][di] = x;
        }
  }
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int dj = 0; dj < 3; ++dj)
#pragma unroll
      for (int di = 0; di < 3; ++di) {
        float x = acc[q][dj][di];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) win[q * 9 + dj * 3 + di] = x;
      }
  __syncwarp();
}

// One kernel per value type (the complex window holds twice the registers);
// instances of the other type return at once.  Lane m < 6 fetches stencil
// point m's offset and extraction operands before the rows stream in.
template <bool C>
__global__ void __launch_bounds__(32 * GB_NODES) gk_gather_extract(const GInst* gi, const int* dj) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  if ((I.C != 0) != C) return;
  ACTIVE_OR_RETURN(I);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * GB_NODES + warp;
  const int nb = I.nb;
  if (k >= nb) return;  // the whole warp
  __shared__ float win[GB_NODES][2 * 9];
  const int Mp = I.Mp;
  int jl = Mp, il = Mp;
  float wm = 0.f, am = 0.f, bm = 0.f, pr = 0.f, pi = 0.f;
  if (lane < 6) {
    const int off = I.node_gidx[lane * nb + k];
    jl = off / Mp;
    il = off - jl * Mp;
    wm = I.node_w32[lane * nb + k];
    am = I.node_a32[lane * nb + k];
    bm = I.node_b32[lane * nb + k];
    int kk = (k - 2 + lane) % nb;
    if (kk < 0) kk += nb;
    const double* phi = (const double*)(I.V + (size_t)(*dj) * nb);
    pr = (float)phi[(size_t)kk * 2];
    if (C) pi = (float)phi[(size_t)kk * 2 + 1];
  }
  // window origin: the least row and column over lanes 0-5
  int jlo = jl, ilo = il;
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    jlo = min(jlo, __shfl_xor_sync(0xffffffffu, jlo, o));
    ilo = min(ilo, __shfl_xor_sync(0xffffffffu, ilo, o));
  }
  jlo = __shfl_sync(0xffffffffu, jlo, 0);
  ilo = __shfl_sync(0xffffffffu, ilo, 0);
  if (I.fft) gather_window<C, true>(I, lane, jlo, ilo, win[warp]);
  else gather_window<C, false>(I, lane, jlo, ilo, win[warp]);
  const float kre = (float)I.kre, kim = (float)I.kim;
  float sr = 0.f, si = 0.f, ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const int w_at = (__shfl_sync(0xffffffffu, jl, m) - jlo) * 3 + __shfl_sync(0xffffffffu, il, m) - ilo;
    const float w_ = __shfl_sync(0xffffffffu, wm, m);
    const float a_ = __shfl_sync(0xffffffffu, am, m);
    const float b_ = __shfl_sync(0xffffffffu, bm, m);
    const float pr_ = __shfl_sync(0xffffffffu, pr, m);
    const float pi_ = C ? __shfl_sync(0xffffffffu, pi, m) : 0.f;
    sr = fmaf(w_, win[warp][w_at], sr);
    if (C) si = fmaf(w_, win[warp][9 + w_at], si);
    ar = fmaf(a_, pr_, ar);
    br = fmaf(b_, pr_, br);
    if (C) {
      ai = fmaf(a_, pi_, ai);
      bi = fmaf(b_, pi_, bi);
    }
  }
  if (lane != 0) return;
  sr += ar + kre * br;
  if (C) {
    sr -= kim * bi;
    si += ai + kre * bi + kim * br;
  }
  I.W[k] = make_double2((double)sr, C ? (double)si : 0.0);
}

// ---- GMRES (as gmres.cu, instance in blockIdx.y) ---------------------------

constexpr int GT = 256;
constexpr int GMAX = 64;

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) red[0] = v;
  }
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

// b = g - ub (real g for heat/wave, complex for Schroedinger)
__global__ void gk_make_b(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= I.nb) return;
  const bool gC = I.eq == KFBI_SCHRODINGER;
  const double gr = gC ? I.g_next[2 * k] : I.g_next[k], gim = gC ? I.g_next[2 * k + 1] : 0.0;
  I.b[k] = make_double2(gr - I.ub[k].x, gim - I.ub[k].y);
}

// ||b|| into scal[0] (tol into scal[3]); one 1024-thread block per instance
__global__ void __launch_bounds__(1024) gk_bnorm(const GInst* gi, double tol, int which) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  __shared__ double red[32];
  const double2* v = which == 0 ? I.b : I.Rv;
  double s = 0.0;
  for (int e = threadIdx.x; e < I.nb; e += 1024) s += v[e].x * v[e].x + v[e].y * v[e].y;
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    I.scal[0] = sqrt(s);
    I.scal[3] = tol;
  }
}

// All instances' scalars and flags into one buffer for a single readback.
__global__ void gk_gather_scal(const GInst* gi, double* out) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.x];
  if (threadIdx.x < 8) out[8 * blockIdx.x + threadIdx.x] = I.scal[threadIdx.x];
}

// All instances' scalars (8 doubles each) and flags (4 ints each) posted to
// host-mapped memory, then, after a system-scope fence, the post's
// sequence number (one more than the last, from a device counter, so that
// posts inside a replayed graph number themselves): slot seq & 1 of mbox,
// scalars at [0, 8 cap), flags from double 8 cap, the sequence number in
// the slot's last double.  The host polls the number instead of copying the
// state back behind a synchronisation.  One block.
__global__ void __launch_bounds__(256) gk_post(const GInst* gi, int n, double* mbox, int slot_stride,
                                              int cap, long long* ctr) {
  KFBI_PDL_ENTRY();
  __shared__ long long s_seq;
  if (threadIdx.x == 0) s_seq = ++(*ctr);
  __syncthreads();
  volatile double* slot = mbox + (s_seq & 1) * (size_t)slot_stride;
  volatile int* fl = reinterpret_cast<volatile int*>(slot + 8 * (size_t)cap);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const GInst& I = gi[i];
#pragma unroll
    for (int k = 0; k < 8; ++k) slot[8 * i + k] = I.scal[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) fl[4 * i + k] = I.flags[k];
  }
  __threadfence_system();
  __syncthreads();
  if (threadIdx.x == 0) reinterpret_cast<volatile long long*>(slot + slot_stride - 1)[0] = s_seq;
}

__global__ void gk_set_tol(const GInst* gi, const double* tol, const int* sel) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.x];
  if (threadIdx.x == 0 && sel[blockIdx.x]) I.scal[3] = tol[blockIdx.x];
}

__global__ void gk_clear_k(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.x];
  if (threadIdx.x == 0) I.flags[1] = 0;
}

// Rv = b - Ax (Ax omitted for x_zero) and ||Rv|| into scal[1]
__global__ void __launch_bounds__(1024) gk_residual(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  __shared__ double red[32];
  const bool skip = I.flags[2] != 0;
  double s = 0.0;
  for (int e = threadIdx.x; e < I.nb; e += 1024) {
    double2 v = I.b[e];
    if (!skip) {
      v.x -= I.Ax[e].x;
      v.y -= I.Ax[e].y;
    }
    I.Rv[e] = v;
    s += v.x * v.x + v.y * v.y;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) I.scal[1] = sqrt(s);
}

// Superposition of the refined step (as the single-instance path): the
// discrete solution is Y f-tilde + W phi, so the grid of the b computation
// is kept, and A phi of a converged residual check is reused by the next
// step's first residual.
__global__ void gk_keep_uf(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  const size_t plane = (size_t)I.Mp * I.Mp;
  const int P = I.C ? 2 : 1;
  INST_QUAD_LOOP(I) {
    for (int p = 0; p < P; ++p) stq(I.uf + p * plane + idx, ldq(I.U64 + p * plane + idx));
  }
}

__global__ void gk_add_uf(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  const size_t plane = (size_t)I.Mp * I.Mp;
  const int P = I.C ? 2 : 1;
  INST_QUAD_LOOP(I) {
    for (int p = 0; p < P; ++p) {
      const size_t i = p * plane + idx;
      Quad u = ldq(I.U64 + i);
      const Quad f = ldq(I.uf + i);
#pragma unroll
      for (int k = 0; k < 4; ++k) u.v[k] += f.v[k];
      stq(I.U64 + i, u);
    }
  }
}

// direction 0: Ax = cached A phi; 1: cache = Ax
__global__ void gk_ax_cache(const GInst* gi, int direction) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < I.nb; k += gridDim.x * blockDim.x) {
    if (direction == 0)
      I.Ax[k] = I.axc[k];
    else
      I.axc[k] = I.Ax[k];
  }
}

// V0 = r/beta with r = Rv - A Dv (restart) or Rv (fresh cycle), g = (beta, 0..)
__global__ void __launch_bounds__(1024) gk_restart(const GInst* gi, int with_ax) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  __shared__ double red[32];
  double s = 0.0;
  for (int e = threadIdx.x; e < I.nb; e += 1024) {
    double2 r = I.Rv[e];
    if (with_ax) {
      r.x -= I.W[e].x;
      r.y -= I.W[e].y;
    }
    I.V[e] = r;
    s += r.x * r.x + r.y * r.y;
  }
  s = block_sum(s, red);
  // the square root and the reciprocal once, not in every thread
  __shared__ double s_beta, s_inv;
  if (threadIdx.x == 0) {
    s_beta = sqrt(s);
    s_inv = s_beta > 0.0 ? 1.0 / s_beta : 0.0;
  }
  __syncthreads();
  const double beta = s_beta, inv = s_inv;
  for (int e = threadIdx.x; e < I.nb; e += 1024) {
    I.V[e].x *= inv;
    I.V[e].y *= inv;
  }
  if (threadIdx.x <= I.m) I.g[threadIdx.x] = make_double2(threadIdx.x == 0 ? beta : 0.0, 0.0);
  if (threadIdx.x == 0) {
    I.scal[1] = beta;
    const double st = !isfinite(beta) ? 2.0 : (beta <= I.scal[3] * I.scal[0] ? 1.0 : 0.0);
    I.scal[2] = st;
    I.flags[1] = 0;
    if (st != 0.0) I.flags[0] = 0;  // converged (or non-finite) before iterating
  }
}

// Same partition of the vectors as the single-instance grid_shape().
__device__ __forceinline__ void shape(int nb, int& G, int& slice) {
  int G0 = (nb + 31) / 32;
  if (G0 > 64) G0 = 64;
  slice = ((nb + G0 - 1) / G0 + 31) / 32 * 32;
  G = (nb + slice - 1) / slice;
}

__device__ __forceinline__ void slice_of(int nb, int b, int, int& e0, int& e1) {
  int G, slice;
  shape(nb, G, slice);
  e0 = b * slice;
  e1 = min(nb, e0 + slice);
}

__device__ __forceinline__ double2 dotpart(const double2* __restrict__ a,
                                           const double2* __restrict__ b, int e0, int e1, int lane,
                                           bool C) {
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

__device__ __forceinline__ int grid_g(int nb) {
  int G, slice;
  shape(nb, G, slice);
  return G;
}

__global__ void __launch_bounds__(GT) gk_cgs_dots(const GInst* gi, const int* dj) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  const int G = grid_g(I.nb);
  if ((int)blockIdx.x >= G) return;
  const int j = *dj;
  int e0, e1;
  slice_of(I.nb, blockIdx.x, G, e0, e1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i <= j; i += GT / 32) {
    const double2 s = dotpart(I.V + (size_t)i * I.nb, I.W, e0, e1, lane, I.C != 0);
    if (lane == 0) I.part[(size_t)i * GMAX + blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(GT) gk_cgs_update(const GInst* gi, const int* dj, int first,
                                                    int mode) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  const int G = grid_g(I.nb);
  if ((int)blockIdx.x >= G) return;
  const int j = *dj;
  const bool C = I.C != 0;
  __shared__ double2 h[65];
  int e0, e1;
  slice_of(I.nb, blockIdx.x, G, e0, e1);
  const double2* part_in = first ? I.part : I.part + (size_t)(I.m + 1) * GMAX;
  double2* part_out = first ? I.part + (size_t)(I.m + 1) * GMAX : I.part;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i <= j; i += GT / 32) {
    double2 s = make_double2(0.0, 0.0);
    for (int b = lane; b < G; b += 32) {
      const double2 v = part_in[(size_t)i * GMAX + b];
      s.x += v.x;
      if (C) s.y += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      if (C) s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (lane == 0) h[i] = s;
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i <= j; i += GT) {
      if (first) {
        I.hcol[i] = h[i];
      } else {
        I.hcol[i].x += h[i].x;
        I.hcol[i].y += h[i].y;
      }
    }
  for (int e = e0 + threadIdx.x; e < e1; e += GT) {
    double2 acc = I.W[e];
    for (int i = 0; i <= j; ++i) {
      const double2 v = I.V[(size_t)i * I.nb + e], hi = h[i];
      if (C) {
        acc.x -= hi.x * v.x - hi.y * v.y;
        acc.y -= hi.x * v.y + hi.y * v.x;
      } else {
        acc.x -= hi.x * v.x;
      }
    }
    I.W[e] = acc;
  }
  __syncthreads();
  if (mode == 0) {
    for (int i = warp; i <= j; i += GT / 32) {
      const double2 s = dotpart(I.V + (size_t)i * I.nb, I.W, e0, e1, lane, C);
      if (lane == 0) part_out[(size_t)i * GMAX + blockIdx.x] = s;
    }
  } else if (warp == 0) {
    const double2 s = dotpart(I.W, I.W, e0, e1, lane, C);
    if (lane == 0) part_out[blockIdx.x] = make_double2(s.x, 0.0);
  }
}

__global__ void __launch_bounds__(GT) gk_cgs_finalize(const GInst* gi, const int* dj) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  const int G = grid_g(I.nb);
  if ((int)blockIdx.x >= G) return;
  const int j = *dj;
  const int m = I.m;
  __shared__ double nrm, nrm_inv;
  int e0, e1;
  slice_of(I.nb, blockIdx.x, G, e0, e1);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double s = 0.0;
    for (int q = lane; q < G; q += 32) s += I.part[q].x;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      nrm = sqrt(s);
      nrm_inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    }
  }
  __syncthreads();
  const double hn = nrm;
  const double inv = nrm_inv;
  double2* vn = I.V + (size_t)(j + 1) * I.nb;
  for (int e = e0 + threadIdx.x; e < e1; e += GT)
    vn[e] = make_double2(I.W[e].x * inv, I.W[e].y * inv);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double2* col = I.H + (size_t)j * (m + 1);
    for (int i = 0; i <= j; ++i) col[i] = I.hcol[i];
    col[j + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < j; ++i) {
      const double c = I.cs[i];
      const double2 sv = I.sn[i], a = col[i], bb = col[i + 1];
      const double2 t = cmul(sv, bb);
      const double2 u = cmul(make_double2(sv.x, -sv.y), a);
      col[i] = make_double2(c * a.x + t.x, c * a.y + t.y);
      col[i + 1] = make_double2(-u.x + c * bb.x, -u.y + c * bb.y);
    }
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
    I.cs[j] = c;
    I.sn[j] = sv;
    col[j] = make_double2(c * a.x + sv.x * bre, c * a.y + sv.y * bre);
    col[j + 1] = make_double2(0.0, 0.0);
    const double2 gj = I.g[j];
    const double2 u = cmul(make_double2(sv.x, -sv.y), gj);
    I.g[j + 1] = make_double2(-u.x, -u.y);
    I.g[j] = make_double2(c * gj.x, c * gj.y);
    const double res = hypot(I.g[j + 1].x, I.g[j + 1].y);
    I.scal[1] = res;
    const double st = !isfinite(res) ? 2.0 : ((res <= I.scal[3] * I.scal[0] || hn == 0.0) ? 1.0 : 0.0);
    I.scal[2] = st;
    I.flags[1] = j + 1;
    if (st != 0.0) I.flags[0] = 0;  // this instance stops iterating
  }
}

// One CGS2 Arnoldi step of an instance in one block (the batch holds many
// small instances: the four-kernel form above spent most of its time in
// cross-block partial sums and launch latency).  W is staged in shared
// memory; each warp forms the dots of one basis vector at a time; the
// Hessenberg column, the earlier rotations and the right-hand side g are
// rotated in shared memory by one thread.  Same arithmetic as
// gk_cgs_dots/update/finalize up to the order of the partial sums.
constexpr int AT = 512;
constexpr int kArnoldiMaxNb = 8192;  // W in shared memory: 128 KiB

template <bool C>
__global__ void __launch_bounds__(AT) gk_arnoldi(const GInst* gi, const int* dj) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.x];
  if ((I.C != 0) != C) return;
  ACTIVE_OR_RETURN(I);
  extern __shared__ double2 Ws[];  // nb
  __shared__ double2 h[2][GMAX + 1];
  __shared__ double2 sn_s[GMAX];
  __shared__ double cs_s[GMAX];
  __shared__ double red[AT / 32];
  const int j = *dj, nb = I.nb, m = I.m;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < nb; e += AT) Ws[e] = I.W[e];
  for (int i = threadIdx.x; i < j; i += AT) {
    cs_s[i] = I.cs[i];
    sn_s[i] = I.sn[i];
  }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    // h_i = V_i^H W
    for (int i = warp; i <= j; i += AT / 32) {
      const double2* v = I.V + (size_t)i * nb;
      double sx = 0.0, sy = 0.0;
      for (int e = lane; e < nb; e += 32) {
        const double2 x = v[e], y = Ws[e];
        if (C) {
          sx += x.x * y.x + x.y * y.y;
          sy += x.x * y.y - x.y * y.x;
        } else {
          sx += x.x * y.x;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        if (C) sy += __shfl_xor_sync(0xffffffffu, sy, o);
      }
      if (lane == 0) h[pass][i] = make_double2(sx, sy);
    }
    __syncthreads();
    // W -= V h
    for (int e = threadIdx.x; e < nb; e += AT) {
      double2 acc = Ws[e];
      for (int i = 0; i <= j; ++i) {
        const double2 v = I.V[(size_t)i * nb + e], hi = h[pass][i];
        if (C) {
          acc.x -= hi.x * v.x - hi.y * v.y;
          acc.y -= hi.x * v.y + hi.y * v.x;
        } else {
          acc.x -= hi.x * v.x;
        }
      }
      Ws[e] = acc;
    }
    __syncthreads();
  }
  // h_{j+1,j} = ||W||, V_{j+1} = W / h_{j+1,j}
  double s = 0.0;
  for (int e = threadIdx.x; e < nb; e += AT) s += Ws[e].x * Ws[e].x + (C ? Ws[e].y * Ws[e].y : 0.0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (warp == 0) {
    double t = lane < AT / 32 ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
      red[0] = sqrt(t);
      red[1] = red[0] > 0.0 ? 1.0 / red[0] : 0.0;
    }
  }
  __syncthreads();
  const double hn = red[0];
  const double inv = red[1];
  double2* vn = I.V + (size_t)(j + 1) * nb;
  for (int e = threadIdx.x; e < nb; e += AT) vn[e] = make_double2(Ws[e].x * inv, Ws[e].y * inv);
  // Hessenberg column j: CGS2 sum, earlier rotations, new rotation, g
  double2* col = h[0];
  for (int i = threadIdx.x; i <= j; i += AT)
    col[i] = make_double2(h[0][i].x + h[1][i].x, h[0][i].y + h[1][i].y);
  __syncthreads();
  if (threadIdx.x == 0) {
    col[j + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < j; ++i) {
      const double c = cs_s[i];
      const double2 sv = sn_s[i], a = col[i], bb = col[i + 1];
      const double2 t = cmul(sv, bb);
      const double2 u = cmul(make_double2(sv.x, -sv.y), a);
      col[i] = make_double2(c * a.x + t.x, c * a.y + t.y);
      col[i + 1] = make_double2(-u.x + c * bb.x, -u.y + c * bb.y);
    }
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
    I.cs[j] = c;
    I.sn[j] = sv;
    col[j] = make_double2(c * a.x + sv.x * bre, c * a.y + sv.y * bre);
    col[j + 1] = make_double2(0.0, 0.0);
    const double2 gj = I.g[j];
    const double2 u = cmul(make_double2(sv.x, -sv.y), gj);
    I.g[j + 1] = make_double2(-u.x, -u.y);
    I.g[j] = make_double2(c * gj.x, c * gj.y);
    const double res = hypot(u.x, u.y);
    I.scal[1] = res;
    const double st = !isfinite(res) ? 2.0 : ((res <= I.scal[3] * I.scal[0] || hn == 0.0) ? 1.0 : 0.0);
    I.scal[2] = st;
    I.flags[1] = j + 1;
  }
  __syncthreads();
  double2* Hc = I.H + (size_t)j * (m + 1);
  for (int i = threadIdx.x; i <= j + 1; i += AT) Hc[i] = col[i];
  // the stop flag last: no other thread of this block reads flags[0] again
  if (threadIdx.x == 0 && I.scal[2] != 0.0) I.flags[0] = 0;
}

// Dv += V y (k = flags[1] iterations); runs for every instance with k > 0.
__global__ void __launch_bounds__(GT) gk_update(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  const int k = I.flags[1];
  if (k == 0) return;
  const int G = grid_g(I.nb);
  if ((int)blockIdx.x >= G) return;
  const int m = I.m;
  __shared__ double2 y[64], gs[64];
  __shared__ double2 R[64 * 65 / 2];  // R[l (l + 1) / 2 + i] = H(i, l), i <= l < k
  int e0, e1;
  slice_of(I.nb, blockIdx.x, G, e0, e1);
  // the triangle and g in one round of independent loads (the solve below
  // is a serial chain and must not wait on global memory)
  for (int t = threadIdx.x; t < k * (k + 1) / 2; t += GT) {
    int l = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while (l * (l + 1) / 2 > t) --l;
    while ((l + 1) * (l + 2) / 2 <= t) ++l;
    R[t] = I.H[(size_t)l * (m + 1) + (t - l * (l + 1) / 2)];
  }
  for (int i = threadIdx.x; i < k; i += GT) gs[i] = I.g[i];
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
        const double dd = d.x * d.x + d.y * d.y;
        y[i] = make_double2((r.x * d.x + r.y * d.y) / dd, (r.y * d.x - r.x * d.y) / dd);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = e0 + threadIdx.x; e < e1; e += GT) {
    double2 acc = I.Dv[e];
    for (int i = 0; i < k; ++i) {
      const double2 t = cmul(y[i], I.V[(size_t)i * I.nb + e]);
      acc.x += t.x;
      acc.y += t.y;
    }
    I.Dv[e] = acc;
  }
}

// x += Dv (Dv stays: the next check may apply it alone; every inner solve
// starts from gk_zero_dv)
__global__ void gk_axpy(const GInst* gi, const int* sel) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  if (!sel[blockIdx.y]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < I.nb; e += gridDim.x * blockDim.x) {
    I.x[e].x += I.Dv[e].x;
    I.x[e].y += I.Dv[e].y;
  }
}

__global__ void gk_zero_dv(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < I.nb; e += gridDim.x * blockDim.x)
    I.Dv[e] = make_double2(0.0, 0.0);
}

// W = A Dv is needed at a restart: copy Dv into V[m] slot? -- the fast
// operator reads V[j]; restarts place Dv into V[0] first (gk_dv_to_v0).
__global__ void gk_dv_to_v0(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  ACTIVE_OR_RETURN(I);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < I.nb; e += gridDim.x * blockDim.x)
    I.V[e] = I.Dv[e];
}

// ---- step updates ----------------------------------------------------------

__global__ void gk_step_update(const GInst* gi) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.y];
  const size_t plane = (size_t)I.Mp * I.Mp;
  if (I.eq == KFBI_HEAT) {
    const double four_dt = 4.0 / I.dt;
    INST_QUAD_LOOP(I) {
      const int r = (int)((unsigned)idx / (unsigned)I.Mp), c0 = (int)idx - r * I.Mp;
      const Quad uu = ldq(I.U64 + idx), F = ldq(I.F + idx);
      Quad f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        f.v[k] = four_dt * uu.v[k] - F.v[k];
        if (I.src && r < I.n1 && c0 + k < I.n1)
          f.v[k] += I.src_scale * I.src[(size_t)r * I.n1 + c0 + k];
      }
      stq(I.u + idx, uu);
      stq(I.F + idx, f);
    }
  } else if (I.eq == KFBI_WAVE) {
    const double k_theta = I.kre / I.theta, c1 = (1.0 - 2.0 * I.theta) / I.theta;
    INST_QUAD_LOOP(I) {
      const Quad uu = ldq(I.U64 + idx), f = ldq(I.F + idx), fp = ldq(I.Fprev + idx);
      Quad fn;
#pragma unroll
      for (int k = 0; k < 4; ++k) fn.v[k] = k_theta * uu.v[k] - c1 * f.v[k] - fp.v[k];
      stq(I.Fprev + idx, f);
      stq(I.F + idx, fn);
      stq(I.u + idx, uu);
    }
  } else {
    INST_QUAD_LOOP(I) {
      for (int p = 0; p < 2; ++p) {
        const size_t q = p * plane + idx;
        const Quad uu = ldq(I.U64 + q), ax = ldq(I.aux + q);
        Quad f;
#pragma unroll
        for (int k = 0; k < 4; ++k) f.v[k] = 2.0 * uu.v[k] - ax.v[k];
        stq(I.u + q, uu);
        stq(I.F + q, f);
      }
    }
  }
}

__global__ void gk_set_flags(const GInst* gi, const int* act, int x_zero_from_state) {
  KFBI_PDL_ENTRY();
  const GInst& I = gi[blockIdx.x];
  if (threadIdx.x == 0) {
    I.flags[0] = act[blockIdx.x];
    if (x_zero_from_state >= 0) I.flags[2] = x_zero_from_state ? act[gridDim.x + blockIdx.x] : 0;
  }
}

__global__ void gk_bump(int* dj) {
  KFBI_PDL_ENTRY();
  if (threadIdx.x == 0) *dj += 1;
}

}  // namespace bt
}  // namespace kfbi

// ============================================================================
// host side
// ============================================================================

using namespace kfbi;
using namespace kfbi::bt;
using kfbi::tc::PassDesc;
using kfbi::tc::GroupArgs;

struct kfbi_batch {
  int n = 0;    // bound instances
  int cap = 0;  // capacity of the per-instance device arrays
  int device = 0;
  int nsm = 148;
  std::vector<kfbi_domain*> doms;
  std::vector<kfbi_state*> states;  // bound at the first step
  std::vector<GInst> h_inst;
  GInst* d_inst = nullptr;
  int* d_flags = nullptr;       // 4 ints per instance
  int* d_j = nullptr;           // lockstep iteration index
  int* d_sel = nullptr;         // 2n ints (selection for axpy / flags)
  double* d_scal_all = nullptr; // 8 doubles per instance (readback staging)
  double* d_tol = nullptr;      // n inner tolerances
  double* h_scal = nullptr;     // pinned: 8 doubles per instance
  int* h_flags = nullptr;       // pinned: 4 ints per instance
  // state mailbox (gk_post): two host-mapped slots of 12 cap + 16 doubles,
  // the device's post counter and its host mirror
  double* h_mbox = nullptr;
  double* d_mbox = nullptr;
  long long* d_postctr = nullptr;
  long long host_posts = 0;
  // grouped pass descriptors and tile prefixes, per pass kind
  enum { kDense1, kDense2, kDense3, kDense4, kSparse2, kSparse3, kPassKinds };
  PassDesc* d_pass[kPassKinds] = {nullptr};
  int* d_prefix[kPassKinds] = {nullptr};
  int total[kPassKinds] = {0};
  double pass_work[kPassKinds] = {0};  // tensor flops of a pass over all instances
  int max_n_irr = 1, max_nb = 1, max_Mp = 128, max_nrows = 1, max_planes_blocks = 1;
  bool bound = false;
  // FFT32 instances: per pass kind one grouped launch per distinct M
  enum { kFftDense1, kFftSolve, kFftFinal, kFftSparse1, kFftSolveS, kFftKinds };
  struct FftPassGroup {
    int M = 0, nblocks = 0, rpb = 8;
    bool sparse = false;
    size_t smem = 0;
    double flops = 0.0, bytes = 0.0;
    FftDesc* d_desc = nullptr;
    int2* d_blk = nullptr;
    int cap_desc = 0, cap_blk = 0;
  };
  std::vector<FftPassGroup> fg[kFftKinds];
  std::vector<int> fft_ms;     // distinct M of the FFT instances
  std::vector<int> fft_rpb;    // rows per block of each M's passes
  std::map<int, int> rpb_of_M;  // autotuned rows per block, kept across rebinds
  std::vector<kfbi_batch_tuning_t> tuning;  // one record per tuned group
  int force = -1;               // >= 0: use this candidate everywhere, no timing
  std::vector<long long> fft_sig;  // launch shapes baked into the captured graph
  int n_fft = 0, n_tc = 0, n_cplx = 0;  // instance counts (FFT32, TF32, complex)
  int gather_mask = 0;                   // gather kernels in the captured iteration
  // autotuned launch shape of the grouped passes (CTAs per SM multiple,
  // tile order) and the CUDA graph of one lockstep GMRES iteration
  int tile_order = 0;  // 0: instances in given order, 1: largest first
  int splitk = 0;      // grouped passes: 0 from the tile count, 1, or 2 (CTA pairs)
  int cta_cap = 0;     // persistent CTAs of a pass without pairs: 0 one per SM, else this many
  bool tuned = false;  // the autotuner ran (its choice is kept across rebinds)
  cudaGraphExec_t iter_graph = nullptr;
  cudaStream_t graph_stream = nullptr;
  double tuned_us[2] = {0.0, 0.0};
  std::vector<int> grid_wx;  // last step: instance's U64 holds W phi at its final phi
  std::string err;
  long long launches = 0;
};

namespace {

dim3 inst_grid(int nblocks_x, int n) { return dim3((unsigned)std::max(1, nblocks_x), (unsigned)n); }

void build_fft_passes(kfbi_batch* B);

void build_passes(kfbi_batch* B) {
  build_fft_passes(B);
  // per-instance descriptors for the dense and sparse tensor passes of the
  // TF32 instances (kappa fixed by the states)
  std::vector<int> tci;
  for (int i = 0; i < B->n; ++i)
    if (!B->h_inst[i].fft) tci.push_back(i);
  B->n_tc = (int)tci.size();
  for (int kind = 0; kind < kfbi_batch::kPassKinds; ++kind) {
    const int nt = B->n_tc;
    std::vector<PassDesc> ds(nt);
    std::vector<int> pref(nt + 1, 0);
    for (int ii = 0; ii < nt; ++ii) {
      const int i = tci[ii];  // tile order is applied by the permutation below
      kfbi_domain* D = B->doms[i];
      TcDst* T = D->tc;
      const GInst& I = B->h_inst[i];
      const int P = I.C ? 2 : 1;
      PassDesc d{};
      d.b_hi = T->d_maps + kMapS_hi;
      d.b_lo = T->d_maps + kMapS_lo;
      d.lam = T->lam;
      d.Mp = T->Mp;
      d.n1 = T->n1;
      d.kb0 = 0;
      d.nk = T->Mp / tc::BK;
      d.ct0 = 0;
      d.nct = T->Mp / tc::BC;
      d.nrt = P * T->Mp / tc::BR;
      d.kre = 0.f;
      d.scale = 0.f;
      d.active = B->d_flags + 4 * i;
      const float scale = (float)((2.0 / D->M) * (2.0 / D->M));
      switch (kind) {
        case kfbi_batch::kDense1:
          d.a_hi = T->d_maps + kMapR_hi; d.a_lo = T->d_maps + kMapR_lo;
          d.out_hi = T->T1h; d.out_lo = T->T1l; d.mode = 0; break;
        case kfbi_batch::kDense2:
          d.a_hi = T->d_maps + kMapT1_hi; d.a_lo = T->d_maps + kMapT1_lo;
          d.out_hi = T->T2h; d.out_lo = T->T2l; d.mode = I.C ? 0 : 1;
          d.kre = (float)I.kre; d.scale = scale; break;
        case kfbi_batch::kDense3:
          d.a_hi = T->d_maps + kMapT2_hi; d.a_lo = T->d_maps + kMapT2_lo;
          d.out_hi = T->T1h; d.out_lo = T->T1l; d.mode = 0; break;
        case kfbi_batch::kDense4:
          d.a_hi = T->d_maps + kMapT1_hi; d.a_lo = T->d_maps + kMapT1_lo;
          d.out_hi = T->U; d.out_lo = nullptr; d.mode = 2; break;
        case kfbi_batch::kSparse2:
          d.a_hi = T->d_maps + kMapT1s_hi; d.a_lo = T->d_maps + kMapT1s_lo;
          d.out_hi = T->T2h; d.out_lo = T->T2l; d.mode = I.C ? 0 : 1;
          d.kre = (float)I.kre; d.scale = scale; d.kb0 = T->kb0; d.nk = T->nk2; break;
        case kfbi_batch::kSparse3:
          d.a_hi = T->d_maps + kMapT2_hi; d.a_lo = T->d_maps + kMapT2_lo;
          d.out_hi = T->U; d.out_lo = nullptr; d.mode = 2; d.ct0 = T->ct0; d.nct = T->nt3; break;
      }
      d.o_hi = tc_out_map(T, d.out_hi);
      d.o_lo = d.out_lo ? tc_out_map(T, d.out_lo) : nullptr;
      ds[ii] = d;
    }
    // tile order: optionally largest instances first (longest-processing-time
    // first keeps the persistent CTAs balanced)
    std::vector<int> order(nt);
    std::iota(order.begin(), order.end(), 0);
    if (B->tile_order == 1)
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)ds[a].nk * ds[a].nct * ds[a].nrt > (long long)ds[b].nk * ds[b].nct * ds[b].nrt;
      });
    std::vector<PassDesc> ordered(nt);
    for (int ii = 0; ii < nt; ++ii) {
      ordered[ii] = ds[order[ii]];
      pref[ii + 1] = pref[ii] + ordered[ii].nct * ordered[ii].nrt;
    }
    B->total[kind] = pref[nt];
    B->pass_work[kind] = 0.0;
    for (int ii = 0; ii < nt; ++ii) B->pass_work[kind] += tc::pass_flops(ordered[ii]);
    if (nt > 0) {
      KFBI_CUDA(cudaMemcpy(B->d_pass[kind], ordered.data(), sizeof(PassDesc) * nt, cudaMemcpyHostToDevice));
      KFBI_CUDA(cudaMemcpy(B->d_prefix[kind], pref.data(), sizeof(int) * (nt + 1), cudaMemcpyHostToDevice));
    }
  }
}

// Descriptors and block maps of the FFT instances' grouped passes: for each
// pass kind, one group per distinct M (one launch each), blocks of every
// instance of that size in instance order.  A change of launch shape (block
// count, rows per block, shared memory) invalidates the captured iteration
// graph.
void build_fft_passes(kfbi_batch* B) {
  std::vector<int> ms;
  for (int i = 0; i < B->n; ++i)
    if (B->h_inst[i].fft) ms.push_back(B->h_inst[i].M);
  std::sort(ms.begin(), ms.end());
  ms.erase(std::unique(ms.begin(), ms.end()), ms.end());
  B->fft_ms = ms;
  B->fft_rpb.assign(ms.size(), 8);
  for (size_t gi = 0; gi < ms.size(); ++gi) {
    auto it = B->rpb_of_M.find(ms[gi]);
    // untuned: 8 rows per block where a complex solve still fits, else 4
    B->fft_rpb[gi] = it != B->rpb_of_M.end() ? it->second : (fft_rpb_fits(ms[gi], 8, 2) ? 8 : 4);
  }
  B->n_fft = 0;
  for (int i = 0; i < B->n; ++i) B->n_fft += B->h_inst[i].fft ? 1 : 0;
  std::vector<long long> sig;
  for (int kind = 0; kind < kfbi_batch::kFftKinds; ++kind) {
    auto& groups = B->fg[kind];
    groups.resize(ms.size());
    for (size_t gi = 0; gi < ms.size(); ++gi) {
      kfbi_batch::FftPassGroup& g = groups[gi];
      g.M = ms[gi];
      g.sparse = kind == kfbi_batch::kFftSparse1;
      int rpb = B->fft_rpb[gi];
      std::vector<FftDesc> ds;
      std::vector<int2> blk;
      double flops = 0.0, bytes = 0.0;
      int pw_max = 1;
      for (int i = 0; i < B->n; ++i) {
        const GInst& I = B->h_inst[i];
        if (!I.fft || I.M != g.M) continue;
        kfbi_domain* D = B->doms[i];
        TcDst* T = D->tc;
        const int P = I.C ? 2 : 1;
        const float kre = (float)I.kre, kim = (float)I.kim, scale = (float)I.scale;
        FftDesc d{};
        switch (kind) {
          case kfbi_batch::kFftDense1:
            d = fft_desc(T, T->Rh, T->T1h, P, false, 0.f, 0.f, 0.f, nullptr, nullptr, rpb);
            break;
          case kfbi_batch::kFftSolve:
            d = fft_desc(T, T->T1h, T->T2h, P, true, kre, kim, scale, nullptr, nullptr, rpb);
            break;
          case kfbi_batch::kFftFinal:
            d = fft_desc(T, T->T2h, T->U, P, false, 0.f, 0.f, 0.f, nullptr, nullptr, rpb);
            d.transpose = 0;
            break;
          case kfbi_batch::kFftSparse1: {
            FftSparseRhs sp{};
            sp.row_start = T->row_start;
            sp.node_col = T->node_col;
            sp.arm_col = T->arm_col;
            sp.rmin = T->rmin;
            sp.nrows = T->nrows;
            sp.arm_start = D->d_arm_start;
            sp.arm_k0 = D->d_arm_k0;
            sp.alpha = D->d_arm_alpha32;
            sp.beta = D->d_arm_beta32;
            sp.n_arms = D->n_arms;
            sp.nb = D->nb;
            sp.phi = (const double*)I.V;  // V[*dj]: the Arnoldi vector of the iteration
            sp.ps = 2;
            sp.kre = kre;
            sp.kim = kim;
            sp.cplx = I.C;
            sp.dj = B->d_j;
            sp.dj_stride = 2LL * I.nb;
            d = fft_desc(T, nullptr, T->T1sh, P, false, 0.f, 0.f, 0.f, nullptr, &sp, rpb);
            break;
          }
          default:  // kFftSolveS
            d = fft_desc(T, T->T1sh, T->U, P, true, kre, kim, scale, nullptr, nullptr, rpb);
            break;
        }
        d.active = B->d_flags + 4 * i;
        const int li = (int)ds.size();
        for (int b = 0; b < fft_blocks(d); ++b) blk.push_back(make_int2(li, b));
        flops += fft_desc_flops(d, rpb);
        bytes += fft_desc_bytes(d, rpb);
        pw_max = std::max(pw_max, d.pw);
        ds.push_back(d);
      }
      g.rpb = rpb;
      g.nblocks = (int)blk.size();
      g.smem = fft_smem(g.M, rpb, pw_max);
      g.flops = flops;
      g.bytes = bytes;
      if ((int)ds.size() > g.cap_desc) {
        if (g.d_desc) KFBI_CUDA(cudaFree(g.d_desc));
        KFBI_CUDA(cudaMalloc(&g.d_desc, ds.size() * sizeof(FftDesc)));
        g.cap_desc = (int)ds.size();
      }
      if ((int)blk.size() > g.cap_blk) {
        if (g.d_blk) KFBI_CUDA(cudaFree(g.d_blk));
        KFBI_CUDA(cudaMalloc(&g.d_blk, blk.size() * sizeof(int2)));
        g.cap_blk = (int)blk.size();
      }
      if (!ds.empty())
        KFBI_CUDA(cudaMemcpy(g.d_desc, ds.data(), ds.size() * sizeof(FftDesc), cudaMemcpyHostToDevice));
      if (!blk.empty())
        KFBI_CUDA(cudaMemcpy(g.d_blk, blk.data(), blk.size() * sizeof(int2), cudaMemcpyHostToDevice));
      sig.insert(sig.end(), {(long long)g.M, (long long)g.nblocks, (long long)g.rpb, (long long)g.smem,
                             (long long)(uintptr_t)g.d_desc, (long long)(uintptr_t)g.d_blk});
    }
  }
  if (sig != B->fft_sig) {
    B->fft_sig = sig;
    if (B->iter_graph) {
      KFBI_CUDA(cudaGraphExecDestroy(B->iter_graph));
      B->iter_graph = nullptr;
    }
  }
}

void fft_group_launch(const kfbi_batch::FftPassGroup& g, int kind, cudaStream_t st) {
  if (g.nblocks == 0) return;
  FftGroup ga{};
  ga.descs = g.d_desc;
  ga.blk = g.d_blk;
  ga.rpb = g.rpb;
  fft_launch(ga, g.M, g.sparse, g.nblocks, g.smem,
             kind == kfbi_batch::kFftSparse1 ? KFBI_PROF_SPARSE : KFBI_PROF_DST, g.flops, g.bytes, st);
}

void fft_grouped(kfbi_batch* B, int kind, cudaStream_t st) {
  for (const kfbi_batch::FftPassGroup& g : B->fg[kind]) fft_group_launch(g, kind, st);
}

void grouped_pass(kfbi_batch* B, int kind, cudaStream_t st) {
  if (B->n_tc == 0) return;
  GroupArgs ga;
  ga.descs = B->d_pass[kind];
  ga.prefix = B->d_prefix[kind];
  ga.n_inst = B->n_tc;
  ga.total = B->total[kind];
  ga.one = PassDesc{};
  ga.err = B->doms[0]->tc->err;
  ga.splitk = B->splitk;
  tc::launch_tc_pass(ga, B->nsm, B->pass_work[kind], st, B->cta_cap);
}

int plane_blocks(kfbi_batch* B) { return B->max_planes_blocks; }

// accurate application for all active instances: which = 0 (zero density),
// 1 (x); with_ft; result grid in U64, u+ into ub (target 0) or Ax (1)
void batch_accurate(kfbi_batch* B, int which, int with_ft, int target, cudaStream_t st) {
  const int n = B->n;
  const int pb = plane_blocks(B);
  KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_base_rhs, inst_grid(pb, n), 256, 0, st, B->d_inst, with_ft);
  KFBI_LAUNCH_P(KFBI_PROF_CORRECT, gk_correct64, inst_grid((B->max_n_irr + 127) / 128, n), 128, 0, st,
                B->d_inst, which, with_ft, (const int*)nullptr);
  if (B->n_tc > 0) KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_split64, inst_grid(pb, n), 256, 0, st, B->d_inst);
  for (int sweep = 0; sweep < 2; ++sweep) {
    if (B->n_tc > 0) {
      grouped_pass(B, kfbi_batch::kDense1, st);
      grouped_pass(B, kfbi_batch::kDense2, st);
      KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_eig_cplx, inst_grid(pb, n), 256, 0, st, B->d_inst);
      grouped_pass(B, kfbi_batch::kDense3, st);
      grouped_pass(B, kfbi_batch::kDense4, st);
    }
    if (B->n_fft > 0) {
      fft_grouped(B, kfbi_batch::kFftDense1, st);
      fft_grouped(B, kfbi_batch::kFftSolve, st);
      fft_grouped(B, kfbi_batch::kFftFinal, st);
    }
    if (sweep == 0) {
      if (B->n_tc > 0) {
        KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_f32_to_f64, inst_grid(pb, n), 256, 0, st, B->d_inst);
        KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_resid_split, inst_grid(pb, n), 256, 0, st, B->d_inst);
      }
      if (B->n_fft > 0)
        KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_resid_u32, inst_grid(pb, n), 256, 0, st, B->d_inst);
    } else {
      KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_add_f32, inst_grid(pb, n), 256, 0, st, B->d_inst);
    }
  }
  KFBI_LAUNCH_P(KFBI_PROF_EXTRACT, gk_extract64, inst_grid((B->max_nb + 127) / 128, n), 128, 0, st,
                B->d_inst, which, with_ft, target);
  KFBI_CHECK_LAUNCH();
}

// Application at x = x_prev + Dv for the active instances, from the grid of
// an accurate application at x_prev in U64 (as tc_apply_correction): one
// unrefined box solve of the correction Dv added to U64, then the FP64
// extraction at x into Ax.
void batch_correction(kfbi_batch* B, cudaStream_t st) {
  const int n = B->n;
  const int pb = plane_blocks(B);
  KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_base_rhs, inst_grid(pb, n), 256, 0, st, B->d_inst, 0);
  KFBI_LAUNCH_P(KFBI_PROF_CORRECT, gk_correct64, inst_grid((B->max_n_irr + 127) / 128, n), 128, 0, st,
                B->d_inst, 3, 0, (const int*)nullptr);
  if (B->n_tc > 0) {
    KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_split64, inst_grid(pb, n), 256, 0, st, B->d_inst);
    grouped_pass(B, kfbi_batch::kDense1, st);
    grouped_pass(B, kfbi_batch::kDense2, st);
    KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_eig_cplx, inst_grid(pb, n), 256, 0, st, B->d_inst);
    grouped_pass(B, kfbi_batch::kDense3, st);
    grouped_pass(B, kfbi_batch::kDense4, st);
  }
  if (B->n_fft > 0) {
    fft_grouped(B, kfbi_batch::kFftDense1, st);
    fft_grouped(B, kfbi_batch::kFftSolve, st);
    fft_grouped(B, kfbi_batch::kFftFinal, st);
  }
  KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_add_f32, inst_grid(pb, n), 256, 0, st, B->d_inst);
  KFBI_LAUNCH_P(KFBI_PROF_EXTRACT, gk_extract64, inst_grid((B->max_nb + 127) / 128, n), 128, 0, st,
                B->d_inst, 1, 0, 1);
  KFBI_CHECK_LAUNCH();
}

// W = A_fast V[j] for every active instance: the sparse route (TF32
// instances: correction values, CUDA-core first pass, two restricted tensor
// passes; FFT instances: first pass built from the arms, solve pass), then
// the gather at the stencil points with the extraction.
void fast_apply(kfbi_batch* B, cudaStream_t st) {
  const int n = B->n;
  if (B->n_tc > 0) {
    KFBI_LAUNCH_P(KFBI_PROF_CORRECT, gk_correct32_rv, inst_grid((B->max_n_irr + 127) / 128, n), 128, 0,
                  st, B->d_inst, (const int*)B->d_j);
    KFBI_LAUNCH_P(KFBI_PROF_SPARSE, gk_sparse_p1, dim3(B->max_Mp / 32, (B->max_nrows + 31) / 32, n),
                  dim3(32, 8), 0, st, B->d_inst);
    grouped_pass(B, kfbi_batch::kSparse2, st);
    KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_eig_cplx, inst_grid(plane_blocks(B), n), 256, 0, st, B->d_inst);
    grouped_pass(B, kfbi_batch::kSparse3, st);
  }
  if (B->n_fft > 0) {
    fft_grouped(B, kfbi_batch::kFftSparse1, st);
    fft_grouped(B, kfbi_batch::kFftSolveS, st);
  }
  const dim3 gg = inst_grid((B->max_nb + GB_NODES - 1) / GB_NODES, n);
  if (B->n_cplx < n)
    KFBI_LAUNCH_P(KFBI_PROF_EXTRACT, gk_gather_extract<false>, gg, 32 * GB_NODES, 0, st, B->d_inst,
                  (const int*)B->d_j);
  if (B->n_cplx > 0)
    KFBI_LAUNCH_P(KFBI_PROF_EXTRACT, gk_gather_extract<true>, gg, 32 * GB_NODES, 0, st, B->d_inst,
                  (const int*)B->d_j);
}

// The state post kernel alone (inside a captured iteration the host counts
// the posts per replay).
void launch_post(kfbi_batch* B, cudaStream_t st) {
  KFBI_LAUNCH(gk_post, 1, 256, 0, st, (const GInst*)B->d_inst, B->n, B->d_mbox,
              (int)(12 * (size_t)B->cap + 16), B->cap, B->d_postctr);
}

// one lockstep GMRES iteration: W = A_fast V[j], CGS2 Arnoldi, j += 1, and
// the post of every instance's state
void batch_iteration(kfbi_batch* B, cudaStream_t st) {
  const int n = B->n;
  fast_apply(B, st);
  if (B->max_nb <= kArnoldiMaxNb) {
    // one block per instance
    const size_t smem = (size_t)B->max_nb * sizeof(double2);
    if (B->n_cplx < n)
      KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_arnoldi<false>, n, AT, smem, st, B->d_inst,
                    (const int*)B->d_j);
    if (B->n_cplx > 0)
      KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_arnoldi<true>, n, AT, smem, st, B->d_inst,
                    (const int*)B->d_j);
  } else {
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_cgs_dots, inst_grid(GMAX, n), GT, 0, st, B->d_inst,
                  (const int*)B->d_j);
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_cgs_update, inst_grid(GMAX, n), GT, 0, st, B->d_inst,
                  (const int*)B->d_j, 1, 0);
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_cgs_update, inst_grid(GMAX, n), GT, 0, st, B->d_inst,
                  (const int*)B->d_j, 0, 1);
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_cgs_finalize, inst_grid(GMAX, n), GT, 0, st, B->d_inst,
                  (const int*)B->d_j);
  }
  KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_bump, 1, 32, 0, st, B->d_j);
  launch_post(B, st);
  KFBI_CHECK_LAUNCH();
}

// Queue a state post (gk_post); returns the sequence number it will carry.
long long post_state(kfbi_batch* B, cudaStream_t st) {
  launch_post(B, st);
  return ++B->host_posts;
}

// Wait for post q and copy its scalars and flags into h_scal / h_flags.
void wait_state(kfbi_batch* B, long long q, cudaStream_t st) {
  const size_t stride = 12 * (size_t)B->cap + 16;
  volatile double* slot = B->h_mbox + (q & 1) * stride;
  volatile long long* seq = reinterpret_cast<volatile long long*>(slot + stride - 1);
  const auto t0 = std::chrono::steady_clock::now();
  for (long long spins = 1; *seq != q; ++spins) {
    if ((spins & 255) != 0) continue;
    const cudaError_t e = cudaStreamQuery(st);
    if (e != cudaSuccess && e != cudaErrorNotReady) KFBI_CUDA(e);
    if (e == cudaSuccess && *seq != q)
      throw Status{KFBI_ERR_CUDA, "batch state post missing after the stream drained"};
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60))
      throw Status{KFBI_ERR_TIMEOUT, "no batch state within 60 s"};
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  const int n = B->n;
  for (int i = 0; i < 8 * n; ++i) B->h_scal[i] = slot[i];
  const volatile int* fl = reinterpret_cast<const volatile int*>(slot + 8 * (size_t)B->cap);
  for (int i = 0; i < 4 * n; ++i) B->h_flags[i] = fl[i];
  for (int i = 0; i < n; ++i) {
    int f = 0;
    std::memcpy(&f, B->h_scal + 8 * i + 6, sizeof(int));
    if (f) throw Status{KFBI_ERR_TIMEOUT, "a tensor-core DST pass gave up waiting on its pipeline"};
  }
}

void read_state(kfbi_batch* B, cudaStream_t st) { wait_state(B, post_state(B, st), st); }

void set_active(kfbi_batch* B, const std::vector<int>& act, const std::vector<int>* xz, cudaStream_t st) {
  std::vector<int> buf(act);
  if (xz) buf.insert(buf.end(), xz->begin(), xz->end());
  KFBI_CUDA(cudaMemcpyAsync(B->d_sel, buf.data(), buf.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  KFBI_LAUNCH(gk_set_flags, B->n, 32, 0, st, B->d_inst, (const int*)B->d_sel, xz ? 1 : -1);
  KFBI_CHECK_LAUNCH();
}

// Per-instance device arrays for at least n instances (contents are
// rebuilt by every step).
void batch_reserve(kfbi_batch* B, int n) {
  if (n <= B->cap) return;
  KFBI_CUDA(cudaDeviceSynchronize());
  void* ds[] = {B->d_inst, B->d_flags, B->d_sel, B->d_scal_all, B->d_tol};
  for (void* p : ds)
    if (p) cudaFree(p);
  for (int k = 0; k < kfbi_batch::kPassKinds; ++k) {
    if (B->d_pass[k]) cudaFree(B->d_pass[k]);
    if (B->d_prefix[k]) cudaFree(B->d_prefix[k]);
    B->d_pass[k] = nullptr;
    B->d_prefix[k] = nullptr;
  }
  if (B->h_scal) cudaFreeHost(B->h_scal);
  if (B->h_flags) cudaFreeHost(B->h_flags);
  if (B->h_mbox) cudaFreeHost(B->h_mbox);
  B->d_inst = nullptr; B->d_flags = nullptr; B->d_sel = nullptr; B->d_scal_all = nullptr;
  B->d_tol = nullptr; B->h_scal = nullptr; B->h_flags = nullptr; B->h_mbox = nullptr;
  B->d_mbox = nullptr;
  const int c = std::max(n, 2 * B->cap);
  B->cap = 0;
  KFBI_CUDA(cudaMalloc(&B->d_inst, sizeof(GInst) * c));
  KFBI_CUDA(cudaMalloc(&B->d_flags, sizeof(int) * 4 * c));
  KFBI_CUDA(cudaMemset(B->d_flags, 0, sizeof(int) * 4 * c));
  KFBI_CUDA(cudaMalloc(&B->d_sel, sizeof(int) * 2 * c));
  KFBI_CUDA(cudaMalloc(&B->d_scal_all, sizeof(double) * 8 * c));
  KFBI_CUDA(cudaMalloc(&B->d_tol, sizeof(double) * c));
  KFBI_CUDA(cudaMallocHost(&B->h_scal, sizeof(double) * 8 * c));
  KFBI_CUDA(cudaMallocHost(&B->h_flags, sizeof(int) * 4 * c));
  {
    const size_t bytes = 2 * (12 * (size_t)c + 16) * sizeof(double);
    KFBI_CUDA(cudaHostAlloc(&B->h_mbox, bytes, cudaHostAllocMapped));
    std::memset(B->h_mbox, 0, bytes);
    KFBI_CUDA(cudaHostGetDevicePointer((void**)&B->d_mbox, B->h_mbox, 0));
  }
  for (int k = 0; k < kfbi_batch::kPassKinds; ++k) {
    KFBI_CUDA(cudaMalloc(&B->d_pass[k], sizeof(PassDesc) * c));
    KFBI_CUDA(cudaMalloc(&B->d_prefix[k], sizeof(int) * (c + 1)));
  }
  B->cap = c;
}

}  // namespace

namespace kfbi {

kfbi_batch* batch_new() {
  kfbi_batch* B = new kfbi_batch();
  KFBI_CUDA(cudaGetDevice(&B->device));
  KFBI_CUDA(cudaDeviceGetAttribute(&B->nsm, cudaDevAttrMultiProcessorCount, B->device));
  KFBI_CUDA(cudaMalloc(&B->d_j, sizeof(int)));
  KFBI_CUDA(cudaMalloc(&B->d_postctr, sizeof(long long)));
  KFBI_CUDA(cudaMemset(B->d_postctr, 0, sizeof(long long)));
  B->host_posts = 0;
  return B;
}

void batch_bind(kfbi_batch* B, kfbi_domain* const* domains, int n) {
  if (!domains || n < 1 || n > 4096) throw Status{KFBI_ERR_ARG, "a batch holds 1 to 4096 domains"};
  for (int i = 0; i < n; ++i)
    if (!domains[i] || !domains[i]->tc || domains[i]->n_irr == 0 ||
        domains[i]->restart != domains[0]->restart || domains[i]->desc.solver != KFBI_GMRES)
      throw Status{KFBI_ERR_ARG,
                   "every domain of a batch must be KFBI_MIXED_TF32 or KFBI_MIXED_FFT32 with an "
                   "interface, the GMRES solver and the same gmres_restart"};
  batch_reserve(B, n);
  if (B->iter_graph) {
    KFBI_CUDA(cudaGraphExecDestroy(B->iter_graph));
    B->iter_graph = nullptr;
  }
  B->bound = false;
  B->n = n;
  B->doms.assign(domains, domains + n);
  B->max_n_irr = 1; B->max_nb = 1; B->max_Mp = 128; B->max_nrows = 1;
  for (int i = 0; i < n; ++i) {
    kfbi_domain* D = domains[i];
    B->max_n_irr = std::max(B->max_n_irr, D->n_irr);
    B->max_nb = std::max(B->max_nb, D->nb);
    B->max_Mp = std::max(B->max_Mp, D->Mp);
    B->max_nrows = std::max(B->max_nrows, D->tc->nrows);
  }
  // grid-stride plane kernels: up to 8 points per thread on the largest
  // plane, at least 8 blocks per SM over the batch (one block per 256 points
  // left most blocks of a mixed-size batch with nothing to do)
  const int full = (B->max_Mp * B->max_Mp + 255) / 256;
  int pb = std::max((full + 7) / 8, (B->nsm * 8 + n - 1) / n);
  B->max_planes_blocks = std::max(1, std::min({pb, full, 1024}));
  // the limit is a property of the kernel, shared by every batch (and
  // server lane): set once, to the largest staging any batch uses
  static std::once_flag arnoldi_attr;
  std::call_once(arnoldi_attr, []() {
    const int smem = (int)(kArnoldiMaxNb * sizeof(double2));
    KFBI_CUDA(cudaFuncSetAttribute(gk_arnoldi<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    KFBI_CUDA(cudaFuncSetAttribute(gk_arnoldi<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  });
}

}  // namespace kfbi

extern "C" {

kfbi_status kfbi_batch_create(kfbi_domain* const* domains, int n, void* stream, kfbi_batch** out) {
  if (!out) return KFBI_ERR_ARG;
  *out = nullptr;
  kfbi_batch* B = nullptr;
  kfbi_status s = guarded(nullptr, [&]() -> kfbi_status {
    B = batch_new();
    batch_bind(B, domains, n);
    KFBI_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return KFBI_OK;
  });
  if (s != KFBI_OK) {
    kfbi_batch_destroy(B);
    return s;
  }
  *out = B;
  return KFBI_OK;
}

void kfbi_batch_destroy(kfbi_batch* B) {
  if (!B) return;
  cudaDeviceSynchronize();
  if (B->iter_graph) cudaGraphExecDestroy(B->iter_graph);
  for (int k = 0; k < kfbi_batch::kPassKinds; ++k) {
    if (B->d_pass[k]) cudaFree(B->d_pass[k]);
    if (B->d_prefix[k]) cudaFree(B->d_prefix[k]);
  }
  for (int k = 0; k < kfbi_batch::kFftKinds; ++k)
    for (auto& g : B->fg[k]) {
      if (g.d_desc) cudaFree(g.d_desc);
      if (g.d_blk) cudaFree(g.d_blk);
    }
  void* ps[] = {B->d_inst, B->d_flags, B->d_j, B->d_sel, B->d_scal_all, B->d_tol};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (B->h_scal) cudaFreeHost(B->h_scal);
  if (B->h_flags) cudaFreeHost(B->h_flags);
  if (B->h_mbox) cudaFreeHost(B->h_mbox);
  if (B->d_postctr) cudaFree(B->d_postctr);
  delete B;
}

const char* kfbi_batch_last_error(const kfbi_batch* B) { return B ? B->err.c_str() : ""; }

}  // extern "C"

namespace {

// Fill the per-instance descriptors for the bound states and this step's
// boundary data / sources.
void fill_instances(kfbi_batch* B, kfbi_state* const* states, const void* const* g_next,
                    const double* const* src, const double* src_scale) {
  B->h_inst.resize(B->n);
  B->n_cplx = 0;
  for (int i = 0; i < B->n; ++i) {
    kfbi_domain* D = B->doms[i];
    kfbi_state* S = states[i];
    B->n_cplx += S->kim != 0.0 ? 1 : 0;
    TcDst* T = D->tc;
    GInst I{};
    I.Mp = D->Mp; I.n1 = D->n1; I.nb = D->nb; I.n_irr = D->n_irr; I.n_arms = D->n_arms;
    I.fft = T->fft ? 1 : 0; I.T1h = T->T1h;
    {
      const double ih2 = 1.0 / (D->h * D->h);
      I.ih_hi = (float)ih2; I.ih_lo = (float)(ih2 - (double)I.ih_hi);
      I.kr_hi = (float)S->kre; I.kr_lo = (float)(S->kre - (double)I.kr_hi);
      I.ki_hi = (float)S->kim; I.ki_lo = (float)(S->kim - (double)I.ki_hi);
    }
    I.M = D->M; I.m = D->restart; I.C = S->kim != 0.0; I.eq = S->eq;
    I.rmin = T->rmin; I.nrows = T->nrows;
    I.h = D->h; I.kre = S->kre; I.kim = S->kim; I.scale = (2.0 / D->M) * (2.0 / D->M);
    I.dt = S->dt; I.theta = S->theta; I.w = S->w;
    I.mask = D->d_mask; I.irr_off = D->d_irr_off; I.arm_start = D->d_arm_start; I.arm_k0 = D->d_arm_k0;
    I.alpha = D->d_arm_alpha; I.beta = D->d_arm_beta; I.arm_fidx = D->d_arm_fidx;
    I.arm_fcoef = D->d_arm_fcoef; I.node_gidx = D->d_node_gidx; I.node_w = D->d_node_w;
    I.node_a = D->d_node_a; I.node_b = D->d_node_b; I.node_fidx = D->d_node_fidx;
    I.node_fcoef = D->d_node_fcoef; I.lam64 = D->d_lam; I.lam32 = T->lam;
    I.alpha32 = D->d_arm_alpha32; I.beta32 = D->d_arm_beta32; I.arm_fcoef32 = D->d_arm_fcoef32;
    I.node_w32 = D->d_node_w32; I.node_a32 = D->d_node_a32; I.node_b32 = D->d_node_b32;
    I.S32 = T->S32; I.row_start = T->row_start; I.node_col = T->node_col;
    I.R64 = D->d_R; I.U64 = D->d_U; I.Rh = T->Rh; I.Rl = T->Rl; I.T2h = T->T2h; I.T2l = T->T2l;
    I.fth = T->T1l; I.ftl = T->T2l;
    I.U32 = T->U; I.T1sh = T->T1sh; I.T1sl = T->T1sl; I.rv = T->rv;
    I.V = (double2*)D->d_V; I.W = (double2*)D->d_W; I.H = (double2*)D->d_H; I.cs = D->d_cs;
    I.sn = (double2*)D->d_sn; I.g = (double2*)D->d_g; I.hcol = (double2*)D->d_hcol;
    I.part = (double2*)D->d_part; I.Rv = (double2*)D->d_Rv; I.Dv = (double2*)D->d_Dv;
    I.Ax = (double2*)D->d_Ax; I.scal = D->d_scal;
    I.u = S->d_u; I.F = S->d_F; I.Fprev = S->d_Fprev; I.ft = S->d_ft; I.aux = S->d_aux;
    I.uf = S->d_uf; I.axc = (double2*)S->d_ax;
    I.x = (double2*)S->d_phi; I.b = (double2*)S->d_b; I.ub = (double2*)S->d_ub;
    I.g_next = (const double*)g_next[i];
    I.src = src ? src[i] : nullptr;
    I.src_scale = src_scale ? src_scale[i] : 1.0;
    I.flags = B->d_flags + 4 * i;
    B->h_inst[i] = I;
  }
  KFBI_CUDA(cudaMemcpy(B->d_inst, B->h_inst.data(), sizeof(GInst) * B->n, cudaMemcpyHostToDevice));
  // the captured iteration launches the real and/or the complex gather
  const int gmask = (B->n_cplx < B->n ? 1 : 0) | (B->n_cplx > 0 ? 2 : 0);
  if (gmask != B->gather_mask) {
    B->gather_mask = gmask;
    if (B->iter_graph) {
      KFBI_CUDA(cudaGraphExecDestroy(B->iter_graph));
      B->iter_graph = nullptr;
    }
  }
}

// Refinement GMRES for every instance, lockstep (see gmres_solve).  An
// instance whose residual turns non-finite is switched off and reported in
// its info (converged 0, rel_residual NaN); the others carry on.  Returns
// KFBI_ERR_NONFINITE if any instance went non-finite, else
// KFBI_ERR_NOT_CONVERGED if any reached gmres_maxit, else KFBI_OK.
kfbi_status batch_gmres(kfbi_batch* B, kfbi_solve_info* infos, cudaStream_t st) {
  const int n = B->n;
  const double kInnerFloor = 1e-6;
  std::vector<int> act(n, 1), xz(n), conv(n, 0), iters(n, 0), apps(n, 0), bad(n, 0);
  std::vector<int> ax_ok(n), fresh(n, 0);
  std::vector<double> bnorm(n, 0.0), rn(n, 0.0);
  // small final corrections (as gmres_solve): r_prev the residual the last
  // correction was solved for, err the bound on |A x - Ax| left by
  // correction applications since the last refined one
  const double kFastRelLinf = 2e-5;
  std::vector<double> r_prev(n, 0.0), err(n, 0.0);
  B->grid_wx.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    xz[i] = B->states[i]->phi_zero ? 1 : 0;
    ax_ok[i] = !xz[i] && B->states[i]->ax_valid && B->states[i]->d_ax ? 1 : 0;
    B->states[i]->ax_valid = false;
    B->states[i]->hist = false;  // batched steps keep no extrapolation history
  }
  // ||b||
  set_active(B, act, &xz, st);
  KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_bnorm, inst_grid(1, n), 1024, 0, st, B->d_inst,
                B->doms[0]->desc.gmres_tol, 0);
  read_state(B, st);
  for (int i = 0; i < n; ++i) bnorm[i] = B->h_scal[8 * i];
  for (int sweep = 0; sweep < 8; ++sweep) {
    // residual r = b - A_accurate x for instances still active; at the
    // first sweep an instance whose A phi is cached (its phi is the
    // previous step's converged phi) copies it instead
    set_active(B, act, &xz, st);
    std::vector<int> need(n), cached(n), corr(n);
    bool any_acc = false, any_cached = false, any_corr = false;
    for (int i = 0; i < n; ++i) {
      const bool has = act[i] && !xz[i];
      cached[i] = has && sweep == 0 && ax_ok[i];
      const double tol = B->doms[i]->desc.gmres_tol;
      const double e = err[i] + 2.0 * kFastRelLinf * std::sqrt((double)B->doms[i]->nb) * r_prev[i];
      corr[i] = has && sweep > 0 && fresh[i] && !B->doms[i]->neumann && e <= 0.1 * tol * bnorm[i];
      need[i] = has && !cached[i] && !corr[i];
      if (corr[i]) err[i] = e;
      else if (has) err[i] = 0.0;
      fresh[i] = need[i] || corr[i];
      any_acc |= need[i] != 0;
      any_cached |= cached[i] != 0;
      any_corr |= corr[i] != 0;
    }
    if (any_cached) {
      set_active(B, cached, nullptr, st);
      KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_ax_cache, inst_grid((B->max_nb + 255) / 256, n), 256, 0, st,
                    B->d_inst, 0);
    }
    if (any_acc) {
      set_active(B, need, nullptr, st);
      batch_accurate(B, 1, 0, 1, st);
      for (int i = 0; i < n; ++i) apps[i] += need[i];
    }
    if (any_corr) {
      set_active(B, corr, nullptr, st);
      batch_correction(B, st);
      for (int i = 0; i < n; ++i) apps[i] += corr[i];
    }
    if (any_cached || any_acc || any_corr) set_active(B, act, &xz, st);
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_residual, inst_grid(1, n), 1024, 0, st, B->d_inst);
    read_state(B, st);
    bool any = false;
    std::vector<double> inner_tol(n, 1.0);
    for (int i = 0; i < n; ++i) {
      if (!act[i]) continue;
      rn[i] = B->h_scal[8 * i + 1];
      if (!std::isfinite(rn[i]) || !std::isfinite(bnorm[i])) {
        bad[i] = 1;
        act[i] = 0;
        continue;
      }
      const double tol = B->doms[i]->desc.gmres_tol;
      const bool ok = rn[i] + err[i] <= tol * bnorm[i];
      if (bnorm[i] == 0.0 || ok || iters[i] >= B->doms[i]->desc.gmres_maxit) {
        conv[i] = ok || bnorm[i] == 0.0;
        B->grid_wx[i] = conv[i] && fresh[i];
        act[i] = 0;
        continue;
      }
      r_prev[i] = rn[i];
      inner_tol[i] = std::max(0.5 * tol * bnorm[i] / rn[i], kInnerFloor);
      any = true;
    }
    if (!any) break;
    for (int i = 0; i < n; ++i) xz[i] = 0;
    // inner GMRES on A_fast d = r, d = 0, lockstep over the active set;
    // the instance's tolerance relative to its ||r|| goes into scal[3]
    std::vector<int> inner(act);
    set_active(B, inner, &xz, st);
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_zero_dv, inst_grid(8, n), 256, 0, st, B->d_inst);
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_bnorm, inst_grid(1, n), 1024, 0, st, B->d_inst, 1.0, 1);
    KFBI_CUDA(cudaMemcpyAsync(B->d_tol, inner_tol.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    KFBI_CUDA(cudaMemcpyAsync(B->d_sel, inner.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    KFBI_LAUNCH(gk_set_tol, n, 32, 0, st, B->d_inst, (const double*)B->d_tol, (const int*)B->d_sel);
    bool first_cycle = true;
    for (int cycle = 0; cycle < 64; ++cycle) {
      bool any_inner = false;
      for (int i = 0; i < n; ++i) any_inner |= inner[i] != 0;
      if (!any_inner) break;
      set_active(B, inner, nullptr, st);
      if (!first_cycle) {
        // restart: W = A_fast Dv (Dv staged in V[0]) then r = Rv - W
        KFBI_CUDA(cudaMemsetAsync(B->d_j, 0, sizeof(int), st));
        KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_dv_to_v0, inst_grid(8, n), 256, 0, st, B->d_inst);
        fast_apply(B, st);
      }
      KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_restart, inst_grid(1, n), 1024, 0, st, B->d_inst,
                    first_cycle ? 0 : 1);
      first_cycle = false;
      KFBI_CUDA(cudaMemsetAsync(B->d_j, 0, sizeof(int), st));
      read_state(B, st);
      int m = 0;
      for (int i = 0; i < n; ++i) {
        if (!inner[i]) continue;
        m = std::max(m, B->doms[i]->restart);
        if (B->h_scal[8 * i + 2] != 0.0) inner[i] = 0;  // converged at the restart
      }
      bool any_left = false;
      for (int i = 0; i < n; ++i) any_left |= inner[i] != 0;
      if (!any_left) break;
      // iteration j + 1 is queued before the host reads iteration j's posted
      // state, so the GPU does not wait for the host between iterations;
      // instances that converged at j are inactive on the device and skip
      // j + 1, and when all have, the queued iteration's kernels only return
      std::vector<long long> qj(m + 1, 0);
      int queued = -1;
      auto queue = [&](int j) {
        if (B->iter_graph) {
          KFBI_CUDA(cudaGraphLaunch(B->iter_graph, st));
          g_launches.fetch_add(B->launches);
        } else {
          batch_iteration(B, st);
        }
        qj[j] = ++B->host_posts;  // the iteration ends with one state post
        queued = j;
      };
      for (int j = 0; j < m; ++j) {
        if (queued < j) queue(j);
        if (j + 1 < m) queue(j + 1);
        wait_state(B, qj[j], st);
        bool still = false;
        for (int i = 0; i < n; ++i) {
          if (!inner[i]) continue;
          ++iters[i];
          ++apps[i];
          if (B->h_flags[4 * i] == 0) {
            if (B->h_scal[8 * i + 2] == 2.0) {
              // non-finite GMRES residual: drop the instance from the sweeps
              bad[i] = 1;
              act[i] = 0;
            }
            inner[i] = 0;  // converged (or dropped)
          }
          still |= inner[i] != 0;
        }
        if (!still) break;
      }
      // x-update for every instance that iterated this cycle (k = flags[1])
      KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_update, inst_grid(GMAX, n), GT, 0, st, B->d_inst);
      // instances still active after m iterations restart (unless out of iterations)
      for (int i = 0; i < n; ++i)
        if (inner[i] && iters[i] >= B->doms[i]->desc.gmres_maxit) inner[i] = 0;
      // clear k so a finished instance does not update twice
      KFBI_LAUNCH(gk_clear_k, n, 32, 0, st, B->d_inst);
      KFBI_CHECK_LAUNCH();
    }
    // x += d for the instances that ran the inner solve
    std::vector<int> ran(n);
    for (int i = 0; i < n; ++i) ran[i] = act[i] && !bad[i];
    KFBI_CUDA(cudaMemcpyAsync(B->d_sel, ran.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_axpy, inst_grid(8, n), 256, 0, st, B->d_inst, (const int*)B->d_sel);
    KFBI_CHECK_LAUNCH();
  }
  bool any_wx = false;
  for (int i = 0; i < n; ++i) any_wx |= B->grid_wx[i] != 0;
  if (any_wx) {
    set_active(B, B->grid_wx, nullptr, st);
    KFBI_LAUNCH_P(KFBI_PROF_KRYLOV, gk_ax_cache, inst_grid((B->max_nb + 255) / 256, n), 256, 0, st,
                  B->d_inst, 1);
  }
  for (int i = 0; i < n; ++i) B->states[i]->ax_valid = B->grid_wx[i] != 0;
  KFBI_CUDA(cudaStreamSynchronize(st));
  bool any_bad = false, any_unconv = false;
  for (int i = 0; i < n; ++i) {
    if (bad[i]) conv[i] = 0;
    if (infos) {
      infos[i].iters = iters[i];
      infos[i].applications = apps[i] + (B->grid_wx[i] ? 1 : 2);
      infos[i].rel_residual = bad[i] ? std::nan("") : (bnorm[i] > 0.0 ? rn[i] / bnorm[i] : 0.0);
      infos[i].converged = conv[i];
    }
    any_bad |= bad[i] != 0;
    any_unconv |= !conv[i] && !bad[i];
    B->states[i]->phi_zero = false;
  }
  if (any_bad) {
    B->err = "non-finite density residual in an instance";
    return KFBI_ERR_NONFINITE;
  }
  if (any_unconv) {
    B->err = "GMRES with refinement reached gmres_maxit for an instance";
    return KFBI_ERR_NOT_CONVERGED;
  }
  return KFBI_OK;
}

// Capture one lockstep iteration into a CUDA graph (kernel arguments are
// fixed: the iteration index and the active flags live in device memory).
void capture_iteration(kfbi_batch* B) {
  if (B->iter_graph) return;
  cudaStream_t cs;
  KFBI_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph;
  const long long before = g_launches.load();
  KFBI_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  const bool prof = g_prof_on;
  g_prof_on = false;  // no event records inside the graph
  batch_iteration(B, cs);
  g_prof_on = prof;
  KFBI_CUDA(cudaStreamEndCapture(cs, &graph));
  KFBI_CUDA(cudaGraphInstantiate(&B->iter_graph, graph, 0));
  KFBI_CUDA(cudaGraphDestroy(graph));
  KFBI_CUDA(cudaStreamDestroy(cs));
  B->launches = g_launches.load() - before;  // kernels per graph replay
  g_launches.fetch_sub(B->launches);
}

// Autotuner.  The candidates of each group are timed on the group's fast
// application (the passes a GMRES iteration runs) with CUDA events: one
// warm-up and three timed repetitions, the fastest kept.
//  - FFT instances, one group per grid size M: rows (warps) per block of the
//    FFT passes, 8 or 4 (4 only where a complex solve does not fit 8); the
//    choice is cached per M and kept across rebinds.
//  - TF32 instances (all sizes in one persistent launch per pass): tile
//    order (instances as given, or largest first) x persistent CTAs (one per
//    SM, or half as many taking twice the tiles each).  Split K stays with
//    the tile-count rule of launch_tc_pass: CTA pairs change the order in
//    which a tile's K range is summed, and a timed choice could then give an
//    instance other bits in another batch.  Every candidate of both engines
//    leaves each tile's and each row's arithmetic unchanged.
// B->force >= 0 skips the timing and takes that candidate (modulo the
// group's candidate count) for every group, so every configuration can be
// checked for correctness.
double time_ms(cudaEvent_t e0, cudaEvent_t e1) {
  float ms = 0.f;
  KFBI_CUDA(cudaEventSynchronize(e1));
  KFBI_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  return ms;
}

void autotune(kfbi_batch* B, cudaStream_t st) {
  cudaEvent_t e0, e1;
  KFBI_CUDA(cudaEventCreate(&e0));
  KFBI_CUDA(cudaEventCreate(&e1));
  std::vector<int> all(B->n, 1), zero(B->n, 0);
  B->tuning.clear();
  const bool prof = g_prof_on;
  g_prof_on = false;  // tuning launches are not part of any profile
  build_passes(B);
  set_active(B, all, &zero, st);
  KFBI_CUDA(cudaMemsetAsync(B->d_j, 0, sizeof(int), st));
  // FFT groups
  for (size_t gi = 0; gi < B->fft_ms.size(); ++gi) {
    const int M = B->fft_ms[gi];
    kfbi_batch_tuning_t rec{};
    rec.engine = 1;
    rec.M = M;
    for (int i = 0; i < B->n; ++i) rec.instances += B->h_inst[i].fft && B->h_inst[i].M == M ? 1 : 0;
    const int cand[2] = {8, 4};
    for (int c = 0; c < 2; ++c) {
      // a complex solve needs room for both planes' rows
      if (!fft_rpb_fits(M, cand[c], 2)) continue;
      rec.param[rec.n_candidates][0] = cand[c];
      rec.us[rec.n_candidates] = 0.0;
      ++rec.n_candidates;
    }
    if (B->force >= 0) {
      rec.chosen = B->force % rec.n_candidates;
    } else {
      for (int c = 0; c < rec.n_candidates; ++c) {
        B->rpb_of_M[M] = rec.param[c][0];
        build_fft_passes(B);
        const auto& g1 = B->fg[kfbi_batch::kFftSparse1][gi];
        const auto& g2 = B->fg[kfbi_batch::kFftSolveS][gi];
        fft_group_launch(g1, kfbi_batch::kFftSparse1, st);
        fft_group_launch(g2, kfbi_batch::kFftSolveS, st);
        KFBI_CUDA(cudaEventRecord(e0, st));
        for (int r = 0; r < 3; ++r) {
          fft_group_launch(g1, kfbi_batch::kFftSparse1, st);
          fft_group_launch(g2, kfbi_batch::kFftSolveS, st);
        }
        KFBI_CUDA(cudaEventRecord(e1, st));
        rec.us[c] = 1e3 * time_ms(e0, e1) / 3.0;
      }
      rec.chosen = 0;
      for (int c = 1; c < rec.n_candidates; ++c)
        if (rec.us[c] < rec.us[rec.chosen]) rec.chosen = c;
    }
    B->rpb_of_M[M] = rec.param[rec.chosen][0];
    B->tuning.push_back(rec);
  }
  // TF32 instances
  if (B->n_tc > 0) {
    kfbi_batch_tuning_t rec{};
    rec.engine = 0;
    rec.M = 0;
    rec.instances = B->n_tc;
    for (int order = 0; order < 2; ++order)
      for (int half = 0; half < 2; ++half) {
        rec.param[rec.n_candidates][0] = order;
        rec.param[rec.n_candidates][1] = half ? B->nsm / 2 : B->nsm;
        ++rec.n_candidates;
      }
    if (B->force >= 0) {
      rec.chosen = B->force % rec.n_candidates;
    } else {
      for (int c = 0; c < rec.n_candidates; ++c) {
        B->tile_order = rec.param[c][0];
        B->cta_cap = rec.param[c][1];
        build_passes(B);
        grouped_pass(B, kfbi_batch::kSparse2, st);
        KFBI_CUDA(cudaEventRecord(e0, st));
        for (int r = 0; r < 3; ++r) {
          grouped_pass(B, kfbi_batch::kSparse2, st);
          grouped_pass(B, kfbi_batch::kSparse3, st);
        }
        KFBI_CUDA(cudaEventRecord(e1, st));
        rec.us[c] = 1e3 * time_ms(e0, e1) / 3.0;
      }
      rec.chosen = 0;
      for (int c = 1; c < rec.n_candidates; ++c)
        if (rec.us[c] < rec.us[rec.chosen]) rec.chosen = c;
    }
    B->tile_order = rec.param[rec.chosen][0];
    B->cta_cap = rec.param[rec.chosen][1];
    B->tuned_us[0] = rec.us[0];
    B->tuned_us[1] = rec.n_candidates > 1 ? rec.us[rec.n_candidates / 2] : 0.0;
    B->tuning.push_back(rec);
  }
  g_prof_on = prof;
  build_passes(B);
  // launch shapes baked into the captured iteration may have changed
  if (B->iter_graph) {
    KFBI_CUDA(cudaGraphExecDestroy(B->iter_graph));
    B->iter_graph = nullptr;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

}  // namespace

namespace kfbi {

kfbi_status batch_step(kfbi_batch* B, kfbi_state* const* states, const void* const* g_next,
                       const double* const* src_or_v, const double* src_scale,
                       kfbi_solve_info* infos, cudaStream_t st) {
  if (!B || !states || !g_next) return KFBI_ERR_ARG;
  B->err.clear();
  for (int i = 0; i < B->n; ++i) {
    if (!states[i] || states[i]->dom != B->doms[i] || !states[i]->initialised || !g_next[i]) {
      B->err = "state i must be initialised on domain i and g_next[i] given";
      return KFBI_ERR_ARG;
    }
    if (states[i]->neumann) {
      B->err = "batches step Dirichlet states only";
      return KFBI_ERR_ARG;
    }
    if (states[i]->eq == KFBI_SCHRODINGER && (!src_or_v || !src_or_v[i])) {
      B->err = "Schroedinger instances need the potential v in src_or_v[i]";
      return KFBI_ERR_ARG;
    }
  }
  kfbi_status s = guarded(nullptr, [&]() -> kfbi_status {
    B->states.assign(states, states + B->n);
    fill_instances(B, states, g_next, src_or_v, src_scale);
    if (!B->bound || !B->tuned) {
      // tune what has no choice yet: the TF32 instances once, and each FFT
      // grid size the first time it appears (choices are kept across
      // rebinds)
      bool need = !B->tuned;
      for (int i = 0; i < B->n && !need; ++i)
        need = B->h_inst[i].fft && !B->rpb_of_M.count(B->h_inst[i].M);
      if (need) {
        autotune(B, st);
        B->tuned = true;
      } else {
        build_passes(B);
      }
      B->bound = true;
    } else {
      build_passes(B);
    }
    // (re)capture when the launch shapes changed or the batch was rebound
    capture_iteration(B);
    const int n = B->n;
    // the state posts of this step count from 1 again (the previous step
    // ended with the stream synchronised, so no post is in flight)
    {
      const size_t stride = 12 * (size_t)B->cap + 16;
      for (int sl = 0; sl < 2; ++sl)
        reinterpret_cast<volatile long long*>(B->h_mbox + sl * stride + stride - 1)[0] = 0;
      KFBI_CUDA(cudaMemsetAsync(B->d_postctr, 0, sizeof(long long), st));
      B->host_posts = 0;
    }
    std::vector<int> all(n, 1);
    set_active(B, all, nullptr, st);
    KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_make_ft, inst_grid(plane_blocks(B), n), 256, 0, st, B->d_inst);
    batch_accurate(B, 0, 1, 0, st);
    KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_keep_uf, inst_grid(plane_blocks(B), n), 256, 0, st, B->d_inst);
    KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_make_b, inst_grid((B->max_nb + 255) / 256, n), 256, 0, st,
                  B->d_inst);
    // per-instance failures (non-finite, not converged) are reported in
    // infos; every instance still completes its step so the batch stays
    // consistent
    kfbi_status gs = batch_gmres(B, infos, st);
    // final grid: W phi (left by the converged residual check) + Y f-tilde,
    // else a refined application with (f-tilde, phi)
    std::vector<int> sum_set(n), full_set(n);
    bool any_sum = false, any_full = false;
    for (int i = 0; i < n; ++i) {
      sum_set[i] = B->grid_wx[i];
      full_set[i] = !B->grid_wx[i];
      any_sum |= sum_set[i] != 0;
      any_full |= full_set[i] != 0;
    }
    if (any_sum) {
      set_active(B, sum_set, nullptr, st);
      KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_add_uf, inst_grid(plane_blocks(B), n), 256, 0, st, B->d_inst);
    }
    if (any_full) {
      set_active(B, full_set, nullptr, st);
      batch_accurate(B, 1, 1, 0, st);
    }
    set_active(B, all, nullptr, st);
    KFBI_LAUNCH_P(KFBI_PROF_GRID, gk_step_update, inst_grid(plane_blocks(B), n), 256, 0, st, B->d_inst);
    KFBI_CHECK_LAUNCH();
    KFBI_CUDA(cudaStreamSynchronize(st));
    return gs;
  });
  if (s != KFBI_OK && B->err.empty()) B->err = kfbi_last_global_error();
  return s;
}

}  // namespace kfbi

extern "C" {

kfbi_status kfbi_batch_step(kfbi_batch* B, kfbi_state* const* states, const void* const* g_next,
                            const double* const* src_or_v, kfbi_solve_info* infos, void* stream) {
  return kfbi::batch_step(B, states, g_next, src_or_v, nullptr, infos, (cudaStream_t)stream);
}

kfbi_status kfbi_batch_tuning(const kfbi_batch* B, int* tile_order, double* us_natural,
                              double* us_largest_first) {
  if (!B) return KFBI_ERR_ARG;
  if (tile_order) *tile_order = B->tile_order;
  if (us_natural) *us_natural = B->tuned_us[0];
  if (us_largest_first) *us_largest_first = B->tuned_us[1];
  return KFBI_OK;
}

int kfbi_batch_tuning_count(const kfbi_batch* B) { return B ? (int)B->tuning.size() : 0; }

kfbi_status kfbi_batch_tuning_get(const kfbi_batch* B, int i, kfbi_batch_tuning_t* out) {
  if (!B || !out || i < 0 || i >= (int)B->tuning.size()) return KFBI_ERR_ARG;
  *out = B->tuning[i];
  return KFBI_OK;
}

kfbi_status kfbi_batch_force_candidate(kfbi_batch* B, int candidate) {
  if (!B || candidate < -1) return KFBI_ERR_ARG;
  B->force = candidate;
  B->tuned = false;  // the next step tunes (or applies the forced candidate) again
  B->rpb_of_M.clear();
  return KFBI_OK;
}

}  // extern "C"
