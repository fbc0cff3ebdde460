// Fast DST-I passes for KFBI_MIXED_FFT32 domains: the box solve of
// Sec. 3.4.2 (arXiv 2404.14864) with each one-dimensional sine transform
// computed by an FP32 FFT on the CUDA cores instead of a dense product.
//
// A transform pass takes every row of P planes of Mp x Mp floats and writes
// the sine transform transposed, out[p][c][r] = sum_n sin(pi (c+1) n / M)
// in[p][r][n-1], c = 0 .. M-2 (output rows c >= M-1 are never written and
// stay zero), or in place of the row (out[p][r][c]).  The box solve
// S (S R S / (lambda_a + lambda_b - kappa)) S of Sec. 3.4.2 needs three
// passes, not four: after the first pass (along x, written transposed) a
// row of the plane holds one x-frequency b and all y samples, and the
// y-transform, the division by lambda_a + lambda_b - kappa and the inverse
// y-transform all run along that row.  The middle pass therefore does
// forward DST, division and inverse DST per row (for complex kappa a warp
// holds the row of both planes) and writes transposed; a row of its output
// holds one y index and all x frequencies, so the third pass transforms
// along x and writes its rows in place: the solution comes out in the
// layout of the right-hand side (row = y, column = x).
//
// DST-I through a complex FFT of length M.  With x_n = in[r][n-1]
// (n = 1 .. M-1), let y be the odd extension of length 2M (y_0 = y_M = 0,
// y_n = x_n, y_{2M-n} = -x_n).  Its DFT is -2i times the DST, so
// DST_k = -Im(Y_k)/2.  Y comes from one complex FFT of length M of the
// packing z_m = y_{2m} + i y_{2m+1}: with Z = FFT_M(z), the even and odd
// parts are E_k = (Z_k + conj Z_{M-k})/2 and O_k = (Z_k - conj Z_{M-k})/(2i),
// and Y_k = E_k + exp(-i pi k/M) O_k.
//
// FFT_M, M = 32 N1 (four-step factorisation n = 32 n1 + n2, k = k1 + N1 k2):
// lane n2 holds z_{32 n1 + n2} for all n1 and does an N1-point DFT in
// registers (mixed radix: one radix-3 step when 3 divides N1, radix-2
// otherwise, every register index a compile-time constant); the result is
// multiplied by W_M^{n2 k1} and transposed through shared memory; lane k1
// (and k1 + 32 when N1 > 32) then does the 32-point DFT over n2 and
// untangles the DST values from Z_k and Z_{M-k} (held by lanes k1 and
// N1 - k1, exchanged by warp shuffles; for N1 > 32 through shared memory in
// natural order).  Twiddles are exact powers computed on the
// host in float64 and rounded.  Supported: M = 32 N1 with N1 in
// {2, 4, 6, 8, 12, 16, 24, 32, 48, 64}, i.e. M = 64 .. 2048 with M / 32 a
// power of two or three times one.
//
// One warp per row (and per plane of a complex solve) for N1 >= 32; for
// smaller N1 a warp carries floor(32 / N1) rows so that every lane works in
// the 32-point DFTs and the untangling.  RPB warps per block (4 or 8, chosen
// at launch).  One kernel per N1; a block of a grouped launch
// may belong to any instance of that size: a per-block map gives its
// instance descriptor.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "tc_internal.h"

namespace kfbi {
namespace ff {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

__host__ __device__ constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

__host__ __device__ constexpr int log2i(int n) { return n <= 1 ? 0 : 1 + log2i(n >> 1); }

// t[i] = a[bitrev(i)] with every index a compile-time constant.
template <int N, int I = 0>
__device__ __forceinline__ void bitrev_copy(float2 (&t)[N], const float2 (&a)[N]) {
  if constexpr (I < N) {
    constexpr int J = bitrev(I, log2i(N));
    t[I] = a[J];
    bitrev_copy<N, I + 1>(t, a);
  }
}

// Radix-2 butterflies of stage LEN (LEN / 2 apart), then the next stage.
// tw[j] = W_M^j and N * S = M, so W_LEN^j = tw[j * (N / LEN) * S].
template <int N, int S, int LEN>
__device__ __forceinline__ void r2_stages(float2 (&t)[N], const float2* tw) {
  if constexpr (LEN <= N) {
#pragma unroll
    for (int i = 0; i < N; i += LEN) {
#pragma unroll
      for (int j = 0; j < LEN / 2; ++j) {
        const float2 u = t[i + j];
        const float2 x = t[i + j + LEN / 2];
        // W^0 = 1 and W_LEN^{LEN/4} = -i need no multiplication
        const float2 v = j == 0 ? x
                         : (4 * j == LEN ? make_float2(x.y, -x.x)
                                         : cmul(x, tw[j * (N / LEN) * S]));
        t[i + j] = cadd(u, v);
        t[i + j + LEN / 2] = csub(u, v);
      }
    }
    r2_stages<N, S, LEN * 2>(t, tw);
  }
}

// In-place DFT of N register values, X_k = sum_n a_n W_N^{nk}, natural
// order in and out; W_N^j = tw[j S] (N S = M).  N = 2^a or 3 * 2^a.
template <int N, int S>
__device__ __forceinline__ void dft(float2 (&a)[N], const float2* tw) {
  if constexpr (N == 1) {
    return;
  } else if constexpr (N % 3 == 0) {
    // decimation in time by 3: three interleaved DFTs of length L, then
    // twiddles W_N^{k}, W_N^{2k} and a 3-point DFT per k
    constexpr int L = N / 3;
    float2 s0[L], s1[L], s2[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      s0[l] = a[3 * l];
      s1[l] = a[3 * l + 1];
      s2[l] = a[3 * l + 2];
    }
    dft<L, 3 * S>(s0, tw);
    dft<L, 3 * S>(s1, tw);
    dft<L, 3 * S>(s2, tw);
    constexpr float kS3 = 0.866025403784438646763723170752936183f;  // sin(pi / 3)
#pragma unroll
    for (int k = 0; k < L; ++k) {
      const float2 t0 = s0[k];
      const float2 t1 = k == 0 ? s1[k] : cmul(s1[k], tw[k * S]);
      const float2 t2 = k == 0 ? s2[k] : cmul(s2[k], tw[2 * k * S]);
      const float2 sm = cadd(t1, t2), df = csub(t1, t2);
      const float2 m = make_float2(t0.x - 0.5f * sm.x, t0.y - 0.5f * sm.y);
      // W_3 = -1/2 - i sqrt(3)/2: X_{k+L} = m - i (sqrt3/2) df, X_{k+2L} = m + i (sqrt3/2) df
      const float2 r = make_float2(kS3 * df.y, -kS3 * df.x);
      a[k] = cadd(t0, sm);
      a[k + L] = cadd(m, r);
      a[k + 2 * L] = csub(m, r);
    }
  } else {
    float2 t[N];
    bitrev_copy<N>(t, a);
    r2_stages<N, S, 2>(t, tw);
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = t[i];
  }
}

// Element y_n of the odd extension of row xr (x_n at xr[n-1]).
__device__ __forceinline__ float yodd(const float* xr, int n, int M) {
  if (n == 0 || n == M) return 0.f;
  return n < M ? xr[n - 1] : -xr[2 * M - n - 1];
}

// Rows per warp: for N1 < 32 the 32-point DFTs of one row occupy only N1
// lanes, so a warp carries R = floor(32 / N1) rows and lane L works on row
// L / N1 in the second step (every lane busy for N1 = 2, 4, 8, 16).
__host__ __device__ constexpr int rows_per_warp(int N1) { return N1 >= 32 ? 1 : 32 / N1; }

// In-place DST-I of the R rows of a warp: row rho held in buf + rho stride
// (as floats: buf[n-1] = x_n on entry, buf[c] = DST_{c+1} on exit,
// c = 0 .. M-2).  Each row buffer holds N1 x 33 float2; the lanes of the
// warp call it together.
template <int N1>
__device__ __forceinline__ void rows_dst(float2* buf, size_t stride, int lane, const float2* s_tw,
                                         const float2* s_twb, const float2* s_tw2) {
  constexpr int M = 32 * N1;
  constexpr int R = rows_per_warp(N1);
  // step 1 (each row): N1-point DFTs over n1 of z_{32 n1 + lane}, then
  // W_M^{lane k1}, written transposed into the row's buffer
#pragma unroll
  for (int rho = 0; rho < R; ++rho) {
    float2* b_ = buf + rho * stride;
    const float* xr = reinterpret_cast<const float*>(b_);
    float2 a[N1];
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const int m = 32 * q + lane;
      a[q] = make_float2(yodd(xr, 2 * m, M), yodd(xr, 2 * m + 1, M));
    }
    dft<N1, 32>(a, s_tw);
    __syncwarp();  // every lane has read its part of the row before the transpose overwrites it
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) b_[k1 * 33 + lane] = cmul(a[k1], s_twb[k1 * 32 + lane]);
  }
  __syncwarp();
  if constexpr (N1 <= 32) {
    // step 2: lane L = rho N1 + k1 does the 32-point DFT over n2 of row rho
    const int rho = lane / N1, k1 = lane - rho * N1;
    const bool act = rho < R;
    float2* b_ = buf + (act ? rho : 0) * stride;
    float* xr = reinterpret_cast<float*>(b_);
    float2 b[32];
    if (act) {
#pragma unroll
      for (int n2 = 0; n2 < 32; ++n2) b[n2] = b_[k1 * 33 + n2];
      dft<32, N1>(b, s_tw);
    } else {
#pragma unroll
      for (int n2 = 0; n2 < 32; ++n2) b[n2] = make_float2(0.f, 0.f);
    }
    __syncwarp();
    // DST_k = -Im(E_k + exp(-i pi k / M) O_k) / 2 from Z_k and Z_{M-k}: lane
    // rho N1 + k1 holds Z_{k1 + N1 k2} of its row in b[k2]; Z_{M-k} is
    // b[31 - k2] of lane rho N1 + N1 - k1 (k1 = 0: its own b[(32 - k2) % 32])
    const int partner = act ? rho * N1 + (k1 == 0 ? 0 : N1 - k1) : lane;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      float2 zc;
      zc.x = __shfl_sync(0xffffffffu, b[31 - k2].x, partner);
      zc.y = __shfl_sync(0xffffffffu, b[31 - k2].y, partner);
      if (k1 == 0) zc = b[(32 - k2) & 31];
      // straight-line body (only the store is predicated) so the unrolled
      // iterations overlap
      const int k = k1 + N1 * k2;
      const float2 zk = b[k2];
      const float ey = 0.5f * (zk.y - zc.y);
      const float ox = 0.5f * (zk.y + zc.y), oy = -0.5f * (zk.x - zc.x);
      const float2 w = s_tw2[k < M ? k : 0];
      const float v = -0.5f * (ey + w.x * oy + w.y * ox);
      if (act && k != 0) xr[k - 1] = v;
    }
  } else {
    // one row (R = 1): lane k1 and k1 + 32 do the 32-point DFTs over n2,
    // then Z in natural order through the buffer (M float2 fit in N1 x 33)
    constexpr int NQ = N1 / 32;
    float* xr = reinterpret_cast<float*>(buf);
    float2 b[NQ][32];
#pragma unroll
    for (int t = 0; t < NQ; ++t) {
      const int k1 = lane + 32 * t;
#pragma unroll
      for (int n2 = 0; n2 < 32; ++n2) b[t][n2] = buf[k1 * 33 + n2];
      dft<32, N1>(b[t], s_tw);
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < NQ; ++t) {
      const int k1 = lane + 32 * t;
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) buf[k1 + N1 * k2] = b[t][k2];
    }
    __syncwarp();
    float v[N1];
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const int k = lane + 32 * q;
      const float2 zk = buf[k];
      const float2 zc = buf[k == 0 ? 0 : M - k];
      const float ey = 0.5f * (zk.y - zc.y);
      const float ox = 0.5f * (zk.y + zc.y), oy = -0.5f * (zk.x - zc.x);
      const float2 w = s_tw2[k];
      v[q] = -0.5f * (ey + w.x * oy + w.y * ox);
    }
    __syncwarp();  // all Z read before the row overwrites them
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const int k = lane + 32 * q;
      if (k > 0) xr[k - 1] = v[q];
    }
  }
  __syncwarp();
}

constexpr size_t buf_floats(int N1) { return (size_t)N1 * 33 * 2; }

// Shared memory of one block (bytes): twiddle tables W_M^j, W_M^{n2 k1} at
// [k1][n2] and exp(-i pi k / M) (M float2 each), eigenvalues (M floats),
// and one N1 x 33 complex row buffer per row slot (rpb warps x R rows) and
// plane.
constexpr size_t smem_for(int N1, int rpb, int pw) {
  return sizeof(float) *
         ((size_t)7 * 32 * N1 + (size_t)rpb * rows_per_warp(N1) * pw * buf_floats(N1));
}

template <int N1, bool SPARSE>
__device__ __forceinline__ void body(const FftDesc& d, int lb, int rpb, float* smem) {
  constexpr int M = 32 * N1;
  constexpr int R = rows_per_warp(N1);
  const int T = 32 * rpb;
  float2* s_tw = reinterpret_cast<float2*>(smem);  // [M] W_M^j
  float2* s_twb = s_tw + M;                         // [N1][32] W_M^{n2 k1}
  float2* s_tw2 = s_twb + M;                        // [M] exp(-i pi k / M)
  float* s_lam = reinterpret_cast<float*>(s_tw2 + M);  // [M]
  float2* s_buf = reinterpret_cast<float2*>(s_lam + M);  // [rpb R slots][pw][N1 * 33]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool solve = d.solve != 0;
  const int pw = d.pw;
  const size_t bstride = (size_t)N1 * 33;  // float2 per row buffer
  // the tables are written once at domain set-up: load them before waiting
  // for the previous kernel
  {
    // four rounds of loads in flight per thread (read-only path), then the
    // stores: one round trip for the tables instead of one per round
    constexpr int CH = 4;
    for (int i0 = threadIdx.x; i0 < M; i0 += CH * T) {
      float2 a[CH], b[CH], c[CH];
      float l[CH];
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int i = i0 + q * T;
        if (i < M) {
          a[q] = __ldg(d.twM + i);
          b[q] = __ldg(d.twB + i);
          c[q] = __ldg(d.tw2M + i);
          l[q] = solve && i < d.n1 ? __ldg(d.lam + i) : 0.f;
        }
      }
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int i = i0 + q * T;
        if (i < M) {
          s_tw[i] = a[q];
          s_twb[i] = b[q];
          s_tw2[i] = c[q];
          s_lam[i] = l[q];
        }
      }
    }
  }
  KFBI_PDL_ENTRY();
  KFBI_STOP_RETURN(d.stop);
  if (d.active && *d.active == 0) return;
  // lb = (plane group) * rblocks + row block; slot s = warp R + rho holds
  // data row rr0 + s
  const int pg = lb / d.rblocks;
  const int rr0 = d.r_lo + (lb - pg * d.rblocks) * rpb * R;
  const size_t plane = (size_t)d.Mp * d.Mp;
  for (int rho = 0; rho < R; ++rho) {
    const int sl = warp * R + rho;
    const int r = rr0 + sl;  // data row within the plane
    for (int pl = 0; pl < pw; ++pl) {
      const int p = pg + pl;  // plane
      float2* buf = s_buf + (size_t)(sl * pw + pl) * bstride;
      float* xrow = reinterpret_cast<float*>(buf);
      if constexpr (SPARSE) {
        const FftSparseRhs& sp = d.sp;
        const double* phi = sp.phi + (sp.dj ? (size_t)(*sp.dj) * sp.dj_stride : 0);
#pragma unroll
        for (int q = 0; q < N1; ++q) xrow[lane + 32 * q] = 0.f;
        __syncwarp();
        const int rl = r - sp.rmin;  // row within the irregular rows
        if (rl >= 0 && rl < sp.nrows) {
          // lanes take the row's correction arms (grouped by node, nodes by
          // column), each one arm with its six density terms; a segmented
          // sum over lanes in a fixed order adds the arms of a node
          const int a0 = sp.arm_start[sp.row_start[rl]], a1 = sp.arm_start[sp.row_start[rl + 1]];
          for (int ab = a0; ab < a1; ab += 32) {
            const int a = ab + lane;
            float val = 0.f;
            int col = -1 - lane;  // distinct keys for idle lanes
            if (a < a1) {
              col = sp.arm_col[a];
              int k = sp.arm_k0[a];
              float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
#pragma unroll
              for (int m = 0; m < 6; ++m) {
                const float al = sp.alpha[m * sp.n_arms + a], be = sp.beta[m * sp.n_arms + a];
                const float pr = (float)phi[(size_t)k * sp.ps];
                ar = fmaf(al, pr, ar);
                br = fmaf(be, pr, br);
                if (sp.cplx) {
                  const float pi = (float)phi[(size_t)k * sp.ps + 1];
                  ai = fmaf(al, pi, ai);
                  bi = fmaf(be, pi, bi);
                }
                k = (k + 1 == sp.nb) ? 0 : k + 1;
              }
              float sr = ar + sp.kre * br, si = 0.f;
              if (sp.cplx) {
                sr -= sp.kim * bi;
                si = ai + sp.kre * bi + sp.kim * br;
              }
              val = p == 0 ? sr : si;
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const float t = __shfl_up_sync(0xffffffffu, val, o);
              const int kc = __shfl_up_sync(0xffffffffu, col, o);
              if (lane >= o && kc == col) val += t;
            }
            const int next = __shfl_down_sync(0xffffffffu, col, 1);
            if (a < a1 && (lane == 31 || next != col)) xrow[col] += val;
            __syncwarp();
          }
        }
      } else if (r < d.n1) {
        // the row (M floats from a 16-byte aligned start): all loads first
        const float4* src = reinterpret_cast<const float4*>(d.in + p * plane + (size_t)r * d.Mp);
        constexpr int NV = (M / 4 + 31) / 32;
        float4 x[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const int i = lane + 32 * q;
          if (i < M / 4) x[q] = src[i];
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const int i = lane + 32 * q;
          if (i < M / 4) reinterpret_cast<float4*>(xrow)[i] = x[q];
        }
      } else {
        // padding rows transform to zero
#pragma unroll
        for (int q = 0; q < N1; ++q) xrow[lane + 32 * q] = 0.f;
      }
    }
  }
  __syncthreads();  // tables (and rows) visible
  // forward transform of each plane's rows; a solve divides by
  // lambda_r + lambda_c - kappa and transforms back.  The loops are kept
  // rolled so the kernel holds one copy of the transform's code (two
  // inlined copies overflowed the instruction cache)
  const int nphase = solve ? 2 : 1;
#pragma unroll 1
  for (int ph = 0; ph < nphase; ++ph) {
#pragma unroll 1
    for (int pl = 0; pl < pw; ++pl)
      rows_dst<N1>(s_buf + (size_t)(warp * R * pw + pl) * bstride, pw * bstride, lane, s_tw, s_twb,
                   s_tw2);
    if (ph + 1 < nphase) {
      __syncwarp();
      for (int rho = 0; rho < R; ++rho) {
        const int sl = warp * R + rho;
        const int r = rr0 + sl;
        float* x0 = reinterpret_cast<float*>(s_buf + (size_t)(sl * pw) * bstride);
        const float lam_r = r < d.n1 ? s_lam[r] : 0.f;
        if (pw == 2) {
          float* x1 = reinterpret_cast<float*>(s_buf + (size_t)(sl * pw + 1) * bstride);
          for (int c = lane; c < M - 1; c += 32) {
            float zr = 0.f, zi = 0.f;
            if (r < d.n1)
              eig_div_cplx32(x0[c], x1[c], lam_r + s_lam[c] - d.kre, d.kim, d.scale, zr, zi);
            x0[c] = zr;
            x1[c] = zi;
          }
        } else {
          for (int c = lane; c < M - 1; c += 32)
            x0[c] = r < d.n1 ? x0[c] * __fdividef(d.scale, lam_r + s_lam[c] - d.kre) : 0.f;
        }
      }
      __syncwarp();
    }
  }
  if (!d.transpose) {
    // the last pass of a box solve: each warp writes its rows as they are
    // (M floats, the slot of index M - 1 zero)
    __syncwarp();
    for (int rho = 0; rho < R; ++rho) {
      const int sl = warp * R + rho;
      const int r = rr0 + sl;
      for (int pl = 0; pl < pw; ++pl) {
        float* xr = reinterpret_cast<float*>(s_buf + (size_t)(sl * pw + pl) * bstride);
        if (lane == 0) xr[M - 1] = 0.f;
        __syncwarp();
        if (r < d.n1) {
          float4* dst = reinterpret_cast<float4*>(d.out + (pg + pl) * plane + (size_t)r * d.Mp);
          for (int i = lane; i < M / 4; i += 32) dst[i] = reinterpret_cast<const float4*>(xr)[i];
        }
      }
    }
    return;
  }
  __syncthreads();
  // transposed write: for each output row c the block's rpb R rows are one
  // contiguous run of rpb R floats (float4 pieces read from four slots' rows)
  const int nq = rpb * R / 4;
  for (int pl = 0; pl < pw; ++pl) {
    float* dst = d.out + (pg + pl) * plane + rr0;
    for (int i = threadIdx.x; i < (M - 1) * nq; i += T) {
      const int c = i / nq, h = i - c * nq;
      float o[4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        o[j] = reinterpret_cast<const float*>(s_buf + (size_t)((4 * h + j) * pw + pl) * bstride)[c];
      *reinterpret_cast<float4*>(dst + (size_t)c * d.Mp + 4 * h) = make_float4(o[0], o[1], o[2], o[3]);
    }
  }
}

// One kernel per transform length (every block of a launch has the same N1;
// a grouped launch over instances of several sizes is one launch per size).
template <int N1, bool SPARSE>
__global__ void __launch_bounds__(256) k_dst_fft(const __grid_constant__ FftGroup g) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  // a private copy of the descriptor: its fields stay in registers instead
  // of being reloaded through a pointer after every shared-memory store
  FftDesc d;
  int lb = blockIdx.x;
  if (g.descs) {
    const int2 m = g.blk[blockIdx.x];
    d = g.descs[m.x];
    lb = m.y;
  } else {
    d = g.one;
  }
  body<N1, SPARSE>(d, lb, g.rpb, smem);
}

}  // namespace ff

// ---- host side --------------------------------------------------------------

bool fft_supported(int M) {
  if (M % 32 != 0) return false;
  switch (M / 32) {
    case 2: case 4: case 6: case 8: case 12: case 16: case 24: case 32: case 48: case 64:
      return true;
    default:
      return false;
  }
}

size_t fft_smem(int M, int rpb, int pw) { return ff::smem_for(M / 32, rpb, pw); }

bool fft_rpb_fits(int M, int rpb, int pw) { return fft_smem(M, rpb, pw) <= (size_t)kMaxSmemOptin; }

// Flops of one row transform as executed: one complex FFT of length M
// (5 M log2 M) and the O(M) untangling (about 10 M).
double fft_pass_flops(int M, int rows) { return (double)rows * (5.0 * M * std::log2((double)M) + 10.0 * M); }

template <int N1>
static void set_attr() {
  KFBI_CUDA(cudaFuncSetAttribute(ff::k_dst_fft<N1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kMaxSmemOptin));
  KFBI_CUDA(cudaFuncSetAttribute(ff::k_dst_fft<N1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kMaxSmemOptin));
}

template <int N1>
static void launch_n1(const FftGroup& g, bool sparse, int nblocks, size_t smem, int prof_class,
                      double flops, double bytes, cudaStream_t st) {
  void* tok = g_prof_on ? prof_begin(prof_class, st) : nullptr;
  if (sparse)
    launch_kernel(ff::k_dst_fft<N1, true>, nblocks, 32 * g.rpb, smem, st, g);
  else
    launch_kernel(ff::k_dst_fft<N1, false>, nblocks, 32 * g.rpb, smem, st, g);
  if (tok) {
    prof_end(tok, st);
    prof_add_work(tok, flops);
    prof_add_bytes(tok, bytes);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void fft_prepare_all() {
  static std::once_flag once;
  std::call_once(once, []() {
    set_attr<2>(); set_attr<4>(); set_attr<6>(); set_attr<8>(); set_attr<12>();
    set_attr<16>(); set_attr<24>(); set_attr<32>(); set_attr<48>(); set_attr<64>();
  });
}

FftDesc fft_desc(const TcDst* T, const float* in, float* out, int P, bool solve, float kre,
                 float kim, float scale, const double* stop, const FftSparseRhs* sp, int rpb) {
  FftDesc d{};
  const int M = T->n1 + 1;
  const int R = ff::rows_per_warp(M / 32);  // rows per warp: a block covers rpb R rows
  d.in = in;
  d.out = out;
  d.twM = T->twM;
  d.twB = T->twB;
  d.tw2M = T->tw2M;
  d.lam = T->lam;
  d.N1 = M / 32;
  d.Mp = T->Mp;
  d.n1 = T->n1;
  d.solve = solve ? 1 : 0;
  d.transpose = 1;
  d.pw = solve && P == 2 ? 2 : 1;
  d.kre = kre;
  d.kim = kim;
  d.scale = scale;
  d.stop = stop;
  d.active = nullptr;
  d.r_lo = 0;
  int rows = T->n1;
  if (sp) {
    d.sparse = 1;
    d.sp = *sp;
    d.r_lo = sp->rmin / (rpb * R) * (rpb * R);
    rows = sp->rmin + sp->nrows - d.r_lo;
  }
  d.rblocks = (rows + rpb * R - 1) / (rpb * R);
  d.pgroups = P / d.pw;
  return d;
}

int fft_blocks(const FftDesc& d) { return d.pgroups * d.rblocks; }

double fft_desc_bytes(const FftDesc& d, int rpb) {
  const int M = 32 * d.N1;
  const int rows =
      std::max(0, std::min(d.r_lo + d.rblocks * rpb * ff::rows_per_warp(d.N1), d.n1) - d.r_lo);
  const double per_row = 4.0 * (M - 1) * (d.sparse ? 1 : 2);  // read (unless built) + write
  return (double)rows * d.pgroups * d.pw * per_row;
}

double fft_desc_flops(const FftDesc& d, int rpb) {
  const int M = 32 * d.N1;
  return fft_pass_flops(M, fft_blocks(d) * rpb * ff::rows_per_warp(d.N1) * d.pw * (d.solve ? 2 : 1));
}

void fft_launch(const FftGroup& g, int M, bool sparse, int nblocks, size_t smem, int prof_class,
                double flops, double bytes, cudaStream_t st) {
  fft_prepare_all();
  if (nblocks <= 0) return;
  switch (M / 32) {
    case 2: launch_n1<2>(g, sparse, nblocks, smem, prof_class, flops, bytes, st); break;
    case 4: launch_n1<4>(g, sparse, nblocks, smem, prof_class, flops, bytes, st); break;
    case 6: launch_n1<6>(g, sparse, nblocks, smem, prof_class, flops, bytes, st); break;
    case 8: launch_n1<8>(g, sparse, nblocks, smem, prof_class, flops, bytes, st); break;
    case 12: launch_n1<12>(g, sparse, nblocks, smem, prof_class, flops, bytes, st); break;
    case 16: launch_n1<16>(g, sparse, nblocks, smem, prof_class, flops, bytes, st); break;
    case 24: launch_n1<24>(g, sparse, nblocks, smem, prof_class, flops, bytes, st); break;
    case 32: launch_n1<32>(g, sparse, nblocks, smem, prof_class, flops, bytes, st); break;
    case 48: launch_n1<48>(g, sparse, nblocks, smem, prof_class, flops, bytes, st); break;
    case 64: launch_n1<64>(g, sparse, nblocks, smem, prof_class, flops, bytes, st); break;
    default: throw Status{KFBI_ERR_UNSUPPORTED, "no FFT pass for this M"};
  }
}

static void launch_one(const TcDst* T, const FftDesc& d, int prof_class, cudaStream_t st, int rpb) {
  const int M = T->n1 + 1;
  FftGroup g{};
  g.descs = nullptr;
  g.blk = nullptr;
  g.one = d;
  g.rpb = rpb;
  fft_launch(g, M, d.sparse != 0, fft_blocks(d), fft_smem(M, rpb, d.pw), prof_class,
             fft_desc_flops(d, rpb), fft_desc_bytes(d, rpb), st);
}

void fft_pass(const TcDst* T, const float* in, float* out, int P, const double* stop,
              cudaStream_t st, const FftSparseRhs* sp, bool transpose, int rpb) {
  if (rpb <= 0) rpb = sp ? T->fft_rpb_sparse : T->fft_rpb;
  FftDesc d = fft_desc(T, in, out, P, false, 0.f, 0.f, 0.f, stop, sp, rpb);
  d.transpose = transpose ? 1 : 0;
  // a sparse first pass is timed with the sparse passes, not the dense DST passes
  launch_one(T, d, sp ? KFBI_PROF_SPARSE : KFBI_PROF_DST, st, rpb);
}

void fft_solve(const TcDst* T, const float* in, float* out, int P, float kre, float kim,
               float scale, const double* stop, cudaStream_t st, int rpb) {
  if (rpb <= 0) rpb = T->fft_rpb_solve;
  if (!fft_rpb_fits(T->n1 + 1, rpb, P == 2 ? 2 : 1)) rpb = 4;
  const FftDesc d = fft_desc(T, in, out, P, true, kre, kim, scale, stop, nullptr, rpb);
  launch_one(T, d, KFBI_PROF_DST, st, rpb);
}

}  // namespace kfbi
