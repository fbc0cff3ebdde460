// Fast DST-I passes for KFBI_MIXED_FFT32 domains: the box solve of
// Sec. 3.4.2 (arXiv 2404.14864) with each one-dimensional sine transform
// computed by an FP32 FFT on the CUDA cores instead of a dense product.
//
// One pass transforms every row of an Mp x Mp plane and writes the result
// transposed, like a dense pass: out[p][c][r] = sum_n sin(pi (c+1) n / M)
// in[p][r][n-1], c = 0 .. M-2 (rows c >= M-1 of the output are never
// written and stay zero).  Two passes give S A S.
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
// registers; the result is multiplied by W_M^{n2 k1} and transposed through
// shared memory; lane k1 then does the 32-point DFT over n2 and holds
// Z_{k1 + N1 k2}.  In-register DFTs are radix-2 with twiddles from a shared
// table of W_M^j (exact powers computed on the host in float64).
//
// One warp per row, RPB rows per block; the block stages its rows' results
// and writes the transposed output as RPB-float runs.  Pass 2 of a box solve
// (real kappa) applies the eigenvalue division as it stages.
#include <cstdint>

#include "tc_internal.h"

namespace kfbi {
namespace ff {
using kfbi::FftSparseRhs;

constexpr int RPB = 8;  // rows (warps) per block

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__host__ __device__ constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

__host__ __device__ constexpr int log2i(int n) { return n <= 1 ? 0 : 1 + log2i(n >> 1); }

// t[i] = a[bitrev(i)] with every index a compile-time constant (a loop
// would leave the permutation to the optimiser and the arrays in memory).
template <int N, int I = 0>
__device__ __forceinline__ void bitrev_copy(float2 (&t)[N], const float2 (&a)[N]) {
  if constexpr (I < N) {
    constexpr int J = bitrev(I, log2i(N));
    t[I] = a[J];
    bitrev_copy<N, I + 1>(t, a);
  }
}

// Butterflies of stage LEN (LEN / 2 apart), then the next stage; one
// template instance per stage keeps every register index a constant.
template <int N, int LEN>
__device__ __forceinline__ void dft_stages(float2 (&t)[N], const float2* tw, int stride) {
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
                                         : cmul(x, tw[j * (N / LEN) * stride]));
        t[i + j] = make_float2(u.x + v.x, u.y + v.y);
        t[i + j + LEN / 2] = make_float2(u.x - v.x, u.y - v.y);
      }
    }
    dft_stages<N, LEN * 2>(t, tw, stride);
  }
}

// In-place radix-2 decimation-in-time DFT of N values in registers;
// tw[j * stride] = exp(-2 pi i j / (N * stride)), so W_len^j is
// tw[j * (N / len) * stride].
template <int N>
__device__ __forceinline__ void dft_reg(float2 (&a)[N], const float2* tw, int stride) {
  float2 t[N];
  bitrev_copy<N>(t, a);
  dft_stages<N, 2>(t, tw, stride);
#pragma unroll
  for (int i = 0; i < N; ++i) a[i] = t[i];
}

// Element y_n of the odd extension of row xr (x_n at xr[n-1]).
__device__ __forceinline__ float yodd(const float* xr, int n, int M) {
  if (n == 0 || n == M) return 0.f;
  return n < M ? xr[n - 1] : -xr[2 * M - n - 1];
}

// Shared memory of one block (floats): twiddle tables W_M^j, W_M^{n2 k1}
// by [k1][n2], exp(-i pi k/M) (2M each), eigenvalues M, and per warp an
// N1 x 33 complex transpose buffer that first holds the warp's input row;
// once every warp has finished its transposes the buffers hold the staged
// output, (M - 1) x (RPB + 1) floats.
constexpr size_t smem_bytes(int M) {
  return sizeof(float) * ((size_t)6 * M + M + (size_t)RPB * (M / 32) * 33 * 2);
}
static_assert((1024 - 1) * (RPB + 1) <= RPB * 32 * 33 * 2, "staged output fits the transposes");

// mode 0: plain transform; mode 1: eigenvalue division of the box solve,
// out *= scale / (lam[r] + lam[c] - kre) for r < n1, 0 for padded rows r.
// SPARSE: the input plane is not read; each warp builds its row from the
// corrected values of the row's irregular nodes (the right-hand side of a
// fast application is zero elsewhere), with the arithmetic of k_correct32.
template <int N1, bool SPARSE>
__global__ void __launch_bounds__(32 * RPB) k_dst_fft(const float* __restrict__ in,
                                                      float* __restrict__ out, int Mp, int n1,
                                                      const float2* __restrict__ twM,
                                                      const float2* __restrict__ twB,
                                                      const float2* __restrict__ tw2M, int mode,
                                                      const float* __restrict__ lam, float kre,
                                                      float scale, const double* stop,
                                                      const FftSparseRhs sp, int r_lo, int bpp) {
  constexpr int M = 32 * N1;
  constexpr int T = 32 * RPB;  // threads
  extern __shared__ float4 smem4[];
  float2* s_tw = reinterpret_cast<float2*>(smem4);  // [M] W_M^j
  float2* s_twb = s_tw + M;                         // [N1][32] W_M^{n2 k1}
  float2* s_tw2 = s_twb + M;                        // [M] exp(-i pi k / M)
  float* s_lam = reinterpret_cast<float*>(s_tw2 + M);  // [M]
  float2* s_ex = reinterpret_cast<float2*>(s_lam + M);   // [RPB][N1][33]
  float* s_out = reinterpret_cast<float*>(s_ex);         // [M - 1][RPB + 1], after the transposes
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the tables are written once at domain set-up: load them before waiting
  // for the previous kernel (every load issued before any is used)
  {
    constexpr int NT = (M + T - 1) / T;
    float2 v0[NT], v1[NT], v2[NT];
    float v3[NT];
#pragma unroll
    for (int q = 0; q < NT; ++q) {
      const int i = threadIdx.x + q * T;
      if (i < M) {
        v0[q] = twM[i];
        v1[q] = twB[i];
        v2[q] = tw2M[i];
        v3[q] = mode == 1 && i < n1 ? lam[i] : 0.f;
      }
    }
#pragma unroll
    for (int q = 0; q < NT; ++q) {
      const int i = threadIdx.x + q * T;
      if (i < M) {
        s_tw[i] = v0[q];
        s_twb[i] = v1[q];
        s_tw2[i] = v2[q];
        s_lam[i] = v3[q];
      }
    }
  }
  KFBI_PDL_ENTRY();
  KFBI_STOP_RETURN(stop);
  // bpp blocks per plane cover rows r_lo .. r_lo + bpp RPB - 1 of each plane
  const int p = blockIdx.x / bpp;
  const int rr0 = r_lo + (blockIdx.x - p * bpp) * RPB;
  const int row0 = p * Mp + rr0;  // first row over all planes
  if constexpr (SPARSE) {
    float* xrow = reinterpret_cast<float*>(s_ex + (size_t)warp * N1 * 33);
#pragma unroll
    for (int q = 0; q < M / 32; ++q) xrow[lane + 32 * q] = 0.f;
    __syncwarp();
    const int rl = rr0 + warp - sp.rmin;  // row within the irregular rows
    if (rl >= 0 && rl < sp.nrows) {
      // lanes take the row's correction arms (grouped by node, nodes by
      // column), each one arm with its six density terms; a segmented sum
      // over lanes in a fixed order adds the arms of a node
      const int a0 = sp.arm_start[sp.row_start[rl]], a1 = sp.arm_start[sp.row_start[rl + 1]];
      for (int ab = a0; ab < a1; ab += 32) {
        const int a = ab + lane;
        float v = 0.f;
        int col = -1 - lane;  // distinct keys for idle lanes
        if (a < a1) {
          col = sp.arm_col[a];
          int k = sp.arm_k0[a];
          float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
#pragma unroll
          for (int m = 0; m < 6; ++m) {
            const float al = sp.alpha[m * sp.n_arms + a], be = sp.beta[m * sp.n_arms + a];
            const float pr = (float)sp.phi[(size_t)k * sp.ps];
            ar = fmaf(al, pr, ar);
            br = fmaf(be, pr, br);
            if (sp.cplx) {
              const float pi = (float)sp.phi[(size_t)k * sp.ps + 1];
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
          v = p == 0 ? sr : si;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const float t = __shfl_up_sync(0xffffffffu, v, o);
          const int kc = __shfl_up_sync(0xffffffffu, col, o);
          if (lane >= o && kc == col) v += t;
        }
        const int next = __shfl_down_sync(0xffffffffu, col, 1);
        if (a < a1 && (lane == 31 || next != col)) xrow[col] += v;
        __syncwarp();
      }
    }
  } else
  // the block's RPB input rows (M floats each) into the warps' transpose
  // buffers: all loads first, then all stores
  {
    const float* src = in + (size_t)row0 * Mp;
    constexpr int NV = RPB * (M / 4) / T;  // float4 per thread (M >= 128)
    constexpr int NVQ = NV > 0 ? NV : 1;
    float4 v[NVQ];
#pragma unroll
    for (int q = 0; q < NVQ; ++q) {
      const int i = threadIdx.x + q * T;
      if (i < RPB * (M / 4)) {
        const int rw = i / (M / 4), cq = i - rw * (M / 4);
        v[q] = *reinterpret_cast<const float4*>(src + (size_t)rw * Mp + 4 * cq);
      }
    }
#pragma unroll
    for (int q = 0; q < NVQ; ++q) {
      const int i = threadIdx.x + q * T;
      if (i < RPB * (M / 4)) {
        const int rw = i / (M / 4), cq = i - rw * (M / 4);
        *reinterpret_cast<float4*>(reinterpret_cast<float*>(s_ex + (size_t)rw * N1 * 33) + 4 * cq) = v[q];
      }
    }
  }
  __syncthreads();
  float2* ex = s_ex + (size_t)warp * N1 * 33;
  const float* xr = reinterpret_cast<const float*>(ex);
  // step 1: N1-point DFTs over n1 of z_{32 n1 + lane}, then W_M^{lane k1}
  float2 a[N1];
#pragma unroll
  for (int q = 0; q < N1; ++q) {
    const int m = 32 * q + lane;
    a[q] = make_float2(yodd(xr, 2 * m, M), yodd(xr, 2 * m + 1, M));
  }
  dft_reg<N1>(a, s_tw, 32);
  __syncwarp();  // every lane has read its part of the row before the transpose overwrites it
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) ex[k1 * 33 + lane] = cmul(a[k1], s_twb[k1 * 32 + lane]);
  __syncwarp();
  // step 3: lane k1 < N1 does the 32-point DFT over n2
  float2 b[32];
  if (lane < N1) {
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) b[n2] = ex[lane * 33 + n2];
    dft_reg<32>(b, s_tw, N1);
  } else {
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) b[n2] = make_float2(0.f, 0.f);
  }
  // every warp is done with its transpose buffer: the staged output may
  // overwrite them
  __syncthreads();
  // DST_k = -Im(E_k + exp(-i pi k / M) O_k) / 2 for k = lane + N1 k2
  // (lanes < N1 hold Z_k in b[k2]); Z_{M-k} is b[31 - k2] of lane N1 - lane,
  // or, for lane 0, its own b[(32 - k2) % 32].  Output row c = k - 1.
  const int r = rr0 + warp;  // data row within the plane
  const float lam_r = r < n1 ? s_lam[r] : 0.f;
  const int partner = lane == 0 ? 0 : N1 - lane;
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) {
    float2 zc;
    zc.x = __shfl_sync(0xffffffffu, b[31 - k2].x, partner);
    zc.y = __shfl_sync(0xffffffffu, b[31 - k2].y, partner);
    if (lane == 0) zc = b[(32 - k2) & 31];
    // straight-line body (only the store is predicated) so the unrolled
    // iterations overlap
    const int k = (lane + N1 * k2) & (M - 1);
    const float2 zk = b[k2];
    const float ey = 0.5f * (zk.y - zc.y);
    const float ox = 0.5f * (zk.y + zc.y), oy = -0.5f * (zk.x - zc.x);
    const float2 w = s_tw2[k];
    float v = -0.5f * (ey + w.x * oy + w.y * ox);
    const int c = k - 1;
    if (mode == 1) v = r < n1 ? v * __fdividef(scale, lam_r + s_lam[c < 0 ? 0 : c] - kre) : 0.f;
    if (lane < N1 && k != 0) s_out[c * (RPB + 1) + warp] = v;
  }
  __syncthreads();
  float* dst = out + (size_t)p * Mp * Mp + rr0;
  constexpr int NW = ((M - 1) * (RPB / 4) + T - 1) / T;
#pragma unroll
  for (int q = 0; q < NW; ++q) {
    const int i = threadIdx.x + q * T;
    if (i < (M - 1) * (RPB / 4)) {
      const int c = i / (RPB / 4), h = i - c * (RPB / 4);
      const float* sv = s_out + c * (RPB + 1) + 4 * h;
      *reinterpret_cast<float4*>(dst + (size_t)c * Mp + 4 * h) = make_float4(sv[0], sv[1], sv[2], sv[3]);
    }
  }
}

template <int N1>
static void set_smem_attr() {
  KFBI_CUDA(cudaFuncSetAttribute(k_dst_fft<N1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes(32 * N1)));
  KFBI_CUDA(cudaFuncSetAttribute(k_dst_fft<N1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes(32 * N1)));
}

template <int N1>
static void launch_n1(const float* in, float* out, int Mp, int n1, const float2* twM,
                      const float2* twB, const float2* tw2M, int mode, const float* lam, float kre,
                      float scale, int P, const double* stop, cudaStream_t st,
                      const FftSparseRhs* sp) {
  // a sparse first pass transforms only the rows that can hold irregular
  // nodes (whole RPB groups); the output columns of the other rows are zero
  // in its dedicated buffer and stay so
  int r_lo = 0, bpp = Mp / RPB;
  if (sp) {
    r_lo = sp->rmin / RPB * RPB;
    bpp = (sp->rmin + sp->nrows - r_lo + RPB - 1) / RPB;
  }
  const int blocks = P * bpp;
  const double fl = fft_pass_flops(32 * N1, blocks * RPB);
  if (sp)  // timed with the sparse first passes, not the dense DST passes
    KFBI_LAUNCH_PW(KFBI_PROF_SPARSE, fl, (k_dst_fft<N1, true>), blocks, 32 * RPB, smem_bytes(32 * N1),
                   st, in, out, Mp, n1, twM, twB, tw2M, mode, lam, kre, scale, stop, *sp, r_lo, bpp);
  else
    KFBI_LAUNCH_PW(KFBI_PROF_DST, fl, (k_dst_fft<N1, false>), blocks, 32 * RPB, smem_bytes(32 * N1),
                   st, in, out, Mp, n1, twM, twB, tw2M, mode, lam, kre, scale, stop, FftSparseRhs{},
                   r_lo, bpp);
}

}  // namespace ff

// Flops of one pass as executed: per row one complex FFT of length M
// (5 M log2 M) and the O(M) untangling (about 10 M).
double fft_pass_flops(int M, int rows) {
  int lg = 0;
  while ((1 << lg) < M) ++lg;
  return (double)rows * (5.0 * M * lg + 10.0 * M);
}

bool fft_supported(int M) { return M >= 64 && M <= 1024 && (M & (M - 1)) == 0; }

size_t fft_smem_bytes(int M) { return ff::smem_bytes(M); }

void fft_prepare(int M) {
  switch (M) {
    case 64: ff::set_smem_attr<2>(); break;
    case 128: ff::set_smem_attr<4>(); break;
    case 256: ff::set_smem_attr<8>(); break;
    case 512: ff::set_smem_attr<16>(); break;
    case 1024: ff::set_smem_attr<32>(); break;
    default: throw Status{KFBI_ERR_UNSUPPORTED, "FFT passes need M = 64 .. 1024, a power of two"};
  }
}

void fft_pass(const TcDst* T, const float* in, float* out, int mode, float kre, float scale, int P,
              const double* stop, cudaStream_t st, const FftSparseRhs* sp) {
  const int M = T->n1 + 1;
  switch (M) {
    case 64: ff::launch_n1<2>(in, out, T->Mp, T->n1, T->twM, T->twB, T->tw2M, mode, T->lam, kre, scale, P, stop, st, sp); break;
    case 128: ff::launch_n1<4>(in, out, T->Mp, T->n1, T->twM, T->twB, T->tw2M, mode, T->lam, kre, scale, P, stop, st, sp); break;
    case 256: ff::launch_n1<8>(in, out, T->Mp, T->n1, T->twM, T->twB, T->tw2M, mode, T->lam, kre, scale, P, stop, st, sp); break;
    case 512: ff::launch_n1<16>(in, out, T->Mp, T->n1, T->twM, T->twB, T->tw2M, mode, T->lam, kre, scale, P, stop, st, sp); break;
    case 1024: ff::launch_n1<32>(in, out, T->Mp, T->n1, T->twM, T->twB, T->tw2M, mode, T->lam, kre, scale, P, stop, st, sp); break;
    default: throw Status{KFBI_ERR_UNSUPPORTED, "FFT passes need M = 64 .. 1024, a power of two"};
  }
}

}  // namespace kfbi
