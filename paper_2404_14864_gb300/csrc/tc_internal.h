// Shared declarations of the tensor-core DST engine (tc_dst.cu) and the
// batch engine (batch.cu).
#pragma once

#include <cuda.h>

#include "internal.h"

namespace kfbi {
namespace tc {

// Output tile of a pass: BC values of the transform index c (rows of S, the
// MMA's M) by BR values of the data index r (rows of the data planes; the
// MMA's N is 2 BR, the hi and lo halves side by side); K-blocks of BK.
constexpr int BC = 128, BR = 128, BK = 32;

// One instance's share of a (possibly grouped) pass.  Tensor maps live in
// device memory (one array per domain).
struct PassDesc {
  const CUtensorMap* a_hi;
  const CUtensorMap* a_lo;
  const CUtensorMap* b_hi;
  const CUtensorMap* b_lo;
  float* out_hi;
  float* out_lo;
  const CUtensorMap* o_hi;  // store maps of out_hi / out_lo ([P Mp rows][Mp], box 32 x 32),
  const CUtensorMap* o_lo;  // written by TMA stores; o_lo unused in mode 2
  const float* lam;
  int Mp, n1;
  int mode;  // 0: TF32 pair out, 1: eigenvalue division + pair, 2: plain fp32
  int kb0;   // first K-block; the pass covers K-blocks kb0 .. kb0 + nk - 1
  int nk;
  int ct0;   // first output column tile
  int nct;   // output column tiles
  int nrt;   // tiles along r (planes x Mp / BR)
  float kre, scale;
  const int* active;  // instance flag (nullptr: always); tiles of inactive instances are skipped
  const double* stop; // speculative GMRES iteration: all tiles skipped while *stop != 0
};

// Tiles of all instances of a grouped launch, in prefix order.  A single
// instance passes its descriptor by value (descs == nullptr).
struct GroupArgs {
  const PassDesc* descs;
  const int* prefix;  // n_inst + 1 tile offsets
  int n_inst;
  int total;
  PassDesc one;
  int* err;
  int splitk;  // 1, or 2: CTA pairs (2-CTA clusters) split each tile's K range
};

__global__ void k_tc_pass(const __grid_constant__ GroupArgs ga);
// Launch one pass (ga.splitk < 1: chosen from the tile count; CTA pairs
// when the tiles fill at most half of the SMs).  work: flops for profiling;
// max_ctas > 0 caps the persistent grid of a pass without pairs.
void launch_tc_pass(GroupArgs ga, int nsm, double work, cudaStream_t st, int max_ctas = 0);
// Tensor flops of one pass of an instance (all its tiles and K-blocks).
double pass_flops(const PassDesc& d);
extern const int kPassThreads;
extern const int kPassSmem;

}  // namespace tc

// Load maps (box 32 x 128 rows) and, for the pass outputs, store maps
// (box 32 x 32 rows: one drain warp's rows).
enum { kMapS_hi, kMapS_lo, kMapR_hi, kMapR_lo, kMapT1_hi, kMapT1_lo, kMapT2_hi, kMapT2_lo,
       kMapT1s_hi, kMapT1s_lo, kStT1_hi, kStT1_lo, kStT2_hi, kStT2_lo, kStU, kNumMaps };

struct TcDst {
  int Mp = 0, n1 = 0;
  // borrowed from the domain's shared DST tables
  float *S_hi = nullptr, *S_lo = nullptr, *lam = nullptr, *S32 = nullptr;
  // sparse route for right-hand sides supported on the irregular nodes
  float *T1sh = nullptr, *T1sl = nullptr, *rv = nullptr;
  int *row_start = nullptr, *node_col = nullptr;
  int* arm_col = nullptr;  // FFT domains: grid column of each arm's irregular node
  int rmin = 0, nrows = 0, kb0 = 0, nk2 = 0, ct0 = 0, nt3 = 0;
  CUtensorMap mT1s_hi, mT1s_lo;
  // device copies of the tensor maps, in kMap* order
  CUtensorMap* d_maps = nullptr;
  int nsm = 148;
  float *Rh = nullptr, *Rl = nullptr, *T1h = nullptr, *T1l = nullptr, *T2h = nullptr,
        *T2l = nullptr, *U = nullptr;
  int* err = nullptr;
  CUtensorMap mS_hi, mS_lo, mR_hi, mR_lo, mT1_hi, mT1_lo, mT2_hi, mT2_lo;
  CUtensorMap sT1_hi, sT1_lo, sT2_hi, sT2_lo, sU;  // store maps
  int rhs_sparse_planes = 0;
  long long bytes = 0;
  // while a GMRES cycle queues iterations ahead: the solver's convergence
  // flag, passed to the kernels of the fast (sparse-route) application
  const double* stop = nullptr;
  // KFBI_MIXED_FFT32: passes by FP32 FFT (fft_dst.cu) on single FP32 planes
  // (Rh, T1h, T2h, U; the lo planes stay unused); twiddles W_M^j,
  // W_M^{n2 k1} at [k1][n2] (n2 < 32) and exp(-i pi j / M), j < M
  bool fft = false;
  float2* twM = nullptr;
  float2* twB = nullptr;
  float2* tw2M = nullptr;
  int fft_rpb = 8;  // warps per block of this domain's plain FFT passes (4 or 8)
  int fft_rpb_sparse = 8;  // ... of its sparse first pass
  int fft_rpb_solve = 8;   // ... of its solve pass
  bool fft_tuned = false;  // the three were timed on this domain (first application)
};


// Right-hand side of a fast application for the FFT first pass: the
// irregular nodes by row (CSR from row rmin, in the order of the correction
// tables) and what the correction of each needs.
struct FftSparseRhs {
  const int* row_start;
  const int* node_col;
  const int* arm_col;  // column of each arm's node (arms grouped by node, nodes by row)
  int rmin, nrows;
  const int* arm_start;
  const int* arm_k0;
  const float* alpha;
  const float* beta;
  int n_arms, nb;
  const double* phi;
  int ps;
  float kre, kim;
  int cplx;
  // batched GMRES: the density is V[*dj], phi + (*dj) * dj_stride doubles
  const int* dj;
  long long dj_stride;
};

// Largest dynamic shared memory a block may opt into (227 KiB).
constexpr int kMaxSmemOptin = 232448;

// One instance's share of an FFT pass (fft_dst.cu).  Rows r_lo ..
// r_lo + rblocks * rpb - 1 of each plane group; rows >= n1 are zero rows.
struct FftDesc {
  const float* in;  // P planes of Mp x Mp (unused when sparse)
  float* out;       // P planes, written transposed
  const float2* twM;
  const float2* twB;
  const float2* tw2M;
  const float* lam;
  int N1, Mp, n1;
  int solve;    // 0: transform; 1: transform, divide by lambda_r + lambda_c - kappa, transform
  int pw;       // planes per warp: 2 for a solve with complex kappa, else 1
  int pgroups;  // plane groups (blocks per row block): P / pw
  int sparse;   // rows built from the corrected irregular nodes (sp)
  int transpose;  // 1: out[p][c][r] (transposed), 0: out[p][r][c] (rows in place)
  float kre, kim, scale;
  int r_lo, rblocks;
  const int* active;   // instance flag (nullptr: always)
  const double* stop;  // as KFBI_STOP_RETURN
  FftSparseRhs sp;
};

// A launch: one descriptor by value (descs == nullptr), or descriptor
// array and per-block (instance, block within instance) map.
struct FftGroup {
  const FftDesc* descs;
  const int2* blk;
  FftDesc one;
  int rpb;
};

// FP32 FFT passes (fft_dst.cu).  fft_pass transforms every row of P planes
// of `in` and writes out transposed (or, transpose false, each row in
// place); with sp the rows are built from the
// corrected irregular nodes instead of read from `in`.  fft_solve is the
// middle pass of a box solve: per row forward DST, division by
// lambda_r + lambda_c - kappa (times scale), inverse DST, written transposed.
// stop as KFBI_STOP_RETURN.
bool fft_supported(int M);
size_t fft_smem(int M, int rpb, int pw);
bool fft_rpb_fits(int M, int rpb, int pw);
double fft_pass_flops(int M, int rows);
void fft_prepare_all();
FftDesc fft_desc(const TcDst* T, const float* in, float* out, int P, bool solve, float kre,
                 float kim, float scale, const double* stop, const FftSparseRhs* sp, int rpb);
int fft_blocks(const FftDesc& d);
double fft_desc_flops(const FftDesc& d, int rpb);
double fft_desc_bytes(const FftDesc& d, int rpb);
void fft_launch(const FftGroup& g, int M, bool sparse, int nblocks, size_t smem, int prof_class,
                double flops, double bytes, cudaStream_t st);
// rpb <= 0: the domain's tuned warps per block for the pass.
void fft_pass(const TcDst* T, const float* in, float* out, int P, const double* stop,
              cudaStream_t st, const FftSparseRhs* sp = nullptr, bool transpose = true,
              int rpb = 0);
void fft_solve(const TcDst* T, const float* in, float* out, int P, float kre, float kim,
               float scale, const double* stop, cudaStream_t st, int rpb = 0);

// Device tensor map of one of the domain's pass output planes (T1, T2 pairs
// or U); throws for any other pointer.
const CUtensorMap* tc_out_map(const TcDst* T, const float* out);

}  // namespace kfbi
