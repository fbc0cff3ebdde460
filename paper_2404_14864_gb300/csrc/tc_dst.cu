// Mixed-precision operator application: the DST-I box solve of Sec. 3.4.2
// (arXiv 2404.14864) as dense GEMMs on the sm_103a tensor cores.
//
// One pass computes out[p][c][r] = sum_k S[c][k] A[p][r][k] (S is
// symmetric; two passes give S A S).  Operands are split into TF32 pairs,
// A = A_hi + A_lo and S = S_hi + S_lo.  Each CTA owns a 128 (c) x 128 (r)
// output tile (64 CTAs per real 1024^2 pass) and runs ten warps:
//   - warp 0 lane 0 streams K-blocks of 32 fp32 (one 128-byte swizzle row)
//     of S_hi, S_lo, A_hi, A_lo into a 3-stage shared-memory ring with TMA
//     (cp.async.bulk.tensor, 128B swizzle, mbarrier completion).  A_hi and
//     A_lo land back to back, so together they are one 256-row operand;
//   - warp 1 lane 0 issues tcgen05.mma kind::tf32 with M = 128 (c), K = 8:
//     S_hi [A_hi | A_lo] with N = 256 (r of A_hi, then r of A_lo) into one
//     TMEM accumulator of 256 columns, and S_lo A_hi with N = 128 into its
//     second half, so columns j and 128 + j hold S_hi A_hi and
//     S_hi A_lo + S_lo A_hi of output column j.  The fourth product
//     S_lo A_lo (below FP32 resolution) is not formed.  Two K-blocks go
//     into one of two accumulators, which tcgen05.commit then publishes;
//     each stage is released by its own commit;
//   - warps 2-9 drain each finished accumulator with tcgen05.ld (one output
//     row c per thread, half of the r columns per warp group) into FP32
//     registers, adding the two halves.  The epilogue splits the result
//     into the next pass's TF32 pair, applies the eigenvalue division of
//     the box solve (pass 2, real kappa) or keeps plain FP32 (pass 4), and
//     writes it through shared memory: each warp group stages 32-column
//     boxes in the 128B-swizzled layout of the output's tensor map and one
//     thread stores them with TMA (cp.async.bulk.tensor, global <- shared).
//     Row-per-thread global stores touched 32 lines per instruction and
//     took longer than the whole K loop.
// N = 256 is the tensor core's full width (three N = 64 products ran it at
// about a third of its rate), and draining every second K-block halves the
// commit round trips; the accumulator sums 64 K-terms, which keeps the
// tensor core's internal FP32 rounding at the level of one group.
// Every mbarrier wait is bounded; on timeout the kernel records an error
// bit, drains its own copies and frees its TMEM.
//
// Correction and extraction run in FP32 from FP32 copies of the domain's
// tables; GMRES and the steppers stay in FP64.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "tc_internal.h"

namespace kfbi {
namespace tc {

constexpr int STAGES = 3;
constexpr int S_BYTES = BC * BK * 4;          // 16 KiB: S_hi or S_lo
constexpr int A_BYTES = BR * BK * 4;          // 16 KiB: A_hi or A_lo
constexpr int STAGE_BYTES = 2 * S_BYTES + 2 * A_BYTES;  // S_hi, S_lo, A_hi, A_lo
constexpr int RECV_BYTES = BC * (BR / 2) * 4;  // 32 KiB: half a tile from the peer CTA
constexpr int SMALL_BYTES = 512;  // descriptor copy, barriers, TMEM slot, state
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + RECV_BYTES + 1024 + SMALL_BYTES;
constexpr int NDRAIN = 8;                     // drain / epilogue warps
constexpr int THREADS = 64 + 32 * NDRAIN;     // producer, MMA, drain warps
constexpr int NW = 2 * BR;                    // MMA width: [A_hi | A_lo]
constexpr int NACC = 2;                       // TMEM accumulators in flight
constexpr int KPA = 4;                        // K-blocks per accumulator
constexpr int RH = BR / 2;                    // r columns per drain warp group
constexpr uint32_t TMEM_COLS = NACC * NW;     // 512 columns: all of TMEM
// kind::tf32, D = F32, A = B = TF32, both K-major, N = NW, M = BC
constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(BC >> 4) << 24);
}
constexpr uint32_t IDESC = idesc_tf32(NW);     // S_hi [A_hi | A_lo]
constexpr uint32_t IDESC_LO = idesc_tf32(BR);  // S_lo A_hi
constexpr long long WAIT_LIMIT = 4000000000LL;  // cycles (~2 s)

// Descriptor of tile t (and its index within its instance).  A single
// instance's descriptor is read from its shared-memory copy `one`.
__device__ __forceinline__ const PassDesc* tile_desc(const GroupArgs& ga, const PassDesc* one,
                                                     int t, int& lt) {
  if (!ga.descs) {
    lt = t;
    return one;
  }
  int lo = 0, hi = ga.n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ga.prefix[mid] <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  lt = t - ga.prefix[lo];
  return ga.descs + lo;
}

// Tiles of an inactive instance, or of a speculative iteration after
// convergence, are skipped (every role of the pass tests the same flags).
__device__ __forceinline__ bool skip_desc(const PassDesc* d) {
  return (d->active && *d->active == 0) || (d->stop && *d->stop != 0.0);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false after `limit` cycles.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// The pipeline waits of the passes: false after WAIT_LIMIT cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  return mbar_wait_for(bar, parity, WAIT_LIMIT);
}

// Wait that also acquires writes other CTAs of the cluster released to
// this barrier (remote stores followed by a remote arrive).
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > WAIT_LIMIT) return false;
  }
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

__device__ __forceinline__ void arrive_peer(uint32_t bar_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_addr)
               : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}

// Byte offset of 16-byte chunk k of row `row` in a buffer of 128-byte-
// aligned rows whose chunk index is XORed with row & 7: the 128B swizzle of
// the tensor maps, and conflict-free for a quarter warp on consecutive rows.
__device__ __forceinline__ uint32_t swz(int row, int row_bytes, int k) {
  return (uint32_t)(row * row_bytes + ((k ^ (row & 7)) << 4));
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(smem_u32(src))
      : "memory");
}

__device__ __forceinline__ void tma_store_2d_addr(const CUtensorMap* map, uint32_t src, int x,
                                                  int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(src)
      : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// The shared-memory source of every committed bulk store has been read.
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// All but the most recent committed bulk group have read their source.
__device__ __forceinline__ void bulk_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}

// Every committed bulk store is complete.
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Bulk copy of `bytes` from this CTA's shared memory to shared memory of a
// CTA of the cluster (peer addresses from mapa), completing `bytes` of
// transaction count on the peer's mbarrier.
__device__ __forceinline__ void bulk_copy_to_peer(uint32_t dst, const void* src, uint32_t bytes,
                                                  uint32_t peer_bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "r"(smem_u32(src)), "r"(bytes), "r"(peer_bar)
      : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile of 128-byte rows, 128B
// swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(const void* p) {
  uint64_t d = (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}

__device__ __forceinline__ void umma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32"
      " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15,"
      " %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31},"
      " [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
}

// TF32 value of x, rounded to nearest (ties away from zero) by the
// conversion instruction.  The split x = hi + lo only needs hi to carry at
// most 10 mantissa bits; lo = x - hi is exact in FP32 either way.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32"
      " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// One DST-I pass (see the file comment).  The tensor core accumulates KPA
// K-blocks (64 terms, both operand halves) into a TMEM accumulator; the
// drain warps add each group's partial tile into FP32 registers with
// round-to-nearest adds while the MMA fills the next of NACC accumulators.
// Accumulating the whole K range inside the tensor core lets its FP32
// rounding error grow linearly with K (measured 2.5e-5 relative at
// K = 1024); per-group draining keeps it at the level of one group.
__global__ void __launch_bounds__(THREADS, 1) k_tc_pass(const __grid_constant__ GroupArgs ga) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* tiles = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* recv = (float*)(tiles + STAGES * STAGE_BYTES);  // [BC rows][BR / 2]
  uint8_t* small = tiles + STAGES * STAGE_BYTES + RECV_BYTES;
  PassDesc* s_one = (PassDesc*)small;  // single-instance descriptor (128 bytes)
  uint64_t* full = (uint64_t*)(small + 128);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;  // accumulator b holds a finished group
  uint64_t* acce = accf + NACC;     // accumulator b has been drained
  uint64_t* done = acce + NACC;     // all MMAs retired
  uint64_t* rfull = done + 1;       // split K: the peer's half tile is in recv
  uint64_t* pfree = rfull + 1;      // split K: the peer has consumed what we sent
  uint32_t* tmem_slot = (uint32_t*)(pfree + 1);
  volatile int* s_state = (volatile int*)(tmem_slot + 1);  // [0] abort, [1] issued, [2] consumed

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  static_assert(sizeof(PassDesc) <= 128, "descriptor copy slot");
  if (threadIdx.x == 64 && !ga.descs) *s_one = ga.one;  // read as kernel parameters
  if (threadIdx.x == 0) {
    if (!ga.descs) {
      // the maps were written at domain set-up, long before any pass
      prefetch_map(ga.one.b_hi);
      prefetch_map(ga.one.b_lo);
      prefetch_map(ga.one.a_hi);
      prefetch_map(ga.one.a_lo);
      prefetch_map(ga.one.o_hi);
      if (ga.one.o_lo) prefetch_map(ga.one.o_lo);
    }
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], NDRAIN);
    }
    mbar_init(done, 1);
    mbar_init(rfull, 1);  // the receiver's expect_tx; the peer's bulk copy completes the bytes
    mbar_init(pfree, 4 * 32);
    s_state[0] = 0;
    s_state[1] = 0;
    s_state[2] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // programmatic dependent launch: the set-up above touches no global
  // memory; wait for the previous kernel here
  KFBI_PDL_ENTRY();
  // tile loop: CTA pairs (split K) walk the tiles together, rank r taking
  // K-block half r; otherwise every CTA walks its own tiles
  const int split = ga.splitk == 2 ? 2 : 1;
  const int rank = split == 2 ? (int)(blockIdx.x & 1) : 0;
  const int unit0 = blockIdx.x / split, nunits = gridDim.x / split;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer: stage ring continues across this CTA's tiles
      int g = 0;
      bool abort = false;
      for (int t = unit0; t < ga.total && !abort; t += nunits) {
        int lt;
        const PassDesc* d = tile_desc(ga, s_one, t, lt);
        if (skip_desc(d)) continue;
        const int r0 = (lt / d->nct) * BR, c0 = (d->ct0 + lt % d->nct) * BC;
        const int kh = split == 2 ? (d->nk + 1) / 2 : d->nk;
        const int kbl = rank ? kh : 0, kbh = rank ? d->nk : kh;
        for (int kb = kbl; kb < kbh; ++kb, ++g) {
          const int s = g % STAGES, n = g / STAGES;
          if (s_state[0] || !mbar_wait(&empty[s], (uint32_t)((n & 1) ^ 1))) {
            s_state[0] = 1;
            atomicOr(ga.err, 1);
            abort = true;
            break;
          }
          uint8_t* st = tiles + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          const int kx = (d->kb0 + kb) * BK;
          tma_load_2d(st, d->b_hi, &full[s], kx, c0);
          tma_load_2d(st + S_BYTES, d->b_lo, &full[s], kx, c0);
          tma_load_2d(st + 2 * S_BYTES, d->a_hi, &full[s], kx, r0);
          tma_load_2d(st + 2 * S_BYTES + A_BYTES, d->a_lo, &full[s], kx, r0);
        }
      }
      s_state[1] = g;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: KPA K-blocks per accumulator, accumulators in a ring
      int g = 0, q = 0;  // K-blocks and accumulator groups issued
      bool abort = false;
      for (int t = unit0; t < ga.total && !abort; t += nunits) {
        int lt;
        const PassDesc* d = tile_desc(ga, s_one, t, lt);
        if (skip_desc(d)) continue;
        const int kh = split == 2 ? (d->nk + 1) / 2 : d->nk;
        const int kbl = rank ? kh : 0, kbh = rank ? d->nk : kh;
        for (int kb = kbl; kb < kbh; ++kb, ++g) {
          const int s = g % STAGES, n = g / STAGES;
          const int b = q % NACC, nbuf = q / NACC;
          const bool first = ((kb - kbl) % KPA) == 0;
          const bool last = ((kb - kbl) % KPA) == KPA - 1 || kb == kbh - 1;
          if (s_state[0] || !mbar_wait(&full[s], (uint32_t)(n & 1)) ||
              (first && !mbar_wait(&acce[b], (uint32_t)((nbuf & 1) ^ 1)))) {
            s_state[0] = 1;
            atomicOr(ga.err, 2);
            abort = true;
            break;
          }
          tc_fence_after();
          uint8_t* st = tiles + s * STAGE_BYTES;
          const uint64_t sh = desc_sw128(st), sl = desc_sw128(st + S_BYTES);
          const uint64_t aa = desc_sw128(st + 2 * S_BYTES);  // [A_hi | A_lo], 256 rows
          const uint32_t td = tmem + (uint32_t)(b * NW);
#pragma unroll
          for (int k = 0; k < BK / 8; ++k) {
            const uint64_t o = (uint64_t)(2 * k);  // 8 tf32 = 32 bytes, in 16-byte units
            umma_tf32(td, sh + o, aa + o, IDESC, (first && k == 0) ? 0u : 1u);
            umma_tf32(td + BR, sl + o, aa + o, IDESC_LO, 1u);
          }
          umma_commit(&empty[s]);
          if (last) {
            umma_commit(&accf[b]);
            ++q;
          }
        }
      }
      s_state[2] = g;
      umma_commit(done);
    }
    __syncwarp();
  } else {
    // drain / epilogue warps: TMEM lane quarter (warp % 4) = 32 output rows
    // c; warps 2-5 take r columns 0..63 of the tile, warps 6-9 64..127
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    int g = 0, ex = 0, nst = 0;  // groups drained, tiles exchanged, bulk stores of this warp
    bool ok = true;
    const int row = q * 32 + lane;  // output row c within the tile
    const uint32_t peer = (uint32_t)(rank ^ 1);
    const bool elected = ((warp - 2) & 3) == 0 && lane == 0;  // arms this half's receive barrier
    // output staging: split K, two 4 KiB slots in this warp's 8 KiB of recv;
    // otherwise one 4 KiB slot per drain warp
    const int nslot = split == 2 ? 2 : 1;
    const uint32_t wslot = smem_u32(recv) + (uint32_t)(split == 2 ? q * 8192 : (warp - 2) * 4096);
    for (int t = unit0; t < ga.total && ok; t += nunits) {
      int lt;
      const PassDesc* d = tile_desc(ga, s_one, t, lt);
      if (skip_desc(d)) continue;
      const int r0 = (lt / d->nct) * BR, c0 = (d->ct0 + lt % d->nct) * BC;
      // eigenvalues of this tile's rows and columns (pass 2), loaded before
      // the accumulation so their latency is hidden behind it
      float lam_c = 0.f, lam_r0 = 0.f, lam_r1 = 0.f;
      if (d->mode == 1) {
        const int rb0 = r0 % d->Mp + half * RH;
        lam_c = d->lam[c0 + row];
        lam_r0 = d->lam[rb0 + lane];
        lam_r1 = d->lam[rb0 + 32 + lane];
      }
      float acc[RH];
#pragma unroll
      for (int j = 0; j < RH; ++j) acc[j] = 0.f;
      const int kh = split == 2 ? (d->nk + 1) / 2 : d->nk;
      const int ngroups = ((rank ? d->nk - kh : kh) + KPA - 1) / KPA;
      for (int gi = 0; gi < ngroups; ++gi, ++g) {
        const int b = g % NACC;
        // one lane waits, the warp follows its result (tcgen05.ld needs the
        // whole warp converged)
        int got = 1;
        if (lane == 0)
          got = (!s_state[0] && mbar_wait(&accf[b], (uint32_t)((g / NACC) & 1))) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) {
          ok = false;
          if (lane == 0) {
            s_state[0] = 1;
            atomicOr(ga.err, 4);
          }
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int cc = 0; cc < RH; cc += 16) {
          uint32_t rh[16], rl[16];
          const uint32_t col = (uint32_t)(b * NW + half * RH + cc);
          tmem_ld16_nowait(tmem + lane_base + col, rh);
          tmem_ld16_nowait(tmem + lane_base + col + BR, rl);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[cc + j] += __uint_as_float(rh[j]) + __uint_as_float(rl[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[b]);
      }
      if (!ok || s_state[0]) break;
      if (split == 2) {
        // rank r finishes r-half r of the tile: send the other half's
        // partial sums to the peer, receive the peer's partials of ours.
        // recv rows are 256 bytes with the chunk index swizzled by row.
        // The sending half stages its partials in stage 0 of its own ring
        // (a CTA pair owns exactly one tile, so the ring is idle once the
        // last group is drained) and one thread moves the 32 KiB to the
        // peer's recv with a bulk copy that completes on the peer's rfull.
        const uint32_t ph = (uint32_t)(ex & 1);
        ++ex;
        if (half != rank) {
          if (!mbar_wait_cluster(pfree, ph ^ 1u)) {
            s_state[0] = 1;
            atomicOr(ga.err, 16);
            ok = false;
            break;
          }
          // this warp's 32 rows: 8 KiB at the same offset here and in recv
          uint8_t* sreg = tiles + q * (RECV_BYTES / 4);
#pragma unroll
          for (int k = 0; k < RH / 4; ++k)
            st_shared_v4(smem_u32(tiles) + swz(row, RH * 4, k), acc[4 * k], acc[4 * k + 1],
                         acc[4 * k + 2], acc[4 * k + 3]);
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) {
            bulk_copy_to_peer(peer_addr(recv, peer) + (uint32_t)(q * (RECV_BYTES / 4)), sreg,
                              (uint32_t)(RECV_BYTES / 4), peer_addr(rfull, peer));
            bulk_commit();
          }
          continue;
        }
        if (elected) mbar_expect_tx(rfull, (uint32_t)RECV_BYTES);
        if (!mbar_wait_cluster(rfull, ph)) {
          s_state[0] = 1;
          atomicOr(ga.err, 32);
          ok = false;
          break;
        }
#pragma unroll
        for (int k = 0; k < RH / 4; ++k) {
          const float4 v = *reinterpret_cast<const float4*>(
              reinterpret_cast<const uint8_t*>(recv) + swz(row, RH * 4, k));
          acc[4 * k] += v.x;
          acc[4 * k + 1] += v.y;
          acc[4 * k + 2] += v.z;
          acc[4 * k + 3] += v.w;
        }
        __syncwarp();  // every lane has read its rows before the warp stages over them
      }
      // Epilogue: scale (pass 2), then per output array (hi, lo; or the
      // plain FP32 plane) and 32-column box, each warp stages its 32 rows
      // (4 KiB, 128B-swizzled) and its lane 0 stores them with TMA: box
      // (x = first r, y = p Mp + c0 + 32 q) of the output's 2-D store map
      // [P Mp rows][Mp].  Warps never wait on one another: the staging
      // slots lie in the warp's own rows of recv (split K: two slots, after
      // the peer's partials there have been read) or its own 4 KiB of it.
      const int Mp = d->Mp, mode = d->mode;
      const int p = r0 / Mp, rb = r0 - p * Mp + half * RH;  // first r of this half
      const int narr = mode == 2 ? 1 : 2;
      const int y = p * Mp + c0 + q * 32;
      const int c = c0 + row, n1 = d->n1;
      const float kre = d->kre, scale = d->scale;
#pragma unroll
      for (int bx = 0; bx < RH / 32; ++bx) {
        if (mode == 1) {
          // eigenvalue division of the box solve: lam[r] is the same for every
          // row, so each lane loads one and the warp shares them
          const int r_lane = rb + bx * 32 + lane;
          const float lam_r = bx ? lam_r1 : lam_r0;
          // padded rows and columns (index n1 and beyond) are zero
          const float cs = c < n1 ? scale : 0.f;
          const unsigned valid = __ballot_sync(0xffffffffu, r_lane < n1);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float den = __shfl_sync(0xffffffffu, lam_r, j) + lam_c - kre;
            acc[bx * 32 + j] *= ((valid >> j) & 1u) ? __fdividef(cs, den) : 0.f;
          }
        }
        for (int a = 0; a < narr; ++a) {
          const CUtensorMap* om = a ? d->o_lo : d->o_hi;
          const int slot = nslot == 2 ? (nst & 1) : 0;
          if (nst >= nslot) {
            // the slot's previous store has read it
            if (lane == 0) {
              if (nslot == 2)
                bulk_wait_read1();
              else
                bulk_wait_read();
            }
            __syncwarp();
          }
          const uint32_t sb = wslot + (uint32_t)(slot * 4096);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float x = acc[bx * 32 + 4 * k + u];
              const float h = tf32_rna(x);
              v[u] = mode == 2 ? x : (a == 0 ? h : tf32_rna(x - h));
            }
            st_shared_v4(sb + swz(lane, 128, k), v[0], v[1], v[2], v[3]);
          }
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d_addr(om, sb, rb + bx * 32, y);
            bulk_commit();
          }
          ++nst;
        }
      }
      if (split == 2) {
        // recv may take the peer's next half tile once the stores have read it
        if (lane == 0) bulk_wait_read();
        __syncwarp();
        arrive_peer(peer_addr(pfree, peer));
      }
    }
    // bulk stores and copies complete before the CTA releases its shared memory
    if (lane == 0) bulk_wait_all();
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_state[0]) {
    // drain TMA copies that were issued but never consumed
    for (int g = s_state[2]; g < s_state[1]; ++g)
      mbar_wait(&full[g % STAGES], (uint32_t)((g / STAGES) & 1));
  }
  if (warp == 1) {
    if (lane == 0) {
      if (!mbar_wait(done, 0u)) atomicOr(ga.err, 8);
    }
    __syncwarp();
    tc_fence_after();
  }
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  if (split == 2) {
    // neither CTA of a pair leaves while the other may still write to its
    // shared memory or arrive on its barriers
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
  }
}

// ---------------------------------------------------------------------------
// FP32 correction / extraction and layout kernels of the mixed path
// ---------------------------------------------------------------------------

// FP64 planes -> TF32 pairs (hi = tf32(x), lo = tf32(x - hi)).
// fp32_lo: FFT domains, whose passes read the FP32 plane hi alone: lo gets
// the FP32 remainder x - hi (the pair keeps ~48 bits of x for the
// double-float refinement residual, k_resid_u32).
// Plane kernels in quads: four consecutive elements per thread and 16-byte
// accesses (n is a multiple of 4: planes are Mp x Mp with Mp a multiple of
// 128), so each thread keeps four elements' loads in flight.
#define QUAD_LOOP(q, n)                                                           \
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < (n) / 4;     \
       q += (size_t)gridDim.x * blockDim.x)

__device__ __forceinline__ void split_one(double x, bool fp32_pair, float& h, float& l) {
  if (fp32_pair) {
    split_f64(x, h, l);
    return;
  }
  h = tf32_round((float)x);
  l = tf32_round((float)(x - (double)h));
}

__global__ void k_split64(const double* __restrict__ src, float* __restrict__ hi,
                          float* __restrict__ lo, size_t n, int fp32_lo) {
  KFBI_PDL_ENTRY();
  // FP32 plane(s) of the FFT passes (hi alone, or hi with its FP32
  // remainder), else a TF32 pair
  const bool f32 = !lo || fp32_lo;
  QUAD_LOOP(q, n) {
    const double2 a = reinterpret_cast<const double2*>(src)[2 * q];
    const double2 b = reinterpret_cast<const double2*>(src)[2 * q + 1];
    float4 h, l;
    split_one(a.x, f32, h.x, l.x);
    split_one(a.y, f32, h.y, l.y);
    split_one(b.x, f32, h.z, l.z);
    split_one(b.y, f32, h.w, l.w);
    reinterpret_cast<float4*>(hi)[q] = h;
    if (lo) reinterpret_cast<float4*>(lo)[q] = l;
  }
}

// Corrected right-hand side at the irregular nodes in FP32, written as a
// TF32 pair (same tables as k_correct, FP32 copies).
template <bool C>
__global__ void k_correct32(float* __restrict__ Rh, float* __restrict__ Rl, size_t plane,
                            const double* __restrict__ ft, const int* __restrict__ irr_off,
                            const int* __restrict__ arm_start, const int* __restrict__ arm_k0,
                            const float* __restrict__ alpha, const float* __restrict__ beta,
                            const int* __restrict__ fidx, const float* __restrict__ fcoef,
                            int n_irr, int n_arms, int nb, const double* __restrict__ phi, int ps,
                            float kre, float kim, float* __restrict__ rv, const double* stop) {
  KFBI_PDL_ENTRY();
  KFBI_STOP_RETURN(stop);
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_irr) return;
  const int off = irr_off[n];
  float sr = ft ? (float)ft[off] : 0.f;
  float si = (C && ft) ? (float)ft[plane + off] : 0.f;
  const int a1 = arm_start[n + 1];
  for (int a = arm_start[n]; a < a1; ++a) {
    int k = arm_k0[a];
    float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      const float al = alpha[m * n_arms + a], be = beta[m * n_arms + a];
      const float pr = (float)phi[(size_t)k * ps];
      ar = fmaf(al, pr, ar);
      br = fmaf(be, pr, br);
      if (C) {
        const float pi = (float)phi[(size_t)k * ps + 1];
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
    if (ft) {
      const int f0 = fidx[a], f1 = fidx[n_arms + a];
      const float c0 = fcoef[a], c1 = fcoef[n_arms + a];
      sr += c0 * (float)ft[f0] + c1 * (float)ft[f1];
      if (C) si += c0 * (float)ft[plane + f0] + c1 * (float)ft[plane + f1];
    }
  }
  if (rv) {  // compact values for the sparse first pass
    rv[n] = sr;
    if (C) rv[n_irr + n] = si;
    return;
  }
  if (!Rl) {  // single FP32 plane (FFT passes)
    Rh[off] = sr;
    if (C) Rh[plane + off] = si;
    return;
  }
  float h = tf32_round(sr);
  Rh[off] = h;
  Rl[off] = tf32_round(sr - h);
  if (C) {
    h = tf32_round(si);
    Rh[plane + off] = h;
    Rl[plane + off] = tf32_round(si - h);
  }
}

// Sparse first pass for a right-hand side supported on the irregular nodes
// only (every GMRES application): T1[p][c][r] = sum over the irregular
// nodes n of row r of v_n S[k_n][c], for the rows rmin .. rmin + nrows - 1
// that hold irregular nodes, written as a TF32 pair.  Rows outside that
// range are never written and stay zero.  32 x 32 tile per block, staged
// through shared memory so both the S reads and the transposed writes are
// coalesced.
__global__ void __launch_bounds__(256) k_sparse_p1(const float* __restrict__ rv, int n_irr,
                                                   const int* __restrict__ row_start,
                                                   const int* __restrict__ node_col, int rmin,
                                                   int nrows, const float* __restrict__ S32,
                                                   float* __restrict__ Th, float* __restrict__ Tl,
                                                   int Mp, int P, const double* stop) {
  KFBI_PDL_ENTRY();
  KFBI_STOP_RETURN(stop);
  __shared__ float tile[2][32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int rr = ty; rr < 32; rr += 8) {
    const int rl = r0 + rr;
    float a0 = 0.f, a1 = 0.f;
    if (rl < nrows) {
      const int ne = row_start[rl + 1];
      for (int n = row_start[rl]; n < ne; ++n) {
        const float sv = S32[(size_t)node_col[n] * Mp + c0 + tx];
        a0 = fmaf(rv[n], sv, a0);
        if (P == 2) a1 = fmaf(rv[n_irr + n], sv, a1);
      }
    }
    tile[0][rr][tx] = a0;
    tile[1][rr][tx] = a1;
  }
  __syncthreads();
  const size_t plane = (size_t)Mp * Mp;
  for (int cc = ty; cc < 32; cc += 8) {
    const int rl = r0 + tx;
    if (rl >= nrows) continue;
    const size_t o = (size_t)(c0 + cc) * Mp + (size_t)(rmin + rl);
    for (int p = 0; p < P; ++p) {
      const float x = tile[p][tx][cc];
      const float h = tf32_round(x);
      Th[p * plane + o] = h;
      Tl[p * plane + o] = tf32_round(x - h);
    }
  }
}

// Last pass restricted to the extraction stencil, fused with Eq. 3.36:
// U(j', i') = sum_a T3[i'][a] S[j'][a] at the six stencil points of node k
// (TY: T3 rows are y indices, U(j', i') = sum_b T3[j'][b] S[i'][b], the
// layout the FFT solve pass leaves),
// then u+ as in k_extract32.  One block of GE_WARPS warps per node: the six
// points lie in a 3 x 3 window of grid rows j and columns i, so the block
// streams three rows of T3 and three rows of S (float4, each warp a
// quarter of them) and forms all nine window sums, reduced over lanes and
// warps; the six it needs are picked from shared memory.  (Six warps per
// node with a full dot product each read twice the rows, 48 MB per
// application at 1024^2; one warp per node left too few warps in flight.)
constexpr int GE_WARPS = 4;
template <bool C, bool TY>
__global__ void __launch_bounds__(32 * GE_WARPS)
    k_gather_extract(const float* __restrict__ T3, const float* __restrict__ S32, int Mp,
                     size_t plane, const int* __restrict__ gidx, const float* __restrict__ w,
                     const float* __restrict__ A, const float* __restrict__ B, int nb,
                     const double* __restrict__ phi, int ps, float kre, float kim,
                     double* __restrict__ out, int os, const double* stop) {
  KFBI_PDL_ENTRY();
  KFBI_STOP_RETURN(stop);
  constexpr int NP = C ? 2 : 1;
  __shared__ float win[GE_WARPS][NP][3][3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x;
  int jm[6], im[6];
  int jlo = Mp, ilo = Mp;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const int off = gidx[m * nb + k];
    jm[m] = off / Mp;
    im[m] = off - jm[m] * Mp;
    jlo = min(jlo, jm[m]);
    ilo = min(ilo, im[m]);
  }
  const float4* tr[NP][3];
  const float4* srow[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    // rows past the plane are clamped; their sums are never picked
    const int ii = min(ilo + d, Mp - 1), jj = min(jlo + d, Mp - 1);
    const int tt = TY ? jj : ii, ss = TY ? ii : jj;
#pragma unroll
    for (int q = 0; q < NP; ++q)
      tr[q][d] = reinterpret_cast<const float4*>(T3 + q * plane + (size_t)tt * Mp);
    srow[d] = reinterpret_cast<const float4*>(S32 + (size_t)ss * Mp);
  }
  float acc[NP][3][3];
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int dj = 0; dj < 3; ++dj)
#pragma unroll
      for (int di = 0; di < 3; ++di) acc[q][dj][di] = 0.f;
  for (int a4 = threadIdx.x; a4 < Mp / 4; a4 += 32 * GE_WARPS) {
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
        if (lane == 0) win[warp][q][dj][di] = x;
      }
  __syncthreads();
  if (threadIdx.x != 0) return;
  float sr_ = 0.f, si = 0.f;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const float wm = w[m * nb + k];
    float ur = 0.f, ui = 0.f;
#pragma unroll
    for (int v = 0; v < GE_WARPS; ++v) {
      ur += win[v][0][jm[m] - jlo][im[m] - ilo];
      if (C) ui += win[v][NP - 1][jm[m] - jlo][im[m] - ilo];
    }
    sr_ = fmaf(wm, ur, sr_);
    if (C) si = fmaf(wm, ui, si);
  }
  float sr = sr_;
  float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
  int kk = k - 2;
  if (kk < 0) kk += nb;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float a = A[j * nb + k], b = B[j * nb + k];
    const float pr = (float)phi[(size_t)kk * ps];
    ar = fmaf(a, pr, ar);
    br = fmaf(b, pr, br);
    if (C) {
      const float pi = (float)phi[(size_t)kk * ps + 1];
      ai = fmaf(a, pi, ai);
      bi = fmaf(b, pi, bi);
    }
    kk = (kk + 1 == nb) ? 0 : kk + 1;
  }
  sr += ar + kre * br;
  if (C) {
    sr -= kim * bi;
    si += ai + kre * bi + kim * br;
  }
  out[(size_t)k * os] = (double)sr;
  if (C)
    out[(size_t)k * os + 1] = (double)si;
  else if (os == 2)
    out[(size_t)k * os + 1] = 0.0;
}

// Complex eigenvalue division on FP32 planes: z *= scale / (lam[a] + lam[b] -
// kappa) with kappa = kre + i kim, i.e. (x + i y)(d + i kim) scale /
// (d^2 + kim^2), d = lam[a] + lam[b] - kre, in FP32.  FFT route (lo null):
// z in hi, the arithmetic of the passes around it.  Tensor route: z = hi + lo
// (a TF32 pair holds 22 significant bits, which FP32 keeps), the quotient is
// split into a TF32 pair again; FP32 rounding (a few 2^-24) stays below the
// pair's resolution.  One block per row a, float4 columns; padded rows and
// columns are left as they are.
__global__ void __launch_bounds__(256) k_eig_cplx32(float* __restrict__ hi, float* __restrict__ lo,
                                                    size_t plane, int Mp, int n1,
                                                    const float* __restrict__ lam, float kre,
                                                    float kim, float scale, const double* stop) {
  KFBI_PDL_ENTRY();
  KFBI_STOP_RETURN(stop);
  for (int a = blockIdx.x; a < n1; a += gridDim.x) {
    const float la = lam[a] - kre;
    const size_t row = (size_t)a * Mp;
    float4* hr = reinterpret_cast<float4*>(hi + row);
    float4* hq = reinterpret_cast<float4*>(hi + plane + row);
    float4* lr = lo ? reinterpret_cast<float4*>(lo + row) : nullptr;
    float4* lq = lo ? reinterpret_cast<float4*>(lo + plane + row) : nullptr;
    for (int q = threadIdx.x; 4 * q < n1; q += blockDim.x) {
      const float4 lb = *reinterpret_cast<const float4*>(lam + 4 * q);
      float4 x = hr[q], y = hq[q];
      float4 xl = make_float4(0.f, 0.f, 0.f, 0.f), yl = xl;
      if (lo) {
        xl = lr[q];
        yl = lq[q];
      }
      float* xs = reinterpret_cast<float*>(&x);
      float* ys = reinterpret_cast<float*>(&y);
      float* xls = reinterpret_cast<float*>(&xl);
      float* yls = reinterpret_cast<float*>(&yl);
      const float* ls = reinterpret_cast<const float*>(&lb);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (4 * q + j >= n1) continue;
        float zr, zi;
        eig_div_cplx32(xs[j] + xls[j], ys[j] + yls[j], la + ls[j], kim, scale, zr, zi);
        if (lo) {
          xs[j] = tf32_round(zr);
          xls[j] = tf32_round(zr - xs[j]);
          ys[j] = tf32_round(zi);
          yls[j] = tf32_round(zi - ys[j]);
        } else {
          xs[j] = zr;
          ys[j] = zi;
        }
      }
      hr[q] = x;
      hq[q] = y;
      if (lo) {
        lr[q] = xl;
        lq[q] = yl;
      }
    }
  }
}

template <bool C>
__global__ void k_extract32(const float* __restrict__ U, size_t plane,
                            const double* __restrict__ ft, const int* __restrict__ gidx,
                            const float* __restrict__ w, const float* __restrict__ A,
                            const float* __restrict__ B, const int* __restrict__ fidx,
                            const float* __restrict__ fcoef, int nb,
                            const double* __restrict__ phi, int ps, float kre, float kim,
                            double* __restrict__ out, int os) {
  KFBI_PDL_ENTRY();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  float sr = 0.f, si = 0.f;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const int g = gidx[m * nb + k];
    const float wm = w[m * nb + k];
    sr = fmaf(wm, U[g], sr);
    if (C) si = fmaf(wm, U[plane + g], si);
  }
  float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
  int kk = k - 2;
  if (kk < 0) kk += nb;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float a = A[j * nb + k], b = B[j * nb + k];
    const float pr = (float)phi[(size_t)kk * ps];
    ar = fmaf(a, pr, ar);
    br = fmaf(b, pr, br);
    if (C) {
      const float pi = (float)phi[(size_t)kk * ps + 1];
      ai = fmaf(a, pi, ai);
      bi = fmaf(b, pi, bi);
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
    const float c = fcoef[k];
    sr += c * (float)ft[g];
    if (C) si += c * (float)ft[plane + g];
  }
  out[(size_t)k * os] = (double)sr;
  if (C)
    out[(size_t)k * os + 1] = (double)si;
  else if (os == 2)
    out[(size_t)k * os + 1] = 0.0;
}

__global__ void k_f32_to_f64(const float* __restrict__ src, double* __restrict__ dst, size_t n) {
  KFBI_PDL_ENTRY();
  QUAD_LOOP(q, n) {
    const float4 v = reinterpret_cast<const float4*>(src)[q];
    reinterpret_cast<double2*>(dst)[2 * q] = make_double2(f32_to_f64(v.x), f32_to_f64(v.y));
    reinterpret_cast<double2*>(dst)[2 * q + 1] = make_double2(f32_to_f64(v.z), f32_to_f64(v.w));
  }
}

// Residual of the five-point system in FP64 for the iterative refinement of
// the box solve: res = R - (D_xx + D_yy - kappa) U with U = 0 outside the
// (n1 x n1) interior, written as a TF32 pair for the correction solve.
template <bool C>
__global__ void k_resid_split(const double* __restrict__ R, const double* __restrict__ U,
                              float* __restrict__ hi, float* __restrict__ lo, int Mp, int n1,
                              double inv_h2, double kre, double kim) {
  KFBI_PDL_ENTRY();
  const size_t plane = (size_t)Mp * Mp;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < plane;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / Mp), c = (int)(idx % Mp);
    for (int p = 0; p < (C ? 2 : 1); ++p) {
      double res = 0.0;
      if (r < n1 && c < n1) {
        const double* Up = U + p * plane;
        const double u = Up[idx];
        const double e = c + 1 < n1 ? Up[idx + 1] : 0.0;
        const double w = c > 0 ? Up[idx - 1] : 0.0;
        const double n = r + 1 < n1 ? Up[idx + Mp] : 0.0;
        const double s = r > 0 ? Up[idx - Mp] : 0.0;
        double Lu = (e + w + n + s - 4.0 * u) * inv_h2 - kre * u;
        if (C) {
          // -kappa u, imaginary part of kappa couples the planes
          const double uo = U[(1 - p) * plane + idx];
          Lu += (p == 0) ? kim * uo : -kim * uo;
        }
        res = R[p * plane + idx] - Lu;
      }
      if (!lo) {  // single FP32 plane (FFT passes)
        hi[p * plane + idx] = (float)res;
        continue;
      }
      const float h = tf32_round((float)res);
      hi[p * plane + idx] = h;
      lo[p * plane + idx] = tf32_round((float)(res - (double)h));
    }
  }
}

// Error-free transformations on FP32 (Knuth's TwoSum; TwoProduct by FMA).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// The residual of the first refinement sweep on an FFT domain, from the
// FP32 solution of the first box solve: r = R - (D_xx + D_yy - kappa) u with
// u = U32 (every neighbour an FP32 number), in double-float arithmetic on
// the FP32 pipe: the five-point sum accumulated by TwoSum with its rounding
// errors kept (hi + lo, ~2^-48 of the terms), 1/h^2 and kappa as FP32 pairs
// (split on the host), the products by TwoProduct, R as the FP32 pair
// (Rh, Rl) that k_split64 wrote, and R - Lu gathered by TwoSum before the
// final rounding: r keeps ~2^-48 of |R| while it is ~1e-6 |R| itself (the
// float64 stencil of k_resid_split gives the same r to FP32 rounding, with
// float64 operations that GB300 issues at a small fraction of the FP32
// rate).  Overwrites Rh with r (each thread reads its own points first) and
// writes U64 = U32, the start of the refined grid.
//
// r = R - L u at one point in double-float arithmetic from FP32 values: u,
// its four neighbours, uo the other plane's u (complex: L couples the planes
// through +-Im kappa, sg = +1 for the real plane, -1 for the imaginary one),
// (R_hi, R_lo) the FP32 pair of R.
template <bool C>
__device__ __forceinline__ float resid_point(float u, float e, float w, float nn, float so, float uo,
                                             float sg, float R_hi, float R_lo, float ih_hi,
                                             float ih_lo, float kr_hi, float kr_lo, float ki_hi,
                                             float ki_lo) {
  // S = e + w + n + s - 4u as hi + lo
  float sh = -4.f * u, sl = 0.f, t;
  two_sum(sh, e, sh, t);
  sl += t;
  two_sum(sh, w, sh, t);
  sl += t;
  two_sum(sh, nn, sh, t);
  sl += t;
  two_sum(sh, so, sh, t);
  sl += t;
  // Lu = S / h^2 - kappa u (+- kim u_other): leading products exact
  float p1, e1, p2, e2;
  two_prod(sh, ih_hi, p1, e1);
  two_prod(kr_hi, u, p2, e2);
  float tail = e1 + fmaf(sh, ih_lo, sl * ih_hi) - e2 - kr_lo * u;
  float lu_hi, t2;
  two_sum(p1, -p2, lu_hi, t2);
  tail += t2;
  if (C) {
    float p3, e3;
    two_prod(ki_hi, uo, p3, e3);
    float t3;
    two_sum(lu_hi, sg * p3, lu_hi, t3);
    tail += t3 + sg * (e3 + ki_lo * uo);
  }
  // res = R - Lu
  float d, t4;
  two_sum(R_hi, -lu_hi, d, t4);
  return d + ((t4 + R_lo) - tail);
}

__device__ __forceinline__ float f4k(const float4& v, int k) {
  return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

// The kernel: four consecutive points of a row per thread; U64 = 0 and r = 0
// outside the n1 x n1 block.
template <bool C>
__global__ void __launch_bounds__(256) k_resid_u32(float* __restrict__ Rh,
                                                   const float* __restrict__ Rl,
                                                   const float* __restrict__ U32,
                                                   double* __restrict__ U64, int Mp, int n1,
                                                   float ih_hi, float ih_lo, float kr_hi,
                                                   float kr_lo, float ki_hi, float ki_lo) {
  KFBI_PDL_ENTRY();
  const size_t plane = (size_t)Mp * Mp;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  QUAD_LOOP(q, plane) {
    const size_t idx = 4 * q;
    const int r = (int)((unsigned)idx / (unsigned)Mp), c0 = (int)idx - r * Mp;
    const bool live = r < n1 && c0 < n1;
#pragma unroll
    for (int p = 0; p < (C ? 2 : 1); ++p) {
      const float* Up = U32 + p * plane;
      float4 res = z4, uq = z4;
      if (live) {
        uq = *reinterpret_cast<const float4*>(Up + idx);
        const float4 un = r + 1 < n1 ? *reinterpret_cast<const float4*>(Up + idx + Mp) : z4;
        const float4 us = r > 0 ? *reinterpret_cast<const float4*>(Up + idx - Mp) : z4;
        const float uw = c0 > 0 ? Up[idx - 1] : 0.f;
        const float ue = c0 + 4 < n1 ? Up[idx + 4] : 0.f;
        const float4 uo = C ? *reinterpret_cast<const float4*>(U32 + (1 - p) * plane + idx) : z4;
        const float4 rh = *reinterpret_cast<const float4*>(Rh + p * plane + idx);
        const float4 rl = *reinterpret_cast<const float4*>(Rl + p * plane + idx);
        float o[4], uu[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = c0 + k;
          const float u = c < n1 ? f4k(uq, k) : 0.f;
          const float e = c + 1 < n1 ? (k < 3 ? f4k(uq, k + 1) : ue) : 0.f;
          const float w = c > 0 ? (k > 0 ? f4k(uq, k - 1) : uw) : 0.f;
          uu[k] = u;
          o[k] = c < n1 ? resid_point<C>(u, e, w, f4k(un, k), f4k(us, k), f4k(uo, k),
                                         p == 0 ? 1.f : -1.f, f4k(rh, k), f4k(rl, k), ih_hi,
                                         ih_lo, kr_hi, kr_lo, ki_hi, ki_lo)
                        : 0.f;
        }
        res = make_float4(o[0], o[1], o[2], o[3]);
        uq = make_float4(uu[0], uu[1], uu[2], uu[3]);
      }
      reinterpret_cast<double2*>(U64 + p * plane + idx)[0] =
          make_double2(f32_to_f64(uq.x), f32_to_f64(uq.y));
      reinterpret_cast<double2*>(U64 + p * plane + idx)[1] =
          make_double2(f32_to_f64(uq.z), f32_to_f64(uq.w));
      *reinterpret_cast<float4*>(Rh + p * plane + idx) = res;
    }
  }
}

__global__ void k_add_f32(double* __restrict__ dst, const float* __restrict__ src, size_t n) {
  KFBI_PDL_ENTRY();
  QUAD_LOOP(q, n) {
    const float4 v = reinterpret_cast<const float4*>(src)[q];
    double2 a = reinterpret_cast<const double2*>(dst)[2 * q];
    double2 b = reinterpret_cast<const double2*>(dst)[2 * q + 1];
    a.x += f32_to_f64(v.x);
    a.y += f32_to_f64(v.y);
    b.x += f32_to_f64(v.z);
    b.y += f32_to_f64(v.w);
    reinterpret_cast<double2*>(dst)[2 * q] = a;
    reinterpret_cast<double2*>(dst)[2 * q + 1] = b;
  }
}

const int kPassThreads = THREADS;
const int kPassSmem = SMEM_BYTES;

}  // namespace tc

using namespace tc;

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// 2-D fp32 tensor map: inner dimension `inner` (contiguous), `rows` rows,
// box 32 x box_rows elements, 128B swizzle.
static void make_map(CUtensorMap* m, float* base, int inner, int rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn) throw Status{KFBI_ERR_CUDA, "cuTensorMapEncodeTiled is not available"};
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)inner * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Status{KFBI_ERR_CUDA, "cuTensorMapEncodeTiled failed"};
}

TcDst* tc_create(kfbi_domain* D, const Plan& P) {
  TcDst* T = new TcDst();
  try {
    T->Mp = D->Mp;
    T->n1 = D->n1;
    const size_t plane = (size_t)D->Mp * D->Mp;
    auto alloc = [&](float** p, size_t n) {
      KFBI_CUDA(cudaMalloc(p, n * sizeof(float)));
      T->bytes += (long long)(n * sizeof(float));
    };
    T->S_hi = D->tables->S_hi;  // borrowed, shared per grid
    T->S_lo = D->tables->S_lo;
    T->S32 = D->tables->S32;
    T->lam = D->tables->lam32;
    alloc(&T->T1sh, 2 * plane);
    alloc(&T->T1sl, 2 * plane);
    alloc(&T->rv, 2 * (size_t)std::max(1, D->n_irr));
    KFBI_CUDA(cudaMemset(T->T1sh, 0, 2 * plane * sizeof(float)));
    KFBI_CUDA(cudaMemset(T->T1sl, 0, 2 * plane * sizeof(float)));
    float** bufs[] = {&T->Rh, &T->Rl, &T->T1h, &T->T1l, &T->T2h, &T->T2l, &T->U};
    // zeroed once: the FFT passes write only the M - 1 data rows of their
    // output planes, and the last pass and the stencil gather contract over
    // all Mp entries of a row, so the padding rows must hold zeros (not
    // whatever an earlier allocation left in recycled memory)
    for (float** b : bufs) {
      alloc(b, 2 * plane);
      KFBI_CUDA(cudaMemset(*b, 0, 2 * plane * sizeof(float)));
    }
    T->rhs_sparse_planes = 2;
    T->err = (int*)(D->d_scal + 6);
    KFBI_CUDA(cudaMemset(T->err, 0, sizeof(int)));
    // sparse route: rows of the right-hand side that hold irregular nodes
    // (the irregular list is sorted by row), the K-blocks they span in the
    // second pass and the output column tiles the extraction stencil reads
    // in the third pass.
    const int n1 = D->n1;
    if (P.n_irr() > 0) {
      T->rmin = P.irr.front() / n1;
      const int rmax = P.irr.back() / n1;
      T->nrows = rmax - T->rmin + 1;
      std::vector<int> rs(T->nrows + 1, 0), col(P.n_irr());
      for (int n = 0; n < P.n_irr(); ++n) {
        rs[P.irr[n] / n1 - T->rmin + 1]++;
        col[n] = P.irr[n] % n1;
      }
      for (int r = 0; r < T->nrows; ++r) rs[r + 1] += rs[r];
      KFBI_CUDA(cudaMalloc(&T->row_start, rs.size() * sizeof(int)));
      KFBI_CUDA(cudaMalloc(&T->node_col, col.size() * sizeof(int)));
      T->bytes += (long long)((rs.size() + col.size()) * sizeof(int));
      KFBI_CUDA(cudaMemcpy(T->row_start, rs.data(), rs.size() * sizeof(int), cudaMemcpyHostToDevice));
      KFBI_CUDA(cudaMemcpy(T->node_col, col.data(), col.size() * sizeof(int), cudaMemcpyHostToDevice));
      if (D->desc.precision == KFBI_MIXED_FFT32) {
        std::vector<int> ac(std::max(1, P.n_arms()), 0);
        for (int a = 0; a < P.n_arms(); ++a) ac[a] = P.irr[P.arm_node[a]] % n1;
        KFBI_CUDA(cudaMalloc(&T->arm_col, ac.size() * sizeof(int)));
        T->bytes += (long long)(ac.size() * sizeof(int));
        KFBI_CUDA(cudaMemcpy(T->arm_col, ac.data(), ac.size() * sizeof(int), cudaMemcpyHostToDevice));
      }
      T->kb0 = T->rmin / BK;
      T->nk2 = rmax / BK + 1 - T->kb0;
      int imin = n1, imax = 0;
      for (int v : P.node_gidx) {
        imin = std::min(imin, v % n1);
        imax = std::max(imax, v % n1);
      }
      T->ct0 = imin / BC;
      T->nt3 = imax / BC + 1 - T->ct0;
    }
    {
      // k_gather_extract reads each node's six stencil points from a 3 x 3
      // window of grid rows and columns
      const int nb = D->nb, n1s = D->n1;
      for (int k = 0; k < nb; ++k) {
        int jlo = 1 << 30, jhi = -1, ilo = 1 << 30, ihi = -1;
        for (int m = 0; m < 6; ++m) {
          const int v = P.node_gidx[(size_t)k * 6 + m];
          const int jj = v / n1s, ii = v % n1s;
          jlo = std::min(jlo, jj);
          jhi = std::max(jhi, jj);
          ilo = std::min(ilo, ii);
          ihi = std::max(ihi, ii);
        }
        if (jhi - jlo > 2 || ihi - ilo > 2)
          throw Status{KFBI_ERR_GEOMETRY, "an extraction stencil spans more than 3 x 3 grid points"};
      }
    }
    const int Mp = D->Mp;
    make_map(&T->mS_hi, T->S_hi, Mp, Mp, BC);
    make_map(&T->mS_lo, T->S_lo, Mp, Mp, BC);
    make_map(&T->mR_hi, T->Rh, Mp, 2 * Mp, BR);
    make_map(&T->mR_lo, T->Rl, Mp, 2 * Mp, BR);
    make_map(&T->mT1_hi, T->T1h, Mp, 2 * Mp, BR);
    make_map(&T->mT1_lo, T->T1l, Mp, 2 * Mp, BR);
    make_map(&T->mT2_hi, T->T2h, Mp, 2 * Mp, BR);
    make_map(&T->mT2_lo, T->T2l, Mp, 2 * Mp, BR);
    make_map(&T->mT1s_hi, T->T1sh, Mp, 2 * Mp, BR);
    make_map(&T->mT1s_lo, T->T1sl, Mp, 2 * Mp, BR);
    make_map(&T->sT1_hi, T->T1h, Mp, 2 * Mp, 32);
    make_map(&T->sT1_lo, T->T1l, Mp, 2 * Mp, 32);
    make_map(&T->sT2_hi, T->T2h, Mp, 2 * Mp, 32);
    make_map(&T->sT2_lo, T->T2l, Mp, 2 * Mp, 32);
    make_map(&T->sU, T->U, Mp, 2 * Mp, 32);
    const CUtensorMap maps[kNumMaps] = {T->mS_hi,  T->mS_lo,  T->mR_hi,   T->mR_lo,
                                        T->mT1_hi, T->mT1_lo, T->mT2_hi,  T->mT2_lo,
                                        T->mT1s_hi, T->mT1s_lo, T->sT1_hi, T->sT1_lo,
                                        T->sT2_hi, T->sT2_lo, T->sU};
    KFBI_CUDA(cudaMalloc(&T->d_maps, sizeof(maps)));
    T->bytes += (long long)sizeof(maps);
    KFBI_CUDA(cudaMemcpy(T->d_maps, maps, sizeof(maps), cudaMemcpyHostToDevice));
    KFBI_CUDA(cudaFuncSetAttribute(k_tc_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   SMEM_BYTES));
    if (D->desc.precision == KFBI_MIXED_FFT32) {
      const int M = D->M;
      if (!fft_supported(M))
        throw Status{KFBI_ERR_UNSUPPORTED,
                     "FFT passes need M = 32 N1, N1 in {2, 4, 6, 8, 12, 16, 24, 32, 48, 64}"};
      // W_M^j and exp(-i pi j / M), j < M, in float64 then rounded
      // (the exponent n2 k1 is reduced mod M before the angle is formed)
      std::vector<float2> tw(M), twb(M), tw2(M);
      auto w = [M](long long j) {
        const double a = -2.0 * M_PI * (double)(j % M) / M;
        return make_float2((float)std::cos(a), (float)std::sin(a));
      };
      for (int j = 0; j < M; ++j) {
        tw[j] = w(j);
        const double b = -M_PI * j / M;
        tw2[j] = make_float2((float)std::cos(b), (float)std::sin(b));
      }
      for (int k1 = 0; k1 < M / 32; ++k1)
        for (int n2 = 0; n2 < 32; ++n2) twb[k1 * 32 + n2] = w((long long)n2 * k1);
      for (float2** pp : {&T->twM, &T->twB, &T->tw2M}) KFBI_CUDA(cudaMalloc(pp, M * sizeof(float2)));
      T->bytes += 3LL * M * (long long)sizeof(float2);
      KFBI_CUDA(cudaMemcpy(T->twM, tw.data(), M * sizeof(float2), cudaMemcpyHostToDevice));
      KFBI_CUDA(cudaMemcpy(T->twB, twb.data(), M * sizeof(float2), cudaMemcpyHostToDevice));
      KFBI_CUDA(cudaMemcpy(T->tw2M, tw2.data(), M * sizeof(float2), cudaMemcpyHostToDevice));
      fft_prepare_all();
      T->fft = true;
      T->fft_rpb = M >= 2048 ? 4 : 8;
    }
    KFBI_CUDA(cudaDeviceGetAttribute(&T->nsm, cudaDevAttrMultiProcessorCount, D->device));
  } catch (...) {
    tc_destroy(T);
    throw;
  }
  return T;
}

void tc_destroy(TcDst* T) {
  if (!T) return;
  float* ptrs[] = {T->T1sh, T->T1sl, T->rv, T->Rh, T->Rl, T->T1h, T->T1l, T->T2h, T->T2l, T->U};
  for (float* p : ptrs)
    if (p) cudaFree(p);
  if (T->row_start) cudaFree(T->row_start);
  if (T->node_col) cudaFree(T->node_col);
  if (T->arm_col) cudaFree(T->arm_col);
  if (T->d_maps) cudaFree(T->d_maps);
  if (T->twM) cudaFree(T->twM);
  if (T->twB) cudaFree(T->twB);
  if (T->tw2M) cudaFree(T->tw2M);
  delete T;
}

long long tc_bytes(const TcDst* T) { return T ? T->bytes : 0; }

// Device bytes tc_create takes for a plan on the padded size Mp.
long long tc_bytes_for(const Plan& P, int Mp) {
  const size_t plane = (size_t)Mp * Mp;
  size_t n = 2 * 2 * plane + 2 * (size_t)std::max(1, P.n_irr()) + 7 * 2 * plane;
  long long b = (long long)(n * sizeof(float));
  if (P.n_irr() > 0) {
    const int rows = P.irr.back() / P.n1 - P.irr.front() / P.n1 + 1;
    b += (long long)((rows + 1 + P.n_irr()) * sizeof(int));
  }
  if (P.desc.precision == KFBI_MIXED_FFT32) {
    b += 3LL * P.M * (long long)sizeof(float2);
    if (P.n_irr() > 0) b += (long long)(std::max(1, P.n_arms()) * sizeof(int));  // arm_col
  }
  return b + (long long)(kNumMaps * sizeof(CUtensorMap));
}

const CUtensorMap* tc_out_map(const TcDst* T, const float* out) {
  if (out == T->T1h) return T->d_maps + kStT1_hi;
  if (out == T->T1l) return T->d_maps + kStT1_lo;
  if (out == T->T2h) return T->d_maps + kStT2_hi;
  if (out == T->T2l) return T->d_maps + kStT2_lo;
  if (out == T->U) return T->d_maps + kStU;
  throw Status{KFBI_ERR_ARG, "pass output is not one of the domain's planes"};
}

// Descriptor of one instance's pass: A operand maps (am_hi, am_lo: kMap*
// indices), output, mode, K-block range and output column-tile range.
static PassDesc pass_desc(TcDst* T, int am_hi, int am_lo, float* oh, float* ol, int mode, int P,
                          float kre, float scale, int kb0 = 0, int nk = -1, int ct0 = 0,
                          int nct = -1) {
  PassDesc d;
  d.a_hi = T->d_maps + am_hi;
  d.a_lo = T->d_maps + am_lo;
  d.b_hi = T->d_maps + kMapS_hi;
  d.b_lo = T->d_maps + kMapS_lo;
  d.out_hi = oh;
  d.out_lo = ol;
  d.o_hi = tc_out_map(T, oh);
  d.o_lo = ol ? tc_out_map(T, ol) : nullptr;
  d.lam = T->lam;
  d.Mp = T->Mp;
  d.n1 = T->n1;
  d.mode = mode;
  d.kb0 = kb0;
  d.nk = nk < 0 ? T->Mp / BK : nk;
  d.ct0 = ct0;
  d.nct = nct < 0 ? T->Mp / BC : nct;
  d.nrt = P * T->Mp / BR;
  d.kre = kre;
  d.scale = scale;
  d.active = nullptr;
  d.stop = nullptr;
  return d;
}

// Tensor flops one pass issues: three TF32 products (hi*hi, hi*lo, lo*hi)
// of BC x BR x BK per tile and K-block.
double tc::pass_flops(const PassDesc& d) {
  return 3.0 * 2.0 * BC * BR * BK * (double)d.nrt * d.nct * d.nk;
}

void tc::launch_tc_pass(GroupArgs ga, int nsm, double work, cudaStream_t st, int max_ctas) {
  // CTA pairs only when every pair owns exactly one tile (the pair
  // exchange reuses the idle stage ring)
  if (ga.splitk < 1 || (ga.splitk == 2 && 2 * ga.total > nsm)) ga.splitk = 2 * ga.total <= nsm ? 2 : 1;
  const int pairs = ga.splitk == 2;
  // persistent CTAs without pairs: one per SM, or max_ctas (> 0) when the
  // autotuner caps them (each CTA then takes more tiles; the per-tile
  // arithmetic is the same)
  const int cap = max_ctas > 0 ? std::min(max_ctas, nsm) : nsm;
  const int grid = pairs ? 2 * std::min(ga.total, nsm / 2) : std::min(ga.total, cap);
  if (grid <= 0) return;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3(THREADS, 1, 1);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = pairs ? 2 : 1;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = pairs ? 1 : 0;
  add_pdl_attr(cfg, at);
  void* tok = g_prof_on ? prof_begin(KFBI_PROF_DST, st) : nullptr;
  KFBI_CUDA(cudaLaunchKernelEx(&cfg, k_tc_pass, ga));
  if (tok) {
    prof_end(tok, st);
    prof_add_work(tok, work);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

// One persistent launch over the tiles of a single instance.
static void launch_pass(TcDst* T, const PassDesc& d, cudaStream_t st) {
  GroupArgs ga;
  ga.descs = nullptr;
  ga.prefix = nullptr;
  ga.n_inst = 1;
  ga.total = d.nct * d.nrt;
  ga.one = d;
  ga.err = T->err;
  ga.splitk = 0;
  tc::launch_tc_pass(ga, T->nsm, tc::pass_flops(d), st);
}

// Four TF32x3 passes: (Rh, Rl) -> U (fp32 planes), eigenvalue division after
// the forward transform.
static void fft_tune(kfbi_domain* D, cudaStream_t st);

static void tc_box_solve(kfbi_domain* D, double kre, double kim, int P, cudaStream_t st) {
  TcDst* T = D->tc;
  const size_t plane = (size_t)T->Mp * T->Mp;
  const bool C = kim != 0.0;
  const float scale = (float)((2.0 / D->M) * (2.0 / D->M));
  if (T->fft) {
    // transform along x (written transposed); along y: transform, divide
    // by the eigenvalues, transform back (one pass); transform along x
    fft_tune(D, st);
    fft_pass(T, T->Rh, T->T1h, P, nullptr, st);
    fft_solve(T, T->T1h, T->T2h, P, (float)kre, (float)kim, scale, nullptr, st);
    fft_pass(T, T->T2h, T->U, P, nullptr, st, nullptr, false);
    return;
  }
  launch_pass(T, pass_desc(T, kMapR_hi, kMapR_lo, T->T1h, T->T1l, 0, P, 0.f, 0.f), st);
  launch_pass(T, pass_desc(T, kMapT1_hi, kMapT1_lo, T->T2h, T->T2l, C ? 0 : 1, P, (float)kre, scale),
              st);
  if (C)
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_eig_cplx32, T->n1, 256, 0, st, T->T2h, T->T2l, plane, T->Mp,
                  T->n1, T->lam, (float)kre, (float)kim, scale, (const double*)nullptr);
  launch_pass(T, pass_desc(T, kMapT2_hi, kMapT2_lo, T->T1h, T->T1l, 0, P, 0.f, 0.f), st);
  launch_pass(T, pass_desc(T, kMapT1_hi, kMapT1_lo, T->U, nullptr, 2, P, 0.f, 0.f), st);
}

// GMRES application (no volume source, only u+ wanted): the right-hand
// side lives on the irregular nodes and only the extraction stencil of the
// grid solution is read, so the first pass is a sparse product on the CUDA
// cores, the second pass runs over the K-blocks of the irregular rows only,
// the third computes only the rows the stencil needs, and the last pass is a
// gather fused with the extraction.  Same discrete operator as the dense
// route; only zero terms and unread outputs are skipped.
// FP32 correction and extraction tables of the operator in use: phi -> u+
// (Dirichlet) or, while a Neumann entry point runs, psi -> d_n u+ with zero
// kappa weights.
struct Tab32 {
  const float *al, *be, *w, *a, *b, *fc;
};
static Tab32 tables32(const kfbi_domain* D) {
  if (D->neumann)
    return {D->d_arm_delta32, D->d_zero_arm32, D->d_node_wn32, D->d_node_e32, D->d_zero_node32,
            D->d_node_fcoef_n32};
  return {D->d_arm_alpha32, D->d_arm_beta32, D->d_node_w32, D->d_node_a32, D->d_node_b32,
          D->d_node_fcoef32};
}

// Right-hand side of an FFT first pass built from the irregular nodes.
static FftSparseRhs fft_sparse_rhs(const kfbi_domain* D, const Tab32& tb, const double* phi, int ps,
                                   double kre, double kim) {
  const TcDst* T = D->tc;
  FftSparseRhs sp;
  sp.row_start = T->row_start;
  sp.node_col = T->node_col;
  sp.arm_col = T->arm_col;
  sp.rmin = T->rmin;
  sp.nrows = T->nrows;
  sp.arm_start = D->d_arm_start;
  sp.arm_k0 = D->d_arm_k0;
  sp.alpha = tb.al;
  sp.beta = tb.be;
  sp.n_arms = D->n_arms;
  sp.nb = D->nb;
  sp.phi = phi;
  sp.ps = ps;
  sp.kre = (float)kre;
  sp.kim = (float)kim;
  sp.cplx = kim != 0.0 ? 1 : 0;
  sp.dj = nullptr;
  sp.dj_stride = 0;
  return sp;
}

// First FFT application of a single domain: each pass kind (sparse first
// pass, solve pass, plain pass) is timed with 8 and 4 warps per block on
// this domain's own work planes (CUDA events, one warm-up, three timed
// repetitions) and the faster is kept.  The results do not depend on the
// choice, only the launch shape does; batches tune their own groups.
static void fft_tune(kfbi_domain* D, cudaStream_t st) {
  TcDst* T = D->tc;
  if (T->fft_tuned) return;
  T->fft_tuned = true;
  const bool prof = g_prof_on;
  g_prof_on = false;
  cudaEvent_t e0, e1;
  KFBI_CUDA(cudaEventCreate(&e0));
  KFBI_CUDA(cudaEventCreate(&e1));
  const FftSparseRhs sp = fft_sparse_rhs(D, tables32(D), D->d_zero_nb, 2, 1.0, 0.0);
  const float scale = (float)((2.0 / D->M) * (2.0 / D->M));
  auto timed = [&](auto&& launch) {
    launch();
    KFBI_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < 3; ++r) launch();
    KFBI_CUDA(cudaEventRecord(e1, st));
    KFBI_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    KFBI_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms;
  };
  float best[3] = {1e30f, 1e30f, 1e30f};
  for (int c : {8, 4}) {
    const float t0 = timed([&]() { fft_pass(T, nullptr, T->T1sh, 1, nullptr, st, &sp, true, c); });
    const float t1 = timed([&]() { fft_solve(T, T->T1sh, T->U, 1, 1.f, 0.f, scale, nullptr, st, c); });
    const float t2 = timed([&]() { fft_pass(T, T->Rh, T->T1h, 1, nullptr, st, nullptr, true, c); });
    if (t0 < best[0]) { best[0] = t0; T->fft_rpb_sparse = c; }
    if (t1 < best[1]) { best[1] = t1; T->fft_rpb_solve = c; }
    if (t2 < best[2]) { best[2] = t2; T->fft_rpb = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g_prof_on = prof;
}

static void tc_apply_sparse(kfbi_domain* D, double kre, double kim, const double* phi, int ps,
                            double* out, int os, cudaStream_t st) {
  TcDst* T = D->tc;
  const Tab32 tb = tables32(D);
  const bool C = kim != 0.0;
  const int P = C ? 2 : 1;
  const int Mp = T->Mp;
  const size_t plane = (size_t)Mp * Mp;
  if (T->fft) {
    // FFT passes cost the same for any right-hand side: the first pass
    // builds its rows from the corrected irregular nodes (no plane is read),
    // then the solve pass and the last pass at the stencil points only
    fft_tune(D, st);
    const FftSparseRhs sp = fft_sparse_rhs(D, tb, phi, ps, kre, kim);
    const float scale = (float)((2.0 / D->M) * (2.0 / D->M));
    // the first pass writes only the columns of the irregular rows; T1sh
    // (zeroed at creation, written by nothing else on an FFT domain) keeps
    // zeros in the others
    fft_pass(T, nullptr, T->T1sh, P, T->stop, st, &sp);
    fft_solve(T, T->T1sh, T->U, P, (float)kre, (float)kim, scale, T->stop, st);
    if (C)
      KFBI_LAUNCH_P(KFBI_PROF_EXTRACT, (k_gather_extract<true, true>), D->nb, 32 * GE_WARPS, 0, st, T->U, T->S32, Mp,
                    plane, D->d_node_gidx, tb.w, tb.a, tb.b, D->nb, phi,
                    ps, (float)kre, (float)kim, out, os, T->stop);
    else
      KFBI_LAUNCH_P(KFBI_PROF_EXTRACT, (k_gather_extract<false, true>), D->nb, 32 * GE_WARPS, 0, st, T->U, T->S32, Mp,
                    plane, D->d_node_gidx, tb.w, tb.a, tb.b, D->nb, phi,
                    ps, (float)kre, (float)kim, out, os, T->stop);
    KFBI_CHECK_LAUNCH();
    return;
  }
  if (C)
    KFBI_LAUNCH_P(KFBI_PROF_CORRECT, k_correct32<true>, (D->n_irr + 127) / 128, 128, 0, st, T->Rh,
                  T->Rl, plane, nullptr, D->d_irr_off, D->d_arm_start, D->d_arm_k0,
                  tb.al, tb.be, D->d_arm_fidx, D->d_arm_fcoef32, D->n_irr,
                  D->n_arms, D->nb, phi, ps, (float)kre, (float)kim, T->rv, T->stop);
  else
    KFBI_LAUNCH_P(KFBI_PROF_CORRECT, k_correct32<false>, (D->n_irr + 127) / 128, 128, 0, st, T->Rh,
                  T->Rl, plane, nullptr, D->d_irr_off, D->d_arm_start, D->d_arm_k0,
                  tb.al, tb.be, D->d_arm_fidx, D->d_arm_fcoef32, D->n_irr,
                  D->n_arms, D->nb, phi, ps, (float)kre, (float)kim, T->rv, T->stop);
  KFBI_LAUNCH_P(KFBI_PROF_SPARSE, k_sparse_p1, dim3(Mp / 32, (T->nrows + 31) / 32), dim3(32, 8), 0, st,
                T->rv, D->n_irr, T->row_start, T->node_col, T->rmin, T->nrows, T->S32, T->T1sh,
                T->T1sl, Mp, P, T->stop);
  const float scale = (float)((2.0 / D->M) * (2.0 / D->M));
  PassDesc d2 = pass_desc(T, kMapT1s_hi, kMapT1s_lo, T->T2h, T->T2l, C ? 0 : 1, P, (float)kre,
                          scale, T->kb0, T->nk2);
  d2.stop = T->stop;
  launch_pass(T, d2, st);
  if (C)
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_eig_cplx32, T->n1, 256, 0, st, T->T2h, T->T2l, plane, Mp,
                  T->n1, T->lam, (float)kre, (float)kim, scale, T->stop);
  PassDesc d3 = pass_desc(T, kMapT2_hi, kMapT2_lo, T->U, nullptr, 2, P, 0.f, 0.f, 0, -1, T->ct0,
                          T->nt3);
  d3.stop = T->stop;
  launch_pass(T, d3, st);
  if (C)
    KFBI_LAUNCH_P(KFBI_PROF_EXTRACT, (k_gather_extract<true, false>), D->nb, 32 * GE_WARPS, 0, st, T->U, T->S32, Mp,
                  plane, D->d_node_gidx, tb.w, tb.a, tb.b, D->nb, phi,
                  ps, (float)kre, (float)kim, out, os, T->stop);
  else
    KFBI_LAUNCH_P(KFBI_PROF_EXTRACT, (k_gather_extract<false, false>), D->nb, 32 * GE_WARPS, 0, st, T->U, T->S32, Mp,
                  plane, D->d_node_gidx, tb.w, tb.a, tb.b, D->nb, phi,
                  ps, (float)kre, (float)kim, out, os, T->stop);
  KFBI_CHECK_LAUNCH();
}

void tc_apply(kfbi_domain* D, double kre, double kim, const double* phi, int ps, const double* ft,
              double* out, int os, bool want_grid, cudaStream_t st) {
  TcDst* T = D->tc;
  const Tab32 tb = tables32(D);
  if (!ft && !want_grid && out && D->n_irr > 0) {
    tc_apply_sparse(D, kre, kim, phi, ps, out, os, st);
    return;
  }
  const bool C = kim != 0.0;
  const int P = C ? 2 : 1;
  const int Mp = T->Mp;
  const size_t plane = (size_t)Mp * Mp;
  if (ft) {
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_split64, grid_for(P * plane / 4, 256), 256, 0, st, ft, T->Rh,
                  T->fft ? nullptr : T->Rl, P * plane, 0);
    T->rhs_sparse_planes = 0;
  } else if (T->rhs_sparse_planes < P) {
    KFBI_CUDA(cudaMemsetAsync(T->Rh, 0, 2 * plane * sizeof(float), st));
    KFBI_CUDA(cudaMemsetAsync(T->Rl, 0, 2 * plane * sizeof(float), st));
    T->rhs_sparse_planes = 2;
  }
  if (D->n_irr > 0) {
    if (C)
      KFBI_LAUNCH_P(KFBI_PROF_CORRECT, k_correct32<true>, (D->n_irr + 127) / 128, 128, 0, st,
                    T->Rh, T->fft ? nullptr : T->Rl, plane, ft, D->d_irr_off, D->d_arm_start, D->d_arm_k0,
                    tb.al, tb.be, D->d_arm_fidx, D->d_arm_fcoef32,
                    D->n_irr, D->n_arms, D->nb, phi, ps, (float)kre, (float)kim, nullptr, nullptr);
    else
      KFBI_LAUNCH_P(KFBI_PROF_CORRECT, k_correct32<false>, (D->n_irr + 127) / 128, 128, 0, st,
                    T->Rh, T->fft ? nullptr : T->Rl, plane, ft, D->d_irr_off, D->d_arm_start, D->d_arm_k0,
                    tb.al, tb.be, D->d_arm_fidx, D->d_arm_fcoef32,
                    D->n_irr, D->n_arms, D->nb, phi, ps, (float)kre, (float)kim, nullptr, nullptr);
  }
  tc_box_solve(D, kre, kim, P, st);
  if (out) {
    if (C)
      KFBI_LAUNCH_P(KFBI_PROF_EXTRACT, k_extract32<true>, (D->nb + 127) / 128, 128, 0, st, T->U,
                    plane, ft, D->d_node_gidx, tb.w, tb.a, tb.b,
                    D->d_node_fidx, tb.fc, D->nb, phi, ps, (float)kre, (float)kim,
                    out, os);
    else
      KFBI_LAUNCH_P(KFBI_PROF_EXTRACT, k_extract32<false>, (D->nb + 127) / 128, 128, 0, st, T->U,
                    plane, ft, D->d_node_gidx, tb.w, tb.a, tb.b,
                    D->d_node_fidx, tb.fc, D->nb, phi, ps, (float)kre, (float)kim,
                    out, os);
  }
  if (want_grid)
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_f32_to_f64, grid_for(P * plane / 4, 256), 256, 0, st, T->U,
                  D->d_U, P * plane);
  KFBI_CHECK_LAUNCH();
}

// Accurate application for the refinement residuals of the steppers: the
// corrected right-hand side in FP64, one TF32x3 box solve, the FP64
// five-point residual, a second box solve for the correction (the solve
// error drops from ~delta to ~delta^2, delta ~ 2e-6), and the FP64
// extraction.  The grid solution is left in D->d_U (FP64 planes).
void tc_apply_accurate(kfbi_domain* D, double kre, double kim, const double* phi, int ps,
                       const double* ft, double* out, int os, cudaStream_t st) {
  TcDst* T = D->tc;
  const bool C = kim != 0.0;
  const int P = C ? 2 : 1;
  const int Mp = T->Mp;
  const size_t plane = (size_t)Mp * Mp;
  correct_fp64(D, kre, kim, phi, ps, ft, st);  // D->d_R: FP64 corrected RHS
  // FFT domains keep the FP32 remainder of R in the (otherwise unused) lo
  // planes for the double-float residual
  KFBI_LAUNCH_P(KFBI_PROF_GRID, k_split64, grid_for(P * plane / 4, 256), 256, 0, st, D->d_R, T->Rh, T->Rl,
                P * plane, T->fft ? 1 : 0);
  T->rhs_sparse_planes = 0;
  tc_box_solve(D, kre, kim, P, st);
  if (!T->fft)
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_f32_to_f64, grid_for(P * plane / 4, 256), 256, 0, st, T->U, D->d_U,
                  P * plane);
  const double inv_h2 = 1.0 / (D->h * D->h);
  // one refinement sweep leaves a relative grid error ~delta^2; the normal
  // derivative of the Neumann operator amplifies grid errors by O(1/h), so
  // its applications take a second sweep.  The first sweep's residual is
  // formed from the FP32 solution in double-float arithmetic (and starts
  // the FP64 grid); a second sweep's grid is no longer FP32, so its
  // residual is the float64 stencil
  const int sweeps = D->neumann ? 2 : 1;
  const float ih_hi = (float)inv_h2, ih_lo = (float)(inv_h2 - (double)ih_hi);
  const float kr_hi = (float)kre, kr_lo = (float)(kre - (double)kr_hi);
  const float ki_hi = (float)kim, ki_lo = (float)(kim - (double)ki_hi);
  for (int sw = 0; sw < sweeps; ++sw) {
    float* rl = T->fft ? nullptr : T->Rl;
    if (sw == 0 && T->fft) {
      if (C)
        KFBI_LAUNCH_P(KFBI_PROF_GRID, k_resid_u32<true>, grid_for(plane / 4, 256), 256, 0, st, T->Rh,
                      (const float*)T->Rl, (const float*)T->U, D->d_U, Mp, T->n1, ih_hi, ih_lo,
                      kr_hi, kr_lo, ki_hi, ki_lo);
      else
        KFBI_LAUNCH_P(KFBI_PROF_GRID, k_resid_u32<false>, grid_for(plane / 4, 256), 256, 0, st, T->Rh,
                      (const float*)T->Rl, (const float*)T->U, D->d_U, Mp, T->n1, ih_hi, ih_lo,
                      kr_hi, kr_lo, ki_hi, ki_lo);
    } else if (C) {
      KFBI_LAUNCH_P(KFBI_PROF_GRID, k_resid_split<true>, grid_for(plane, 256), 256, 0, st, D->d_R,
                    D->d_U, T->Rh, rl, Mp, T->n1, inv_h2, kre, kim);
    } else {
      KFBI_LAUNCH_P(KFBI_PROF_GRID, k_resid_split<false>, grid_for(plane, 256), 256, 0, st, D->d_R,
                    D->d_U, T->Rh, rl, Mp, T->n1, inv_h2, kre, kim);
    }
    tc_box_solve(D, kre, kim, P, st);
    KFBI_LAUNCH_P(KFBI_PROF_GRID, k_add_f32, grid_for(P * plane / 4, 256), 256, 0, st, D->d_U, T->U,
                  P * plane);
  }
  if (out) extract_fp64(D, kre, kim, phi, ps, ft, out, os, st);
  KFBI_CHECK_LAUNCH();
}

// Application at phi = phi_prev + d for a small correction d, given the
// grid of an accurate application at phi_prev in D->d_U (no volume
// source): the grid is affine in the density, so W phi = W phi_prev + W d,
// and W d needs only one FP32 box solve (no refinement sweep) because its
// error scales with |d|.  D->d_U becomes W phi and out the FP64 extraction
// at phi from that grid.
void tc_apply_correction(kfbi_domain* D, double kre, double kim, const double* d, const double* phi,
                         int ps, double* out, int os, cudaStream_t st) {
  TcDst* T = D->tc;
  const bool C = kim != 0.0;
  const int P = C ? 2 : 1;
  const size_t plane = (size_t)T->Mp * T->Mp;
  correct_fp64(D, kre, kim, d, ps, nullptr, st);
  KFBI_LAUNCH_P(KFBI_PROF_GRID, k_split64, grid_for(P * plane / 4, 256), 256, 0, st, D->d_R, T->Rh,
                T->fft ? nullptr : T->Rl, P * plane, 0);
  T->rhs_sparse_planes = 0;
  tc_box_solve(D, kre, kim, P, st);
  KFBI_LAUNCH_P(KFBI_PROF_GRID, k_add_f32, grid_for(P * plane / 4, 256), 256, 0, st, D->d_U, T->U,
                P * plane);
  if (out) extract_fp64(D, kre, kim, phi, ps, nullptr, out, os, st);
  KFBI_CHECK_LAUNCH();
}

}  // namespace kfbi

// ---- self-check of the integer-pipe conversions ----------------------------

namespace kfbi {
namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  // splitmix64 finaliser
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void k_check_conversions(unsigned long long seed, long long n,
                                    unsigned long long* bad) {
  unsigned long long local = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long z = mix64(seed ^ mix64((unsigned long long)i));
    unsigned long long b = z;
    const unsigned long long sign = z & 0x8000000000000000ull;
    switch (i & 3) {
      case 0: break;  // any bit pattern
      case 1:         // exponents around the handled range
        b = sign | ((unsigned long long)(900 + (z >> 40) % 300) << 52) | (z & 0xfffffffffffffull);
        break;
      case 2:  // rounding ties: the 29 bits below the FP32 significand are 1000...0
        b = sign | ((unsigned long long)(940 + (z >> 40) % 220) << 52) |
            (z & 0xfffffe0000000ull) | 0x10000000ull;
        break;
      default:  // all-ones significand: the rounding carries into the exponent
        b = sign | ((unsigned long long)(940 + (z >> 40) % 220) << 52) |
            (0xfffffe0000000ull | ((z >> 11) & 0x1fffffffull));
        break;
    }
    const double x = __longlong_as_double((long long)b);
    float hi, lo;
    split_f64(x, hi, lo);
    const float h_ref = (float)x;
    const float l_ref = (float)(x - (double)h_ref);
    if (h_ref != h_ref) {
      local += hi == hi;
    } else {
      local += __float_as_uint(hi) != __float_as_uint(h_ref);
      local += __float_as_uint(lo) != __float_as_uint(l_ref);
    }
    const float f = __uint_as_float((uint32_t)(z >> 17));
    const double d = f32_to_f64(f), d_ref = (double)f;
    if (d_ref != d_ref) local += d == d;  // a NaN must stay a NaN (payloads may differ)
    else local += __double_as_longlong(d) != __double_as_longlong(d_ref);
  }
  if (local) atomicAdd(bad, local);
}

}  // namespace
}  // namespace kfbi

namespace kfbi {
namespace {

// A wait that must give up: an mbarrier expecting one arrival that never
// comes, waited on with the passes' bounded wait, which then records the
// failure in the error word as a pass does.
__global__ void k_wait_selftest(long long limit, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_for(&bar, 0u, limit)) atomicOr(err, 64);
}

}  // namespace
}  // namespace kfbi

extern "C" kfbi_status kfbi_check_wait_timeout(double seconds, void* stream) {
  if (!(seconds > 0.0 && seconds <= 1.0)) return KFBI_ERR_ARG;
  return kfbi::guarded(nullptr, [&]() -> kfbi_status {
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, khz = 0;
    KFBI_CUDA(cudaGetDevice(&dev));
    KFBI_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    const long long limit = (long long)(seconds * 1e3 * (double)khz);
    int* d_err = nullptr;
    KFBI_CUDA(cudaMallocAsync(&d_err, sizeof(int), st));
    KFBI_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    kfbi::k_wait_selftest<<<1, 32, 0, st>>>(limit, d_err);
    KFBI_CHECK_LAUNCH();
    int h_err = 0;
    KFBI_CUDA(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    KFBI_CUDA(cudaFreeAsync(d_err, st));
    KFBI_CUDA(cudaStreamSynchronize(st));
    if (h_err != 0)
      throw kfbi::Status{KFBI_ERR_TIMEOUT, "bounded wait gave up (flags " + std::to_string(h_err) + ")"};
    return KFBI_OK;
  });
}

extern "C" kfbi_status kfbi_check_conversions(unsigned long long seed, long long n,
                                              long long* mismatches, void* stream) {
  if (!mismatches || n < 1) return KFBI_ERR_ARG;
  return kfbi::guarded(nullptr, [&]() -> kfbi_status {
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long* d_bad = nullptr;
    KFBI_CUDA(cudaMallocAsync(&d_bad, sizeof(unsigned long long), st));
    KFBI_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), st));
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    kfbi::k_check_conversions<<<(unsigned)blocks, 256, 0, st>>>(seed, n, d_bad);
    KFBI_CHECK_LAUNCH();
    unsigned long long h_bad = 0;
    KFBI_CUDA(cudaMemcpyAsync(&h_bad, d_bad, sizeof(h_bad), cudaMemcpyDeviceToHost, st));
    KFBI_CUDA(cudaFreeAsync(d_bad, st));
    KFBI_CUDA(cudaStreamSynchronize(st));
    *mismatches = (long long)h_bad;
    return KFBI_OK;
  });
}
