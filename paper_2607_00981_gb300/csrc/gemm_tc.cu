// Split-precision GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   C[m, n] (+)= alpha[m] * sum_k (Ahi Bhi + Ahi Blo + Alo Bhi)[m, n]
//
// A [M][Kpad] and B [N][Kpad] are K-major panels split into hi/lo planes (BF16,
// or TF32 held in FP32 words); the three products accumulate in FP32 in tensor
// memory.  This is the 3-term split product of Henry, Tang & Heinecke (ARITH 2019)
// for BF16 and of Ootomo & Yokota (2022) for TF32: dropping lo*lo leaves a
// relative error of about 2^-16 (BF16) or 2^-21 (TF32) per product.
//
// Persistent kernel, one CTA per SM, 320 threads:
//   warp 0     TMA producer: swizzled K-major tiles of 128 rows of A and 128,
//              144 or 256 rows of B, hi and lo planes, into a ring of stages (256-
//              wide tiles: four stages of 64-byte K rows; narrower: three of 128);
//   warp 1     TMEM owner and MMA issuer (one thread): 3 tcgen05.mma per 32-byte
//              K slice into a 128 x 256 FP32 accumulator, double buffered in
//              TMEM (512 columns) so the epilogue of one tile overlaps the MMAs
//              of the next;
//   warps 2-9  epilogue: tcgen05.ld of the accumulator (one row per thread; the
//              two warps of a lane quadrant take alternate 32-column chunks) and
//              the table-driven scatter C[row_base[m] + col_off[sel[m]][n]] +=
//              alpha[m] * acc, or FP32 partial tiles when K is split.  Two warps
//              per quadrant double the loads in flight of read-modify-write
//              epilogues (short K, large outputs), which are latency bound.
// Every mbarrier wait is bounded by a clock64 budget; on expiry the kernel sets
// *status, drains its own copies and MMAs (bounded by at least kDrainFloor cycles,
// whatever the budget), frees TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>

#include "elem.cuh"
#include "kernels.h"

namespace rcc {
namespace {

constexpr int BM = 128;
constexpr int kEpiWarps = 8;                 // two epilogue warps per TMEM lane quadrant
constexpr int kThreads = 64 + 32 * kEpiWarps;

// Tile width BN (256 or 128 columns): B planes, stage and shared-memory sizes.
// 256-wide tiles: four stages of 64-byte K rows (48 KiB per stage; two stages of
// 128-byte rows in the same memory kept one stage in flight behind the MMAs).  128-
// and 144-wide tiles (GEMMs of few tiles, the hh-ladder): three stages of 128-byte rows
// (64 / 68 KiB per stage), whose larger copies suit these mostly load-bound GEMMs.
constexpr int row_bytes(int BN) { return BN == 256 ? 64 : 128; }
template <int BN>
struct TileCfg {
  static constexpr int ROWB = row_bytes(BN);  // bytes of one K-row of a tile (swizzle span)
  static constexpr int STAGES = BN == 256 ? 4 : 3;
  static constexpr int A_PLANE = BM * ROWB;
  static constexpr int B_PLANE = BN * ROWB;
  static constexpr int STAGE_BYTES = 2 * A_PLANE + 2 * B_PLANE;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
  static constexpr int TMEM_COLS = 2 * BN <= 256 ? 256 : 512;      // double-buffered accumulator (power of 2)
  static constexpr int FULL = BN / 32, HALF = (BN % 32) / 16;      // 32- and 16-column epilogue chunks
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false on timeout or when another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget, volatile int* abort_flag) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// Waits that retire the CTA's own asynchronous work before its shared memory and
// TMEM are released (the producer's bulk copies, the MMA issuer's tcgen05.mma) are
// bounded too, but never below kDrainFloor cycles (about a second), whatever budget
// the caller gave: a short watchdog makes the pipeline waits give up early, never
// these, so no copy or MMA outlives its CTA.
constexpr long long kDrainFloor = 1LL << 31;
__device__ __forceinline__ long long drain_budget(long long budget) { return budget > kDrainFloor ? budget : kDrainFloor; }

// Producer epilogue: wait for every bulk copy this thread issued (stage q's last copy
// has parity issued[q], -1 = never used).  In the normal path they have landed or are
// about to (the MMA issuer consumes them); after an abort nobody consumes them.
template <int NST>
__device__ __forceinline__ void drain_copies(uint64_t* full, const int (&issued)[NST], long long budget) {
  const long long lim = drain_budget(budget);
  for (int q = 0; q < NST; ++q) {
    if (issued[q] < 0) continue;
    const long long t0 = clock64();
    while (!mbar_try(&full[q], (uint32_t)issued[q]) && clock64() - t0 < lim) {
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          su32(dst)),
      "l"((uint64_t)map), "r"(su32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          su32(dst)),
      "l"((uint64_t)map), "r"(su32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// K-major, 64-byte swizzle (rows of 32 BF16), 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t sdesc64(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((512u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;  // SWIZZLE_64B
  return d;
}

// SM100 shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), version 1; tiles are 1024-byte aligned (base offset 0).
__device__ __forceinline__ uint64_t sdesc128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;                      // SWIZZLE_128B
  return d;
}
// the k_gemm_tc tiles' descriptor for K rows of ROWB bytes (swizzle span = row)
template <int ROWB>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  static_assert(ROWB == 64 || ROWB == 128, "64- or 128-byte K rows");
  if constexpr (ROWB == 64) return sdesc64(saddr);
  else return sdesc128(saddr);
}

// Instruction descriptor: D = F32, A = B = fmt (1 BF16, 2 TF32), both K-major, N = BN, M = BM.
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, int BN) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int FMT, int BN>
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  if constexpr (FMT == 1) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc(1, BN)), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc(2, BN)), "r"(acc));
  }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 16; j < 32; ++j) r[j] = 0u;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Scatter 32 accumulator columns of row m: every address and old value is
// loaded before any store, so the loads of a row overlap in flight.  A mirrored
// row (row_base2) repeats the pass at its second base; column offsets < 0 are
// skipped (the unmirrored columns of a column mirror).
__device__ __forceinline__ void epilogue_row(const EpiArgs& e, int m, int n0, const uint32_t (&r)[32]) {
  const i64* co = e.col_off + (i64)e.row_sel[m] * e.N;
  const int nv = min(32, e.N - n0);
  const int nout = (e.row_base2 && e.row_base2[m] >= 0) ? 2 : 1;
  for (int q = 0; q < nout; ++q) {
    const i64 rb = q ? e.row_base2[m] : e.row_base[m];
    const double alq = q ? e.row_alpha2[m] : e.row_alpha[m];
    if (e.c_f32) {
      float* C = (float*)epi_out(e, m);
      const float al = (float)alq;
#pragma unroll
      for (int h = 0; h < 32; h += 16) {
        i64 ad[16];
        float old[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const i64 cv = (h + j < nv) ? __ldg(co + n0 + h + j) : -1;
          ad[j] = cv >= 0 ? rb + cv : -1;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) old[j] = ad[j] >= 0 ? C[ad[j]] : 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (ad[j] >= 0) C[ad[j]] = fmaf(al, __uint_as_float(r[h + j]), old[j]);
      }
    } else {
      double* C = (double*)epi_out(e, m);
      const double al = alq;
#pragma unroll
      for (int h = 0; h < 32; h += 16) {
        i64 ad[16];
        double old[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const i64 cv = (h + j < nv) ? __ldg(co + n0 + h + j) : -1;
          ad[j] = cv >= 0 ? rb + cv : -1;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) old[j] = ad[j] >= 0 ? C[ad[j]] : 0.0;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (ad[j] >= 0) C[ad[j]] = old[j] + al * (double)__uint_as_float(r[h + j]);
      }
    }
  }
}

struct TileGeom {
  int mt, nt, splitk, kblocks, kb_per;
};

constexpr int GROUP_N = 8;  // tiles of one wave span 8 column tiles x (SMs / 8) row tiles

// One output tile: problem p, row tile tm, column tile tn, K blocks [kb0, kb1), split slice ks.
struct Tile {
  int p, tm, tn, kb0, kb1, ks;
};

// Grouped raster order: within a group of GROUP_N column tiles, the column tile
// varies fastest, then the row tile, so the A and B tiles one wave reads stay
// L2-resident (about 4x less HBM traffic than a plain row-major order on the
// largest GEMMs).
__device__ __forceinline__ void raster(int mt, int nt, int t, int& tm, int& tn) {
  const int per_group = mt * GROUP_N;
  const int grp = t / per_group, idx = t % per_group;
  const int gw = min(GROUP_N, nt - grp * GROUP_N);
  tm = idx / gw;
  tn = grp * GROUP_N + idx % gw;
}

// Schedule of a single GEMM (optionally split along K) with the table-driven
// scatter epilogue or FP32 partial tiles.  Tensor maps live in the kernel's
// parameter space (__grid_constant__).
template <bool COLM>  // COLM: the epilogue adds the column mirror (EpiArgs::col_off2) in a second pass
struct PlainSchedT {
  CUtensorMap ah, al, bh, bl;
  TileGeom g;
  EpiArgs e;
  float* partial;  // [splitk][M][N] partial tiles, or the dense raw result when splitk == 1
  int colmajor;    // raw result stored as [N][M] (each thread's row runs along memory)
  __device__ __forceinline__ int ntiles() const { return g.mt * g.nt * g.splitk; }
  __device__ __forceinline__ void tile(int t, Tile& x) const {
    // split slices K-range-major: the CTAs of one wave take every tile of the same
    // K ranges, so the A and B slices they read are shared through L2
    const int nmn = g.mt * g.nt;
    x.p = 0;
    x.ks = t / nmn;
    raster(g.mt, g.nt, t - x.ks * nmn, x.tm, x.tn);
    x.kb0 = x.ks * g.kb_per;
    x.kb1 = min(g.kblocks, x.kb0 + g.kb_per);
  }
  __device__ __forceinline__ const CUtensorMap* map(int q, const Tile&) const {
    return q == 0 ? &ah : q == 1 ? &al : q == 2 ? &bh : &bl;
  }
  __device__ __forceinline__ void store(const Tile& x, int m, int n0, const uint32_t (&r)[32], int ncols) const {
    if (m >= e.M) return;
    if (partial && colmajor) {
      float* dst = partial + (i64)n0 * e.M + m;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < ncols && n0 + j < e.N) dst[(i64)j * e.M] = __uint_as_float(r[j]);
    } else if (partial) {
      float* dst = partial + ((i64)x.ks * e.M + m) * e.N;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < ncols && n0 + j < e.N) dst[n0 + j] = __uint_as_float(r[j]);
    } else {
      EpiArgs e2 = e;
      if (ncols < 32) e2.N = min(e.N, n0 + ncols);
      // with the column mirror, a second pass over the mirrored offsets (one loop body)
#pragma unroll 1
      for (int q = 0; q < (COLM ? 2 : 1); ++q) {
        if (q) {
          e2.col_off = e.col_off2;
          e2.row_alpha = e.row_alpha2;
          e2.row_base2 = nullptr;
        }
        epilogue_row(e2, m, n0, r);
      }
    }
  }
};

using PlainSched = PlainSchedT<false>;

// Schedule of a group of independent GEMMs of different shapes (problem table in
// device memory, tensor maps included): one persistent launch runs every tile
// of every problem; problem p owns the tiles [tile0_p, tile0_p + mt_p nt_p).
// Each problem writes its dense FP32 result out_p[M_p][N_p].
struct GroupSched {
  const GProblem* probs;
  int nprob, total;
  __device__ __forceinline__ int ntiles() const { return total; }
  __device__ __forceinline__ void tile(int t, Tile& x) const {
    int lo = 0, hi = nprob - 1;  // last problem with tile0 <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&probs[mid].tile0) <= t) lo = mid;
      else hi = mid - 1;
    }
    const GProblem& P = probs[lo];
    x.p = lo;
    x.ks = 0;
    raster(__ldg(&P.mt), __ldg(&P.nt), t - __ldg(&P.tile0), x.tm, x.tn);
    x.kb0 = 0;
    x.kb1 = __ldg(&P.kblocks);
  }
  __device__ __forceinline__ const CUtensorMap* map(int q, const Tile& x) const {
    const GProblem& P = probs[x.p];
    return q == 0 ? &P.ah : q == 1 ? &P.al : q == 2 ? &P.bh : &P.bl;
  }
  __device__ __forceinline__ void store(const Tile& x, int m, int n0, const uint32_t (&r)[32], int ncols) const {
    const GProblem& P = probs[x.p];
    const int M = __ldg(&P.M), N = __ldg(&P.N);
    if (m >= M) return;
    if (__ldg(&P.colmajor)) {
      float* dst = P.out + (i64)n0 * M + m;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < ncols && n0 + j < N) dst[(i64)j * M] = __uint_as_float(r[j]);
      return;
    }
    float* dst = P.out + (i64)m * N + n0;
    if ((N & 3) == 0 && ncols == 32 && n0 + 32 <= N) {
#pragma unroll
      for (int j = 0; j < 32; j += 4)
        *(float4*)(dst + j) = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                          __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < ncols && n0 + j < N) dst[j] = __uint_as_float(r[j]);
    }
  }
};

// A group whose tile count (and the problems' tile0) an earlier kernel of the same
// stream or graph wrote to device memory (a batch of instances, some of which sit
// out an iteration).
struct GroupSchedDev : GroupSched {
  const int* total_dev;
  __device__ __forceinline__ int ntiles() const { return *(volatile const int*)total_dev; }
};

template <int FMT, int BN, class S>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ S sch, int* __restrict__ status, long long budget) {
  constexpr int B_PLANE = TileCfg<BN>::B_PLANE, STAGE_BYTES = TileCfg<BN>::STAGE_BYTES;
  constexpr int ROWB = TileCfg<BN>::ROWB, STAGES = TileCfg<BN>::STAGES, A_PLANE = TileCfg<BN>::A_PLANE;
  constexpr int TMEM_COLS = TileCfg<BN>::TMEM_COLS;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ntiles = sch.ntiles();

  if (warp == 0) {
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int issued[STAGES];
      for (int q = 0; q < STAGES; ++q) issued[q] = -1;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        Tile x;
        sch.tile(tile, x);
        const CUtensorMap *mah = sch.map(0, x), *mal = sch.map(1, x), *mbh = sch.map(2, x), *mbl = sch.map(3, x);
        for (int kb = x.kb0; kb < x.kb1; ++kb) {
          if (!mbar_wait(&empty[s], ph ^ 1, budget, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          const int kx = kb * (ROWB / (FMT == 1 ? 2 : 4));
          tma_load_2d(st, mah, &full[s], kx, x.tm * BM);
          tma_load_2d(st + A_PLANE, mal, &full[s], kx, x.tm * BM);
          tma_load_2d(st + 2 * A_PLANE, mbh, &full[s], kx, x.tn * BN);
          tma_load_2d(st + 2 * A_PLANE + B_PLANE, mbl, &full[s], kx, x.tn * BN);
          issued[s] = (int)ph;
          if (++s == STAGES) {
            s = 0;
            ph ^= 1;
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(status, 1);
      }
      // drain: every copy this thread issued has landed before the CTA may exit
      drain_copies<STAGES>(full, issued, budget);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int it = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
        Tile x;
        sch.tile(tile, x);
        const int b = it & 1;
        const uint32_t aph = (it >> 1) & 1;
        if (!mbar_wait(&tempty[b], aph ^ 1, budget, abort_flag)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(b * BN);
        for (int kb = x.kb0; kb < x.kb1; ++kb) {
          if (!mbar_wait(&full[s], ph, budget, abort_flag)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t base = su32(smem + s * STAGE_BYTES);
          const uint64_t ah = sdesc<ROWB>(base), al = sdesc<ROWB>(base + A_PLANE);
          const uint64_t bh = sdesc<ROWB>(base + 2 * A_PLANE), bl = sdesc<ROWB>(base + 2 * A_PLANE + B_PLANE);
#pragma unroll
          for (int j = 0; j < ROWB / 32; ++j) {
            const uint64_t adv = (uint64_t)(j * 32 >> 4);  // 32-byte K slice inside the swizzled row
            umma<FMT, BN>(d, ah + adv, bh + adv, (kb > x.kb0 || j > 0) ? 1u : 0u);
            umma<FMT, BN>(d, ah + adv, bl + adv, 1u);
            umma<FMT, BN>(d, al + adv, bh + adv, 1u);
          }
          umma_commit(&empty[s]);
          if (++s == STAGES) {
            s = 0;
            ph ^= 1;
          }
        }
        if (!ok) break;
        umma_commit(&tfull[b]);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(status, 1);
      }
      // make sure every MMA this thread issued has completed before TMEM is freed
      umma_commit(drain);
      const long long t0 = clock64(), lim = drain_budget(budget);
      while (!mbar_try(drain, 0) && clock64() - t0 < lim) {
      }
    }
  } else {
    const int q = warp & 3;        // TMEM lane quadrant this warp may read
    const int h = (warp - 2) >> 2;  // which of the quadrant's two warps
    const int row = q * 32 + lane;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      Tile x;
      sch.tile(tile, x);
      const int b = it & 1;
      const uint32_t aph = (it >> 1) & 1;
      if (!mbar_wait(&tfull[b], aph, budget, abort_flag)) {
        *abort_flag = 1;
        atomicExch(status, 1);
        break;
      }
      fence_after();
      const int m = x.tm * BM + row;
      for (int c = h; c < TileCfg<BN>::FULL; c += 2) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + c * 32), r);
        sch.store(x, m, x.tn * BN + c * 32, r, 32);
      }
      if (TileCfg<BN>::HALF && h == (TileCfg<BN>::FULL & 1)) {
        uint32_t r[32];
        const int c0 = TileCfg<BN>::FULL * 32;
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + c0), r);
        sch.store(x, m, x.tn * BN + c0, r, 16);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------------------------------
// FP64-accurate GEMM on the BF16 tensor cores (FP64 bodies):
//   C[m, n] (+)= alpha[m] * sum_k A[m, k] B[n, k],  A = 2^(e_m - 7) sum_s a_s, B likewise
// with the digit planes of slice_digits (elem.cuh).  Of the 36 digit products the 21
// with s + t <= 5 are summed on the tensor cores into four FP32 accumulators in TMEM,
// by digit level d = s + t: d = 0, 1, 2 each in its own (values are multiples of
// 2^-7d), d = 3..5 together.  Over a chunk of 256 K values the first three stay below
// 2^24 units of their granularity (|d_s| <= 128, at most three products per level),
// so they are exact however the tensor cores align and truncate partial sums; the
// last is about 2^-21 of the first, so its truncation errors (measured: a few 2^-24
// of it per chunk) stay near 2^-37 of the result.  (One accumulator for all levels
// d >= 2 measured 2^-30.)  After each chunk the epilogue warps add the four to a
// double-float (two FP32) running sum per element, and the tile ends with one FP64
// step: C += alpha * 2^(e_m + f_n - 14) * (hi + lo).
// This is the error-free splitting of matrix products (Ozaki, Ogita, Oishi, Rump,
// Numer. Algorithms 59, 2012) with fixed 7-bit digits; the neglected digits and digit
// products leave about 2^-38 of the row and column maxima times K.
//
// Persistent CTA per SM, 320 threads: warp 0 TMA (both operands' six planes of a
// 128 x 32 tile in one 3D copy each, 64-byte swizzle, 2 stages of 96 KiB), warp 1
// TMEM owner and MMA issuer, warps 2-9 epilogue (two per TMEM lane quadrant, 64
// columns each).  All waits are bounded as in k_gemm_tc.
// ---------------------------------------------------------------------------
constexpr int EBN = 64;                          // tile width (two double-float sums of 32 columns per thread)
constexpr int EKB = 32;                          // K per stage (64-byte rows)
constexpr int E_APLANE = 128 * EKB * 2;          // one digit plane of a 128-row A tile: 8 KiB
constexpr int E_BPLANE = EBN * EKB * 2;          // one digit plane of a 64-row B tile: 4 KiB
constexpr int E_AOPER = kSlices * E_APLANE, E_BOPER = kSlices * E_BPLANE;
constexpr int E_STAGE = E_AOPER + E_BOPER;       // 72 KiB
constexpr int E_STAGES = 3;
constexpr int E_CHUNK = 256 / EKB;               // stages per exact chunk
constexpr int E_SMEM = E_STAGES * E_STAGE + 1024 + 256;
constexpr int E_NACC = 4;                        // accumulators per buffer (digit levels 0, 1, 2, >= 3)
constexpr int E_ACC = E_NACC * EBN;              // one buffer (two buffers in 512 columns)

struct F64ESched {
  CUtensorMap a, b;        // 3D maps {Kpad, rows, kSlices} of the digit planes
  const int* ea;           // per-row scale exponents of A and B
  const int* eb;
  EpiArgs e;
  int mt, nt, kstages;
};

__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {  // (hi, lo) += x, TwoSum
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_f64e(const __grid_constant__ F64ESched sch, int* __restrict__ status, long long budget) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + E_STAGES * E_STAGE);
  uint64_t* empty = full + E_STAGES;
  uint64_t* tfull = empty + E_STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int q = 0; q < E_STAGES; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEpiWarps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ntiles = sch.mt * sch.nt;
  const int ks = sch.kstages;
  const int nchunk = (ks + E_CHUNK - 1) / E_CHUNK;

  if (warp == 0) {
    if (lane == 0) {
      int st = 0;
      uint32_t ph = 0;
      int issued[E_STAGES];
      for (int q = 0; q < E_STAGES; ++q) issued[q] = -1;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int tm, tn;
        raster(sch.mt, sch.nt, tile, tm, tn);
        for (int kb = 0; kb < ks; ++kb) {
          if (!mbar_wait(&empty[st], ph ^ 1, budget, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* sp = smem + st * E_STAGE;
          mbar_expect_tx(&full[st], E_STAGE);
          tma_load_3d(sp, &sch.a, &full[st], kb * EKB, tm * BM, 0);
          tma_load_3d(sp + E_AOPER, &sch.b, &full[st], kb * EKB, tn * EBN, 0);
          issued[st] = (int)ph;
          if (++st == E_STAGES) {
            st = 0;
            ph ^= 1;
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(status, 1);
      }
      drain_copies<E_STAGES>(full, issued, budget);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int st = 0;
      uint32_t ph = 0;
      int chunk = 0;  // chunks issued by this CTA; buffer chunk & 1
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int c = 0; c < nchunk && ok; ++c, ++chunk) {
          const int b = chunk & 1;
          if (!mbar_wait(&tempty[b], (uint32_t)((chunk >> 1) & 1) ^ 1u, budget, abort_flag)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t d0 = tmem + (uint32_t)(b * E_ACC);
          bool first[E_NACC] = {true, true, true, true};
          const int kb1 = min(ks, (c + 1) * E_CHUNK);
          for (int kb = c * E_CHUNK; kb < kb1; ++kb) {
            if (!mbar_wait(&full[st], ph, budget, abort_flag)) {
              ok = false;
              break;
            }
            fence_after();
            const uint32_t base = su32(smem + st * E_STAGE);
#pragma unroll
            for (int sa = 0; sa < kSlices; ++sa) {
#pragma unroll
              for (int sb = 0; sb < kSlices - sa; ++sb) {
                const int acc = sa + sb < 3 ? sa + sb : 3;
                const uint64_t da = sdesc64(base + sa * E_APLANE), db = sdesc64(base + E_AOPER + sb * E_BPLANE);
#pragma unroll
                for (int j = 0; j < EKB / 16; ++j) {
                  const uint64_t adv = (uint64_t)(j * 32 >> 4);
                  umma<1, EBN>(d0 + (uint32_t)(acc * EBN), da + adv, db + adv, first[acc] ? 0u : 1u);
                  first[acc] = false;
                }
              }
            }
            umma_commit(&empty[st]);
            if (++st == E_STAGES) {
              st = 0;
              ph ^= 1;
            }
          }
          if (!ok) break;
          umma_commit(&tfull[b]);
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(status, 1);
      }
      umma_commit(drain);
      const long long t0 = clock64(), lim = drain_budget(budget);
      while (!mbar_try(drain, 0) && clock64() - t0 < lim) {
      }
    }
  } else {
    const int q = warp & 3, h = (warp - 2) >> 2;  // lane quadrant, column half
    const int row = q * 32 + lane;
    int chunk = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      int tm, tn;
      raster(sch.mt, sch.nt, tile, tm, tn);
      float shi[32], slo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) shi[j] = slo[j] = 0.f;
      for (int c = 0; c < nchunk; ++c, ++chunk) {
        const int b = chunk & 1;
        if (!mbar_wait(&tfull[b], (uint32_t)((chunk >> 1) & 1), budget, abort_flag)) {
          *abort_flag = 1;
          atomicExch(status, 1);
          ok = false;
          break;
        }
        fence_after();
#pragma unroll
        for (int acc = 0; acc < E_NACC; ++acc) {
          uint32_t r[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * E_ACC + acc * EBN + h * 32), r);
#pragma unroll
          for (int j = 0; j < 32; ++j) df_add(shi[j], slo[j], __uint_as_float(r[j]));
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
      }
      if (!ok) break;
      // finish the tile in FP64: C += alpha * 2^(e_m + f_n - 14) * (hi + lo)
      const EpiArgs& e = sch.e;
      const int m = tm * BM + row;
      if (m < e.M) {
        const i64* co0 = e.col_off + (i64)e.row_sel[m] * e.N;
        const int em = sch.ea[m];
        void* C = epi_out(e, m);
        const bool rowm = e.row_base2 && e.row_base2[m] >= 0;
        const int nout = (rowm || e.col_off2) ? 2 : 1;
        for (int q = 0; q < nout; ++q) {
          const i64 rb = (q && rowm) ? e.row_base2[m] : e.row_base[m];
          const i64* co = (q && !rowm) ? e.col_off2 : co0;  // column offsets < 0: no second copy
          const double al = q ? e.row_alpha2[m] : e.row_alpha[m];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int n = tn * EBN + h * 32 + j;
            const i64 cv = n < e.N ? __ldg(co + n) : -1;
            if (cv >= 0) {
              const int sc = em + __ldg(sch.eb + n) - 14;
              const double pw = __longlong_as_double((long long)(sc + 1023) << 52);  // |sc| < 1000 for finite data
              const double val = ((double)shi[j] + (double)slo[j]) * pw;
              const i64 ad = rb + cv;
              if (e.c_f32)  // FP32 storage (R3 of split contexts)
                ((float*)C)[ad] = (float)((double)((float*)C)[ad] + al * val);
              else
                ((double*)C)[ad] += al * val;
            }
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// Digit planes of an FP64 panel: one CTA per row (grid-strided), the row's scale
// exponent from an integer max over the magnitudes' bit patterns, then the digits.
__global__ void __launch_bounds__(256) k_slice_f64(const double* __restrict__ P, int R, int Kpad,
                                                   __nv_bfloat16* __restrict__ planes, int* __restrict__ exps) {
  __shared__ unsigned long long red[8];
  const i64 plane = (i64)R * Kpad;
  for (int r = blockIdx.x; r < R; r += gridDim.x) {
    const double* row = P + (i64)r * Kpad;
    unsigned long long mx = 0;
    for (int k = threadIdx.x; k < Kpad; k += blockDim.x) mx = max(mx, f64_magnitude_bits(row[k]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
      unsigned long long v = threadIdx.x < 8 ? red[threadIdx.x] : 0ull;
#pragma unroll
      for (int off = 4; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
      if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const int ex = slice_exponent(red[0]);
    if (threadIdx.x == 0) exps[r] = ex;
    for (int k = threadIdx.x; k < Kpad; k += blockDim.x) {
      float a[kSlices];
      slice_digits(row[k], ex, a);
#pragma unroll
      for (int s = 0; s < kSlices; ++s) planes[s * plane + (i64)r * Kpad + k] = __float2bfloat16_rn(a[s]);
    }
    __syncthreads();  // red[] is reused by the next row
  }
}

__global__ void k_splitk_reduce_f32(const float* __restrict__ partial, int splitk, EpiArgs e) {
  const i64 MN = (i64)e.M * e.N;
  for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < MN; x += (i64)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splitk; ++z) s += (double)partial[z * MN + x];
    epi_apply(e, (int)(x / e.N), (int)(x % e.N), s);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// rowb: bytes of one K row of the kernel's tiles (64 or 128, the swizzle span)
bool make_map(CUtensorMap* map, const void* ptr, int rows, int Kpad, int kind, int box_rows, int rowb) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int esz = kind == PANEL_BF16X2 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)Kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kpad * esz};
  if (rowb != 64 && rowb != 128) return false;
  cuuint32_t box[2] = {(cuuint32_t)(rowb / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = kind == PANEL_BF16X2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  return fn(map, dt, 2, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            rowb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

}  // namespace

template <int FMT, int BN, class S>
static void launch_sched(const S& sch, int grid, int* status_flag, long long budget, cudaStream_t s) {
  constexpr int SMEM = TileCfg<BN>::SMEM_BYTES;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_tc<FMT, BN, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    attr = true;
  }
  ++g_launch_count;
  k_gemm_tc<FMT, BN, S><<<grid, kThreads, SMEM, s>>>(sch, status_flag, budget);
}

template <class S>
static void launch_any(int kind, int bn, const S& sch, int grid, int* status_flag, long long budget, cudaStream_t s) {
  if (kind == PANEL_BF16X2) {
    if (bn == 128) launch_sched<1, 128>(sch, grid, status_flag, budget, s);
    else if (bn == 144) launch_sched<1, 144>(sch, grid, status_flag, budget, s);
    else launch_sched<1, 256>(sch, grid, status_flag, budget, s);
  } else {
    if (bn == 128) launch_sched<2, 128>(sch, grid, status_flag, budget, s);
    else if (bn == 144) launch_sched<2, 144>(sch, grid, status_flag, budget, s);
    else launch_sched<2, 256>(sch, grid, status_flag, budget, s);
  }
}

int launch_gemm_tc(int kind, const void* Ahi, const void* Alo, const void* Bhi, const void* Blo, int Kpad,
                   const EpiArgs& e, int* status_flag, long long watchdog, cudaStream_t s, float* scratch,
                   long long scratch_elems, float* raw_out, int bn, int colmajor) {
  if (kind != PANEL_BF16X2 && kind != PANEL_TF32X2) return 1;
  int BN = (bn == 128 || bn == 144) ? bn : 256;
  const int esz = kind == PANEL_BF16X2 ? 2 : 4;
  if (e.M <= 0 || e.N <= 0) return 1;
  if (e.col_off2 && (BN != 256 || raw_out || e.row_base2)) return 1;  // column mirror: 256-wide, direct epilogue
  // A table-epilogue GEMM of few 256-wide tiles is bound by its epilogue's chains of
  // dependent loads (eight warps per tile): with at most half the SMs busy, 128-wide
  // tiles give twice the CTAs and half the epilogue work each.
  if (BN == 256 && !raw_out && !e.col_off2 &&
      2LL * ((e.M + BM - 1) / BM) * ((e.N + 255) / 256) <= (long long)num_sms())
    BN = 128;
  const int rowb = row_bytes(BN), bk = rowb / esz;
  if (Kpad % bk != 0) return 1;
  PlainSched sch;
  if (!make_map(&sch.ah, Ahi, e.M, Kpad, kind, BM, rowb) || !make_map(&sch.al, Alo, e.M, Kpad, kind, BM, rowb) ||
      !make_map(&sch.bh, Bhi, e.N, Kpad, kind, BN, rowb) || !make_map(&sch.bl, Blo, e.N, Kpad, kind, BN, rowb))
    return 2;
  TileGeom& g = sch.g;
  g.mt = (e.M + BM - 1) / BM;
  g.nt = (e.N + BN - 1) / BN;
  g.kblocks = Kpad / bk;
  g.splitk = 1;
  const int sms = num_sms();
  const int tiles = g.mt * g.nt;
  if (tiles < sms && g.kblocks >= 8 && scratch && !raw_out) {
    // split factor with the shortest critical path: whole waves of tile slices times
    // the K blocks of one slice (plus a few K blocks' worth of epilogue per slice), so
    // that the last wave is not a sliver of the SMs
    const int max_sk = std::min(g.kblocks / 4, 64);
    long long best = -1;
    int best_sk = 1;
    for (int sk = 1; sk <= max_sk; ++sk) {
      const int kb_per = (g.kblocks + sk - 1) / sk;
      const int real = (g.kblocks + kb_per - 1) / kb_per;
      if (real > 1 && (long long)real * e.M * e.N > scratch_elems) break;
      const long long waves = ((long long)tiles * real + sms - 1) / sms;
      const long long cost = waves * (kb_per + 4);
      if (best < 0 || cost < best) {
        best = cost;
        best_sk = real;
      }
    }
    g.splitk = best_sk;
  }
  g.kb_per = (g.kblocks + g.splitk - 1) / g.splitk;
  g.splitk = (g.kblocks + g.kb_per - 1) / g.kb_per;
  const int ntiles = tiles * g.splitk;
  const int grid = std::min(ntiles, sms);
  const long long budget = watchdog > 0 ? watchdog : 4000000000LL;
  float* part = raw_out ? raw_out : (g.splitk > 1 ? scratch : nullptr);
  sch.e = e;
  sch.partial = part;
  sch.colmajor = raw_out && colmajor ? 1 : 0;
  if (e.col_off2 && !part) {
    PlainSchedT<true> schm;
    schm.ah = sch.ah;
    schm.al = sch.al;
    schm.bh = sch.bh;
    schm.bl = sch.bl;
    schm.g = sch.g;
    schm.e = sch.e;
    schm.partial = sch.partial;
    schm.colmajor = sch.colmajor;
    if (kind == PANEL_BF16X2) launch_sched<1, 256>(schm, grid, status_flag, budget, s);
    else launch_sched<2, 256>(schm, grid, status_flag, budget, s);
  } else {
    launch_any(kind, BN, sch, grid, status_flag, budget, s);
  }
  if (part && !raw_out) {
    const long long MN = (long long)e.M * e.N;
    long long blocks = (MN + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    ++g_launch_count;
    k_splitk_reduce_f32<<<(unsigned)blocks, 256, 0, s>>>(part, g.splitk, e);
  }
  return 0;
}

int gemm_tc_block_k(int kind, int bn) {
  const int BN = (bn == 128 || bn == 144) ? bn : 256;
  return row_bytes(BN) / (kind == PANEL_BF16X2 ? 2 : 4);
}

int make_gproblem(GProblem* p, int kind, const void* Ahi, const void* Alo, const void* Bhi, const void* Blo, int M,
                  int N, int Kpad, float* out, int bn) {
  if (kind != PANEL_BF16X2 && kind != PANEL_TF32X2) return 1;
  const int BN = (bn == 128 || bn == 144) ? bn : 256;
  const int bk = gemm_tc_block_k(kind, BN), rowb = row_bytes(BN);
  if (Kpad % bk != 0 || M <= 0 || N <= 0) return 1;
  if (!make_map(&p->ah, Ahi, M, Kpad, kind, BM, rowb) || !make_map(&p->al, Alo, M, Kpad, kind, BM, rowb) ||
      !make_map(&p->bh, Bhi, N, Kpad, kind, BN, rowb) || !make_map(&p->bl, Blo, N, Kpad, kind, BN, rowb))
    return 2;
  p->a_hi = Ahi;
  p->a_lo = Alo;
  p->b_hi = Bhi;
  p->b_lo = Blo;
  p->out = out;
  p->colmajor = 0;
  p->M = M;
  p->N = N;
  p->Kpad = Kpad;
  p->kblocks = Kpad / bk;
  p->mt = (M + BM - 1) / BM;
  p->nt = (N + BN - 1) / BN;
  return 0;
}

int gproblem_tiles(const GProblem& p) { return p.mt * p.nt; }

int launch_gemm_tc_grouped(int kind, const GProblem* probs, int nprob, int total_tiles, int grid, int bn,
                           int* status_flag, long long watchdog, cudaStream_t s) {
  if ((kind != PANEL_BF16X2 && kind != PANEL_TF32X2) || nprob <= 0 || total_tiles <= 0) return 1;
  GroupSched sch;
  sch.probs = probs;
  sch.nprob = nprob;
  sch.total = total_tiles;
  const int g = std::max(1, std::min(grid > 0 ? grid : num_sms(), total_tiles));
  const long long budget = watchdog > 0 ? watchdog : 4000000000LL;
  launch_any(kind, (bn == 128 || bn == 144) ? bn : 256, sch, g, status_flag, budget, s);
  return 0;
}

int launch_gemm_tc_grouped_dev(int kind, const GProblem* probs, int nprob, int max_tiles, const int* total_dev,
                               int grid, int bn, int* status_flag, long long watchdog, cudaStream_t s) {
  if ((kind != PANEL_BF16X2 && kind != PANEL_TF32X2) || nprob <= 0 || max_tiles <= 0 || !total_dev) return 1;
  GroupSchedDev sch;
  sch.probs = probs;
  sch.nprob = nprob;
  sch.total = max_tiles;
  sch.total_dev = total_dev;
  const int g = std::max(1, std::min(grid > 0 ? grid : num_sms(), max_tiles));
  const long long budget = watchdog > 0 ? watchdog : 4000000000LL;
  launch_any(kind, (bn == 128 || bn == 144) ? bn : 256, sch, g, status_flag, budget, s);
  return 0;
}

bool make_map_planes(CUtensorMap* map, const void* planes, int rows, int Kpad, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)rows, (cuuint64_t)kSlices};
  cuuint64_t strides[2] = {(cuuint64_t)Kpad * 2, (cuuint64_t)rows * Kpad * 2};
  cuuint32_t box[3] = {(cuuint32_t)EKB, (cuuint32_t)box_rows, (cuuint32_t)kSlices};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(planes), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void launch_slice_f64(const double* P, int R, int Kpad, void* planes, int* exps, cudaStream_t s) {
  if (R <= 0) return;
  ++g_launch_count;
  k_slice_f64<<<(unsigned)std::min(R, 152 * 16), 256, 0, s>>>(P, R, Kpad, (__nv_bfloat16*)planes, exps);
}

int launch_gemm_f64e(const void* Aplanes, const int* ea, const void* Bplanes, const int* eb, int Kpad, const EpiArgs& e,
                     int* status_flag, long long watchdog, cudaStream_t s) {
  if (Kpad % 64 != 0 || e.M <= 0 || e.N <= 0) return 1;
  F64ESched sch;
  if (!make_map_planes(&sch.a, Aplanes, e.M, Kpad, BM) || !make_map_planes(&sch.b, Bplanes, e.N, Kpad, EBN)) return 2;
  sch.ea = ea;
  sch.eb = eb;
  sch.e = e;
  sch.mt = (e.M + BM - 1) / BM;
  sch.nt = (e.N + EBN - 1) / EBN;
  sch.kstages = Kpad / EKB;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_f64e, cudaFuncAttributeMaxDynamicSharedMemorySize, E_SMEM);
    attr = true;
  }
  const int grid = std::min(sch.mt * sch.nt, num_sms());
  ++g_launch_count;
  k_gemm_f64e<<<grid, kThreads, E_SMEM, s>>>(sch, status_flag, watchdog > 0 ? watchdog : 4000000000LL);
  return 0;
}

}  // namespace rcc
