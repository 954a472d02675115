// Bandwidth-bound and FP64 kernels of the RCCSDT iteration (sm_103a).
//
//  k_pack        strided / permuted / spin-summed gather of a GEMM operand panel
//                (the "unpacking" of Sec. II.C.2), optionally split into hi/lo halves
//  k_gemm_f64    FP64 DFMA GEMM C += A B^T with the table-driven scatter epilogue
//  k_combine     out = beta*out + sum_t c_t in_t[perm_t(idx)] on dense tensors <= rank 6
//  k_post        symmetrise / purify / orthogonalise compact R3 (Sec. II.D)
//  k_update_*    Jacobi step t += r / eps (appendix A.1)
//  k_wdot, k_sum deterministic weighted dot products (norms, DIIS B matrix)
//  k_diis_*      DIIS bordered solve and extrapolation (Sec. III.A.5)
#include <algorithm>
#include <type_traits>

#include "elem.cuh"
#include "kernels.h"

namespace rcc {

long long g_launch_count = 0;  // kernels launched by this library (host-side count)

// The six orderings of three virtual labels (lexicographic); index = selector.
__constant__ int c_perm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// ---------------------------------------------------------------------------
// Panel gather.  32 x 32 tile per block of 32 x 8 threads; reads go along the
// source's contiguous direction, writes along k (the output's contiguous axis).
// ---------------------------------------------------------------------------
// One 32 x 32 tile per step; the tile's column tables (coefficient, base offset,
// selector of up to 3 terms) and, with a single selector, its 32 row offsets
// are staged in shared memory, so an element costs one source load.
// F32: FP32 arithmetic into split panels (FP32 sources read directly, FP64 sources
// converted on the integer path); otherwise FP64 arithmetic (FP64 panels).
template <bool F32>
__device__ __forceinline__ void pack_tiles(const PackArgs& a, int r0, int kfirst, int kstep) {
  typedef typename std::conditional<F32, float, double>::type T;
  __shared__ T tile[32][33];
  __shared__ i64 cb[3][32];
  __shared__ T cf[3][32];
  __shared__ int sl[3][32];
  __shared__ i64 ro[32];
  __shared__ int lab[3][32];   // computed row offsets: the tile rows' labels ...
  __shared__ i64 cs[3][3][32];  // ... and, per term and column, the label strides
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int nterm = a.nterm < 3 ? a.nterm : 3;
  const int rm = a.row_mode;
  if (!rm && a.one_sel && tid < 32) ro[tid] = (r0 + tid < a.R) ? a.rowoff[r0 + tid] : 0;
  if (rm && tid < 32) {
    const int r = r0 + tid < a.R ? r0 + tid : 0, lv = a.lv;
    lab[0][tid] = rm == 2 ? r / lv : r / (lv * lv);
    lab[1][tid] = rm == 2 ? r % lv : (r / lv) % lv;
    lab[2][tid] = rm == 2 ? 0 : r % lv;
  }
  auto value = [&](int rr, int kk) -> T {
    const int r = r0 + rr;
    T s = (T)0;
    for (int t = 0; t < nterm; ++t) {
      const T c = cf[t][kk];
      if (c != (T)0) {
        const i64 off = cb[t][kk] + (rm ? lab[0][rr] * cs[t][0][kk] + lab[1][rr] * cs[t][1][kk] +
                                              lab[2][rr] * cs[t][2][kk]
                                        : (a.one_sel ? ro[rr] : a.rowoff[(i64)sl[t][kk] * a.R + r]));
        if constexpr (F32)  // no FP64 instructions on the FP32 path
          s += c * (a.src_f32 ? ((const float*)a.src)[off] : f64_to_f32_rn(((const double*)a.src)[off]));
        else
          s += c * (T)load_src(a.src, a.src_f32, off);
      }
    }
    return s;
  };
  auto store = [&](int r, int k, T x) {
    if constexpr (F32)
      store_panel_f(a, r, k, x);
    else
      store_panel(a, r, k, x);
  };
  for (int k0 = kfirst; k0 < a.Kpad; k0 += kstep) {
    __syncthreads();
    if (tid < nterm * 32) {
      const int t = tid >> 5, kk = tid & 31, k = k0 + kk;
      const bool ok = k < a.K;
      const i64 idx = (i64)t * a.K + k;
      cb[t][kk] = ok ? a.colbase[idx] : 0;
      cf[t][kk] = ok ? (T)a.coef[idx] : (T)0;
      const int sel = ok ? a.sel[idx] : 0;
      sl[t][kk] = sel;
      if (rm) {
        const i64 v = a.lv;
        auto S = [&](int axis) { return axis == 0 ? v * v : (axis == 1 ? v : (i64)1); };
        cs[t][0][kk] = rm == 2 ? S(sel / 3) : S(perm3(sel, 0));
        cs[t][1][kk] = rm == 2 ? S(sel % 3) : S(perm3(sel, 1));
        cs[t][2][kk] = rm == 2 ? 0 : S(perm3(sel, 2));
      }
    }
    __syncthreads();
    if (a.read_k_fast) {
      for (int rr = ty; rr < 32; rr += 8) {
        const int r = r0 + rr, k = k0 + tx;
        if (r < a.R && k < a.Kpad) store(r, k, value(rr, tx));
      }
    } else {
      for (int kk = ty; kk < 32; kk += 8) tile[kk][tx] = (r0 + tx < a.R) ? value(tx, kk) : (T)0;
      __syncthreads();
      for (int rr = ty; rr < 32; rr += 8) {
        const int r = r0 + rr, k = k0 + tx;
        if (r < a.R && k < a.Kpad) store(r, k, tile[tx][rr]);
      }
    }
  }
}

// Lean FP32-source gather into split panels (the common case): NT terms at most,
// panel kind KIND, 32-bit offsets inside a stored block (v^3 < 2^31), one row
// pointer per output row.  Same tiles and semantics as pack_tiles<true>.
template <int NT, int KIND>
__device__ __forceinline__ void pack_tiles_f32(const PackArgs& a, int r0, int kfirst, int kstep) {
  __shared__ float tile[32][33];
  __shared__ i64 cb[NT][32];
  __shared__ float cf[NT][32];
  __shared__ int sl[NT][32];
  __shared__ int cs[NT][3][32];
  __shared__ i64 ro[32];
  __shared__ int lab[3][32];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int nterm = a.nterm < NT ? a.nterm : NT;
  const int rm = a.row_mode;
  const float* src = (const float*)a.src;
  if (tid < 32) {
    const int r = r0 + tid < a.R ? r0 + tid : 0, lv = a.lv;
    if (rm) {
      lab[0][tid] = rm == 2 ? r / lv : r / (lv * lv);
      lab[1][tid] = rm == 2 ? r % lv : (r / lv) % lv;
      lab[2][tid] = rm == 2 ? 0 : r % lv;
    } else if (a.one_sel) {
      ro[tid] = a.rowoff[r];
    }
  }
  auto value = [&](int rr, int kk) -> float {
    float s = 0.f;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      if (t >= nterm) break;
      const float c = cf[t][kk];
      if (c != 0.f) {
        i64 off = cb[t][kk];
        if (rm)
          off += lab[0][rr] * cs[t][0][kk] + lab[1][rr] * cs[t][1][kk] + lab[2][rr] * cs[t][2][kk];
        else
          off += a.one_sel ? ro[rr] : a.rowoff[(i64)sl[t][kk] * a.R + r0 + rr];
        s = fmaf(c, __ldg(src + off), s);
      }
    }
    return s;
  };
  auto store = [&](int r, int k, float x) {
    const i64 o = (i64)r * a.Kpad + k;
    if constexpr (KIND == PANEL_BF16X2) {
      const __nv_bfloat16 hi = __float2bfloat16_rn(x);
      ((__nv_bfloat16*)a.out_hi)[o] = hi;
      ((__nv_bfloat16*)a.out_lo)[o] = __float2bfloat16_rn(x - __bfloat162float(hi));
    } else {
      const float hi = tf32_round(x);
      ((float*)a.out_hi)[o] = hi;
      ((float*)a.out_lo)[o] = tf32_round(x - hi);
    }
  };
  for (int k0 = kfirst; k0 < a.Kpad; k0 += kstep) {
    __syncthreads();
    if (tid < nterm * 32) {
      const int t = tid >> 5, kk = tid & 31, k = k0 + kk;
      const bool ok = k < a.K;
      const i64 idx = (i64)t * a.K + k;
      cb[t][kk] = ok ? a.colbase[idx] : 0;
      cf[t][kk] = ok ? (float)a.coef[idx] : 0.f;
      const int sel = ok ? a.sel[idx] : 0;
      sl[t][kk] = sel;
      if (rm) {
        const int v = a.lv;
        auto S = [&](int axis) { return axis == 0 ? v * v : (axis == 1 ? v : 1); };
        cs[t][0][kk] = rm == 2 ? S(sel / 3) : S(perm3(sel, 0));
        cs[t][1][kk] = rm == 2 ? S(sel % 3) : S(perm3(sel, 1));
        cs[t][2][kk] = rm == 2 ? 0 : S(perm3(sel, 2));
      }
    }
    __syncthreads();
    if (a.read_k_fast) {
      float x[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = (r0 + ty + 8 * j < a.R && k0 + tx < a.Kpad) ? value(ty + 8 * j, tx) : 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (r0 + ty + 8 * j < a.R && k0 + tx < a.Kpad) store(r0 + ty + 8 * j, k0 + tx, x[j]);
    } else {
      float x[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = (r0 + tx < a.R) ? value(tx, ty + 8 * j) : 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) tile[ty + 8 * j][tx] = x[j];
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = r0 + ty + 8 * j, k = k0 + tx;
        if (r < a.R && k < a.Kpad) store(r, k, tile[tx][ty + 8 * j]);
      }
    }
  }
}

template <bool F32>
__device__ __forceinline__ void pack_tiles_any(const PackArgs& a, int r0, int kfirst, int kstep) {
  if constexpr (F32) {
    if (a.nterm <= 1) {
      if (a.kind == PANEL_BF16X2) pack_tiles_f32<1, PANEL_BF16X2>(a, r0, kfirst, kstep);
      else pack_tiles_f32<1, PANEL_TF32X2>(a, r0, kfirst, kstep);
    } else {
      if (a.kind == PANEL_BF16X2) pack_tiles_f32<3, PANEL_BF16X2>(a, r0, kfirst, kstep);
      else pack_tiles_f32<3, PANEL_TF32X2>(a, r0, kfirst, kstep);
    }
  } else if (a.kind != PANEL_F64) {
    pack_tiles<true>(a, r0, kfirst, kstep);  // FP64 source into split panels
  } else {
    pack_tiles<false>(a, r0, kfirst, kstep);
  }
}

// One 32 x 32 tile per step; the tile's column tables (coefficient, base offset,
// selector of up to 3 terms) and, with a single selector, its 32 row offsets
// are staged in shared memory, so an element costs one source load.
template <bool F32>
__global__ void __launch_bounds__(256, 6) k_pack(PackArgs a) {
  pack_tiles_any<F32>(a, blockIdx.x * 32, blockIdx.y * 32, gridDim.y * 32);
}

void launch_pack(const PackArgs& a, cudaStream_t s) {
  // rows on grid x (up to 2^31 - 1 blocks); K on grid y, grid-strided past 65535
  const int gy = std::min((a.Kpad + 31) / 32, 65535);
  dim3 grid((a.R + 31) / 32, gy), block(32, 8);
  ++g_launch_count;
  if (a.src_f32 && a.kind != PANEL_F64)
    k_pack<true><<<grid, block, 0, s>>>(a);
  else
    k_pack<false><<<grid, block, 0, s>>>(a);
}

// Many gathers in one launch: block b packs one 32 x 32 tile of the gather p with
// tile0[p] <= b < tile0[p + 1] (row tiles outer, K tiles inner).  All gathers of
// one launch share the source type (F32: FP32 sources into split panels).
template <bool F32>
__global__ void __launch_bounds__(256, 6) k_pack_grouped(const PackArgs* __restrict__ list,
                                                      const int* __restrict__ tile0, int npack) {
  const int b = blockIdx.x;
  int lo = 0, hi = npack - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile0[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  const PackArgs a = list[lo];
  const int kt = (a.Kpad + 31) / 32;
  const int local = b - tile0[lo];
  pack_tiles_any<F32>(a, (local / kt) * 32, (local % kt) * 32, 1 << 30);
}

int pack_tiles_of(const PackArgs& a) { return ((a.R + 31) / 32) * ((a.Kpad + 31) / 32); }

void launch_pack_grouped(const PackArgs* list, const int* tile0, int npack, int total_tiles, int f32_src,
                         cudaStream_t s) {
  if (npack <= 0 || total_tiles <= 0) return;
  ++g_launch_count;
  if (f32_src)
    k_pack_grouped<true><<<total_tiles, dim3(32, 8), 0, s>>>(list, tile0, npack);
  else
    k_pack_grouped<false><<<total_tiles, dim3(32, 8), 0, s>>>(list, tile0, npack);
}

// ---------------------------------------------------------------------------
// Output-stationary reduction of the dense GEMM results into compact R3.
// Every contribution is a contiguous v^3 block X[x0][x1][x2] of a GEMM result
// whose axis q lands on stored axis pos[q] of its target block, with a weight.
// Block (cube, target) of the grid owns one 16^3 cube of one target block and
// sums all of that block's contributions in a fixed order (no atomics): per
// contribution, the permuted 16^3 cube of X is staged in shared memory with
// coalesced loads and added into registers; the cube is written once.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_r3_gather(const float* __restrict__ X, const i64* __restrict__ target,
                                                   const int* __restrict__ cstart, const i64* __restrict__ xoff,
                                                   const int* __restrict__ csel, const float* __restrict__ calpha,
                                                   int v, int accumulate, T* __restrict__ r3) {
  __shared__ float xs[16][17][17];  // odd outer strides: permuted reads stay below 2-way conflicts
  const int nc = (v + 15) / 16;
  const int cube = blockIdx.x, t = blockIdx.y;
  const int y0[3] = {(cube / (nc * nc)) * 16, ((cube / nc) % nc) * 16, (cube % nc) * 16};
  const i64 V2 = (i64)v * v;
  const int tb = threadIdx.x >> 4, tc = threadIdx.x & 15;  // output (b, c) of this thread; a loops
  float acc[16];
#pragma unroll
  for (int a = 0; a < 16; ++a) acc[a] = 0.f;
  const int c0 = cstart[t], c1 = cstart[t + 1];
  for (int c = c0; c < c1; ++c) {
    const int sel = csel[c];
    const int p0 = c_perm3[sel][0], p1 = c_perm3[sel][1], p2 = c_perm3[sel][2];
    const int xo0 = y0[p0], xo1 = y0[p1], xo2 = y0[p2];
    const float* xb = X + xoff[c];
    __syncthreads();
    float ld[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int x0 = xo0 + i, x1 = xo1 + tb, x2 = xo2 + tc;
      ld[i] = (x0 < v && x1 < v && x2 < v) ? __ldg(xb + x0 * V2 + (i64)x1 * v + x2) : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) xs[i][tb][tc] = ld[i];
    __syncthreads();
    const float al = calpha[c];
#pragma unroll
    for (int a = 0; a < 16; ++a) {
      const int yl[3] = {a, tb, tc};
      acc[a] = fmaf(al, xs[yl[p0]][yl[p1]][yl[p2]], acc[a]);
    }
  }
  T* out = r3 + target[t];
  const int yb = y0[1] + tb, yc = y0[2] + tc;
  if (yb >= v || yc >= v) return;
#pragma unroll
  for (int a = 0; a < 16; ++a) {
    const int ya = y0[0] + a;
    if (ya < v) {
      const i64 o = ya * V2 + (i64)yb * v + yc;
      out[o] = accumulate ? (T)(out[o] + (T)acc[a]) : (T)acc[a];
    }
  }
}

template <typename T>
void launch_r3_gather(const float* X, const i64* target, int ntarget, const int* cstart, const i64* xoff,
                      const int* csel, const float* calpha, int v, int accumulate, T* r3, cudaStream_t s) {
  if (ntarget <= 0) return;
  const int nc = (v + 15) / 16;
  ++g_launch_count;
  k_r3_gather<T><<<dim3(nc * nc * nc, ntarget), 256, 0, s>>>(X, target, cstart, xoff, csel, calpha, v, accumulate,
                                                             r3);
}
template void launch_r3_gather<float>(const float*, const i64*, int, const int*, const i64*, const int*, const float*,
                                      int, int, float*, cudaStream_t);
template void launch_r3_gather<double>(const float*, const i64*, int, const int*, const i64*, const int*,
                                       const float*, int, int, double*, cudaStream_t);

// ---------------------------------------------------------------------------
// FP64 GEMM, C[m, n] += alpha[m] * sum_k A[m, k] B[n, k]; A [M][lda], B [N][ldb]
// (k contiguous, zero padded to a multiple of 16).  64 x 64 tile, 4 x 4 per thread.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gemm_f64(const double* __restrict__ A,
                                                  const double* __restrict__ B, int K, int lda,
                                                  int ldb, EpiArgs e, int kz_len,
                                                  double* __restrict__ partial) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int lrow = tid >> 2, lk = (tid & 3) * 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int kbeg = blockIdx.z * kz_len;
  const int kend = min(K, kbeg + kz_len);
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    const int am = m0 + lrow, bn = n0 + lrow;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      As[lk + q][lrow] = am < e.M ? A[(i64)am * lda + k0 + lk + q] : 0.0;
      Bs[lk + q][lrow] = bn < e.N ? B[(i64)bn * ldb + k0 + lk + q] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= e.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= e.N) continue;
      if (partial)
        partial[((i64)blockIdx.z * e.M + m) * e.N + n] = acc[i][j];
      else
        epi_apply(e, m, n, acc[i][j]);
    }
  }
}

// Split-K reduction in a fixed order, then the scatter epilogue.
__global__ void k_splitk_reduce(const double* __restrict__ partial, int splitk, EpiArgs e) {
  const i64 MN = (i64)e.M * e.N;
  for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < MN; x += (i64)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splitk; ++z) s += partial[z * MN + x];
    epi_apply(e, (int)(x / e.N), (int)(x % e.N), s);
  }
}

// Launches with split-K when the output has few tiles and K is long; `scratch`
// (scratch_elems doubles) holds the partial tiles.  Deterministic in both paths.
void launch_gemm_f64(const double* A, const double* B, int K, int lda, int ldb, const EpiArgs& e,
                     double* scratch, i64 scratch_elems, cudaStream_t s) {
  // The FP64 pipe does about 2 FMA per clock per SM, so a GEMM is only fast when
  // every SM works on it: a grid below 2 x 152 tiles splits K (chunks of >= 32).
  const int tiles = ((e.N + 63) / 64) * ((e.M + 63) / 64);
  int splitk = 1;
  if (tiles < 304 && K >= 64 && scratch) {
    splitk = (608 + tiles - 1) / tiles;
    splitk = std::min(splitk, K / 32);
    const i64 MN = (i64)e.M * e.N;
    while (splitk > 1 && (i64)splitk * MN > scratch_elems) --splitk;
  }
  if (splitk <= 1) {
    dim3 grid((e.N + 63) / 64, (e.M + 63) / 64, 1);
    ++g_launch_count;
    k_gemm_f64<<<grid, 256, 0, s>>>(A, B, K, lda, ldb, e, K, nullptr);
    return;
  }
  const int kz = ((K + splitk - 1) / splitk + 15) / 16 * 16;
  splitk = (K + kz - 1) / kz;
  dim3 grid((e.N + 63) / 64, (e.M + 63) / 64, splitk);
  ++g_launch_count;
  k_gemm_f64<<<grid, 256, 0, s>>>(A, B, K, lda, ldb, e, kz, scratch);
  const i64 MN = (i64)e.M * e.N;
  i64 blocks = (MN + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  ++g_launch_count;
  k_splitk_reduce<<<(unsigned)blocks, 256, 0, s>>>(scratch, splitk, e);
}

// ---------------------------------------------------------------------------
// Dense permuted linear combination.
// ---------------------------------------------------------------------------
template <bool FAST>
__global__ void k_combine(CombineArgs c) {
  const i64 total = c.total;
  for (i64 idx = blockIdx.x * (i64)blockDim.x + threadIdx.x; idx < total;
       idx += (i64)gridDim.x * blockDim.x) {
    i64 ooff = 0;
    i64 ioff[4] = {0, 0, 0, 0};
    if constexpr (FAST) {
      unsigned rem = (unsigned)idx;
#pragma unroll
      for (int d = 5; d >= 0; --d) {
        if (d >= c.rank) continue;
        const unsigned q = (__umulhi(c.fdm[d], rem) + rem) >> c.fdl[d];
        const i64 x = (i64)(rem - q * (unsigned)c.shape[d]);
        rem = q;
        ooff += x * c.ostride[d];
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (t < c.nterm) ioff[t] += x * c.istride[t][d];
      }
    } else {
      i64 rem = idx;
      for (int d = c.rank - 1; d >= 0; --d) {
        const i64 x = rem % c.shape[d];
        rem /= c.shape[d];
        ooff += x * c.ostride[d];
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (t < c.nterm) ioff[t] += x * c.istride[t][d];
      }
    }
    if (c.beta == 0.0 && c.nterm == 1 && c.coef[0] == 1.0) {  // a permuted copy: no FP64 arithmetic
      c.out[ooff] = c.in[0][ioff[0]];
      continue;
    }
    double s = c.beta == 0.0 ? 0.0 : c.beta * c.out[ooff];
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (t < c.nterm) s += c.coef[t] * c.in[t][ioff[t]];
    c.out[ooff] = s;
  }
}

void launch_combine(const CombineArgs& c0, cudaStream_t s) {
  if (c0.total <= 0) return;
  CombineArgs c = c0;
  const bool fast = c.total < (1LL << 31);
  if (fast) {
    // divisor d < 2^31: l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1 < 2^32;
    // then n / d = (umulhi(m, n) + n) >> l for every n < 2^31
    for (int d = 0; d < c.rank; ++d) {
      const unsigned long long dv = (unsigned long long)c.shape[d];
      int l = 0;
      while ((1ULL << l) < dv) ++l;
      c.fdl[d] = l;
      c.fdm[d] = (unsigned)(((1ULL << 32) * ((1ULL << l) - dv)) / dv + 1);
    }
  }
  i64 blocks = (c.total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  ++g_launch_count;
  if (fast)
    k_combine<true><<<(unsigned)blocks, 256, 0, s>>>(c);
  else
    k_combine<false><<<(unsigned)blocks, 256, 0, s>>>(c);
}

// ---------------------------------------------------------------------------
// R3 post-processing: rp[blk] = post(r[blk]) (symmetrise, purify, orthogonalise).
// Every element needs its six virtual permutations, which lie in the six cubes
// of one orbit of 8^3 tiles {(TA,TB,TC) permuted}.  One CTA takes one orbit of
// one block at a time: it loads the orbit's distinct cubes (1, 3 or 6) into shared
// memory along the unit-stride axis (each thread two rows of every cube, all loads
// issued before the first store).  Each thread then reads the six values of the
// element orbits of its two elements of cube 0 once, forms all six outputs of each
// orbit (one mean, the block's column-swap average) and writes them back into the
// cubes, one writer per element; the cubes are then stored along the unit-stride
// axis -- one HBM read and one write per element, about four shared-memory accesses
// per element (seven when every output read its six permutations).  Small cubes
// keep six CTAs on an SM, so one CTA's loads overlap another's stores.  The squared
// norm of each block is summed in the storage type per thread and in FP64 across
// blocks and threads.
// ---------------------------------------------------------------------------
constexpr int kPostTL = 8;

__device__ __forceinline__ double block_sum(double x);
__global__ void k_sum(const double* __restrict__ partial, int np, double* __restrict__ out, double scale,
                      int accumulate);

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 4) k_post(const T* __restrict__ r, T* __restrict__ rp,
                                              const int4* __restrict__ blocks, int v, i64 n3,
                                              const double* __restrict__ wblk, double* __restrict__ partial) {
  constexpr int TL = kPostTL;
  // [8][9][9]: odd strides on both outer axes keep the permuted reads within 2-way bank conflicts
  typedef T Cube[TL][TL + 1][TL + 1];
  extern __shared__ __align__(16) unsigned char post_smem[];
  Cube* cube = reinterpret_cast<Cube*>(post_smem);
  __shared__ int tcoord[6][3];
  __shared__ int slot[6][6];
  __shared__ bool first[6];
  __shared__ int ncube;
  const i64 V2 = (i64)v * v, V3 = V2 * v;
  // orbit index -> sorted tile triple (TA <= TB <= TC), colex like the blocks; the
  // orbit's distinct cubes and, per cube and label permutation, the cube holding it
  if (threadIdx.x == 0) {
    int rem = blockIdx.x, tc = 0;
    while ((tc + 1) * (tc + 2) * (tc + 3) / 6 <= rem) ++tc;
    rem -= tc * (tc + 1) * (tc + 2) / 6;
    int tb = 0;
    while ((tb + 1) * (tb + 2) / 2 <= rem) ++tb;
    const int T0[3] = {rem - tb * (tb + 1) / 2, tb, tc};
    int n = 0;
    for (int q = 0; q < 6; ++q) {
      const int x = T0[c_perm3[q][0]], y = T0[c_perm3[q][1]], z = T0[c_perm3[q][2]];
      bool dup = false;
      for (int k = 0; k < n; ++k) dup |= tcoord[k][0] == x && tcoord[k][1] == y && tcoord[k][2] == z;
      if (!dup) {
        tcoord[n][0] = x;
        tcoord[n][1] = y;
        tcoord[n][2] = z;
        ++n;
      }
    }
    ncube = n;
  }
  __syncthreads();
  if (threadIdx.x < 36) {
    const int k = threadIdx.x / 6, q = threadIdx.x % 6;
    if (k < ncube) {
      const int x = tcoord[k][c_perm3[q][0]], y = tcoord[k][c_perm3[q][1]], z = tcoord[k][c_perm3[q][2]];
      for (int k2 = 0; k2 < ncube; ++k2)
        if (tcoord[k2][0] == x && tcoord[k2][1] == y && tcoord[k2][2] == z) slot[k][q] = k2;
    }
  }
  if (threadIdx.x < 6) {  // q is the first label permutation of cube 0 that lands in its cube
    bool f = true;
    for (int q2 = 0; q2 < (int)threadIdx.x; ++q2) f = f && slot[0][q2] != slot[0][threadIdx.x];
    first[threadIdx.x] = f;
  }
  __syncthreads();
  const int n = ncube;
  // thread (xg, ty, tz): rows x = xg and xg + 4 of every cube, local (ty, tz) along them
  const int tz = threadIdx.x & 7, ty = (threadIdx.x >> 3) & 7, xg = threadIdx.x >> 6;
  // sum over this CTA's outputs of m(blk) val^2 (the |R3|^2 share), in the storage
  // type across its blocks (FP32 storage: no per-block FP64 work)
  T nrm = (T)0;
  for (i64 b = blockIdx.y; b < n3; b += gridDim.y) {
    const T wb = (T)wblk[b];
    const int4 ijk = blocks[b];
    const T* rb = r + b * V3;
    T ld[6][2];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int kk = k < n ? k : 0;
      const int x0 = tcoord[kk][0] * TL + xg, gy = tcoord[kk][1] * TL + ty, gz = tcoord[kk][2] * TL + tz;
      const bool in = k < n && gy < v && gz < v;
      const T* src = rb + (i64)gy * v + gz;
#pragma unroll
      for (int h = 0; h < 2; ++h) ld[k][h] = (in && x0 + 4 * h < v) ? src[(i64)(x0 + 4 * h) * V2] : (T)0;
    }
    __syncthreads();  // the previous block's cubes are consumed
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (k < n) {
        cube[k][xg][ty][tz] = ld[k][0];
        cube[k][xg + 4][ty][tz] = ld[k][1];
      }
    __syncthreads();
    T* out = rp + b * V3;
    const bool all_eq = ijk.x == ijk.y && ijk.y == ijk.z;
    if (!all_eq) {
      // the orbit of element e = (x, ty, tz) of cube 0: v[q] = R(e o perm_q) lies in
      // cube slot[0][q] at e's local coordinates permuted by q
      const int s1 = slot[0][1], s2 = slot[0][2], s3 = slot[0][3], s4 = slot[0][4], s5 = slot[0][5];
      T vv[2][6];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int x = xg + 4 * h;
        vv[h][0] = cube[0][x][ty][tz];
        vv[h][1] = cube[s1][x][tz][ty];
        vv[h][2] = cube[s2][ty][x][tz];
        vv[h][3] = cube[s3][ty][tz][x];
        vv[h][4] = cube[s4][tz][x][ty];
        vv[h][5] = cube[s5][tz][ty][x];
      }
      __syncthreads();  // every orbit read before the outputs overwrite the cubes
      // out(e o q) = sym(e o q) - mean over the orbit; sym averages e o q with its
      // image under the block's column swap (positions 0 1 for i = j, 1 2 for j = k)
      const int mode = ijk.x == ijk.y ? 1 : (ijk.y == ijk.z ? 2 : 0);
      constexpr int kS01[6] = {2, 4, 0, 5, 1, 3}, kS12[6] = {1, 0, 3, 2, 5, 4};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int x = xg + 4 * h;
        const T* w = vv[h];
        const T mean = (w[0] + w[1] + w[2] + w[3] + w[4] + w[5]) * (T)(1.0 / 6.0);
        T o6[6];
#pragma unroll
        for (int qq = 0; qq < 6; ++qq)
          o6[qq] = (mode == 1 ? (T)0.5 * (w[qq] + w[kS01[qq]])
                              : (mode == 2 ? (T)0.5 * (w[qq] + w[kS12[qq]]) : w[qq])) - mean;
        // one writer per output: cube slot[0][q] is written through its first q
        if (first[0]) cube[0][x][ty][tz] = o6[0];
        if (first[1]) cube[s1][x][tz][ty] = o6[1];
        if (first[2]) cube[s2][ty][x][tz] = o6[2];
        if (first[3]) cube[s3][ty][tz][x] = o6[3];
        if (first[4]) cube[s4][tz][x][ty] = o6[4];
        if (first[5]) cube[s5][tz][ty][x] = o6[5];
      }
      __syncthreads();
    }
    T bs = (T)0;
    for (int k = 0; k < n; ++k) {
      const int gy = tcoord[k][1] * TL + ty, gz = tcoord[k][2] * TL + tz;
      if (gy >= v || gz >= v) continue;
      T* dst = out + (i64)gy * v + gz;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int x = xg + 4 * h, gx = tcoord[k][0] * TL + x;
        if (gx >= v) break;
        const T val = all_eq ? (T)0 : cube[k][x][ty][tz];
        dst[(i64)gx * V2] = val;
        bs += val * val;
      }
    }
    nrm += wb * bs;
  }
  const double tot = block_sum((double)nrm);
  if (threadIdx.x == 0) partial[(i64)blockIdx.y * gridDim.x + blockIdx.x] = tot;
}

// about 64 CTAs per SM in all (six resident at a time); each keeps its orbit tables
// across the blocks it visits
static i64 post_grid_y(int norb, i64 n3) {
  return std::max<i64>(1, std::min<i64>(n3, (152 * 8 * 8 + norb - 1) / norb));
}

int post_partials(int v, i64 n3) {
  const int nt = (v + kPostTL - 1) / kPostTL;
  const int norb = nt * (nt + 1) * (nt + 2) / 6;
  return (int)(norb * post_grid_y(norb, n3));
}

template <typename T>
void launch_post(const T* r, T* rp, const int4* blocks, int v, i64 n3, const double* wblk, double* partial,
                 double* norm2, cudaStream_t s) {
  if (n3 <= 0) return;
  const int nt = (v + kPostTL - 1) / kPostTL;
  const int norb = nt * (nt + 1) * (nt + 2) / 6;
  const i64 gy = post_grid_y(norb, n3);
  const size_t smem = 6 * sizeof(T) * kPostTL * (kPostTL + 1) * (kPostTL + 1);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_post<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  ++g_launch_count;
  k_post<T><<<dim3((unsigned)norb, (unsigned)gy), 256, smem, s>>>(r, rp, blocks, v, n3, wblk, partial);
  ++g_launch_count;
  k_sum<<<1, 256, 0, s>>>(partial, norb * (int)gy, norm2, 1.0, 0);
}
template void launch_post<double>(const double*, double*, const int4*, int, i64, const double*, double*, double*,
                                  cudaStream_t);
template void launch_post<float>(const float*, float*, const int4*, int, i64, const double*, double*, double*,
                                 cudaStream_t);

// ---------------------------------------------------------------------------
// Jacobi updates with the bare Fock diagonal (orbital energies e[0..n)).
// ---------------------------------------------------------------------------
__global__ void k_update_t1(double* t1, const double* r1, const double* e, int o, int v, double shift) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= o * v) return;
  const int i = idx / v, a = idx % v;
  t1[idx] += r1[idx] / (e[i] - e[o + a] - shift);
}

__global__ void k_update_t2(double* t2, const double* r2, const double* e, int o, int v, double shift) {
  const i64 n = (i64)o * o * v * v;
  for (i64 idx = blockIdx.x * (i64)blockDim.x + threadIdx.x; idx < n; idx += (i64)gridDim.x * blockDim.x) {
    const int b = (int)(idx % v), a = (int)((idx / v) % v);
    const int j = (int)((idx / ((i64)v * v)) % o), i = (int)(idx / ((i64)v * v * o));
    t2[idx] += r2[idx] / (e[i] + e[j] - e[o + a] - e[o + b] - shift);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_update_t3(T* __restrict__ t3, const T* __restrict__ rp3,
                                                   const double* __restrict__ e, const int4* __restrict__ blocks,
                                                   int o, int v, double shift) {
  // block (a, blk): the slab t3[blk][a][:][:], threads 32 along c x 8 along b.
  // The denominator is assembled in FP64; the step r / eps is taken in the
  // storage precision of T3 (FP32 storage: FP32 division, as precise as the store)
  const int a = blockIdx.x;
  const i64 b = blockIdx.y;
  const int4 ijk = blocks[b];
  const double ea = e[ijk.x] + e[ijk.y] + e[ijk.z] - e[o + a] - shift;
  const i64 V2 = (i64)v * v;
  T* tb = t3 + (b * v + a) * V2;
  const T* rb = rp3 + (b * v + a) * V2;
  if constexpr (sizeof(T) == 4) {
    // FP32 storage: the FP64 row parts e_ijk - e_a - e_b and the e_c are carried as
    // float pairs (hi + lo) in shared memory, so the FP32 denominator is the FP64
    // one rounded once, without FP64 arithmetic per element
    extern __shared__ float upd_smem[];  // 4 v floats (launch_update_t3)
    float *rh = upd_smem, *rl = rh + v, *ch = rl + v, *cl = ch + v;
    for (int q = threadIdx.y * 32 + threadIdx.x; q < v; q += 256) {
      const double eab = ea - e[o + q], ec = e[o + q];
      rh[q] = (float)eab;
      rl[q] = (float)(eab - (double)rh[q]);
      ch[q] = (float)ec;
      cl[q] = (float)(ec - (double)ch[q]);
    }
    __syncthreads();
    for (int bb = threadIdx.y; bb < v; bb += 8) {
      const float eh = rh[bb], el = rl[bb];
      for (int c = threadIdx.x; c < v; c += 32) {
        const int idx = bb * v + c;
        const float d = (eh - ch[c]) + (el - cl[c]);
        tb[idx] = tb[idx] + rb[idx] / d;
      }
    }
  } else {
    for (int bb = threadIdx.y; bb < v; bb += 8) {
      const double eab = ea - e[o + bb];
      for (int c = threadIdx.x; c < v; c += 32) {
        const int idx = bb * v + c;
        const T d = (T)(eab - e[o + c]);
        tb[idx] = tb[idx] + rb[idx] / d;
      }
    }
  }
}

void launch_update_t12(double* t1, const double* r1, double* t2, const double* r2, const double* e,
                       int o, int v, double shift, cudaStream_t s) {
  ++g_launch_count;
  k_update_t1<<<(o * v + 255) / 256, 256, 0, s>>>(t1, r1, e, o, v, shift);
  const i64 n = (i64)o * o * v * v;
  i64 blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  ++g_launch_count;
  k_update_t2<<<(unsigned)blocks, 256, 0, s>>>(t2, r2, e, o, v, shift);
}

template <typename T>
void launch_update_t3(T* t3, const T* rp3, const double* e, const int4* blocks, int o, int v, i64 n3,
                      double shift, cudaStream_t s) {
  if (n3 <= 0) return;
  ++g_launch_count;
  const size_t smem = sizeof(T) == 4 ? (size_t)16 * v : 0;
  static bool attr = false;
  if (!attr) {  // v up to 4096: 64 KB of float pairs
    cudaFuncSetAttribute(k_update_t3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 16 * 4096);
    attr = true;
  }
  k_update_t3<T><<<dim3((unsigned)v, (unsigned)n3), dim3(32, 8), smem, s>>>(t3, rp3, e, blocks, o, v, shift);
}
template void launch_update_t3<double>(double*, const double*, const double*, const int4*, int, int,
                                       i64, double, cudaStream_t);
template void launch_update_t3<float>(float*, const float*, const double*, const int4*, int, int, i64,
                                      double, cudaStream_t);

// ---------------------------------------------------------------------------
// Deterministic weighted dot products: sum_i x[i] y[i] w[i / seg] (w NULL = 1).
// Stage 1 writes one partial per block (fixed grid), stage 2 sums in order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ double block_sum(double x) {
  __shared__ double ws[32];
  x = warp_sum(x);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    x = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
    x = warp_sum(x);
  }
  return x;
}

// Piece p of the weighted sum: with w, segment p / P, part p % P of P equal parts
// (P pieces per segment, so that every block of the fixed grid has work even with
// few long segments); without w, a grid-stride slice.
struct Pieces {
  i64 n, seg, nseg, len;
  int P;
};
__host__ __device__ inline Pieces make_pieces(i64 n, i64 seg, bool weighted, int grid) {
  Pieces q;
  q.n = n;
  q.seg = weighted ? seg : n;
  q.nseg = weighted ? (n + seg - 1) / seg : 1;
  // about 16 pieces per block (balanced tail), each of at least 2048 elements
  i64 per = (16LL * grid + q.nseg - 1) / q.nseg;
  const i64 cap = (q.seg + 2047) / 2048;
  if (per > cap) per = cap;
  q.P = (int)(per < 1 ? 1 : per);
  q.len = ((q.seg + q.P - 1) / q.P + 3) & ~(i64)3;  // a multiple of 4 (vector loads)
  return q;
}

// sum_i x[i] y[i] over [b0, b1) by this block's threads, four loads in flight each.
// FP32 data: products and runs of 32 terms are summed in FP32 and every run is
// added to an FP64 total (the FP64 pipe of this part does about 2 operations per
// clock per SM, too few for one conversion and FMA per element).
template <typename T>
__device__ __forceinline__ double dot_range(const T* __restrict__ x, const T* __restrict__ y, i64 b0, i64 b1) {
  const i64 step = blockDim.x;
  i64 i = b0 + threadIdx.x;
  if constexpr (sizeof(T) == 4) {
    double tot = 0.0;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int run = 0;
    for (; i + 3 * step < b1; i += 4 * step) {
      const float x0 = x[i], x1 = x[i + step], x2 = x[i + 2 * step], x3 = x[i + 3 * step];
      const float y0 = y[i], y1 = y[i + step], y2 = y[i + 2 * step], y3 = y[i + 3 * step];
      s0 = fmaf(x0, y0, s0);
      s1 = fmaf(x1, y1, s1);
      s2 = fmaf(x2, y2, s2);
      s3 = fmaf(x3, y3, s3);
      if (++run == 8) {
        tot += (double)((s0 + s1) + (s2 + s3));
        s0 = s1 = s2 = s3 = 0.f;
        run = 0;
      }
    }
    for (; i < b1; i += step) s0 = fmaf((float)x[i], (float)y[i], s0);
    return tot + (double)((s0 + s1) + (s2 + s3));
  } else {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (; i + 3 * step < b1; i += 4 * step) {
      const T x0 = x[i], x1 = x[i + step], x2 = x[i + 2 * step], x3 = x[i + 3 * step];
      const T y0 = y[i], y1 = y[i + step], y2 = y[i + 2 * step], y3 = y[i + 3 * step];
      s0 += (double)x0 * (double)y0;
      s1 += (double)x1 * (double)y1;
      s2 += (double)x2 * (double)y2;
      s3 += (double)x3 * (double)y3;
    }
    for (; i < b1; i += step) s0 += (double)x[i] * (double)y[i];
    return (s0 + s1) + (s2 + s3);
  }
}

template <typename T>
__global__ void k_wdot(const T* __restrict__ x, const T* __restrict__ y, i64 n, i64 seg,
                       const double* __restrict__ w, double* __restrict__ partial) {
  const Pieces pc = make_pieces(n, seg, w != nullptr, gridDim.x);
  double s = 0.0;
  for (i64 p = blockIdx.x; p < pc.nseg * pc.P; p += gridDim.x) {
    const i64 sg = p / pc.P, part = p % pc.P;
    const i64 b0 = sg * pc.seg + part * pc.len;
    i64 b1 = b0 + pc.len;
    const i64 send = sg * pc.seg + pc.seg < n ? sg * pc.seg + pc.seg : n;
    if (b1 > send) b1 = send;
    s += (w ? w[sg] : 1.0) * dot_range<T>(x, y, b0, b1);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_sum(const double* __restrict__ partial, int np, double* __restrict__ out, double scale,
                      int accumulate) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = (accumulate ? *out : 0.0) + scale * s;
}

template <typename T>
void launch_wdot(const T* x, const T* y, i64 n, i64 seg, const double* w, double* partial,
                 double* out, double scale, int accumulate, cudaStream_t s) {
  ++g_launch_count;
  k_wdot<T><<<kDotBlocks, 256, 0, s>>>(x, y, n, seg, w, partial);
  ++g_launch_count;
  k_sum<<<1, 256, 0, s>>>(partial, kDotBlocks, out, scale, accumulate);
}
template void launch_wdot<double>(const double*, const double*, i64, i64, const double*, double*,
                                  double*, double, int, cudaStream_t);
template void launch_wdot<float>(const float*, const float*, i64, i64, const double*, double*, double*,
                                 double, int, cudaStream_t);

// ---------------------------------------------------------------------------
// DIIS (Sec. III.A.5) with its bookkeeping on the device, so one iteration is a
// fixed sequence of launches (capturable in a CUDA graph).  State st[8]:
//   st[0] updates done, st[1] history entries written, st[2] slot of the current
//   update, st[3] entries in use after it, st[4] 1 if this update extrapolates.
// History slot q of a segment starts at base + q * stride + off (bytes).
// ---------------------------------------------------------------------------
__global__ void k_diis_begin(int* st, int M, int diis_start) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int iter = st[0] + 1, count = st[1];
  st[0] = iter;
  st[2] = count % M;
  st[1] = count + 1;
  st[3] = count + 1 < M ? count + 1 : M;
  st[4] = (iter >= diis_start && st[3] >= 2) ? 1 : 0;
}

void launch_diis_begin(int* st, int M, int diis_start, cudaStream_t s) {
  ++g_launch_count;
  k_diis_begin<<<1, 32, 0, s>>>(st, M, diis_start);
}

static unsigned ew_blocks(i64 n) {
  i64 blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  return (unsigned)blocks;
}

// slot[st[2]] = src (the amplitudes before the Jacobi step)
template <typename T>
__global__ void k_slot_save(char* __restrict__ base, i64 stride, i64 off, const int* __restrict__ st,
                            const T* __restrict__ src, i64 n) {
  T* dst = (T*)(base + (i64)st[2] * stride + off);
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) dst[i] = src[i];
}

template <typename T>
void launch_slot_save(char* base, i64 stride, i64 off, const int* st, const T* src, i64 n, cudaStream_t s) {
  if (n <= 0) return;
  ++g_launch_count;
  k_slot_save<T><<<ew_blocks(n), 256, 0, s>>>(base, stride, off, st, src, n);
}
template void launch_slot_save<double>(char*, i64, i64, const int*, const double*, i64, cudaStream_t);
template void launch_slot_save<float>(char*, i64, i64, const int*, const float*, i64, cudaStream_t);

// Virtual subspace of compact T3 (the T3 part of the DIIS vectors restricted to the
// first ns virtual orbitals, the lowest in energy): sub[blk][a][b][c] <-> t3[blk][a][b][c]
// for a, b, c < ns.  dir 0 gathers t3 -> sub, dir 1 scatters sub -> t3.
// Vector variant (FP32, ns and v multiples of 4): float4 units, four of them in flight
// per thread, one division per unit.
__global__ void k_subcube4(float* __restrict__ t3, float* __restrict__ sub, i64 n3, int v, int ns, int dir) {
  const int q4 = ns / 4;
  const i64 V3 = (i64)v * v * v, n4 = n3 * ns * ns * q4;
  const i64 step = (i64)gridDim.x * blockDim.x;
  for (i64 i0 = blockIdx.x * (i64)blockDim.x + threadIdx.x; i0 < n4; i0 += 4 * step) {
    float4* fp[4];
    float4* sp[4];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const i64 i = i0 + u * step;
      ok[u] = i < n4;
      const i64 row = ok[u] ? i / q4 : 0;
      const int c4 = (int)(i - row * q4);
      const i64 blk = row / ((i64)ns * ns);
      const int ab = (int)(row - blk * ns * ns), a = ab / ns, b = ab - a * ns;
      fp[u] = reinterpret_cast<float4*>(t3 + blk * V3 + ((i64)a * v + b) * v) + c4;
      sp[u] = reinterpret_cast<float4*>(sub) + i;
    }
    float4 x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (ok[u]) x[u] = dir == 0 ? *fp[u] : *sp[u];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (ok[u]) {
        if (dir == 0) *sp[u] = x[u];
        else *fp[u] = x[u];
      }
  }
}

template <typename T>
__global__ void k_subcube(T* __restrict__ t3, T* __restrict__ sub, i64 n3, int v, int ns, int dir) {
  // rows (blk, a, b) of ns contiguous values in both layouts: no division per element
  const i64 V3 = (i64)v * v * v, nrow = n3 * ns * ns;
  for (i64 row = blockIdx.x; row < nrow; row += gridDim.x) {
    const i64 blk = row / ((i64)ns * ns);
    const int ab = (int)(row - blk * ns * ns), a = ab / ns, b = ab - a * ns;
    T* full = t3 + blk * V3 + ((i64)a * v + b) * v;
    T* s = sub + row * ns;
    for (int c = threadIdx.x; c < ns; c += blockDim.x) {
      if (dir == 0) s[c] = full[c];
      else full[c] = s[c];
    }
  }
}

template <typename T>
void launch_subcube(T* t3, T* sub, i64 n3, int v, int ns, int dir, cudaStream_t s) {
  const i64 nrow = n3 * ns * ns;
  if (nrow <= 0) return;
  ++g_launch_count;
  if (sizeof(T) == 4 && ns % 4 == 0 && v % 4 == 0) {
    const i64 n4 = nrow * (ns / 4);
    const i64 blocks = std::min<i64>((n4 + 1023) / 1024, (i64)152 * 16);
    k_subcube4<<<(unsigned)blocks, 256, 0, s>>>((float*)t3, (float*)sub, n3, v, ns, dir);
    return;
  }
  const int threads = ns <= 64 ? 64 : 128;
  const i64 blocks = std::min<i64>(nrow, (i64)152 * 64);
  k_subcube<T><<<(unsigned)blocks, threads, 0, s>>>(t3, sub, n3, v, ns, dir);
}
template void launch_subcube<double>(double*, double*, i64, int, int, int, cudaStream_t);
template void launch_subcube<float>(float*, float*, i64, int, int, int, cudaStream_t);

// error slot: e = t - e (new minus old); amplitude slot: t
template <typename T>
__global__ void k_slot_diff_store(char* __restrict__ hist_t, char* __restrict__ hist_e, i64 stride, i64 off,
                                  const int* __restrict__ st, const T* __restrict__ t, i64 n) {
  const i64 o = (i64)st[2] * stride + off;
  T* ts = (T*)(hist_t + o);
  T* es = (T*)(hist_e + o);
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    const T x = t[i];
    es[i] = x - es[i];
    ts[i] = x;
  }
}

template <typename T>
void launch_slot_diff_store(char* hist_t, char* hist_e, i64 stride, i64 off, const int* st, const T* t, i64 n,
                            cudaStream_t s) {
  if (n <= 0) return;
  ++g_launch_count;
  k_slot_diff_store<T><<<ew_blocks(n), 256, 0, s>>>(hist_t, hist_e, stride, off, st, t, n);
}
template void launch_slot_diff_store<double>(char*, char*, i64, i64, const int*, const double*, i64, cudaStream_t);
template void launch_slot_diff_store<float>(char*, char*, i64, i64, const int*, const float*, i64, cudaStream_t);

// partial[q][block] = sum_x w(x) e_s[x] e_q[x] for q < st[3] (0 otherwise); weights
// per segment of `seg` elements when w is given.  One pass: e_s is read once and
// every e_q once.  Fixed grid and pieces: deterministic.
template <typename T>
__global__ void k_diis_dots(const char* __restrict__ hist_e, i64 stride, i64 off, const int* __restrict__ st, int M,
                            i64 n, i64 seg, const double* __restrict__ w, double* __restrict__ partial) {
  const int m = st[3];
  const T* es = (const T*)(hist_e + (i64)st[2] * stride + off);
  const Pieces pc = make_pieces(n, seg, w != nullptr, gridDim.x);
  double s[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) s[q] = 0.0;
  for (i64 p = blockIdx.x; p < pc.nseg * pc.P; p += gridDim.x) {
    const i64 sg = p / pc.P, part = p % pc.P;
    const i64 b0 = sg * pc.seg + part * pc.len;
    i64 b1 = b0 + pc.len;
    const i64 send = sg * pc.seg + pc.seg < n ? sg * pc.seg + pc.seg : n;
    if (b1 > send) b1 = send;
    const double wt = w ? w[sg] : 1.0;
    if constexpr (sizeof(T) == 4) {
      // runs of 64 terms per thread in FP32, each run added (weighted) to the FP64
      // sums of the m live slots: the FP64 units run at a small fraction of the FP32
      // rate on this part.  16-byte aligned data: four elements per load.
      float fs[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) fs[q] = 0.f;
      auto flush = [&]() {
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (q < m) {
            s[q] += wt * (double)fs[q];
            fs[q] = 0.f;
          }
      };
      const bool vec = (((uintptr_t)(hist_e + off)) & 15) == 0 && (stride & 15) == 0 && (b0 & 3) == 0 && (b1 & 3) == 0;
      int run = 0;
      if (vec) {
        for (i64 i = b0 + 4 * (i64)threadIdx.x; i < b1; i += 4 * (i64)blockDim.x) {
          const float4 x = *reinterpret_cast<const float4*>(es + i);
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (q < m) {
              const float4 y = *reinterpret_cast<const float4*>((const float*)(hist_e + (i64)q * stride + off) + i);
              fs[q] = fmaf(x.x, y.x, fs[q]);
              fs[q] = fmaf(x.y, y.y, fs[q]);
              fs[q] = fmaf(x.z, y.z, fs[q]);
              fs[q] = fmaf(x.w, y.w, fs[q]);
            }
          if (++run == 16) {
            flush();
            run = 0;
          }
        }
      } else {
        for (i64 i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
          const float x = es[i];
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (q < m) fs[q] = fmaf(x, ((const float*)(hist_e + (i64)q * stride + off))[i], fs[q]);
          if (++run == 64) {
            flush();
            run = 0;
          }
        }
      }
      flush();
    } else {
      double ss[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) ss[q] = 0.0;
      for (i64 i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const double x = (double)es[i];
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (q < m) ss[q] += x * (double)((const T*)(hist_e + (i64)q * stride + off))[i];
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) s[q] += wt * ss[q];
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    if (q >= M) break;  // M is uniform over the block
    const double t = block_sum(q < m ? s[q] : 0.0);
    if (threadIdx.x == 0) partial[(i64)q * gridDim.x + blockIdx.x] = t;
  }
}

template <typename T>
void launch_diis_dots(const char* hist_e, i64 stride, i64 off, const int* st, int M, i64 n, i64 seg, const double* w,
                      double* partial, cudaStream_t s) {
  ++g_launch_count;
  k_diis_dots<T><<<kDotBlocks, 256, 0, s>>>(hist_e, stride, off, st, M, n, seg, w, partial);
}
template void launch_diis_dots<double>(const char*, i64, i64, const int*, int, i64, i64, const double*, double*,
                                       cudaStream_t);
template void launch_diis_dots<float>(const char*, i64, i64, const int*, int, i64, i64, const double*, double*,
                                      cudaStream_t);

// B[s][q] = B[q][s] = sum over the nseg segment partials (fixed order); block q.
__global__ void k_diis_row(const double* __restrict__ partial, int nseg, const int* __restrict__ st, int M,
                           double* __restrict__ B) {
  const int q = blockIdx.x, slot = st[2];
  if (q >= st[3]) return;
  double tot = 0.0;
  for (int g = 0; g < nseg; ++g) {
    const double* p = partial + ((i64)g * M + q) * kDotBlocks;
    double s = 0.0;
    for (int i = threadIdx.x; i < kDotBlocks; i += blockDim.x) s += p[i];
    s = block_sum(s);
    tot += s;  // meaningful in thread 0
  }
  if (threadIdx.x == 0) {
    B[slot * M + q] = tot;
    B[q * M + slot] = tot;
  }
}

void launch_diis_row(const double* partial, int nseg, const int* st, int M, double* B, cudaStream_t s) {
  ++g_launch_count;
  k_diis_row<<<M, 256, 0, s>>>(partial, nseg, st, M, B);
}

// Bordered solve [B 1; 1 0] [c; lambda] = [0; 1] over the st[3] entries in use by
// partial-pivoting Gaussian elimination; a pivot below 1e-14 of max|B| drops that
// direction (coefficient 0), the least-squares limit for a singular B.  Runs only
// when st[4] is set.
__global__ void k_diis_solve(const double* __restrict__ Bmat, const int* __restrict__ st, int ld,
                             double* __restrict__ coef) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || !st[4]) return;
  const int m = st[3];
  double A[17][18];
  const int n = m + 1;
  double scale = 0.0;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) scale = fmax(scale, fabs(Bmat[i * ld + j]));
  if (scale == 0.0) scale = 1.0;
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      double x;
      if (i < m && j < m) x = Bmat[i * ld + j] / scale;
      else if (i == m && j == m) x = 0.0;
      else x = 1.0;
      A[i][j] = x;
    }
    A[i][n] = (i == m) ? 1.0 : 0.0;
  }
  int piv_ok[17];
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int i = c + 1; i < n; ++i)
      if (fabs(A[i][c]) > fabs(A[p][c])) p = i;
    if (p != c)
      for (int j = 0; j <= n; ++j) { double t = A[c][j]; A[c][j] = A[p][j]; A[p][j] = t; }
    piv_ok[c] = fabs(A[c][c]) > 1e-14;
    if (!piv_ok[c]) continue;
    for (int i = c + 1; i < n; ++i) {
      const double f = A[i][c] / A[c][c];
      for (int j = c; j <= n; ++j) A[i][j] -= f * A[c][j];
    }
  }
  double x[17];
  for (int c = n - 1; c >= 0; --c) {
    if (!piv_ok[c]) { x[c] = 0.0; continue; }
    double s = A[c][n];
    for (int j = c + 1; j < n; ++j) s -= A[c][j] * x[j];
    x[c] = s / A[c][c];
  }
  for (int i = 0; i < m; ++i) coef[i] = x[i];
}

void launch_diis_solve(const double* B, const int* st, int ld, double* coef, cudaStream_t s) {
  ++g_launch_count;
  k_diis_solve<<<1, 32, 0, s>>>(B, st, ld, coef);
}

// out[i] = sum_q coef[q] * hist[q][i] over the st[3] entries (hist slots `stride`
// elements apart); runs only when st[4] is set.
template <typename T>
__global__ void k_diis_extrapolate(T* __restrict__ out, const T* __restrict__ hist, i64 stride, i64 n,
                                   const double* __restrict__ coef, const int* __restrict__ st) {
  if (!st[4]) return;
  const int m = st[3];
  if constexpr (sizeof(T) == 4) {
    // FP32 history: sum_q c_q x_q as a double-float sum (c_q split into two floats,
    // each product exact through an FMA, the running sum kept by TwoSum), so the FP64
    // units (a small fraction of the FP32 rate on this part) see no per-element work;
    // the result is the FP64 sum to about 2^-44 before the final rounding to FP32
    float ch[16], cl[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const double cq = q < m ? coef[q] : 0.0;
      ch[q] = (float)cq;
      cl[q] = (float)(cq - (double)ch[q]);
    }
    for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
      float sh = 0.f, sl = 0.f;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        if (q >= m) break;
        const float x = (float)hist[q * stride + i];
        const float p = ch[q] * x;
        const float e = fmaf(ch[q], x, -p);  // p + e = ch x exactly
        const float t = sh + p;              // TwoSum(sh, p)
        const float bp = t - sh;
        sl += ((sh - (t - bp)) + (p - bp)) + fmaf(cl[q], x, e);
        sh = t;
      }
      out[i] = (T)(sh + sl);
    }
  } else {
    for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < m; ++q) s += coef[q] * (double)hist[q * stride + i];
      out[i] = (T)s;
    }
  }
}

// FP32 vector variant (16-byte aligned history, stride and output): four elements per
// access, the same double-float sum per element.
__global__ void k_diis_extrapolate4(float4* __restrict__ out, const float4* __restrict__ hist, i64 stride4, i64 n4,
                                    const double* __restrict__ coef, const int* __restrict__ st) {
  if (!st[4]) return;
  const int m = st[3];
  float ch[16], cl[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const double cq = q < m ? coef[q] : 0.0;
    ch[q] = (float)cq;
    cl[q] = (float)(cq - (double)ch[q]);
  }
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n4; i += (i64)gridDim.x * blockDim.x) {
    float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (q >= m) break;
      const float4 x4 = hist[q * stride4 + i];
      const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float p = ch[q] * xs[j];
        const float e = fmaf(ch[q], xs[j], -p);
        const float t = sh[j] + p;
        const float bp = t - sh[j];
        sl[j] += ((sh[j] - (t - bp)) + (p - bp)) + fmaf(cl[q], xs[j], e);
        sh[j] = t;
      }
    }
    out[i] = make_float4(sh[0] + sl[0], sh[1] + sl[1], sh[2] + sl[2], sh[3] + sl[3]);
  }
}

template <typename T>
void launch_diis_extrapolate(T* out, const T* hist, i64 stride, i64 n, const double* coef, const int* st,
                             cudaStream_t s) {
  if (n <= 0) return;
  ++g_launch_count;
  if (sizeof(T) == 4 && n % 4 == 0 && stride % 4 == 0 && ((uintptr_t)out & 15) == 0 && ((uintptr_t)hist & 15) == 0) {
    const i64 n4 = n / 4;
    k_diis_extrapolate4<<<ew_blocks(n4), 256, 0, s>>>((float4*)out, (const float4*)hist, stride / 4, n4, coef, st);
    return;
  }
  k_diis_extrapolate<T><<<ew_blocks(n), 256, 0, s>>>(out, hist, stride, n, coef, st);
}
template void launch_diis_extrapolate<double>(double*, const double*, i64, i64, const double*, const int*,
                                              cudaStream_t);
template void launch_diis_extrapolate<float>(float*, const float*, i64, i64, const double*, const int*,
                                             cudaStream_t);

// Type conversion between FP64 and FP32 storage.
template <typename TO, typename TI>
__global__ void k_convert(TO* __restrict__ out, const TI* __restrict__ in, i64 n) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}
template <typename TO, typename TI>
void launch_convert(TO* out, const TI* in, i64 n, cudaStream_t s) {
  if (n <= 0) return;
  i64 blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  ++g_launch_count;
  k_convert<TO, TI><<<(unsigned)blocks, 256, 0, s>>>(out, in, n);
}
template void launch_convert<float, double>(float*, const double*, i64, cudaStream_t);
template void launch_convert<double, float>(double*, const float*, i64, cudaStream_t);
template void launch_convert<double, double>(double*, const double*, i64, cudaStream_t);
template void launch_convert<float, float>(float*, const float*, i64, cudaStream_t);

}  // namespace rcc

namespace rcc {

__global__ void k_energy(const double* __restrict__ g, const double* __restrict__ t1,
                         const double* __restrict__ t2, int o, int v, double* __restrict__ partial) {
  const i64 total = (i64)o * o * v * v;
  double s = 0.0;
  for (i64 idx = blockIdx.x * (i64)blockDim.x + threadIdx.x; idx < total; idx += (i64)gridDim.x * blockDim.x) {
    const int b = (int)(idx % v), a = (int)((idx / v) % v);
    const int j = (int)((idx / ((i64)v * v)) % o), i = (int)(idx / ((i64)v * v * o));
    const double giajb = g[(((i64)i * v + a) * o + j) * v + b];
    const double gibja = g[(((i64)i * v + b) * o + j) * v + a];
    s += (2.0 * giajb - gibja) * (t2[idx] + t1[i * v + a] * t1[j * v + b]);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

void launch_energy(const double* g, const double* t1, const double* t2, int o, int v, double* partial,
                   double* out, cudaStream_t s) {
  ++g_launch_count;
  k_energy<<<kDotBlocks, 256, 0, s>>>(g, t1, t2, o, v, partial);
  ++g_launch_count;
  k_sum<<<1, 256, 0, s>>>(partial, kDotBlocks, out, 1.0, 0);
}

__global__ void k_mp2(double* __restrict__ t2, const double* __restrict__ g, const double* __restrict__ e, int o,
                      int v) {
  const i64 total = (i64)o * o * v * v;
  for (i64 idx = blockIdx.x * (i64)blockDim.x + threadIdx.x; idx < total; idx += (i64)gridDim.x * blockDim.x) {
    const int b = (int)(idx % v), a = (int)((idx / v) % v);
    const int j = (int)((idx / ((i64)v * v)) % o), i = (int)(idx / ((i64)v * v * o));
    t2[idx] = g[(((i64)i * v + a) * o + j) * v + b] / (e[i] + e[j] - e[o + a] - e[o + b]);
  }
}

void launch_mp2(double* t2, const double* g, const double* e, int o, int v, cudaStream_t s) {
  const i64 total = (i64)o * o * v * v;
  i64 blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  ++g_launch_count;
  k_mp2<<<(unsigned)blocks, 256, 0, s>>>(t2, g, e, o, v);
}

// S = (2 - P_a^b - P_a^c) U for each occupied triple, U = t_{trip} read from its
// stored block.  One CTA computes a 16^3 tile of one triple: the three source
// cubes (U^{abc}, U^{bac}, U^{cba} over the tile's label ranges) are loaded into
// shared memory with the threads running along the stored block's unit-stride
// axis, then S is written along c.
template <typename T>
__global__ void __launch_bounds__(256) k_unpack_spin(const void* __restrict__ t3, int f32, int ntrip,
                                                     const i64* __restrict__ base, const int* __restrict__ pos, int v,
                                                     T* __restrict__ S) {
  constexpr int TL = 16;
  // padded [TL][TL+1][TL+2] cubes in dynamic shared memory (59 KB for FP32, 118 KB for FP64)
  extern __shared__ __align__(16) unsigned char unpack_smem[];
  typedef T Cube[TL][TL + 1][TL + 2];
  Cube* cube = reinterpret_cast<Cube*>(unpack_smem);
  const int nt = (v + TL - 1) / TL;
  const i64 V3 = (i64)v * v * v;
  const i64 sv[3] = {(i64)v * v, v, 1};
  const int lf = threadIdx.x & 15, lm = threadIdx.x >> 4;  // lane along the fast slot, row along the middle slot
  for (int t = blockIdx.y; t < ntrip; t += gridDim.y) {
    const i64 b0 = base[t];
    const int p[3] = {pos[3 * t], pos[3 * t + 1], pos[3 * t + 2]};
    const i64 st[3] = {p[0] == 0 ? sv[0] : (p[0] == 1 ? sv[1] : sv[2]), p[1] == 0 ? sv[0] : (p[1] == 1 ? sv[1] : sv[2]),
                       p[2] == 0 ? sv[0] : (p[2] == 1 ? sv[1] : sv[2])};
    // slot (position) whose label runs along the stored unit-stride axis, and the other two
    const int fast = p[0] == 2 ? 0 : (p[1] == 2 ? 1 : 2);
    const int mid = (fast + 1) % 3, slow = (fast + 2) % 3;
    for (int tile = blockIdx.x; tile < nt * nt * nt; tile += gridDim.x) {
      const int lo[3] = {(tile / (nt * nt)) * TL, ((tile / nt) % nt) * TL, (tile % nt) * TL};
      (void)sv;
      // term q reads U at slots (x0, x1, x2) whose label ranges are, in output label order:
      //   q=0: (a, b, c)   q=1: (b, a, c)   q=2: (c, b, a)
      auto label = [](int q, int slot_) {
        return q == 0 ? slot_ : (q == 1 ? (slot_ == 2 ? 2 : 1 - slot_) : 2 - slot_);
      };
      auto sel3 = [](int i, int x0, int x1, int x2) { return i == 0 ? x0 : (i == 1 ? x1 : x2); };
      auto sel3l = [](int i, i64 x0, i64 x1, i64 x2) { return i == 0 ? x0 : (i == 1 ? x1 : x2); };
      const i64 sf = sel3l(fast, st[0], st[1], st[2]), sm = sel3l(mid, st[0], st[1], st[2]),
                ss = sel3l(slow, st[0], st[1], st[2]);
      // shared offsets of the slots in a [TL][TL+1][TL+2] cube
      const int cf = sel3(fast, (TL + 1) * (TL + 2), TL + 2, 1), cm = sel3(mid, (TL + 1) * (TL + 2), TL + 2, 1),
                cs = sel3(slow, (TL + 1) * (TL + 2), TL + 2, 1);
      __syncthreads();
      for (int q = 0; q < 3; ++q) {
        const int xf = sel3(label(q, fast), lo[0], lo[1], lo[2]) + lf;
        const int xm = sel3(label(q, mid), lo[0], lo[1], lo[2]) + lm;
        const int xs0 = sel3(label(q, slow), lo[0], lo[1], lo[2]);
        const bool in = xf < v && xm < v;
        const i64 off0 = b0 + xf * sf + xm * sm + xs0 * ss;
        T ld[TL];
#pragma unroll
        for (int u = 0; u < TL; ++u) {
          T val = (T)0;
          if (in && xs0 + u < v) {
            const i64 off = off0 + u * ss;
            if constexpr (sizeof(T) == 4)
              val = ((const float*)t3)[off];  // FP32 storage: no FP64 conversions
            else
              val = (T)load_src(t3, f32, off);
          }
          ld[u] = val;
        }
        T* cq = &cube[q][0][0][0] + lf * cf + lm * cm;
#pragma unroll
        for (int u = 0; u < TL; ++u) cq[u * cs] = ld[u];
      }
      __syncthreads();
      // S along c: thread (bb, c), loop a
      const int bb = threadIdx.x >> 4, c = threadIdx.x & 15;
      const int gb = lo[1] + bb, gc = lo[2] + c;
      if (gb < v && gc < v) {
        T* dst = S + (i64)t * V3 + (i64)gb * v + gc;
#pragma unroll 4
        for (int a = 0; a < TL; ++a) {
          const int ga = lo[0] + a;
          if (ga >= v) break;
          // U^{abc} = cube0[a][b][c], U^{bac} = cube1[b][a][c], U^{cba} = cube2[c][b][a]
          dst[(i64)ga * v * v] = (T)2 * cube[0][a][bb][c] - cube[1][bb][a][c] - cube[2][c][bb][a];
        }
      }
    }
  }
}

template <typename T>
void launch_unpack_spin(const void* t3, int f32, int ntrip, const i64* base, const int* pos, int v, T* S,
                        cudaStream_t s) {
  const int nt = (v + 15) / 16;
  unsigned gx = (unsigned)(nt * nt * nt);
  if (gx > 1024) gx = 1024;
  unsigned gy = (unsigned)(ntrip < 1024 ? ntrip : 1024);
  const size_t smem = 3 * sizeof(T) * 16 * 17 * 18;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_unpack_spin<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  ++g_launch_count;
  k_unpack_spin<T><<<dim3(gx, gy), 256, smem, s>>>(t3, f32, ntrip, base, pos, v, S);
}
template void launch_unpack_spin<double>(const void*, int, int, const i64*, const int*, int, double*, cudaStream_t);
template void launch_unpack_spin<float>(const void*, int, int, const i64*, const int*, int, float*, cudaStream_t);

// ---------------------------------------------------------------------------
// T3 contribution to R1 for one batch z of unpacked, spin-summed blocks
// S[x][y][e1][e2][e3] (the double check is D^{x0x1x2} = 2 S^{x0x1x2} - S^{x0x2x1}):
//   dR1[z][a] += sum_{x,y,b} sum_c v^{xy}_{bc} (S[x,y,b,c,a] - 1/2 S[x,y,b,a,c])
// One pass over S; per-block partial sums, then a fixed-order reduction.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_r1_t3(const T* __restrict__ S, const double* __restrict__ oovv, int o,
                                               int v, double* __restrict__ partial) {
  // per slab (x, y, b) = sl[c][a]: term 1 sum_c w[c] sl[c][a] with threads along a,
  // term 2 sum_c w[c] sl[a][c] with a warp per row a and lanes along c (both coalesced);
  // term 2 of each row is owned by one warp and kept in shared memory per warp.
  // a = threadIdx.x + 256 j, j < 16 (v <= 4096).
  extern __shared__ __align__(16) unsigned char r1_smem[];
  T* t2s = reinterpret_cast<T*>(r1_smem);  // [8 warps][v]
  T* ws = t2s + 8 * v;                     // the slab's weights in the storage type
  const i64 nslab = (i64)o * o * v;
  const i64 V2 = (i64)v * v;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = threadIdx.x; q < 8 * v; q += blockDim.x) t2s[q] = (T)0;
  T acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = (T)0;
  for (i64 sgi = blockIdx.x; sgi < nslab; sgi += gridDim.x) {
    const T* sl = S + sgi * V2;          // slab (x, y, b): [c][a]
    __syncthreads();                     // the previous slab's weights are consumed
    for (int c = threadIdx.x; c < v; c += blockDim.x) ws[c] = (T)oovv[sgi * v + c];  // v^{xy}_{bc}
    __syncthreads();
    const T* w = ws;
    for (int c = 0; c < v; ++c) {
      const T wc = w[c];
      const T* row = sl + (i64)c * v;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int a = threadIdx.x + 256 * j;
        if (a < v) acc[j] += wc * row[a];
      }
    }
    for (int ar = warp; ar < v; ar += 8) {
      T part = (T)0;
      for (int c = lane; c < v; c += 32) part += w[c] * sl[(i64)ar * v + c];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
      if (lane == 0) t2s[warp * v + ar] += part;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int a = threadIdx.x + 256 * j;
    if (a < v) {
      T t2 = (T)0;
      for (int q = 0; q < 8; ++q) t2 += t2s[q * v + a];
      partial[(i64)blockIdx.x * v + a] = (double)acc[j] - 0.5 * (double)t2;
    }
  }
}

// Same sums with the whole slab staged in shared memory ([c][a] rows padded to v+1):
// every element of S is read from memory once and both terms come from shared
// memory (used when a slab fits, v up to about 220 in FP32).
template <typename T>
__global__ void __launch_bounds__(256) k_r1_slab(const T* __restrict__ S, const double* __restrict__ oovv, int o,
                                                 int v, double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char r1s_smem[];
  T* sl = reinterpret_cast<T*>(r1s_smem);  // [v][v + 1]
  T* ws = sl + (i64)v * (v + 1);           // [v]
  const i64 nslab = (i64)o * o * v;
  const i64 V2 = (i64)v * v;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, a = threadIdx.x;
  T t1 = (T)0, t2 = (T)0;
  for (i64 sgi = blockIdx.x; sgi < nslab; sgi += gridDim.x) {
    const T* src = S + sgi * V2;
    __syncthreads();  // the previous slab is consumed
    // asynchronous element copies (cp.async, no register staging): all of a thread's
    // loads of the slab are in flight at once
    for (int c = warp; c < v; c += 8) {
      const T* row = src + (i64)c * v;
      T* dst = sl + c * (v + 1);
      for (int x = lane; x < v; x += 32) {
        if constexpr (sizeof(T) == 4)
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst + x)),
                       "l"(row + x)
                       : "memory");
        else
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst + x)),
                       "l"(row + x)
                       : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int c = threadIdx.x; c < v; c += blockDim.x) ws[c] = (T)oovv[sgi * v + c];
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    if (a < v) {
      const T* col = sl + a;                 // sl[c][a] over c
      const T* row = sl + a * (v + 1);       // sl[a][c] over c
      for (int c = 0; c < v; ++c) {
        const T w = ws[c];
        t1 += w * col[c * (v + 1)];
        t2 += w * row[c];
      }
    }
  }
  if (a < v) partial[(i64)blockIdx.x * v + a] = (double)t1 - 0.5 * (double)t2;
}

// One block per a: the nblk partials are summed in a fixed order.
__global__ void k_r1_reduce(const double* __restrict__ partial, int nblk, int v, double* __restrict__ out) {
  const int a = blockIdx.x;
  double s = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) s += partial[(i64)q * v + a];
  s = block_sum(s);
  if (threadIdx.x == 0) out[a] += s;
}

template <typename T>
void launch_r1_t3(const T* S, const double* oovv, int o, int v, double* dR1_z, double* scratch, i64 scratch_elems,
                  cudaStream_t s) {
  const i64 nslab = (i64)o * o * v;
  int nblk = (int)std::min<i64>(nslab, 1216);
  while ((i64)nblk * v > scratch_elems && nblk > 1) nblk /= 2;
  const size_t slab = ((size_t)v * (v + 1) + v) * sizeof(T);
  if (v <= 256 && slab <= (200u << 10)) {
    static size_t attr_s = 48 << 10;
    if (slab > attr_s) {
      cudaFuncSetAttribute(k_r1_slab<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)slab);
      attr_s = slab;
    }
    ++g_launch_count;
    k_r1_slab<T><<<nblk, 256, slab, s>>>(S, oovv, o, v, scratch);
  } else {
    const size_t smem = (size_t)9 * v * sizeof(T);
    static size_t attr = 48 << 10;  // above the default 48 KB the kernel opts in (up to the 227 KB limit)
    if (smem > attr) {
      cudaFuncSetAttribute(k_r1_t3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr = smem;
    }
    ++g_launch_count;
    k_r1_t3<T><<<nblk, 256, smem, s>>>(S, oovv, o, v, scratch);
  }
  ++g_launch_count;
  k_r1_reduce<<<v, 256, 0, s>>>(scratch, nblk, v, dR1_z);
}
template void launch_r1_t3<double>(const double*, const double*, int, int, double*, double*, i64, cudaStream_t);
template void launch_r1_t3<float>(const float*, const double*, int, int, double*, double*, i64, cudaStream_t);

// ---------------------------------------------------------------------------
// Two-phase scatter of whole v^3 rows: X[m] in natural (a,b,c) order is added to
// the stored block at row_base[m] with the virtual axes permuted by the sort
// permutation perm_sel[m].  One CTA moves a 16^3 cube: the cube is read along c
// (coalesced), staged in shared memory, and added along the target's unit-stride
// axis (coalesced read-modify-write).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256, 5) k_scatter_rows3(const float* __restrict__ X, int M, int v,
                                                       const i64* __restrict__ row_base,
                                                       const int* __restrict__ row_sel,
                                                       const double* __restrict__ row_alpha, T* __restrict__ C) {
  constexpr int TL = 16;
  __shared__ float cube[TL][TL + 1][TL + 2];
  constexpr int SA = (TL + 1) * (TL + 2), SB = TL + 2;  // shared strides of the cube's a and b slots
  const int nt = (v + TL - 1) / TL;
  const i64 V2 = (i64)v * v, V3 = V2 * v;
  const int lf = threadIdx.x & 15, lm = threadIdx.x >> 4;
  for (int m = blockIdx.y; m < M; m += gridDim.y) {
    const int sel = row_sel[m];
    const int p0 = perm3(sel, 0), p1 = perm3(sel, 1), p2 = perm3(sel, 2);  // stored axis of X slot q
    // slot whose label lands on the target's unit-stride axis, and the other two
    const int fast = p0 == 2 ? 0 : (p1 == 2 ? 1 : 2);
    const int mid = fast == 0 ? 1 : 0, slow = 3 - fast - mid;
    auto pq = [&](int q) { return q == 0 ? p0 : (q == 1 ? p1 : p2); };
    auto sv = [&](int axis) { return axis == 0 ? V2 : (axis == 1 ? (i64)v : (i64)1); };
    auto ss = [&](int q) { return q == 0 ? SA : (q == 1 ? SB : 1); };
    const i64 stm = sv(pq(mid)), sts = sv(pq(slow));
    const int cF = ss(fast), cM = ss(mid), cS = ss(slow);
    const i64 base = row_base[m];
    const T al = (T)row_alpha[m];
    const float* xm = X + (i64)m * V3;
    for (int tile = blockIdx.x; tile < nt * nt * nt; tile += gridDim.x) {
      const int lo0 = tile / (nt * nt) * TL, lo1 = (tile / nt) % nt * TL, lo2 = tile % nt * TL;
      __syncthreads();
      {  // X cube along c: thread (b, c) = (lm, lf), 16 loads in flight (one running pointer)
        const int gb = lo1 + lm, gc = lo2 + lf;
        const int na = (gb < v && gc < v) ? min(TL, v - lo0) : 0;
        const float* px = xm + lo0 * V2 + (i64)gb * v + gc;
        float ld[TL];
#pragma unroll
        for (int a = 0; a < TL; ++a) {
          ld[a] = a < na ? __ldg(px) : 0.f;
          px += V2;
        }
#pragma unroll
        for (int a = 0; a < TL; ++a) cube[a][lm][lf] = ld[a];
      }
      __syncthreads();
      // add along the target's unit-stride axis: slot fast = lf, mid = lm, slow = u
      const int lofast = fast == 0 ? lo0 : (fast == 1 ? lo1 : lo2);
      const int lomid = mid == 0 ? lo0 : (mid == 1 ? lo1 : lo2);
      const int loslow = slow == 0 ? lo0 : (slow == 1 ? lo1 : lo2);
      const int gf = lofast + lf, gm = lomid + lm;
      if (gf < v && gm < v) {
        T* dst = C + base + gf + gm * stm + (i64)loslow * sts;
        const float* src = &cube[0][0][0] + lf * cF + lm * cM;
        const int nu = min(TL, v - loslow);
#pragma unroll
        for (int h = 0; h < TL; h += 8) {  // two halves of 8 read-modify-writes in flight
          T old[8];
          T* pd = dst + h * sts;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            old[u] = h + u < nu ? pd[0] : (T)0;
            pd += sts;
          }
          pd = dst + h * sts;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (h + u < nu) pd[0] = old[u] + al * (T)src[(h + u) * cS];
            pd += sts;
          }
        }
      }
    }
  }
}

template <typename T>
void launch_scatter_rows3(const float* X, int M, int v, const i64* row_base, const int* row_sel,
                          const double* row_alpha, T* C, cudaStream_t s) {
  const int nt = (v + 15) / 16;
  unsigned gx = (unsigned)std::min(nt * nt * nt, 1024);
  unsigned gy = (unsigned)std::min(M, 65535);
  ++g_launch_count;
  k_scatter_rows3<T><<<dim3(gx, gy), 256, 0, s>>>(X, M, v, row_base, row_sel, row_alpha, C);
}
template void launch_scatter_rows3<float>(const float*, int, int, const i64*, const int*, const double*, float*,
                                          cudaStream_t);
template void launch_scatter_rows3<double>(const float*, int, int, const i64*, const int*, const double*, double*,
                                           cudaStream_t);

// ---------------------------------------------------------------------------
// T2-driven term of Eq. resi-rccsdt with K = o, output-stationary:
//   r_{ijk}^{abc} += sum over the six column permutations of
//                    -sum_l W^{a1 l}_{i1 i2} t_{l i3}^{a2 a3}
// One CTA of 64 threads owns a 16^3 tile of one stored block and accumulates all six
// terms in registers, each thread a 4 x 4 x 4 sub-cube (register blocking: per l one
// 4-vector of W and a 4 x 4 patch of t2 from shared memory feed 64 FMAs).  Per term
// and chunk of 8 values of l the W slice [l][a1] and the t2 slice [l][a2][a3] of the
// tile are copied to shared memory with cp.async (zero-filled outside the block and
// beyond o), two stages in flight (three measured slower: fewer CTAs per SM).  The
// block is read and written once.
// Wvooo[a][l][i][j] = W^{al}_{ij}; t2[l][k][b][c] = t_lk^bc (T precision copies).
// ---------------------------------------------------------------------------
constexpr int kT2oTL = 16, kT2oLC = 8, kT2oThreads = 64, kT2oStages = 2;

template <typename T>
struct T2oLayout {
  static constexpr int EPC = 16 / (int)sizeof(T);      // elements per 16-byte chunk
  static constexpr int PW = kT2oTL + EPC;              // padded row, 16-byte multiple
  static constexpr int WS = kT2oLC * PW;               // W slice [l][a1]
  static constexpr int TS = kT2oLC * kT2oTL * PW;      // t2 slice [l][a2][a3]
  static constexpr int STAGE = WS + TS;
};

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

template <typename T>
__device__ __forceinline__ void load4(const T* p, T (&x)[4]) {  // p 16-byte aligned
  if constexpr (sizeof(T) == 4) {
    const float4 f = *reinterpret_cast<const float4*>(p);
    x[0] = f.x;
    x[1] = f.y;
    x[2] = f.z;
    x[3] = f.w;
  } else {
    const double2 f0 = reinterpret_cast<const double2*>(p)[0], f1 = reinterpret_cast<const double2*>(p)[1];
    x[0] = f0.x;
    x[1] = f0.y;
    x[2] = f1.x;
    x[3] = f1.y;
  }
}

// acc[a0][a1][a2] -= sum_l W[l][a_X1] t[l][a_X2][a_X3] over the thread's sub-cube
template <int X1, int X2, int X3, typename T>
__device__ __forceinline__ void t2o_step(T (&acc)[4][4][4], const T* __restrict__ Wb, const T* __restrict__ Tb,
                                         int lc, const int (&u)[3]) {
  using Lay = T2oLayout<T>;
#pragma unroll 2
  for (int l = 0; l < lc; ++l) {
    T w[4], t[4][4];
    load4(Wb + l * Lay::PW + 4 * u[X1], w);
#pragma unroll
    for (int i = 0; i < 4; ++i) load4(Tb + (l * kT2oTL + 4 * u[X2] + i) * Lay::PW + 4 * u[X3], t[i]);
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c0 = X1 == 0 ? m : (X2 == 0 ? i : j);
          const int c1 = X1 == 1 ? m : (X2 == 1 ? i : j);
          const int c2 = X1 == 2 ? m : (X2 == 2 ? i : j);
          acc[c0][c1][c2] -= w[m] * t[i][j];
        }
  }
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(kT2oThreads) k_t2_outer(T* __restrict__ r3, const T* __restrict__ Wvooo,
                                                          const T* __restrict__ t2, const int4* __restrict__ blocks,
                                                          int o, int v, i64 n3) {
  using Lay = T2oLayout<T>;
  constexpr int TL = kT2oTL, LC = kT2oLC;
  extern __shared__ __align__(16) unsigned char t2o_smem[];
  T* sm = reinterpret_cast<T*>(t2o_smem);  // [2][STAGE]: W slice then t2 slice
  const int nt = (v + TL - 1) / TL;
  const i64 V2 = (i64)v * v, V3 = V2 * v;
  const int tid = threadIdx.x;
  const int u[3] = {tid >> 4, (tid >> 2) & 3, tid & 3};
  const int nch = (o + LC - 1) / LC, nstage = 6 * nch;  // stage = (ordering q, chunk of l)
  for (i64 blk = blockIdx.y; blk < n3; blk += gridDim.y) {
    const int4 ijk = blocks[blk];
    auto occ = [&](int x) { return x == 0 ? ijk.x : (x == 1 ? ijk.y : ijk.z); };
    for (int tile = blockIdx.x; tile < nt * nt * nt; tile += gridDim.x) {
      const int lo0 = tile / (nt * nt) * TL, lo1 = (tile / nt) % nt * TL, lo2 = tile % nt * TL;
      auto lo = [&](int x) { return x == 0 ? lo0 : (x == 1 ? lo1 : lo2); };
      auto issue = [&](int st) {
        T* Wb = sm + (st % kT2oStages) * Lay::STAGE;
        T* Tb = Wb + Lay::WS;
        const int q = st / nch, l0 = (st % nch) * LC, lc = min(LC, o - l0);
        const int x1 = perm3(q, 0), x2 = perm3(q, 1), x3 = perm3(q, 2);
        const int i1 = occ(x1), i2 = occ(x2), i3 = occ(x3);
        for (int e = tid; e < LC * TL; e += kT2oThreads) {  // W[l][a1]
          const int l = e / TL, a = e % TL, ga = lo(x1) + a;
          const bool ok = l < lc && ga < v;
          cp_async_elem(Wb + l * Lay::PW + a, ok ? Wvooo + (((i64)ga * o + l0 + l) * o + i1) * o + i2 : Wvooo, ok);
        }
        if constexpr (VEC) {  // t2 rows of 16 elements in 16-byte chunks (v a multiple of the chunk)
          constexpr int CPR = TL / Lay::EPC;
          for (int e = tid; e < LC * TL * CPR; e += kT2oThreads) {
            const int row = e / CPR, part = e % CPR, l = row / TL, r2 = row % TL;
            const int g2 = lo(x2) + r2, g3 = lo(x3) + part * Lay::EPC;
            const bool ok = l < lc && g2 < v && g3 < v;
            const T* src = ok ? t2 + ((i64)(l0 + l) * o + i3) * V2 + (i64)g2 * v + g3 : t2;
            cp_async16(Tb + (l * TL + r2) * Lay::PW + part * Lay::EPC, src, ok);
          }
        } else {
          for (int e = tid; e < LC * TL * TL; e += kT2oThreads) {
            const int row = e / TL, c = e % TL, l = row / TL, r2 = row % TL;
            const int g2 = lo(x2) + r2, g3 = lo(x3) + c;
            const bool ok = l < lc && g2 < v && g3 < v;
            cp_async_elem(Tb + (l * TL + r2) * Lay::PW + c, ok ? t2 + ((i64)(l0 + l) * o + i3) * V2 + (i64)g2 * v + g3 : t2,
                          ok);
          }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
      };
      T acc[4][4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
          for (int z = 0; z < 4; ++z) acc[x][y][z] = (T)0;
      __syncthreads();  // the previous tile's last stage is consumed
      for (int st = 0; st < kT2oStages - 1; ++st) {
        if (st < nstage) issue(st);
        else asm volatile("cp.async.commit_group;" ::: "memory");  // an empty group keeps the count
      }
#pragma unroll 1
      for (int st = 0; st < nstage; ++st) {
        // the stage kT2oStages - 1 ahead; its buffer's last reader was stage st - 1
        if (st + kT2oStages - 1 < nstage) issue(st + kT2oStages - 1);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group %0;" ::"n"(kT2oStages - 1) : "memory");  // stage st has landed
        __syncthreads();
        const T* Wb = sm + (st % kT2oStages) * Lay::STAGE;
        const T* Tb = Wb + Lay::WS;
        const int q = st / nch, lc = min(LC, o - (st % nch) * LC);
        switch (perm3(q, 0) * 3 + perm3(q, 1)) {
          case 1: t2o_step<0, 1, 2>(acc, Wb, Tb, lc, u); break;
          case 2: t2o_step<0, 2, 1>(acc, Wb, Tb, lc, u); break;
          case 3: t2o_step<1, 0, 2>(acc, Wb, Tb, lc, u); break;
          case 5: t2o_step<1, 2, 0>(acc, Wb, Tb, lc, u); break;
          case 6: t2o_step<2, 0, 1>(acc, Wb, Tb, lc, u); break;
          default: t2o_step<2, 1, 0>(acc, Wb, Tb, lc, u); break;
        }
        __syncthreads();
      }
      // read-modify-write of the sub-cube: rows of 4 along the unit-stride axis
#pragma unroll
      for (int m0 = 0; m0 < 4; ++m0)
#pragma unroll
        for (int m1 = 0; m1 < 4; ++m1) {
          const int g0 = lo0 + 4 * u[0] + m0, g1 = lo1 + 4 * u[1] + m1, g2 = lo2 + 4 * u[2];
          if (g0 >= v || g1 >= v || g2 >= v) continue;
          T* dst = r3 + blk * V3 + (i64)g0 * V2 + (i64)g1 * v + g2;
          if constexpr (VEC && sizeof(T) == 4) {
            float4 x = *reinterpret_cast<float4*>(dst);
            x.x += acc[m0][m1][0];
            x.y += acc[m0][m1][1];
            x.z += acc[m0][m1][2];
            x.w += acc[m0][m1][3];
            *reinterpret_cast<float4*>(dst) = x;
          } else {
#pragma unroll
            for (int m2 = 0; m2 < 4; ++m2)
              if (g2 + m2 < v) dst[m2] += acc[m0][m1][m2];
          }
        }
    }
  }
}

template <typename T>
void launch_t2_outer(T* r3, const T* Wvooo, const T* t2, const int4* blocks, int o, int v, i64 n3, cudaStream_t s) {
  const int nt = (v + kT2oTL - 1) / kT2oTL;
  const unsigned gx = (unsigned)std::min(nt * nt * nt, 65535);
  const unsigned gy = (unsigned)std::min<i64>(n3, 65535);
  const size_t smem = (size_t)kT2oStages * T2oLayout<T>::STAGE * sizeof(T);
  const bool vec = v % T2oLayout<T>::EPC == 0;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_t2_outer<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_t2_outer<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  ++g_launch_count;
  if (vec)
    k_t2_outer<T, true><<<dim3(gx, gy), kT2oThreads, smem, s>>>(r3, Wvooo, t2, blocks, o, v, n3);
  else
    k_t2_outer<T, false><<<dim3(gx, gy), kT2oThreads, smem, s>>>(r3, Wvooo, t2, blocks, o, v, n3);
}
template void launch_t2_outer<double>(double*, const double*, const double*, const int4*, int, int, i64, cudaStream_t);
template void launch_t2_outer<float>(float*, const float*, const float*, const int4*, int, int, i64, cudaStream_t);

}  // namespace rcc
