// Pair-symmetric operand panels of the pp-ladder (Sec. II.C.1).
//
// The ladder intermediate is symmetric under the joint exchange of its two pairs,
// W^{xy}_{de} = W^{yx}_{ed}.  For one view X^{xy}(w) = sum_{de} W^{xy}_{de} T(d, e, w)
// of a stored block, the sum and difference over the exchange x <-> y are
//   X^{xy} + X^{yx} = sum_{d <= e} W+^{xy}_{de} T+(d, e, w),
//   X^{xy} - X^{yx} = sum_{d <  e} W-^{xy}_{de} T-(d, e, w),
// with W+ = W_de + W_ed (W_dd on the diagonal), W- = W_de - W_ed,
// T+ = T(d, e) + T(e, d), T- = T(d, e) - T(e, d); rows x <= y (x < y for the
// difference).  Two GEMMs of about (v^2 / 2)^2 v FMA each replace one of v^4 v.
// These kernels gather the four panels (K-major, pairs numbered tile-major as
// pair_decode describes); the GEMM epilogue adds each product half to X^{xy} and
// half, with the sign of its part, to X^{yx}.
#include <cstdint>
#include <type_traits>

#include "elem.cuh"
#include "kernels.h"

namespace rcc {
namespace {

constexpr int kPT = 16;         // labels per tile
constexpr int kPS = kPT + 1;    // padded stride of the staged cubes

template <int KIND>
__device__ __forceinline__ void put_f(const CubeDst& d, i64 o, float x) {
  if constexpr (KIND == PANEL_BF16X2) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    ((__nv_bfloat16*)d.out_hi)[o] = hi;
    ((__nv_bfloat16*)d.out_lo)[o] = __float2bfloat16_rn(x - __bfloat162float(hi));
  } else {
    const float hi = tf32_round(x);
    ((float*)d.out_hi)[o] = hi;
    ((float*)d.out_lo)[o] = tf32_round(x - hi);
  }
}

// Stores one panel element computed in AT (double for FP64 panels).
template <int KIND, typename AT>
__device__ __forceinline__ void put(const CubeDst& d, i64 row, int k, AT x) {
  const i64 o = row * d.Kpad + k;
  if constexpr (KIND == PANEL_F64) {
    ((double*)d.out_hi)[o] = (double)x;
  } else if constexpr (sizeof(AT) == 8) {
    put_f<KIND>(d, o, f64_to_f32_rn((double)x));  // integer-path rounding (no FP64 pipe)
  } else {
    put_f<KIND>(d, o, (float)x);
  }
}

// A panels from W [x][y][d][e] (FP64): one CTA per row pair (x, y), x <= y, taking
// the chunks in order; each chunk stages W_{de} and W_{ed} as 16 x 16 tiles.
template <int KIND>
__global__ void __launch_bounds__(256) k_pair_pack_w(const double* __restrict__ W, int v,
                                                     const int4* __restrict__ rows, int Mp,
                                                     const PairChunk* __restrict__ ch, int nchunk, int Kp, int Km,
                                                     CubeDst dp, CubeDst dm) {
  __shared__ double sA[kPT][kPS], sB[kPT][kPS];
  const int t = threadIdx.x;
  const i64 V2 = (i64)v * v;
  for (int m = blockIdx.x; m < Mp; m += gridDim.x) {
    const int4 rw = rows[m];  // x, y, row of the difference (-1 when x = y)
    const double* Wr = W + ((i64)rw.x * v + rw.y) * V2;
    for (int ci = 0; ci < nchunk; ++ci) {
      const PairChunk c = ch[ci];
      const int d0 = c.P * kPT, e0 = c.Q * kPT;
      const int nd = min(kPT, v - d0), ne = min(kPT, v - e0);
      const bool diag = c.P == c.Q;
      {
        const int i = t >> 4, j = t & 15;
        if (i < nd && j < ne) sA[i][j] = Wr[(i64)(d0 + i) * v + e0 + j];  // W_{de}
        if (i < ne && j < nd) sB[i][j] = Wr[(i64)(e0 + i) * v + d0 + j];  // W_{ed}
      }
      __syncthreads();
      const int np = diag ? nd * (nd + 1) / 2 : nd * ne;
      const int nm = diag ? nd * (nd - 1) / 2 : nd * ne;
      if (t < np) {
        int a, b;
        pair_decode(t, diag, true, nd, ne, a, b);
        const double x = (diag && a == b) ? sA[a][a] : sA[a][b] + sB[b][a];
        put<KIND, double>(dp, m, c.offp + t, x);
      }
      if (rw.z >= 0 && t < nm) {
        int a, b;
        pair_decode(t, diag, false, nd, ne, a, b);
        put<KIND, double>(dm, rw.z, c.offm + t, sA[a][b] - sB[b][a]);
      }
      __syncthreads();
    }
    for (int k = Kp + t; k < dp.Kpad; k += blockDim.x) put<KIND, double>(dp, m, k, 0.0);
    if (rw.z >= 0)
      for (int k = Km + t; k < dm.Kpad; k += blockDim.x) put<KIND, double>(dm, rw.z, k, 0.0);
  }
}

// B panels of one view of stored blocks: CTA (chunk, w tile, block) stages the
// label cubes T(d0.., e0.., w0..) and T(e0.., d0.., w0..) (read along the view's
// unit-stride axis), then writes 16 panel rows of the chunk's pairs.  The last
// chunk's CTAs also zero the padding columns.
// (Also the T4 views: grid z = (block, w1) pairs with `inner` values of w1 at stride
// `sinner` inside a block of `vblk` elements; T3: inner 1, vblk v^3.)
template <int KIND, typename TS>
__global__ void __launch_bounds__(256) k_pair_pack_t(const TS* __restrict__ t3, i64 b0, int v, i64 sd, i64 se,
                                                     i64 sw, const PairChunk* __restrict__ ch, int nchunk, int Kp,
                                                     int Km, CubeDst dp, CubeDst dm, int inner, i64 sinner,
                                                     i64 vblk) {
  using AT = typename std::conditional<KIND == PANEL_F64, double, float>::type;
  extern __shared__ __align__(16) unsigned char pp_smem[];
  TS* X = (TS*)pp_smem;            // X[a][b][w] = T(d0 + a, e0 + b, w0 + w)
  TS* Y = X + kPT * kPS * kPS;     // Y[a][b][w] = T(e0 + a, d0 + b, w0 + w)
  const PairChunk c = ch[blockIdx.x];
  const int w0 = blockIdx.y * kPT;
  const i64 zb = blockIdx.z / inner, zi = blockIdx.z - zb * inner;
  const TS* T = t3 + (b0 + zb) * vblk + zi * sinner;
  const int d0 = c.P * kPT, e0 = c.Q * kPT;
  const int nd = min(kPT, v - d0), ne = min(kPT, v - e0), nw = min(kPT, v - w0);
  const bool diag = c.P == c.Q;
  const bool wfast = sw == 1;
  {
    // thread (f, g) holds the labels (b, w) (the unit-stride one on f) and reads the
    // 16 values of a of both cubes; every load is issued before any is stored
    const int f = threadIdx.x & 15, g = threadIdx.x >> 4;
    const int b = wfast ? g : f, w = wfast ? f : g;
    const bool inx = w < nw && b < ne, iny = !diag && w < nw && b < nd;
    const TS* px = T + (i64)d0 * sd + (e0 + b) * se + (w0 + w) * sw;
    const TS* py = T + (i64)e0 * sd + (d0 + b) * se + (w0 + w) * sw;
    TS vx[kPT], vy[kPT];
#pragma unroll
    for (int a = 0; a < kPT; ++a) vx[a] = (inx && a < nd) ? __ldg(px + a * sd) : (TS)0;
#pragma unroll
    for (int a = 0; a < kPT; ++a) vy[a] = (iny && a < ne) ? __ldg(py + a * sd) : (TS)0;
    TS* x = X + b * kPS + w;
    TS* y = Y + b * kPS + w;
#pragma unroll
    for (int a = 0; a < kPT; ++a) x[a * kPS * kPS] = vx[a];
    if (!diag) {
#pragma unroll
      for (int a = 0; a < kPT; ++a) y[a * kPS * kPS] = vy[a];
    }
  }
  __syncthreads();
  const TS* Z = diag ? X : Y;
  const int np = diag ? nd * (nd + 1) / 2 : nd * ne;
  const int nm = diag ? nd * (nd - 1) / 2 : nd * ne;
  const int t = threadIdx.x;
  int ap = 0, bp = 0, am = 0, bm = 0;
  if (t < np) pair_decode(t, diag, true, nd, ne, ap, bp);
  if (t < nm) pair_decode(t, diag, false, nd, ne, am, bm);
  const i64 row0 = (i64)blockIdx.z * v + w0;
  for (int w = 0; w < nw; ++w) {
    if (t < np)
      put<KIND, AT>(dp, row0 + w, c.offp + t, (AT)X[(ap * kPS + bp) * kPS + w] + (AT)Z[(bp * kPS + ap) * kPS + w]);
    if (t < nm)
      put<KIND, AT>(dm, row0 + w, c.offm + t, (AT)X[(am * kPS + bm) * kPS + w] - (AT)Z[(bm * kPS + am) * kPS + w]);
  }
  if (blockIdx.x == nchunk - 1) {
    for (int w = 0; w < nw; ++w) {
      for (int k = Kp + t; k < dp.Kpad; k += blockDim.x) put<KIND, AT>(dp, row0 + w, k, (AT)0);
      for (int k = Km + t; k < dm.Kpad; k += blockDim.x) put<KIND, AT>(dm, row0 + w, k, (AT)0);
    }
  }
}

template <int KIND, typename TS>
void pack_t(const TS* t3, i64 b0, int nblk, int v, i64 sd, i64 se, i64 sw, const PairChunk* ch, int nchunk, int Kp,
            int Km, const CubeDst& dp, const CubeDst& dm, cudaStream_t s, int inner = 1, i64 sinner = 0,
            i64 vblk = -1) {
  if (vblk < 0) vblk = (i64)v * v * v;
  const size_t smem = (size_t)2 * kPT * kPS * kPS * sizeof(TS);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_pair_pack_t<KIND, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const int nw = (v + kPT - 1) / kPT;
  dim3 grid((unsigned)nchunk, (unsigned)nw, (unsigned)((i64)nblk * inner));
  ++g_launch_count;
  k_pair_pack_t<KIND, TS><<<grid, 256, smem, s>>>(t3, b0, v, sd, se, sw, ch, nchunk, Kp, Km, dp, dm, inner, sinner,
                                                  vblk);
}

}  // namespace

void launch_pair_pack_w(int kind, const double* W, int v, const int4* rows, int Mp, const PairChunk* ch, int nchunk,
                        int Kp, int Km, const CubeDst& dp, const CubeDst& dm, cudaStream_t s) {
  if (Mp <= 0) return;
  const unsigned grid = (unsigned)Mp;
  ++g_launch_count;
  if (kind == PANEL_F64)
    k_pair_pack_w<PANEL_F64><<<grid, 256, 0, s>>>(W, v, rows, Mp, ch, nchunk, Kp, Km, dp, dm);
  else if (kind == PANEL_BF16X2)
    k_pair_pack_w<PANEL_BF16X2><<<grid, 256, 0, s>>>(W, v, rows, Mp, ch, nchunk, Kp, Km, dp, dm);
  else
    k_pair_pack_w<PANEL_TF32X2><<<grid, 256, 0, s>>>(W, v, rows, Mp, ch, nchunk, Kp, Km, dp, dm);
}

void launch_pair_pack_t(int kind, const void* t3, int t3_f32, i64 b0, int nblk, int v, i64 sd, i64 se, i64 sw,
                        const PairChunk* ch, int nchunk, int Kp, int Km, const CubeDst& dp, const CubeDst& dm,
                        cudaStream_t s) {
  if (nblk <= 0 || nchunk <= 0) return;
  if (t3_f32) {
    const float* t = (const float*)t3;
    if (kind == PANEL_F64) pack_t<PANEL_F64, float>(t, b0, nblk, v, sd, se, sw, ch, nchunk, Kp, Km, dp, dm, s);
    else if (kind == PANEL_BF16X2) pack_t<PANEL_BF16X2, float>(t, b0, nblk, v, sd, se, sw, ch, nchunk, Kp, Km, dp, dm, s);
    else pack_t<PANEL_TF32X2, float>(t, b0, nblk, v, sd, se, sw, ch, nchunk, Kp, Km, dp, dm, s);
  } else {  // FP64 storage: FP64 panels only
    pack_t<PANEL_F64, double>((const double*)t3, b0, nblk, v, sd, se, sw, ch, nchunk, Kp, Km, dp, dm, s);
  }
}

void launch_pair_pack_t4(int kind, const void* t4, int t4_f32, i64 b0, int nblk, int v, i64 sd, i64 se, i64 sw,
                         i64 sr, const PairChunk* ch, int nchunk, int Kp, int Km, const CubeDst& dp,
                         const CubeDst& dm, cudaStream_t s) {
  if (nblk <= 0 || nchunk <= 0) return;
  const i64 V4 = (i64)v * v * v * v;
  if (t4_f32) {
    const float* t = (const float*)t4;
    if (kind == PANEL_BF16X2)
      pack_t<PANEL_BF16X2, float>(t, b0, nblk, v, sd, se, sw, ch, nchunk, Kp, Km, dp, dm, s, v, sr, V4);
    else
      pack_t<PANEL_TF32X2, float>(t, b0, nblk, v, sd, se, sw, ch, nchunk, Kp, Km, dp, dm, s, v, sr, V4);
  } else {
    pack_t<PANEL_F64, double>((const double*)t4, b0, nblk, v, sd, se, sw, ch, nchunk, Kp, Km, dp, dm, s, v, sr, V4);
  }
}

}  // namespace rcc
