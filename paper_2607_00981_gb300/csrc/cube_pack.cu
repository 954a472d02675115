// Operand panels read from compact T3 blocks through 16^3 (or 8^3) cubes.
//
// The tensor-core operands of the ring and hh-ladder terms are unpacked T3 blocks
// (Sec. II.C.2): each "piece" of a panel is one stored v^3 block, or a linear
// combination of up to three label permutations of stored blocks (the spin
// summation 2U^{dbc} - U^{bdc} - U^{cbd}), written into the K-major panel.  A
// table-driven gather reads such a block with the virtual axes permuted, which for
// most permutations touches one 32-byte sector per element.  Here a CTA stages a
// cube of the labels in shared memory, reading every source cube along its stored
// unit-stride axis, and writes the panel in runs along K:
//   mode 0  the piece's label L0 runs along K (K = k0 + L0 + L1 ks1) and the rows
//           are row0 + L1 rs1 + L2 rs2 (ring terms: K = (part, l, d), rows (b, c) or
//           (a, c); the panels of step (iii) read from the unpacked batch S);
//   mode 1  each piece is one column (K = k0) of one term and the rows are
//           row0 + L0 v^2 + L1 v + L2 (hh-ladder: K = (l, m), rows (a, b, c)); a CTA
//           takes 16 consecutive columns and an 8^3 cube of rows.
// A term's `pos` packs the stored axis of labels L0, L1, L2 (2 bits each).
#include <cstdint>

#include "elem.cuh"
#include "kernels.h"

namespace rcc {
namespace {

__device__ __forceinline__ int pos_of(int pos, int q) { return (pos >> (2 * q)) & 3; }
__device__ __forceinline__ i64 axis_stride(int axis, int v) {
  return axis == 0 ? (i64)v * v : (axis == 1 ? (i64)v : (i64)1);
}

template <int KIND>
__device__ __forceinline__ void store_run(const CubeDst& d, i64 row, int k, const float (&x)[16], int n, bool vec) {
  // n <= 16 consecutive K values of one row
  if constexpr (KIND == PANEL_BF16X2) {
    __nv_bfloat16* hi = (__nv_bfloat16*)d.out_hi + row * d.Kpad + k;
    __nv_bfloat16* lo = (__nv_bfloat16*)d.out_lo + row * d.Kpad + k;
    if (vec && n == 16) {
      uint32_t h[8], l[8];  // bf16 pairs, first element in the low half
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const __nv_bfloat162 hp = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
        const float2 hf = __bfloat1622float2(hp);
        const __nv_bfloat162 lp = __floats2bfloat162_rn(x[2 * j] - hf.x, x[2 * j + 1] - hf.y);
        h[j] = *reinterpret_cast<const uint32_t*>(&hp);
        l[j] = *reinterpret_cast<const uint32_t*>(&lp);
      }
      ((uint4*)hi)[0] = make_uint4(h[0], h[1], h[2], h[3]);
      ((uint4*)hi)[1] = make_uint4(h[4], h[5], h[6], h[7]);
      ((uint4*)lo)[0] = make_uint4(l[0], l[1], l[2], l[3]);
      ((uint4*)lo)[1] = make_uint4(l[4], l[5], l[6], l[7]);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < n) {
          const __nv_bfloat16 h = __float2bfloat16_rn(x[j]);
          hi[j] = h;
          lo[j] = __float2bfloat16_rn(x[j] - __bfloat162float(h));
        }
    }
  } else {
    float* hi = (float*)d.out_hi + row * d.Kpad + k;
    float* lo = (float*)d.out_lo + row * d.Kpad + k;
    if (vec && n == 16) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          h[j] = tf32_round(x[4 * q + j]);
          l[j] = tf32_round(x[4 * q + j] - h[j]);
        }
        ((float4*)hi)[q] = make_float4(h[0], h[1], h[2], h[3]);
        ((float4*)lo)[q] = make_float4(l[0], l[1], l[2], l[3]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < n) {
          const float h = tf32_round(x[j]);
          hi[j] = h;
          lo[j] = tf32_round(x[j] - h);
        }
    }
  }
}

// Mode 0: grid (label cubes of 16^3, pieces).  Shared: one [16][17][18] cube that
// accumulates the terms one after the other (19 KB, so small enough for the
// register limit, not shared memory, to set the occupancy).
//
// R1 (the variant for the S panels of step (iii)): piece p is the spin-summed block
// S^{xy}[e1][e2][e3] of one z (L0, L1, L2 = e1, e2, e3) and the CTA also forms the
// two partial sums of the T3 term of R1 over its cube,
//   A[e3] = sum_{e1,e2} v^{xy}_{e1 e2} S[e1][e2][e3],  B[e2] = sum_{e1,e3} v^{xy}_{e1 e3} S[e1][e2][e3]
// (w + wbase[p] = v^{xy} as [v][v] floats), written in a fixed order to
// part[(p * cubes + cube) * 32 + (0..15: A, 16..31: B)].
template <int KIND, bool R1>
__global__ void __launch_bounds__(256) k_cube_pack_k(const CubePiece* __restrict__ pieces,
                                                     const CubeDst* __restrict__ dsts, CubeDst d0,
                                                     const float* __restrict__ src, int v,
                                                     const float* __restrict__ w, const i64* __restrict__ wbase,
                                                     float* __restrict__ part) {
  constexpr int TL = 16, CA = (TL + 1) * (TL + 2), CB = TL + 2;
  extern __shared__ __align__(16) float cube_smem[];
  // R1 weights transposed (wAT[e2][e1], wBT[e3][e1]; rows of 20 floats, 16-byte aligned)
  __shared__ __align__(16) float wAT[R1 ? TL : 1][TL + 4], wBT[R1 ? TL : 1][TL + 4];
  __shared__ float red[R1 ? TL : 1][TL + 1];
  const CubePiece& P = pieces[blockIdx.y];
  const int nterm = P.nterm;
  const int nc = (v + TL - 1) / TL;
  const int cb = blockIdx.x;
  const int lo[3] = {(cb / (nc * nc)) * TL, ((cb / nc) % nc) * TL, (cb % nc) * TL};
  const int lf = threadIdx.x & 15, lm = threadIdx.x >> 4;
  if constexpr (R1) {
    // weights v^{xy}_{e1 e2} and v^{xy}_{e1 e3} of this cube (zero outside v)
    const float* wp = w + wbase[blockIdx.y];
    const int e1 = lo[0] + lm;
    wAT[lf][lm] = (e1 < v && lo[1] + lf < v) ? wp[(i64)e1 * v + lo[1] + lf] : 0.f;
    wBT[lf][lm] = (e1 < v && lo[2] + lf < v) ? wp[(i64)e1 * v + lo[2] + lf] : 0.f;
  }
  for (int t = 0; t < nterm; ++t) {
    const int pos = P.t[t].pos;
    const int p0 = pos_of(pos, 0), p1 = pos_of(pos, 1);
    // label on the stored unit-stride axis, then the other two
    const int fast = p0 == 2 ? 0 : (p1 == 2 ? 1 : 2);
    const int mid = fast == 0 ? 1 : 0, slow = 3 - fast - mid;
    // offsets inside one stored block in 32 bits (v^3 < 2^31 for every accepted v)
    const int sm = (int)axis_stride(pos_of(pos, mid), v), ss = (int)axis_stride(pos_of(pos, slow), v);
    const int cf = fast == 0 ? CA : (fast == 1 ? CB : 1), cmid = mid == 0 ? CA : (mid == 1 ? CB : 1),
              cs = slow == 0 ? CA : (slow == 1 ? CB : 1);
    const int xf = (fast == 0 ? lo[0] : fast == 1 ? lo[1] : lo[2]) + lf;
    const int xm = (mid == 0 ? lo[0] : mid == 1 ? lo[1] : lo[2]) + lm;
    const int xs = slow == 0 ? lo[0] : slow == 1 ? lo[1] : lo[2];
    const int nrun = (xf < v && xm < v) ? min(TL, v - xs) : 0;  // valid labels along the slow axis
    const float* s0 = src + P.t[t].base + (xf + xm * sm + xs * ss);
    float ld[TL];
    if (nrun == TL) {
#pragma unroll
      for (int u = 0; u < TL; ++u) ld[u] = __ldg(s0 + u * ss);
    } else {
#pragma unroll
      for (int u = 0; u < TL; ++u) ld[u] = u < nrun ? __ldg(s0 + u * ss) : 0.f;
    }
    float* c = cube_smem + lf * cf + lm * cmid;
    const float coef = P.t[t].coef;
    if (t == 0) {
#pragma unroll
      for (int u = 0; u < TL; ++u) c[u * cs] = fmaf(coef, ld[u], 0.f);
    } else {
      __syncthreads();  // the previous term's updates of these positions are done
#pragma unroll
      for (int u = 0; u < TL; ++u) c[u * cs] = fmaf(coef, ld[u], c[u * cs]);
    }
  }
  __syncthreads();
  // thread (L1, L2) = (lm, lf) writes its row's run of 16 K values (L0)
  const int g1 = lo[1] + lm, g2 = lo[2] + lf;
  float x[TL];
  {
    const float* c = cube_smem + lm * CB + lf;
#pragma unroll
    for (int u = 0; u < TL; ++u) x[u] = nterm > 0 ? c[u * CA] : 0.f;
  }
  if constexpr (R1) {
    // labels outside v hold zeros in the cube, so every thread takes part
    float sa = 0.f, sb = 0.f;
#pragma unroll
    for (int q = 0; q < TL / 4; ++q) {
      const float4 a4 = reinterpret_cast<const float4*>(&wAT[lm][0])[q];
      const float4 b4 = reinterpret_cast<const float4*>(&wBT[lf][0])[q];
      sa = fmaf(a4.x, x[4 * q], sa);
      sa = fmaf(a4.y, x[4 * q + 1], sa);
      sa = fmaf(a4.z, x[4 * q + 2], sa);
      sa = fmaf(a4.w, x[4 * q + 3], sa);
      sb = fmaf(b4.x, x[4 * q], sb);
      sb = fmaf(b4.y, x[4 * q + 1], sb);
      sb = fmaf(b4.z, x[4 * q + 2], sb);
      sb = fmaf(b4.w, x[4 * q + 3], sb);
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) sb += __shfl_xor_sync(0xffffffffu, sb, off);  // over e3 (lf)
    red[lm][lf] = sa;
    __syncthreads();
    float* out = part + ((i64)blockIdx.y * gridDim.x + blockIdx.x) * 32;
    if (threadIdx.x < TL) {  // over e2 (lm), fixed order
      float a = 0.f;
#pragma unroll
      for (int q = 0; q < TL; ++q) a += red[q][threadIdx.x];
      out[threadIdx.x] = a;
    }
    if (lf == 0) out[TL + lm] = sb;
  }
  if (g1 >= v || g2 >= v) return;
  const CubeDst d = dsts ? dsts[P.dst] : d0;
  const int n = min(TL, v - lo[0]);
  const int k = P.k0 + lo[0] + g1 * P.ks1;
  const bool vec = (k & 7) == 0 && (KIND == PANEL_BF16X2 || (k & 3) == 0);
  store_run<KIND>(d, P.row0 + (i64)g1 * P.rs1 + (i64)g2 * P.rs2, k, x, n, vec);
}

// Mode 1: grid (label cubes of 8^3, groups of 16 pieces = 16 consecutive columns).
// The 16 columns' source geometry is decoded once into shared memory, then every
// thread issues its 32 loads (2 elements x 16 columns) before staging any of them.
template <int KIND>
__global__ void __launch_bounds__(256) k_cube_pack_col(const CubePiece* __restrict__ pieces,
                                                       const CubeDst* __restrict__ dsts, CubeDst d0,
                                                       const float* __restrict__ src, int v) {
  constexpr int TL = 8, CS = TL * TL * (TL + 1) + 1;  // one padded 8^3 cube per column
  __shared__ float cols[16 * CS];
  __shared__ i64 g_off[16];
  __shared__ int g_sm[16], g_ss[16];  // strides inside one stored block (v^3 < 2^31)
  __shared__ int g_n[16], g_map[16];
  __shared__ float g_coef[16];
  const int nc = (v + TL - 1) / TL;
  const int cb = blockIdx.x;
  const int lo[3] = {(cb / (nc * nc)) * TL, ((cb / nc) % nc) * TL, (cb % nc) * TL};
  const CubePiece* G = pieces + (i64)blockIdx.y * 16;
  const int tid = threadIdx.x;
  if (tid < 16) {
    const CubePiece& P = G[tid];
    // load order: the label on the stored unit-stride axis (fast), then mid, slow
    const int pos = P.t[0].pos;
    const int p0 = pos_of(pos, 0), p1 = pos_of(pos, 1);
    const int fast = P.nterm > 0 ? (p0 == 2 ? 0 : (p1 == 2 ? 1 : 2)) : 2;
    const int mid = P.nterm > 0 ? (fast == 0 ? 1 : 0) : 1, slow = 3 - fast - mid;
    const i64 sm = axis_stride(pos_of(pos, mid), v), ss = axis_stride(pos_of(pos, slow), v);
    const int lf = fast == 0 ? lo[0] : (fast == 1 ? lo[1] : lo[2]);
    const int lm = mid == 0 ? lo[0] : (mid == 1 ? lo[1] : lo[2]);
    const int ls = slow == 0 ? lo[0] : (slow == 1 ? lo[1] : lo[2]);
    g_off[tid] = P.t[0].base + lf + lm * sm + (i64)ls * ss;
    g_sm[tid] = (int)sm;
    g_ss[tid] = (int)ss;
    // valid extents along fast, mid, slow (8 bits each; 0 for a zero column)
    const int nf = P.nterm > 0 ? min(TL, v - lf) : 0, nm = min(TL, v - lm), ns = min(TL, v - ls);
    g_n[tid] = nf | (nm << 8) | (ns << 16);
    g_map[tid] = fast | (mid << 2) | (slow << 4);  // label of each load coordinate
    g_coef[tid] = P.t[0].coef;
  }
  __syncthreads();
  float ld[16][2];
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const float* base = src + g_off[c];
    const int sm = g_sm[c], ss = g_ss[c];
    const int n = g_n[c];
    const float cf = g_coef[c];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + 256 * h;  // (slow, mid, fast) of 8^3
      const int uf = e & 7, um = (e >> 3) & 7, us = e >> 6;
      const bool ok = uf < (n & 255) && um < ((n >> 8) & 255) && us < (n >> 16);
      ld[c][h] = ok ? cf * __ldg(base + (uf + um * sm + us * ss)) : 0.f;
    }
  }
  // stage by label order (L0, L1, L2), whatever the load order was
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const int mp = g_map[c];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + 256 * h;
      const int u[3] = {e & 7, (e >> 3) & 7, e >> 6};  // fast, mid, slow coordinates
      const int lab_f = mp & 3, lab_m = (mp >> 2) & 3;
      // coordinate of label q: the load coordinate whose label is q
      const int u0 = lab_f == 0 ? u[0] : (lab_m == 0 ? u[1] : u[2]);
      const int u1 = lab_f == 1 ? u[0] : (lab_m == 1 ? u[1] : u[2]);
      const int u2 = lab_f == 2 ? u[0] : (lab_m == 2 ? u[1] : u[2]);
      cols[c * CS + (u0 * TL + u1) * (TL + 1) + u2] = ld[c][h];
    }
  }
  __syncthreads();
  const CubeDst d = dsts ? dsts[G[0].dst] : d0;
  const int k = G[0].k0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = tid + 256 * h;
    const int u0 = e >> 6, u1 = (e >> 3) & 7, u2 = e & 7;
    const int g0 = lo[0] + u0, g1 = lo[1] + u1, g2 = lo[2] + u2;
    if (g0 >= v || g1 >= v || g2 >= v) continue;
    float x[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) x[c] = cols[c * CS + (u0 * TL + u1) * (TL + 1) + u2];
    store_run<KIND>(d, G[0].row0 + ((i64)g0 * v + g1) * v + g2, k, x, 16, true);
  }
}

__global__ void k_zero_cols(CubeDst d, i64 rows, int k0, int esz) {
  const int w = d.Kpad - k0;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < rows * w; i += (i64)gridDim.x * blockDim.x) {
    const i64 r = i / w, k = k0 + i % w;
    if (esz == 2) {
      ((__nv_bfloat16*)d.out_hi)[r * d.Kpad + k] = __float2bfloat16_rn(0.f);
      ((__nv_bfloat16*)d.out_lo)[r * d.Kpad + k] = __float2bfloat16_rn(0.f);
    } else {
      ((float*)d.out_hi)[r * d.Kpad + k] = 0.f;
      ((float*)d.out_lo)[r * d.Kpad + k] = 0.f;
    }
  }
}

}  // namespace

void launch_cube_pack(int mode, int kind, const CubePiece* pieces, int npieces, const CubeDst* dsts,
                      const CubeDst& d0, const float* src, int v, cudaStream_t s) {
  if (npieces <= 0) return;
  if (mode == 0) {
    const int nc = (v + 15) / 16;
    const size_t smem = (size_t)16 * 17 * 18 * sizeof(float);
    dim3 grid((unsigned)(nc * nc * nc), (unsigned)npieces);
    ++g_launch_count;
    if (kind == PANEL_BF16X2)
      k_cube_pack_k<PANEL_BF16X2, false><<<grid, 256, smem, s>>>(pieces, dsts, d0, src, v, nullptr, nullptr, nullptr);
    else
      k_cube_pack_k<PANEL_TF32X2, false><<<grid, 256, smem, s>>>(pieces, dsts, d0, src, v, nullptr, nullptr, nullptr);
  } else {
    const int nc = (v + 7) / 8;
    dim3 grid((unsigned)(nc * nc * nc), (unsigned)(npieces / 16));
    ++g_launch_count;
    if (kind == PANEL_BF16X2)
      k_cube_pack_col<PANEL_BF16X2><<<grid, 256, 0, s>>>(pieces, dsts, d0, src, v);
    else
      k_cube_pack_col<PANEL_TF32X2><<<grid, 256, 0, s>>>(pieces, dsts, d0, src, v);
  }
}

void launch_cube_pack_r1(int kind, const CubePiece* pieces, int npieces, const CubeDst& d0,
                         const float* src, int v, const float* w, const i64* wbase, float* part, cudaStream_t s) {
  if (npieces <= 0) return;
  const int nc = (v + 15) / 16;
  const size_t smem = (size_t)16 * 17 * 18 * sizeof(float);
  dim3 grid((unsigned)(nc * nc * nc), (unsigned)npieces);
  ++g_launch_count;
  if (kind == PANEL_BF16X2)
    k_cube_pack_k<PANEL_BF16X2, true><<<grid, 256, smem, s>>>(pieces, nullptr, d0, src, v, w, wbase, part);
  else
    k_cube_pack_k<PANEL_TF32X2, true><<<grid, 256, smem, s>>>(pieces, nullptr, d0, src, v, w, wbase, part);
}

// dR1[z][a] += sum over the pieces of z and the cubes holding a of A[a] - B[a] / 2
// (the partials of k_cube_pack_k<R1>).  One block per (z, a); each thread sums a
// fixed strided subset in FP64, then a fixed-order tree: deterministic.
__global__ void __launch_bounds__(256) k_r1_cubes_reduce(const float* __restrict__ part, int ppz, int nc, int v,
                                                         double* __restrict__ dR1) {
  __shared__ double acc[256];
  const int z = blockIdx.y, a = blockIdx.x;
  const int ta = a / 16, r = a % 16;
  const int per = nc * nc;  // cubes of one piece whose e3 (or e2) tile is ta
  const i64 total = (i64)ppz * per * 2;
  double s = 0.0;
  for (i64 q = threadIdx.x; q < total; q += blockDim.x) {
    const int kind = (int)(q % 2);
    const i64 rest = q / 2;
    const int c2 = (int)(rest % per);
    const i64 p = (i64)z * ppz + rest / per;
    // cube index (t0, t1, t2) = lo / 16: A needs t2 = ta, B needs t1 = ta
    const int t0 = c2 / nc, tx = c2 % nc;
    const int cube = kind == 0 ? (t0 * nc + tx) * nc + ta : (t0 * nc + ta) * nc + tx;
    const float val = part[(p * (i64)(nc * nc * nc) + cube) * 32 + kind * 16 + r];
    s += kind == 0 ? (double)val : -0.5 * (double)val;
  }
  acc[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) acc[threadIdx.x] += acc[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) dR1[(i64)z * v + a] += acc[0];
}

void launch_r1_cubes_reduce(const float* part, int ppz, int nz, int v, double* dR1, cudaStream_t s) {
  if (ppz <= 0 || nz <= 0) return;
  ++g_launch_count;
  k_r1_cubes_reduce<<<dim3((unsigned)v, (unsigned)nz), 256, 0, s>>>(part, ppz, (v + 15) / 16, v, dR1);
}

void launch_zero_cols(const CubeDst& d, i64 rows, int k0, int kind, cudaStream_t s) {
  if (k0 >= d.Kpad || rows <= 0) return;
  const i64 n = rows * (d.Kpad - k0);
  i64 blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  ++g_launch_count;
  k_zero_cols<<<(unsigned)blocks, 256, 0, s>>>(d, rows, k0, kind == PANEL_BF16X2 ? 2 : 4);
}

}  // namespace rcc
