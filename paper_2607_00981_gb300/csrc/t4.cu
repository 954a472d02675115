// Compact T4 of RCCSDTQ: the W^vv_vv * T4 particle-particle ladder by direct traversal
// (Sec. II.C.4) and the post-processing of R4 (Sec. II.D with the projector of
// appendix B), on the same GEMM engines as the RCCSDT path.
//
// Storage: T4 and R4 hold the occupied quadruples i <= j <= k <= l in colex order,
// blk = C(l+3,4) + C(k+2,3) + C(j+1,2) + i, each a contiguous v^4 block over abcd
// (FP64, or FP32 in the split precisions); W[a][b][e][f] = W^{ab}_{ef} (FP64).
//
// pp-ladder: for a stored block the six terms of Sec. II.C.4 are
//   R[p <- x, q <- y, r <- w1, s <- w2] += sum_ef W^{xy}_{ef} T[p <- e, q <- f, r <- w1, s <- w2]
// over the six position pairs (p, q) of the W labels ((0,1), (0,2), (0,3), (1,2),
// (1,3), (2,3); (r, s) the other two positions in order).  Per term and range of
// stored blocks this is one GEMM: rows (x, y) (M = v^2), columns (blk, w1, w2)
// (N = v^2 per block), K = (e, f) (v^2), with A = W reshaped (the same panel for all
// six terms) and B gathered from the stored blocks through 32 x 32 shared-memory
// tiles (one of f and w2 always runs along the block's unit-stride axis).  The
// table epilogue adds row x, y and column blk, w1, w2 at its place in R4; the six
// terms run one after another on the stream, each GEMM writes every element once.
//
// Post-processing (one pass, out of place): with x o rho the labels of element x
// permuted by rho, out(x) = sum_rho d_rho R(x o rho) where d convolves the projector
// 1 - Pi_[4] - Pi_[3,1] (a class function: 14/24 on the identity, -4/24 on a
// transposition, 2/24 on a double transposition or a 4-cycle, -1/24 on a 3-cycle;
// appendix B) with the average over the block's symmetrisation group (the column
// swaps of its equal occupied indices, Sec. II.D.1); blocks with three equal
// occupied indices are zero (purification).  The pass also sums the squared
// full-tensor norm (block multiplicities 24 / 12 / 6 / 4 / 1) in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/rccsdt.h"
#include "elem.cuh"
#include "kernels.h"

using rcc::i64;

namespace {

constexpr int kPos[6][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2}, {1, 2, 0, 3}, {1, 3, 0, 2}, {2, 3, 0, 1}};

__constant__ unsigned char c_t4perm[24][4];
__constant__ double c_t4coef[5][24];  // per symmetrisation type
__constant__ float c_t4coef_f[5][24];  // the same in FP32 (FP32 storage)

// A panel: A[(x, y)][(e, f)] = W^{xy}_{ef} (W row-major is already [v^2][v^2]).
__global__ void k_t4_pack_w(const double* __restrict__ W, int v, int kind, void* hi, void* lo, int Kpad) {
  const i64 V2 = (i64)v * v, tot = V2 * Kpad;
  for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < tot; x += (i64)gridDim.x * blockDim.x) {
    const i64 r = x / Kpad, k = x - r * Kpad;
    rcc::panel_put(kind, hi, lo, x, k < V2 ? W[r * V2 + k] : 0.0);
  }
}

// B panel of one term for stored blocks b0 .. b0 + nblk - 1:
//   B[((blk - b0) v + w1) v + w2][e v + f] = T[blk][p <- e, q <- f, r <- w1, s <- w2]
// CTA = one (blk, w1); per e it stages the (w2, f) plane in chunks of up to 32 rows
// w2 in shared memory, read along f or w2, whichever has the block's unit stride (one
// always does), and writes each row's run of v K values (f) with 8 values per
// thread (16-byte stores when the run starts on an 8-element boundary); the K
// padding v^2 .. Kpad of its rows is zeroed once.
template <typename T>
__global__ void __launch_bounds__(256) k_t4_pack_t(const T* __restrict__ t4, i64 b0, int nblk, int v, int sp,
                                                   int sq, int sr, int ss, int kind, void* hi, void* lo,
                                                   int Kpad) {
  extern __shared__ __align__(16) unsigned char t4p_smem[];
  T* tile = reinterpret_cast<T*>(t4p_smem);  // [32][v + 1]
  const int P = v + 1;
  const i64 blk = blockIdx.x / v;
  const int w1 = (int)(blockIdx.x - blk * v);
  const i64 V4 = (i64)v * v * v * v, V2 = (i64)v * v;
  const T* base = t4 + (b0 + blk) * V4 + (i64)w1 * sr;
  const bool f_fast = sq == 1;
  const int nf8 = (v + 7) / 8;
  const bool vec = (v & 7) == 0 && (Kpad & 7) == 0;
  for (int e = 0; e < v; ++e) {
    const T* pe = base + (i64)e * sp;
    for (int r0 = 0; r0 < v; r0 += 32) {
      const int nr = min(32, v - r0);
      __syncthreads();  // the previous chunk is written out
      for (int idx = threadIdx.x; idx < nr * v; idx += blockDim.x) {
        int r, f;
        if (f_fast) {
          r = idx / v;
          f = idx - r * v;
        } else {
          f = idx / nr;
          r = idx - f * nr;
        }
        tile[r * P + f] = pe[(i64)f * sq + (i64)(r0 + r) * ss];
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < nr * nf8; idx += blockDim.x) {
        const int r = idx / nf8, f0 = (idx - r * nf8) * 8;
        const i64 o = ((blk * v + w1) * v + r0 + r) * (i64)Kpad + (i64)e * v + f0;
        const T* src = tile + r * P + f0;
        if (vec && kind == rcc::PANEL_BF16X2 && sizeof(T) == 4) {
          uint32_t h[4], l[4];  // bf16 pairs, first element in the low half
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const __nv_bfloat162 hp = __floats2bfloat162_rn((float)src[2 * j], (float)src[2 * j + 1]);
            const float2 hf = __bfloat1622float2(hp);
            const __nv_bfloat162 lp = __floats2bfloat162_rn((float)src[2 * j] - hf.x, (float)src[2 * j + 1] - hf.y);
            h[j] = *reinterpret_cast<const uint32_t*>(&hp);
            l[j] = *reinterpret_cast<const uint32_t*>(&lp);
          }
          *reinterpret_cast<uint4*>((__nv_bfloat16*)hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<uint4*>((__nv_bfloat16*)lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
        } else {
          const int n = min(8, v - f0);
          for (int j = 0; j < n; ++j) {
            if constexpr (sizeof(T) == 4)
              rcc::panel_put_f(kind, hi, lo, o + j, src[j]);
            else
              rcc::panel_put(kind, hi, lo, o + j, src[j]);
          }
        }
      }
    }
  }
  // zero the padding columns K = v^2 .. Kpad of this CTA's v rows
  if (Kpad > V2) {
    const int np = Kpad - (int)V2;
    for (int idx = threadIdx.x; idx < v * np; idx += blockDim.x) {
      const int w2 = idx / np;
      const i64 k = V2 + (idx - w2 * np);
      rcc::panel_put_f(kind, hi, lo, ((blk * v + w1) * v + w2) * (i64)Kpad + k, 0.f);
    }
  }
}

template <typename T>
__device__ __forceinline__ double t4_block_sum(double x, double* ws) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) x += __shfl_xor_sync(0xffffffffu, x, s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
  __syncthreads();
  return t;
}

// Post-processing pass, orbit-tiled: the labels are cut into tiles of 4 (the last
// one ragged); CTA (x, blk) takes the tile quadruples A <= B <= C <= D numbered x,
// x + gridDim.x, ... of stored block blk.  The 24 label permutations map the tiles
// (A, B, C, D) permuted onto one another, so a quadruple's distinct permuted tiles
// (its orbit, at most 24 tiles of 256 elements) hold every input its outputs read:
// they are staged in shared memory once, and each output element of the orbit
// is the 24-term sum over them.  Slot s holds the tile whose position x has tile
// index Q[perm_s(x)]; the input of term p of an output in slot s lies in slot
// (s o p) at the output's local coordinates permuted by p.  Shared strides
// (69, 17, 4, 1) keep every permuted read of a warp within two-way bank conflicts.
// Writes the block's partial squared norm (times the block multiplicity) to
// partial[blk * gridDim.x + x].
constexpr int kT4Tile = 4;
constexpr int kT4S0 = 69, kT4S1 = 17, kT4S2 = 4;
constexpr int kT4Slot = 3 * (kT4S0 + kT4S1 + kT4S2 + 1) + 1;  // 274 elements per staged tile
__constant__ unsigned char c_t4comp[24][24];  // index of the permutation y -> s(p(y))

template <typename T>
__global__ void __launch_bounds__(256) k_t4_post(const T* __restrict__ r, T* __restrict__ out,
                                                 const int4* __restrict__ info, const int4* __restrict__ quads,
                                                 int nq, int v, double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char t4_smem[];
  T* tiles = reinterpret_cast<T*>(t4_smem);
  __shared__ int canon[24];
  __shared__ double ws[8];
  const i64 blk = blockIdx.y;
  const int4 q = info[blk];  // x: coefficient row (5 = purified block), y: multiplicity
  const i64 V4 = (i64)v * v * v * v;
  const T* rb = r + blk * V4;
  T* ob = out + blk * V4;
  const int l = threadIdx.x;
  auto lx = [l](int x) { return (l >> (6 - 2 * x)) & 3; };  // local coordinate of label position x
  const int own = lx(0) * kT4S0 + lx(1) * kT4S1 + lx(2) * kT4S2 + lx(3);
  int paddr[24];
#pragma unroll
  for (int p = 0; p < 24; ++p)
    paddr[p] = lx(c_t4perm[p][0]) * kT4S0 + lx(c_t4perm[p][1]) * kT4S1 + lx(c_t4perm[p][2]) * kT4S2 +
               lx(c_t4perm[p][3]);
  double s = 0.0;
  for (int qi = blockIdx.x; qi < nq; qi += gridDim.x) {
    const int4 Q4 = quads[qi];
    // tile index of label position x (tile indices < 256 since v <= 200)
    const unsigned Qp = (unsigned)Q4.x | ((unsigned)Q4.y << 8) | ((unsigned)Q4.z << 16) | ((unsigned)Q4.w << 24);
    auto Qa = [Qp](int x) { return (int)((Qp >> (8 * x)) & 255u); };
    if (l < 24) {  // first slot with the same tile as slot l
      int c = l;
      for (int u = 0; u < l; ++u) {
        bool same = true;
        for (int x = 0; x < 4; ++x) same &= Qa(c_t4perm[u][x]) == Qa(c_t4perm[l][x]);
        if (same) {
          c = u;
          break;
        }
      }
      canon[l] = c;
    }
    __syncthreads();
    for (int sl = 0; sl < 24; ++sl) {
      if (canon[sl] != sl) continue;
      int g[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) g[x] = kT4Tile * Qa(c_t4perm[sl][x]) + lx(x);
      const bool in = g[0] < v && g[1] < v && g[2] < v && g[3] < v;
      const i64 off = (((i64)g[0] * v + g[1]) * v + g[2]) * v + g[3];
      if (q.x < 5) tiles[sl * kT4Slot + own] = in ? rb[off] : (T)0;
    }
    __syncthreads();
    T qs = (T)0;  // this quadruple's squared outputs, in the storage type
    for (int sl = 0; sl < 24; ++sl) {
      if (canon[sl] != sl) continue;
      int g[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) g[x] = kT4Tile * Qa(c_t4perm[sl][x]) + lx(x);
      T acc = (T)0;
      if (q.x < 5) {
#pragma unroll
        for (int p = 0; p < 24; ++p) {
          T d;
          if constexpr (sizeof(T) == 4) d = c_t4coef_f[q.x][p];
          else d = c_t4coef[q.x][p];
          acc += d * tiles[canon[c_t4comp[sl][p]] * kT4Slot + paddr[p]];
        }
      }
      if (g[0] < v && g[1] < v && g[2] < v && g[3] < v) {
        ob[(((i64)g[0] * v + g[1]) * v + g[2]) * v + g[3]] = acc;
        qs += acc * acc;
      }
    }
    s += (double)qs;
    __syncthreads();  // the next quadruple restages the tiles
  }
  const double bs = t4_block_sum<T>(s, ws);
  if (threadIdx.x == 0) partial[blk * gridDim.x + blockIdx.x] = bs * (double)q.y;
}

// Sum of the partials in a fixed order: 256 strided runs, then a fixed tree.
__global__ void k_t4_reduce(const double* __restrict__ partial, i64 n, double* __restrict__ out) {
  __shared__ double ws[8];
  double s = 0.0;
  for (i64 i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  const double t = t4_block_sum<double>(s, ws);
  if (threadIdx.x == 0) out[0] = t;
}

template <typename TO, typename TI>
__global__ void k_t4_convert(TO* __restrict__ out, const TI* __restrict__ in, i64 n) {
  for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < n; x += (i64)gridDim.x * blockDim.x)
    out[x] = (TO)in[x];
}

unsigned grid_of(i64 n) { return (unsigned)std::max<i64>(1, std::min<i64>((n + 255) / 256, 152 * 32)); }

}  // namespace

struct rccsdt_t4 {
  int o = 0, v = 0, prec = 0, kind = 0, Kpad = 0;
  i64 n4 = 0, V4 = 0, unit = 1;
  cudaStream_t s = nullptr;
  std::vector<void*> allocs;
  void *t4 = nullptr, *r4 = nullptr, *rp4 = nullptr, *stage = nullptr;
  double* W = nullptr;
  void *Ahi = nullptr, *Alo = nullptr, *Bhi = nullptr, *Blo = nullptr;
  i64* rowbase = nullptr;   // [6][v^2]
  i64* coloff = nullptr;    // [6][n4 v^2]
  int* rowsel = nullptr;
  double* alpha = nullptr;
  int4* info = nullptr;
  double* partial = nullptr;
  int4* quads = nullptr;    // tile quadruples A <= B <= C <= D of the post-processing pass
  int nq = 0, qgrid = 1;
  double* scal = nullptr;   // [0] squared norm, [8..] watchdog flag (int)
  float* splitk = nullptr;
  i64 splitk_elems = 0;
  bool have_w = false, have_t = false, have_r = false;
  std::string err;
  ~rccsdt_t4() {
    for (void* p : allocs) cudaFree(p);
  }
  void* alloc(size_t bytes, bool* ok) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
      *ok = false;
      cudaGetLastError();
      return nullptr;
    }
    allocs.push_back(p);
    return p;
  }
  int fail(int code, const std::string& m) {
    err = m;
    return code;
  }
};

namespace {

void t4_tables_once() {
  static bool done = false;
  if (done) return;
  std::vector<std::array<int, 4>> perms;
  std::array<int, 4> p = {0, 1, 2, 3};
  do perms.push_back(p);
  while (std::next_permutation(p.begin(), p.end()));
  auto index_of = [&](const std::array<int, 4>& q) {
    for (int i = 0; i < 24; ++i)
      if (perms[i] == q) return i;
    return -1;
  };
  // projector coefficient by cycle type (class function): fixed points decide it here
  double proj[24];
  for (int i = 0; i < 24; ++i) {
    int fixed = 0;
    for (int x = 0; x < 4; ++x) fixed += perms[i][x] == x;
    const int chi31 = fixed - 1;  // character of [3,1]
    proj[i] = (i == 0 ? 1.0 : 0.0) - 1.0 / 24.0 - 3.0 / 24.0 * chi31;
  }
  // symmetrisation groups: none, swap (0 1), swap (1 2), swap (2 3), swaps (0 1) and (2 3)
  const std::vector<std::vector<std::array<int, 4>>> groups = {
      {{0, 1, 2, 3}},
      {{0, 1, 2, 3}, {1, 0, 2, 3}},
      {{0, 1, 2, 3}, {0, 2, 1, 3}},
      {{0, 1, 2, 3}, {0, 1, 3, 2}},
      {{0, 1, 2, 3}, {1, 0, 2, 3}, {0, 1, 3, 2}, {1, 0, 3, 2}}};
  double coef[5][24] = {};
  for (int g = 0; g < 5; ++g)
    for (int i = 0; i < 24; ++i)
      for (const auto& h : groups[g]) {
        std::array<int, 4> rho;  // (pi o h)(x) = pi(h(x))
        for (int x = 0; x < 4; ++x) rho[x] = perms[i][h[x]];
        coef[g][index_of(rho)] += proj[i] / (double)groups[g].size();
      }
  unsigned char hp[24][4], comp[24][24];
  for (int i = 0; i < 24; ++i)
    for (int x = 0; x < 4; ++x) hp[i][x] = (unsigned char)perms[i][x];
  for (int a = 0; a < 24; ++a)
    for (int b = 0; b < 24; ++b) {
      std::array<int, 4> ab;  // y -> a(b(y))
      for (int y = 0; y < 4; ++y) ab[y] = perms[a][perms[b][y]];
      comp[a][b] = (unsigned char)index_of(ab);
    }
  cudaMemcpyToSymbol(c_t4perm, hp, sizeof(hp));
  cudaMemcpyToSymbol(c_t4comp, comp, sizeof(comp));
  cudaMemcpyToSymbol(c_t4coef, coef, sizeof(coef));
  float coef_f[5][24];
  for (int g = 0; g < 5; ++g)
    for (int i = 0; i < 24; ++i) coef_f[g][i] = (float)coef[g][i];
  cudaMemcpyToSymbol(c_t4coef_f, coef_f, sizeof(coef_f));
  done = true;
}

template <typename T>
int t4_copy_in(rccsdt_t4* c, void* dst, const double* src, i64 n) {
  if (std::is_same<T, double>::value)
    return cudaMemcpyAsync(dst, src, (size_t)n * 8, cudaMemcpyDefault, c->s) == cudaSuccess ? 0 : 1;
  // FP32 storage: stage FP64 chunks and convert
  const i64 chunk = (i64)32 << 20;
  for (i64 off = 0; off < n; off += chunk) {
    const i64 len = std::min(chunk, n - off);
    if (cudaMemcpyAsync(c->stage, src + off, (size_t)len * 8, cudaMemcpyDefault, c->s) != cudaSuccess) return 1;
    ++rcc::g_launch_count;
    k_t4_convert<float, double><<<grid_of(len), 256, 0, c->s>>>((float*)dst + off, (const double*)c->stage, len);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) return 1;
  }
  return 0;
}

}  // namespace

#define RCC_API extern "C" __attribute__((visibility("default")))

RCC_API int rccsdt_t4_create(int o, int v, int precision, void* stream, rccsdt_t4** out) {
  if (!out) return RCCSDT_ERR_ARG;
  *out = nullptr;
  if (o < 1 || v < 1 || o > 32 || v > 200 || precision < 0 || precision > 2) return RCCSDT_ERR_ARG;
  auto* c = new rccsdt_t4();
  c->o = o;
  c->v = v;
  c->prec = precision;
  c->kind = precision == RCCSDT_FP64 ? rcc::PANEL_F64 : (precision == RCCSDT_SPLIT_BF16X3 ? rcc::PANEL_BF16X2
                                                                                          : rcc::PANEL_TF32X2);
  c->n4 = (i64)o * (o + 1) * (o + 2) * (o + 3) / 24;
  const i64 V2 = (i64)v * v;
  c->V4 = V2 * V2;
  c->s = (cudaStream_t)stream;
  c->Kpad = (int)((V2 + 63) / 64 * 64);
  const size_t es = precision == RCCSDT_FP64 ? 8 : 4;
  const size_t pe = precision == RCCSDT_FP64 ? 8 : (precision == RCCSDT_SPLIT_BF16X3 ? 2 : 4);
  // blocks per B panel: about 1 GiB of FP64-sized panel
  const i64 per_blk = V2 * c->Kpad * 8;
  c->unit = std::max<i64>(1, std::min<i64>(c->n4, ((i64)1 << 30) / per_blk));
  bool ok = true;
  c->t4 = c->alloc(c->n4 * c->V4 * es, &ok);
  c->r4 = c->alloc(c->n4 * c->V4 * es, &ok);
  c->rp4 = c->alloc(c->n4 * c->V4 * es, &ok);
  c->stage = c->alloc(precision == RCCSDT_FP64 ? 16 : ((size_t)32 << 20) * 8, &ok);
  c->W = (double*)c->alloc(c->V4 * 8, &ok);
  c->Ahi = c->alloc(V2 * c->Kpad * pe, &ok);
  c->Alo = c->alloc(precision == RCCSDT_FP64 ? 16 : V2 * c->Kpad * pe, &ok);
  c->Bhi = c->alloc(c->unit * V2 * c->Kpad * pe, &ok);
  c->Blo = c->alloc(precision == RCCSDT_FP64 ? 16 : c->unit * V2 * c->Kpad * pe, &ok);
  c->rowbase = (i64*)c->alloc(6 * V2 * 8, &ok);
  c->coloff = (i64*)c->alloc(6 * c->n4 * V2 * 8, &ok);
  c->rowsel = (int*)c->alloc(std::max<i64>(V2, c->unit * V2) * 4, &ok);
  c->alpha = (double*)c->alloc(std::max<i64>(V2, c->unit * V2) * 8, &ok);
  c->info = (int4*)c->alloc(c->n4 * sizeof(int4), &ok);
  const int ntile = (v + kT4Tile - 1) / kT4Tile;
  c->nq = (int)((i64)ntile * (ntile + 1) * (ntile + 2) * (ntile + 3) / 24);
  c->qgrid = std::max(1, std::min(c->nq, 64));
  c->quads = (int4*)c->alloc((size_t)c->nq * sizeof(int4), &ok);
  c->partial = (double*)c->alloc(c->n4 * c->qgrid * 8, &ok);
  c->scal = (double*)c->alloc(64 * 8, &ok);
  c->splitk_elems = (i64)8 << 20;
  c->splitk = (float*)c->alloc((size_t)c->splitk_elems * 8, &ok);
  if (!ok) {
    delete c;
    return RCCSDT_ERR_OOM;
  }
  // tables: strides of the four label positions in a v^4 block
  const i64 st[4] = {V2 * v, V2, (i64)v, 1};
  std::vector<i64> rb(6 * V2), co((size_t)6 * c->n4 * V2);
  for (int t = 0; t < 6; ++t) {
    const int p = kPos[t][0], q = kPos[t][1], r = kPos[t][2], s = kPos[t][3];
    for (int x = 0; x < v; ++x)
      for (int y = 0; y < v; ++y) rb[t * V2 + x * v + y] = x * st[p] + y * st[q];
    for (i64 b = 0; b < c->n4; ++b)
      for (int w1 = 0; w1 < v; ++w1)
        for (int w2 = 0; w2 < v; ++w2) co[(size_t)t * c->n4 * V2 + (b * v + w1) * v + w2] = b * c->V4 + w1 * st[r] + w2 * st[s];
  }
  // per block: x = the coefficient row of the post-processing pass (0 none, 1 swap of
  // columns 1 2, 2 of 2 3, 3 of 3 4, 4 both 1 2 and 3 4; 5 = a purified block), y = the
  // number of occupied quadruples the block stands for
  std::vector<int4> info;
  for (int l = 0; l < o; ++l)
    for (int k = 0; k <= l; ++k)
      for (int j = 0; j <= k; ++j)
        for (int i = 0; i <= j; ++i) {
          int type, mult;
          if ((i == j && j == k) || (j == k && k == l)) {
            type = 5;
            mult = (i == l) ? 1 : 4;
          } else if (i == j && k == l) {
            type = 4;
            mult = 6;
          } else if (i == j || j == k || k == l) {
            type = i == j ? 1 : (j == k ? 2 : 3);
            mult = 12;
          } else {
            type = 0;
            mult = 24;
          }
          info.push_back(make_int4(type, mult, 0, 0));
        }
  std::vector<int4> quads;
  for (int D = 0; D < ntile; ++D)
    for (int C = 0; C <= D; ++C)
      for (int B = 0; B <= C; ++B)
        for (int A = 0; A <= B; ++A) quads.push_back(make_int4(A, B, C, D));
  std::vector<int> sel(std::max<i64>(V2, c->unit * V2), 0);
  std::vector<double> al(std::max<i64>(V2, c->unit * V2), 1.0);
  bool cp = cudaMemcpy(c->rowbase, rb.data(), rb.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->coloff, co.data(), co.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->info, info.data(), info.size() * sizeof(int4), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->quads, quads.data(), quads.size() * sizeof(int4), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->rowsel, sel.data(), sel.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->alpha, al.data(), al.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemset(c->scal, 0, 64 * 8) == cudaSuccess;
  if (!cp) {
    cudaGetLastError();
    delete c;
    return RCCSDT_ERR_CUDA;
  }
  t4_tables_once();
  if (cudaFuncSetAttribute(k_t4_post<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 24 * kT4Slot * 8) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_t4_pack_t<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 32 * (200 + 1) * 8) !=
          cudaSuccess) {
    cudaGetLastError();
    delete c;
    return RCCSDT_ERR_CUDA;
  }
  *out = c;
  return RCCSDT_OK;
}

RCC_API int rccsdt_t4_set(rccsdt_t4* c, const double* W, const double* t4c) {
  if (!c) return RCCSDT_ERR_ARG;
  if (W) {
    if (cudaMemcpyAsync(c->W, W, (size_t)c->V4 * 8, cudaMemcpyDefault, c->s) != cudaSuccess)
      return c->fail(RCCSDT_ERR_CUDA, "copy of W failed");
    ++rcc::g_launch_count;
    k_t4_pack_w<<<grid_of((i64)c->v * c->v * c->Kpad), 256, 0, c->s>>>(c->W, c->v, c->kind, c->Ahi, c->Alo,
                                                                        c->Kpad);
    c->have_w = true;
  }
  if (t4c) {
    const int st = c->prec == RCCSDT_FP64 ? t4_copy_in<double>(c, c->t4, t4c, c->n4 * c->V4)
                                          : t4_copy_in<float>(c, c->t4, t4c, c->n4 * c->V4);
    if (st) return c->fail(RCCSDT_ERR_CUDA, "copy of T4 failed");
    c->have_t = true;
  }
  if (cudaStreamSynchronize(c->s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return c->fail(RCCSDT_ERR_CUDA, "rccsdt_t4_set failed");
  return RCCSDT_OK;
}

RCC_API int rccsdt_t4_pp_ladder(rccsdt_t4* c) {
  if (!c) return RCCSDT_ERR_ARG;
  if (!c->have_w || !c->have_t) return c->fail(RCCSDT_ERR_STATE, "W or T4 not set");
  const int v = c->v;
  const i64 V2 = (i64)v * v;
  const size_t es = c->prec == RCCSDT_FP64 ? 8 : 4;
  if (cudaMemsetAsync(c->r4, 0, (size_t)(c->n4 * c->V4 * es), c->s) != cudaSuccess)
    return c->fail(RCCSDT_ERR_CUDA, "memset failed");
  cudaMemsetAsync(c->scal, 0, 64 * 8, c->s);
  const i64 st[4] = {V2 * v, V2, (i64)v, 1};
  int* flag = (int*)(c->scal + 8);
  for (int t = 0; t < 6; ++t) {
    const int p = kPos[t][0], q = kPos[t][1], r = kPos[t][2], s = kPos[t][3];
    for (i64 b0 = 0; b0 < c->n4; b0 += c->unit) {
      const int nblk = (int)std::min<i64>(c->unit, c->n4 - b0);
      const i64 ncta = (i64)nblk * v;
      const size_t tsm = (size_t)32 * (v + 1);
      ++rcc::g_launch_count;
      if (c->prec == RCCSDT_FP64)
        k_t4_pack_t<double><<<(unsigned)ncta, 256, tsm * 8, c->s>>>((const double*)c->t4, b0, nblk, v, (int)st[p],
                                                                     (int)st[q], (int)st[r], (int)st[s], c->kind,
                                                                     c->Bhi, c->Blo, c->Kpad);
      else
        k_t4_pack_t<float><<<(unsigned)ncta, 256, tsm * 4, c->s>>>((const float*)c->t4, b0, nblk, v, (int)st[p],
                                                                    (int)st[q], (int)st[r], (int)st[s], c->kind,
                                                                    c->Bhi, c->Blo, c->Kpad);
      rcc::EpiArgs e{};
      e.C = c->r4;
      e.c_f32 = c->prec != RCCSDT_FP64;
      e.M = (int)V2;
      e.N = (int)(nblk * V2);
      e.row_base = c->rowbase + t * V2;
      e.row_sel = c->rowsel;
      e.row_alpha = c->alpha;
      e.col_off = c->coloff + (size_t)t * c->n4 * V2 + b0 * V2;
      if (c->prec == RCCSDT_FP64) {
        rcc::launch_gemm_f64((const double*)c->Ahi, (const double*)c->Bhi, (int)((V2 + 15) / 16 * 16), c->Kpad,
                             c->Kpad, e, (double*)c->splitk, c->splitk_elems, c->s);
      } else if (rcc::launch_gemm_tc(c->kind, c->Ahi, c->Alo, c->Bhi, c->Blo, c->Kpad, e, flag, 0, c->s, c->splitk,
                                     c->splitk_elems * 2, nullptr, e.N <= 128 ? 128 : 256)) {
        return c->fail(RCCSDT_ERR_ARG, "tensor-core GEMM configuration unsupported");
      }
    }
  }
  int hf = 0;
  if (cudaMemcpyAsync(&hf, flag, 4, cudaMemcpyDeviceToHost, c->s) != cudaSuccess ||
      cudaStreamSynchronize(c->s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return c->fail(RCCSDT_ERR_CUDA, "pp-ladder failed");
  if (hf) return c->fail(RCCSDT_ERR_TIMEOUT, "a device-side wait exceeded its watchdog budget");
  c->have_r = true;
  return RCCSDT_OK;
}

RCC_API int rccsdt_t4_postprocess(rccsdt_t4* c, double* norm) {
  if (!c) return RCCSDT_ERR_ARG;
  if (!c->have_r) return c->fail(RCCSDT_ERR_STATE, "R4 not computed");
  const i64 ncta = c->n4 * c->qgrid;
  const dim3 grid((unsigned)c->qgrid, (unsigned)c->n4);
  ++rcc::g_launch_count;
  if (c->prec == RCCSDT_FP64)
    k_t4_post<double><<<grid, 256, 24 * kT4Slot * 8, c->s>>>((const double*)c->r4, (double*)c->rp4, c->info,
                                                             c->quads, c->nq, c->v, c->partial);
  else
    k_t4_post<float><<<grid, 256, 24 * kT4Slot * 4, c->s>>>((const float*)c->r4, (float*)c->rp4, c->info,
                                                            c->quads, c->nq, c->v, c->partial);
  ++rcc::g_launch_count;
  k_t4_reduce<<<1, 256, 0, c->s>>>(c->partial, ncta, c->scal);
  std::swap(c->r4, c->rp4);
  double h = 0.0;
  if (cudaMemcpyAsync(&h, c->scal, 8, cudaMemcpyDeviceToHost, c->s) != cudaSuccess ||
      cudaStreamSynchronize(c->s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return c->fail(RCCSDT_ERR_CUDA, "post-processing failed");
  if (!std::isfinite(h)) return c->fail(RCCSDT_ERR_NONFINITE, "non-finite R4 norm");
  if (norm) *norm = std::sqrt(h);
  return RCCSDT_OK;
}

RCC_API int rccsdt_t4_get_r4(rccsdt_t4* c, double* r4c) {
  if (!c || !r4c) return RCCSDT_ERR_ARG;
  const i64 n = c->n4 * c->V4;
  if (c->prec == RCCSDT_FP64) {
    if (cudaMemcpyAsync(r4c, c->r4, (size_t)n * 8, cudaMemcpyDefault, c->s) != cudaSuccess)
      return c->fail(RCCSDT_ERR_CUDA, "copy failed");
  } else {
    const i64 chunk = (i64)32 << 20;
    for (i64 off = 0; off < n; off += chunk) {
      const i64 len = std::min(chunk, n - off);
      ++rcc::g_launch_count;
      k_t4_convert<double, float><<<grid_of(len), 256, 0, c->s>>>((double*)c->stage, (const float*)c->r4 + off, len);
      if (cudaMemcpyAsync(r4c + off, c->stage, (size_t)len * 8, cudaMemcpyDefault, c->s) != cudaSuccess ||
          cudaStreamSynchronize(c->s) != cudaSuccess)
        return c->fail(RCCSDT_ERR_CUDA, "copy failed");
    }
  }
  return cudaStreamSynchronize(c->s) == cudaSuccess ? RCCSDT_OK : c->fail(RCCSDT_ERR_CUDA, "copy failed");
}

RCC_API const char* rccsdt_t4_last_error(const rccsdt_t4* c) { return c ? c->err.c_str() : "null T4 engine"; }

RCC_API void rccsdt_t4_destroy(rccsdt_t4* c) {
  if (!c) return;
  cudaStreamSynchronize(c->s);
  delete c;
}
