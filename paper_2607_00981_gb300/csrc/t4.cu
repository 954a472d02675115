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
// (1,3), (2,3); (r, s) the other two positions in order).  W is pair-symmetric
// (W^{xy}_{ef} = W^{yx}_{fe}), so each term runs as the sum and difference products of
// the RCCSDT pp-ladder: per term and range of stored blocks two GEMMs with K over the
// label pairs e <= f (sum) and e < f (difference), rows the pairs x <= y and x < y of
// W+ / W- (one panel pair for all six terms), columns (blk, w1, w2), B the T+ / T-
// panels gathered from the stored blocks; each product is added half to (x, y) and
// half, with its part's sign, to (y, x).  Half the multiply-adds of the plain
// v^2 x v^2 product.  Where the block's unit-stride label is free (s = 3) the GEMMs
// run with the operands exchanged and write R4 from the epilogue (both writes run
// along w2); otherwise the unit-stride label is y, the mirrored writes would run
// across it, so in the split precisions the GEMMs write their raw products and
// k_t4_pair_scatter combines both parts per 16 x 16 label tile, writing 64-byte runs
// for (x, y) and (y, x) (FP64 keeps the epilogue's writes).
// The six terms run one after another on the stream.
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
#include <utility>
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
// they are staged in shared memory once.  Slot s holds the tile whose position x has
// tile index Q[perm_s(x)].  Thread l takes the element e of slot 0 at local
// coordinates l and its orbit {e o s}: it reads the 24 values v_s = R(e o s) once
// (slot s at l's coordinates permuted by s), forms out(e o s) = sum_p d_p v_(s o p)
// for every distinct slot s (24 x 24 multiply-adds in registers, the permutation
// indices compile-time constants), and writes them back into the staged tiles in
// place; the tiles are then stored to R4 along the unit-stride axis.  Each output
// element of a distinct slot comes from exactly one thread (l -> l o s is a
// bijection), so the pass is deterministic.  Shared strides (69, 17, 4, 1) keep every
// permuted access of a warp within two-way bank conflicts.  Writes the block's
// partial squared norm (times the block multiplicity) to partial[blk * gridDim.x + x].
constexpr int kT4Tile = 4;
constexpr int kT4S0 = 69, kT4S1 = 17, kT4S2 = 4;
constexpr int kT4Slot = 3 * (kT4S0 + kT4S1 + kT4S2 + 1) + 1;  // 274 elements per staged tile

// The 24 permutations of (0, 1, 2, 3) in lexicographic order (the order of the
// coefficient tables) and their composition, as compile-time constants.
__host__ __device__ constexpr int t4_perm(int i, int x) {
  int n = 0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c)
        for (int d = 0; d < 4; ++d)
          if (a != b && a != c && a != d && b != c && b != d && c != d) {
            if (n == i) return x == 0 ? a : (x == 1 ? b : (x == 2 ? c : d));
            ++n;
          }
  return -1;
}
__host__ __device__ constexpr int t4_comp(int i, int j) {  // index of y -> perm_i(perm_j(y))
  for (int k = 0; k < 24; ++k) {
    bool eq = true;
    for (int y = 0; y < 4; ++y) eq = eq && t4_perm(k, y) == t4_perm(i, t4_perm(j, y));
    if (eq) return k;
  }
  return -1;
}
template <int I, int J>
constexpr int kT4Comp = t4_comp(I, J);
template <int I, int X>
constexpr int kT4Perm = t4_perm(I, X);
static_assert(kT4Comp<5, 0> == 5 && kT4Comp<0, 7> == 7 && kT4Perm<23, 0> == 3, "permutation tables");

// staged address of slot-local coordinates l permuted by permutation I
template <int I>
__device__ __forceinline__ int t4_paddr(const int (&lx)[4]) {
  return lx[kT4Perm<I, 0>] * kT4S0 + lx[kT4Perm<I, 1>] * kT4S1 + lx[kT4Perm<I, 2>] * kT4S2 + lx[kT4Perm<I, 3>];
}

template <typename T, int S, int... P>
__device__ __forceinline__ T t4_orbit_out(const T (&vv)[24], const T (&d)[24], std::integer_sequence<int, P...>) {
  T acc = (T)0;
  ((acc += d[P] * vv[kT4Comp<S, P>]), ...);
  return acc;
}

template <typename T, int... S>
__device__ __forceinline__ void t4_orbit_read(T (&vv)[24], const T* tiles, const int* canon, const int (&lx)[4],
                                              std::integer_sequence<int, S...>) {
  ((vv[S] = tiles[canon[S] * kT4Slot + t4_paddr<S>(lx)]), ...);
}

template <typename T, int... S>
__device__ __forceinline__ void t4_orbit_write(const T (&vv)[24], const T (&d)[24], T* tiles, const int* canon,
                                               const int (&lx)[4], std::integer_sequence<int, S...>) {
  ((canon[S] == S ? (void)(tiles[S * kT4Slot + t4_paddr<S>(lx)] =
                               t4_orbit_out<T, S>(vv, d, std::make_integer_sequence<int, 24>{}))
                  : (void)0),
   ...);
}

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
  const int lx[4] = {(l >> 6) & 3, (l >> 4) & 3, (l >> 2) & 3, l & 3};  // local coordinate of label position x
  const int own = lx[0] * kT4S0 + lx[1] * kT4S1 + lx[2] * kT4S2 + lx[3];
  T d[24];  // this block's coefficients (uniform over the CTA)
#pragma unroll
  for (int p = 0; p < 24; ++p) {
    if constexpr (sizeof(T) == 4) d[p] = q.x < 5 ? c_t4coef_f[q.x][p] : 0.f;
    else d[p] = q.x < 5 ? c_t4coef[q.x][p] : 0.0;
  }
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
    if (q.x < 5) {
      for (int sl = 0; sl < 24; ++sl) {
        if (canon[sl] != sl) continue;
        int g[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) g[x] = kT4Tile * Qa(c_t4perm[sl][x]) + lx[x];
        const bool in = g[0] < v && g[1] < v && g[2] < v && g[3] < v;
        const i64 off = (((i64)g[0] * v + g[1]) * v + g[2]) * v + g[3];
        tiles[sl * kT4Slot + own] = in ? rb[off] : (T)0;
      }
      __syncthreads();
      T vv[24];
      t4_orbit_read<T>(vv, tiles, canon, lx, std::make_integer_sequence<int, 24>{});
      __syncthreads();  // every orbit read before the outputs overwrite the tiles
      t4_orbit_write<T>(vv, d, tiles, canon, lx, std::make_integer_sequence<int, 24>{});
      __syncthreads();
    }
    T qs = (T)0;  // this quadruple's squared outputs, in the storage type
    for (int sl = 0; sl < 24; ++sl) {
      if (canon[sl] != sl) continue;
      int g[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) g[x] = kT4Tile * Qa(c_t4perm[sl][x]) + lx[x];
      const T val = q.x < 5 ? tiles[sl * kT4Slot + own] : (T)0;
      if (g[0] < v && g[1] < v && g[2] < v && g[3] < v) {
        ob[(((i64)g[0] * v + g[1]) * v + g[2]) * v + g[3]] = val;
        qs += val * val;
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

// Second phase of a ladder term whose GEMM wrote its sum and difference products raw
// (column-major: P[n][m] over the sum pairs, M[n][m] over the difference pairs, n =
// (blk, w1, w2) of the range): per column and chunk of 16-label tiles, both parts are
// staged as full 16 x 16 tiles, then thread (r, c) adds
//   R(d0 + r, e0 + c) += (P + M) / 2 at pair (r, c) and R(e0 + r, d0 + c) += (P - M) / 2
// at pair (c, r) (a diagonal chunk: the one element (r, c), from the pair with r <= c).
// Consecutive threads run along c, the label at the second W position, so the writes
// are 64-byte runs when that position has unit stride.  Chunks and columns write
// disjoint elements (no atomics).
constexpr int kT4ScCols = 8;
__global__ void __launch_bounds__(256, 3) k_t4_pair_scatter(const float* __restrict__ P, const float* __restrict__ M,
                                                         int Kp, int Km, const rcc::PairChunk* __restrict__ ch,
                                                         int v, const i64* __restrict__ colo, i64 sp, i64 sq,
                                                         i64 N, float* __restrict__ r4) {
  __shared__ float SP[kT4ScCols][16][17], SM[kT4ScCols][16][17];
  const rcc::PairChunk c = ch[blockIdx.x];
  const int d0 = c.P * 16, e0 = c.Q * 16;
  const int nd = min(16, v - d0), ne = min(16, v - e0);
  const bool diag = c.P == c.Q;
  const int np = diag ? nd * (nd + 1) / 2 : nd * ne;
  const int nm = diag ? nd * (nd - 1) / 2 : nd * ne;
  const int t = threadIdx.x;
  int ap = 0, bp = 0, am = 0, bm = 0;
  if (t < np) rcc::pair_decode(t, diag, true, nd, ne, ap, bp);
  if (t < nm) rcc::pair_decode(t, diag, false, nd, ne, am, bm);
  const int r = t >> 4, q = t & 15;
  for (i64 n0 = (i64)blockIdx.y * kT4ScCols; n0 < N; n0 += (i64)gridDim.y * kT4ScCols) {
    const int ncol = (int)min((i64)kT4ScCols, N - n0);
    __syncthreads();  // the previous group's tiles are consumed
    {
      float vp[kT4ScCols], vm[kT4ScCols];
#pragma unroll
      for (int j = 0; j < kT4ScCols; ++j) {
        const i64 n = n0 + j;
        vp[j] = (j < ncol && t < np) ? __ldg(P + n * Kp + c.offp + t) : 0.f;
        vm[j] = (j < ncol && t < nm) ? __ldg(M + n * Km + c.offm + t) : 0.f;
      }
#pragma unroll
      for (int j = 0; j < kT4ScCols; ++j) {
        if (t < np) SP[j][ap][bp] = vp[j];
        if (t < nm) SM[j][am][bm] = vm[j];
      }
    }
    __syncthreads();
    // all read-modify-write loads of the group first (independent, in flight together)
    i64 base[kT4ScCols];
    const bool w1 = diag ? (r < nd && q < nd) : (r < nd && q < ne);
    const bool w2 = !diag && r < ne && q < nd;
    const i64 off1 = (i64)(d0 + r) * sp + (i64)((diag ? d0 : e0) + q) * sq;
    const i64 off2 = (i64)(e0 + r) * sp + (i64)(d0 + q) * sq;
#pragma unroll
    for (int j = 0; j < kT4ScCols; ++j) base[j] = j < ncol ? __ldg(colo + n0 + j) : 0;
    float o[kT4ScCols];
    // the (d, e) elements: loads of the group in flight together, then the stores
#pragma unroll
    for (int j = 0; j < kT4ScCols; ++j) o[j] = (j < ncol && w1) ? r4[base[j] + off1] : 0.f;
#pragma unroll
    for (int j = 0; j < kT4ScCols; ++j) {
      const float x = !diag || r < q ? 0.5f * (SP[j][r][q] + SM[j][r][q])
                                     : (r > q ? 0.5f * (SP[j][q][r] - SM[j][q][r]) : 0.5f * SP[j][r][r]);
      if (j < ncol && w1) r4[base[j] + off1] = o[j] + x;
    }
    // the mirrored (e, d) elements of an off-diagonal chunk
    if (w2) {
#pragma unroll
      for (int j = 0; j < kT4ScCols; ++j) o[j] = j < ncol ? r4[base[j] + off2] : 0.f;
#pragma unroll
      for (int j = 0; j < kT4ScCols; ++j)
        if (j < ncol) r4[base[j] + off2] = o[j] + 0.5f * (SP[j][q][r] - SM[j][q][r]);
    }
  }
}

template <typename TO, typename TI>
__global__ void k_t4_convert(TO* __restrict__ out, const TI* __restrict__ in, i64 n) {
  for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < n; x += (i64)gridDim.x * blockDim.x)
    out[x] = (TO)in[x];
}

unsigned grid_of(i64 n) { return (unsigned)std::max<i64>(1, std::min<i64>((n + 255) / 256, 152 * 32)); }

}  // namespace

struct rccsdt_t4 {
  int o = 0, v = 0, prec = 0, kind = 0;
  i64 n4 = 0, V4 = 0, unit = 1;
  cudaStream_t s = nullptr;
  std::vector<void*> allocs;
  void *t4 = nullptr, *r4 = nullptr, *rp4 = nullptr, *stage = nullptr;
  double* W = nullptr;
  void *Ahi = nullptr, *Alo = nullptr, *Bhi = nullptr, *Blo = nullptr;
  i64* coloff = nullptr;    // [6][n4 v^2]: R4 offset of column (blk, w1, w2) of each term
  // pair-symmetric ladder (W^{ab}_{ef} = W^{ba}_{fe}): sum and difference panels over the
  // label pairs; K numbered by chunks of 16-label tiles, rows x <= y (sum), x < y (difference)
  rcc::PairChunk* pchunks = nullptr;
  int nchunk = 0, Kp = 0, Km = 0, Kpadp = 0, Kpadm = 0;
  int4* prows = nullptr;    // [Kp] (x, y, row of (x, y) among the difference pairs or -1)
  i64* prb = nullptr;       // [6][2][Kp] R4 offset of (x, y) at the term's W label positions
  i64* prb2 = nullptr;      // the mirrored (y, x); -1 on the diagonal
  i64 nal = 0;              // rows of the alpha and selector tables: max(Kp, unit v^2)
  double* pal = nullptr;    // [2][nal] 1/2
  double* pal2 = nullptr;   // [2][nal] +1/2 (sum), -1/2 (difference)
  int* psel = nullptr;      // [nal] zeros
  float* raw = nullptr;     // split kinds: raw sum and difference products of one range, [unit v^2][Kp + Km]
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
  unsigned char hp[24][4];  // lexicographic, as t4_perm (the kernel's compile-time tables)
  for (int i = 0; i < 24; ++i)
    for (int x = 0; x < 4; ++x) hp[i][x] = (unsigned char)perms[i][x];
  cudaMemcpyToSymbol(c_t4perm, hp, sizeof(hp));
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
  const size_t es = precision == RCCSDT_FP64 ? 8 : 4;
  const size_t pe = precision == RCCSDT_FP64 ? 8 : (precision == RCCSDT_SPLIT_BF16X3 ? 2 : 4);
  // pair numbering (16-label tiles P <= Q; inside a chunk as pair_decode describes)
  std::vector<rcc::PairChunk> ch;
  {
    const int nt = (v + 15) / 16;
    int offp = 0, offm = 0;
    for (int P = 0; P < nt; ++P)
      for (int Q = P; Q < nt; ++Q) {
        const int nd = std::min(16, v - 16 * P), ne = std::min(16, v - 16 * Q);
        const bool diag = P == Q;
        ch.push_back({P, Q, offp, offm});
        offp += diag ? nd * (nd + 1) / 2 : nd * ne;
        offm += diag ? nd * (nd - 1) / 2 : nd * ne;
      }
    c->nchunk = (int)ch.size();
    c->Kp = offp;
    c->Km = offm;
    c->Kpadp = (offp + 63) / 64 * 64;
    c->Kpadm = (offm + 63) / 64 * 64;
  }
  // blocks per B panel: about 1 GiB of FP64-sized panel, and at most 65535 (block, w1)
  // pairs (the pair gather's grid)
  const i64 kcols = c->Kpadp + std::max(c->Kpadm, 64);
  const i64 per_blk = V2 * kcols * 8;
  c->unit = std::max<i64>(1, std::min<i64>(std::min<i64>(c->n4, ((i64)1 << 30) / per_blk), 65535 / v));
  bool ok = true;
  c->t4 = c->alloc(c->n4 * c->V4 * es, &ok);
  c->r4 = c->alloc(c->n4 * c->V4 * es, &ok);
  c->rp4 = c->alloc(c->n4 * c->V4 * es, &ok);
  c->stage = c->alloc(precision == RCCSDT_FP64 ? 16 : ((size_t)32 << 20) * 8, &ok);
  c->W = (double*)c->alloc(c->V4 * 8, &ok);
  const i64 abytes = ((i64)c->Kp * c->Kpadp + (i64)c->Km * c->Kpadm) * (i64)pe;
  const i64 bbytes = c->unit * V2 * kcols * (i64)pe;
  c->Ahi = c->alloc(abytes, &ok);
  c->Alo = c->alloc(precision == RCCSDT_FP64 ? 16 : abytes, &ok);
  c->Bhi = c->alloc(bbytes, &ok);
  c->Blo = c->alloc(precision == RCCSDT_FP64 ? 16 : bbytes, &ok);
  c->coloff = (i64*)c->alloc(6 * c->n4 * V2 * 8, &ok);
  c->pchunks = (rcc::PairChunk*)c->alloc(ch.size() * sizeof(rcc::PairChunk), &ok);
  c->prows = (int4*)c->alloc((size_t)c->Kp * sizeof(int4), &ok);
  c->prb = (i64*)c->alloc((size_t)12 * c->Kp * 8, &ok);
  c->prb2 = (i64*)c->alloc((size_t)12 * c->Kp * 8, &ok);
  c->nal = std::max<i64>(c->Kp, std::min(c->n4, c->unit) * V2);
  c->pal = (double*)c->alloc((size_t)2 * c->nal * 8, &ok);
  c->pal2 = (double*)c->alloc((size_t)2 * c->nal * 8, &ok);
  c->psel = (int*)c->alloc((size_t)c->nal * 4, &ok);
  if (precision != RCCSDT_FP64) c->raw = (float*)c->alloc((size_t)(c->unit * V2) * (c->Kp + c->Km) * 4, &ok);
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
  // rows of both parts in the K order of the chunks (pair_decode inside a chunk), so the
  // raw products' row index is the pair's K index: sum rows x <= y, difference rows x < y
  std::vector<std::array<int, 2>> rp, rm;
  std::vector<int> mrow((size_t)V2, -1);
  for (const rcc::PairChunk& q : ch) {
    const int nd = std::min(16, v - 16 * q.P), ne = std::min(16, v - 16 * q.Q);
    const bool diag = q.P == q.Q;
    const int np = diag ? nd * (nd + 1) / 2 : nd * ne, nm = diag ? nd * (nd - 1) / 2 : nd * ne;
    for (int t = 0; t < np; ++t) {
      int a, b;
      rcc::pair_decode(t, diag, true, nd, ne, a, b);
      rp.push_back({16 * q.P + a, 16 * q.Q + b});
    }
    for (int t = 0; t < nm; ++t) {
      int a, b;
      rcc::pair_decode(t, diag, false, nd, ne, a, b);
      mrow[(size_t)(16 * q.P + a) * v + 16 * q.Q + b] = (int)rm.size();
      rm.push_back({16 * q.P + a, 16 * q.Q + b});
    }
  }
  std::vector<int4> prows(rp.size());
  for (size_t m = 0; m < rp.size(); ++m) prows[m] = make_int4(rp[m][0], rp[m][1], mrow[(size_t)rp[m][0] * v + rp[m][1]], 0);
  std::vector<i64> prb((size_t)12 * c->Kp, -1), prb2((size_t)12 * c->Kp, -1), co((size_t)6 * c->n4 * V2);
  std::vector<double> pal((size_t)2 * c->nal, 0.5), pal2((size_t)2 * c->nal, 0.5);
  for (i64 m = 0; m < c->nal; ++m) pal2[(size_t)(c->nal + m)] = -0.5;
  for (int t = 0; t < 6; ++t) {
    const int p = kPos[t][0], q = kPos[t][1], r = kPos[t][2], s = kPos[t][3];
    for (int part = 0; part < 2; ++part) {
      const auto& pr = part == 0 ? rp : rm;
      i64* b1 = prb.data() + (size_t)(t * 2 + part) * c->Kp;
      i64* b2 = prb2.data() + (size_t)(t * 2 + part) * c->Kp;
      for (size_t m = 0; m < pr.size(); ++m) {
        const i64 x = pr[m][0], y = pr[m][1];
        b1[m] = x * st[p] + y * st[q];
        b2[m] = x == y ? -1 : y * st[p] + x * st[q];
      }
    }
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
  std::vector<int> sel((size_t)c->nal, 0);
  bool cp = cudaMemcpy(c->coloff, co.data(), co.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->pchunks, ch.data(), ch.size() * sizeof(rcc::PairChunk), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->prows, prows.data(), prows.size() * sizeof(int4), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->prb, prb.data(), prb.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->prb2, prb2.data(), prb2.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->pal, pal.data(), pal.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->pal2, pal2.data(), pal2.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->psel, sel.data(), sel.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->info, info.data(), info.size() * sizeof(int4), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(c->quads, quads.data(), quads.size() * sizeof(int4), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemset(c->scal, 0, 64 * 8) == cudaSuccess;
  if (!cp) {
    cudaGetLastError();
    delete c;
    return RCCSDT_ERR_CUDA;
  }
  t4_tables_once();
  if (cudaFuncSetAttribute(k_t4_post<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 24 * kT4Slot * 8) !=
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
    // W+ / W- panels (both parts side by side in the A buffers)
    const size_t pe = c->prec == RCCSDT_FP64 ? 8 : (c->prec == RCCSDT_SPLIT_BF16X3 ? 2 : 4);
    const size_t aoff = (size_t)c->Kp * c->Kpadp * pe;
    const rcc::CubeDst Ap{c->Ahi, c->prec == RCCSDT_FP64 ? nullptr : c->Alo, c->Kpadp};
    const rcc::CubeDst Am{(char*)c->Ahi + aoff, c->prec == RCCSDT_FP64 ? nullptr : (char*)c->Alo + aoff, c->Kpadm};
    rcc::launch_pair_pack_w(c->kind, c->W, c->v, c->prows, c->Kp, c->pchunks, c->nchunk, c->Kp, c->Km, Ap, Am, c->s);
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
  const bool f64 = c->prec == RCCSDT_FP64;
  const size_t pe = f64 ? 8 : (c->prec == RCCSDT_SPLIT_BF16X3 ? 2 : 4);
  const size_t aoff = (size_t)c->Kp * c->Kpadp * pe;
  for (int t = 0; t < 6; ++t) {
    const int p = kPos[t][0], q = kPos[t][1], r = kPos[t][2], s = kPos[t][3];
    for (i64 b0 = 0; b0 < c->n4; b0 += c->unit) {
      const int nblk = (int)std::min<i64>(c->unit, c->n4 - b0);
      const i64 N = nblk * V2;
      // T+ / T- panels of this view: rows (blk, w1, w2), K the pairs of the labels at p, q
      const size_t boff = (size_t)N * c->Kpadp * pe;
      char* bh = (char*)c->Bhi;
      char* bl = f64 ? nullptr : (char*)c->Blo;
      const rcc::CubeDst Bp{bh, bl, c->Kpadp}, Bm{bh + boff, bl ? bl + boff : nullptr, c->Kpadm};
      rcc::launch_pair_pack_t4(c->kind, c->t4, f64 ? 0 : 1, b0, nblk, v, st[p], st[q], st[s], st[r], c->pchunks,
                               c->nchunk, c->Kp, c->Km, Bp, Bm, c->s);
      for (int part = 0; part < 2; ++part) {
        const int K = part ? c->Km : c->Kp, Kpad = part ? c->Kpadm : c->Kpadp;
        if (K == 0) continue;
        // With the unit-stride label free (s = 3) the operands are exchanged: rows
        // (blk, w1, w2), so an epilogue warp's 32 rows are 32 consecutive elements for both
        // the (x, y) write and its mirror (the column mirror); otherwise rows are the pairs
        // and the direct write runs along y at unit stride.
        const bool swap = s == 3;
        const i64* pb = c->prb + (size_t)(t * 2 + part) * c->Kp;
        const i64* pb2 = c->prb2 + (size_t)(t * 2 + part) * c->Kp;
        const i64* co = c->coloff + (size_t)t * c->n4 * V2 + b0 * V2;
        rcc::EpiArgs e{};
        e.C = c->r4;
        e.c_f32 = f64 ? 0 : 1;
        e.row_sel = c->psel;
        e.row_alpha = c->pal + (size_t)part * c->nal;
        e.row_alpha2 = c->pal2 + (size_t)part * c->nal;
        if (swap) {
          e.M = (int)N;
          e.N = K;
          e.row_base = co;
          e.col_off = pb;
          e.col_off2 = pb2;
        } else {
          e.M = K;
          e.N = (int)N;
          e.row_base = pb;
          e.row_base2 = pb2;
          e.col_off = co;
        }
        const char* wh = (const char*)c->Ahi + (part ? aoff : 0);
        const char* wl = f64 ? nullptr : (const char*)c->Alo + (part ? aoff : 0);
        const char* th = bh + (part ? boff : 0);
        const char* tl = bl ? bl + (part ? boff : 0) : nullptr;
        const char* ah = swap ? th : wh;
        const char* al = swap ? tl : wl;
        const char* bhp = swap ? wh : th;
        const char* blp = swap ? wl : tl;
        if (f64) {
          rcc::launch_gemm_f64((const double*)ah, (const double*)bhp, (K + 15) / 16 * 16, Kpad, Kpad, e,
                               (double*)c->splitk, c->splitk_elems, c->s);
        } else if (rcc::launch_gemm_tc(c->kind, ah, al, bhp, blp, Kpad, e, flag, 0, c->s, c->splitk,
                                       c->splitk_elems * 2, swap ? nullptr : c->raw + (part ? N * c->Kp : 0), 256,
                                       1)) {
          return c->fail(RCCSDT_ERR_ARG, "tensor-core GEMM configuration unsupported");
        }
      }
      if (!f64 && s != 3) {
        // raw products of both parts -> R4 (the direct epilogue's mirrored writes would
        // run across the unit-stride label)
        ++rcc::g_launch_count;
        k_t4_pair_scatter<<<dim3((unsigned)c->nchunk, (unsigned)std::min<i64>(65535, (N + kT4ScCols - 1) / kT4ScCols)),
                            256, 0, c->s>>>(
            c->raw, c->raw + N * c->Kp, c->Kp, c->Km, c->pchunks, v, c->coloff + (size_t)t * c->n4 * V2 + b0 * V2,
            st[p], st[q], N, (float*)c->r4);
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
