// RCCSDT(Q): the perturbative quadruples energy correction on the converged
// amplitudes of a context, evaluated by the ABC-based algorithm of Sec. II.E.2.
//
// The energy of Eq. ener-pt-q,
//   E_(Q) = 1/24 sum_{ijkl,abcd} z_{ijkl}^{abcd} t~_{ijkl}^{abcd}  (t~ fully spin summed),
// with t = r / eps (Eq. orb-energy-deno), r = P(X + Y), z = P(X + V) (Eq. resi-pt-q;
// P the sum over the 24 joint permutations of the column pairs, Eq. rcc-perm-op) and
// X, Y, V of Eq. q_t3_terms, is restricted, as in Eq. ener-pt-q-abc, to sorted virtual
// quadruples a <= b <= c <= d weighted by their degeneracy factor (24 / 12 / 6, and 0
// when three or four labels are equal).  Y uses the alternative intermediates of
// Eq. q_w_alter (the ABC-based form):
//   Wbar^{abc}_{ejk} = P_(jb)(kc) ( -sum_m v^{mb}_{ej} t^{ac}_{mk} - sum_m v^{ma}_{je} t^{bc}_{mk}
//                                   + 1/2 sum_f v^{ab}_{ef} t^{fc}_{jk} ),
//   Wbar^{abm}_{ijk} = P_(ia)(jb) ( -1/2 sum_n v^{mn}_{ki} t^{ab}_{nj} ),
// and every integral is the BARE v^{pq}_{rs} = (pr|qs) (T1 does not enter).
//
// GPU design (one GB300):
//   1. k_q_eri: (pq|rs) from the factors once (n^4, FP64);
//   2. k_q_t3v: the one-time transposition of compact T3 from the occupied-triangular
//      layout (i <= j <= k, v^3 blocks) to the virtual-triangular one (a <= b <= c,
//      o^3 blocks, Fig. q_operation_counts(a)), so that a task's amplitudes t^{xyz}
//      for fixed labels are o^3 contiguous values;
//   3. k_q_layout / k_q_wbar1 / k_q_wbar2: the integrals and Wbar in the layouts the
//      main kernel reads with its summation index innermost;
//   4. k_q_main: a persistent grid; each CTA takes sorted quadruples in a fixed
//      round-robin order and, per quadruple, (a) accumulates R = P(X + Y) and
//      Z = P(X + V) for all o^4 occupied tuples in shared memory (each thread owns
//      tuples; per joint permutation sigma two sums over v and two over o), then
//      (b) forms t~ from R at the 24 occupied permutations (the spin summation is a
//      class function of the virtual permutation, and t^{L o pi}_{O} = t^{L}_{O o pi^-1}
//      by the joint column symmetry) and adds f_abcd sum Z t~ to its FP64 partial;
//   5. k_q_reduce: the partials in index order (deterministic).
// Arithmetic: FP64 throughout, or FP32 operands and dot products with FP64
// partial sums of the energy (option `arith`).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/rccsdt.h"
#include "internal.h"
#include "kernels.h"

namespace {

using rcc::i64;

constexpr int kThreadsQ = 256;
constexpr int kMaxVQ = 256;  // largest v of the (Q) kernels (per-CTA tables)

// The 24 permutations of four positions (sigma[x] = source position of position x)
__constant__ unsigned char c_perm[24][4];
// spin summation: t~(O, L) = sum_pi c_pi R(O o pi^-1, L) / eps; per pi the inverse map and c_pi
__constant__ unsigned char c_pinv[24][4];
__constant__ double c_coef[24];

__host__ __device__ __forceinline__ i64 tri3(i64 a, i64 b, i64 c) {  // colex a <= b <= c
  return c * (c + 1) * (c + 2) / 6 + b * (b + 1) / 2 + a;
}

// Offset of t^{xyz}_{alpha beta gamma} in the virtual-triangular layout
// [tri3(sorted labels)][occupied of the smallest label][middle][largest].
__device__ __forceinline__ i64 t3v_off(int x, int y, int z, int al, int be, int ga, int o) {
  if (x > y) { int t = x; x = y; y = t; t = al; al = be; be = t; }
  if (y > z) { int t = y; y = z; z = t; t = be; be = ga; ga = t; }
  if (x > y) { int t = x; x = y; y = t; t = al; al = be; be = t; }
  return tri3(x, y, z) * o * o * o + ((i64)al * o + be) * o + ga;
}

// 1. chemists' ERIs G[p][q][r][s] = (pq|rs) = sum_P L[P][p][q] L[P][r][s]
__global__ void k_q_eri(const double* __restrict__ L, int naux, int n, double* __restrict__ G) {
  const i64 n2 = (i64)n * n, tot = n2 * n2;
  for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < tot; x += (i64)gridDim.x * blockDim.x) {
    const i64 pq = x / n2, rs = x - pq * n2;
    double s = 0.0;
    for (int P = 0; P < naux; ++P) s += L[P * n2 + pq] * L[P * n2 + rs];
    G[x] = s;
  }
}

// 2. virtual-triangular T3: out[tri3(a<=b<=c)][i][j][k] = t^{abc}_{ijk}, read from the
// compact occupied-triangular t3c[tri3(i<=j<=k)][x][y][z] = t^{xyz}_{ijk}
template <typename S, typename T>
__global__ void k_q_t3v(const S* __restrict__ t3c, int o, int v, const int4* __restrict__ vtrip, i64 nv3,
                        T* __restrict__ out) {
  const i64 o3 = (i64)o * o * o, V3 = (i64)v * v * v, tot = nv3 * o3;
  for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < tot; x += (i64)gridDim.x * blockDim.x) {
    const i64 blk = x / o3;
    int r = (int)(x - blk * o3);
    int k = r % o, j = (r / o) % o, i = r / (o * o);
    const int4 lab = vtrip[blk];
    int a = lab.x, b = lab.y, c = lab.z;
    // sort the (occupied, label) pairs by the occupied index
    if (i > j) { int t = i; i = j; j = t; t = a; a = b; b = t; }
    if (j > k) { int t = j; j = k; k = t; t = b; b = c; c = t; }
    if (i > j) { int t = i; i = j; j = t; t = a; a = b; b = t; }
    out[x] = (T)t3c[tri3(i, j, k) * V3 + ((i64)a * v + b) * v + c];
  }
}

// 3a. main-kernel layouts of integrals and t2 (G and t2 FP64; output T)
//   kind 0: A1[p][q][j][e]    = v^{pq}_{ej} = (pe|qj)
//   kind 1: A2[p][i][j][m]    = v^{pm}_{ij} = (pi|mj)
//   kind 2: Vv[p][q][i][j]    = v^{pq}_{ij} = (pi|qj)
//   kind 3: T2e[i][l][s][e]   = t^{es}_{il} = t2[i][l][e][s]
//   kind 4: T2m[l][r][s][m]   = t^{rs}_{ml} = t2[m][l][r][s]
//   kind 5: T2v[k][l][r][s]   = t^{rs}_{kl} = t2[k][l][r][s]
template <typename T>
__global__ void k_q_layout(int kind, const double* __restrict__ G, const double* __restrict__ t2, int o, int v,
                           T* __restrict__ out, i64 tot) {
  const int n = o + v;
  const i64 n1 = n, n2 = n1 * n, n3 = n2 * n;
  for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < tot; x += (i64)gridDim.x * blockDim.x) {
    double val;
    if (kind == 0) {  // [p][q][j][e]
      const int e = (int)(x % v), j = (int)((x / v) % o), q = (int)((x / ((i64)v * o)) % v),
                p = (int)(x / ((i64)v * o * v));
      val = G[(o + p) * n3 + (o + e) * n2 + (o + q) * n1 + j];
    } else if (kind == 1) {  // [p][i][j][m]
      const int m = (int)(x % o), j = (int)((x / o) % o), i = (int)((x / ((i64)o * o)) % o),
                p = (int)(x / ((i64)o * o * o));
      val = G[(o + p) * n3 + i * n2 + m * n1 + j];
    } else if (kind == 2) {  // [p][q][i][j]
      const int j = (int)(x % o), i = (int)((x / o) % o), q = (int)((x / ((i64)o * o)) % v),
                p = (int)(x / ((i64)o * o * v));
      val = G[(o + p) * n3 + i * n2 + (o + q) * n1 + j];
    } else if (kind == 3) {  // [i][l][s][e]
      const int e = (int)(x % v), s = (int)((x / v) % v), l = (int)((x / ((i64)v * v)) % o),
                i = (int)(x / ((i64)v * v * o));
      val = t2[(((i64)i * o + l) * v + e) * v + s];
    } else if (kind == 4) {  // [l][r][s][m]
      const int m = (int)(x % o), s = (int)((x / o) % v), r = (int)((x / ((i64)o * v)) % v),
                l = (int)(x / ((i64)o * v * v));
      val = t2[(((i64)m * o + l) * v + r) * v + s];
    } else {  // [k][l][r][s]
      val = t2[x];
    }
    out[x] = (T)val;
  }
}

// 3b. W1[p][q][r][j][k][e] = Wbar^{pqr}_{ejk} = w(p,q,r; e,j,k) + w(p,r,q; e,k,j), with
//   w(a,b,c; e,j,k) = -sum_m v^{mb}_{ej} t^{ac}_{mk} - sum_m v^{ma}_{je} t^{bc}_{mk}
//                     + 1/2 sum_f v^{ab}_{ef} t^{fc}_{jk}
// (v^{mb}_{ej} = (me|bj), v^{ma}_{je} = (mj|ae), v^{ab}_{ef} = (ae|bf)); arithmetic in T,
// on ERI and t2 copies of T's precision (FP32: converted once, so that the sums do no
// per-product conversions on the FP64 units).
template <typename T, typename TI>
__device__ __forceinline__ T q_w1(const TI* __restrict__ G, const TI* __restrict__ t2, int o, int v, int a,
                                  int b, int c, int e, int j, int k) {
  const int n = o + v;
  const i64 n1 = n, n2 = n1 * n, n3 = n2 * n;
  const i64 V2 = (i64)v * v;
  T s = 0;
  for (int m = 0; m < o; ++m) {
    s -= (T)G[m * n3 + (o + e) * n2 + (o + b) * n1 + j] * (T)t2[((i64)m * o + k) * V2 + (i64)a * v + c];
    s -= (T)G[m * n3 + j * n2 + (o + a) * n1 + (o + e)] * (T)t2[((i64)m * o + k) * V2 + (i64)b * v + c];
  }
  T h = 0;
  for (int f = 0; f < v; ++f)
    h += (T)G[(o + a) * n3 + (o + e) * n2 + (o + b) * n1 + (o + f)] * (T)t2[((i64)j * o + k) * V2 + (i64)f * v + c];
  return s + (T)0.5 * h;
}

template <typename T, typename TI>  // TI: the type of the ERI and t2 copies read (T's precision)
__global__ void k_q_wbar1(const TI* __restrict__ G, const TI* __restrict__ t2, int o, int v,
                          T* __restrict__ W1) {
  const i64 tot = (i64)v * v * v * o * o * v;
  for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < tot; x += (i64)gridDim.x * blockDim.x) {
    const int e = (int)(x % v);
    i64 r = x / v;
    const int k = (int)(r % o);
    r /= o;
    const int j = (int)(r % o);
    r /= o;
    const int c = (int)(r % v);
    r /= v;
    const int b = (int)(r % v), a = (int)(r / v);
    W1[x] = q_w1<T, TI>(G, t2, o, v, a, b, c, e, j, k) + q_w1<T, TI>(G, t2, o, v, a, c, b, e, k, j);
  }
}

// 3c. W2[p][q][i][j][k][m] = Wbar^{pqm}_{ijk} = w2(p,q,m; i,j,k) + w2(q,p,m; j,i,k),
//   w2(a,b,m; i,j,k) = -1/2 sum_n v^{mn}_{ki} t^{ab}_{nj}   (v^{mn}_{ki} = (mk|ni))
template <typename T, typename TI>
__global__ void k_q_wbar2(const TI* __restrict__ G, const TI* __restrict__ t2, int o, int v,
                          T* __restrict__ W2) {
  const int n = o + v;
  const i64 n1 = n, n2 = n1 * n, n3 = n2 * n, V2 = (i64)v * v;
  const i64 tot = V2 * o * o * o * o;
  for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < tot; x += (i64)gridDim.x * blockDim.x) {
    const int m = (int)(x % o);
    i64 r = x / o;
    const int k = (int)(r % o);
    r /= o;
    const int j = (int)(r % o);
    r /= o;
    const int i = (int)(r % o);
    r /= o;
    const int b = (int)(r % v), a = (int)(r / v);
    T s = 0;
    for (int q = 0; q < o; ++q) {
      s += (T)G[m * n3 + k * n2 + q * n1 + i] * (T)t2[((i64)q * o + j) * V2 + (i64)a * v + b];
      s += (T)G[m * n3 + k * n2 + q * n1 + j] * (T)t2[((i64)q * o + i) * V2 + (i64)b * v + a];
    }
    W2[x] = (T)-0.5 * s;
  }
}

struct QArgs {
  const int4* quads;   // sorted (a, b, c, d) with a nonzero degeneracy factor (w = factor)
  i64 nquad;
  int o, v;
  const double* eps;   // Fock diagonal, occupied first
  const void* t3v;
  const void* A1;
  const void* A2;
  const void* Vv;
  const void* W1;
  const void* W2;
  const void* T2e;
  const void* T2m;
  const void* T2v;
  void* scratch;       // [gridDim][2][o^4] when R and Z do not fit shared memory
  int smem_rz;         // 1: R and Z in shared memory
  double* partial;     // [gridDim]
};

__device__ __forceinline__ double block_sum_q(double x, double* ws) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) x += __shfl_xor_sync(0xffffffffu, x, s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) ws[wid] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
  return t;  // valid in thread 0
}

// Position pair {x, y} (x < y) of the quadruple's labels -> index 0..5.
__device__ __forceinline__ int pair_index(int x, int y) {
  // (0,1) 0, (0,2) 1, (0,3) 2, (1,2) 3, (1,3) 4, (2,3) 5
  return x == 0 ? y - 1 : (x == 1 ? y + 1 : 5);
}

template <typename T>
__global__ void __launch_bounds__(kThreadsQ) k_q_main(const QArgs q) {
  extern __shared__ unsigned char q_smem[];
  __shared__ double ws[32];
  // per label-position pair {x < y} and summation label e: the element offset (block
  // index times o^3) of the stored block sorted(e, L[x], L[y]); the rank of e in that
  // triple, which fixes the occupied order, follows from the range of e
  __shared__ i64 s_blk[6][kMaxVQ];
  const int o = q.o, v = q.v;
  const i64 O4 = (i64)o * o * o * o;
  T* R = q.smem_rz ? (T*)q_smem : (T*)q.scratch + (i64)blockIdx.x * 2 * O4;
  T* Z = R + O4;
  const T* t3v = (const T*)q.t3v;
  const T* A1 = (const T*)q.A1;
  const T* A2 = (const T*)q.A2;
  const T* Vv = (const T*)q.Vv;
  const T* W1 = (const T*)q.W1;
  const T* W2 = (const T*)q.W2;
  const T* T2e = (const T*)q.T2e;
  const T* T2m = (const T*)q.T2m;
  const T* T2v = (const T*)q.T2v;
  const i64 o2 = (i64)o * o, o3 = o2 * o;
  double total = 0.0;
  for (i64 qi = blockIdx.x; qi < q.nquad; qi += gridDim.x) {
    const int4 L4 = q.quads[qi];
    const int L[4] = {L4.x & 0xffff, L4.x >> 16, L4.y & 0xffff, L4.y >> 16};
    const double fac = (double)L4.z;
    __syncthreads();  // s_blk of the previous quadruple is consumed
    for (int t = threadIdx.x; t < 6 * v; t += blockDim.x) {
      const int pi = t / v, e = t % v;
      const int x = pi < 3 ? 0 : (pi < 5 ? 1 : 2), y = pi < 3 ? pi + 1 : (pi < 5 ? pi - 1 : 3);
      const int r0 = L[x], s0 = L[y];  // r0 <= s0 (L is sorted)
      const i64 b = e <= r0 ? tri3(e, r0, s0) : (e <= s0 ? tri3(r0, e, s0) : tri3(r0, s0, e));
      s_blk[pi][e] = b * o3;
    }
    __syncthreads();
    // (a) R = P(X + Y), Z = P(X + V) for every occupied tuple
    for (i64 el = threadIdx.x; el < O4; el += blockDim.x) {
      const int Oc[4] = {(int)(el / o3), (int)((el / o2) % o), (int)((el / o) % o), (int)(el % o)};
      T rr = 0, zz = 0;
      for (int sg = 0; sg < 24; ++sg) {
        const int c0 = c_perm[sg][0], c1 = c_perm[sg][1], c2 = c_perm[sg][2], c3 = c_perm[sg][3];
        const int p = L[c0], qq = L[c1], r = L[c2], s = L[c3];
        const int i = Oc[c0], j = Oc[c1], k = Oc[c2], l = Oc[c3];
        // X: 1/2 sum_e v^{pq}_{ej} t^{ers}_{ikl} - 1/2 sum_m v^{pm}_{ij} t^{qrs}_{mkl}
        // t^{ers}_{ikl}: sorted triple (e, r0, s0) | (r0, e, s0) | (r0, s0, e) by the range of e,
        // (r0, s0) = the pair's labels in position order with their occupied indices (k0, l0)
        const bool rs = c2 < c3;
        const int r0 = rs ? r : s, s0 = rs ? s : r, k0 = rs ? k : l, l0 = rs ? l : k;
        const i64* bt = s_blk[pair_index(rs ? c2 : c3, rs ? c3 : c2)];
        const T* a1 = A1 + (((i64)p * v + qq) * o + j) * v;
        T x1 = 0;
        {
          const i64 f0 = ((i64)i * o + k0) * o + l0, f1 = ((i64)k0 * o + i) * o + l0, f2 = ((i64)k0 * o + l0) * o + i;
          int e = 0;
          for (; e <= r0; ++e) x1 += a1[e] * t3v[bt[e] + f0];
          for (; e <= s0; ++e) x1 += a1[e] * t3v[bt[e] + f1];
          for (; e < v; ++e) x1 += a1[e] * t3v[bt[e] + f2];
        }
        const T* a2 = A2 + (((i64)p * o + i) * o + j) * o;
        const i64 b0 = t3v_off(qq, r, s, 0, k, l, o), bm = t3v_off(qq, r, s, 1, k, l, o) - b0;
        T x2 = 0;
        for (int m = 0; m < o; ++m) x2 += a2[m] * t3v[b0 + m * bm];
        // Y: 1/2 sum_e Wbar^{pqr}_{ejk} t^{es}_{il} - 1/2 sum_m Wbar^{pqm}_{ijk} t^{rs}_{ml}
        const T* w1 = W1 + ((((i64)p * v + qq) * v + r) * o2 + (i64)j * o + k) * v;
        const T* t2e = T2e + (((i64)i * o + l) * v + s) * v;
        T y1 = 0;
        for (int e = 0; e < v; ++e) y1 += w1[e] * t2e[e];
        const T* w2 = W2 + ((((i64)p * v + qq) * o + i) * o2 + (i64)j * o + k) * o;
        const T* t2m = T2m + (((i64)l * v + r) * v + s) * o;
        T y2 = 0;
        for (int m = 0; m < o; ++m) y2 += w2[m] * t2m[m];
        // V: 1/4 v^{pq}_{ij} t^{rs}_{kl}
        const T vv = Vv[(((i64)p * v + qq) * o + i) * o + j] * T2v[(((i64)k * o + l) * v + r) * v + s];
        const T X = (T)0.5 * (x1 - x2);
        rr += X + (T)0.5 * (y1 - y2);
        zz += X + (T)0.25 * vv;
      }
      R[el] = rr;
      Z[el] = zz;
    }
    __syncthreads();
    // (b) f_abcd sum_O Z(O) t~(O), t~(O) = sum_pi c_pi R(O o pi^-1) / eps(O)
    const double ev = q.eps[o + L[0]] + q.eps[o + L[1]] + q.eps[o + L[2]] + q.eps[o + L[3]];
    double part = 0.0;
    for (i64 el = threadIdx.x; el < O4; el += blockDim.x) {
      const int Oc[4] = {(int)(el / o3), (int)((el / o2) % o), (int)((el / o) % o), (int)(el % o)};
      double ts = 0.0;
      for (int pi = 0; pi < 24; ++pi) {
        const i64 idx = (((i64)Oc[c_pinv[pi][0]] * o + Oc[c_pinv[pi][1]]) * o + Oc[c_pinv[pi][2]]) * o +
                        Oc[c_pinv[pi][3]];
        ts += c_coef[pi] * (double)R[idx];
      }
      const double eo = q.eps[Oc[0]] + q.eps[Oc[1]] + q.eps[Oc[2]] + q.eps[Oc[3]];
      part += (double)Z[el] * ts / (eo - ev);
    }
    const double bs = block_sum_q(part, ws);
    if (threadIdx.x == 0) total += fac * bs;
  }
  if (threadIdx.x == 0) q.partial[blockIdx.x] = total;
}

// Operand-staged variant of k_q_main (FP32, o <= 16, everything in shared memory).  Per joint
// permutation sigma the four sums of phase (a) are small products: with the labels
// (p, q, r, s) = sigma(L) fixed, a thread owns an occupied triple (i, k, l) and forms
// the sums for all o values of j at once, so that each gathered T3 / t2 value feeds o
// FMAs; the W / integral slices of this sigma, which every thread reads, are staged in
// shared memory first ([e][j], [k][e][j], [i][m][j], [i][k][m][j], [i][j]: j innermost).
// Each sum is written into R / Z at the occupied tuple O with O[c_x] = (i, j, k, l)_x.
// Phase (b) is the same as in k_q_main.
constexpr int kMaxOQ = 16;

struct QStage {  // element offsets of the staged slices in the dynamic shared memory
  int a1, w1, a2, w2, vs, w2_staged;
  i64 total;  // elements (R, Z and the slices)
};

__host__ __device__ inline i64 q_pad4(i64 x) { return (x + 3) & ~(i64)3; }

__host__ __device__ inline QStage q_stage_layout(int o, int v) {
  const i64 o2 = (i64)o * o, o4 = o2 * o2;
  QStage L;
  i64 off = 2 * q_pad4(o4);
  L.a1 = (int)off;
  off += q_pad4((i64)v * o);
  L.w1 = (int)off;
  off += q_pad4((i64)o * v * o);
  L.a2 = (int)off;
  off += q_pad4(o2 * o);
  L.w2_staged = o4 <= 4096;
  L.w2 = (int)off;
  off += L.w2_staged ? q_pad4(o4) : 0;
  L.vs = (int)off;
  off += q_pad4(o2);
  L.total = off;
  return L;
}

template <typename T, int JM>  // JM >= o: the per-j accumulators and loops (o rounded up to 4)
__global__ void __launch_bounds__(kThreadsQ, 2) k_q_main_staged(const QArgs q) {
  extern __shared__ __align__(16) unsigned char q_smem[];
  __shared__ double ws[32];
  __shared__ i64 s_blk[6][kMaxVQ];
  const int o = q.o, v = q.v;
  const i64 o2 = (i64)o * o, o3 = o2 * o, O4 = o2 * o2;
  const QStage lay = q_stage_layout(o, v);
  T* sm = (T*)q_smem;
  T* R = sm;
  T* Z = sm + q_pad4(O4);
  T* A1s = sm + lay.a1;
  T* W1s = sm + lay.w1;
  T* A2s = sm + lay.a2;
  T* W2s = sm + lay.w2;
  T* Vs = sm + lay.vs;
  const T* t3v = (const T*)q.t3v;
  const T* A1 = (const T*)q.A1;
  const T* A2 = (const T*)q.A2;
  const T* Vv = (const T*)q.Vv;
  const T* W1 = (const T*)q.W1;
  const T* W2 = (const T*)q.W2;
  const T* T2e = (const T*)q.T2e;
  const T* T2m = (const T*)q.T2m;
  const T* T2v = (const T*)q.T2v;
  double total = 0.0;
  for (i64 qi = blockIdx.x; qi < q.nquad; qi += gridDim.x) {
    const int4 L4 = q.quads[qi];
    const int L[4] = {L4.x & 0xffff, L4.x >> 16, L4.y & 0xffff, L4.y >> 16};
    const double fac = (double)L4.z;
    __syncthreads();  // the previous quadruple's tables and R, Z are consumed
    for (int t = threadIdx.x; t < 6 * v; t += blockDim.x) {
      const int pi = t / v, e = t % v;
      const int x = pi < 3 ? 0 : (pi < 5 ? 1 : 2), y = pi < 3 ? pi + 1 : (pi < 5 ? pi - 1 : 3);
      const int r0 = L[x], s0 = L[y];
      const i64 b = e <= r0 ? tri3(e, r0, s0) : (e <= s0 ? tri3(r0, e, s0) : tri3(r0, s0, e));
      s_blk[pi][e] = b * o3;
    }
    for (i64 t = threadIdx.x; t < 2 * q_pad4(O4); t += blockDim.x) R[t] = (T)0;  // R and Z
    for (int sg = 0; sg < 24; ++sg) {
      const int c0 = c_perm[sg][0], c1 = c_perm[sg][1], c2 = c_perm[sg][2], c3 = c_perm[sg][3];
      const int p = L[c0], qq = L[c1], r = L[c2], s = L[c3];
      __syncthreads();  // the previous sigma's slices are consumed (and R, Z, s_blk are set)
      for (i64 t = threadIdx.x; t < (i64)o * v; t += blockDim.x) {  // A1s[e][j] = v^{pq}_{ej}
        const int j = (int)(t / v), e = (int)(t % v);
        A1s[e * o + j] = A1[(((i64)p * v + qq) * o + j) * v + e];
      }
      for (i64 t = threadIdx.x; t < o2 * v; t += blockDim.x) {  // W1s[k][e][j] = Wbar^{pqr}_{ejk}
        const int j = (int)(t / ((i64)o * v)), k = (int)((t / v) % o), e = (int)(t % v);
        W1s[((i64)k * v + e) * o + j] = W1[((((i64)p * v + qq) * v + r) * o2 + (i64)j * o + k) * v + e];
      }
      for (i64 t = threadIdx.x; t < o3; t += blockDim.x) {  // A2s[i][m][j] = v^{pm}_{ij}
        const int i = (int)(t / o2), j = (int)((t / o) % o), m = (int)(t % o);
        A2s[((i64)i * o + m) * o + j] = A2[(((i64)p * o + i) * o + j) * o + m];
      }
      if (lay.w2_staged)
        for (i64 t = threadIdx.x; t < O4; t += blockDim.x) {  // W2s[i][k][m][j] = Wbar^{pqm}_{ijk}
          const int i = (int)(t / o3), j = (int)((t / o2) % o), k = (int)((t / o) % o), m = (int)(t % o);
          W2s[(((i64)i * o + k) * o + m) * o + j] = W2[((((i64)p * v + qq) * o + i) * o2 + (i64)j * o + k) * o + m];
        }
      for (i64 t = threadIdx.x; t < o2; t += blockDim.x)  // Vs[i][j] = v^{pq}_{ij}
        Vs[t] = Vv[(((i64)p * v + qq) * o) * o + t];
      __syncthreads();
      // weights of the permuted occupied positions in R's index
      const int w[4] = {(int)(c0 == 0 ? o3 : c0 == 1 ? o2 : c0 == 2 ? o : 1),
                        (int)(c1 == 0 ? o3 : c1 == 1 ? o2 : c1 == 2 ? o : 1),
                        (int)(c2 == 0 ? o3 : c2 == 1 ? o2 : c2 == 2 ? o : 1),
                        (int)(c3 == 0 ? o3 : c3 == 1 ? o2 : c3 == 2 ? o : 1)};
      const bool rs = c2 < c3;
      const i64* bt = s_blk[pair_index(rs ? c2 : c3, rs ? c3 : c2)];
      const int r0 = rs ? r : s, s0 = rs ? s : r;
      for (i64 t = threadIdx.x; t < o3; t += blockDim.x) {
        const int i = (int)(t / o2), k = (int)((t / o) % o), l = (int)(t % o);
        T ax[JM], ay[JM];  // per j: x1 - x2 and y1 - y2
#pragma unroll
        for (int j = 0; j < JM; ++j) ax[j] = ay[j] = (T)0;
        {  // x1 = sum_e v^{pq}_{ej} t^{ers}_{ikl}
          const int k0 = rs ? k : l, l0 = rs ? l : k;
          const i64 f0 = ((i64)i * o + k0) * o + l0, f1 = ((i64)k0 * o + i) * o + l0, f2 = ((i64)k0 * o + l0) * o + i;
          for (int e0 = 0; e0 < v; e0 += 8) {  // eight gathers in flight, then their FMAs
            T tv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int e = e0 + u;
              tv[u] = e < v ? t3v[bt[e] + (e <= r0 ? f0 : (e <= s0 ? f1 : f2))] : (T)0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              if (e0 + u >= v) break;
              const T* a = A1s + (e0 + u) * o;
#pragma unroll
              for (int j = 0; j < JM; ++j)
                if (j < o) ax[j] += a[j] * tv[u];
            }
          }
        }
        {  // x2 = sum_m v^{pm}_{ij} t^{qrs}_{mkl}
          const i64 b0 = t3v_off(qq, r, s, 0, k, l, o), bm = t3v_off(qq, r, s, 1, k, l, o) - b0;
          for (int m = 0; m < o; ++m) {
            const T tv = t3v[b0 + m * bm];
            const T* a = A2s + ((i64)i * o + m) * o;
#pragma unroll
            for (int j = 0; j < JM; ++j)
              if (j < o) ax[j] -= a[j] * tv;
          }
        }
        {  // y1 = sum_e Wbar^{pqr}_{ejk} t^{es}_{il}
          const T* t2e = T2e + (((i64)i * o + l) * v + s) * v;
          const T* wk = W1s + (i64)k * v * o;
          for (int e0 = 0; e0 < v; e0 += 8) {
            T tv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) tv[u] = e0 + u < v ? t2e[e0 + u] : (T)0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              if (e0 + u >= v) break;
              const T* a = wk + (e0 + u) * o;
#pragma unroll
              for (int j = 0; j < JM; ++j)
                if (j < o) ay[j] += a[j] * tv[u];
            }
          }
        }
        {  // y2 = sum_m Wbar^{pqm}_{ijk} t^{rs}_{ml}
          const T* t2m = T2m + (((i64)l * v + r) * v + s) * o;
          for (int m = 0; m < o; ++m) {
            const T tv = t2m[m];
            if (lay.w2_staged) {
              const T* a = W2s + (((i64)i * o + k) * o + m) * o;
#pragma unroll
              for (int j = 0; j < JM; ++j)
                if (j < o) ay[j] -= a[j] * tv;
            } else {
#pragma unroll
              for (int j = 0; j < JM; ++j)
                if (j < o) ay[j] -= W2[((((i64)p * v + qq) * o + i) * o2 + (i64)j * o + k) * o + m] * tv;
            }
          }
        }
        // V: 1/4 v^{pq}_{ij} t^{rs}_{kl}; then R += X + Y, Z += X + V with X = (x1 - x2) / 2
        const T t2v = T2v[(((i64)k * o + l) * v + r) * v + s];
        const i64 base = (i64)i * w[0] + (i64)k * w[2] + (i64)l * w[3];
#pragma unroll
        for (int j = 0; j < JM; ++j)
          if (j < o) {
            const i64 el = base + (i64)j * w[1];
            const T X = (T)0.5 * ax[j];
            R[el] += X + (T)0.5 * ay[j];
            Z[el] += X + (T)0.25 * Vs[i * o + j] * t2v;
          }
      }
    }
    __syncthreads();
    // (b) f_abcd sum_O Z(O) t~(O), t~(O) = sum_pi c_pi R(O o pi^-1) / eps(O)
    const double ev = q.eps[o + L[0]] + q.eps[o + L[1]] + q.eps[o + L[2]] + q.eps[o + L[3]];
    double part = 0.0;
    for (i64 el = threadIdx.x; el < O4; el += blockDim.x) {
      const int Oc[4] = {(int)(el / o3), (int)((el / o2) % o), (int)((el / o) % o), (int)(el % o)};
      double ts = 0.0;
      for (int pi = 0; pi < 24; ++pi) {
        const i64 idx = (((i64)Oc[c_pinv[pi][0]] * o + Oc[c_pinv[pi][1]]) * o + Oc[c_pinv[pi][2]]) * o +
                        Oc[c_pinv[pi][3]];
        ts += c_coef[pi] * (double)R[idx];
      }
      const double eo = q.eps[Oc[0]] + q.eps[Oc[1]] + q.eps[Oc[2]] + q.eps[Oc[3]];
      part += (double)Z[el] * ts / (eo - ev);
    }
    const double bs = block_sum_q(part, ws);
    if (threadIdx.x == 0) total += fac * bs;
  }
  if (threadIdx.x == 0) q.partial[blockIdx.x] = total;
}

__global__ void k_q_reduce(const double* __restrict__ partial, int n, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += partial[i];
  out[0] = s / 24.0;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// Coefficients of the full spin summation 2 (2 - P_c^d)(2 - P_b^c - P_b^d)(2 - P_a^b - P_a^c - P_a^d)
// (Eq. quadruples-spin-sum and the (Q) appendix) as sum_pi c_pi t(L o pi), where a swap
// P_x^y acts on a function of the labels as g(L) -> g(L o tau_xy).
void spin_sum_table(const std::vector<std::array<int, 4>>& perms, double coef[24]) {
  auto index_of = [&](const std::array<int, 4>& p) {
    for (int i = 0; i < 24; ++i)
      if (perms[i] == p) return i;
    return -1;
  };
  std::vector<double> g(24, 0.0);
  g[index_of({0, 1, 2, 3})] = 1.0;
  auto apply = [&](double diag, const std::vector<std::array<int, 2>>& swaps) {
    std::vector<double> out(24, 0.0);
    for (int i = 0; i < 24; ++i) {
      if (g[i] == 0.0) continue;
      out[i] += diag * g[i];
      for (const auto& sw : swaps) {
        std::array<int, 4> np;  // (tau o pi)(x) = tau(pi(x))
        for (int x = 0; x < 4; ++x) {
          const int y = perms[i][x];
          np[x] = y == sw[0] ? sw[1] : (y == sw[1] ? sw[0] : y);
        }
        out[index_of(np)] -= g[i];
      }
    }
    g = out;
  };
  apply(2.0, {{0, 1}, {0, 2}, {0, 3}});
  apply(2.0, {{1, 2}, {1, 3}});
  apply(2.0, {{2, 3}});
  for (int i = 0; i < 24; ++i) coef[i] = 2.0 * g[i];
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  bool alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 16) == cudaSuccess; }
};

unsigned grid_for(i64 tot) { return (unsigned)std::max<i64>(1, std::min<i64>((tot + 255) / 256, 152 * 32)); }

void init_tables() {
  static bool done = false;
  if (done) return;
  std::vector<std::array<int, 4>> perms;
  std::array<int, 4> p = {0, 1, 2, 3};
  do perms.push_back(p);
  while (std::next_permutation(p.begin(), p.end()));
  unsigned char hp[24][4], hinv[24][4];
  for (int i = 0; i < 24; ++i)
    for (int x = 0; x < 4; ++x) {
      hp[i][x] = (unsigned char)perms[i][x];
      hinv[i][perms[i][x]] = (unsigned char)x;
    }
  double coef[24];
  spin_sum_table(perms, coef);
  cudaMemcpyToSymbol(c_perm, hp, sizeof(hp));
  cudaMemcpyToSymbol(c_pinv, hinv, sizeof(hinv));
  cudaMemcpyToSymbol(c_coef, coef, sizeof(coef));
  done = true;
}

// The one-time transposition into `out` (device, T elements).
template <typename T>
int transpose_t3(const rcc::QInputs& in, T* out, i64 nv3, const int4* vtrip) {
  const i64 tot = nv3 * in.o * in.o * in.o;
  ++rcc::g_launch_count;
  if (in.t3_f32)
    k_q_t3v<float, T><<<grid_for(tot), 256, 0, in.stream>>>((const float*)in.t3, in.o, in.v, vtrip, nv3, out);
  else
    k_q_t3v<double, T><<<grid_for(tot), 256, 0, in.stream>>>((const double*)in.t3, in.o, in.v, vtrip, nv3, out);
  return cudaGetLastError() == cudaSuccess ? 0 : RCCSDT_ERR_CUDA;
}

std::vector<int4> virtual_triples(int v) {
  std::vector<int4> out;
  for (int c = 0; c < v; ++c)
    for (int b = 0; b <= c; ++b)
      for (int a = 0; a <= b; ++a) out.push_back(make_int4(a, b, c, 0));
  return out;
}

template <typename T>
int q_energy(rccsdt_ctx* ctx, const rcc::QInputs& in, double* e_q, double* info) {
  const int o = in.o, v = in.v, n = o + v;
  const i64 n4 = (i64)n * n * n * n, o2 = (i64)o * o, o4 = o2 * o2, V2 = (i64)v * v;
  const std::vector<int4> vt = virtual_triples(v);
  const i64 nv3 = (i64)vt.size();
  // sorted quadruples with their degeneracy factor (Eq. ener-pt-q-abc)
  std::vector<int4> quads;
  for (int d = 0; d < v; ++d)
    for (int c = 0; c <= d; ++c)
      for (int b = 0; b <= c; ++b)
        for (int a = 0; a <= b; ++a) {
          const int eq = (a == b) + (b == c) + (c == d);
          const int f = eq == 0 ? 24 : (eq == 1 ? 12 : (eq == 2 && a == b && c == d ? 6 : 0));
          if (f) quads.push_back(make_int4(a | (b << 16), c | (d << 16), f, 0));
        }
  const i64 nquad = (i64)quads.size();
  const size_t es = sizeof(T);
  const size_t rz_bytes = (size_t)2 * o4 * es;
  int dev = 0, nsm = 152, smem_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const bool in_smem = rz_bytes + 1024 <= (size_t)std::min(smem_optin, 200 * 1024);
  // the operand-staged kernel when o <= 16 and R, Z and the slices fit shared memory
  const size_t staged_bytes = (size_t)q_stage_layout(o, v).total * es;
  // (FP32 only: in FP64 the sums are bound by the FP64 units either way, and the
  // per-j accumulators of the staged form cost the FP64 kernel its occupancy)
  const bool staged = sizeof(T) == 4 && o <= kMaxOQ && staged_bytes + 1024 <= (size_t)std::min(smem_optin, 200 * 1024);
  // resident CTAs per SM: the dynamic shared memory plus the static tables (about 13 KB)
  const size_t dyn = staged ? staged_bytes : rz_bytes;
  const int per_sm = (staged || in_smem) ? std::max(1, std::min(4, (int)((224 * 1024) / (dyn + 14 * 1024)))) : 4;
  const int grid = (int)std::max<i64>(1, std::min<i64>(nquad, (i64)nsm * per_sm));

  DevBuf G, Gf_buf, t3v, A1, A2, Vv, W1, W2, T2e, T2m, T2v, vtr, qd, scratch, partial, outd;
  if (!G.alloc(n4 * 8) || !Gf_buf.alloc(sizeof(T) == 4 ? (size_t)(n4 + o2 * V2) * 4 : 16) || !t3v.alloc(nv3 * o2 * o * es) || !A1.alloc(V2 * o * v * es) ||
      !A2.alloc((i64)v * o2 * o * es) || !Vv.alloc(V2 * o2 * es) || !W1.alloc(V2 * V2 * o2 * es) ||
      !W2.alloc(V2 * o4 * es) || !T2e.alloc(o2 * V2 * es) || !T2m.alloc(o2 * V2 * es) ||
      !T2v.alloc(o2 * V2 * es) || !vtr.alloc(vt.size() * sizeof(int4)) || !qd.alloc(quads.size() * sizeof(int4)) ||
      !scratch.alloc(in_smem ? 16 : (size_t)grid * rz_bytes) || !partial.alloc((size_t)grid * 8) || !outd.alloc(8)) {
    cudaGetLastError();
    return rcc::ctx_fail(ctx, RCCSDT_ERR_OOM, "(Q): device allocation failed");
  }
  init_tables();
  cudaStream_t s = in.stream;
  cudaEvent_t ev[5];
  for (auto& e : ev) cudaEventCreate(&e);
  cudaEventRecord(ev[0], s);
  cudaMemcpyAsync(vtr.p, vt.data(), vt.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(qd.p, quads.data(), quads.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
  int st = transpose_t3<T>(in, (T*)t3v.p, nv3, (const int4*)vtr.p);
  cudaEventRecord(ev[1], s);
  rcc::g_launch_count += 10;
  k_q_eri<<<grid_for(n4), 256, 0, s>>>(in.L, in.naux, n, (double*)G.p);
  const i64 sizes[6] = {V2 * o * v, (i64)v * o2 * o, V2 * o2, o2 * V2, o2 * V2, o2 * V2};
  void* dst[6] = {A1.p, A2.p, Vv.p, T2e.p, T2m.p, T2v.p};
  for (int kind = 0; kind < 6; ++kind)
    k_q_layout<T><<<grid_for(sizes[kind]), 256, 0, s>>>(kind, (const double*)G.p, in.t2, o, v, (T*)dst[kind],
                                                        sizes[kind]);
  if (sizeof(T) == 8) {
    k_q_wbar1<T, double><<<grid_for(V2 * V2 * o2), 256, 0, s>>>((const double*)G.p, in.t2, o, v, (T*)W1.p);
    k_q_wbar2<T, double><<<grid_for(V2 * o4), 256, 0, s>>>((const double*)G.p, in.t2, o, v, (T*)W2.p);
  } else {
    // FP32 copies of the ERIs and t2, read by the FP32 sums
    float* Gf = (float*)Gf_buf.p;
    float* t2f = Gf + n4;
    rcc::launch_convert<float, double>(Gf, (const double*)G.p, n4, s);
    rcc::launch_convert<float, double>(t2f, in.t2, o2 * V2, s);
    k_q_wbar1<T, float><<<grid_for(V2 * V2 * o2), 256, 0, s>>>(Gf, t2f, o, v, (T*)W1.p);
    k_q_wbar2<T, float><<<grid_for(V2 * o4), 256, 0, s>>>(Gf, t2f, o, v, (T*)W2.p);
  }
  cudaEventRecord(ev[2], s);
  QArgs qa;
  qa.quads = (const int4*)qd.p;
  qa.nquad = nquad;
  qa.o = o;
  qa.v = v;
  qa.eps = in.e;
  qa.t3v = t3v.p;
  qa.A1 = A1.p;
  qa.A2 = A2.p;
  qa.Vv = Vv.p;
  qa.W1 = W1.p;
  qa.W2 = W2.p;
  qa.T2e = T2e.p;
  qa.T2m = T2m.p;
  qa.T2v = T2v.p;
  qa.scratch = scratch.p;
  qa.smem_rz = in_smem ? 1 : 0;
  qa.partial = (double*)partial.p;
  const int smem = in_smem ? (int)rz_bytes : 0;
  ++rcc::g_launch_count;
  if (staged) {
    auto launch = [&](auto kern) {
      if (staged_bytes > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)staged_bytes);
      kern<<<grid, kThreadsQ, staged_bytes, s>>>(qa);
    };
    if (o <= 4) launch(k_q_main_staged<T, 4>);
    else if (o <= 8) launch(k_q_main_staged<T, 8>);
    else if (o <= 12) launch(k_q_main_staged<T, 12>);
    else launch(k_q_main_staged<T, 16>);
  } else {
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_q_main<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_q_main<T><<<grid, kThreadsQ, smem, s>>>(qa);
  }
  cudaEventRecord(ev[3], s);
  ++rcc::g_launch_count;
  k_q_reduce<<<1, 32, 0, s>>>((const double*)partial.p, grid, (double*)outd.p);
  cudaEventRecord(ev[4], s);
  double e = 0.0;
  if (!st && (cudaMemcpyAsync(&e, outd.p, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess))
    st = RCCSDT_ERR_CUDA;
  if (!st && info) {
    float ms[4];
    for (int q = 0; q < 4; ++q) cudaEventElapsedTime(&ms[q], ev[q], ev[q + 1]);
    info[0] = ms[0];  // transposition
    info[1] = ms[1];  // integrals, layouts and Wbar
    info[2] = ms[2];  // main kernel
    info[3] = (double)nquad * 24.0 * (double)o4 * (2.0 * v + 2.0 * o) * 2.0;  // flop of the main kernel
    info[4] = (double)nquad;
    info[5] = (double)grid;
  }
  for (auto& x : ev) cudaEventDestroy(x);
  if (st) return rcc::ctx_fail(ctx, st, "(Q): a CUDA call failed");
  if (!std::isfinite(e)) return rcc::ctx_fail(ctx, RCCSDT_ERR_NONFINITE, "(Q): non-finite energy");
  *e_q = e;
  return RCCSDT_OK;
}

}  // namespace

#define RCC_API extern "C" __attribute__((visibility("default")))

RCC_API int rccsdt_q_energy(rccsdt_ctx* ctx, int arith, double* e_q, double* info) {
  if (!ctx || !e_q || (arith != RCCSDT_Q_FP64 && arith != RCCSDT_Q_FP32)) return RCCSDT_ERR_ARG;
  rcc::QInputs in;
  int st = rcc::ctx_q_inputs(ctx, &in);
  if (st) return st;
  if (cudaPeekAtLastError() != cudaSuccess) return rcc::ctx_fail(ctx, RCCSDT_ERR_CUDA, "(Q): pending CUDA error");
  if (in.v > kMaxVQ) return rcc::ctx_fail(ctx, RCCSDT_ERR_ARG, "(Q): v above 256");
  return arith == RCCSDT_Q_FP64 ? q_energy<double>(ctx, in, e_q, info) : q_energy<float>(ctx, in, e_q, info);
}

RCC_API int rccsdt_t3_virtual_triangular(rccsdt_ctx* ctx, double* t3v) {
  if (!ctx || !t3v) return RCCSDT_ERR_ARG;
  rcc::QInputs in;
  int st = rcc::ctx_q_inputs(ctx, &in);
  if (st) return st;
  const std::vector<int4> vt = virtual_triples(in.v);
  const i64 nv3 = (i64)vt.size(), cnt = nv3 * in.o * in.o * in.o;
  DevBuf out, vtr;
  if (!out.alloc((size_t)cnt * 8) || !vtr.alloc(vt.size() * sizeof(int4))) {
    cudaGetLastError();
    return rcc::ctx_fail(ctx, RCCSDT_ERR_OOM, "transposition: device allocation failed");
  }
  if (cudaMemcpyAsync(vtr.p, vt.data(), vt.size() * sizeof(int4), cudaMemcpyHostToDevice, in.stream) != cudaSuccess)
    return rcc::ctx_fail(ctx, RCCSDT_ERR_CUDA, "transposition: copy failed");
  st = transpose_t3<double>(in, (double*)out.p, nv3, (const int4*)vtr.p);
  if (st || cudaMemcpyAsync(t3v, out.p, (size_t)cnt * 8, cudaMemcpyDefault, in.stream) != cudaSuccess ||
      cudaStreamSynchronize(in.stream) != cudaSuccess)
    return rcc::ctx_fail(ctx, RCCSDT_ERR_CUDA, "transposition failed");
  return RCCSDT_OK;
}
