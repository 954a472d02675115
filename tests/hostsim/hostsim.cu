// TEST-ONLY host simulation of the RCCSDT library's kernels.
//
// Built together with the library's runtime (compiled with -DRCC_HOSTSIM) into a
// separate shared object that only the CPU tests load.  It executes the very
// plans (gather tables, scatter tables, term lists) of the CUDA library with
// plain host loops over the same per-element functions (elem.cuh), so the host
// logic can be checked against the oracle without a GPU.  The product binding
// never loads it; the CUDA library has no CPU path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "elem.cuh"
#include "kernels.h"

namespace rcc {

long long g_launch_count = 0;

void launch_pack(const PackArgs& a, cudaStream_t) {
  for (int r = 0; r < a.R; ++r)
    for (int k = 0; k < a.Kpad; ++k) store_panel(a, r, k, k < a.K ? pack_value(a, r, k) : 0.0);
}

int pack_tiles_of(const PackArgs& a) { return ((a.R + 31) / 32) * ((a.Kpad + 31) / 32); }

void launch_pack_grouped(const PackArgs* list, const int*, int npack, int, int, cudaStream_t s) {
  for (int p = 0; p < npack; ++p) launch_pack(list[p], s);
}

void launch_gemm_f64(const double* A, const double* B, int K, int lda, int ldb, const EpiArgs& e, double*, i64,
                     cudaStream_t) {
  for (int m = 0; m < e.M; ++m)
    for (int n = 0; n < e.N; ++n) {
      double s = 0.0;
      for (int k = 0; k < K; ++k) s += A[(i64)m * lda + k] * B[(i64)n * ldb + k];
      epi_apply(e, m, n, s);
    }
}

// Split-precision product hi*hi + hi*lo + lo*hi with float products and a float
// accumulator (the order of the tensor-core sum is not modelled).
int launch_gemm_tc(int kind, const void* Ahi, const void* Alo, const void* Bhi, const void* Blo, int Kpad,
                   const EpiArgs& e, int*, long long, cudaStream_t, float*, long long, float* raw_out, int,
                   int colmajor) {
  auto get = [&](const void* p, i64 i) -> float {
    if (kind == PANEL_BF16X2) return __bfloat162float(((const __nv_bfloat16*)p)[i]);
    return ((const float*)p)[i];
  };
  for (int m = 0; m < e.M; ++m)
    for (int n = 0; n < e.N; ++n) {
      float s = 0.f;
      for (int k = 0; k < Kpad; ++k) {
        const i64 ia = (i64)m * Kpad + k, ib = (i64)n * Kpad + k;
        const float ah = get(Ahi, ia), al = get(Alo, ia), bh = get(Bhi, ib), bl = get(Blo, ib);
        s += ah * bh + ah * bl + al * bh;
      }
      if (raw_out)
        raw_out[colmajor ? (i64)n * e.M + m : (i64)m * e.N + n] = s;
      else
        epi_apply(e, m, n, (double)s);
    }
  return 0;
}

void launch_combine(const CombineArgs& c, cudaStream_t) {
  for (i64 idx = 0; idx < c.total; ++idx) {
    i64 rem = idx, ooff = 0;
    i64 ioff[4] = {0, 0, 0, 0};
    for (int d = c.rank - 1; d >= 0; --d) {
      const i64 x = rem % c.shape[d];
      rem /= c.shape[d];
      ooff += x * c.ostride[d];
      for (int t = 0; t < c.nterm; ++t) ioff[t] += x * c.istride[t][d];
    }
    double s = c.beta == 0.0 ? 0.0 : c.beta * c.out[ooff];
    for (int t = 0; t < c.nterm; ++t) s += c.coef[t] * c.in[t][ioff[t]];
    c.out[ooff] = s;
  }
}

static void host_store_split(int kind, void* hi, void* lo, long long o, float x) {
  if (kind == PANEL_BF16X2) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    ((__nv_bfloat16*)hi)[o] = h;
    ((__nv_bfloat16*)lo)[o] = __float2bfloat16_rn(x - __bfloat162float(h));
  } else {
    const float h = tf32_round(x);
    ((float*)hi)[o] = h;
    ((float*)lo)[o] = tf32_round(x - h);
  }
}

void launch_cube_pack(int mode, int kind, const CubePiece* pieces, int npieces, const CubeDst* dsts,
                      const CubeDst& d0, const float* src, int v, cudaStream_t) {
  const i64 S[3] = {(i64)v * v, v, 1};
  for (int q = 0; q < npieces; ++q) {
    const CubePiece& P = pieces[q];
    const CubeDst d = dsts ? dsts[P.dst] : d0;
    const int nt = mode == 1 ? (P.nterm > 0 ? 1 : 0) : P.nterm;
    for (int l0 = 0; l0 < v; ++l0)
      for (int l1 = 0; l1 < v; ++l1)
        for (int l2 = 0; l2 < v; ++l2) {
          float x = 0.f;
          for (int t = 0; t < nt; ++t) {
            const int ps = P.t[t].pos;
            const i64 off = P.t[t].base + l0 * S[ps & 3] + l1 * S[(ps >> 2) & 3] + l2 * S[(ps >> 4) & 3];
            x = std::fma(P.t[t].coef, src[off], x);
          }
          const i64 row = mode == 0 ? P.row0 + (i64)l1 * P.rs1 + (i64)l2 * P.rs2 : P.row0 + ((i64)l0 * v + l1) * v + l2;
          const i64 k = mode == 0 ? P.k0 + l0 + (i64)l1 * P.ks1 : P.k0;
          host_store_split(kind, d.out_hi, d.out_lo, row * d.Kpad + k, x);
        }
  }
}

void launch_pair_pack_w(int kind, const double* W, int v, const int4* rows, int Mp, const PairChunk* ch, int nchunk,
                        int Kp, int Km, const CubeDst& dp, const CubeDst& dm, cudaStream_t) {
  const i64 V2 = (i64)v * v;
  for (int m = 0; m < Mp; ++m) {
    const int4 rw = rows[m];
    const double* Wr = W + ((i64)rw.x * v + rw.y) * V2;
    for (int ci = 0; ci < nchunk; ++ci) {
      const PairChunk c = ch[ci];
      const int d0 = c.P * 16, e0 = c.Q * 16, nd = std::min(16, v - d0), ne = std::min(16, v - e0);
      const bool diag = c.P == c.Q;
      const int np = diag ? nd * (nd + 1) / 2 : nd * ne, nm = diag ? nd * (nd - 1) / 2 : nd * ne;
      for (int t = 0; t < np; ++t) {
        int a, b;
        pair_decode(t, diag, true, nd, ne, a, b);
        const int d = d0 + a, e = e0 + b;
        const double x = d == e ? Wr[(i64)d * v + d] : Wr[(i64)d * v + e] + Wr[(i64)e * v + d];
        panel_put(kind, dp.out_hi, dp.out_lo, (i64)m * dp.Kpad + c.offp + t, x);
      }
      if (rw.z >= 0)
        for (int t = 0; t < nm; ++t) {
          int a, b;
          pair_decode(t, diag, false, nd, ne, a, b);
          const int d = d0 + a, e = e0 + b;
          panel_put(kind, dm.out_hi, dm.out_lo, (i64)rw.z * dm.Kpad + c.offm + t,
                    Wr[(i64)d * v + e] - Wr[(i64)e * v + d]);
        }
    }
    for (int k = Kp; k < dp.Kpad; ++k) panel_put(kind, dp.out_hi, dp.out_lo, (i64)m * dp.Kpad + k, 0.0);
    if (rw.z >= 0)
      for (int k = Km; k < dm.Kpad; ++k) panel_put(kind, dm.out_hi, dm.out_lo, (i64)rw.z * dm.Kpad + k, 0.0);
  }
}

void launch_pair_pack_t(int kind, const void* t3, int t3_f32, i64 b0, int nblk, int v, i64 sd, i64 se, i64 sw,
                        const PairChunk* ch, int nchunk, int Kp, int Km, const CubeDst& dp, const CubeDst& dm,
                        cudaStream_t) {
  const i64 V3 = (i64)v * v * v;
  for (int q = 0; q < nblk; ++q) {
    const i64 base = (b0 + q) * V3;
    auto T = [&](int d, int e, int w) { return load_src(t3, t3_f32, base + d * sd + e * se + w * sw); };
    for (int w = 0; w < v; ++w) {
      const i64 row = (i64)q * v + w;
      for (int ci = 0; ci < nchunk; ++ci) {
        const PairChunk c = ch[ci];
        const int d0 = c.P * 16, e0 = c.Q * 16, nd = std::min(16, v - d0), ne = std::min(16, v - e0);
        const bool diag = c.P == c.Q;
        const int np = diag ? nd * (nd + 1) / 2 : nd * ne, nm = diag ? nd * (nd - 1) / 2 : nd * ne;
        for (int t = 0; t < np; ++t) {
          int a, b;
          pair_decode(t, diag, true, nd, ne, a, b);
          const double x = kind == PANEL_F64 ? T(d0 + a, e0 + b, w) + T(e0 + b, d0 + a, w)
                                             : (double)((float)T(d0 + a, e0 + b, w) + (float)T(e0 + b, d0 + a, w));
          panel_put(kind, dp.out_hi, dp.out_lo, row * dp.Kpad + c.offp + t, x);
        }
        for (int t = 0; t < nm; ++t) {
          int a, b;
          pair_decode(t, diag, false, nd, ne, a, b);
          const double x = kind == PANEL_F64 ? T(d0 + a, e0 + b, w) - T(e0 + b, d0 + a, w)
                                             : (double)((float)T(d0 + a, e0 + b, w) - (float)T(e0 + b, d0 + a, w));
          panel_put(kind, dm.out_hi, dm.out_lo, row * dm.Kpad + c.offm + t, x);
        }
      }
      for (int k = Kp; k < dp.Kpad; ++k) panel_put(kind, dp.out_hi, dp.out_lo, row * dp.Kpad + k, 0.0);
      for (int k = Km; k < dm.Kpad; ++k) panel_put(kind, dm.out_hi, dm.out_lo, row * dm.Kpad + k, 0.0);
    }
  }
}

void launch_cube_pack_r1(int kind, const CubePiece* pieces, int npieces, const CubeDst& d0,
                         const float* src, int v, const float* w, const i64* wbase, float* part, cudaStream_t st) {
  launch_cube_pack(0, kind, pieces, npieces, nullptr, d0, src, v, st);
  const i64 S[3] = {(i64)v * v, v, 1};
  const int nc = (v + 15) / 16;
  auto sval = [&](const CubePiece& P, int l0, int l1, int l2) {
    if (l0 >= v || l1 >= v || l2 >= v) return 0.f;
    float x = 0.f;
    for (int t = 0; t < P.nterm; ++t) {
      const int ps = P.t[t].pos;
      x = std::fma(P.t[t].coef, src[P.t[t].base + l0 * S[ps & 3] + l1 * S[(ps >> 2) & 3] + l2 * S[(ps >> 4) & 3]], x);
    }
    return x;
  };
  for (int q = 0; q < npieces; ++q) {
    const CubePiece& P = pieces[q];
    const float* wp = w + wbase[q];
    for (int cb = 0; cb < nc * nc * nc; ++cb) {
      const int t0 = cb / (nc * nc), t1 = (cb / nc) % nc, t2 = cb % nc;
      float* out = part + ((i64)q * nc * nc * nc + cb) * 32;
      for (int r = 0; r < 16; ++r) {
        float a = 0.f, b = 0.f;
        for (int u = 0; u < 16; ++u)
          for (int m = 0; m < 16; ++m) {
            const int e1 = t0 * 16 + u;
            if (e1 >= v) continue;
            if (t1 * 16 + m < v) a += wp[(i64)e1 * v + t1 * 16 + m] * sval(P, e1, t1 * 16 + m, t2 * 16 + r);
            if (t2 * 16 + m < v) b += wp[(i64)e1 * v + t2 * 16 + m] * sval(P, e1, t1 * 16 + r, t2 * 16 + m);
          }
        out[r] = a;
        out[16 + r] = b;
      }
    }
  }
}

void launch_r1_cubes_reduce(const float* part, int ppz, int nz, int v, double* dR1, cudaStream_t) {
  const int nc = (v + 15) / 16, ncube = nc * nc * nc;
  for (int z = 0; z < nz; ++z)
    for (int a = 0; a < v; ++a) {
      double s = 0.0;
      for (int p = 0; p < ppz; ++p)
        for (int cb = 0; cb < ncube; ++cb) {
          const int t1 = (cb / nc) % nc, t2 = cb % nc;
          const float* pp = part + ((i64)(z * ppz + p) * ncube + cb) * 32;
          if (t2 == a / 16) s += pp[a % 16];
          if (t1 == a / 16) s -= 0.5 * pp[16 + a % 16];
        }
      dR1[(i64)z * v + a] += s;
    }
}

void launch_slice_f64(const double* P, int R, int Kpad, void* planes, int* exps, cudaStream_t) {
  __nv_bfloat16* pl = (__nv_bfloat16*)planes;
  const i64 plane = (i64)R * Kpad;
  for (int r = 0; r < R; ++r) {
    unsigned long long mx = 0;
    for (int k = 0; k < Kpad; ++k) mx = std::max(mx, f64_magnitude_bits(P[(i64)r * Kpad + k]));
    exps[r] = slice_exponent(mx);
    for (int k = 0; k < Kpad; ++k) {
      float a[kSlices];
      slice_digits(P[(i64)r * Kpad + k], exps[r], a);
      for (int s = 0; s < kSlices; ++s) pl[s * plane + (i64)r * Kpad + k] = __float2bfloat16_rn(a[s]);
    }
  }
}

// The digit products with s + t <= 5, summed in FP64 (the device sums them exactly,
// up to the FP32 rounding of the smallest ones).
int launch_gemm_f64e(const void* Aplanes, const int* ea, const void* Bplanes, const int* eb, int Kpad, const EpiArgs& e,
                     int*, long long, cudaStream_t) {
  if (Kpad % 64 != 0) return 1;
  const __nv_bfloat16* A = (const __nv_bfloat16*)Aplanes;
  const __nv_bfloat16* B = (const __nv_bfloat16*)Bplanes;
  const i64 pa = (i64)e.M * Kpad, pb = (i64)e.N * Kpad;
  for (int m = 0; m < e.M; ++m)
    for (int n = 0; n < e.N; ++n) {
      double s = 0.0;
      for (int k = 0; k < Kpad; ++k)
        for (int sa = 0; sa < kSlices; ++sa)
          for (int sb = 0; sb + sa < kSlices; ++sb)
            s += (double)__bfloat162float(A[sa * pa + (i64)m * Kpad + k]) *
                 (double)__bfloat162float(B[sb * pb + (i64)n * Kpad + k]);
      epi_apply(e, m, n, std::ldexp(s, ea[m] + eb[n] - 14));
    }
  return 0;
}

void launch_zero_cols(const CubeDst& d, i64 rows, int k0, int kind, cudaStream_t) {
  for (i64 r = 0; r < rows; ++r)
    for (int k = k0; k < d.Kpad; ++k) host_store_split(kind, d.out_hi, d.out_lo, r * d.Kpad + k, 0.f);
}

int gemm_tc_block_k(int kind) { return kind == PANEL_BF16X2 ? 64 : 32; }

int make_gproblem(GProblem* p, int kind, const void* Ahi, const void* Alo, const void* Bhi, const void* Blo, int M,
                  int N, int Kpad, float* out, int bn) {
  if (kind != PANEL_BF16X2 && kind != PANEL_TF32X2) return 1;
  if (Kpad % gemm_tc_block_k(kind) != 0 || M <= 0 || N <= 0) return 1;
  memset((void*)p, 0, sizeof(*p));
  p->colmajor = 0;
  p->a_hi = Ahi;
  p->a_lo = Alo;
  p->b_hi = Bhi;
  p->b_lo = Blo;
  p->out = out;
  p->M = M;
  p->N = N;
  p->Kpad = Kpad;
  p->kblocks = Kpad / gemm_tc_block_k(kind);
  p->mt = (M + 127) / 128;
  p->nt = (N + (bn == 128 ? 127 : 255)) / (bn == 128 ? 128 : 256);
  return 0;
}

int gproblem_tiles(const GProblem& p) { return p.mt * p.nt; }

int launch_gemm_tc_grouped(int kind, const GProblem* probs, int nprob, int, int, int, int* flag, long long wd,
                           cudaStream_t s) {
  for (int q = 0; q < nprob; ++q) {
    const GProblem& P = probs[q];
    EpiArgs e{};
    e.M = P.M;
    e.N = P.N;
    if (launch_gemm_tc(kind, P.a_hi, P.a_lo, P.b_hi, P.b_lo, P.Kpad, e, flag, wd, s, nullptr, 0, P.out, 256,
                       P.colmajor))
      return 1;
  }
  return 0;
}

template <typename T>
void launch_r3_gather(const float* X, const i64* target, int ntarget, const int* cstart, const i64* xoff,
                      const int* csel, const float* calpha, int v, int accumulate, T* r3, cudaStream_t) {
  static const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const i64 V2 = (i64)v * v, V3 = V2 * v;
  std::vector<float> acc((size_t)V3);
  for (int t = 0; t < ntarget; ++t) {
    std::fill(acc.begin(), acc.end(), 0.f);
    for (int c = cstart[t]; c < cstart[t + 1]; ++c) {
      const int* p = P[csel[c]];
      const float* xb = X + xoff[c];
      for (int a = 0; a < v; ++a)
        for (int b = 0; b < v; ++b)
          for (int cc = 0; cc < v; ++cc) {
            const int y[3] = {a, b, cc};
            acc[(size_t)(a * V2 + b * v + cc)] =
                std::fma(calpha[c], xb[y[p[0]] * V2 + (i64)y[p[1]] * v + y[p[2]]], acc[(size_t)(a * V2 + b * v + cc)]);
          }
    }
    T* out = r3 + target[t];
    for (i64 e = 0; e < V3; ++e) out[e] = accumulate ? (T)(out[e] + (T)acc[(size_t)e]) : (T)acc[(size_t)e];
  }
}
template void launch_r3_gather<float>(const float*, const i64*, int, const int*, const i64*, const int*, const float*,
                                      int, int, float*, cudaStream_t);
template void launch_r3_gather<double>(const float*, const i64*, int, const int*, const i64*, const int*,
                                       const float*, int, int, double*, cudaStream_t);

template <typename T>
void launch_post(const T* r, T* rp, const int4* blocks, int v, i64 n3, const double* wblk, double*, double* norm2,
                 cudaStream_t) {
  const i64 V3 = (i64)v * v * v;
  double s = 0.0;
  for (i64 b = 0; b < n3; ++b) {
    double bs = 0.0;
    for (i64 e = 0; e < V3; ++e) {
      const int c = (int)(e % v), bb = (int)((e / v) % v), a = (int)(e / ((i64)v * v));
      const T x = post_value<T>(r + b * V3, v, blocks[b].x, blocks[b].y, blocks[b].z, a, bb, c);
      rp[b * V3 + e] = x;
      bs += (double)x * (double)x;
    }
    s += wblk[b] * bs;
  }
  *norm2 = s;
}
template void launch_post<double>(const double*, double*, const int4*, int, i64, const double*, double*, double*,
                                  cudaStream_t);
template void launch_post<float>(const float*, float*, const int4*, int, i64, const double*, double*, double*,
                                 cudaStream_t);
int post_partials(int, i64) { return 1; }

void launch_update_t12(double* t1, const double* r1, double* t2, const double* r2, const double* e, int o, int v,
                       double shift, cudaStream_t) {
  for (int i = 0; i < o; ++i)
    for (int a = 0; a < v; ++a) t1[i * v + a] += r1[i * v + a] / (e[i] - e[o + a] - shift);
  for (int i = 0; i < o; ++i)
    for (int j = 0; j < o; ++j)
      for (int a = 0; a < v; ++a)
        for (int b = 0; b < v; ++b) {
          const i64 x = (((i64)i * o + j) * v + a) * v + b;
          t2[x] += r2[x] / (e[i] + e[j] - e[o + a] - e[o + b] - shift);
        }
}

template <typename T>
void launch_update_t3(T* t3, const T* rp3, const double* e, const int4* blocks, int o, int v, i64 n3, double shift,
                      cudaStream_t) {
  const i64 V3 = (i64)v * v * v;
  for (i64 b = 0; b < n3; ++b)
    for (i64 x = 0; x < V3; ++x) {
      const int c = (int)(x % v), bb = (int)((x / v) % v), a = (int)(x / ((i64)v * v));
      const T d = (T)(e[blocks[b].x] + e[blocks[b].y] + e[blocks[b].z] - e[o + a] - e[o + bb] - e[o + c] - shift);
      t3[b * V3 + x] = t3[b * V3 + x] + rp3[b * V3 + x] / d;
    }
}
template void launch_update_t3<double>(double*, const double*, const double*, const int4*, int, int, i64, double,
                                       cudaStream_t);
template void launch_update_t3<float>(float*, const float*, const double*, const int4*, int, int, i64, double,
                                      cudaStream_t);

template <typename T>
void launch_wdot(const T* x, const T* y, i64 n, i64 seg, const double* w, double*, double* out, double scale,
                 int accumulate, cudaStream_t) {
  double s = 0.0;
  for (i64 i = 0; i < n; ++i) s += (double)x[i] * (double)y[i] * (w ? w[i / seg] : 1.0);
  *out = (accumulate ? *out : 0.0) + scale * s;
}
template void launch_wdot<double>(const double*, const double*, i64, i64, const double*, double*, double*, double,
                                  int, cudaStream_t);
template void launch_wdot<float>(const float*, const float*, i64, i64, const double*, double*, double*, double, int,
                                 cudaStream_t);

void launch_diis_begin(int* st, int M, int diis_start, cudaStream_t) {
  const int iter = st[0] + 1, count = st[1];
  st[0] = iter;
  st[2] = count % M;
  st[1] = count + 1;
  st[3] = std::min(count + 1, M);
  st[4] = (iter >= diis_start && st[3] >= 2) ? 1 : 0;
}

template <typename T>
void launch_slot_save(char* base, i64 stride, i64 off, const int* st, const T* src, i64 n, cudaStream_t) {
  T* dst = (T*)(base + (i64)st[2] * stride + off);
  for (i64 i = 0; i < n; ++i) dst[i] = src[i];
}
template void launch_slot_save<double>(char*, i64, i64, const int*, const double*, i64, cudaStream_t);
template void launch_slot_save<float>(char*, i64, i64, const int*, const float*, i64, cudaStream_t);

template <typename T>
void launch_slot_diff_store(char* hist_t, char* hist_e, i64 stride, i64 off, const int* st, const T* t, i64 n,
                            cudaStream_t) {
  T* ts = (T*)(hist_t + (i64)st[2] * stride + off);
  T* es = (T*)(hist_e + (i64)st[2] * stride + off);
  for (i64 i = 0; i < n; ++i) {
    es[i] = t[i] - es[i];
    ts[i] = t[i];
  }
}
template void launch_slot_diff_store<double>(char*, char*, i64, i64, const int*, const double*, i64, cudaStream_t);
template void launch_slot_diff_store<float>(char*, char*, i64, i64, const int*, const float*, i64, cudaStream_t);

template <typename T>
void launch_subcube(T* t3, T* sub, i64 n3, int v, int ns, int dir, cudaStream_t) {
  const i64 S3 = (i64)ns * ns * ns, V3 = (i64)v * v * v;
  for (i64 blk = 0; blk < n3; ++blk)
    for (int a = 0; a < ns; ++a)
      for (int b = 0; b < ns; ++b)
        for (int c = 0; c < ns; ++c) {
          T* full = t3 + blk * V3 + ((i64)a * v + b) * v + c;
          T* part = sub + blk * S3 + ((i64)a * ns + b) * ns + c;
          if (dir == 0) *part = *full;
          else *full = *part;
        }
}
template void launch_subcube<double>(double*, double*, i64, int, int, int, cudaStream_t);
template void launch_subcube<float>(float*, float*, i64, int, int, int, cudaStream_t);

// the host version keeps one partial per q (the device splits it over its fixed grid)
template <typename T>
void launch_diis_dots(const char* hist_e, i64 stride, i64 off, const int* st, int M, i64 n, i64 seg, const double* w,
                      double* partial, cudaStream_t) {
  const T* es = (const T*)(hist_e + (i64)st[2] * stride + off);
  for (int q = 0; q < M; ++q) {
    double s = 0.0;
    if (q < st[3]) {
      const T* eq = (const T*)(hist_e + (i64)q * stride + off);
      for (i64 i = 0; i < n; ++i) s += (double)es[i] * (double)eq[i] * (w ? w[i / seg] : 1.0);
    }
    for (int b = 0; b < kDotBlocks; ++b) partial[(i64)q * kDotBlocks + b] = b == 0 ? s : 0.0;
  }
}
template void launch_diis_dots<double>(const char*, i64, i64, const int*, int, i64, i64, const double*, double*,
                                       cudaStream_t);
template void launch_diis_dots<float>(const char*, i64, i64, const int*, int, i64, i64, const double*, double*,
                                      cudaStream_t);

void launch_diis_row(const double* partial, int nseg, const int* st, int M, double* B, cudaStream_t) {
  for (int q = 0; q < st[3]; ++q) {
    double tot = 0.0;
    for (int g = 0; g < nseg; ++g)
      for (int b = 0; b < kDotBlocks; ++b) tot += partial[((i64)g * M + q) * kDotBlocks + b];
    B[st[2] * M + q] = tot;
    B[q * M + st[2]] = tot;
  }
}

void launch_diis_solve(const double* Bm, const int* st, int ld, double* coef, cudaStream_t) {
  if (!st[4]) return;
  const int m = st[3];
  const int n = m + 1;
  std::vector<double> A((size_t)n * (n + 1));
  double scale = 0.0;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) scale = std::fmax(scale, std::fabs(Bm[i * ld + j]));
  if (scale == 0.0) scale = 1.0;
  auto at = [&](int i, int j) -> double& { return A[(size_t)i * (n + 1) + j]; };
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) at(i, j) = (i < m && j < m) ? Bm[i * ld + j] / scale : (i == m && j == m ? 0.0 : 1.0);
    at(i, n) = i == m ? 1.0 : 0.0;
  }
  std::vector<int> ok(n);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(at(i, c)) > std::fabs(at(p, c))) p = i;
    if (p != c)
      for (int j = 0; j <= n; ++j) std::swap(at(c, j), at(p, j));
    ok[c] = std::fabs(at(c, c)) > 1e-14;
    if (!ok[c]) continue;
    for (int i = c + 1; i < n; ++i) {
      const double f = at(i, c) / at(c, c);
      for (int j = c; j <= n; ++j) at(i, j) -= f * at(c, j);
    }
  }
  std::vector<double> x(n);
  for (int c = n - 1; c >= 0; --c) {
    if (!ok[c]) { x[c] = 0.0; continue; }
    double s = at(c, n);
    for (int j = c + 1; j < n; ++j) s -= at(c, j) * x[j];
    x[c] = s / at(c, c);
  }
  for (int i = 0; i < m; ++i) coef[i] = x[i];
}

template <typename T>
void launch_diis_extrapolate(T* out, const T* hist, i64 stride, i64 n, const double* coef, const int* st,
                             cudaStream_t) {
  if (!st[4]) return;
  for (i64 i = 0; i < n; ++i) {
    double s = 0.0;
    for (int q = 0; q < st[3]; ++q) s += coef[q] * (double)hist[q * stride + i];
    out[i] = (T)s;
  }
}
template void launch_diis_extrapolate<double>(double*, const double*, i64, i64, const double*, const int*,
                                              cudaStream_t);
template void launch_diis_extrapolate<float>(float*, const float*, i64, i64, const double*, const int*,
                                             cudaStream_t);

template <typename TO, typename TI>
void launch_convert(TO* out, const TI* in, i64 n, cudaStream_t) {
  for (i64 i = 0; i < n; ++i) out[i] = (TO)in[i];
}
template void launch_convert<float, double>(float*, const double*, i64, cudaStream_t);
template void launch_convert<double, float>(double*, const float*, i64, cudaStream_t);
template void launch_convert<double, double>(double*, const double*, i64, cudaStream_t);

void launch_energy(const double* g, const double* t1, const double* t2, int o, int v, double*, double* out,
                   cudaStream_t) {
  double s = 0.0;
  for (int i = 0; i < o; ++i)
    for (int j = 0; j < o; ++j)
      for (int a = 0; a < v; ++a)
        for (int b = 0; b < v; ++b) {
          const double giajb = g[(((i64)i * v + a) * o + j) * v + b], gibja = g[(((i64)i * v + b) * o + j) * v + a];
          s += (2.0 * giajb - gibja) * (t2[(((i64)i * o + j) * v + a) * v + b] + t1[i * v + a] * t1[j * v + b]);
        }
  *out = s;
}

void launch_mp2(double* t2, const double* g, const double* e, int o, int v, cudaStream_t) {
  for (int i = 0; i < o; ++i)
    for (int j = 0; j < o; ++j)
      for (int a = 0; a < v; ++a)
        for (int b = 0; b < v; ++b)
          t2[(((i64)i * o + j) * v + a) * v + b] =
              g[(((i64)i * v + a) * o + j) * v + b] / (e[i] + e[j] - e[o + a] - e[o + b]);
}

template <typename T>
void launch_unpack_spin(const void* t3, int f32, int ntrip, const i64* base, const int* pos, int v, T* S,
                        cudaStream_t) {
  const i64 V3 = (i64)v * v * v;
  const i64 sv[3] = {(i64)v * v, v, 1};
  for (int t = 0; t < ntrip; ++t) {
    const i64 s0 = sv[pos[3 * t]], s1 = sv[pos[3 * t + 1]], s2 = sv[pos[3 * t + 2]];
    auto U = [&](int x, int y, int z) { return load_src(t3, f32, base[t] + x * s0 + y * s1 + z * s2); };
    for (i64 e = 0; e < V3; ++e) {
      const int c = (int)(e % v), b = (int)((e / v) % v), a = (int)(e / ((i64)v * v));
      S[t * V3 + e] = (T)(2.0 * U(a, b, c) - U(b, a, c) - U(c, b, a));
    }
  }
}
template void launch_unpack_spin<double>(const void*, int, int, const i64*, const int*, int, double*, cudaStream_t);
template void launch_unpack_spin<float>(const void*, int, int, const i64*, const int*, int, float*, cudaStream_t);

template <typename T>
void launch_r1_t3(const T* S, const double* oovv, int o, int v, double* dR1_z, double*, i64, cudaStream_t) {
  const i64 nslab = (i64)o * o * v, V2 = (i64)v * v;
  for (int a = 0; a < v; ++a) {
    double acc = 0.0;
    for (i64 s = 0; s < nslab; ++s)
      for (int c = 0; c < v; ++c)
        acc += oovv[s * v + c] * ((double)S[s * V2 + (i64)c * v + a] - 0.5 * (double)S[s * V2 + (i64)a * v + c]);
    dR1_z[a] += acc;
  }
}
template void launch_r1_t3<double>(const double*, const double*, int, int, double*, double*, i64, cudaStream_t);
template void launch_r1_t3<float>(const float*, const double*, int, int, double*, double*, i64, cudaStream_t);
template <typename T>
void launch_scatter_rows3(const float* X, int M, int v, const i64* row_base, const int* row_sel,
                          const double* row_alpha, T* C, cudaStream_t) {
  const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const i64 V3 = (i64)v * v * v, S[3] = {(i64)v * v, v, 1};
  for (int m = 0; m < M; ++m) {
    const int* p = P[row_sel[m]];
    for (i64 e = 0; e < V3; ++e) {
      const int a = (int)(e / ((i64)v * v)), b = (int)((e / v) % v), c = (int)(e % v);
      C[row_base[m] + a * S[p[0]] + b * S[p[1]] + c * S[p[2]]] += (T)(row_alpha[m] * (double)X[(i64)m * V3 + e]);
    }
  }
}
template void launch_scatter_rows3<float>(const float*, int, int, const i64*, const int*, const double*, float*,
                                          cudaStream_t);
template void launch_scatter_rows3<double>(const float*, int, int, const i64*, const int*, const double*, double*,
                                           cudaStream_t);
template <typename T>
void launch_t2_outer(T* r3, const T* Wvooo, const T* t2, const int4* blocks, int o, int v, i64 n3, cudaStream_t) {
  const i64 V3 = (i64)v * v * v;
  const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (i64 b = 0; b < n3; ++b) {
    const int occ[3] = {blocks[b].x, blocks[b].y, blocks[b].z};
    for (i64 x = 0; x < V3; ++x) {
      const int lab[3] = {(int)(x / ((i64)v * v)), (int)((x / v) % v), (int)(x % v)};
      double s = 0.0;
      for (int q = 0; q < 6; ++q) {
        const int i1 = occ[P[q][0]], i2 = occ[P[q][1]], i3 = occ[P[q][2]];
        const int a1 = lab[P[q][0]], a2 = lab[P[q][1]], a3 = lab[P[q][2]];
        for (int l = 0; l < o; ++l)
          s -= (double)Wvooo[(((i64)a1 * o + l) * o + i1) * o + i2] * (double)t2[(((i64)l * o + i3) * v + a2) * v + a3];
      }
      r3[b * V3 + x] = (T)((double)r3[b * V3 + x] + s);
    }
  }
}
template void launch_t2_outer<double>(double*, const double*, const double*, const int4*, int, int, i64, cudaStream_t);
template void launch_t2_outer<float>(float*, const float*, const float*, const int4*, int, int, i64, cudaStream_t);
}  // namespace rcc

// Test hook: the integer-path binary64 -> binary32 conversion of the panel gathers.
extern "C" void rcc_test_f64_to_f32(const double* x, float* y, long long n) {
  for (long long i = 0; i < n; ++i) y[i] = rcc::f64_to_f32_rn(x[i]);
}
