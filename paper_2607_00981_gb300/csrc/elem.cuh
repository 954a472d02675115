// Per-element arithmetic shared by the device kernels and by the test-only host
// simulation build (RCC_HOSTSIM), so both execute the same plans.
#pragma once
#include "common.cuh"

#define RCC_HD __host__ __device__ __forceinline__

namespace rcc {

RCC_HD double load_src(const void* p, int f32, i64 off) {
  return f32 ? (double)((const float*)p)[off] : ((const double*)p)[off];
}

// Round-to-nearest, ties away from zero, to the 10-bit TF32 mantissa, done on the
// integer representation (finite inputs).  Returns the value as a float.
RCC_HD float tf32_round(float x) {
  union { float f; unsigned u; } c;
  c.f = x;
  c.u = (c.u + 0x1000u) & 0xffffe000u;
  return c.f;
}

// IEEE 754 binary64 -> binary32, round to nearest even, on the integer
// representation (no FP64 instructions: this part's FP64 pipe is about 1/64 of its
// FP32 rate, which made FP64-source panel gathers compute bound).  Overflow gives
// infinity, binary64 subnormals give zero, NaN stays NaN.
RCC_HD float f64_to_f32_rn(double x) {
  union { double d; unsigned long long u; } in;
  union { unsigned u; float f; } out;
  in.d = x;
  const unsigned long long b = in.u;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = b & 0xfffffffffffffull;
  if (e == 0x7ff) {
    out.u = sign | 0x7f800000u | (m ? 0x00400000u : 0u);
    return out.f;
  }
  int fe = e - 1023 + 127;
  if (fe >= 255) {
    out.u = sign | 0x7f800000u;
    return out.f;
  }
  unsigned long long sig = m;
  int shift = 29;  // 52 - 23 fraction bits dropped
  if (fe <= 0) {   // binary32 subnormal: value = q 2^-149, q = sig 2^(fe - 30)
    if (e == 0 || fe < -24) {
      out.u = sign;
      return out.f;
    }
    sig = m | (1ull << 52);
    shift = 30 - fe;
    fe = 0;
  }
  unsigned long long q = sig >> shift;
  const unsigned long long rem = sig & ((1ull << shift) - 1), half = 1ull << (shift - 1);
  if (rem > half || (rem == half && (q & 1ull))) ++q;
  // a carry out of the fraction moves into the exponent (up to infinity)
  out.u = sign | (unsigned)(((unsigned long long)fe << 23) + q);
  return out.f;
}

// FP64-accurate products on the BF16 tensor cores (the FP64 bodies' emulated GEMM):
// a row of an operand is scaled by 2^-e (e: its largest magnitude is below 2^e) and
// each element's magnitude, as a 42-bit fixed-point fraction N (round to nearest), is
// cut into six 7-bit digits d_0..d_5 (d_0 <= 128, the others <= 127), stored
// pre-scaled as a_s = sign * d_s * 2^(-7 s), which BF16 holds exactly:
//   x = 2^(e - 7) * sum_s a_s   (up to 2^-42 of the row's largest magnitude).
// Everything works on the binary64 bit patterns (subnormals count as zero).
constexpr int kSlices = 6;
RCC_HD unsigned long long f64_magnitude_bits(double x) {
  union { double d; unsigned long long u; } c;
  c.d = x;
  return c.u & 0x7fffffffffffffffull;  // orders like |x| for finite values
}
RCC_HD int slice_exponent(unsigned long long max_bits) {
  const int ex = (int)(max_bits >> 52);
  return ex == 0 ? 0 : ex - 1022;  // |x| < 2^(ex - 1023 + 1)
}
RCC_HD void slice_digits(double x, int e, float (&a)[kSlices]) {
  union { double d; unsigned long long u; } c;
  c.d = x;
  const int ex = (int)((c.u >> 52) & 0x7ff);
  unsigned long long n = 0;
  if (ex != 0) {
    const unsigned long long m = (c.u & 0xfffffffffffffull) | (1ull << 52);
    const int sh = 1033 + e - ex;  // N = m 2^(ex - 1033 - e), and |x| < 2^e makes sh >= 11
    if (sh < 64) n = (m + (1ull << (sh - 1))) >> sh;
  }
  const float sign = (c.u >> 63) ? -1.f : 1.f;
  const float d[kSlices] = {(float)(n >> 35), (float)((n >> 28) & 127), (float)((n >> 21) & 127),
                            (float)((n >> 14) & 127), (float)((n >> 7) & 127), (float)(n & 127)};
  float scale = sign;
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    a[s] = d[s] * scale;
    scale *= 0.0078125f;  // 2^-7
  }
}

// Stored-axis index of label q under ordering s (the six orderings, lexicographic).
RCC_HD int perm3(int s, int q) {
  // {0,1,2} {0,2,1} {1,0,2} {1,2,0} {2,0,1} {2,1,0}
  const int first = s >> 1;
  const int rest0 = first == 0 ? 1 : 0, rest1 = first == 2 ? 1 : 2;
  return q == 0 ? first : ((q == 1) == ((s & 1) == 0) ? rest0 : rest1);
}

// Row offset of row r under selector s (table or computed, see PackArgs).
RCC_HD i64 row_offset(const PackArgs& a, int s, int r) {
  if (a.row_mode == 0) return a.rowoff[(i64)s * a.R + r];
  const i64 v = a.lv;
  auto S = [v](int axis) { return axis == 0 ? v * v : (axis == 1 ? v : (i64)1); };
  if (a.row_mode == 2) return (r / a.lv) * S(s / 3) + (r % a.lv) * S(s % 3);
  const int x = r / (a.lv * a.lv), y = (r / a.lv) % a.lv, z = r % a.lv;
  return x * S(perm3(s, 0)) + y * S(perm3(s, 1)) + z * S(perm3(s, 2));
}

RCC_HD double pack_value(const PackArgs& a, int r, int k) {
  double s = 0.0;
  for (int t = 0; t < a.nterm; ++t) {
    const i64 idx = (i64)t * a.K + k;
    const double c = a.coef[idx];
    if (c != 0.0) {
      const i64 off = a.colbase[idx] + row_offset(a, a.sel[idx], r);
      s += c * load_src(a.src, a.src_f32, off);
    }
  }
  return s;
}

RCC_HD void store_panel(const PackArgs& a, int r, int k, double x) {
  const i64 o = (i64)r * a.Kpad + k;
  if (a.kind == PANEL_F64) {
    ((double*)a.out_hi)[o] = x;
  } else if (a.kind == PANEL_BF16X2) {
    const __nv_bfloat16 hi = __float2bfloat16_rn((float)x);
    const double rem = x - (double)__bfloat162float(hi);
    ((__nv_bfloat16*)a.out_hi)[o] = hi;
    ((__nv_bfloat16*)a.out_lo)[o] = __float2bfloat16_rn((float)rem);
  } else {
    const float hi = tf32_round((float)x);
    ((float*)a.out_hi)[o] = hi;
    ((float*)a.out_lo)[o] = tf32_round((float)(x - (double)hi));
  }
}

// FP32 variants for FP32 sources packed into split panels (no FP64 arithmetic).
RCC_HD float pack_value_f(const PackArgs& a, int r, int k) {
  float s = 0.f;
  for (int t = 0; t < a.nterm; ++t) {
    const i64 idx = (i64)t * a.K + k;
    const float c = (float)a.coef[idx];
    if (c != 0.f) {
      const i64 off = a.colbase[idx] + row_offset(a, a.sel[idx], r);
      s += c * ((const float*)a.src)[off];
    }
  }
  return s;
}

RCC_HD void store_panel_f(const PackArgs& a, int r, int k, float x) {
  const i64 o = (i64)r * a.Kpad + k;
  if (a.kind == PANEL_BF16X2) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    ((__nv_bfloat16*)a.out_hi)[o] = hi;
    ((__nv_bfloat16*)a.out_lo)[o] = __float2bfloat16_rn(x - __bfloat162float(hi));
  } else {
    const float hi = tf32_round(x);
    ((float*)a.out_hi)[o] = hi;
    ((float*)a.out_lo)[o] = tf32_round(x - hi);
  }
}

// Pair-symmetric operands of the pp-ladder.  Pairs of virtual labels are
// numbered tile-major: the 16-label tiles P <= Q form chunks, and inside a chunk
// of n0 x n1 labels the pair of local labels (a, b) sits at a n1 + b (P < Q), or,
// on a diagonal chunk (P = Q, n0 = n1), row-major over a <= b (plus) or a < b
// (minus).  Returns the local pair of index idx.
RCC_HD void pair_decode(int idx, bool diag, bool plus, int n0, int n1, int& a, int& b) {
  if (!diag) {
    a = idx / n1;
    b = idx - a * n1;
    return;
  }
  a = 0;
  int len = plus ? n0 : n0 - 1;
  while (idx >= len) {
    idx -= len;
    ++a;
    --len;
  }
  b = a + (plus ? 0 : 1) + idx;
}

// One element of a K-major panel of `kind` (FP64, or split into hi + lo planes
// from the FP32 value of x).
RCC_HD void panel_put(int kind, void* out_hi, void* out_lo, i64 o, double x) {
  if (kind == PANEL_F64) {
    ((double*)out_hi)[o] = x;
  } else if (kind == PANEL_BF16X2) {
    const float f = f64_to_f32_rn(x);  // integer-path rounding (no FP64 pipe)
    const __nv_bfloat16 hi = __float2bfloat16_rn(f);
    ((__nv_bfloat16*)out_hi)[o] = hi;
    ((__nv_bfloat16*)out_lo)[o] = __float2bfloat16_rn(f - __bfloat162float(hi));
  } else {
    const float f = f64_to_f32_rn(x);
    const float hi = tf32_round(f);
    ((float*)out_hi)[o] = hi;
    ((float*)out_lo)[o] = tf32_round(f - hi);
  }
}

// The same for an FP32 value (no round trip through FP64: on this part the FP64
// units convert at a small fraction of the FP32 rate).
RCC_HD void panel_put_f(int kind, void* out_hi, void* out_lo, i64 o, float f) {
  if (kind == PANEL_F64) {
    ((double*)out_hi)[o] = (double)f;
  } else if (kind == PANEL_BF16X2) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(f);
    ((__nv_bfloat16*)out_hi)[o] = hi;
    ((__nv_bfloat16*)out_lo)[o] = __float2bfloat16_rn(f - __bfloat162float(hi));
  } else {
    const float hi = tf32_round(f);
    ((float*)out_hi)[o] = hi;
    ((float*)out_lo)[o] = tf32_round(f - hi);
  }
}

// Output tensor of row m (see EpiArgs).
RCC_HD void* epi_out(const EpiArgs& e, int m) { return (e.C2 && m >= e.m2) ? e.C2 : e.C; }

RCC_HD void epi_apply(const EpiArgs& e, int m, int n, double acc) {
  const i64 co = e.col_off[(i64)e.row_sel[m] * e.N + n];
  const bool rowm = e.row_base2 && e.row_base2[m] >= 0, colm = e.col_off2 && e.col_off2[n] >= 0;
  const int nout = (rowm || colm) ? 2 : 1;
  for (int q = 0; q < nout; ++q) {
    const i64 addr = q == 0 ? e.row_base[m] + co : (rowm ? e.row_base2[m] + co : e.row_base[m] + e.col_off2[n]);
    const double val = (q ? e.row_alpha2[m] : e.row_alpha[m]) * acc;
    if (e.c_f32)
      ((float*)epi_out(e, m))[addr] += (float)val;
    else
      ((double*)epi_out(e, m))[addr] += val;
  }
}

// ---------------------------------------------------------------------------
// Compact-block helpers.  blk(i<=j<=k) = C(k+2,3) + C(j+1,2) + i.
// ---------------------------------------------------------------------------
RCC_HD i64 blk_index(int i, int j, int k) {
  return (i64)k * (k + 1) * (k + 2) / 6 + (i64)j * (j + 1) / 2 + i;
}

// Virtual element offset inside a v^3 block for labels (x0, x1, x2) of one
// triple, given the stored-axis position of each label: pos[q] = stored axis
// that label q lands on.
RCC_HD i64 perm_offset(int v, const int* pos, int x0, int x1, int x2) {
  i64 s[3];
  s[0] = (i64)v * v; s[1] = v; s[2] = 1;
  return s[pos[0]] * x0 + s[pos[1]] * x1 + s[pos[2]] * x2;
}

// Post-processing of one element of a compact R3 block (Sec. II.D):
// symmetrise degenerate blocks, purify i=j=k, subtract the S3 mean.
// r points at the block; returns the processed value at (a, b, c).
// Arithmetic in the storage type T (FP32 storage computes in FP32).
template <typename T>
RCC_HD T post_value(const T* r, int v, int i, int j, int k, int a, int b, int c) {
  if (i == j && j == k) return (T)0;
  const i64 V2 = (i64)v * v;
  const T rabc = r[a * V2 + b * v + c], racb = r[a * V2 + c * v + b];
  const T rbac = r[b * V2 + a * v + c], rbca = r[b * V2 + c * v + a];
  const T rcab = r[c * V2 + a * v + b], rcba = r[c * V2 + b * v + a];
  T s;
  if (i == j)
    s = (T)0.5 * (rabc + rbac);
  else if (j == k)
    s = (T)0.5 * (rabc + racb);
  else
    s = rabc;
  // the symmetrisations above keep the sum over the six permutations unchanged
  const T mean = (rabc + racb + rbac + rbca + rcab + rcba) * (T)(1.0 / 6.0);
  return s - mean;
}

}  // namespace rcc
