// Shared device-side definitions of the RCCSDT kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace rcc {

typedef long long i64;

// Operand storage of packed GEMM panels.
enum PanelKind : int { PANEL_F64 = 0, PANEL_BF16X2 = 1, PANEL_TF32X2 = 2 };
// (FP64 bodies on the tensor cores keep the FP64 panel and add its BF16 digit planes,
// kSlices x [rows][Kpad], with one scale exponent per row: see elem.cuh.)

// A packed panel out[r][k] (row-major, k contiguous) is gathered as
//   out[r][k] = sum_{t < nterm} coef[t*K + k] * src[colbase[t*K + k] + rowoff[sel[t*K + k]*R + r]]
// which covers strided views of dense tensors (nterm = 1, one selector) and
// permuted/spin-summed reads of compact T3 blocks (selector = virtual permutation).
struct PackArgs {
  const void* src;       // double or float
  int src_f32;           // 1: src is float
  int R, K, nterm;
  const double* coef;    // [nterm][K]
  const i64* colbase;    // [nterm][K]
  const int* sel;        // [nterm][K]
  const i64* rowoff;     // [nsel][R]
  int kind;              // PanelKind of the output
  void* out_hi;          // [R][Kpad] double / bf16 / float(tf32)
  void* out_lo;          // [R][Kpad] second half of a split (unused for F64)
  int Kpad;              // leading dimension of the output (>= K, zero filled)
  int read_k_fast;       // 1: source contiguous along k, 0: along r
  int one_sel;           // 1: every selector is 0 (rowoff is a single table of R entries)
  // Row offsets computed instead of looked up (rowoff then unused): rows are the
  // labels (x, y) (row_mode 2, R = lv^2) or (x, y, z) (row_mode 3, R = lv^3) in
  // base lv; with stored-block strides S = {lv^2, lv, 1}, selector s gives
  //   mode 2: x S[s / 3] + y S[s % 3]
  //   mode 3: x S[p0] + y S[p1] + z S[p2], (p0, p1, p2) the s-th of the six orderings.
  int row_mode;
  int lv;
};

// Table-driven epilogue: C[row_base[m] + col_off[row_sel[m]*N + n]] += row_alpha[m] * acc(m, n)
// where rows m >= m2 write to C2 instead of C (a GEMM whose stacked A operand
// feeds two output tensors of the same element type; C2 null: C only).
// With row_base2 set, every value is also added, times row_alpha2[m], at
// row_base2[m] + the same column offset of the same tensor (rows with
// row_base2[m] < 0 write once): the mirrored element of a pair-symmetric product.
// With col_off2 set instead, the second copy goes to row_base[m] + col_off2[n]
// (columns with col_off2[n] < 0 write once), times row_alpha2[m]: the same mirror
// when the pairs index the columns.
struct EpiArgs {
  void* C;               // double or float
  int c_f32;
  int M, N;
  const i64* row_base;   // [M]
  const int* row_sel;    // [M]
  const double* row_alpha; // [M]
  const i64* col_off;    // [nsel][N]
  void* C2;
  int m2;
  const i64* row_base2;     // [M] or null
  const double* row_alpha2; // [M] (with row_base2 or col_off2)
  const i64* col_off2;      // [N] or null (row_sel 0 only)
};

}  // namespace rcc
