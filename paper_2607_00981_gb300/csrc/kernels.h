// Launch wrappers of the RCCSDT kernels (host-callable).
#pragma once
#include <cuda.h>

#include "common.cuh"

namespace rcc {

constexpr int kDotBlocks = 608;
extern long long g_launch_count;  // 4 x 152 SMs, fixed so reductions are deterministic

struct CombineArgs {
  double* out;
  i64 total;
  int rank;
  i64 shape[6];
  i64 ostride[6];
  int nterm;
  const double* in[4];
  i64 istride[4][6];
  double coef[4];
  double beta;
  // filled by launch_combine: 32-bit index division by shape[d] as a multiply-high
  // and shift (Granlund & Montgomery, PLDI 1994, round-up method) when total < 2^31
  unsigned fdm[6];
  int fdl[6];
};

void launch_pack(const PackArgs& a, cudaStream_t s);
// Grouped gathers (FP32 sources into split panels): list and tile0 in device
// memory, tile0[p] = sum of pack_tiles_of() over the gathers before p.
int pack_tiles_of(const PackArgs& a);
void launch_pack_grouped(const PackArgs* list, const int* tile0, int npack, int total_tiles, int f32_src,
                         cudaStream_t s);
// Output-stationary reduction into compact R3: target block t (element offset
// target[t] into r3) receives, in order, the contributions cstart[t] ..
// cstart[t+1]-1: alpha * X[xoff + permuted v^3 block] with the virtual
// permutation csel (index into the 6 orderings, X axis q -> stored axis).
// accumulate = 0 overwrites the target blocks.
template <typename T>
void launch_r3_gather(const float* X, const i64* target, int ntarget, const int* cstart, const i64* xoff,
                      const int* csel, const float* calpha, int v, int accumulate, T* r3, cudaStream_t s);
void launch_gemm_f64(const double* A, const double* B, int K, int lda, int ldb, const EpiArgs& e,
                     double* scratch, i64 scratch_elems, cudaStream_t s);
void launch_combine(const CombineArgs& c, cudaStream_t s);
// Symmetrise, purify and orthogonalise compact R3 (r -> rp) and, in the same pass,
// *norm2 = sum over blocks of wblk[b] |rp_b|^2 (fixed-order sums over the
// post_partials(v, n3) entries of `partial`).
template <typename T>
void launch_post(const T* r, T* rp, const int4* blocks, int v, i64 n3, const double* wblk, double* partial,
                 double* norm2, cudaStream_t s);
int post_partials(int v, i64 n3);
void launch_update_t12(double* t1, const double* r1, double* t2, const double* r2, const double* e,
                       int o, int v, double shift, cudaStream_t s);
template <typename T>
void launch_update_t3(T* t3, const T* rp3, const double* e, const int4* blocks, int o, int v, i64 n3,
                      double shift, cudaStream_t s);
template <typename T>
void launch_wdot(const T* x, const T* y, i64 n, i64 seg, const double* w, double* partial, double* out,
                 double scale, int accumulate, cudaStream_t s);
// DIIS with device-side bookkeeping (st[8]: updates, entries written, slot, entries
// in use, extrapolate flag); every launch reads the state, none needs the host.
void launch_diis_begin(int* st, int M, int diis_start, cudaStream_t s);
template <typename T>
void launch_slot_save(char* base, i64 stride, i64 off, const int* st, const T* src, i64 n, cudaStream_t s);
template <typename T>
void launch_slot_diff_store(char* hist_t, char* hist_e, i64 stride, i64 off, const int* st, const T* t, i64 n,
                            cudaStream_t s);
// Virtual-subspace part of compact T3: sub[n3][ns][ns][ns] = t3[.][a<ns][b<ns][c<ns]
// (dir 0), or written back into t3 (dir 1).
template <typename T>
void launch_subcube(T* t3, T* sub, i64 n3, int v, int ns, int dir, cudaStream_t s);
template <typename T>
void launch_diis_dots(const char* hist_e, i64 stride, i64 off, const int* st, int M, i64 n, i64 seg, const double* w,
                      double* partial, cudaStream_t s);
void launch_diis_row(const double* partial, int nseg, const int* st, int M, double* B, cudaStream_t s);
void launch_diis_solve(const double* B, const int* st, int ld, double* coef, cudaStream_t s);
template <typename T>
void launch_diis_extrapolate(T* out, const T* hist, i64 stride, i64 n, const double* coef, const int* st,
                             cudaStream_t s);
template <typename TO, typename TI>
void launch_convert(TO* out, const TI* in, i64 n, cudaStream_t s);

// tcgen05 split-precision GEMM (gemm_tc.cu): C += alpha * (Ahi Bhi + Ahi Blo + Alo Bhi)
// with A [M][Kpad], B [N][Kpad] in two planes each.  kind: PANEL_BF16X2 or PANEL_TF32X2.
// Returns 0 on success, nonzero if the configuration is unsupported.
// `scratch` (scratch_elems floats) holds FP32 partial tiles when K is split.
// With raw_out, the raw FP32 result is written densely to raw_out[m * N + n] (no
// alpha, no scatter, no split-K) for a separate scatter pass.
// bn: tile width, 256 (default), 144 or 128 columns.
// colmajor (raw output only): the result is stored as raw_out[n * M + m].
int launch_gemm_tc(int kind, const void* Ahi, const void* Alo, const void* Bhi, const void* Blo,
                   int Kpad, const EpiArgs& e, int* status_flag, long long watchdog, cudaStream_t s,
                   float* scratch, long long scratch_elems, float* raw_out = nullptr, int bn = 256,
                   int colmajor = 0);
// One GEMM of a grouped launch: X[M][N] = (Ahi Bhi + Ahi Blo + Alo Bhi) with A
// [M][Kpad], B [N][Kpad] split panels; the tensor maps are encoded on the host
// (make_gproblem) and the table is copied to device memory before the launch.
struct alignas(128) GProblem {
  CUtensorMap ah, al, bh, bl;
  const void* a_hi;
  const void* a_lo;
  const void* b_hi;
  const void* b_lo;
  float* out;  // dense FP32 result, row-major [M][N] (colmajor: [N][M])
  int M, N, Kpad, kblocks, mt, nt;
  int tile0;   // first tile of this problem in the launch's tile order (set by the caller)
  int colmajor;
};
// Fills p (except tile0) for panels of `kind`; nonzero if unsupported.
int make_gproblem(GProblem* p, int kind, const void* Ahi, const void* Alo, const void* Bhi, const void* Blo, int M,
                  int N, int Kpad, float* out, int bn = 256);
int gproblem_tiles(const GProblem& p);
int gemm_tc_block_k(int kind, int bn);
// One persistent launch over every tile of the nprob problems (device table,
// tile0 prefix order, tables made with the same bn); grid <= 0 picks one CTA per SM.
// FP64-accurate GEMM on the BF16 tensor cores (digit planes, see elem.cuh):
// launch_slice_f64 cuts an FP64 panel [R][Kpad] into kSlices BF16 planes
// [kSlices][R][Kpad] and one scale exponent per row; launch_gemm_f64e then applies
// the table epilogue e (FP64 or FP32 outputs, FP64 arithmetic) to the product of two such panels.
// Kpad a multiple of 64.  Returns nonzero for an unsupported configuration.
void launch_slice_f64(const double* P, int R, int Kpad, void* planes, int* exps, cudaStream_t s);
int launch_gemm_f64e(const void* Aplanes, const int* ea, const void* Bplanes, const int* eb, int Kpad, const EpiArgs& e,
                     int* status_flag, long long watchdog, cudaStream_t s);
int launch_gemm_tc_grouped(int kind, const GProblem* probs, int nprob, int total_tiles, int grid, int bn,
                           int* status_flag, long long watchdog, cudaStream_t s);
// The same with the tile count and every problem's tile0 read from device memory
// when the kernel starts (written by an earlier kernel: problems of instances that
// do not run this time get no tiles); max_tiles bounds the grid.
int launch_gemm_tc_grouped_dev(int kind, const GProblem* probs, int nprob, int max_tiles, const int* total_dev,
                               int grid, int bn, int* status_flag, long long watchdog, cudaStream_t s);
// Operand panels read from compact T3 through label cubes (cube_pack.cu).
struct CubeTerm {
  i64 base;    // element offset of the stored block
  float coef;
  int pos;     // stored axis of labels L0, L1, L2: pos0 | pos1 << 2 | pos2 << 4
};
struct CubePiece {
  int dst;     // index into the destination table (0 without a table)
  int k0;      // mode 0: panel column of L0 = 0; mode 1: the piece's column
  i64 row0;    // panel row of the labels' origin
  int nterm;   // 0 (zeros), 1..3 (mode 1: at most 1)
  int ks1;     // mode 0: K stride of L1 (0 when L1 indexes rows)
  int rs1, rs2;  // mode 0: row strides of L1 and L2
  CubeTerm t[3];
};
struct CubeDst {
  void* out_hi;
  void* out_lo;
  int Kpad;
};
// mode 0: K = k0 + L0 + L1 ks1, rows row0 + L1 rs1 + L2 rs2 (pieces in any order);
// mode 1: K = k0, rows row0 + L0 v^2 + L1 v + L2, pieces in groups of 16 consecutive
// columns of one panel (npieces a multiple of 16).  Panels of `kind` (split).
void launch_cube_pack(int mode, int kind, const CubePiece* pieces, int npieces, const CubeDst* dsts,
                      const CubeDst& d0, const float* src, int v, cudaStream_t s);
// Mode 0 for the S panels of step (iii) (pieces ordered by (z, x, y), ppz per z),
// also writing the per-cube partial sums of the T3 term of R1 to `part`
// [npieces][cubes][32] (w + wbase[p] = v^{xy}_{..} of piece p as [v][v] floats);
// launch_r1_cubes_reduce then adds them into dR1[z][a] for z < nz (dR1 at z0).
void launch_cube_pack_r1(int kind, const CubePiece* pieces, int npieces, const CubeDst& d0,
                         const float* src, int v, const float* w, const i64* wbase, float* part, cudaStream_t s);
void launch_r1_cubes_reduce(const float* part, int ppz, int nz, int v, double* dR1, cudaStream_t s);
// Pair-symmetric pp-ladder panels (pair_pack.cu).  Chunk (P, Q), P <= Q, of the
// 16-label tiles holds its pairs at K offsets offp (d <= e) and offm (d < e); inside
// a chunk pairs are numbered as pair_decode (elem.cuh) describes.
struct PairChunk {
  int P, Q, offp, offm;
};
// A panels: row m of dp is the pair (x, y) = rows[m].x, .y (x <= y) with
// dp[m][k] = W^{xy}_{de} + W^{xy}_{ed} (W^{xy}_{dd} for d = e), and row rows[m].z
// (>= 0 when x < y) of dm holds W^{xy}_{de} - W^{xy}_{ed}; (d, e) the pair of
// column k.  W is FP64 [x][y][d][e]; Kp = v(v+1)/2, Km = v(v-1)/2 columns, the
// padding up to each Kpad zero.
void launch_pair_pack_w(int kind, const double* W, int v, const int4* rows, int Mp, const PairChunk* ch, int nchunk,
                        int Kp, int Km, const CubeDst& dp, const CubeDst& dm, cudaStream_t s);
// B panels of one view of the stored blocks b0 .. b0 + nblk - 1 (element strides
// sd, se, sw of the view's axes d, e, w inside a v^3 block): row (blk - b0) v + w,
// dp = T(d, e, w) + T(e, d, w), dm = T(d, e, w) - T(e, d, w); padding zero.
// FP32 T3 fills any panel kind, FP64 T3 FP64 panels.
void launch_pair_pack_t(int kind, const void* t3, int t3_f32, i64 b0, int nblk, int v, i64 sd, i64 se, i64 sw,
                        const PairChunk* ch, int nchunk, int Kp, int Km, const CubeDst& dp, const CubeDst& dm,
                        cudaStream_t s);
// The same for one view of compact T4 blocks (v^4, a second free label w1 at stride sr):
// row ((blk - b0) v + w1) v + w, dp = T(d, e, w1, w) + T(e, d, w1, w), dm = the difference.
void launch_pair_pack_t4(int kind, const void* t4, int t4_f32, i64 b0, int nblk, int v, i64 sd, i64 se, i64 sw,
                         i64 sr, const PairChunk* ch, int nchunk, int Kp, int Km, const CubeDst& dp,
                         const CubeDst& dm, cudaStream_t s);
// Zero the panel columns [k0, Kpad) of `rows` rows.
void launch_zero_cols(const CubeDst& d, i64 rows, int k0, int kind, cudaStream_t s);
// Second phase of a two-phase scatter: for each row m of the dense FP32 result X
// [M][v^3] (natural (a,b,c) order), C[row_base[m] + perm_sel[m](a,b,c)] +=
// row_alpha[m] * X[m][abc]; perm_sel indexes the 6 virtual permutations.
template <typename T>
void launch_scatter_rows3(const float* X, int M, int v, const i64* row_base, const int* row_sel,
                          const double* row_alpha, T* C, cudaStream_t s);

}  // namespace rcc

namespace rcc {
// E partials: sum_{ijab} (2 g[i,a,j,b] - g[i,b,j,a]) (t2[i,j,a,b] + t1[i,a] t1[j,b]), g = (ia|jb)
void launch_energy(const double* g, const double* t1, const double* t2, int o, int v, double* partial,
                   double* out, cudaStream_t s);
// t2[i,j,a,b] = g[i,a,j,b] / (e_i + e_j - e_a - e_b)
void launch_mp2(double* t2, const double* g, const double* e, int o, int v, cudaStream_t s);
// For each of ntrip occupied triples: U = t_{trip} unpacked from compact storage,
// S = (2 - P_a^b - P_a^c) U  (output [ntrip][v^3])
template <typename T>
void launch_unpack_spin(const void* t3, int f32, int ntrip, const i64* base, const int* pos, int v, T* S,
                        cudaStream_t s);
// dR1_z[a] += sum_{x,y,b,c} v^{xy}_{bc} (S[x,y,b,c,a] - 1/2 S[x,y,b,a,c]) (T3 term of R1, one batch z)
template <typename T>
void launch_r1_t3(const T* S, const double* oovv, int o, int v, double* dR1_z, double* scratch, i64 scratch_elems,
                  cudaStream_t s);
// T2-driven R3 term with K = o, all six column permutations, output-stationary
// (Wvooo[a][l][i][j], t2[l][k][b][c] in the precision T of R3).
template <typename T>
void launch_t2_outer(T* r3, const T* Wvooo, const T* t2, const int4* blocks, int o, int v, i64 n3, cudaStream_t s);
}  // namespace rcc
