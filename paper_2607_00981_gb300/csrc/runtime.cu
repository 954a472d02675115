// Host runtime of the RCCSDT library: context, plans, iteration driver, C ABI.
//
// Every contraction of one iteration is planned once, when the context is
// created: operand panels are described by gather tables (PackArgs) and the
// output by a scatter table (EpiArgs); an iteration only launches kernels.
// Dense contractions are written as einsum-like specs (appendix A.5 term by
// term); the compact-T3 terms of Eq. resi-rccsdt use hand-built tables:
//   pp-ladder   direct traversal, three GEMM views of each stored block
//               (W^{ab}_{de} t^{dec}, W^{ac}_{de} t^{dbe}, W^{bc}_{de} t^{ade}), Sec. II.C.1
//   ring, hh    unpacking (Sec. II.C.2): for a fixed pair of occupied indices the
//               unpacked (and spin-summed) blocks form one GEMM operand; the GEMM
//               result X_{ijk} for every i lands in the stored block sorted(i,j,k)
//               with the virtual axes permuted by the same sort and a weight that
//               counts the column permutations mapping onto that triple.  For a
//               block with two equal occupied indices this accumulates twice the
//               sum over the coset representatives, which the symmetrisation of
//               Sec. II.D.1 turns into the exact permutation-operator sum.
//   F_vv, F_oo  folded into W_vvvv and W_oooo, the groupings (F^v_v + W^vv_vv) and
//               (F^o_o + W^oo_oo) of steps (iv) and (v) of Sec. III.A.2.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <array>
#include <limits>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/rccsdt.h"
#include "elem.cuh"
#include "internal.h"
#include "solve_sm.h"
#include "kernels.h"

using rcc::i64;

namespace {

// ---------------------------------------------------------------------------
// Device abstraction (the test-only host simulation swaps these for host calls)
// ---------------------------------------------------------------------------
#ifdef RCC_HOSTSIM
void* dev_alloc(size_t bytes, int* err) {
  void* p = calloc(bytes ? bytes : 1, 1);
  if (!p) *err = RCCSDT_ERR_OOM;
  return p;
}
void dev_free(void* p) { free(p); }
int dev_copy(void* dst, const void* src, size_t bytes, cudaStream_t) {
  memcpy(dst, src, bytes);
  return 0;
}
int dev_zero(void* p, size_t bytes, cudaStream_t) {
  memset(p, 0, bytes);
  return 0;
}
int dev_sync(cudaStream_t) { return 0; }
int dev_check() { return 0; }
#else
void* dev_alloc(size_t bytes, int* err) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    *err = RCCSDT_ERR_OOM;
    return nullptr;
  }
  cudaMemset(p, 0, bytes ? bytes : 16);
  return p;
}
void dev_free(void* p) {
  if (p) cudaFree(p);
}
int dev_copy(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s) == cudaSuccess ? 0 : RCCSDT_ERR_CUDA;
}
int dev_zero(void* p, size_t bytes, cudaStream_t s) {
  return cudaMemsetAsync(p, 0, bytes, s) == cudaSuccess ? 0 : RCCSDT_ERR_CUDA;
}
int dev_sync(cudaStream_t s) { return cudaStreamSynchronize(s) == cudaSuccess ? 0 : RCCSDT_ERR_CUDA; }
int dev_check() { return cudaGetLastError() == cudaSuccess ? 0 : RCCSDT_ERR_CUDA; }
#endif
i64 n3_of(int o) { return (i64)o * (o + 1) * (o + 2) / 6; }
int multiplicity(int i, int j, int k) {
  if (i == j && j == k) return 1;
  if (i == j || j == k || i == k) return 3;
  return 6;
}
// pos[q] = stored axis of position q after sorting (occ[0], occ[1], occ[2]); stable.
void sort_positions(const int occ[3], int pos[3], int sorted[3]) {
  int idx[3] = {0, 1, 2};
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b)
      if (occ[idx[b]] < occ[idx[a]]) std::swap(idx[a], idx[b]);
  for (int s = 0; s < 3; ++s) {
    pos[idx[s]] = s;
    sorted[s] = occ[idx[s]];
  }
}

// ---------------------------------------------------------------------------
// Owned device buffer
// ---------------------------------------------------------------------------
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { dev_free(p); }
  double* d() const { return (double*)p; }
  float* f() const { return (float*)p; }
};

// A strided view of a dense tensor (element strides).
struct View {
  void* p = nullptr;
  int f32 = 0;
  std::vector<i64> shape, stride;
};

View dense(void* p, std::vector<i64> shape, int f32 = 0) {
  View v;
  v.p = p;
  v.f32 = f32;
  v.shape = shape;
  v.stride.assign(shape.size(), 1);
  for (int d = (int)shape.size() - 2; d >= 0; --d) v.stride[d] = v.stride[d + 1] * shape[d + 1];
  return v;
}

// Restrict dimension `dim` to [start, start + len).
View sub(View v, int dim, i64 start, i64 len) {
  v.p = (char*)v.p + start * v.stride[dim] * (v.f32 ? 4 : 8);
  v.shape[dim] = len;
  return v;
}

}  // namespace

// ---------------------------------------------------------------------------
// Plans
// ---------------------------------------------------------------------------
struct PackPlan {
  rcc::PackArgs a{};
  std::unique_ptr<DBuf> coef, colbase, sel, rowoff;
};

struct EpiPlan {
  rcc::EpiArgs e{};
  std::unique_ptr<DBuf> row_base, row_sel, row_alpha, col_off;
};

struct GemmPlan {
  PackPlan A, B;        // A panel rows = M, B panel rows = N, common K
  EpiPlan E;
  int K = 0, Kpad = 0;
  double fma = 0;
  int big = 0;          // large contraction (reported; every contraction runs split in split modes)
  int f64_only = 0;     // always FP64 (the bare integrals of the energy and the MP2 guess)
  int step = 0;         // timing bucket
  int reuse_A = 0;      // the A panel packed by the previous plan of the group is still valid
  int reuse_B = 0;      // likewise for the B panel
  // Two-phase scatter on the tensor cores: the GEMM result X [M][N] is written
  // densely; consecutive groups of M / s3_rows rows form one v^3 block of X whose
  // axes map to stored axes by s3_sel, added to C[s3_base] with weight s3_alpha.
  int s3_rows = 0;
  std::unique_ptr<DBuf> s3_base, s3_sel, s3_alpha;
  // host copies of the block tables (grouped residual); swap_ab: the grouped form
  // exchanges the operands so that each v^3 block of the result is contiguous
  std::vector<i64> h_base;
  std::vector<int> h_sel;
  std::vector<double> h_alpha;
  int swap_ab = 0;
  // split modes: the tensor-core GEMM runs with the operands exchanged and stores its
  // result column-major (same dense layout), so that a short M becomes the tile width
  int tc_swap = 0;
  // split modes: the B operand is gathered from T3 through label cubes (cube_pack.cu)
  std::vector<rcc::CubePiece> h_cube;
  std::unique_ptr<DBuf> cube;
  int cube_mode = -1;
  const float* cube_src = nullptr;  // the pieces' source (default: the B operand's)
  // step (iii): the cube gather also forms the partial sums of the T3 term of R1
  // (per piece, the offset of v^{xy} in the FP32 copy of the oovv integrals)
  std::unique_ptr<DBuf> r1_wbase;
  // stacked rows: the A panel is the concatenation of these plans' A operands
  // (each packed into its row range); the plan stands for all of them
  std::vector<GemmPlan*> a_parts;
  // split modes: an A panel of its own, shared by plans with the same A operand (the
  // step (iii) plans of every z batch); the plan with own_pack packs it, the others
  // reuse it while own_kind matches
  struct OwnPanel {
    DBuf hi, lo;
    int kind = -1;
  };
  std::shared_ptr<OwnPanel> own;
  int own_pack = 0;
};

struct rccsdt_ctx {
  int o = 0, v = 0, n = 0, naux = 0;
  i64 n3 = 0, V3 = 0;
  rccsdt_options opt{};
  int precision = RCCSDT_FP64;
  cudaStream_t stream = nullptr;
  std::string err;
  int have_ham = 0, have_amp = 0, have_int = 0, have_res = 0;
  int timing = 0;
  int concurrent = 0;  // other contexts share the GPU (batch): GEMMs keep their natural grids
  int batch_gemm = 0;  // a batch runs this context's grouped GEMM in its own batch-wide launch
  double step_ms[16] = {0};
  // event pool for non-blocking interval timing: tag < 16 = step slots, 16 = GEMM engine
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_tag;
  std::vector<double> ev_flop;
  int ev_used = 0;
  long long launches = 0;
  size_t total_bytes = 0;

  // buffers
  std::map<std::string, std::unique_ptr<DBuf>> buf;
  std::vector<std::unique_ptr<GemmPlan>> plans;
  // panels (engine scratch)
  std::unique_ptr<DBuf> panelA_hi, panelA_lo, panelB_hi, panelB_lo;
  size_t panel_bytes = 0;
  int panel_rows = 0;  // the most rows of any operand panel
  int packedA_kind = -1, packedB_kind = -1;  // panel kinds last written (reuse needs a match)
  // FP64 contractions on the tensor cores: digit planes and row exponents of the
  // FP64 panels (which stay in panelA_hi / panelB_hi)
  std::unique_ptr<DBuf> planesA, planesB, expA, expB;
  // the planes hold the current FP64 panels cut into rows of this many K values
  // (0: stale; a reused panel read with another row length is cut again)
  int slicedA = 0, slicedB = 0;

  // plan groups
  std::vector<GemmPlan*> p_dress, p_fock, p_eri, p_int, p_r12, p_energy_bare;
  std::vector<std::vector<GemmPlan*>> p_a3;  // per batch of a3_Z values of z
  std::vector<GemmPlan*> p_wbar;             // the W-bar contractions before step (iii)
  int a3_Z = 1;
  int a3_direct = 0;  // batches whose split-body panels are gathered from T3 (all of them, or none used)
  std::vector<GemmPlan*> p_pp, p_hh, p_ringab, p_ringc, p_t2a;
  // pp-ladder of the per-plan engine on pair-symmetric operands (pair_pack.cu): the
  // sum and difference parts of each view of a block range, two GEMMs per unit
  struct PpSym {
    int on = 0, nchunk = 0, Kp = 0, Km = 0, Kpadp = 0, Kpadm = 0;
    std::unique_ptr<DBuf> chunks, rows;  // PairChunk[nchunk], int4[Kp] (x, y, row of the difference)
    std::unique_ptr<DBuf> rb[3][2], rb2[3][2], al[2], al2[2], sel;  // per view / part: row tables
    struct Unit {
      int term = 0, nblk = 0, N = 0, swap = 0;
      i64 b0 = 0;
      std::unique_ptr<DBuf> col;  // [N] column offsets into R3
      rcc::EpiArgs e[2]{};        // sum and difference GEMMs
      double fma[2] = {0, 0};
    };
    std::vector<std::unique_ptr<Unit>> units;
  } pps;
  // combines
  std::vector<rcc::CombineArgs> c_fock, c_helpers, c_int_base, c_r12_base, c_r2_sym, c_wt;
  rcc::CombineArgs c_Lt_copy{}, c_ft_copy{};
  std::vector<std::vector<rcc::CombineArgs>> c_int_after;
  // per-z unpack tables for a3
  std::unique_ptr<DBuf> a3_base, a3_pos;

  // Grouped residual (split modes): every tensor-core contraction of the R3
  // residual in one grouped GEMM launch, its operands gathered by two grouped
  // launches, its results reduced into R3 by one output-stationary launch.
  struct Grouped {
    int on = 0, kind = -1;
    size_t bytes = 0;
    std::unique_ptr<DBuf> panels, raw;
    std::unique_ptr<DBuf> packs[2], ptile[2];  // [0] FP64 sources, [1] FP32 sources
    int npack[2] = {0, 0}, ntile[2] = {0, 0};
    std::unique_ptr<DBuf> cubes[2], cube_dst;     // label-cube gathers from T3, modes 0 and 1
    int ncube[2] = {0, 0};
    std::unique_ptr<DBuf> probs;
    int nprob = 0, ntiles = 0, grid = 0;
    double flop = 0.0;
    std::unique_ptr<DBuf> target, cstart, xoff, csel, calpha;
    int ntarget = 0;
    // launch shape: tile width, problem order (0 longest K first, 1 plan order), grid
    int bn = 256, ord = 0, tuned = 0;
    double tuned_ms = 0.0, fixed_ms = 0.0;
    struct Src {
      const void *ahi, *alo, *bhi, *blo;
      int M, N, Kpad;
      float* out;
      int colmajor;
    };
    std::vector<Src> src;
  } gr;

  // DIIS state
  int diis_count = 0, iter = 0;
  std::unique_ptr<DBuf> blocks_info, blk_weight;
  std::unique_ptr<DBuf> hist_t, hist_e;     // M slots each: t1 | t2 | t3 (padded)
  i64 hist_stride = 0;                      // bytes per slot
  i64 seg1 = 0, seg2 = 0, seg3 = 0;         // element counts
  int ns = 0;                               // virtual orbitals of the T3 part of the DIIS vectors
  std::unique_ptr<DBuf> diis_st, diis_partial;  // device DIIS counters int[8]; dot partials [3][M][blocks]
  std::unique_ptr<DBuf> scalars, partial, splitk, rawX;

  DBuf* B(const std::string& k) { return buf.at(k).get(); }
  double* D(const std::string& k) { return buf.at(k)->d(); }
};

namespace {

// clock64 budgets of the device-side pipeline waits (the drains that retire a CTA's
// own copies and MMAs have a floor of their own in the GEMM kernels)
constexpr long long kDefaultWatchdog = 4000000000LL, kMinWatchdog = 64;

int fail(rccsdt_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

DBuf* alloc_buf(rccsdt_ctx* c, const std::string& name, size_t bytes, int* err) {
  auto b = std::make_unique<DBuf>();
  b->p = dev_alloc(bytes, err);
  b->bytes = bytes;
  c->total_bytes += bytes;
  DBuf* raw = b.get();
  c->buf[name] = std::move(b);
  return raw;
}

std::unique_ptr<DBuf> upload(rccsdt_ctx* c, const void* host, size_t bytes, int* err) {
  auto b = std::make_unique<DBuf>();
  b->p = dev_alloc(bytes, err);
  b->bytes = bytes;
  c->total_bytes += bytes;
  if (b->p && bytes) {
#ifdef RCC_HOSTSIM
    memcpy(b->p, host, bytes);
#else
    if (cudaMemcpy(b->p, host, bytes, cudaMemcpyHostToDevice) != cudaSuccess) *err = RCCSDT_ERR_CUDA;
#endif
  }
  return b;
}

template <typename T>
std::unique_ptr<DBuf> upload_vec(rccsdt_ctx* c, const std::vector<T>& v, int* err) {
  return upload(c, v.data(), v.size() * sizeof(T), err);
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Fill a PackPlan from host tables; `shared_rowoff` (device) replaces rowoff if given.
void make_pack(rccsdt_ctx* c, PackPlan& P, const void* src, int src_f32, int R, int K, int nterm,
               const std::vector<double>& coef, const std::vector<i64>& colbase,
               const std::vector<int>& sel, const std::vector<i64>& rowoff, int read_k_fast, int* err,
               const i64* shared_rowoff = nullptr, int row_mode = 0) {
  P.coef = upload_vec(c, coef, err);
  P.colbase = upload_vec(c, colbase, err);
  P.sel = upload_vec(c, sel, err);
  if (!shared_rowoff) P.rowoff = upload_vec(c, rowoff, err);
  rcc::PackArgs& a = P.a;
  a.src = src;
  a.src_f32 = src_f32;
  a.R = R;
  a.K = K;
  a.nterm = nterm;
  a.coef = (const double*)P.coef->p;
  a.colbase = (const i64*)P.colbase->p;
  a.sel = (const int*)P.sel->p;
  a.rowoff = shared_rowoff ? shared_rowoff : (const i64*)P.rowoff->p;
  a.read_k_fast = read_k_fast;
  a.one_sel = 1;
  for (int x : sel)
    if (x != 0) a.one_sel = 0;
  // the shared selector tables are the computed forms (rows = 2 or 3 virtual labels)
  a.row_mode = row_mode;
  a.lv = c->v;
}

void make_epi(rccsdt_ctx* c, EpiPlan& E, void* C, int c_f32, int M, int N,
              const std::vector<i64>& row_base, const std::vector<int>& row_sel,
              const std::vector<double>& row_alpha, const std::vector<i64>& col_off, int* err,
              const i64* shared_col_off = nullptr) {
  E.row_base = upload_vec(c, row_base, err);
  E.row_sel = upload_vec(c, row_sel, err);
  E.row_alpha = upload_vec(c, row_alpha, err);
  if (!shared_col_off) E.col_off = upload_vec(c, col_off, err);
  rcc::EpiArgs& e = E.e;
  e.C = C;
  e.c_f32 = c_f32;
  e.M = M;
  e.N = N;
  e.row_base = (const i64*)E.row_base->p;
  e.row_sel = (const int*)E.row_sel->p;
  e.row_alpha = (const double*)E.row_alpha->p;
  e.col_off = shared_col_off ? shared_col_off : (const i64*)E.col_off->p;
}

// Block-row tables of the two-phase scatter; xaxes[r] = stored axis of each X axis.
void set_two_phase(rccsdt_ctx* c, GemmPlan* g, const std::vector<i64>& base, const std::vector<std::array<int, 3>>& xaxes,
                   const std::vector<double>& alpha, int* err);

void finish_plan(rccsdt_ctx* c, GemmPlan* g, int K) {
  g->K = K;
  g->Kpad = round_up(K, 64);
  g->A.a.Kpad = g->Kpad;
  g->B.a.Kpad = g->Kpad;
  g->fma = (double)g->E.e.M * g->E.e.N * K;
  size_t need = (size_t)std::max(g->A.a.R, g->B.a.R) * g->Kpad * 8;
  if (need > c->panel_bytes) c->panel_bytes = need;
  c->panel_rows = std::max(c->panel_rows, std::max(g->A.a.R, g->B.a.R));
}

// Bytes of one pp-ladder launch unit's T panel (FP64-sized, v rows of v^2 per stored
// block): options.pp_unit_bytes, 2 GiB when not positive.  The stored blocks are cut
// into ranges of that size, one GEMM per view and range.
i64 pp_unit_bytes(const rccsdt_ctx* c) { return c->opt.pp_unit_bytes > 0 ? c->opt.pp_unit_bytes : (2LL << 30); }

// Tables of the pair-symmetric pp-ladder (see PpSym): tile-major pair numbering,
// W panel rows, per-view epilogue rows (each x <= y writes (x, y) and, mirrored,
// (y, x)), and units of the same block ranges as the plain plans.
void build_pp_sym(rccsdt_ctx* c, bool t3f, void* r3p, int* err) {
  auto& S = c->pps;
  const int v = c->v;
  const i64 V2 = (i64)v * v, V3 = c->V3;
  const int nt = (v + 15) / 16;
  // K numbering: chunk (P, Q) of the 16-label tiles holds its sum pairs at offp and
  // its difference pairs at offm (inside a chunk as pair_decode describes)
  std::vector<rcc::PairChunk> ch;
  int offp = 0, offm = 0;
  for (int P = 0; P < nt; ++P)
    for (int Q = P; Q < nt; ++Q) {
      const int nd = std::min(16, v - 16 * P), ne = std::min(16, v - 16 * Q);
      const bool diag = P == Q;
      ch.push_back({P, Q, offp, offm});
      offp += diag ? nd * (nd + 1) / 2 : nd * ne;
      offm += diag ? nd * (nd - 1) / 2 : nd * ne;
    }
  S.nchunk = (int)ch.size();
  S.Kp = offp;
  S.Km = offm;
  S.Kpadp = round_up(S.Kp, 64);
  S.Kpadm = round_up(S.Km, 64);
  // GEMM row orders (independent of the K numbering): full 4 x 8 blocks of (x, y)
  // first, y fastest, so that the 32 rows of an epilogue warp write 8-element runs
  // along y for (x, y) and 4-element runs along x for the mirrored (y, x); then the
  // pairs of the partial blocks
  auto row_order = [&](bool plus) {
    std::vector<std::array<int, 2>> full, rest;
    for (int x0 = 0; x0 < v; x0 += 4)
      for (int y0 = 0; y0 < v; y0 += 8) {
        const bool whole = x0 + 4 <= v && y0 + 8 <= v && (plus ? x0 + 3 <= y0 : x0 + 3 < y0);
        for (int x = x0; x < std::min(x0 + 4, v); ++x)
          for (int y = y0; y < std::min(y0 + 8, v); ++y)
            if (plus ? x <= y : x < y) (whole ? full : rest).push_back({x, y});
      }
    full.insert(full.end(), rest.begin(), rest.end());
    return full;
  };
  const std::vector<std::array<int, 2>> rp = row_order(true), rm = row_order(false);
  std::vector<int> mrow((size_t)V2, -1);
  for (size_t q = 0; q < rm.size(); ++q) mrow[(size_t)rm[q][0] * v + rm[q][1]] = (int)q;
  std::vector<int4> rows(rp.size());
  for (size_t q = 0; q < rp.size(); ++q) rows[q] = make_int4(rp[q][0], rp[q][1], mrow[(size_t)rp[q][0] * v + rp[q][1]], 0);
  S.chunks = upload_vec(c, ch, err);
  S.rows = upload_vec(c, rows, err);
  // R3 offset of the result element (x, y, w) of view `term` is ebase(x, y) + col(blk, w)
  auto ebase = [&](int term, i64 x, i64 y) { return term == 0 ? x * V2 + y * v : term == 1 ? x * V2 + y : x * v + y; };
  // units: each view of nb stored blocks (N = nb v panel rows)
  const i64 per_blk = (i64)v * round_up((int)V2, 64) * 8;
  const i64 nb = std::max<i64>(1, std::min<i64>(c->n3, pp_unit_bytes(c) / per_blk));
  const int maxN0 = (int)(std::min<i64>(c->n3, nb) * v);
  for (int part = 0; part < 2; ++part) {
    const auto& pr = part == 0 ? rp : rm;
    const size_t M = pr.size();
    for (int term = 0; term < 3; ++term) {
      std::vector<i64> rb(M), rb2(M);
      for (size_t q = 0; q < M; ++q) {
        rb[q] = ebase(term, pr[q][0], pr[q][1]);
        rb2[q] = pr[q][0] == pr[q][1] ? -1 : ebase(term, pr[q][1], pr[q][0]);
      }
      S.rb[term][part] = upload_vec(c, rb, err);
      S.rb2[term][part] = upload_vec(c, rb2, err);
    }
    const size_t R = std::max<size_t>(std::max<size_t>(M, (size_t)maxN0), 1);  // rows of either orientation
    S.al[part] = upload_vec(c, std::vector<double>(R, 0.5), err);
    S.al2[part] = upload_vec(c, std::vector<double>(R, part == 0 ? 0.5 : -0.5), err);
  }
  S.sel = upload_vec(c, std::vector<int>(std::max(std::max(S.Kp, maxN0), 1), 0), err);
  int maxN = 0;
  for (int term = 0; term < 3; ++term)
    for (i64 b0 = 0; b0 < c->n3; b0 += nb) {
      auto u = std::make_unique<rccsdt_ctx::PpSym::Unit>();
      u->term = term;
      u->b0 = b0;
      u->nblk = (int)(std::min(c->n3, b0 + nb) - b0);
      u->N = u->nblk * v;
      maxN = std::max(maxN, u->N);
      std::vector<i64> col(u->N);
      for (int q = 0; q < u->N; ++q) {
        const i64 blk = b0 + q / v, w = q % v;
        col[q] = blk * V3 + (term == 0 ? w : term == 1 ? w * v : w * V2);
      }
      u->col = upload_vec(c, col, err);
      // the view with w on the unit-stride axis runs with the operands exchanged
      // (rows (blk, w), columns the pairs): an epilogue warp's rows are consecutive w,
      // so both the (x, y) and the mirrored (y, x) writes are coalesced
      u->swap = term == 0;
      for (int part = 0; part < 2; ++part) {
        rcc::EpiArgs& e = u->e[part];
        const int P = part == 0 ? S.Kp : S.Km;
        e.C = r3p;
        e.c_f32 = t3f ? 1 : 0;
        e.row_sel = (const int*)S.sel->p;
        e.row_alpha = (const double*)S.al[part]->p;
        e.row_alpha2 = (const double*)S.al2[part]->p;
        if (u->swap) {
          e.M = u->N;
          e.N = P;
          e.row_base = (const i64*)u->col->p;
          e.col_off = (const i64*)S.rb[term][part]->p;
          e.col_off2 = (const i64*)S.rb2[term][part]->p;
        } else {
          e.M = P;
          e.N = u->N;
          e.row_base = (const i64*)S.rb[term][part]->p;
          e.col_off = (const i64*)u->col->p;
          e.row_base2 = (const i64*)S.rb2[term][part]->p;
        }
        u->fma[part] = (double)P * u->N * P;
      }
      S.units.push_back(std::move(u));
    }
  // engine panels: both A parts side by side, both B parts side by side
  const size_t needA = ((size_t)S.Kp * S.Kpadp + (size_t)S.Km * S.Kpadm) * 8;
  const size_t needB = (size_t)maxN * (S.Kpadp + S.Kpadm) * 8;
  c->panel_bytes = std::max(c->panel_bytes, std::max(needA, needB));
  c->panel_rows = std::max(c->panel_rows, std::max(S.Kp + S.Km, 2 * maxN));
  S.on = 1;
}

// The allocation holding p (start pointer and element offset of p in it).
static bool locate(rccsdt_ctx* c, const void* p, size_t esz, void** start, i64* off) {
  for (auto& kv : c->buf) {
    const char* b = (const char*)kv.second->p;
    if (b && (const char*)p >= b && (const char*)p < b + kv.second->bytes) {
      *start = kv.second->p;
      *off = (i64)(((const char*)p - b) / esz);
      return ((const char*)p - b) % esz == 0;
    }
  }
  return false;
}

// One GEMM for plans that share their B operand (same N, K and K order; the first
// part's B is taken over): their A operands are stacked into one panel, so the B
// panel is streamed once for all of them.  The parts' outputs may lie in at most
// two allocations of one element type, the parts writing the first one coming
// first, and the address ranges of parts in one allocation must not overlap
// (rows of one GEMM update their elements concurrently, without atomics).
// Returns null (parts unchanged) when the parts do not fit this form.
GemmPlan* stack_rows(rccsdt_ctx* c, const std::vector<GemmPlan*>& parts, int* err) {
  if (parts.size() < 2) return nullptr;
  const GemmPlan* p0 = parts[0];
  const size_t esz = p0->E.e.c_f32 ? 4 : 8;
  void* bufs[2] = {nullptr, nullptr};
  int m2 = -1, M = 0, nsel_total = 0;
  const int N = p0->E.e.N;
  std::vector<i64> rb, co;
  std::vector<int> rs;
  std::vector<double> ra;
  std::vector<std::array<i64, 3>> span;  // per part: slot, first and last element written
  for (const GemmPlan* q : parts) {
    const rcc::EpiArgs& e = q->E.e;
    if (e.N != N || q->K != p0->K || e.c_f32 != p0->E.e.c_f32 || q->s3_rows || q->tc_swap || e.C2) return nullptr;
    void* start = nullptr;
    i64 off = 0;
    if (!locate(c, e.C, esz, &start, &off)) return nullptr;
    int slot = start == bufs[0] ? 0 : (start == bufs[1] ? 1 : -1);
    if (slot < 0) {
      if (!bufs[0]) slot = 0;
      else if (!bufs[1]) slot = 1;
      else return nullptr;
      bufs[slot] = start;
      if (slot == 1) m2 = M;
    }
    if (slot == 0 && m2 >= 0) return nullptr;  // rows of the first output must come first
    std::vector<i64> hb(e.M);
    std::vector<int> hs(e.M);
    std::vector<double> ha(e.M);
    if (dev_copy(hb.data(), e.row_base, hb.size() * 8, c->stream) ||
        dev_copy(hs.data(), e.row_sel, hs.size() * 4, c->stream) ||
        dev_copy(ha.data(), e.row_alpha, ha.size() * 8, c->stream) || dev_sync(c->stream)) {
      *err = RCCSDT_ERR_CUDA;
      return nullptr;
    }
    int nsel = 0;
    for (int x : hs) nsel = std::max(nsel, x + 1);
    std::vector<i64> hc((size_t)nsel * N);
    if (dev_copy(hc.data(), e.col_off, hc.size() * 8, c->stream) || dev_sync(c->stream)) {
      *err = RCCSDT_ERR_CUDA;
      return nullptr;
    }
    i64 lo = std::numeric_limits<i64>::max(), hi = std::numeric_limits<i64>::min();
    for (int m = 0; m < e.M; ++m) {
      rb.push_back(hb[m] + off);
      rs.push_back(hs[m] + nsel_total);
      ra.push_back(ha[m]);
      for (int n = 0; n < N; ++n) {
        const i64 a = hb[m] + off + hc[(size_t)hs[m] * N + n];
        lo = std::min(lo, a);
        hi = std::max(hi, a);
      }
    }
    for (const auto& sp : span)
      if (sp[0] == slot && lo <= sp[2] && sp[1] <= hi) return nullptr;
    span.push_back({(i64)slot, lo, hi});
    co.insert(co.end(), hc.begin(), hc.end());
    nsel_total += nsel;
    M += e.M;
  }
  c->plans.push_back(std::make_unique<GemmPlan>());
  GemmPlan* g = c->plans.back().get();
  GemmPlan* b0 = parts[0];
  g->B = std::move(b0->B);
  g->h_cube = std::move(b0->h_cube);
  g->cube = std::move(b0->cube);
  g->cube_mode = b0->cube_mode;
  g->cube_src = b0->cube_src;
  g->r1_wbase = std::move(b0->r1_wbase);
  make_epi(c, g->E, bufs[0], p0->E.e.c_f32, M, N, rb, rs, ra, co, err);
  g->E.e.C2 = bufs[1];
  g->E.e.m2 = m2 >= 0 ? m2 : M;
  g->a_parts = parts;
  g->reuse_B = b0->reuse_B;  // the first part's B may be the panel of the plan before
  g->A.a.R = M;
  g->step = p0->step;
  g->big = 1;
  finish_plan(c, g, p0->K);
  return g;
}

// Multi-index enumeration: offsets sum_d idx_d * stride_d over dims in order.
std::vector<i64> offsets(const std::vector<i64>& size, const std::vector<i64>& stride) {
  i64 total = 1;
  for (i64 s : size) total *= s;
  std::vector<i64> out((size_t)total);
  std::vector<i64> idx(size.size(), 0);
  for (i64 t = 0; t < total; ++t) {
    i64 off = 0;
    for (size_t d = 0; d < size.size(); ++d) off += idx[d] * stride[d];
    out[(size_t)t] = off;
    for (int d = (int)size.size() - 1; d >= 0; --d) {
      if (++idx[d] < size[d]) break;
      idx[d] = 0;
    }
  }
  return out;
}

// C += alpha * contract(A, B) by an einsum-like spec "ab,bc->ac" (no batch labels).
GemmPlan* contraction(rccsdt_ctx* c, const char* spec, double alpha, const View& A, const View& Bv,
                      const View& C, int* err, int big = 0) {
  std::string s(spec);
  size_t comma = s.find(','), arrow = s.find("->");
  std::string la = s.substr(0, comma), lb = s.substr(comma + 1, arrow - comma - 1), lc = s.substr(arrow + 2);
  if (la.size() != A.shape.size() || lb.size() != Bv.shape.size() || lc.size() != C.shape.size()) {
    *err = RCCSDT_ERR_ARG;
    c->err = std::string("internal: rank mismatch in ") + spec;
    return nullptr;
  }
  auto find = [](const std::string& l, char ch) { return (int)l.find(ch); };
  std::vector<i64> mA, mC, mS, nB, nC, nS, kA, kB, kS;
  for (size_t q = 0; q < lc.size(); ++q) {
    char ch = lc[q];
    int ia = find(la, ch), ib = find(lb, ch);
    if (ia >= 0 && ib >= 0) {
      *err = RCCSDT_ERR_ARG;
      c->err = std::string("internal: batch label in ") + spec;
      return nullptr;
    }
    if (ia >= 0) {
      mA.push_back(A.stride[ia]); mC.push_back(C.stride[q]); mS.push_back(C.shape[q]);
    } else {
      nB.push_back(Bv.stride[ib]); nC.push_back(C.stride[q]); nS.push_back(C.shape[q]);
    }
  }
  for (size_t q = 0; q < la.size(); ++q) {
    char ch = la[q];
    if (find(lc, ch) >= 0) continue;
    int ib = find(lb, ch);
    if (ib < 0) {
      *err = RCCSDT_ERR_ARG;
      c->err = std::string("internal: free label in ") + spec;
      return nullptr;
    }
    kA.push_back(A.stride[q]); kB.push_back(Bv.stride[ib]); kS.push_back(A.shape[q]);
  }
  std::vector<i64> rowA = offsets(mS, mA), rowC = offsets(mS, mC);
  std::vector<i64> rowB = offsets(nS, nB), colC = offsets(nS, nC);
  std::vector<i64> kAo = offsets(kS, kA), kBo = offsets(kS, kB);
  const int M = (int)rowA.size(), N = (int)rowB.size(), K = (int)kAo.size();
  auto g = std::make_unique<GemmPlan>();
  std::vector<double> coefK(K, 1.0);
  std::vector<int> selK(K, 0);
  auto unit_fast = [](const std::vector<i64>& st) { return !st.empty() && st.back() == 1; };
  make_pack(c, g->A, A.p, A.f32, M, K, 1, coefK, kAo, selK, rowA, unit_fast(kA) ? 1 : 0, err);
  make_pack(c, g->B, Bv.p, Bv.f32, N, K, 1, coefK, kBo, selK, rowB, unit_fast(kB) ? 1 : 0, err);
  make_epi(c, g->E, C.p, C.f32, M, N, rowC, std::vector<int>(M, 0), std::vector<double>(M, alpha), colC, err);
  finish_plan(c, g.get(), K);
  // in the split modes every contraction of 1e7 FMA or more runs on the tensor cores
  g->big = big || g->fma >= 1e7;
  GemmPlan* raw = g.get();
  c->plans.push_back(std::move(g));
  return raw;
}

// Permuted linear combination out = beta*out + sum coef_t in_t; views share a shape.
rcc::CombineArgs combine(const View& out, double beta, std::vector<std::pair<double, View>> terms) {
  rcc::CombineArgs a{};
  a.out = (double*)out.p;
  a.rank = (int)out.shape.size();
  a.total = 1;
  for (int d = 0; d < a.rank; ++d) {
    a.shape[d] = out.shape[d];
    a.ostride[d] = out.stride[d];
    a.total *= out.shape[d];
  }
  a.nterm = (int)terms.size();
  for (int t = 0; t < a.nterm; ++t) {
    a.coef[t] = terms[t].first;
    a.in[t] = (const double*)terms[t].second.p;
    for (int d = 0; d < a.rank; ++d) a.istride[t][d] = terms[t].second.stride[d];
  }
  a.beta = beta;
  return a;
}

// A view with explicit shape and strides (for diagonal and permuted access).
View strided(void* p, std::vector<i64> shape, std::vector<i64> stride) {
  View v;
  v.p = p;
  v.shape = shape;
  v.stride = stride;
  return v;
}

// Permuted view: out axis d reads input axis perm[d].
View permuted(const View& in, std::vector<int> perm) {
  View v = in;
  for (size_t d = 0; d < perm.size(); ++d) {
    v.shape[d] = in.shape[perm[d]];
    v.stride[d] = in.stride[perm[d]];
  }
  return v;
}

}  // namespace

// ---------------------------------------------------------------------------
// Interval timing with pooled CUDA events (recorded, never waited on until the
// totals are read), so timing does not serialise the iteration.
// ---------------------------------------------------------------------------
static int timer_begin(rccsdt_ctx* c, int tag, double flop = 0.0) {
#ifdef RCC_HOSTSIM
  (void)c; (void)tag; (void)flop;
  return -1;
#else
  if (!c->timing) return -1;
  if (c->ev_used + 2 > (int)c->ev.size()) {
    // grow the pool (fresh events, nothing pending on them)
    const int add = 1024;
    for (int q = 0; q < add; ++q) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      c->ev.push_back(e);
    }
    c->ev_tag.resize(c->ev.size() / 2);
    c->ev_flop.resize(c->ev.size() / 2);
  }
  const int idx = c->ev_used / 2;
  c->ev_tag[idx] = tag;
  c->ev_flop[idx] = flop;
  cudaEventRecord(c->ev[c->ev_used], c->stream);
  c->ev_used += 2;
  return idx;
#endif
}

static void timer_end(rccsdt_ctx* c, int idx) {
#ifndef RCC_HOSTSIM
  if (idx >= 0) cudaEventRecord(c->ev[2 * idx + 1], c->stream);
#else
  (void)c; (void)idx;
#endif
}

// Sums the recorded intervals: ms per tag into out_ms[17], GEMM launches and flop.
static void timer_collect(rccsdt_ctx* c, double* out_ms, double* gemm_launches, double* gemm_flop) {
  for (int q = 0; q < 17; ++q) out_ms[q] = 0.0;
  *gemm_launches = 0.0;
  *gemm_flop = 0.0;
#ifndef RCC_HOSTSIM
  if (c->ev_used == 0) return;
  cudaEventSynchronize(c->ev[c->ev_used - 1]);
  for (int idx = 0; idx < c->ev_used / 2; ++idx) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev[2 * idx], c->ev[2 * idx + 1]);
    out_ms[c->ev_tag[idx]] += ms;
    if (c->ev_tag[idx] == 16) {
      *gemm_launches += 1.0;
      *gemm_flop += c->ev_flop[idx];
    }
  }
#endif
}

// ---------------------------------------------------------------------------
// Engine: run one GemmPlan
// ---------------------------------------------------------------------------
static int run_gemm(rccsdt_ctx* c, GemmPlan* g) {
  // in the split modes every contraction runs as a split product on the tensor
  // cores (FP64 throughput on this part is 2 FMA per clock per SM), except the
  // bare integrals that define the energy
  const bool tc = c->precision != RCCSDT_FP64 && !g->f64_only;
  const int kind = !tc ? rcc::PANEL_F64 : (c->precision == RCCSDT_SPLIT_BF16X3 ? rcc::PANEL_BF16X2 : rcc::PANEL_TF32X2);
  rcc::PackArgs pa = g->A.a, pb = g->B.a;
  pa.kind = pb.kind = kind;
  const bool own = tc && g->own;  // the plan's own A panel (split modes)
  pa.out_hi = own ? g->own->hi.p : c->panelA_hi->p;
  pa.out_lo = own ? g->own->lo.p : (c->panelA_lo ? c->panelA_lo->p : nullptr);
  pb.out_hi = c->panelB_hi->p;
  pb.out_lo = c->panelB_lo ? c->panelB_lo->p : nullptr;
  // FP64 contractions on the tensor cores (option f64_tc): the large ones only
  const bool f64e = !tc && c->opt.f64_tc && c->planesA && (c->opt.f64_tc == 2 || g->fma >= 3e7) && !g->f64_only;
  const bool packA = own ? (g->own_pack || g->own->kind != kind)
                         : (!g->a_parts.empty() || !g->reuse_A || c->packedA_kind != kind);
  const bool packB = !g->reuse_B || c->packedB_kind != kind;
  if (!packA) {
  } else if (!g->a_parts.empty()) {
    const size_t esz = kind == rcc::PANEL_F64 ? 8 : (kind == rcc::PANEL_BF16X2 ? 2 : 4);
    size_t r0 = 0;
    for (GemmPlan* q : g->a_parts) {
      rcc::PackArgs pq = q->A.a;
      pq.kind = kind;
      pq.out_hi = (char*)pa.out_hi + r0 * g->Kpad * esz;
      pq.out_lo = pa.out_lo ? (void*)((char*)pa.out_lo + r0 * g->Kpad * esz) : nullptr;
      rcc::launch_pack(pq, c->stream);
      r0 += (size_t)pq.R;
    }
  } else {
    rcc::launch_pack(pa, c->stream);
  }
  if (own) {
    if (packA) g->own->kind = kind;
  } else if (packA) {
    c->slicedA = 0;
  }
  if (packB) c->slicedB = 0;
  if (packB) {
    if (tc && g->cube) {
      const rcc::CubeDst d0{pb.out_hi, pb.out_lo, g->Kpad};
      const float* src = g->cube_src ? g->cube_src : (const float*)pb.src;
      if (g->r1_wbase)
        rcc::launch_cube_pack_r1(kind, (const rcc::CubePiece*)g->cube->p, (int)g->h_cube.size(), d0, src, c->v,
                                 c->B("oovv_f")->f(), (const i64*)g->r1_wbase->p, c->B("r1_part")->f(), c->stream);
      else
        rcc::launch_cube_pack(g->cube_mode, kind, (const rcc::CubePiece*)g->cube->p, (int)g->h_cube.size(),
                              nullptr, d0, src, c->v, c->stream);
      if (g->cube_mode == 0) rcc::launch_zero_cols(d0, pb.R, g->K, kind, c->stream);
    } else {
      rcc::launch_pack(pb, c->stream);
    }
  }
  c->packedA_kind = c->packedB_kind = kind;
  const int tidx = g->step == 1 ? timer_begin(c, 16, 2.0 * g->fma) : -1;
  if (f64e) {
    if (c->slicedA != g->Kpad)
      rcc::launch_slice_f64((const double*)pa.out_hi, g->E.e.M, g->Kpad, c->planesA->p, (int*)c->expA->p, c->stream);
    if (c->slicedB != g->Kpad)
      rcc::launch_slice_f64((const double*)pb.out_hi, g->E.e.N, g->Kpad, c->planesB->p, (int*)c->expB->p, c->stream);
    c->slicedA = c->slicedB = g->Kpad;
    int* flag = (int*)((double*)c->scalars->p + 1000);
    if (rcc::launch_gemm_f64e(c->planesA->p, (const int*)c->expA->p, c->planesB->p, (const int*)c->expB->p, g->Kpad,
                              g->E.e, flag, c->opt.watchdog_cycles, c->stream))
      return fail(c, RCCSDT_ERR_ARG, "tensor-core FP64 GEMM configuration unsupported");
  } else if (!tc) {
    rcc::launch_gemm_f64((const double*)pa.out_hi, (const double*)pb.out_hi, round_up(g->K, 16), g->Kpad, g->Kpad,
                         g->E.e, c->concurrent ? nullptr : c->splitk->d(), (i64)(c->splitk->bytes / 8), c->stream);
  } else {
    int* flag = (int*)((double*)c->scalars->p + 1000);
    float* raw = g->s3_rows > 0 && c->rawX ? (float*)c->rawX->p : nullptr;
    // tile width from the output columns: 128, 144 (e.g. the 136 pairs i <= j of o = 16) or 256
    auto width = [](int n) { return n <= 128 ? 128 : (n <= 144 ? 144 : 256); };
    int lst;
    if (raw && g->tc_swap) {
      rcc::EpiArgs et = g->E.e;
      std::swap(et.M, et.N);
      lst = rcc::launch_gemm_tc(kind, pb.out_hi, pb.out_lo, pa.out_hi, pa.out_lo, g->Kpad, et, flag,
                                c->opt.watchdog_cycles, c->stream, nullptr, 0, raw, width(et.N), 1);
    } else {
      lst = rcc::launch_gemm_tc(kind, pa.out_hi, pa.out_lo, pb.out_hi, pb.out_lo, g->Kpad, g->E.e, flag,
                                c->opt.watchdog_cycles, c->stream, c->concurrent ? nullptr : (float*)c->splitk->p,
                                (long long)(c->splitk->bytes / 4), raw, width(g->E.e.N));
    }
    if (lst) return fail(c, RCCSDT_ERR_ARG, "tensor-core GEMM configuration unsupported");
    if (raw) {
      const rcc::EpiArgs& e = g->E.e;
      const i64* sb = (const i64*)g->s3_base->p;
      const int* ss = (const int*)g->s3_sel->p;
      const double* sa = (const double*)g->s3_alpha->p;
      if (e.c_f32)
        rcc::launch_scatter_rows3<float>(raw, g->s3_rows, c->v, sb, ss, sa, (float*)e.C, c->stream);
      else
        rcc::launch_scatter_rows3<double>(raw, g->s3_rows, c->v, sb, ss, sa, (double*)e.C, c->stream);
    }
  }
  timer_end(c, tidx);
#ifndef RCC_HOSTSIM
  const cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return fail(c, RCCSDT_ERR_CUDA, std::string("GEMM launch: ") + cudaGetErrorString(ce));
#endif
  return 0;
}

static int run_plans(rccsdt_ctx* c, const std::vector<GemmPlan*>& ps) {
  for (GemmPlan* g : ps) {
    int st = run_gemm(c, g);
    if (st) return st;
  }
  return 0;
}

// pp-ladder on pair-symmetric operands: the two W panels once, then per unit the
// two T panels of its view and the sum and difference GEMMs (tensor cores in the
// split modes; FP64 on the tensor cores or the FP64 units otherwise).
static int run_pp_sym(rccsdt_ctx* c) {
  auto& S = c->pps;
  const int v = c->v;
  const i64 V2 = (i64)v * v;
  const bool tc = c->precision != RCCSDT_FP64;
  const int kind = !tc ? rcc::PANEL_F64 : (c->precision == RCCSDT_SPLIT_BF16X3 ? rcc::PANEL_BF16X2 : rcc::PANEL_TF32X2);
  const size_t esz = kind == rcc::PANEL_F64 ? 8 : (kind == rcc::PANEL_BF16X2 ? 2 : 4);
  const bool f64e = !tc && c->opt.f64_tc && c->planesA && !S.units.empty() &&
                    (c->opt.f64_tc == 2 || S.units[0]->fma[0] >= 3e7);
  char* ahi = (char*)c->panelA_hi->p;
  char* alo = c->panelA_lo ? (char*)c->panelA_lo->p : nullptr;
  char* bhi = (char*)c->panelB_hi->p;
  char* blo = c->panelB_lo ? (char*)c->panelB_lo->p : nullptr;
  const size_t aoff = (size_t)S.Kp * S.Kpadp * esz;
  const rcc::CubeDst Ap{ahi, alo, S.Kpadp}, Am{ahi + aoff, alo ? alo + aoff : nullptr, S.Kpadm};
  const auto* ch = (const rcc::PairChunk*)S.chunks->p;
  // the shared panels hold other operands afterwards
  c->packedA_kind = c->packedB_kind = -1;
  c->slicedA = c->slicedB = 0;
  rcc::launch_pair_pack_w(kind, c->D("Wvvvv"), v, (const int4*)S.rows->p, S.Kp, ch, S.nchunk, S.Kp, S.Km, Ap, Am,
                          c->stream);
  char* pA[2] = {nullptr, nullptr};
  int* eA[2] = {nullptr, nullptr};
  if (f64e) {
    pA[0] = (char*)c->planesA->p;
    pA[1] = pA[0] + (size_t)rcc::kSlices * S.Kp * S.Kpadp * 2;
    eA[0] = (int*)c->expA->p;
    eA[1] = eA[0] + S.Kp;
    rcc::launch_slice_f64((const double*)Ap.out_hi, S.Kp, S.Kpadp, pA[0], eA[0], c->stream);
    if (S.Km) rcc::launch_slice_f64((const double*)Am.out_hi, S.Km, S.Kpadm, pA[1], eA[1], c->stream);
  }
  int* flag = (int*)((double*)c->scalars->p + 1000);
  const i64 sd[3] = {V2, V2, v}, se[3] = {v, 1, 1}, sw[3] = {1, v, V2};
  const bool t3f = c->opt.precision != RCCSDT_FP64;
  for (auto& up : S.units) {
    auto& u = *up;
    const size_t boff = (size_t)u.N * S.Kpadp * esz;
    const rcc::CubeDst Bp{bhi, blo, S.Kpadp}, Bm{bhi + boff, blo ? blo + boff : nullptr, S.Kpadm};
    rcc::launch_pair_pack_t(kind, c->B("t3")->p, t3f ? 1 : 0, u.b0, u.nblk, v, sd[u.term], se[u.term], sw[u.term], ch,
                            S.nchunk, S.Kp, S.Km, Bp, Bm, c->stream);
    for (int part = 0; part < 2; ++part) {
      const int K = part ? S.Km : S.Kp, Kpad = part ? S.Kpadm : S.Kpadp;
      if (K == 0) continue;
      const rcc::CubeDst& A = part ? Am : Ap;
      const rcc::CubeDst& Bq = part ? Bm : Bp;
      const rcc::EpiArgs& e = u.e[part];
      const int tidx = timer_begin(c, 16, 2.0 * u.fma[part]);
      int lst = 0;
      // operands in GEMM order: rows of e.M first (the T panel when the unit is exchanged)
      const rcc::CubeDst& X = u.swap ? Bq : A;
      const rcc::CubeDst& Y = u.swap ? A : Bq;
      if (f64e) {
        rcc::launch_slice_f64((const double*)Bq.out_hi, u.N, Kpad, c->planesB->p, (int*)c->expB->p, c->stream);
        const void* px = u.swap ? c->planesB->p : (const void*)pA[part];
        const void* py = u.swap ? (const void*)pA[part] : c->planesB->p;
        const int* ex = u.swap ? (const int*)c->expB->p : eA[part];
        const int* ey = u.swap ? eA[part] : (const int*)c->expB->p;
        lst = rcc::launch_gemm_f64e(px, ex, py, ey, Kpad, e, flag, c->opt.watchdog_cycles, c->stream);
      } else if (!tc) {
        rcc::launch_gemm_f64((const double*)X.out_hi, (const double*)Y.out_hi, round_up(K, 16), Kpad, Kpad, e,
                             c->concurrent ? nullptr : c->splitk->d(), (i64)(c->splitk->bytes / 8), c->stream);
      } else {
        // (the column-mirror epilogue exists for 256-wide tiles only)
        const int bn = u.swap ? 256 : (e.N <= 128 ? 128 : (e.N <= 144 ? 144 : 256));
        lst = rcc::launch_gemm_tc(kind, X.out_hi, X.out_lo, Y.out_hi, Y.out_lo, Kpad, e, flag, c->opt.watchdog_cycles,
                                  c->stream, c->concurrent ? nullptr : (float*)c->splitk->p,
                                  (long long)(c->splitk->bytes / 4), nullptr, bn);
      }
      timer_end(c, tidx);
      if (lst) return fail(c, RCCSDT_ERR_ARG, "pair-symmetric pp-ladder GEMM configuration unsupported");
    }
  }
#ifndef RCC_HOSTSIM
  const cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return fail(c, RCCSDT_ERR_CUDA, std::string("pp-ladder: ") + cudaGetErrorString(ce));
#endif
  return 0;
}

static void run_combines(rccsdt_ctx* c, const std::vector<rcc::CombineArgs>& cs) {
  for (const auto& a : cs) rcc::launch_combine(a, c->stream);
}

// ---------------------------------------------------------------------------
// Context construction: buffers and every plan of one iteration
// ---------------------------------------------------------------------------
namespace {

// Virtual-permutation index of pos (the 6 orderings in lexicographic order).
int perm_id(const int pos[3]) {
  static const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int q = 0; q < 6; ++q)
    if (P[q][0] == pos[0] && P[q][1] == pos[1] && P[q][2] == pos[2]) return q;
  return 0;
}

}  // namespace

namespace {
void set_two_phase(rccsdt_ctx* c, GemmPlan* g, const std::vector<i64>& base, const std::vector<std::array<int, 3>>& xaxes,
                   const std::vector<double>& alpha, int* err) {
  std::vector<int> sel(xaxes.size());
  for (size_t r = 0; r < xaxes.size(); ++r) sel[r] = perm_id(xaxes[r].data());
  g->h_base = base;
  g->h_sel = sel;
  g->h_alpha = alpha;
  g->s3_base = upload_vec(c, base, err);
  g->s3_sel = upload_vec(c, sel, err);
  g->s3_alpha = upload_vec(c, alpha, err);
  g->s3_rows = (int)base.size();
}

struct TripleInfo {
  i64 blk;
  int pos[3];
  int m;
};

int packpos(int a, int b, int c) { return a | (b << 2) | (c << 4); }

// A piece with rows row0 + L1 rs1 + L2 rs2 (mode 0: default rows L1 v + L2).
rcc::CubePiece cube_piece(int k0, int nterm, int v = 0) {
  rcc::CubePiece p;
  memset(&p, 0, sizeof(p));
  p.k0 = k0;
  p.nterm = nterm;
  p.rs1 = v;
  p.rs2 = 1;
  return p;
}

void set_cube(rccsdt_ctx* c, GemmPlan* g, int mode, std::vector<rcc::CubePiece> pieces, int* err) {
  g->cube_mode = mode;
  g->h_cube = std::move(pieces);
  g->cube = upload_vec(c, g->h_cube, err);
}
TripleInfo triple(int i, int j, int k) {
  TripleInfo t;
  int occ[3] = {i, j, k}, srt[3];
  sort_positions(occ, t.pos, srt);
  t.blk = rcc::blk_index(srt[0], srt[1], srt[2]);
  t.m = multiplicity(i, j, k);
  return t;
}

struct Builder {
  rccsdt_ctx* c;
  int* err;
  int o, v, n, naux;
  i64 V2, V3, S[3];
  const i64* RT2 = nullptr;  // [9][v^2]
  const i64* RT3 = nullptr;  // [6][v^3]

  View T(const std::string& name, std::vector<i64> shape) { return dense(c->D(name), shape); }
  DBuf* mk(const std::string& name, size_t count, size_t elem = 8) { return alloc_buf(c, name, count * elem, err); }
  GemmPlan* ct(std::vector<GemmPlan*>& grp, const char* spec, double alpha, const View& A, const View& B,
               const View& C, int big = 0) {
    GemmPlan* g = contraction(c, spec, alpha, A, B, C, err, big);
    if (g) grp.push_back(g);
    return g;
  }
  GemmPlan* new_plan() {
    c->plans.push_back(std::make_unique<GemmPlan>());
    return c->plans.back().get();
  }
};

int build_context(rccsdt_ctx* c) {
  int err = 0;
  Builder b{c, &err, c->o, c->v, c->n, c->naux};
  const int o = c->o, v = c->v, n = c->n, naux = c->naux;
  b.V2 = (i64)v * v;
  b.V3 = b.V2 * v;
  b.S[0] = b.V2; b.S[1] = v; b.S[2] = 1;
  const i64 V2 = b.V2, V3 = b.V3, n3 = c->n3;
  const int t3f = c->opt.precision != RCCSDT_FP64;
  const size_t t3e = t3f ? 4 : 8;

  // --- data buffers
  b.mk("e", n); b.mk("L", (size_t)naux * n * n); b.mk("Lt", (size_t)naux * n * n);
  b.mk("F", (size_t)n * n); b.mk("ft", (size_t)n * n); b.mk("J", (size_t)n * n); b.mk("Kx", (size_t)n * n);
  b.mk("gamma", naux); b.mk("Y", (size_t)naux * v * n);
  const char* blocks[] = {"oooo", "ooov", "oovo", "oovv", "ovov", "ovvo", "ovvv", "vovv", "vooo", "vvoo", "vvvo", "vvvv"};
  for (const char* s : blocks) {
    size_t cnt = 1;
    for (int q = 0; q < 4; ++q) cnt *= (s[q] == 'o' ? o : v);
    b.mk(s, cnt);
  }
  b.mk("ovov_bare", (size_t)o * v * o * v);
  b.mk("vs_oovv", (size_t)o * o * v * v); b.mk("ts2", (size_t)o * o * v * v);
  b.mk("vs_ovvv", (size_t)o * v * v * v); b.mk("vs_oovo", (size_t)o * o * v * o);
  b.mk("Fvv", V2); b.mk("Foo", (size_t)o * o); b.mk("Woooo", (size_t)o * o * o * o);
  b.mk("Wt_oooo", (size_t)o * o * o * o);
  b.mk("Wovvo", (size_t)o * v * v * o); b.mk("Wovov", (size_t)o * v * o * v);
  b.mk("Wvvvo", (size_t)v * v * v * o); b.mk("Wvooo", (size_t)v * o * o * o);
  b.mk("Wb_ovvo", (size_t)o * v * v * o); b.mk("Wb_ovov", (size_t)o * v * o * v);
  b.mk("Wvvvv", (size_t)V2 * V2);
  b.mk("Wring_ab", (size_t)o * v * 2 * o * v); b.mk("Wring_c", (size_t)o * v * o * v);
  b.mk("t1", (size_t)o * v); b.mk("t2", (size_t)o * o * v * v); b.mk("r1", (size_t)o * v);
  b.mk("r2", (size_t)o * o * v * v); b.mk("X2", (size_t)o * o * v * v);
  b.mk("dR1", (size_t)o * v); b.mk("dX2", (size_t)o * o * v * v);
  b.mk("t3", (size_t)n3 * V3, t3e); b.mk("r3", (size_t)n3 * V3, t3e); b.mk("rp3", (size_t)n3 * V3, t3e);
  // step (iii) unpacks the blocks t_{xyz} of a3_Z values of z at a time (options.unpack_bytes)
  const i64 ub = c->opt.unpack_bytes > 0 ? c->opt.unpack_bytes : (1LL << 30);
  c->a3_Z = (int)std::max<i64>(1, std::min<i64>(o, ub / std::max<i64>(1, (i64)o * o * V3 * (i64)t3e)));
  b.mk("Sz", (size_t)c->a3_Z * o * o * V3, t3e);
  if (t3f) {  // split bodies of step (iii): panels gathered from T3, R1 partials per cube
    const i64 nc = (v + 15) / 16;
    b.mk("oovv_f", (size_t)o * o * V2, 4);
    b.mk("r1_part", (size_t)c->a3_Z * o * o * nc * nc * nc * 32, 4);
  }
  if (err) return fail(c, err, "device allocation failed");

  // --- block info and weights
  {
    std::vector<int4> info((size_t)n3);
    std::vector<double> w((size_t)n3);
    for (int k = 0; k < o; ++k)
      for (int j = 0; j <= k; ++j)
        for (int i = 0; i <= j; ++i) {
          i64 bi = rcc::blk_index(i, j, k);
          info[bi] = make_int4(i, j, k, 0);
          w[bi] = multiplicity(i, j, k);
        }
    c->blocks_info = upload_vec(c, info, &err);
    c->blk_weight = upload_vec(c, w, &err);
    // per-CTA partial sums of |R3|^2 formed by the post-processing pass
    alloc_buf(c, "post_partial", (size_t)rcc::post_partials(v, n3) * 8, &err);
  }
  // --- selector tables
  std::unique_ptr<DBuf> rt2, rt3;
  {
    std::vector<i64> t2tab((size_t)9 * V2), t3tab((size_t)6 * V3);
    for (int al = 0; al < 3; ++al)
      for (int be = 0; be < 3; ++be)
        for (int x = 0; x < v; ++x)
          for (int y = 0; y < v; ++y) t2tab[(size_t)(al * 3 + be) * V2 + x * v + y] = x * b.S[al] + y * b.S[be];
    static const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int q = 0; q < 6; ++q)
      for (i64 e = 0; e < V3; ++e) {
        i64 a = e / V2, bb = (e / v) % v, cc = e % v;
        t3tab[(size_t)q * V3 + e] = a * b.S[P[q][0]] + bb * b.S[P[q][1]] + cc * b.S[P[q][2]];
      }
    rt2 = upload_vec(c, t2tab, &err);
    rt3 = upload_vec(c, t3tab, &err);
    b.RT2 = (const i64*)rt2->p;
    b.RT3 = (const i64*)rt3->p;
    c->buf["RT2"] = std::move(rt2);
    c->buf["RT3"] = std::move(rt3);
  }

  const i64 O0 = 0, V0 = o;
  View L = b.T("L", {naux, n, n}), Lt = b.T("Lt", {naux, n, n});
  View t1 = b.T("t1", {o, v}), t2 = b.T("t2", {o, o, v, v}), ts2 = b.T("ts2", {o, o, v, v});
  View ft = b.T("ft", {n, n}), F = b.T("F", {n, n});
  auto eri = [&](const char* s) {
    std::vector<i64> sh;
    for (int q = 0; q < 4; ++q) sh.push_back(s[q] == 'o' ? o : v);
    return b.T(s, sh);
  };

  // bare (ia|jb) for the energy and the MP2 guess
  b.ct(c->p_energy_bare, "Pia,Pjb->iajb", 1.0, sub(sub(L, 1, O0, o), 2, V0, v), sub(sub(L, 1, O0, o), 2, V0, v),
       b.T("ovov_bare", {o, v, o, v}));
  for (GemmPlan* g : c->p_energy_bare) g->f64_only = 1;

  // --- (i) T1 dressing: Lt = (1 - t1) L (1 + t1), ft = (1 - t1) [f + G(t1)] (1 + t1)
  c->c_Lt_copy = combine(Lt, 0.0, {{1.0, L}});
  b.ct(c->p_dress, "Ppa,ia->Ppi", 1.0, sub(L, 2, V0, v), t1, sub(Lt, 2, O0, o));
  b.ct(c->p_dress, "ia,Piq->Paq", -1.0, t1, sub(Lt, 1, O0, o), sub(Lt, 1, V0, v));
  b.ct(c->p_fock, "Pia,ia->P", 1.0, sub(sub(L, 1, O0, o), 2, V0, v), t1, b.T("gamma", {naux}));
  b.ct(c->p_fock, "Prs,P->rs", 1.0, L, b.T("gamma", {naux}), b.T("J", {n, n}));
  b.ct(c->p_fock, "ia,Pis->Pas", 1.0, t1, sub(L, 1, O0, o), b.T("Y", {naux, v, n}));
  b.ct(c->p_fock, "Pra,Pas->rs", 1.0, sub(L, 2, V0, v), b.T("Y", {naux, v, n}), b.T("Kx", {n, n}));
  c->c_fock.push_back(combine(F, 0.0, {{2.0, b.T("J", {n, n})}, {-1.0, b.T("Kx", {n, n})}}));
  c->c_fock.push_back(combine(strided(c->D("F"), {n}, {n + 1}), 1.0, {{1.0, b.T("e", {n})}}));
  c->c_fock.push_back(combine(ft, 0.0, {{1.0, F}}));
  std::vector<GemmPlan*> p_ft;
  b.ct(p_ft, "pa,ia->pi", 1.0, sub(F, 1, V0, v), t1, sub(ft, 1, O0, o));
  b.ct(p_ft, "ia,iq->aq", -1.0, t1, sub(ft, 0, O0, o), sub(ft, 0, V0, v));
  for (GemmPlan* g : p_ft) c->p_fock.push_back(g);  // run after the combines (see run order)

  // --- ERI blocks v~^{pq}_{rs} = sum_P Lt[P,p,r] Lt[P,q,s]
  for (const char* s : blocks) {
    auto sp = [&](char ch) { return ch == 'o' ? std::make_pair(O0, (i64)o) : std::make_pair(V0, (i64)v); };
    auto p = sp(s[0]), q = sp(s[1]), r = sp(s[2]), t = sp(s[3]);
    View A = sub(sub(Lt, 1, p.first, p.second), 2, r.first, r.second);
    View Bv = sub(sub(Lt, 1, q.first, q.second), 2, t.first, t.second);
    b.ct(c->p_eri, "Ppr,Pqs->pqrs", 1.0, A, Bv, eri(s), std::string(s) == "vvvv");
  }

  // --- spin-summed helpers
  c->c_helpers.push_back(combine(b.T("vs_oovv", {o, o, v, v}), 0.0,
                                 {{2.0, eri("oovv")}, {-1.0, permuted(eri("oovv"), {0, 1, 3, 2})}}));
  c->c_helpers.push_back(combine(ts2, 0.0, {{2.0, t2}, {-1.0, permuted(t2, {0, 1, 3, 2})}}));
  c->c_helpers.push_back(combine(b.T("vs_ovvv", {o, v, v, v}), 0.0,
                                 {{2.0, eri("ovvv")}, {-1.0, permuted(eri("ovvv"), {0, 1, 3, 2})}}));
  c->c_helpers.push_back(combine(b.T("vs_oovo", {o, o, v, o}), 0.0,
                                 {{2.0, eri("oovo")}, {-1.0, permuted(eri("ooov"), {0, 1, 3, 2})}}));

  // --- RCCSD and RCCSDT intermediates (appendix A.5)
  View vs_oovv = b.T("vs_oovv", {o, o, v, v}), vs_ovvv = b.T("vs_ovvv", {o, v, v, v});
  View vs_oovo = b.T("vs_oovo", {o, o, v, o});
  View Fvv = b.T("Fvv", {v, v}), Foo = b.T("Foo", {o, o}), Woooo = b.T("Woooo", {o, o, o, o});
  View Wovvo = b.T("Wovvo", {o, v, v, o}), Wovov = b.T("Wovov", {o, v, o, v});
  // W^{ab}_{dj} is stored [j][a][b][d]: the T3 contribution of step (iii) writes it
  // along d (the rows of its GEMM) and the T2-driven R3 term reads it along d (K)
  View Wvvvo = strided(c->D("Wvvvo"), {v, v, v, o}, {V2, v, 1, V3}), Wvooo = b.T("Wvooo", {v, o, o, o});
  View Wb_ovvo = b.T("Wb_ovvo", {o, v, v, o}), Wb_ovov = b.T("Wb_ovov", {o, v, o, v});
  View Wvvvv = b.T("Wvvvv", {v, v, v, v});
  c->c_int_base.push_back(combine(Fvv, 0.0, {{1.0, sub(sub(ft, 0, V0, v), 1, V0, v)}}));
  c->c_int_base.push_back(combine(Foo, 0.0, {{1.0, sub(sub(ft, 0, O0, o), 1, O0, o)}}));
  c->c_int_base.push_back(combine(Woooo, 0.0, {{1.0, eri("oooo")}}));
  c->c_int_base.push_back(combine(Wovvo, 0.0, {{2.0, eri("ovvo")}, {-1.0, permuted(eri("ovov"), {0, 1, 3, 2})}}));
  c->c_int_base.push_back(combine(Wovov, 0.0, {{1.0, eri("ovov")}}));
  c->c_int_base.push_back(combine(permuted(Wvvvo, {3, 0, 1, 2}), 0.0, {{1.0, permuted(eri("vvvo"), {3, 0, 1, 2})}}));
  c->c_int_base.push_back(combine(Wvooo, 0.0, {{1.0, eri("vooo")}}));
  c->c_int_base.push_back(combine(Wvvvv, 0.0, {{1.0, eri("vvvv")}}));
  b.ct(c->p_int, "kldc,kldb->bc", -1.0, vs_oovv, t2, Fvv);
  b.ct(c->p_int, "lkcd,ljcd->kj", 1.0, vs_oovv, t2, Foo);
  b.ct(c->p_int, "klcd,ijcd->klij", 1.0, eri("oovv"), t2, Woooo);
  b.ct(c->p_int, "lkdc,lida->kaci", 0.5, vs_oovv, ts2, Wovvo);
  b.ct(c->p_int, "lkcd,ilda->kaic", -0.5, eri("oovv"), t2, Wovov);
  b.ct(c->p_int, "laed,ljeb->abdj", 0.5, vs_ovvv, ts2, Wvvvo);
  b.ct(c->p_int, "lade,jleb->abdj", -0.5, eri("ovvv"), t2, Wvvvo);
  b.ct(c->p_int, "lbde,jlea->abdj", -1.0, eri("ovvv"), t2, Wvvvo);
  b.ct(c->p_int, "lmdj,lmab->jabd", 1.0, eri("oovo"), t2, permuted(Wvvvo, {3, 0, 1, 2}));  // rows (j, d)
  b.ct(c->p_int, "ld,ijad->alij", 1.0, sub(sub(ft, 0, O0, o), 1, V0, v), t2, Wvooo);
  b.ct(c->p_int, "mldj,mida->alij", 0.5, vs_oovo, ts2, Wvooo);
  b.ct(c->p_int, "mljd,imda->alij", -0.5, eri("ooov"), t2, Wvooo);
  b.ct(c->p_int, "mlid,jmda->alij", -1.0, eri("ooov"), t2, Wvooo);
  b.ct(c->p_int, "alde,ijde->alij", 1.0, eri("vovv"), t2, Wvooo);
  b.ct(c->p_int, "lmde,lmab->abde", 1.0, eri("oovv"), t2, Wvvvv, 1);
  c->c_int_after.resize(1);
  c->c_int_after[0].push_back(combine(Wb_ovvo, 0.0, {{1.0, Wovvo}}));
  c->c_int_after[0].push_back(combine(Wb_ovov, 0.0, {{1.0, Wovov}}));
  std::vector<GemmPlan*> p_int2;
  b.ct(p_int2, "mled,miea->ladi", 0.5, vs_oovv, ts2, Wb_ovvo);
  b.ct(p_int2, "mlde,imea->laid", -0.5, eri("oovv"), t2, Wb_ovov);
  c->p_wbar = p_int2;

  // --- step (iii): T3 contributions, per z batch of unpacked blocks t_{xyz}
  {
    std::vector<i64> base((size_t)o * o * o);
    std::vector<int> pos((size_t)o * o * o * 3);
    for (int z = 0; z < o; ++z)
      for (int x = 0; x < o; ++x)
        for (int y = 0; y < o; ++y) {
          TripleInfo ti = triple(x, y, z);
          size_t id = ((size_t)z * o + x) * o + y;
          base[id] = ti.blk * V3;
          for (int q = 0; q < 3; ++q) pos[id * 3 + q] = ti.pos[q];
        }
    c->a3_base = upload_vec(c, base, &err);
    c->a3_pos = upload_vec(c, pos, &err);
    View dR1 = b.T("dR1", {o, v}), dX2 = b.T("dX2", {o, o, v, v});
    const int Z = c->a3_Z;
    std::shared_ptr<GemmPlan::OwnPanel> own45;
    for (int z0 = 0; z0 < o; z0 += Z) {
      const int Zb = std::min(Z, o - z0);
      View Sz = dense(c->B("Sz")->p, {Zb, o, o, v, v, v}, t3f);  // S[z][x][y][e1][e2][e3]
      c->p_a3.emplace_back();
      auto& g = c->p_a3.back();
      // (the T3 term of R1: k_r1_t3 on the unpacked batch, or the first panel's gather)
      View dX2z = sub(permuted(dX2, {1, 0, 2, 3}), 0, z0, Zb);  // dX2[y, z, a, b] over (z, y, a, b)
      GemmPlan* q1 = b.ct(g, "xc,zxycab->zyab", 0.5, sub(sub(ft, 0, O0, o), 1, V0, v), Sz, dX2z);
      // S panel [(y,e2,e3)][(z,x,e1)], shared by two contractions (and the first one when Zb = 1)
      GemmPlan* q2 = b.ct(g, "zxjc,zxycab->yjab", -1.0, sub(eri("ooov"), 0, z0, Zb), Sz, dX2);
      if (q2 && Zb == 1) q2->reuse_B = 1;
      GemmPlan* q3 = b.ct(g, "zxde,zxyeba->ybad", -1.0, sub(eri("oovv"), 0, z0, Zb), Sz,
                          permuted(Wvvvo, {3, 1, 0, 2}), 1);
      if (q3) q3->reuse_B = 1;
      // two contractions over (x, e3, e1), rows (z, y, e2)
      GemmPlan* q4 = b.ct(g, "bxcd,zxydac->zyab", 1.0, eri("vovv"), Sz, dX2z, 1);
      GemmPlan* q5 = b.ct(g, "lxde,zxyead->zyal", 1.0, eri("oovv"), Sz,
                          permuted(sub(permuted(Wvooo, {3, 0, 1, 2}), 0, z0, Zb), {0, 3, 1, 2}));
      if (q5) q5->reuse_B = 1;
      // The last two contractions sum over (x, e3, e1): they read the first panel
      // P1 [(z, y, e2, e3)][(x, e1)] (K padded to Kp1) as [(z, y, e2)][(e3, x, e1)],
      // the same memory with K blocks of Kp1 per e3, so they need no panel of their
      // own; their A operands are laid out with the same padded K.
      if (q1 && q4 && q5) {
        const int Kp1 = q1->Kpad, K45 = v * Kp1;
        std::vector<double> cf((size_t)K45, 0.0);
        std::vector<i64> cbase((size_t)K45, 0);
        for (int e3 = 0; e3 < v; ++e3)
          for (int x = 0; x < o; ++x)
            for (int e1 = 0; e1 < v; ++e1) {
              const size_t k = (size_t)e3 * Kp1 + (size_t)x * v + e1;
              cf[k] = 1.0;
              cbase[k] = (i64)x * V2 + (i64)e3 * v + e1;  // vovv[b][x][e3][e1], oovv[l][x][e3][e1]
            }
        std::vector<i64> rb(v), rl(o);
        for (int bb = 0; bb < v; ++bb) rb[bb] = (i64)bb * o * V2;
        for (int l = 0; l < o; ++l) rl[l] = (i64)l * o * V2;
        make_pack(c, q4->A, c->D("vovv"), 0, v, K45, 1, cf, cbase, std::vector<int>((size_t)K45, 0), rb, 1, &err);
        make_pack(c, q5->A, c->D("oovv"), 0, o, K45, 1, cf, cbase, std::vector<int>((size_t)K45, 0), rl, 1, &err);
        for (GemmPlan* q : {q4, q5}) {
          q->B = PackPlan();
          q->B.a.R = q->E.e.N;
          q->reuse_B = 1;  // the panel of q1
          finish_plan(c, q, K45);
        }
      }
      if (t3f && q1 && q2 && q3 && q4 && q5) {
        // split bodies: the S panels straight from T3 through label cubes, one piece
        // per block S^{xy} = 2 U^{e1e2e3} - U^{e2e1e3} - U^{e3e2e1}, U = t_{x y z}
        // (no unpacked batch); the first panel's gather also forms the R1 partials
        auto spin = [&](rcc::CubePiece& pc, int x, int y, int z, const int lab[3]) {
          // lab[q]: the S label (0 e1, 1 e2, 2 e3) of the piece's label Lq; term t
          // reads S label s in slot slot[t][s] of U
          static const int slot[3][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0}};
          static const float coef[3] = {2.f, -1.f, -1.f};
          const TripleInfo u = triple(x, y, z);
          pc.nterm = 3;
          for (int t = 0; t < 3; ++t)
            pc.t[t] = {u.blk * V3, coef[t],
                       packpos(u.pos[slot[t][lab[0]]], u.pos[slot[t][lab[1]]], u.pos[slot[t][lab[2]]])};
        };
        const int l123[3] = {0, 1, 2};
        std::vector<rcc::CubePiece> pa_, pb_;
        std::vector<i64> wb;
        for (int z = 0; z < Zb; ++z)
          for (int x = 0; x < o; ++x)
            for (int y = 0; y < o; ++y) {
              rcc::CubePiece p1 = cube_piece(x * v, 3, v);  // rows (z, y, e2, e3), K (x, e1)
              p1.row0 = ((i64)z * o + y) * V2;
              spin(p1, x, y, z0 + z, l123);
              rcc::CubePiece p2 = cube_piece((z * o + x) * v, 3, v);  // rows (y, e2, e3), K (z, x, e1)
              p2.row0 = (i64)y * V2;
              spin(p2, x, y, z0 + z, l123);
              pa_.push_back(p1);
              pb_.push_back(p2);
              wb.push_back(((i64)x * o + y) * V2);  // v^{xy} in oovv [x][y][b][c]
            }
        for (GemmPlan* q : {q1, q2, q3}) q->cube_src = c->B("t3")->f();
        set_cube(c, q1, 0, pa_, &err);
        q1->r1_wbase = upload_vec(c, wb, &err);
        ++c->a3_direct;
        set_cube(c, q2, 0, pb_, &err);
        set_cube(c, q3, 0, std::move(pb_), &err);
      }
      // one pass over each S panel: the contractions sharing it run as one GEMM with
      // stacked A operands.  (With Zb = 1 the first contraction's panel is the
      // second's too, but both write dX2[y][z0], so they stay two GEMMs.)
      if (q1 && q2 && q3 && q4 && q5) {
        auto replace = [&](const std::vector<GemmPlan*>& parts) -> GemmPlan* {
          GemmPlan* m = stack_rows(c, parts, &err);
          if (!m) return nullptr;
          auto at = std::find(g.begin(), g.end(), parts[0]);
          const size_t pos = (size_t)(at - g.begin());
          for (GemmPlan* q : parts) g.erase(std::find(g.begin(), g.end(), q));
          g.insert(g.begin() + pos, m);
          return m;
        };
        replace({q2, q3});
        GemmPlan* m45 = replace({q4, q5});
        // the A operand of (q4 q5) (vovv and oovv over (e3, x, e1)) is the same for every
        // z batch: in the split modes it is packed once per iteration into a panel of
        // its own (the first batch packs it)
        if (m45 && t3f) {
          if (!own45) {
            own45 = std::make_shared<GemmPlan::OwnPanel>();
            const size_t bytes = (size_t)m45->A.a.R * m45->Kpad * 4;  // widest split element (TF32)
            own45->hi.p = dev_alloc(bytes, &err);
            own45->hi.bytes = bytes;
            own45->lo.p = dev_alloc(bytes, &err);
            own45->lo.bytes = bytes;
            m45->own_pack = 1;
          }
          m45->own = own45;
        }
        // q1's panel must still be in place for the reshaped read: q1, (q4 q5), (q2 q3)
        std::stable_partition(g.begin(), g.end(), [&](GemmPlan* p) {
          return p == q1 || (!p->a_parts.empty() && p->a_parts[0] == q4) || p == q4 || p == q5;
        });
      }
    }
  }

  // --- R1, R2
  View r1 = b.T("r1", {o, v}), X2 = b.T("X2", {o, o, v, v});
  c->c_r12_base.push_back(combine(r1, 0.0, {{1.0, permuted(sub(sub(ft, 0, V0, v), 1, O0, o), {1, 0})},
                                            {1.0, b.T("dR1", {o, v})}}));
  b.ct(c->p_r12, "kc,ikac->ia", 1.0, sub(sub(ft, 0, O0, o), 1, V0, v), ts2, r1);
  b.ct(c->p_r12, "akcd,ikcd->ia", 1.0, eri("vovv"), ts2, r1);
  b.ct(c->p_r12, "klic,klac->ia", -1.0, eri("ooov"), ts2, r1);
  c->c_r12_base.push_back(combine(X2, 0.0, {{0.5, permuted(eri("vvoo"), {2, 3, 0, 1})},
                                            {1.0, b.T("dX2", {o, o, v, v})}}));
  b.ct(c->p_r12, "bc,ijac->ijab", 1.0, Fvv, t2, X2);
  b.ct(c->p_r12, "kj,ikab->ijab", -1.0, Foo, t2, X2);
  b.ct(c->p_r12, "abcd,ijcd->ijab", 0.5, eri("vvvv"), t2, X2, 1);
  b.ct(c->p_r12, "klij,klab->ijab", 0.5, Woooo, t2, X2);
  b.ct(c->p_r12, "kaci,kjcb->ijab", 0.5, Wovvo, ts2, X2);
  b.ct(c->p_r12, "kaic,jkcb->ijab", -0.5, Wovov, t2, X2);
  b.ct(c->p_r12, "kbic,jkca->ijab", -1.0, Wovov, t2, X2);
  c->c_r2_sym.push_back(combine(b.T("r2", {o, o, v, v}), 0.0, {{1.0, X2}, {1.0, permuted(X2, {1, 0, 3, 2})}}));

  // --- R3 operands: F folded into W_vvvv and W_oooo, ring A operands
  {
    View Wt = b.T("Wt_oooo", {o, o, o, o});
    c->c_wt.push_back(combine(Wt, 0.0, {{1.0, Woooo}}));
    // W~^{lm}_{ij} -= 1/2 F^l_i delta_mj ; -= 1/2 delta_li F^m_j
    c->c_wt.push_back(combine(strided(c->D("Wt_oooo"), {o, o, o}, {(i64)o * o * o, (i64)o * o + 1, o}), 1.0,
                              {{-0.5, strided(c->D("Foo"), {o, o, o}, {o, 0, 1})}}));
    c->c_wt.push_back(combine(strided(c->D("Wt_oooo"), {o, o, o}, {(i64)o * o * o + o, (i64)o * o, 1}), 1.0,
                              {{-0.5, strided(c->D("Foo"), {o, o, o}, {0, o, 1})}}));
    // W~^{ab}_{de} += 1/2 F^a_d delta_be ; += 1/2 delta_ad F^b_e
    c->c_wt.push_back(combine(strided(c->D("Wvvvv"), {v, v, v}, {V3, V2 + 1, v}), 1.0,
                              {{0.5, strided(c->D("Fvv"), {v, v, v}, {v, 0, 1})}}));
    c->c_wt.push_back(combine(strided(c->D("Wvvvv"), {v, v, v}, {V3 + v, V2, 1}), 1.0,
                              {{0.5, strided(c->D("Fvv"), {v, v, v}, {0, v, 1})}}));
    // Wring_ab[i][a][0][l][d] = 1/4 Wbar^{la}_{di};  [1][l][d] = -1/4 Wbar^{la}_{id}
    const i64 K2 = 2LL * o * v;
    View Wab0 = strided(c->D("Wring_ab"), {o, v, o, v}, {v * K2, K2, v, 1});
    View Wab1 = strided(c->D("Wring_ab") + (i64)o * v, {o, v, o, v}, {v * K2, K2, v, 1});
    c->c_wt.push_back(combine(Wab0, 0.0, {{0.25, permuted(Wb_ovvo, {3, 1, 0, 2})}}));
    c->c_wt.push_back(combine(Wab1, 0.0, {{-0.25, permuted(Wb_ovov, {2, 1, 0, 3})}}));
    // Wring_c[i][b][l][d] = -Wbar^{lb}_{id}
    c->c_wt.push_back(combine(b.T("Wring_c", {o, v, o, v}), 0.0, {{-1.0, permuted(Wb_ovov, {2, 1, 0, 3})}}));
  }

  void* r3p = c->B("r3")->p;
  void* t3p = c->B("t3")->p;
  // --- pp-ladder: three views of each stored block (direct traversal)
  {
    i64 per_blk = (i64)v * round_up((int)V2, 64) * 8;
    i64 nb = std::max<i64>(1, std::min<i64>(n3, pp_unit_bytes(c) / per_blk));
    for (int term = 0; term < 3; ++term)
      for (i64 b0 = 0; b0 < n3; b0 += nb) {
        i64 b1 = std::min(n3, b0 + nb);
        int N = (int)((b1 - b0) * v);
        GemmPlan* g = b.new_plan();
        std::vector<i64> arow(V2), acol(V2), brow(N), bcol(V2), ebase(V2), ecol(N);
        for (i64 r = 0; r < V2; ++r) { arow[r] = r * V2; acol[r] = r; }
        for (i64 q = 0; q < V2; ++q) {
          i64 d = q / v, e = q % v;
          bcol[q] = term == 0 ? d * V2 + e * v : term == 1 ? d * V2 + e : d * v + e;
        }
        for (int q = 0; q < N; ++q) {
          i64 blk = b0 + q / v, w = q % v;
          brow[q] = blk * V3 + (term == 0 ? w : term == 1 ? w * v : w * V2);
          ecol[q] = brow[q];
        }
        for (i64 r = 0; r < V2; ++r) {
          i64 x = r / v, y = r % v;
          ebase[r] = term == 0 ? x * V2 + y * v : term == 1 ? x * V2 + y : x * v + y;
        }
        make_pack(c, g->A, c->D("Wvvvv"), 0, (int)V2, (int)V2, 1, std::vector<double>(V2, 1.0), acol,
                  std::vector<int>(V2, 0), arow, 1, &err);
        make_pack(c, g->B, t3p, t3f, N, (int)V2, 1, std::vector<double>(V2, 1.0), bcol, std::vector<int>(V2, 0),
                  brow, term == 0 ? 0 : 1, &err);
        make_epi(c, g->E, r3p, t3f, (int)V2, N, ebase, std::vector<int>(V2, 0), std::vector<double>(V2, 1.0),
                 ecol, &err);
        g->big = 1;
        g->step = 1;
        // grouped form: X = T3 view x W^T, rows (blk, w), columns (x, y) -- each block
        // of v rows is the contiguous v^3 block [w][x][y] of stored block blk
        {
          static const int ax[3][3] = {{2, 0, 1}, {1, 0, 2}, {0, 1, 2}};
          int pos[3] = {ax[term][0], ax[term][1], ax[term][2]};
          for (i64 blk = b0; blk < b1; ++blk) {
            g->h_base.push_back(blk * V3);
            g->h_sel.push_back(perm_id(pos));
            g->h_alpha.push_back(1.0);
          }
          g->swap_ab = 1;
        }
        finish_plan(c, g, (int)V2);
        if (t3f) {  // split bodies: B through label cubes, one piece per block, K = (d, e), rows w
          static const int vp[3][3] = {{1, 0, 2}, {2, 0, 1}, {2, 1, 0}};  // stored axes of (e, d, w)
          std::vector<rcc::CubePiece> pcs;
          for (i64 blk = b0; blk < b1; ++blk) {
            rcc::CubePiece pc = cube_piece(0, 1);
            pc.ks1 = v;
            pc.rs1 = 0;
            pc.rs2 = 1;
            pc.row0 = (blk - b0) * v;
            pc.t[0] = {blk * V3, 1.f, packpos(vp[term][0], vp[term][1], vp[term][2])};
            pcs.push_back(pc);
          }
          set_cube(c, g, 0, std::move(pcs), &err);
        }
        c->p_pp.push_back(g);
      }
    build_pp_sym(c, t3f, r3p, &err);
  }

  // --- hh-ladder (with F_oo folded in), unit k: rows (i<=j), cols abc, K = (l,m)
  {
    std::vector<std::pair<int, int>> pairs;
    for (int i = 0; i < o; ++i)
      for (int j = i; j < o; ++j) pairs.push_back({i, j});
    const int M = (int)pairs.size(), K = o * o;
    for (int k = 0; k < o; ++k) {
      GemmPlan* g = b.new_plan();
      std::vector<i64> arow(M), acol(K), bcol(K), ebase(M);
      std::vector<int> bsel(K), esel(M);
      std::vector<double> ealpha(M);
      for (int q = 0; q < M; ++q) arow[q] = (i64)pairs[q].first * o + pairs[q].second;
      for (int l = 0; l < o; ++l)
        for (int m = 0; m < o; ++m) {
          acol[l * o + m] = (i64)l * o * o * o + (i64)m * o * o;
          TripleInfo ti = triple(l, m, k);
          bcol[l * o + m] = ti.blk * V3;
          bsel[l * o + m] = perm_id(ti.pos);
        }
      for (int q = 0; q < M; ++q) {
        TripleInfo ti = triple(pairs[q].first, pairs[q].second, k);
        ebase[q] = ti.blk * V3;
        esel[q] = perm_id(ti.pos);
        ealpha[q] = (6.0 / ti.m) * (pairs[q].first < pairs[q].second ? 2.0 : 1.0);
      }
      make_pack(c, g->A, c->D("Wt_oooo"), 0, M, K, 1, std::vector<double>(K, 0.5), acol, std::vector<int>(K, 0),
                arow, 0, &err);
      make_pack(c, g->B, t3p, t3f, (int)V3, K, 1, std::vector<double>(K, 1.0), bcol, bsel, {}, 0, &err, b.RT3, 3);
      make_epi(c, g->E, r3p, t3f, M, (int)V3, ebase, esel, ealpha, {}, &err, b.RT3);
      g->big = 1;
      g->step = 3;
      {
        std::vector<std::array<int, 3>> ax(M);
        for (int q = 0; q < M; ++q) {
          TripleInfo ti = triple(pairs[q].first, pairs[q].second, k);
          ax[q] = {ti.pos[0], ti.pos[1], ti.pos[2]};                       // X block [a][b][c]
        }
        set_two_phase(c, g, ebase, ax, ealpha, &err);
      }
      finish_plan(c, g, K);
      if (t3f) {  // B columns (l, m): the block t_{lmk} with rows (a, b, c); zero columns to Kpad
        std::vector<rcc::CubePiece> pcs;
        for (int q = 0; q < g->Kpad; ++q) {
          rcc::CubePiece pc = cube_piece(q, q < K ? 1 : 0);
          if (q < K) {
            TripleInfo ti = triple(q / o, q % o, k);
            pc.t[0].base = ti.blk * V3;
            pc.t[0].coef = 1.f;
            pc.t[0].pos = packpos(ti.pos[0], ti.pos[1], ti.pos[2]);
          }
          pcs.push_back(pc);
        }
        set_cube(c, g, 1, std::move(pcs), &err);
        g->tc_swap = 1;  // rows (i <= j) become the 144/128-wide tile columns
      }
      c->p_hh.push_back(g);
    }
  }

  // --- ring terms (a) + (b): unit (j <= k); rows (i,a), cols (b,c), K = (part, l, d)
  {
    const int M = o * v, K = 2 * o * v;
    for (int j = 0; j < o; ++j)
      for (int k = j; k < o; ++k) {
        GemmPlan* g = b.new_plan();
        std::vector<i64> arow(M), acol(K), bcol((size_t)3 * K), ebase(M);
        std::vector<int> bsel((size_t)3 * K, 0), esel(M);
        std::vector<double> bcoef((size_t)3 * K, 0.0), ealpha(M);
        for (int r = 0; r < M; ++r) arow[r] = (i64)r * K;
        for (int q = 0; q < K; ++q) acol[q] = q;
        for (int l = 0; l < o; ++l) {
          TripleInfo u = triple(l, j, k), u1 = triple(j, l, k), u2 = triple(k, l, j);
          for (int d = 0; d < v; ++d) {
            int q0 = l * v + d, q1 = o * v + l * v + d;
            // part 0: 2 U^{dbc} - U^{bdc} - U^{cbd}, U = t_{ljk}
            bcoef[q0] = 2.0; bcol[q0] = u.blk * V3 + d * b.S[u.pos[0]]; bsel[q0] = u.pos[1] * 3 + u.pos[2];
            bcoef[K + q0] = -1.0; bcol[K + q0] = u.blk * V3 + d * b.S[u.pos[1]]; bsel[K + q0] = u.pos[0] * 3 + u.pos[2];
            bcoef[2 * K + q0] = -1.0; bcol[2 * K + q0] = u.blk * V3 + d * b.S[u.pos[2]]; bsel[2 * K + q0] = u.pos[1] * 3 + u.pos[0];
            // part 1: t_{jlk}^{dbc} + t_{klj}^{dcb}
            bcoef[q1] = 1.0; bcol[q1] = u1.blk * V3 + d * b.S[u1.pos[0]]; bsel[q1] = u1.pos[1] * 3 + u1.pos[2];
            bcoef[K + q1] = 1.0; bcol[K + q1] = u2.blk * V3 + d * b.S[u2.pos[0]]; bsel[K + q1] = u2.pos[2] * 3 + u2.pos[1];
            bcol[2 * K + q1] = u1.blk * V3;
          }
        }
        for (int i = 0; i < o; ++i) {
          TripleInfo ti = triple(i, j, k);
          for (int a = 0; a < v; ++a) {
            ebase[i * v + a] = ti.blk * V3 + a * b.S[ti.pos[0]];
            esel[i * v + a] = ti.pos[1] * 3 + ti.pos[2];
            ealpha[i * v + a] = (6.0 / ti.m) * (j < k ? 2.0 : 1.0);
          }
        }
        make_pack(c, g->A, c->D("Wring_ab"), 0, M, K, 1, std::vector<double>(K, 1.0), acol, std::vector<int>(K, 0),
                  arow, 1, &err);
        make_pack(c, g->B, t3p, t3f, (int)V2, K, 3, bcoef, bcol, bsel, {}, 0, &err, b.RT2, 2);
        make_epi(c, g->E, r3p, t3f, M, (int)V2, ebase, esel, ealpha, {}, &err, b.RT2);
        g->big = 1;
        g->step = 2;
        {
          std::vector<i64> tb(o);
          std::vector<std::array<int, 3>> ax(o);
          std::vector<double> ta(o);
          for (int i = 0; i < o; ++i) {
            TripleInfo ti = triple(i, j, k);
            tb[i] = ti.blk * V3;
            ax[i] = {ti.pos[0], ti.pos[1], ti.pos[2]};                        // X block [a][b][c]
            ta[i] = (6.0 / ti.m) * (j < k ? 2.0 : 1.0);
          }
          set_two_phase(c, g, tb, ax, ta, &err);
        }
        finish_plan(c, g, K);
        g->tc_swap = 1;  // column-major dense result: coalesced rows of the raw output
        if (t3f) {  // B: labels (d, b, c), K = (part, l, d), rows (b, c)
          std::vector<rcc::CubePiece> pcs;
          for (int l = 0; l < o; ++l) {
            TripleInfo u = triple(l, j, k), u1 = triple(j, l, k), u2 = triple(k, l, j);
            rcc::CubePiece p0 = cube_piece(l * v, 3, v);
            p0.t[0] = {u.blk * V3, 2.f, packpos(u.pos[0], u.pos[1], u.pos[2])};
            p0.t[1] = {u.blk * V3, -1.f, packpos(u.pos[1], u.pos[0], u.pos[2])};
            p0.t[2] = {u.blk * V3, -1.f, packpos(u.pos[2], u.pos[1], u.pos[0])};
            rcc::CubePiece p1 = cube_piece(o * v + l * v, 2, v);
            p1.t[0] = {u1.blk * V3, 1.f, packpos(u1.pos[0], u1.pos[1], u1.pos[2])};
            p1.t[1] = {u2.blk * V3, 1.f, packpos(u2.pos[0], u2.pos[2], u2.pos[1])};
            pcs.push_back(p0);
            pcs.push_back(p1);
          }
          set_cube(c, g, 0, std::move(pcs), &err);
        }
        c->p_ringab.push_back(g);
      }
  }

  // --- ring term (c): unit (j,k); rows (i,b), cols (a,c), K = (l,d)
  {
    const int M = o * v, K = o * v;
    for (int j = 0; j < o; ++j)
      for (int k = 0; k < o; ++k) {
        GemmPlan* g = b.new_plan();
        std::vector<i64> arow(M), acol(K), bcol(K), ebase(M);
        std::vector<int> bsel(K), esel(M);
        std::vector<double> ealpha(M);
        for (int r = 0; r < M; ++r) arow[r] = (i64)r * K;
        for (int q = 0; q < K; ++q) acol[q] = q;
        for (int l = 0; l < o; ++l) {
          TripleInfo u = triple(j, l, k);
          for (int d = 0; d < v; ++d) {
            bcol[l * v + d] = u.blk * V3 + d * b.S[u.pos[0]];
            bsel[l * v + d] = u.pos[1] * 3 + u.pos[2];
          }
        }
        for (int i = 0; i < o; ++i) {
          TripleInfo ti = triple(i, j, k);
          for (int bb = 0; bb < v; ++bb) {
            ebase[i * v + bb] = ti.blk * V3 + bb * b.S[ti.pos[1]];
            esel[i * v + bb] = ti.pos[0] * 3 + ti.pos[2];
            ealpha[i * v + bb] = 6.0 / ti.m;
          }
        }
        make_pack(c, g->A, c->D("Wring_c"), 0, M, K, 1, std::vector<double>(K, 1.0), acol, std::vector<int>(K, 0),
                  arow, 1, &err);
        make_pack(c, g->B, t3p, t3f, (int)V2, K, 1, std::vector<double>(K, 1.0), bcol, bsel, {}, 0, &err, b.RT2, 2);
        make_epi(c, g->E, r3p, t3f, M, (int)V2, ebase, esel, ealpha, {}, &err, b.RT2);
        g->big = 1;
        g->step = 2;
        {
          std::vector<i64> tb(o);
          std::vector<std::array<int, 3>> ax(o);
          std::vector<double> ta(o);
          for (int i = 0; i < o; ++i) {
            TripleInfo ti = triple(i, j, k);
            tb[i] = ti.blk * V3;
            ax[i] = {ti.pos[1], ti.pos[0], ti.pos[2]};                        // X block [b][a][c]
            ta[i] = 6.0 / ti.m;
          }
          set_two_phase(c, g, tb, ax, ta, &err);
        }
        finish_plan(c, g, K);
        g->tc_swap = 1;
        if (t3f) {  // B: labels (d, a, c) of t_{jlk}, K = (l, d), rows (a, c)
          std::vector<rcc::CubePiece> pcs;
          for (int l = 0; l < o; ++l) {
            TripleInfo u = triple(j, l, k);
            rcc::CubePiece pc = cube_piece(l * v, 1, v);
            pc.t[0] = {u.blk * V3, 1.f, packpos(u.pos[0], u.pos[1], u.pos[2])};
            pcs.push_back(pc);
          }
          set_cube(c, g, 0, std::move(pcs), &err);
        }
        c->p_ringc.push_back(g);
      }
  }

  // --- T2-driven term sum_d W^{ab}_{dj} t_ik^{dc}: unit (j, i<k | i>k | i=k);
  //     rows (pair, c), cols (a, b), K = d
  for (int j = 0; j < o; ++j)
    for (int region = 0; region < 3; ++region) {
      std::vector<std::pair<int, int>> pairs;
      for (int i = 0; i < o; ++i)
        for (int k = 0; k < o; ++k)
          if ((region == 0 && i < k) || (region == 1 && i > k) || (region == 2 && i == k)) pairs.push_back({i, k});
      if (pairs.empty()) continue;
      const int M = (int)pairs.size() * v, K = v;
      GemmPlan* g = b.new_plan();
      std::vector<i64> arow(M), acol(K), brow(V2), bcol(K), ebase(M);
      std::vector<int> esel(M);
      std::vector<double> ealpha(M);
      for (int q = 0; q < (int)pairs.size(); ++q)
        for (int cc = 0; cc < v; ++cc) {
          int r = q * v + cc;
          arow[r] = ((i64)pairs[q].first * o + pairs[q].second) * V2 + cc;
          TripleInfo ti = triple(pairs[q].first, j, pairs[q].second);
          ebase[r] = ti.blk * V3 + cc * b.S[ti.pos[2]];
          esel[r] = ti.pos[0] * 3 + ti.pos[1];
          ealpha[r] = 6.0 / ti.m;
        }
      for (int d = 0; d < v; ++d) { acol[d] = (i64)d * v; bcol[d] = d; }
      for (i64 ab = 0; ab < V2; ++ab) brow[ab] = (i64)j * V3 + ab * v;  // W stored [j][a][b][d]
      make_pack(c, g->A, c->D("t2"), 0, M, K, 1, std::vector<double>(K, 1.0), acol, std::vector<int>(K, 0), arow, 0,
                &err);
      make_pack(c, g->B, c->D("Wvvvo"), 0, (int)V2, K, 1, std::vector<double>(K, 1.0), bcol, std::vector<int>(K, 0),
                brow, 1, &err);
      make_epi(c, g->E, r3p, t3f, M, (int)V2, ebase, esel, ealpha, {}, &err, b.RT2);
      g->big = 1;
      g->step = 4;
      {
        const int np = (int)pairs.size();
        std::vector<i64> tb(np);
        std::vector<std::array<int, 3>> ax(np);
        std::vector<double> ta(np);
        for (int q = 0; q < np; ++q) {
          TripleInfo ti = triple(pairs[q].first, j, pairs[q].second);
          tb[q] = ti.blk * V3;
          ax[q] = {ti.pos[2], ti.pos[0], ti.pos[1]};                          // X block [c][a][b]
          ta[q] = 6.0 / ti.m;
        }
        set_two_phase(c, g, tb, ax, ta, &err);
      }
      finish_plan(c, g, K);
      g->tc_swap = 1;  // K = v is short: the GEMM streams its result, written column-major (coalesced)
      c->p_t2a.push_back(g);
    }

  // (the T2-driven term -sum_l W^{al}_{ij} t_lk^{bc} runs output-stationary in k_t2_outer)
  if (t3f) {
    b.mk("t2_f", (size_t)o * o * V2, 4);
    b.mk("Wvooo_f", (size_t)v * o * o * o, 4);
  }

  // the A panel is shared by consecutive plans of these groups
  for (auto* grp : {&c->p_pp, &c->p_hh, &c->p_ringab, &c->p_ringc})
    for (size_t q = 1; q < grp->size(); ++q) (*grp)[q]->reuse_A = 1;

  if (err) return fail(c, err, "plan construction failed");
  return 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// Grouped residual setup.  The problems are the tensor-core contractions of the
// R3 residual (pp-ladder with exchanged operands, ring, hh-ladder, T2 terms);
// panels whose plans share an operand are gathered once.  Returns 0 and leaves
// gr.on = 0 when the mode does not apply or exceeds its memory budget.
// ---------------------------------------------------------------------------
namespace {

struct GPanel {
  const rcc::PackArgs* src;
  size_t hi = 0, lo = 0;  // byte offsets in the panel arena
  const GemmPlan* cube = nullptr;  // gathered through label cubes (the plan's pieces)
};

// Problem table of the grouped GEMM for tile width bn and problem order ord
// (0: longest K first -- the persistent CTAs take tiles round robin; 1: plan order).
int grouped_table(rccsdt_ctx* c, int bn, int ord, std::unique_ptr<DBuf>* out, int* ntiles) {
  auto& G = c->gr;
  const size_t n = G.src.size();
  std::vector<rcc::GProblem> probs(n);
  for (size_t q = 0; q < n; ++q) {
    const auto& x = G.src[q];
    if (rcc::make_gproblem(&probs[q], G.kind, x.ahi, x.alo, x.bhi, x.blo, x.M, x.N, x.Kpad, x.out, bn))
      return fail(c, RCCSDT_ERR_CUDA, "grouped residual: tensor map encoding failed");
    probs[q].colmajor = x.colmajor;
  }
  std::vector<int> order(n);
  for (size_t q = 0; q < n; ++q) order[q] = (int)q;
  if (ord == 0)
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return probs[x].kblocks > probs[y].kblocks; });
  std::vector<rcc::GProblem> sorted;
  int t0 = 0;
  for (int q : order) {
    rcc::GProblem P = probs[q];
    P.tile0 = t0;
    t0 += rcc::gproblem_tiles(P);
    sorted.push_back(P);
  }
  int err = 0;
  *out = upload_vec(c, sorted, &err);
  *ntiles = t0;
  if (err) return fail(c, RCCSDT_ERR_OOM, "grouped residual: table upload failed");
  return 0;
}

int build_grouped(rccsdt_ctx* c) {
  auto& G = c->gr;
  G.on = 0;
  if (c->opt.precision == RCCSDT_FP64 || c->opt.grouped_bytes <= 0) return 0;
  const int kind = c->opt.precision == RCCSDT_SPLIT_BF16X3 ? rcc::PANEL_BF16X2 : rcc::PANEL_TF32X2;
  const size_t esz = kind == rcc::PANEL_BF16X2 ? 2 : 4;
  std::vector<GemmPlan*> plans;
  for (auto* grp : {&c->p_pp, &c->p_ringab, &c->p_ringc, &c->p_hh, &c->p_t2a})
    for (GemmPlan* g : *grp) plans.push_back(g);
  if (plans.empty()) return 0;
  // panels: the shared operand of a group (reuse_A) is gathered once
  std::vector<GPanel> panels;
  std::vector<int> pa(plans.size()), pb(plans.size());
  size_t off = 0;
  auto add_panel = [&](const rcc::PackArgs* a) {
    GPanel p;
    p.src = a;
    const size_t plane = (size_t)a->R * a->Kpad * esz;
    p.hi = off;
    off += (plane + 255) / 256 * 256;
    p.lo = off;
    off += (plane + 255) / 256 * 256;
    panels.push_back(p);
    return (int)panels.size() - 1;
  };
  for (size_t q = 0; q < plans.size(); ++q) {
    GemmPlan* g = plans[q];
    const rcc::PackArgs* shared = &g->A.a;  // the operand reuse_A refers to
    const rcc::PackArgs* other = &g->B.a;
    int ish = (g->reuse_A && q > 0) ? -1 : add_panel(shared);
    if (ish < 0) ish = plans[q - 1]->swap_ab ? pb[q - 1] : pa[q - 1];
    const int iot = add_panel(other);
    if (!g->swap_ab && g->cube) panels[iot].cube = g;
    if (g->swap_ab) {
      pa[q] = iot;
      pb[q] = ish;
    } else {
      pa[q] = ish;
      pb[q] = iot;
    }
  }
  const size_t panel_bytes = off;
  // dense results
  std::vector<size_t> xo(plans.size());
  size_t xel = 0;
  for (size_t q = 0; q < plans.size(); ++q) {
    xo[q] = xel;
    xel += ((size_t)plans[q]->E.e.M * plans[q]->E.e.N + 63) / 64 * 64;
  }
  const size_t need = panel_bytes + xel * 4;
  G.flop = 0.0;
  for (GemmPlan* g : plans) G.flop += 2.0 * g->fma;
  if ((long long)need > c->opt.grouped_bytes) return 0;
  int err = 0;
  G.panels = std::make_unique<DBuf>();
  G.panels->bytes = panel_bytes;
  G.panels->p = dev_alloc(panel_bytes, &err);
  G.raw = std::make_unique<DBuf>();
  G.raw->bytes = xel * 4;
  G.raw->p = dev_alloc(G.raw->bytes, &err);
  if (err) return fail(c, RCCSDT_ERR_OOM, "grouped residual: device allocation failed");
  c->total_bytes += need;
  G.bytes = need;
  char* base = (char*)G.panels->p;
  float* raw = (float*)G.raw->p;
  // gathers, split by source type
  // the padding columns of every panel stay zero (gathers write columns < K only)
  if (dev_zero(G.panels->p, panel_bytes, c->stream) || dev_sync(c->stream))
    return fail(c, RCCSDT_ERR_CUDA, "grouped residual: panel clear failed");
  std::vector<rcc::PackArgs> packs[2];
  std::vector<int> ptile[2];
  std::vector<rcc::CubePiece> cubes[2];
  std::vector<rcc::CubeDst> cdst;
  int tiles[2] = {0, 0};
  for (const GPanel& p : panels) {
    if (p.cube) {
      const int d = (int)cdst.size();
      cdst.push_back({base + p.hi, base + p.lo, p.src->Kpad});
      for (rcc::CubePiece pc : p.cube->h_cube) {
        pc.dst = d;
        cubes[p.cube->cube_mode].push_back(pc);
      }
      continue;
    }
    rcc::PackArgs a = *p.src;
    a.kind = kind;
    a.out_hi = base + p.hi;
    a.out_lo = base + p.lo;
    const int t = a.src_f32 ? 1 : 0;
    packs[t].push_back(a);
    ptile[t].push_back(tiles[t]);
    tiles[t] += rcc::pack_tiles_of(a);
  }
  for (int t = 0; t < 2; ++t) {
    G.npack[t] = (int)packs[t].size();
    G.ntile[t] = tiles[t];
    if (G.npack[t]) {
      G.packs[t] = upload_vec(c, packs[t], &err);
      G.ptile[t] = upload_vec(c, ptile[t], &err);
    }
    G.ncube[t] = (int)cubes[t].size();
    if (G.ncube[t]) G.cubes[t] = upload_vec(c, cubes[t], &err);
  }
  if (!cdst.empty()) G.cube_dst = upload_vec(c, cdst, &err);
  // problems (kept as sources so that other launch shapes can be encoded later)
  for (size_t q = 0; q < plans.size(); ++q) {
    GemmPlan* g = plans[q];
    const GPanel &A = panels[pa[q]], &B = panels[pb[q]];
    rccsdt_ctx::Grouped::Src x;
    x.ahi = base + A.hi;
    x.alo = base + A.lo;
    x.bhi = base + B.hi;
    x.blo = base + B.lo;
    x.M = (g->swap_ab || g->tc_swap) ? g->E.e.N : g->E.e.M;
    x.N = (g->swap_ab || g->tc_swap) ? g->E.e.M : g->E.e.N;
    x.colmajor = g->tc_swap;
    if (g->tc_swap) {  // exchanged operands, column-major result
      std::swap(x.ahi, x.bhi);
      std::swap(x.alo, x.blo);
    }
    x.Kpad = g->Kpad;
    x.out = raw + xo[q];
    G.src.push_back(x);
  }
  G.kind = kind;
  if (int e2 = grouped_table(c, 256, 0, &G.probs, &G.ntiles)) return e2;
  G.nprob = (int)plans.size();
  // contributions per stored block, in plan order
  const i64 V3 = c->V3;
  std::vector<std::vector<std::array<i64, 2>>> per(c->n3);  // (xoff, q * 64 + r-th) -> resolved below
  std::vector<std::vector<std::pair<int, float>>> meta(c->n3);
  for (size_t q = 0; q < plans.size(); ++q) {
    GemmPlan* g = plans[q];
    for (size_t r = 0; r < g->h_base.size(); ++r) {
      const i64 blk = g->h_base[r] / V3;
      per[blk].push_back({(i64)xo[q] + (i64)r * V3, 0});
      meta[blk].push_back({g->h_sel[r], (float)g->h_alpha[r]});
    }
  }
  std::vector<i64> target(c->n3), xoff;
  std::vector<int> cstart(c->n3 + 1, 0), csel;
  std::vector<float> calpha;
  for (i64 b = 0; b < c->n3; ++b) {
    target[b] = b * V3;
    cstart[b] = (int)xoff.size();
    for (size_t k = 0; k < per[b].size(); ++k) {
      xoff.push_back(per[b][k][0]);
      csel.push_back(meta[b][k].first);
      calpha.push_back(meta[b][k].second);
    }
  }
  cstart[c->n3] = (int)xoff.size();
  G.ntarget = (int)c->n3;
  G.target = upload_vec(c, target, &err);
  G.cstart = upload_vec(c, cstart, &err);
  G.xoff = upload_vec(c, xoff, &err);
  G.csel = upload_vec(c, csel, &err);
  G.calpha = upload_vec(c, calpha, &err);
  if (err) return fail(c, RCCSDT_ERR_OOM, "grouped residual: table upload failed");
  G.on = 1;
  return 0;
}

int check(rccsdt_ctx* c, const char* where);

// Autotuner of the grouped GEMM: times each candidate launch shape (tile width,
// problem order, persistent grid) on the panels of the current iteration and
// keeps the fastest.  The first candidate is the fixed shape (256-wide tiles,
// longest K first, one CTA per SM); its time is kept for comparison.
int autotune_grouped(rccsdt_ctx* c) {
  auto& G = c->gr;
  G.tuned = 1;
#ifdef RCC_HOSTSIM
  return 0;
#else
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  struct Cand {
    int bn, ord, grid;
  };
  const Cand cands[] = {{256, 0, 0}, {256, 1, 0}, {128, 0, 0}, {128, 1, 0}, {256, 0, sms / 2}, {128, 0, sms / 2}};
  int* flag = (int*)((double*)c->scalars->p + 1000);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(c, RCCSDT_ERR_CUDA, "autotune: event creation failed");
  double best = 1e300;
  Cand bc = cands[0];
  std::unique_ptr<DBuf> best_tab;
  int best_tiles = 0, st = 0;
  const int ncand = (int)(sizeof(cands) / sizeof(cands[0]));
  const int only = c->opt.autotune >= 2 ? c->opt.autotune - 2 : -1;  // a fixed candidate (testing)
  for (const Cand& k : cands) {
    if (only >= 0 && only < ncand && &k != &cands[only] && &k != &cands[0]) continue;
    std::unique_ptr<DBuf> tab;
    int nt = 0;
    if ((st = grouped_table(c, k.bn, k.ord, &tab, &nt))) break;
    const rcc::GProblem* P = (const rcc::GProblem*)tab->p;
    rcc::launch_gemm_tc_grouped(G.kind, P, G.nprob, nt, k.grid, k.bn, flag, c->opt.watchdog_cycles, c->stream);
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < 2; ++r)
      rcc::launch_gemm_tc_grouped(G.kind, P, G.nprob, nt, k.grid, k.bn, flag, c->opt.watchdog_cycles, c->stream);
    cudaEventRecord(e1, c->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = fail(c, RCCSDT_ERR_CUDA, "autotune: launch failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double t = ms / 2.0;
    if (&k == &cands[0]) G.fixed_ms = t;
    if (only >= 0 && only < ncand ? &k == &cands[only] : t < best) {
      best = t;
      bc = k;
      best_tab = std::move(tab);
      best_tiles = nt;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  G.probs = std::move(best_tab);
  G.ntiles = best_tiles;
  G.bn = bc.bn;
  G.ord = bc.ord;
  G.grid = bc.grid;
  G.tuned_ms = best;
  return check(c, "autotune");
#endif
}

// Operand gathers of the grouped residual.
int run_grouped_gathers(rccsdt_ctx* c) {
  auto& G = c->gr;
  for (int t = 0; t < 2; ++t)
    if (G.npack[t])
      rcc::launch_pack_grouped((const rcc::PackArgs*)G.packs[t]->p, (const int*)G.ptile[t]->p, G.npack[t], G.ntile[t],
                               t == 1, c->stream);
  for (int m = 0; m < 2; ++m)
    if (G.ncube[m])
      rcc::launch_cube_pack(m, G.kind, (const rcc::CubePiece*)G.cubes[m]->p, G.ncube[m],
                            (const rcc::CubeDst*)G.cube_dst->p, rcc::CubeDst{nullptr, nullptr, 0}, c->B("t3")->f(),
                            c->v, c->stream);
  return 0;
}

int run_grouped_gemm(rccsdt_ctx* c) {
  auto& G = c->gr;
  if (c->opt.autotune && !G.tuned) {
    const int st = autotune_grouped(c);
    if (st) return st;
  }
  int* flag = (int*)((double*)c->scalars->p + 1000);
  const int tidx = timer_begin(c, 16, G.flop);
  if (rcc::launch_gemm_tc_grouped(G.kind, (const rcc::GProblem*)G.probs->p, G.nprob, G.ntiles, G.grid, G.bn, flag,
                                  c->opt.watchdog_cycles, c->stream))
    return fail(c, RCCSDT_ERR_ARG, "grouped GEMM configuration unsupported");
  timer_end(c, tidx);
  return 0;
}

void run_grouped_reduce(rccsdt_ctx* c) {
  auto& G = c->gr;
  const float* X = (const float*)G.raw->p;
  if (c->opt.precision != RCCSDT_FP64)
    rcc::launch_r3_gather<float>(X, (const i64*)G.target->p, G.ntarget, (const int*)G.cstart->p,
                                 (const i64*)G.xoff->p, (const int*)G.csel->p, (const float*)G.calpha->p, c->v, 0,
                                 c->B("r3")->f(), c->stream);
}


}  // namespace

// ---------------------------------------------------------------------------
// Iteration steps
// ---------------------------------------------------------------------------
namespace {

struct StepTimer {
  rccsdt_ctx* c;
  int slot;
  int idx = -1;
  StepTimer(rccsdt_ctx* c_, int slot_) : c(c_), slot(slot_) { idx = timer_begin(c, slot); }
  ~StepTimer() { timer_end(c, idx); }
};

int check(rccsdt_ctx* c, const char* where) {
#ifndef RCC_HOSTSIM
  const cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return fail(c, RCCSDT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(ce));
#else
  (void)c; (void)where;
#endif
  return 0;
}

int zero(rccsdt_ctx* c, const char* name) { return dev_zero(c->B(name)->p, c->B(name)->bytes, c->stream); }

int do_intermediates(rccsdt_ctx* c) {
  StepTimer tm(c, 0);
  int st = 0;
  rcc::launch_combine(c->c_Lt_copy, c->stream);
  if ((st = run_plans(c, c->p_dress))) return st;
  for (const char* z : {"gamma", "J", "Y", "Kx"}) zero(c, z);
  // gamma, J, Y, Kx, then F and ft = F, then the two ft dressing plans
  for (int q = 0; q < 4; ++q)
    if ((st = run_gemm(c, c->p_fock[q]))) return st;
  run_combines(c, c->c_fock);
  for (size_t q = 4; q < c->p_fock.size(); ++q)
    if ((st = run_gemm(c, c->p_fock[q]))) return st;
  for (const char* s : {"oooo", "ooov", "oovo", "oovv", "ovov", "ovvo", "ovvv", "vovv", "vooo", "vvoo", "vvvo", "vvvv"})
    zero(c, s);
  if ((st = run_plans(c, c->p_eri))) return st;
  run_combines(c, c->c_helpers);
  run_combines(c, c->c_int_base);
  if ((st = run_plans(c, c->p_int))) return st;
  run_combines(c, c->c_int_after[0]);
  if ((st = run_plans(c, c->p_wbar))) return st;
  // step (iii): T3 -> R1, R2, W^{ab}_{dj}, W^{al}_{ij}, a3_Z values of z at a time
  zero(c, "dR1");
  zero(c, "dX2");
  const int o = c->o;
  const int t3f = c->opt.precision != RCCSDT_FP64;
  // split bodies gather the S panels from T3 directly (cube pieces, R1 partials);
  // FP64 bodies unpack each batch of S and run the generic gathers
  const bool direct = t3f && c->precision != RCCSDT_FP64 && c->a3_direct == (int)c->p_a3.size();
  if (direct)
    rcc::launch_convert<float, double>(c->B("oovv_f")->f(), c->D("oovv"), (i64)o * o * c->v * c->v, c->stream);
  const i64 slab = (i64)o * o * c->V3;  // S of one z
  for (int z0 = 0, bz = 0; z0 < o; z0 += c->a3_Z, ++bz) {
    const int Zb = std::min(c->a3_Z, o - z0);
    const i64* zb = (const i64*)c->a3_base->p + (size_t)z0 * o * o;
    const int* zp = (const int*)c->a3_pos->p + (size_t)z0 * o * o * 3;
    if (direct) {
      if ((st = run_plans(c, c->p_a3[bz]))) return st;
      rcc::launch_r1_cubes_reduce(c->B("r1_part")->f(), o * o, Zb, c->v, c->D("dR1") + (size_t)z0 * c->v, c->stream);
      continue;
    }
    if (t3f)
      rcc::launch_unpack_spin<float>(c->B("t3")->p, 1, Zb * o * o, zb, zp, c->v, c->B("Sz")->f(), c->stream);
    else
      rcc::launch_unpack_spin<double>(c->B("t3")->p, 0, Zb * o * o, zb, zp, c->v, c->D("Sz"), c->stream);
    if ((st = run_plans(c, c->p_a3[bz]))) return st;
    for (int z = z0; z < z0 + Zb; ++z) {
      if (t3f)
        rcc::launch_r1_t3<float>(c->B("Sz")->f() + (z - z0) * slab, c->D("oovv"), o, c->v,
                                 c->D("dR1") + (size_t)z * c->v, c->splitk->d(), (i64)(c->splitk->bytes / 8),
                                 c->stream);
      else
        rcc::launch_r1_t3<double>(c->D("Sz") + (z - z0) * slab, c->D("oovv"), o, c->v, c->D("dR1") + (size_t)z * c->v,
                                  c->splitk->d(), (i64)(c->splitk->bytes / 8), c->stream);
    }
  }
  c->have_int = 1;
  return check(c, "do_intermediates");
}

// Residuals R1, R2, R3.  part -1: all of it.  For a batch that runs the grouped
// GEMMs of all its instances in one launch, part 0 stops after the grouped operand
// gathers and part 1 starts with the reduction of the GEMM results into R3 (a
// context off the grouped path does everything in part 0).
int do_residual(rccsdt_ctx* c, int part = -1) {
  int st = 0;
  const bool grouped = c->gr.on && c->precision == c->opt.precision;
  if (part == 1 && !grouped) return 0;
  if (part != 1) {
  {
    StepTimer tm(c, 5);
    run_combines(c, c->c_r12_base);
    if ((st = run_plans(c, c->p_r12))) return st;
    run_combines(c, c->c_r2_sym);
    if (!grouped) zero(c, "r3");
    run_combines(c, c->c_wt);
  }
  if (grouped) {
    // pp-ladder, ring, hh-ladder and the T2 term with W^{ab}_{dj}: one grouped pass
    StepTimer tm(c, 1);
    if ((st = run_grouped_gathers(c))) return st;
    if (part == 0) return check(c, "do_residual");
    if ((st = run_grouped_gemm(c))) return st;
  } else {
    {
      StepTimer tm(c, 1);
      if ((st = c->pps.on ? run_pp_sym(c) : run_plans(c, c->p_pp))) return st;
    }
    {
      StepTimer tm(c, 2);
      if ((st = run_plans(c, c->p_ringab))) return st;
      if ((st = run_plans(c, c->p_ringc))) return st;
    }
    {
      StepTimer tm(c, 3);
      if ((st = run_plans(c, c->p_hh))) return st;
    }
  }
  }
  if (grouped) {
    StepTimer tm(c, 1);
    run_grouped_reduce(c);
  }
  {
    StepTimer tm(c, 4);
    if (!grouped && (st = run_plans(c, c->p_t2a))) return st;
    const int4* blk = (const int4*)c->blocks_info->p;
    if (c->opt.precision != RCCSDT_FP64) {
      rcc::launch_convert<float, double>(c->B("t2_f")->f(), c->D("t2"), (i64)c->o * c->o * c->v * c->v, c->stream);
      rcc::launch_convert<float, double>(c->B("Wvooo_f")->f(), c->D("Wvooo"), (i64)c->v * c->o * c->o * c->o,
                                         c->stream);
      rcc::launch_t2_outer<float>(c->B("r3")->f(), c->B("Wvooo_f")->f(), c->B("t2_f")->f(), blk, c->o, c->v, c->n3,
                                  c->stream);
    } else {
      rcc::launch_t2_outer<double>(c->D("r3"), c->D("Wvooo"), c->D("t2"), blk, c->o, c->v, c->n3, c->stream);
    }
  }
  c->have_res = 1;
  return check(c, "do_residual");
}

double* scal(rccsdt_ctx* c, int i) { return (double*)c->scalars->p + i; }
double* partials(rccsdt_ctx* c) { return (double*)c->partial->p; }

// scalars layout: [0..3] norms^2 (r1, r2, r3, total) [4] energy [16..16+M*M) DIIS B, [300..316) coef
constexpr int kB = 16, kCoef = 300;

int do_postprocess(rccsdt_ctx* c, double norms[4]) {
  StepTimer tm(c, 6);
  const int4* blk = (const int4*)c->blocks_info->p;
  const bool f = c->opt.precision != RCCSDT_FP64;
  // post-processing with |R3|^2 (block multiplicities) formed in the same pass
  double* pp = (double*)c->B("post_partial")->p;
  if (f)
    rcc::launch_post<float>(c->B("r3")->f(), c->B("rp3")->f(), blk, c->v, c->n3, c->blk_weight->d(), pp, scal(c, 2),
                            c->stream);
  else
    rcc::launch_post<double>(c->D("r3"), c->D("rp3"), blk, c->v, c->n3, c->blk_weight->d(), pp, scal(c, 2),
                             c->stream);

  rcc::launch_wdot<double>(c->D("r1"), c->D("r1"), (i64)c->o * c->v, 1, nullptr, partials(c), scal(c, 0), 1.0, 0,
                           c->stream);
  rcc::launch_wdot<double>(c->D("r2"), c->D("r2"), (i64)c->o * c->o * c->v * c->v, 1, nullptr, partials(c),
                           scal(c, 1), 1.0, 0, c->stream);
  if (norms) {
    double h[3];
    if (dev_copy(h, scal(c, 0), sizeof(h), c->stream) || dev_sync(c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
    norms[0] = sqrt(h[0]);
    norms[1] = sqrt(h[1]);
    norms[2] = sqrt(h[2]);
    norms[3] = sqrt(h[0] + h[1] + h[2]);
    for (int q = 0; q < 4; ++q)
      if (!std::isfinite(norms[q])) return fail(c, RCCSDT_ERR_NONFINITE, "non-finite residual norm");
  }
  return check(c, "do_postprocess");
}

// Segment views of history slot s: t1 | t2 | t3 (t3 of the storage type).
struct Seg {
  double* t1;
  double* t2;
  void* t3;
};
Seg slot(rccsdt_ctx* c, int q) {
  const int M = c->opt.diis_space;
  char* p = q < M ? (char*)c->hist_t->p + (i64)q * c->hist_stride : (char*)c->hist_e->p + (i64)(q - M) * c->hist_stride;
  Seg s;
  s.t1 = (double*)p;
  s.t2 = (double*)(p + c->seg1 * 8);
  s.t3 = p + (c->seg1 + c->seg2) * 8;
  return s;
}

int do_update(rccsdt_ctx* c) {
  StepTimer tm(c, 7);
  const int o = c->o, v = c->v;
  const bool f = c->opt.precision != RCCSDT_FP64;
  const int4* blk = (const int4*)c->blocks_info->p;
  const int M = c->opt.diis_space;
  const bool dt3 = c->opt.diis_t3 != 0;
  c->iter += 1;
  int* st = c->diis_st ? (int*)c->diis_st->p : nullptr;
  char* ht = c->hist_t ? (char*)c->hist_t->p : nullptr;
  char* he = c->hist_e ? (char*)c->hist_e->p : nullptr;
  const i64 S = c->hist_stride, off1 = 0, off2 = c->seg1 * 8, off3 = (c->seg1 + c->seg2) * 8;
  // the T3 part of the DIIS vectors: T3 itself, or its virtual subspace gathered into t3sub
  const bool sub = dt3 && M > 0 && c->ns < v;
  void* t3d = sub ? c->B("t3sub")->p : c->B("t3")->p;
  auto gather_sub = [&](int dir) {
    if (!sub) return;
    if (f) rcc::launch_subcube<float>(c->B("t3")->f(), (float*)t3d, c->n3, v, c->ns, dir, c->stream);
    else rcc::launch_subcube<double>(c->D("t3"), (double*)t3d, c->n3, v, c->ns, dir, c->stream);
  };
  if (M > 0) {
    // slot and counters on the device; the amplitudes before the step go to the error slot
    rcc::launch_diis_begin(st, M, c->opt.diis_start, c->stream);
    rcc::launch_slot_save<double>(he, S, off1, st, c->D("t1"), c->seg1, c->stream);
    rcc::launch_slot_save<double>(he, S, off2, st, c->D("t2"), c->seg2, c->stream);
    if (dt3) {
      gather_sub(0);
      if (f) rcc::launch_slot_save<float>(he, S, off3, st, (const float*)t3d, c->seg3, c->stream);
      else rcc::launch_slot_save<double>(he, S, off3, st, (const double*)t3d, c->seg3, c->stream);
    }
  }
  rcc::launch_update_t12(c->D("t1"), c->D("r1"), c->D("t2"), c->D("r2"), c->D("e"), o, v, 0.0, c->stream);
  if (f)
    rcc::launch_update_t3<float>(c->B("t3")->f(), c->B("rp3")->f(), c->D("e"), blk, o, v, c->n3, 0.0, c->stream);
  else
    rcc::launch_update_t3<double>(c->D("t3"), c->D("rp3"), c->D("e"), blk, o, v, c->n3, 0.0, c->stream);
  if (M <= 0) return check(c, "do_update");
  // error vector e = t_new - t_old and the new amplitudes into slot st[2]
  rcc::launch_slot_diff_store<double>(ht, he, S, off1, st, c->D("t1"), c->seg1, c->stream);
  rcc::launch_slot_diff_store<double>(ht, he, S, off2, st, c->D("t2"), c->seg2, c->stream);
  if (dt3) {
    gather_sub(0);
    if (f) rcc::launch_slot_diff_store<float>(ht, he, S, off3, st, (const float*)t3d, c->seg3, c->stream);
    else rcc::launch_slot_diff_store<double>(ht, he, S, off3, st, (const double*)t3d, c->seg3, c->stream);
  }
  c->diis_count += 1;
  // new row / column of B: <e_s, e_q> with the multiplicity weights on t3
  double* dp = (double*)c->diis_partial->p;
  const i64 G = (i64)M * rcc::kDotBlocks;
  rcc::launch_diis_dots<double>(he, S, off1, st, M, c->seg1, 1, nullptr, dp, c->stream);
  rcc::launch_diis_dots<double>(he, S, off2, st, M, c->seg2, 1, nullptr, dp + G, c->stream);
  if (dt3) {
    if (f)
      rcc::launch_diis_dots<float>(he, S, off3, st, M, c->seg3, c->seg3 / c->n3, c->blk_weight->d(), dp + 2 * G,
                                   c->stream);
    else
      rcc::launch_diis_dots<double>(he, S, off3, st, M, c->seg3, c->seg3 / c->n3, c->blk_weight->d(), dp + 2 * G,
                                    c->stream);
  }
  rcc::launch_diis_row(dp, dt3 ? 3 : 2, st, M, scal(c, kB), c->stream);
  // extrapolation (the kernels skip themselves before diis_start or with one entry)
  rcc::launch_diis_solve(scal(c, kB), st, M, scal(c, kCoef), c->stream);
  rcc::launch_diis_extrapolate<double>(c->D("t1"), slot(c, 0).t1, c->hist_stride / 8, c->seg1, scal(c, kCoef), st,
                                       c->stream);
  rcc::launch_diis_extrapolate<double>(c->D("t2"), slot(c, 0).t2, c->hist_stride / 8, c->seg2, scal(c, kCoef), st,
                                       c->stream);
  if (dt3) {
    if (f)
      rcc::launch_diis_extrapolate<float>((float*)t3d, (const float*)slot(c, 0).t3, c->hist_stride / 4, c->seg3,
                                          scal(c, kCoef), st, c->stream);
    else
      rcc::launch_diis_extrapolate<double>((double*)t3d, (const double*)slot(c, 0).t3, c->hist_stride / 8, c->seg3,
                                           scal(c, kCoef), st, c->stream);
    // the subspace back into T3 (without extrapolation t3sub holds T3's own values)
    gather_sub(1);
  }
  return check(c, "do_update");
}

int do_energy(rccsdt_ctx* c, double* e_out) {
  StepTimer tm(c, 8);
  rcc::launch_energy(c->D("ovov_bare"), c->D("t1"), c->D("t2"), c->o, c->v, partials(c), scal(c, 4), c->stream);
  if (e_out) {
    if (dev_copy(e_out, scal(c, 4), 8, c->stream) || dev_sync(c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
    if (!std::isfinite(*e_out)) return fail(c, RCCSDT_ERR_NONFINITE, "non-finite energy");
  }
  return check(c, "do_energy");
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
#define RCC_API extern "C" __attribute__((visibility("default")))

RCC_API int rccsdt_options_default(rccsdt_options* opt) {
  if (!opt) return RCCSDT_ERR_ARG;
  memset(opt, 0, sizeof(*opt));
  opt->precision = RCCSDT_FP64;
  opt->diis_space = 8;
  opt->diis_start = 2;
  opt->diis_t3 = 1;
  opt->max_iter = 100;
  opt->tol = 1e-8;
  opt->watchdog_cycles = 0;
  opt->grouped_bytes = 8LL << 30;
  opt->unpack_bytes = 1LL << 30;
  opt->autotune = 0;
  opt->f64_tc = 0;
  opt->pp_unit_bytes = 0;
  opt->diis_t3_nvir = 0;
  return RCCSDT_OK;
}

RCC_API int rccsdt_create(int o, int v, int naux, const rccsdt_options* opt, void* stream, rccsdt_ctx** out) {
  if (!out) return RCCSDT_ERR_ARG;
  *out = nullptr;
  if (o < 1 || v < 1 || naux < 1 || o > 64 || v > 1024) return RCCSDT_ERR_ARG;
  rccsdt_options def;
  rccsdt_options_default(&def);
  const rccsdt_options& op = opt ? *opt : def;
  if (op.precision < 0 || op.precision > 2 || op.diis_space < 0 || op.diis_space > 16 || op.f64_tc < 0 ||
      op.f64_tc > 2 || op.watchdog_cycles < 0)
    return RCCSDT_ERR_ARG;
  auto* c = new rccsdt_ctx();
  c->o = o; c->v = v; c->n = o + v; c->naux = naux;
  c->n3 = n3_of(o);
  c->V3 = (i64)v * v * v;
  c->opt = op;
  // device-side wait budget: 0 selects the default; very small values are raised
  c->opt.watchdog_cycles = op.watchdog_cycles == 0 ? kDefaultWatchdog : std::max(op.watchdog_cycles, kMinWatchdog);
  c->precision = op.precision;
  c->stream = (cudaStream_t)stream;
  int err = 0;
  c->scalars = upload_vec(c, std::vector<double>(2048, 0.0), &err);
  c->partial = upload_vec(c, std::vector<double>(rcc::kDotBlocks, 0.0), &err);
  c->splitk = std::make_unique<DBuf>();
  c->splitk->bytes = (size_t)32 << 20;  // split-K partial tiles (4 Mi doubles)
  c->splitk->p = dev_alloc(c->splitk->bytes, &err);
  c->total_bytes += c->splitk->bytes;
  int st = err ? RCCSDT_ERR_OOM : build_context(c);
  if (!st) {
    // engine panels (hi planes hold doubles in FP64 mode; lo planes only for split modes)
    c->panelA_hi = std::make_unique<DBuf>();
    c->panelB_hi = std::make_unique<DBuf>();
    c->panelA_hi->p = dev_alloc(c->panel_bytes, &err);
    c->panelB_hi->p = dev_alloc(c->panel_bytes, &err);
    if (op.f64_tc) {  // digit planes (kSlices BF16 per FP64 panel element) and row exponents
      const size_t pb = c->panel_bytes / 8 * rcc::kSlices * 2;
      for (auto* q : {&c->planesA, &c->planesB}) {
        *q = std::make_unique<DBuf>();
        (*q)->p = dev_alloc(pb, &err);
        (*q)->bytes = pb;
        c->total_bytes += pb;
      }
      for (auto* q : {&c->expA, &c->expB}) {
        *q = std::make_unique<DBuf>();
        (*q)->p = dev_alloc((size_t)c->panel_rows * 4 + 16, &err);
        (*q)->bytes = (size_t)c->panel_rows * 4 + 16;
      }
    }
    c->total_bytes += 2 * c->panel_bytes;
    if (op.precision != RCCSDT_FP64) {
      c->panelA_lo = std::make_unique<DBuf>();
      c->panelB_lo = std::make_unique<DBuf>();
      c->panelA_lo->p = dev_alloc(c->panel_bytes / 2, &err);
      c->panelB_lo->p = dev_alloc(c->panel_bytes / 2, &err);
      c->total_bytes += c->panel_bytes;
    }
    // dense FP32 result of the hh-ladder GEMM for its two-phase scatter (split modes)
    if (op.precision != RCCSDT_FP64) {
      c->rawX = std::make_unique<DBuf>();
      size_t mx = 0;
      for (auto& g : c->plans)
        if (g->s3_rows > 0) mx = std::max(mx, (size_t)g->E.e.M * g->E.e.N);
      c->rawX->bytes = mx * 4;
      c->rawX->p = dev_alloc(c->rawX->bytes, &err);
      c->total_bytes += c->rawX->bytes;
    }
    // DIIS history
    c->seg1 = (i64)o * v;
    c->seg2 = (i64)o * o * v * v;
    // the T3 part of the DIIS vectors: all of T3, or its first ns virtual orbitals
    c->ns = (op.diis_t3_nvir > 0 && op.diis_t3_nvir < v) ? op.diis_t3_nvir : v;
    const i64 S3 = (i64)c->ns * c->ns * c->ns;
    c->seg3 = op.diis_t3 ? c->n3 * S3 : 0;
    if (op.diis_t3 && op.diis_space > 0 && c->ns < v) {
      const i64 t3b = op.precision != RCCSDT_FP64 ? 4 : 8;
      alloc_buf(c, "t3sub", (size_t)(c->n3 * S3 * t3b), &err);
    }
    const i64 t3e = op.precision != RCCSDT_FP64 ? 4 : 8;
    c->hist_stride = ((c->seg1 + c->seg2) * 8 + c->seg3 * t3e + 15) / 16 * 16;
    if (op.diis_space > 0) {
      c->hist_t = std::make_unique<DBuf>();
      c->hist_e = std::make_unique<DBuf>();
      c->hist_t->p = dev_alloc((size_t)c->hist_stride * op.diis_space, &err);
      c->hist_e->p = dev_alloc((size_t)c->hist_stride * op.diis_space, &err);
      c->total_bytes += 2 * (size_t)c->hist_stride * op.diis_space;
      c->diis_st = upload_vec(c, std::vector<int>(8, 0), &err);
      c->diis_partial = upload_vec(c, std::vector<double>((size_t)3 * op.diis_space * rcc::kDotBlocks, 0.0), &err);
    }
    if (err) st = fail(c, RCCSDT_ERR_OOM, "device allocation failed");
  }
  if (!st) st = build_grouped(c);
  if (st) {
    delete c;
    return st;
  }
  *out = c;
  return RCCSDT_OK;
}

RCC_API long long rccsdt_device_bytes(const rccsdt_ctx* c) { return c ? (long long)c->total_bytes : 0; }

RCC_API int rccsdt_set_hamiltonian(rccsdt_ctx* c, const double* fock_diag, const double* L) {
  if (!c || !fock_diag || !L) return fail(c, RCCSDT_ERR_ARG, "null argument");
  if (dev_copy(c->D("e"), fock_diag, (size_t)c->n * 8, c->stream) ||
      dev_copy(c->D("L"), L, (size_t)c->naux * c->n * c->n * 8, c->stream))
    return fail(c, RCCSDT_ERR_CUDA, "copy failed");
  dev_zero(c->B("ovov_bare")->p, c->B("ovov_bare")->bytes, c->stream);
  int st = run_plans(c, c->p_energy_bare);
  if (st) return st;
  if (dev_sync(c->stream)) return fail(c, RCCSDT_ERR_CUDA, "set_hamiltonian failed");
  c->have_ham = 1;
  c->have_int = c->have_res = 0;
  return RCCSDT_OK;
}

// RCCSDT_ERR_TIMEOUT once a tensor-core GEMM of this context has given up a wait (the
// kernels set the flag; it stays set until new amplitudes are given).  Synchronises.
static int watchdog_status(rccsdt_ctx* c) {
  int flag = 0;
  if (dev_copy(&flag, (double*)c->scalars->p + 1000, sizeof(int), c->stream) || dev_sync(c->stream))
    return fail(c, RCCSDT_ERR_CUDA, "status read failed");
  return flag ? fail(c, RCCSDT_ERR_TIMEOUT, "a device-side wait exceeded its watchdog budget") : 0;
}

static int clear_watchdog(rccsdt_ctx* c) { return dev_zero((double*)c->scalars->p + 1000, sizeof(double), c->stream); }

static void reset_diis(rccsdt_ctx* c) {
  c->diis_count = 0;
  c->iter = 0;
  if (c->diis_st) dev_zero(c->diis_st->p, c->diis_st->bytes, c->stream);
}

// Device address of caller memory that kernels can access in place: device memory,
// or pinned / registered host memory mapped into the device's address space (read
// over the host link by the conversion kernel itself, without a staging copy).
// nullptr for pageable host memory.
static const void* device_view(const void* p) {
#ifndef RCC_HOSTSIM
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if ((at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeManaged) &&
      at.devicePointer)
    return at.devicePointer;
#else
  (void)p;
#endif
  return nullptr;
}

RCC_API int rccsdt_set_amplitudes(rccsdt_ctx* c, const double* t1, const double* t2, const double* t3c) {
  if (!c) return RCCSDT_ERR_ARG;
  const bool f = c->opt.precision != RCCSDT_FP64;
  if (t1 && dev_copy(c->D("t1"), t1, (size_t)c->seg1 * 8, c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
  if (t2 && dev_copy(c->D("t2"), t2, (size_t)c->o * c->o * c->v * c->v * 8, c->stream))
    return fail(c, RCCSDT_ERR_CUDA, "copy");
  if (t3c) {
    const i64 cnt = c->n3 * c->V3;
    if (!f) {
      if (dev_copy(c->D("t3"), t3c, (size_t)cnt * 8, c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
    } else if (const double* dv = (const double*)device_view(t3c)) {
      // device or mapped pinned host memory: one conversion pass reads it in place
      rcc::launch_convert<float, double>(c->B("t3")->f(), dv, cnt, c->stream);
    } else {
      // pageable host memory: stage the FP64 values in rp3's storage (chunked) and convert
      const i64 chunk = c->B("rp3")->bytes / 8;
      for (i64 off = 0; off < cnt; off += chunk) {
        const i64 len = std::min(chunk, cnt - off);
        if (dev_copy(c->B("rp3")->p, t3c + off, (size_t)len * 8, c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
        rcc::launch_convert<float, double>(c->B("t3")->f() + off, (const double*)c->B("rp3")->p, len, c->stream);
        if (dev_sync(c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
      }
    }
  }
  clear_watchdog(c);
  if (dev_sync(c->stream)) return fail(c, RCCSDT_ERR_CUDA, "set_amplitudes failed");
  c->have_amp = 1;
  c->have_int = c->have_res = 0;
  reset_diis(c);
  return RCCSDT_OK;
}

RCC_API int rccsdt_set_amplitudes_t3f32(rccsdt_ctx* c, const double* t1, const double* t2, const float* t3c) {
  if (!c) return RCCSDT_ERR_ARG;
  if (c->opt.precision == RCCSDT_FP64) return fail(c, RCCSDT_ERR_ARG, "FP32 T3 exchange needs a split-precision context");
  if (t3c) {
    const i64 cnt = c->n3 * c->V3;
    if (const float* dv = (const float*)device_view(t3c))
      rcc::launch_convert<float, float>(c->B("t3")->f(), dv, cnt, c->stream);  // in place (SM loads over the link)
    else if (dev_copy(c->B("t3")->p, t3c, (size_t)cnt * 4, c->stream))
      return fail(c, RCCSDT_ERR_CUDA, "copy");
  }
  return rccsdt_set_amplitudes(c, t1, t2, nullptr);  // stream order; synchronises, resets DIIS
}

RCC_API int rccsdt_init_mp2(rccsdt_ctx* c) {
  if (!c) return RCCSDT_ERR_ARG;
  if (!c->have_ham) return fail(c, RCCSDT_ERR_STATE, "hamiltonian not set");
  zero(c, "t1");
  zero(c, "t3");
  rcc::launch_mp2(c->D("t2"), c->D("ovov_bare"), c->D("e"), c->o, c->v, c->stream);
  clear_watchdog(c);
  if (dev_sync(c->stream) || dev_check()) return fail(c, RCCSDT_ERR_CUDA, "init_mp2 failed");
  c->have_amp = 1;
  c->have_int = c->have_res = 0;
  reset_diis(c);
  return RCCSDT_OK;
}

RCC_API int rccsdt_set_precision(rccsdt_ctx* c, int precision) {
  if (!c || precision < 0 || precision > 2) return fail(c, RCCSDT_ERR_ARG, "bad precision");
  if ((precision != RCCSDT_FP64) != (c->opt.precision != RCCSDT_FP64) && precision != RCCSDT_FP64)
    return fail(c, RCCSDT_ERR_ARG, "a context created in FP64 mode has no split-precision panels");
  c->precision = precision;
  return RCCSDT_OK;
}

static int need(rccsdt_ctx* c, bool amp, bool inter, bool res) {
  if (!c) return RCCSDT_ERR_ARG;
  if (!c->have_ham) return fail(c, RCCSDT_ERR_STATE, "hamiltonian not set");
  if (amp && !c->have_amp) return fail(c, RCCSDT_ERR_STATE, "amplitudes not set");
  if (inter && !c->have_int) return fail(c, RCCSDT_ERR_STATE, "intermediates not built");
  if (res && !c->have_res) return fail(c, RCCSDT_ERR_STATE, "residual not computed");
  return 0;
}

RCC_API int rccsdt_build_intermediates(rccsdt_ctx* c) {
  int st = need(c, true, false, false);
  if (st) return st;
  st = do_intermediates(c);
  if (!st && dev_sync(c->stream)) st = fail(c, RCCSDT_ERR_CUDA, "intermediates failed");
  return st ? st : watchdog_status(c);
}

RCC_API int rccsdt_residual(rccsdt_ctx* c) {
  int st = need(c, true, true, false);
  if (st) return st;
  st = do_residual(c);
  if (!st && dev_sync(c->stream)) st = fail(c, RCCSDT_ERR_CUDA, "residual failed");
  return st ? st : watchdog_status(c);
}

RCC_API int rccsdt_postprocess(rccsdt_ctx* c, double norms[4]) {
  int st = need(c, true, true, true);
  if (st) return st;
  return do_postprocess(c, norms);
}

RCC_API int rccsdt_update(rccsdt_ctx* c) {
  int st = need(c, true, true, true);
  if (st) return st;
  st = do_update(c);
  c->have_int = c->have_res = 0;
  return st ? st : (dev_sync(c->stream) ? fail(c, RCCSDT_ERR_CUDA, "update failed") : 0);
}

RCC_API int rccsdt_energy(rccsdt_ctx* c, double* e) {
  int st = need(c, true, false, false);
  if (st) return st;
  double tmp;
  return do_energy(c, e ? e : &tmp);
}

RCC_API int rccsdt_iterate(rccsdt_ctx* c, double* e, double norms[4]) {
  int st = need(c, true, false, false);
  if (st) return st;
  double tmp[4], et;
  if ((st = do_energy(c, nullptr))) return st;
  if ((st = do_intermediates(c))) return st;
  if ((st = do_residual(c))) return st;
  if ((st = do_postprocess(c, norms ? norms : tmp))) return st;
  if ((st = do_update(c))) return st;
  c->have_int = c->have_res = 0;
  if (dev_copy(&et, scal(c, 4), 8, c->stream) || dev_sync(c->stream)) return fail(c, RCCSDT_ERR_CUDA, "iterate");
  if ((st = watchdog_status(c))) return st;
  if (!std::isfinite(et)) return fail(c, RCCSDT_ERR_NONFINITE, "non-finite energy");
  if (e) *e = et;
  return RCCSDT_OK;
}

RCC_API int rccsdt_solve(rccsdt_ctx* c, double* e_corr, int* iterations, double* final_norm) {
  int st = need(c, true, false, false);
  if (st) return st;
  rcc::SolveState S;
  for (;;) {
    const int code = rcc::next_code(c->opt, S);
    if (code >= rcc::kSkip) break;
    if ((st = rcc::ctx_enqueue_code(c, code))) return st;
    double out[6];
    if ((st = rcc::ctx_read_scalars(c, out))) return st;
    rcc::take_result(c->opt, S, code, out);
  }
  c->have_int = c->have_res = 0;
  if (iterations) *iterations = S.it;
  if (final_norm) *final_norm = S.norm;
  if (e_corr) *e_corr = S.e;
  if (S.status == RCCSDT_ERR_TIMEOUT) return fail(c, S.status, "a device-side wait exceeded its watchdog budget");
  if (S.status == RCCSDT_ERR_NONFINITE) return fail(c, S.status, "non-finite residual norm or energy");
  return S.status;
}

RCC_API int rccsdt_get_amplitudes(rccsdt_ctx* c, double* t1, double* t2, double* t3c) {
  if (!c) return RCCSDT_ERR_ARG;
  const bool f = c->opt.precision != RCCSDT_FP64;
  if (t1 && dev_copy(t1, c->D("t1"), (size_t)c->seg1 * 8, c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
  if (t2 && dev_copy(t2, c->D("t2"), (size_t)c->o * c->o * c->v * c->v * 8, c->stream))
    return fail(c, RCCSDT_ERR_CUDA, "copy");
  if (t3c) {
    const i64 cnt = c->n3 * c->V3;
    if (!f) {
      if (dev_copy(t3c, c->D("t3"), (size_t)cnt * 8, c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
    } else if (double* dv = (double*)device_view(t3c)) {
      // device or mapped pinned host memory: the conversion writes it in place
      rcc::launch_convert<double, float>(dv, c->B("t3")->f(), cnt, c->stream);
    } else {
      const i64 chunk = c->B("Sz")->bytes / 8;
      double* stage = (double*)c->B("Sz")->p;  // FP64 staging through the unpack scratch
      for (i64 off = 0; off < cnt; off += chunk) {
        const i64 len = std::min(chunk, cnt - off);
        rcc::launch_convert<double, float>(stage, c->B("t3")->f() + off, len, c->stream);
        if (dev_copy(t3c + off, stage, (size_t)len * 8, c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
        if (dev_sync(c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
      }
    }
  }
  return dev_sync(c->stream) ? fail(c, RCCSDT_ERR_CUDA, "get_amplitudes failed") : 0;
}

RCC_API int rccsdt_get_amplitudes_t3f32(rccsdt_ctx* c, double* t1, double* t2, float* t3c) {
  if (!c) return RCCSDT_ERR_ARG;
  if (c->opt.precision == RCCSDT_FP64) return fail(c, RCCSDT_ERR_ARG, "FP32 T3 exchange needs a split-precision context");
  if (t3c) {
    const i64 cnt = c->n3 * c->V3;
    if (float* dv = (float*)device_view(t3c))
      rcc::launch_convert<float, float>(dv, c->B("t3")->f(), cnt, c->stream);  // in place (SM stores over the link)
    else if (dev_copy(t3c, c->B("t3")->p, (size_t)cnt * 4, c->stream))
      return fail(c, RCCSDT_ERR_CUDA, "copy");
  }
  return rccsdt_get_amplitudes(c, t1, t2, nullptr);  // stream order; synchronises
}

// ---------------------------------------------------------------------------
// Checkpoint: the iteration state (amplitudes in their storage type, the DIIS
// history, its device counters and B matrix, the host counters) as a raw
// little-endian file, so that an iteration resumed in a new context with the same
// Hamiltonian and options repeats the one the saved context would take next.
// ---------------------------------------------------------------------------
namespace {

constexpr char kCkMagic[8] = {'R', 'C', 'C', 'S', 'D', 'T', 'c', 'k'};
constexpr int kCkVersion = 1;

struct CkHeader {
  char magic[8];
  int32_t version, o, v, t3_bytes, diis_space, diis_t3, precision, pad;
  int64_t iter, diis_count, hist_stride, seg1, seg2, seg3;
};

struct CkRegion {
  void* dev;
  size_t bytes;
};

// The device regions of the state, in file order.
std::vector<CkRegion> ck_regions(rccsdt_ctx* c) {
  const bool f = c->opt.precision != RCCSDT_FP64;
  std::vector<CkRegion> r;
  r.push_back({c->D("t1"), (size_t)c->seg1 * 8});
  r.push_back({c->D("t2"), (size_t)c->seg2 * 8});
  r.push_back({c->B("t3")->p, (size_t)(c->n3 * c->V3) * (f ? 4 : 8)});
  const int M = c->opt.diis_space;
  if (M > 0) {
    r.push_back({c->diis_st->p, 8 * sizeof(int)});
    r.push_back({scal(c, kB), (size_t)M * M * 8});
    r.push_back({c->hist_t->p, (size_t)c->hist_stride * M});
    r.push_back({c->hist_e->p, (size_t)c->hist_stride * M});
  }
  return r;
}

CkHeader ck_header(rccsdt_ctx* c) {
  CkHeader h{};
  memcpy(h.magic, kCkMagic, 8);
  h.version = kCkVersion;
  h.o = c->o;
  h.v = c->v;
  h.t3_bytes = c->opt.precision != RCCSDT_FP64 ? 4 : 8;
  h.diis_space = c->opt.diis_space;
  h.diis_t3 = c->opt.diis_t3;
  h.precision = c->precision;
  h.iter = c->iter;
  h.diis_count = c->diis_count;
  h.hist_stride = c->hist_stride;
  h.seg1 = c->seg1;
  h.seg2 = c->seg2;
  h.seg3 = c->seg3;
  return h;
}

constexpr size_t kCkChunk = (size_t)64 << 20;  // host staging per copy

}  // namespace

RCC_API int rccsdt_save(rccsdt_ctx* c, const char* path) {
  if (!c) return RCCSDT_ERR_ARG;
  if (!path) return fail(c, RCCSDT_ERR_ARG, "null path");
  if (!c->have_amp) return fail(c, RCCSDT_ERR_STATE, "no amplitudes to save");
  if (dev_sync(c->stream)) return fail(c, RCCSDT_ERR_CUDA, "save: pending work failed");
  FILE* fp = fopen(path, "wb");
  if (!fp) return fail(c, RCCSDT_ERR_ARG, std::string("cannot open ") + path + " for writing");
  const CkHeader h = ck_header(c);
  bool ok = fwrite(&h, sizeof(h), 1, fp) == 1;
  std::vector<char> buf;
  for (const CkRegion& r : ck_regions(c)) {
    for (size_t off = 0; ok && off < r.bytes; off += kCkChunk) {
      const size_t len = std::min(kCkChunk, r.bytes - off);
      buf.resize(len);
      if (dev_copy(buf.data(), (const char*)r.dev + off, len, c->stream) || dev_sync(c->stream)) {
        fclose(fp);
        return fail(c, RCCSDT_ERR_CUDA, "save: copy failed");
      }
      ok = fwrite(buf.data(), 1, len, fp) == len;
    }
  }
  if (fclose(fp) != 0) ok = false;
  return ok ? RCCSDT_OK : fail(c, RCCSDT_ERR_ARG, std::string("write to ") + path + " failed");
}

RCC_API int rccsdt_load(rccsdt_ctx* c, const char* path) {
  if (!c) return RCCSDT_ERR_ARG;
  if (!path) return fail(c, RCCSDT_ERR_ARG, "null path");
  FILE* fp = fopen(path, "rb");
  if (!fp) return fail(c, RCCSDT_ERR_ARG, std::string("cannot open ") + path);
  CkHeader h{};
  const CkHeader want = ck_header(c);
  if (fread(&h, sizeof(h), 1, fp) != 1 || memcmp(h.magic, kCkMagic, 8) != 0 || h.version != kCkVersion) {
    fclose(fp);
    return fail(c, RCCSDT_ERR_ARG, "not an RCCSDT checkpoint");
  }
  if (h.o != want.o || h.v != want.v || h.t3_bytes != want.t3_bytes || h.diis_space != want.diis_space ||
      h.diis_t3 != want.diis_t3 || h.hist_stride != want.hist_stride || h.seg1 != want.seg1 ||
      h.seg2 != want.seg2 || h.seg3 != want.seg3) {
    fclose(fp);
    return fail(c, RCCSDT_ERR_ARG, "checkpoint does not match this context (sizes, storage or DIIS options)");
  }
  if (h.precision != c->opt.precision && (c->opt.precision == RCCSDT_FP64 || h.precision < 0 || h.precision > 2)) {
    fclose(fp);
    return fail(c, RCCSDT_ERR_ARG, "checkpoint precision not accepted by this context");
  }
  std::vector<char> buf;
  for (const CkRegion& r : ck_regions(c)) {
    for (size_t off = 0; off < r.bytes; off += kCkChunk) {
      const size_t len = std::min(kCkChunk, r.bytes - off);
      buf.resize(len);
      if (fread(buf.data(), 1, len, fp) != len) {
        fclose(fp);
        return fail(c, RCCSDT_ERR_ARG, "checkpoint truncated");
      }
      if (dev_copy((char*)r.dev + off, buf.data(), len, c->stream) || dev_sync(c->stream)) {
        fclose(fp);
        return fail(c, RCCSDT_ERR_CUDA, "load: copy failed");
      }
    }
  }
  fclose(fp);
  c->precision = h.precision;
  c->iter = (int)h.iter;
  c->diis_count = (int)h.diis_count;
  c->have_amp = 1;
  c->have_int = c->have_res = 0;
  return RCCSDT_OK;
}

RCC_API int rccsdt_get_residuals(rccsdt_ctx* c, double* r1, double* r2, double* r3c) {
  if (!c) return RCCSDT_ERR_ARG;
  const bool f = c->opt.precision != RCCSDT_FP64;
  if (r1 && dev_copy(r1, c->D("r1"), (size_t)c->seg1 * 8, c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
  if (r2 && dev_copy(r2, c->D("r2"), (size_t)c->o * c->o * c->v * c->v * 8, c->stream))
    return fail(c, RCCSDT_ERR_CUDA, "copy");
  if (r3c) {
    const i64 cnt = c->n3 * c->V3;
    if (!f) {
      if (dev_copy(r3c, c->D("r3"), (size_t)cnt * 8, c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
    } else if (double* dv = (double*)device_view(r3c)) {
      rcc::launch_convert<double, float>(dv, c->B("r3")->f(), cnt, c->stream);  // converted in place
    } else {
      const i64 chunk = c->B("Sz")->bytes / 8;
      double* stage = (double*)c->B("Sz")->p;
      for (i64 off = 0; off < cnt; off += chunk) {
        const i64 len = std::min(chunk, cnt - off);
        rcc::launch_convert<double, float>(stage, c->B("r3")->f() + off, len, c->stream);
        if (dev_copy(r3c + off, stage, (size_t)len * 8, c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
        if (dev_sync(c->stream)) return fail(c, RCCSDT_ERR_CUDA, "copy");
      }
    }
  }
  return dev_sync(c->stream) ? fail(c, RCCSDT_ERR_CUDA, "get_residuals failed") : 0;
}

RCC_API int rccsdt_debug_copy(rccsdt_ctx* c, const char* name, double* out, long long count) {
  if (!c || !name || !out) return RCCSDT_ERR_ARG;
  auto it = c->buf.find(name);
  if (it == c->buf.end()) return fail(c, RCCSDT_ERR_ARG, std::string("no tensor ") + name);
  if (count < 0 || (size_t)count * 8 > it->second->bytes) return fail(c, RCCSDT_ERR_ARG, "count too large");
  if (std::string(name) == "Wvvvo") {
    // stored [j][a][b][d]; returned in the symbol's order [a][b][d][j]
    const i64 o = c->o, V3 = c->V3;
    std::vector<double> h((size_t)(o * V3));
    if (dev_copy(h.data(), it->second->p, h.size() * 8, c->stream) || dev_sync(c->stream))
      return fail(c, RCCSDT_ERR_CUDA, "copy");
    for (i64 x = 0; x < count; ++x) {
      const i64 j = x % o, abd = x / o;
      out[x] = h[(size_t)(j * V3 + abd)];  // a V^2 + b v + d = abd
    }
    return RCCSDT_OK;
  }
  if (dev_copy(out, it->second->p, (size_t)count * 8, c->stream) || dev_sync(c->stream))
    return fail(c, RCCSDT_ERR_CUDA, "copy");
  return RCCSDT_OK;
}

RCC_API double rccsdt_iteration_fma(int o, int v) {
  const double n3 = (double)o * (o + 1) * (o + 2) / 6.0, V = v;
  return n3 * (3.0 * V * V * V * V * V + 12.0 * o * V * V * V * V + 3.0 * (double)o * o * V * V * V);
}

RCC_API int rccsdt_enable_timing(rccsdt_ctx* c, int on) {
  if (!c) return RCCSDT_ERR_ARG;
  c->timing = on ? 1 : 0;
  c->ev_used = 0;  // starts a new measurement window
  return RCCSDT_OK;
}

RCC_API int rccsdt_step_times(rccsdt_ctx* c, double* ms, int cap) {
  if (!c || !ms) return RCCSDT_ERR_ARG;
  double all[17], gl, gf;
  timer_collect(c, all, &gl, &gf);
  const int n = std::min(cap, 12);
  for (int q = 0; q < n; ++q) {
    if (q < 9) ms[q] = all[q];
    else if (q == 9) ms[q] = all[16];
    else if (q == 10) ms[q] = gl;
    else ms[q] = gf;
  }
  return n;
}

RCC_API long long rccsdt_kernel_launches(void) { return rcc::g_launch_count; }

RCC_API int rccsdt_engine_info(const rccsdt_ctx* c, long long* out, int cap) {
  if (!c || !out) return RCCSDT_ERR_ARG;
  const auto& G = c->gr;
  const long long v[13] = {G.on, G.nprob, G.ntiles, (long long)G.npack[0] + G.npack[1],
                           G.on ? (long long)(G.xoff ? G.xoff->bytes / 8 : 0) : 0, (long long)(G.on ? G.bytes : 0),
                           G.grid, G.kind, G.bn, G.ord, G.tuned, (long long)(G.tuned_ms * 1e3),
                           (long long)(G.fixed_ms * 1e3)};
  const int k = cap < 13 ? cap : 13;
  for (int q = 0; q < k; ++q) out[q] = v[q];
  return k;
}

RCC_API const char* rccsdt_last_error(const rccsdt_ctx* c) { return c ? c->err.c_str() : "null context"; }

RCC_API void rccsdt_destroy(rccsdt_ctx* c) {
  if (!c) return;
  dev_sync(c->stream);
#ifndef RCC_HOSTSIM
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
#endif
  delete c;
}

// ---------------------------------------------------------------------------
// Internal entry points for the batched driver (batch.cu); not part of the ABI.
// ---------------------------------------------------------------------------
namespace rcc {

int ctx_enqueue(rccsdt_ctx* c, int update_first, int precision) {
  c->precision = precision;
  int st = 0;
  if (update_first && (st = do_update(c))) return st;
  if ((st = do_energy(c, nullptr))) return st;
  if ((st = do_intermediates(c))) return st;
  if ((st = do_residual(c))) return st;
  return do_postprocess(c, nullptr);
}

int ctx_body_grouped(const rccsdt_ctx* c, int code) {
  return c->gr.on && body_precision(c->opt, code) == c->opt.precision ? 1 : 0;
}

int ctx_enqueue_part(rccsdt_ctx* c, int code, int part) {
  if (code < 0 || code >= kBodies) return fail(c, RCCSDT_ERR_ARG, "internal: unknown body");
  const int precision = body_precision(c->opt, code);
  const bool split = ctx_body_grouped(c, code) != 0;
  c->precision = precision;
  int st = 0;
  if (part == 0) {
    if (rcc::body_updates(code) && (st = do_update(c))) return st;
    if ((st = do_energy(c, nullptr))) return st;
    if ((st = do_intermediates(c))) return st;
    if ((st = do_residual(c, split ? 0 : -1))) return st;
    if (!split && (st = do_postprocess(c, nullptr))) return st;
  } else if (split) {
    if ((st = do_residual(c, 1))) return st;
    if ((st = do_postprocess(c, nullptr))) return st;
  }
  c->precision = c->opt.precision;
  return check(c, "ctx_enqueue_part");
}

int ctx_grouped_problems(rccsdt_ctx* c, int bn, std::vector<GProblem>* out) {
  auto& G = c->gr;
  out->clear();
  for (const auto& x : G.src) {
    GProblem P;
    if (make_gproblem(&P, G.kind, x.ahi, x.alo, x.bhi, x.blo, x.M, x.N, x.Kpad, x.out, bn))
      return fail(c, RCCSDT_ERR_CUDA, "grouped residual: tensor map encoding failed");
    P.colmajor = x.colmajor;
    out->push_back(P);
  }
  return 0;
}
int ctx_grouped_kind(const rccsdt_ctx* c) { return c->gr.on ? c->gr.kind : -1; }
void ctx_set_batch_gemm(rccsdt_ctx* c, int on) { c->batch_gemm = on; }
int ctx_run_grouped_gemm(rccsdt_ctx* c) { return run_grouped_gemm(c); }

// Queues one body of the solver (solve_sm.h) without host synchronisation.
int ctx_enqueue_code(rccsdt_ctx* c, int code) {
  if (code < 0 || code >= kBodies) return fail(c, RCCSDT_ERR_ARG, "internal: unknown body");
  const int st = ctx_enqueue(c, rcc::body_updates(code), body_precision(c->opt, code));
  c->precision = c->opt.precision;
  return st ? st : check(c, "ctx_enqueue_code");
}

// Device scalars of the last evaluation into out[0..5] (host), synchronising.
int ctx_read_scalars(rccsdt_ctx* c, double* out) {
  double h[6];
  if (dev_copy(h, c->scalars->p, 5 * sizeof(double), c->stream) ||
      dev_copy(&h[5], (double*)c->scalars->p + 1000, sizeof(double), c->stream) || dev_sync(c->stream))
    return fail(c, RCCSDT_ERR_CUDA, "scalar read failed");
  const int flag = *(const int*)&h[5];
  for (int q = 0; q < 5; ++q) out[q] = h[q];
  out[3] = 0.0;
  out[5] = (double)flag;
  return 0;
}

const double* ctx_scalars(const rccsdt_ctx* c) { return (const double*)c->scalars->p; }
cudaStream_t ctx_stream(const rccsdt_ctx* c) { return c->stream; }
void ctx_set_stream(rccsdt_ctx* c, cudaStream_t s) { c->stream = s; }
int ctx_main_precision(const rccsdt_ctx* c) { return c->opt.precision; }
void ctx_reset_precision(rccsdt_ctx* c) { c->precision = c->opt.precision; }
void ctx_set_concurrent(rccsdt_ctx* c, int on) { c->concurrent = on; }
void ctx_begin_capture(rccsdt_ctx* c) {
  c->packedA_kind = c->packedB_kind = -1;
  c->timing = 0;
}
int ctx_ready(rccsdt_ctx* c) { return need(c, true, false, false); }
int ctx_prepare(rccsdt_ctx* c) {
  // (a batch that runs the grouped GEMMs itself tunes its own launch)
  if (!c->opt.autotune || !c->gr.on || c->gr.tuned || c->batch_gemm) return 0;
  // one evaluation in the main precision runs the autotuner on real panels
  const int st = ctx_enqueue(c, 0, c->opt.precision);
  c->precision = c->opt.precision;
  if (st) return st;
  return dev_sync(c->stream) ? fail(c, RCCSDT_ERR_CUDA, "autotune evaluation failed") : 0;
}
int ctx_q_inputs(rccsdt_ctx* c, QInputs* q) {
  if (!c || !q) return RCCSDT_ERR_ARG;
  if (!c->have_ham) return fail(c, RCCSDT_ERR_STATE, "hamiltonian not set");
  if (!c->have_amp) return fail(c, RCCSDT_ERR_STATE, "amplitudes not set");
  q->L = c->D("L");
  q->e = c->D("e");
  q->t2 = c->D("t2");
  q->t3 = c->B("t3")->p;
  q->t3_f32 = c->opt.precision != RCCSDT_FP64 ? 1 : 0;
  q->o = c->o;
  q->v = c->v;
  q->naux = c->naux;
  q->stream = c->stream;
  return 0;
}
int ctx_fail(rccsdt_ctx* c, int code, const char* msg) { return fail(c, code, msg); }

int ctx_dims(const rccsdt_ctx* c, int* o, int* v) {
  *o = c->o;
  *v = c->v;
  return 0;
}

}  // namespace rcc
