/*
 * rccsdt.h -- C ABI of the GB300 (sm_103a) RCCSDT residual library.
 *
 * One spin-restricted CCSDT iteration on compact triples storage: the T1-dressed
 * Hamiltonian and intermediates, the residuals R1, R2 and R3 (the T3 residual
 * keeps only the occupied triples i <= j <= k, each a full v^3 block over abc),
 * the post-processing of R3, the orbital-energy denominator update with DIIS and
 * the correlation energy.  The method is the one of arXiv 2607.00981:
 *   - working equations: appendix A.5 (RCCSD R1/R2, RCCSDT T3 corrections,
 *     Eq. resi-rccsdt, the RCCSDT intermediates), with the T1-dressed integrals
 *     of appendix A.4 and the spin summations of Eq. triples-spin-sum;
 *   - compact storage and contractions: Sec. II.B.1 and Sec. II.C (direct
 *     traversal of the pp-ladder, unpacking for the hh-ladder and ring terms,
 *     the representative contractions of the operation-count table); the
 *     pp-ladder runs as sum and difference products over the exchange symmetry
 *     W^{ab}_{de} = W^{ba}_{ed} (same result, about half its FMA);
 *   - post-processing: Sec. II.D (symmetrise, purify, orthogonalise);
 *   - update: Jacobi step t += r / eps of appendix A.1; DIIS of Sec. III.A.5;
 *   - energy: the E_CC expression of appendix A.5 with bare integrals.
 *
 * Conventions (all arrays dense, row-major, float64 unless stated):
 *   n = o + v spatial orbitals, occupied first.
 *   L[naux][n][n]   factors of the chemists' ERIs, (pq|rs) = sum_P L[P,p,q] L[P,r,s];
 *                   symmetric in the last two indices.
 *   fock_diag[n]    canonical (diagonal) Fock matrix.
 *   t1[o][v], t2[o][o][v][v]        spin-free amplitudes t_i^a, t_ij^ab.
 *   t3c[n3][v][v][v], n3 = o(o+1)(o+2)/6, block blk(i<=j<=k) =
 *                   C(k+2,3) + C(j+1,2) + i  (colex order), element [a][b][c] = t_ijk^abc.
 *   Residuals r1, r2, r3c use the same layouts.
 * Pointers passed in or out may be host or device memory (the library copies with
 * cudaMemcpyDefault on the context's stream and synchronises before returning
 * from calls that read or write caller memory; an FP32-storage context converts
 * T3 from or to device memory and pinned host memory in place, with one kernel
 * over the host link, and stages pageable host memory in chunks).  The caller
 * keeps ownership of its buffers; the context owns every buffer it allocates.
 *
 * Errors: every call returns an rccsdt_status; nothing aborts, traps or prints.
 * rccsdt_last_error() gives a text for the last failing call on a context.
 */
#ifndef RCCSDT_H
#define RCCSDT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rccsdt_ctx rccsdt_ctx;

typedef enum {
  RCCSDT_OK = 0,
  RCCSDT_ERR_ARG = -1,        /* invalid size, pointer or option */
  RCCSDT_ERR_OOM = -2,        /* device allocation failed */
  RCCSDT_ERR_CUDA = -3,       /* a CUDA runtime or driver call failed */
  RCCSDT_ERR_NONFINITE = -4,  /* NaN or Inf found in a residual norm or the energy */
  RCCSDT_ERR_TIMEOUT = -5,    /* a device-side wait exceeded its watchdog budget */
  RCCSDT_ERR_STATE = -6,      /* call made before the data it needs was set */
  RCCSDT_NOT_CONVERGED = 1    /* rccsdt_solve reached max_iter */
} rccsdt_status;

typedef enum {
  RCCSDT_FP64 = 0,            /* FP64 contractions (SIMT DFMA), FP64 T3 storage */
  RCCSDT_SPLIT_BF16X3 = 1,    /* FP32 T3; large contractions as hi*hi + hi*lo + lo*hi in BF16
                                 on tcgen05 with FP32 accumulation in TMEM */
  RCCSDT_SPLIT_TF32X3 = 2     /* as above with TF32 halves */
} rccsdt_precision;

typedef struct {
  int precision;          /* rccsdt_precision */
  int diis_space;         /* DIIS history length M (0 = plain Jacobi) */
  int diis_start;         /* first iteration (1-based) that extrapolates */
  int diis_t3;            /* 1: DIIS vectors include T3; 0: T1 and T2 only */
  int max_iter;           /* rccsdt_solve iteration cap */
  double tol;             /* convergence threshold on the residual norm */
  long long watchdog_cycles; /* clock64 budget of each device-side pipeline wait of the tensor-core
                                GEMMs (0 = default 4e9, about 2 s; values below 64 are raised to 64;
                                negative: RCCSDT_ERR_ARG).  A wait that runs out makes the GEMM stop
                                and the next call that reads results return RCCSDT_ERR_TIMEOUT; the
                                kernel still retires its own copies and MMAs (waiting at least about
                                a second for them) before it exits. */
  long long grouped_bytes;   /* split modes: device bytes the grouped residual may hold (all
                                operand panels and dense results of the R3 contractions at
                                once); when an instance needs more, or 0, its contractions
                                run one by one through shared panels */
  long long unpack_bytes;    /* device bytes for the unpacked, spin-summed T3 blocks t_{xyz} of
                                the T3 -> R1/R2/W step (as many values of z as fit, at least
                                one; <= 0 means 1 GiB) */
  int autotune;              /* 1: time candidate launch shapes of the grouped GEMM on the
                                first iteration and keep the fastest; 0: fixed shape;
                                2 + i: always candidate i (0..5) of the autotuner's list */
  int f64_tc;                /* FP64 contractions (FP64 contexts, and the final FP64
                                iterations of split contexts): 0 on the FP64 units (DFMA);
                                1 those of 3e7 FMA or more on the BF16 tensor cores, exact to
                                about 2^-37 of the operands' row and column maxima (six 7-bit
                                digit planes per operand, 21 digit products, exact FP32
                                partial sums of the leading digit levels over K chunks of
                                256, double-float and FP64 totals); 2 every contraction there */
  long long pp_unit_bytes;   /* device bytes of one pp-ladder launch unit's T operand (v rows of
                                v^2 doubles per stored block): the stored blocks are cut into
                                ranges of that size, one GEMM per view and range (<= 0: 2 GiB) */
  int diis_t3_nvir;          /* with diis_t3: the T3 part of the DIIS vectors keeps only the
                                components t_ijk^abc with a, b, c < diis_t3_nvir (the lowest
                                virtual orbitals in the given order; the subspace DIIS of
                                Sec. III.A.5), the rest of T3 takes the plain Jacobi step;
                                <= 0 or >= v: all of T3 */
} rccsdt_options;

/* Fills *opt with the defaults: FP64, DIIS(8) from iteration 2 including T3,
 * max_iter 100, tol 1e-8, grouped_bytes 8 GiB, unpack_bytes 1 GiB, autotune 0,
 * f64_tc 0, pp_unit_bytes 2 GiB, diis_t3_nvir 0 (all of T3). */
int rccsdt_options_default(rccsdt_options* opt);

/* Creates a context for o occupied / v virtual orbitals and naux factors, on the
 * CUDA stream `stream` (a cudaStream_t, NULL = legacy default stream) of the
 * current device.  Allocates all device memory the iteration needs.
 * Limits: o <= 64, v <= 1024 (offsets inside one v^3 block are 32-bit; W^{ab}_{cd}
 * alone, v^4 doubles, exceeds any device's memory well before that).
 * Errors: RCCSDT_ERR_ARG (o, v, naux < 1, o or v above the limits, or out == NULL),
 * RCCSDT_ERR_OOM. */
int rccsdt_create(int o, int v, int naux, const rccsdt_options* opt, void* stream,
                  rccsdt_ctx** out);

/* Bytes of device memory the context holds. */
long long rccsdt_device_bytes(const rccsdt_ctx* ctx);

/* Sets the Hamiltonian (appendix A.3): fock_diag[n], L[naux][n][n]. */
int rccsdt_set_hamiltonian(rccsdt_ctx* ctx, const double* fock_diag, const double* L);

/* Sets the amplitudes (float64 in every precision mode; stored as FP32 T3 in the
 * split modes).  Any pointer may be NULL to leave that amplitude unchanged.
 * Clears the DIIS history and a watchdog timeout (as does rccsdt_init_mp2). */
int rccsdt_set_amplitudes(rccsdt_ctx* ctx, const double* t1, const double* t2, const double* t3c);

/* The same with T3 in FP32, the storage type of the split modes (RCCSDT_SPLIT_*
 * contexts only): t3c is copied as it is, half the bytes of the float64 call (pinned
 * host or device memory: one copy kernel reads it in place; pageable host memory: a
 * staged copy).  t1 and t2 stay float64.  Errors: RCCSDT_ERR_ARG (an FP64 context), RCCSDT_ERR_CUDA. */
int rccsdt_set_amplitudes_t3f32(rccsdt_ctx* ctx, const double* t1, const double* t2, const float* t3c);

/* t1 = 0, t2 = first-order (MP2) doubles v^{ab}_{ij} / eps_ij^ab, t3 = 0. */
int rccsdt_init_mp2(rccsdt_ctx* ctx);

/* Switches the precision of later contractions (rccsdt_precision).  A split context
 * may switch between the split modes and FP64 contractions (its T3 and R3 stay in
 * FP32 storage); a context created in FP64 mode accepts FP64 only (RCCSDT_ERR_ARG). */
int rccsdt_set_precision(rccsdt_ctx* ctx, int precision);

/* Step (i)-(iii) of one iteration: T1-dressing, the RCCSD and RCCSDT
 * intermediates, and the T3 contributions to R1, R2, W^{ab}_{dj}, W^{al}_{ij}.
 * This call, rccsdt_residual and rccsdt_iterate return RCCSDT_ERR_TIMEOUT once a
 * device-side wait of the context has run out (options.watchdog_cycles); the
 * results are then undefined until new amplitudes are set. */
int rccsdt_build_intermediates(rccsdt_ctx* ctx);

/* Steps (iv)-(v): R1, R2 and the raw compact R3 (requires the intermediates). */
int rccsdt_residual(rccsdt_ctx* ctx);

/* Symmetrise, purify and orthogonalise R3 (Sec. II.D) and return
 * norms[4] = {|R1|, |R2|, |R3|, |R|}, |R3| the full-tensor norm
 * (block multiplicities 6/3/1).  norms may be NULL. */
int rccsdt_postprocess(rccsdt_ctx* ctx, double norms[4]);

/* Jacobi step t += r / eps (bare Fock diagonal) for t1, t2, t3, then DIIS. */
int rccsdt_update(rccsdt_ctx* ctx);

/* Correlation energy of the current amplitudes (bare integrals). */
int rccsdt_energy(rccsdt_ctx* ctx, double* e_corr);

/* One whole iteration: energy of the current amplitudes, intermediates,
 * residuals, post-processing, update.  e_corr and norms (as above) describe the
 * amplitudes the residual was evaluated at; either may be NULL. */
int rccsdt_iterate(rccsdt_ctx* ctx, double* e_corr, double norms[4]);

/* Iterates from the current amplitudes until |R| <= tol or max_iter evaluations.
 * In the split modes the iterations run in the context's split precision until
 * |R| <= sqrt(tol); a 3xBF16 context then runs 3xTF32 iterations until
 * |R| <= tol^(3/4) or until they stop improving (no 10 % gain in three evaluations);
 * the rest run with FP64 contractions (options.f64_tc chooses the engine), and
 * convergence is only accepted on an FP64 evaluation (iterative refinement).
 * Outputs describe the last residual evaluated (iterations counts evaluations).
 * Returns RCCSDT_NOT_CONVERGED if max_iter is reached. */
int rccsdt_solve(rccsdt_ctx* ctx, double* e_corr, int* iterations, double* final_norm);

/* Checkpoint (the restart from amplitudes on disk of Sec. II.B.1, "Amplitude tensors").
 * rccsdt_save writes the iteration state -- t1, t2, compact t3 in the context's
 * storage type, the DIIS history with its counters and B matrix, the iteration
 * counters and the current precision -- to `path` (raw little-endian with a
 * header); rccsdt_load reads it into a context created with the same o, v,
 * storage precision and DIIS options (the Hamiltonian is not part of the file:
 * set it before iterating).  An iteration after rccsdt_load repeats the one the
 * saved context would have taken next.  Errors: RCCSDT_ERR_ARG (NULL path, file
 * not readable or writable, not a checkpoint, truncated, or made for other sizes
 * or options), RCCSDT_ERR_STATE (save without amplitudes), RCCSDT_ERR_CUDA. */
int rccsdt_save(rccsdt_ctx* ctx, const char* path);
int rccsdt_load(rccsdt_ctx* ctx, const char* path);

/* Copies out the amplitudes / the current residuals (float64). NULL skips. */
int rccsdt_get_amplitudes(rccsdt_ctx* ctx, double* t1, double* t2, double* t3c);
/* Copies out the amplitudes with T3 in its FP32 storage (split modes only; errors as
 * rccsdt_set_amplitudes_t3f32). */
int rccsdt_get_amplitudes_t3f32(rccsdt_ctx* ctx, double* t1, double* t2, float* t3c);
int rccsdt_get_residuals(rccsdt_ctx* ctx, double* r1, double* r2, double* r3c);

/* Leading algorithmic FMA count of the compact contractions of one iteration,
 * n3 (3 v^5 + 12 o v^4 + 3 o^2 v^3) (operation-count table). */
double rccsdt_iteration_fma(int o, int v);

/* Timing window.  rccsdt_enable_timing(ctx, 1) starts a window: from then on
 * the library records CUDA events (never waited on) around each step and around
 * each GEMM launch of the pp-ladder on the context's stream.  rccsdt_step_times
 * waits for the last event and writes, summed over the window:
 *   ms[0..8]  device ms of: intermediates, pp-ladder, ring, hh-ladder, T2 terms,
 *             R1/R2 and setup, postprocess, update, energy;
 *   ms[9]     device ms inside the pp-ladder GEMM kernels alone;
 *   ms[10]    number of those GEMM launches;  ms[11]  the flop they execute
 *             (2 M N K each; with the pair-symmetric form of the per-plan engine,
 *             about half the paper's pp-ladder count).
 * Returns the number of entries written (<= cap, at most 12). */
int rccsdt_step_times(rccsdt_ctx* ctx, double* ms, int cap);
int rccsdt_enable_timing(rccsdt_ctx* ctx, int on);

/* Number of CUDA kernels this library has launched in the process so far. */
long long rccsdt_kernel_launches(void);

/* Contraction engine of the context: out[0] 1 if the grouped residual is on,
 * [1] its GEMM problems, [2] their output tiles, [3] operand gathers, [4] block
 * contributions reduced into R3, [5] device bytes it holds, [6] persistent grid
 * of its GEMM launch (0 = one CTA per SM), [7] panel kind, [8] tile width,
 * [9] problem order (0 longest K first, 1 plan order), [10] 1 once the autotuner
 * has run, [11] its chosen shape's GEMM time and [12] the fixed shape's (256-wide
 * tiles, longest K first, one CTA per SM), in microseconds.  Returns entries written. */
int rccsdt_engine_info(const rccsdt_ctx* ctx, long long* out, int cap);

/* Diagnostic: copies the first `count` float64 values of a named internal tensor
 * (e.g. "Fvv", "Wvvvo", "Wvvvv", "Wb_ovov", "r1", "X2") to `out`.  Layouts are the
 * index orders of the paper's symbols, upper indices first.  RCCSDT_ERR_ARG for
 * an unknown name or a count beyond the tensor. */
int rccsdt_debug_copy(rccsdt_ctx* ctx, const char* name, double* out, long long count);

const char* rccsdt_last_error(const rccsdt_ctx* ctx);
void rccsdt_destroy(rccsdt_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Batched instances.  A batch holds n independent contexts (instance i has
 * o[i], v[i], naux[i]; all share *opt) and iterates them together: one CUDA
 * graph launch per iteration runs every unconverged instance's iteration
 * concurrently, each as the body of a conditional node chosen on the device from
 * a per-instance code the host writes before the launch.  In the split precisions
 * the residuals' tensor-core products of every instance on the grouped path run
 * as ONE persistent grouped-GEMM launch inside that graph (the instances' bodies
 * are captured in two parts around it; its launch shape is tuned on the batch's
 * own problem table when options.autotune is set).  The graph is built on the
 * first rccsdt_batch_solve (capture of each instance's launch sequence) and
 * replayed afterwards.
 * --------------------------------------------------------------------------- */
typedef struct rccsdt_batch rccsdt_batch;

/* Creates the batch and its n contexts on `stream` (used by the per-instance
 * calls below); the batch launches its graph on a stream of its own.
 * Errors: RCCSDT_ERR_ARG (n < 1, NULL arrays, an invalid size), RCCSDT_ERR_OOM. */
int rccsdt_batch_create(int n, const int* o, const int* v, const int* naux, const rccsdt_options* opt,
                        void* stream, rccsdt_batch** out);

/* Context of instance i (owned by the batch, NULL if i is out of range).  Use it
 * with rccsdt_set_hamiltonian, rccsdt_init_mp2 / rccsdt_set_amplitudes and
 * rccsdt_get_amplitudes; do not destroy it. */
rccsdt_ctx* rccsdt_batch_instance(rccsdt_batch* b, int i);

/* Iterates every instance from its current amplitudes with the rule of
 * rccsdt_solve (including the FP64 final phase of the split modes) until each has
 * converged, failed or reached max_iter.  Host arrays of n entries receive each
 * instance's energy, evaluations, final |R| and status (any may be NULL).
 * Returns RCCSDT_OK when all converged, the most severe negative status if one
 * failed, else RCCSDT_NOT_CONVERGED.  Unlike rccsdt_solve, an instance that stops
 * at max_iter keeps the amplitudes its last residual was evaluated at. */
int rccsdt_batch_solve(rccsdt_batch* b, double* e_corr, int* iterations, double* final_norm, int* status);

/* Statistics of the last rccsdt_batch_solve: out[0] graph launches, [1] device ms
 * over those launches (CUDA events around each launch), [2] algorithmic flop of
 * the evaluations run, [3] kernels executed, [4] nodes of the top-level graph,
 * [5] host ms to build the graph (captures included), [6] host ms to instantiate
 * and upload it, [7] device ms of the first launch, [8] 1 when the residuals'
 * grouped GEMMs of all instances run as one batch-wide persistent launch (split
 * precisions), [9] its problems, [10] its tiles with every instance active, [11] its
 * tile width, [12] its tuned and [13] its fixed-shape time in ms (all instances
 * active).  Returns entries written (at most 14). */
int rccsdt_batch_stats(const rccsdt_batch* b, double* out, int cap);
/* Device ms of each launch of the last rccsdt_batch_solve; returns the count. */
int rccsdt_batch_launch_times(const rccsdt_batch* b, double* ms, int cap);

const char* rccsdt_batch_last_error(const rccsdt_batch* b);
void rccsdt_batch_destroy(rccsdt_batch* b);

/* ---------------------------------------------------------------------------
 * RCCSDT(Q): the perturbative quadruples energy correction on the context's
 * current (converged) t2 and compact t3 with the BARE Hamiltonian (T1 does not
 * enter), Eq. ener-pt-q of the (Q) appendix with r = P(X + Y), z = P(X + V)
 * (Eqs. resi-pt-q, q_t3_terms), the alternative intermediates of Eq. q_w_alter and
 * the orbital-energy denominators, evaluated by the ABC-based algorithm of
 * Sec. II.E.2: the one-time transposition of compact T3 to the virtual-triangular
 * layout, then the sum over sorted virtual quadruples a <= b <= c <= d weighted by
 * their degeneracy factors (Eq. ener-pt-q-abc).
 * --------------------------------------------------------------------------- */
typedef enum {
  RCCSDT_Q_FP64 = 0,   /* FP64 arithmetic throughout */
  RCCSDT_Q_FP32 = 1    /* FP32 operands and dot products, FP64 energy partial sums */
} rccsdt_q_arith;

/* Writes E_(Q) to *e_q (host).  info, if not NULL, receives 6 values: device ms of
 * the T3 transposition, of the integrals and intermediates, and of the main kernel;
 * the flop the main kernel executes (24 joint permutations x o^4 x (2v + 2o) FMA per
 * sorted quadruple with a nonzero degeneracy factor); the number of such
 * quadruples; the persistent grid.  Allocates its working buffers (the bare ERIs
 * n^4, Wbar^{abc}_{ejk} o^2 v^4 and Wbar^{abm}_{ijk} o^4 v^2 in the arithmetic's
 * type, the transposed T3) for the duration of the call and frees them.
 * Errors: RCCSDT_ERR_ARG (NULL pointers, unknown arith), RCCSDT_ERR_STATE (no
 * Hamiltonian or amplitudes), RCCSDT_ERR_OOM, RCCSDT_ERR_CUDA (also when a CUDA
 * error was pending before the call), RCCSDT_ERR_NONFINITE. */
int rccsdt_q_energy(rccsdt_ctx* ctx, int arith, double* e_q, double* info);

/* The one-time transposition of Sec. II.E.2 (Fig. q_operation_counts(a)): compact
 * T3 of the context (occupied-triangular, [n3][v][v][v]) written to t3v (host or
 * device, float64) in the virtual-triangular layout t3v[nv3][o][o][o],
 * nv3 = v(v+1)(v+2)/6, block (a <= b <= c) at C(c+2,3) + C(b+1,2) + a (colex, as
 * the occupied blocks), element [i][j][k] = t_ijk^abc. */
int rccsdt_t3_virtual_triangular(rccsdt_ctx* ctx, double* t3v);

/* ---------------------------------------------------------------------------
 * Compact T4 of RCCSDTQ (the step one rank above this library's RCCSDT path):
 * the W^vv_vv * T4 particle-particle ladder on compact storage by direct
 * traversal (Sec. II.C.4: six terms per stored block, each read from the same
 * block after relabelling the paired columns), and the post-processing of R4
 * (Sec. II.D: symmetrisation of blocks with two equal occupied indices as the
 * average over the column swap, purification of blocks with three equal ones, and
 * the projection 1 - Pi_[4] - Pi_[3,1] of Eq. T4ortho on every block).
 * Storage: t4c[n4][v][v][v][v], n4 = o(o+1)(o+2)(o+3)/24, block (i<=j<=k<=l) at
 * C(l+3,4) + C(k+2,3) + C(j+1,2) + i, element [a][b][c][d] = t_ijkl^abcd;
 * W[a][b][e][f] = W^{ab}_{ef}, symmetric under (a,e) <-> (b,f) (the ladder runs as
 * sum and difference products over the label pairs and relies on it).  In the split
 * precisions T4 and R4 are stored in FP32 and the ladder runs as 3xBF16 / 3xTF32
 * products on the tensor cores; in FP64 on the FP64 units.
 * --------------------------------------------------------------------------- */
typedef struct rccsdt_t4 rccsdt_t4;

/* Allocates T4, R4 and the operand panels on the current device, work on `stream`.
 * Limits: 1 <= o <= 32, 1 <= v <= 200.  Errors: RCCSDT_ERR_ARG, RCCSDT_ERR_OOM. */
int rccsdt_t4_create(int o, int v, int precision, void* stream, rccsdt_t4** out);
/* Sets W (v^4) and/or compact T4 (host or device float64; NULL leaves one as is). */
int rccsdt_t4_set(rccsdt_t4* t4, const double* W, const double* t4c);
/* R4 = the six-term ladder of the current W and T4 (overwrites R4).
 * Errors: RCCSDT_ERR_STATE (W or T4 not set), RCCSDT_ERR_TIMEOUT, RCCSDT_ERR_CUDA. */
int rccsdt_t4_pp_ladder(rccsdt_t4* t4);
/* Symmetrise, purify and project R4 in place; *norm (if not NULL) = the full-tensor
 * norm of the result (block multiplicities 24 / 12 / 6 / 4 / 1). */
int rccsdt_t4_postprocess(rccsdt_t4* t4, double* norm);
/* Copies R4 out (host or device float64, n4 v^4 values). */
int rccsdt_t4_get_r4(rccsdt_t4* t4, double* r4c);
const char* rccsdt_t4_last_error(const rccsdt_t4* t4);
void rccsdt_t4_destroy(rccsdt_t4* t4);

/* ---------------------------------------------------------------------------
 * IJK-partitioned multi-process planning (Sec. III.A.1-III.A.3).  Host-only: no
 * call in this section touches a GPU, and none needs one.
 *
 * The stored blocks of compact T3/R3 (i <= j <= k, storage order of the context)
 * are distributed over `nranks` processes as individual IJK triples (Sec. III.A.1:
 * the finest of the three partitions the paper weighs, chosen for load balance);
 * lower-order quantities stay replicated.  Ownership balances a per-block cost
 * (longest-processing-time-first: blocks by decreasing cost, ties by storage order,
 * each to the least-loaded rank, ties to the lowest rank).  The exchange of step
 * (v) of Sec. III.A.2 (F_oo, W_oooo and the two W_ov rings on T3 blocks owned
 * elsewhere) runs in batches (Sec. III.A.3): the batches partition the stored
 * blocks, so each T3 element is sent once per cycle; a batch holds consecutive
 * blocks in storage order, cut so that the batches carry equal shares of the step
 * (v) work, and lists its blocks grouped by owner in rank order (the layout of an
 * all-gather with per-rank counts).  The step (v) work of a gathered block u on rank
 * r is the work of the contractions of r's blocks that read u: v^3 FMA per F_oo or
 * W_oooo read, v^4 per ring read, over the reads of every term with unpacking of a
 * block's residual (F_oo 3o, W_oooo 3o^2, rings 15o reads per block).
 * --------------------------------------------------------------------------- */
typedef struct rccsdt_ijk_plan rccsdt_ijk_plan;

/* The default per-block cost: the FMA count of one stored block's residual terms,
 * 3v^5 (W_vvvv, direct traversal) + 15 o v^4 (rings) + 9 v^4 (F_vv and the T2 terms
 * with W_vvvo) + 3 o^2 v^3 (W_oooo) + 9 o v^3 (F_oo and the T2 terms with W_vooo),
 * and 0 for the blocks i = j = k, whose residual purification sets to zero
 * (Sec. II.D.2), so they need no contraction.  cost[n3] (host).
 * Errors: RCCSDT_ERR_ARG (o, v < 1, o > 64, NULL cost). */
int rccsdt_ijk_block_costs(int o, int v, double* cost);

/* Plans the partition and the exchange batches.  batch_triples (>= 1) is the
 * paper's N_IJK^batch, the mean number of blocks per batch (the batch count is
 * ceil(n3 / batch_triples)); cost[n3] (host, >= 0 and finite) replaces the default
 * model when not NULL.  A block of zero cost is owned like any other but reads
 * nothing in step (v).  Limits: 1 <= o <= 64, 1 <= nranks <= 4096, batches x
 * nranks <= 2^27.  Errors: RCCSDT_ERR_ARG (limits, NULL out, a negative or
 * non-finite cost), RCCSDT_ERR_OOM. */
int rccsdt_ijk_plan_create(int o, int v, int nranks, int batch_triples, const double* cost,
                           rccsdt_ijk_plan** out);
void rccsdt_ijk_plan_destroy(rccsdt_ijk_plan* plan);
/* info[6] = {n3, nranks, number of batches, most blocks one rank owns, most
 * blocks in one batch, most blocks one rank sends in one batch}. */
int rccsdt_ijk_plan_info(const rccsdt_ijk_plan* plan, long long info[6]);
/* owner[n3]: the rank that owns each stored block. */
int rccsdt_ijk_plan_owners(const rccsdt_ijk_plan* plan, int* owner);
/* The blocks `rank` owns, in storage order: *count is set; blocks (may be NULL to
 * query the count) receives *count indices.  Errors: RCCSDT_ERR_ARG (rank out of
 * range, NULL count). */
int rccsdt_ijk_plan_local(const rccsdt_ijk_plan* plan, int rank, int* blocks, int* count);
/* Batch b: counts[nranks] = the blocks each rank contributes; blocks (may be NULL)
 * receives the batch's block indices grouped by owner in rank order, each group in
 * storage order.  Errors: RCCSDT_ERR_ARG (b out of range, NULL counts). */
int rccsdt_ijk_plan_batch(const rccsdt_ijk_plan* plan, int b, int* counts, int* blocks);
/* rank_cost[nranks] (may be NULL): the summed cost of each rank's blocks;
 * batch_work[nbatches][nranks] (may be NULL): the step (v) FMA each batch's
 * gathered blocks cause on each rank. */
int rccsdt_ijk_plan_work(const rccsdt_ijk_plan* plan, double* rank_cost, double* batch_work);

/* Residual norms for callers that cannot allocate device memory.  The paper has
 * no counterpart: this entry point exists for callers such as a framework that
 * owns all device memory through its own pool allocator (a raw cudaMalloc would
 * bypass its accounting), or a service that reserves its memory at start-up and
 * must not allocate in steady state (cudaMalloc may synchronise the device, add
 * latency, or fail near the HBM limit).  It needs no context and allocates
 * nothing: its scratch is a fixed device array in the library image.
 *
 * Computes norms[4] = {|R1|, |R2|, |R3|, |R|} exactly as rccsdt_postprocess does
 * (|R3| weights each stored block by 6, 3 or 1 occupied triples) from the caller's
 * device buffers r1[o][v], r2[o][o][v][v] and the post-processed compact
 * r3c[n3][v][v][v] (float64), writing the four values to the device pointer
 * `norms`.  Work is queued on `stream` (a cudaStream_t, NULL = legacy default) and
 * the call returns without waiting.
 *
 * Limit: n3 = o(o+1)(o+2)/6 <= 4096, i.e. o <= 28; larger o, o or v < 1, or a NULL
 * pointer return RCCSDT_ERR_ARG before any GPU work.  RCCSDT_ERR_CUDA if the
 * device lookup or a launch fails, or if a CUDA error was already pending when the
 * call was made (that error is left pending for the caller, not cleared).
 * The first call on each device looks up the scratch's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  All calls on a device share the scratch and every call
 * overwrites the slots it uses before reading them; calls whose kernels overlap
 * on the GPU race on it, so order them on one stream. */
int rccsdt_residual_norms_noalloc(int o, int v, const double* r1, const double* r2, const double* r3c,
                                  double* norms, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RCCSDT_H */
