// Internal interface between the single-instance runtime and the batched driver.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "kernels.h"

struct rccsdt_ctx;

namespace rcc {

// Queues one evaluation on the context's stream without any host synchronisation:
// [the update of the amplitudes from the last residual when update_first], then the
// energy, intermediates, residuals and post-processed R3 with its norms, with the
// contractions in `precision`.  Results stay in the device scalars.
int ctx_enqueue(rccsdt_ctx* c, int update_first, int precision);
// Queues body `code` of the solver's state machine (solve_sm.h).
int ctx_enqueue_code(rccsdt_ctx* c, int code);
// Reads the last evaluation's scalars (norms squared [0..2], energy [4], watchdog
// flag [5]) to the host, synchronising the context's stream.
int ctx_read_scalars(rccsdt_ctx* c, double* out);
// Device scalars: [0..2] squared norms of R1, R2, R3 (block-weighted), [4] energy;
// the int at byte offset 8000 is the tensor-core watchdog flag.
const double* ctx_scalars(const rccsdt_ctx* c);
cudaStream_t ctx_stream(const rccsdt_ctx* c);
void ctx_set_stream(rccsdt_ctx* c, cudaStream_t s);
int ctx_main_precision(const rccsdt_ctx* c);
void ctx_reset_precision(rccsdt_ctx* c);
// 1: other contexts run concurrently on the GPU (a batch), so GEMMs are launched
// with their natural grids instead of splitting K across every SM.
void ctx_set_concurrent(rccsdt_ctx* c, int on);
// Resets host-side launch bookkeeping (operand reuse tracking, timing) so that a
// captured sequence does not depend on what ran before it.
void ctx_begin_capture(rccsdt_ctx* c);
// 0 when the Hamiltonian and amplitudes are set, else an rccsdt_status.
int ctx_ready(rccsdt_ctx* c);
// Runs what must not happen inside a graph capture (the grouped GEMM's autotuner,
// on one eager evaluation) when the context asks for it; 0 otherwise.
int ctx_prepare(rccsdt_ctx* c);
int ctx_dims(const rccsdt_ctx* c, int* o, int* v);

// Batch-wide grouped GEMM.  A body `code` whose evaluation takes the grouped path
// (ctx_body_grouped) is queued in two parts around its grouped GEMM: part 0 up to
// the operand gathers, part 1 from the reduction of the GEMM results into R3 to the
// post-processed norms; other bodies run whole in part 0.
int ctx_body_grouped(const rccsdt_ctx* c, int code);
int ctx_enqueue_part(rccsdt_ctx* c, int code, int part);
// The context's grouped GEMM problems (plan order) with tile width bn.
int ctx_grouped_problems(rccsdt_ctx* c, int bn, std::vector<GProblem>* out);
// Panel kind of the grouped path (-1 when the context has none).
int ctx_grouped_kind(const rccsdt_ctx* c);
void ctx_set_batch_gemm(rccsdt_ctx* c, int on);
// The context's own grouped GEMM launch (the host simulation of a batch).
int ctx_run_grouped_gemm(rccsdt_ctx* c);

// What the (Q) correction reads from a context: the bare factors L[naux][n][n], the
// Fock diagonal e[n], t2[o][o][v][v] (FP64) and compact T3 (FP32 in split contexts).
struct QInputs {
  const double* L;
  const double* e;
  const double* t2;
  const void* t3;
  int t3_f32;
  int o, v, naux;
  cudaStream_t stream;
};
// Fills *q; RCCSDT_ERR_STATE (with the context's error text) when the Hamiltonian or
// the amplitudes are not set.
int ctx_q_inputs(rccsdt_ctx* c, QInputs* q);
// Records msg as the context's last error and returns code.
int ctx_fail(rccsdt_ctx* c, int code, const char* msg);

}  // namespace rcc
