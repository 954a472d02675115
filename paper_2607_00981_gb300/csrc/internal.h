// Internal interface between the single-instance runtime and the batched driver.
#pragma once
#include <cuda_runtime.h>

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
