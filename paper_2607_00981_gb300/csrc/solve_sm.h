// Host-side iteration control of rccsdt_solve, shared by the single-context
// solver and the batched driver so that both take exactly the same steps.
//
// Every step is one "body" queued on a context (ctx_enqueue_code):
//   kEvalMain  evaluation in the main precision at the current amplitudes (first step)
//   kEvalF64   evaluation with FP64 contractions
//   kStepMain  update from the last residual, then a main-precision evaluation
//   kStepF64   update, then an FP64 evaluation
//
// FP64 contexts iterate kStepMain.  Split contexts run split iterations until
// |R| <= sqrt(tol) and then FP64 iterations (iterative refinement: the split
// residual carries a rounding error of about 2^-16 (3xBF16) or 2^-21 (3xTF32) of
// the terms it sums, which the FP64 iterations remove); convergence is only
// accepted on an FP64 evaluation.
#pragma once
#include <cmath>

#include "../../include/rccsdt.h"

namespace rcc {

enum { kEvalMain = 0, kEvalF64 = 1, kStepMain = 2, kStepF64 = 3, kBodies = 4, kSkip = 4 };

struct SolveState {
  int it = 0;     // evaluations done
  int phase = 0;  // 0 split, 1 FP64
  int done = 0;
  int status = RCCSDT_NOT_CONVERGED;
  double e = 0.0, norm = 0.0;
};

inline bool split_opt(const rccsdt_options& o) { return o.precision != RCCSDT_FP64; }

// Precision of a body's contractions.
inline int body_precision(const rccsdt_options& o, int code) {
  return (code == kEvalF64 || code == kStepF64) ? RCCSDT_FP64 : o.precision;
}

inline int next_code(const rccsdt_options& o, SolveState& s) {
  if (s.done) return kSkip;
  if (s.it == 0) return kEvalMain;
  if (!split_opt(o)) return kStepMain;
  if (s.phase == 0 && s.norm <= std::sqrt(o.tol)) s.phase = 1;
  return s.phase == 1 ? kStepF64 : kStepMain;
}

// out: squared norms of R1, R2, R3 in [0..2], energy in [4], watchdog flag in [5].
inline void take_result(const rccsdt_options& o, SolveState& s, int code, const double* out) {
  s.it += 1;
  s.norm = std::sqrt(out[0] + out[1] + out[2]);
  s.e = out[4];
  const bool fp64_eval = body_precision(o, code) == RCCSDT_FP64;
  if (out[5] != 0.0) {
    s.status = RCCSDT_ERR_TIMEOUT;
    s.done = 1;
  } else if (!std::isfinite(s.norm) || !std::isfinite(s.e)) {
    s.status = RCCSDT_ERR_NONFINITE;
    s.done = 1;
  } else if (s.norm <= o.tol && fp64_eval) {
    s.status = RCCSDT_OK;
    s.done = 1;
  } else if (s.it >= o.max_iter) {
    s.status = RCCSDT_NOT_CONVERGED;
    s.done = 1;
  }
}

}  // namespace rcc
