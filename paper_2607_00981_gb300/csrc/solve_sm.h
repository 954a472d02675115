// Host-side iteration control of rccsdt_solve, shared by the single-context solver
// and the batched driver so that both take exactly the same steps.
//
// Every step is one "body" queued on a context (ctx_enqueue_code):
//   kEvalMain  evaluation in the main precision at the current amplitudes (first step)
//   kEvalF64   evaluation with FP64 contractions
//   kStepMain  update from the last residual, then a main-precision evaluation
//   kStepF64   update, then an FP64 evaluation
//   kStepMid   update, then a 3xTF32 evaluation (3xBF16 contexts only)
//
// FP64 contexts iterate kStepMain.  Split contexts refine in a ladder of precisions:
// the main precision until |R| <= sqrt(tol); for 3xBF16 then 3xTF32 until
// |R| <= tol^(3/4) or until it stalls (no 10 % improvement over three evaluations);
// then FP64 iterations.  Each rung's rounding error (about 2^-16 of the summed terms
// for 3xBF16, 2^-21 for 3xTF32) bounds how far its residual can be trusted; the
// cheaper rungs take the iterations they can, the FP64 ones remove the rest.
// Convergence is only accepted on an FP64 evaluation.
#pragma once
#include <cmath>

#include "../../include/rccsdt.h"

namespace rcc {

enum { kEvalMain = 0, kEvalF64 = 1, kStepMain = 2, kStepF64 = 3, kStepMid = 4, kBodies = 5, kSkip = 5 };

struct SolveState {
  int it = 0;     // evaluations done
  int phase = 0;  // 0 main precision, 1 3xTF32 (from 3xBF16), 2 FP64
  int done = 0;
  int status = RCCSDT_NOT_CONVERGED;
  double e = 0.0, norm = 0.0;
  double best = INFINITY;  // the phase's smallest |R| so far
  int since = 0;           // evaluations since it last improved by 10 %
};

inline bool split_opt(const rccsdt_options& o) { return o.precision != RCCSDT_FP64; }
inline bool has_mid(const rccsdt_options& o) { return o.precision == RCCSDT_SPLIT_BF16X3; }

// Precision of a body's contractions.
inline int body_precision(const rccsdt_options& o, int code) {
  if (code == kEvalF64 || code == kStepF64) return RCCSDT_FP64;
  if (code == kStepMid) return RCCSDT_SPLIT_TF32X3;
  return o.precision;
}

inline bool body_updates(int code) { return code == kStepMain || code == kStepF64 || code == kStepMid; }

inline int next_code(const rccsdt_options& o, SolveState& s) {
  if (s.done) return kSkip;
  if (s.it == 0) return kEvalMain;
  if (!split_opt(o)) return kStepMain;
  const int before = s.phase;
  if (s.phase == 0 && s.norm <= std::sqrt(o.tol)) s.phase = has_mid(o) ? 1 : 2;
  if (s.phase == 1 && (s.norm <= std::pow(o.tol, 0.75) || s.since >= 3)) s.phase = 2;
  if (s.phase != before) {
    s.best = INFINITY;
    s.since = 0;
  }
  return s.phase == 0 ? kStepMain : (s.phase == 1 ? kStepMid : kStepF64);
}

// out: squared norms of R1, R2, R3 in [0..2], energy in [4], watchdog flag in [5].
inline void take_result(const rccsdt_options& o, SolveState& s, int code, const double* out) {
  s.it += 1;
  s.norm = std::sqrt(out[0] + out[1] + out[2]);
  s.e = out[4];
  if (s.norm < 0.9 * s.best) {
    s.best = s.norm;
    s.since = 0;
  } else {
    s.since += 1;
  }
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
