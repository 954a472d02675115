// Batched driver: many independent RCCSDT instances of different (o, v) iterated
// together, one CUDA graph launch per iteration of the whole batch.
//
// Each instance owns a full context (its own plans and buffers).  Its steps are
// captured once into the bodies of a conditional SWITCH node of one graph, one
// body per step kind of the solver (solve_sm.h: evaluation, or update followed
// by evaluation, in the main precision or with FP64 contractions); a code past
// the last body runs nothing (converged or stopped instances).  A control kernel at the top of the graph sets each SWITCH
// from a code array that the host writes before the launch; a gather kernel at
// the bottom copies every instance's norms and energy into one array read back
// with one copy.  The SWITCH nodes have no edges between them, so the instances
// run concurrently.  The host runs, per instance, the state machine of
// rccsdt_solve, so a batched instance takes the same steps as rccsdt_solve on a
// context of its own.
//
// Batch-wide grouped GEMM (split precisions): the residual's tensor-core products of
// every instance on the grouped path run in ONE persistent launch per batch
// iteration.  Each such body is captured in two parts around its grouped GEMM
// (SWITCH A: update, energy, intermediates, residual up to the operand gathers;
// SWITCH B: the reduction of the products into R3, the rest of the residual, the
// post-processed norms); between the two rows of SWITCH nodes one GEMM node runs the
// problems of all instances from one table.  A table kernel after the control kernel
// gives the problems of instances that do not take the grouped path this iteration
// (converged, or in an FP64 phase) no tiles, and writes the tile count the
// persistent kernel reads.  The launch shape (tile width, problem order) is tuned
// once on the batch's own table before the graph is captured.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rccsdt.h"
#include "internal.h"
#include "kernels.h"
#include "solve_sm.h"

namespace {

using rcc::kBodies;
using rcc::kSkip;
using rcc::SolveState;
constexpr int kOutStride = 8;  // per instance: |R1|^2 |R2|^2 |R3|^2 - E flag - -

#ifndef RCC_HOSTSIM
// handles[h] for h < nh takes the code of instance h % n (one or two SWITCH rows)
__global__ void k_batch_switch(const unsigned long long* __restrict__ handles, const int* __restrict__ codes, int n,
                               int nh) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h < nh) cudaGraphSetConditional((cudaGraphConditionalHandle)handles[h], (unsigned)codes[h % n]);
}

// Tile offsets of the batch-wide grouped GEMM: problems of instances whose body of
// this iteration takes the grouped path get their tiles, in table order; the others
// none.  One thread (a few hundred problems).
__global__ void k_batch_table(rcc::GProblem* __restrict__ probs, const int* __restrict__ pinst,
                              const int* __restrict__ ptiles, int nprob, const int* __restrict__ codes,
                              const int* __restrict__ gcode, int* __restrict__ total) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int t0 = 0;
  for (int p = 0; p < nprob; ++p) {
    probs[p].tile0 = t0;
    const int i = pinst[p], code = codes[i];
    if (code < kSkip && gcode[i * kBodies + code]) t0 += ptiles[p];
  }
  *total = t0;
}

__global__ void k_batch_gather(const double* const* __restrict__ scal, int n, const int* __restrict__ bflag,
                               double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* s = scal[i];
  double* o = out + (size_t)i * kOutStride;
  o[0] = s[0];
  o[1] = s[1];
  o[2] = s[2];
  o[3] = 0.0;
  o[4] = s[4];
  o[5] = (double)(((const int*)(s + 1000))[0] | (bflag ? *bflag : 0));
}
#endif

}  // namespace

struct rccsdt_batch {
  int n = 0;
  rccsdt_options opt{};
  cudaStream_t stream = nullptr;  // caller's stream (instance API calls)
  cudaStream_t run = nullptr;     // owned: capture and graph launches
  std::vector<rccsdt_ctx*> inst;
  std::vector<SolveState> state;
  std::vector<long long> body_launches;  // [n][kBodies]
  std::string err;
  // graph
  int built = 0;
  long long graph_nodes = 0;
  double capture_ms = 0.0, instantiate_ms = 0.0;
#ifndef RCC_HOSTSIM
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
#endif
  void* d_handles = nullptr;
  void* d_codes = nullptr;
  void* d_scal = nullptr;
  void* d_out = nullptr;
  int* h_codes = nullptr;
  double* h_out = nullptr;
  // batch-wide grouped GEMM (bgemm = 1): table of every grouped instance's problems
  int bgemm = 0, bg_kind = -1, bg_bn = 256, bg_ord = 0, bg_nprob = 0, bg_maxtiles = 0;
  double bg_ms = 0.0, bg_fixed_ms = 0.0;
  std::vector<int> gcode;   // [n][kBodies]: 1 if that body takes the grouped path
  void* d_probs = nullptr;
  void* d_pinst = nullptr;
  void* d_ptiles = nullptr;
  void* d_gcode = nullptr;
  void* d_total = nullptr;
  void* d_bflag = nullptr;
  // statistics of the last rccsdt_batch_solve
  long long launches = 0, kernels = 0;
  double device_ms = 0.0, flop = 0.0;
  std::vector<double> launch_ms;
};

namespace {

int bfail(rccsdt_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

#ifndef RCC_HOSTSIM
double ms_since(const std::chrono::steady_clock::time_point& t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// The batch-wide problem table for tile width bn and problem order ord (0 longest K
// first over the whole batch, 1 instance and plan order); every problem active.
int batch_table(rccsdt_batch* b, int bn, int ord) {
  std::vector<rcc::GProblem> all;
  std::vector<int> inst;
  for (int i = 0; i < b->n; ++i) {
    if (rcc::ctx_grouped_kind(b->inst[i]) < 0) continue;
    std::vector<rcc::GProblem> pr;
    const int st = rcc::ctx_grouped_problems(b->inst[i], bn, &pr);
    if (st) return bfail(b, st, std::string("instance ") + std::to_string(i) + ": " + rccsdt_last_error(b->inst[i]));
    for (const auto& P : pr) {
      all.push_back(P);
      inst.push_back(i);
    }
  }
  std::vector<int> order(all.size());
  for (size_t q = 0; q < all.size(); ++q) order[q] = (int)q;
  if (ord == 0)
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return all[x].kblocks > all[y].kblocks; });
  std::vector<rcc::GProblem> probs;
  std::vector<int> pinst, ptiles;
  int t0 = 0;
  for (int q : order) {
    rcc::GProblem P = all[q];
    P.tile0 = t0;
    t0 += rcc::gproblem_tiles(P);
    probs.push_back(P);
    pinst.push_back(inst[q]);
    ptiles.push_back(rcc::gproblem_tiles(P));
  }
  b->bg_nprob = (int)probs.size();
  b->bg_maxtiles = t0;
  b->bg_bn = bn;
  b->bg_ord = ord;
  if (cudaMemcpy(b->d_probs, probs.data(), probs.size() * sizeof(rcc::GProblem), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(b->d_pinst, pinst.data(), pinst.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_ptiles, ptiles.data(), ptiles.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_total, &t0, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return bfail(b, RCCSDT_ERR_CUDA, "batch GEMM table upload failed");
  return 0;
}

int launch_batch_gemm(rccsdt_batch* b, cudaStream_t s) {
  if (rcc::launch_gemm_tc_grouped_dev(b->bg_kind, (const rcc::GProblem*)b->d_probs, b->bg_nprob, b->bg_maxtiles,
                                      (const int*)b->d_total, 0, b->bg_bn, (int*)b->d_bflag, b->opt.watchdog_cycles, s))
    return bfail(b, RCCSDT_ERR_ARG, "batch GEMM configuration unsupported");
  return 0;
}

// Times the candidate launch shapes of the batch-wide grouped GEMM on its table (all
// problems active; the values in the panels do not matter for the time) and keeps
// the fastest.  The first candidate is the fixed shape (256-wide tiles, longest K first).
int tune_batch_gemm(rccsdt_batch* b) {
  const int cands[4][2] = {{256, 0}, {128, 0}, {256, 1}, {128, 1}};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return bfail(b, RCCSDT_ERR_CUDA, "event creation failed");
  double best = 1e300;
  int bi = 0, st = 0;
  const int ncand = b->opt.autotune ? 4 : 1;
  for (int k = 0; k < ncand && !st; ++k) {
    if ((st = batch_table(b, cands[k][0], cands[k][1]))) break;
    if ((st = launch_batch_gemm(b, b->run))) break;
    cudaEventRecord(e0, b->run);
    for (int r = 0; r < 2 && !st; ++r) st = launch_batch_gemm(b, b->run);
    cudaEventRecord(e1, b->run);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = bfail(b, RCCSDT_ERR_CUDA, "batch GEMM tuning launch failed");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (k == 0) b->bg_fixed_ms = ms / 2.0;
    if (ms / 2.0 < best) {
      best = ms / 2.0;
      bi = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  b->bg_ms = best;
  // the tuning launches may have set the flag on garbage panels: clear it
  if (cudaMemset(b->d_bflag, 0, sizeof(int)) != cudaSuccess) return bfail(b, RCCSDT_ERR_CUDA, "flag reset failed");
  return batch_table(b, cands[bi][0], cands[bi][1]);
}

// Captures the bodies of one SWITCH row: part < 0 whole bodies, else that part.
int capture_bodies(rccsdt_batch* b, int i, cudaGraph_t* bodies, int part) {
  rccsdt_ctx* c = b->inst[i];
  const bool split = rcc::split_opt(b->opt);
  for (int code = 0; code < kBodies; ++code) {
    const bool unused = (!split && (code == rcc::kEvalF64 || code == rcc::kStepF64 || code == rcc::kStepMid)) ||
                        (code == rcc::kStepMid && !rcc::has_mid(b->opt)) ||
                        (part == 1 && !b->gcode[(size_t)i * kBodies + code]);
    if (unused) {
      cudaGraphNode_t e;
      cudaGraphAddEmptyNode(&e, bodies[code], nullptr, 0);
      continue;
    }
    rcc::ctx_set_stream(c, b->run);
    rcc::ctx_begin_capture(c);
    const long long l0 = rcc::g_launch_count;
    if (cudaStreamBeginCaptureToGraph(b->run, bodies[code], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess) {
      rcc::ctx_set_stream(c, b->stream);
      return bfail(b, RCCSDT_ERR_CUDA, "capture start failed");
    }
    const int st = part < 0 ? rcc::ctx_enqueue_code(c, code) : rcc::ctx_enqueue_part(c, code, part);
    cudaGraph_t out = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->run, &out);
    b->body_launches[(size_t)i * kBodies + code] += rcc::g_launch_count - l0;
    rcc::g_launch_count = l0;  // captured, not run: counted when a launch executes them
    rcc::ctx_set_stream(c, b->stream);
    rcc::ctx_reset_precision(c);
    if (st) return bfail(b, st, std::string("instance ") + std::to_string(i) + ": " + rccsdt_last_error(c));
    if (ce != cudaSuccess) return bfail(b, RCCSDT_ERR_CUDA, std::string("capture failed: ") + cudaGetErrorString(ce));
    size_t cnt = 0;
    cudaGraphGetNodes(bodies[code], nullptr, &cnt);
    if (cnt == 0) {
      cudaGraphNode_t e;
      cudaGraphAddEmptyNode(&e, bodies[code], nullptr, 0);
    }
  }
  return 0;
}

// One row of SWITCH nodes (handles h0 .. h0 + n - 1), each depending on `deps`.
int add_switch_row(rccsdt_batch* b, cudaGraph_t g, const std::vector<cudaGraphConditionalHandle>& handles, int h0,
                   const cudaGraphNode_t* deps, size_t ndeps, int part, std::vector<cudaGraphNode_t>* row) {
  row->resize(b->n);
  for (int i = 0; i < b->n; ++i) {
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = handles[h0 + i];
    p.conditional.type = cudaGraphCondTypeSwitch;
    p.conditional.size = kBodies;
    if (cudaGraphAddNode(&(*row)[i], g, deps, nullptr, ndeps, &p) != cudaSuccess)
      return bfail(b, RCCSDT_ERR_CUDA, "conditional node failed");
    const int st = capture_bodies(b, i, p.conditional.phGraph_out, part);
    if (st) return st;
  }
  return 0;
}

// Builds and instantiates the batch graph (once per batch).
int build_graph(rccsdt_batch* b) {
  auto t0 = std::chrono::steady_clock::now();
  const int n = b->n;
  if (b->bgemm) {
    const int st = tune_batch_gemm(b);
    if (st) return st;
  }
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return bfail(b, RCCSDT_ERR_CUDA, "cudaGraphCreate failed");
  b->graph = g;
  const int nh = b->bgemm ? 2 * n : n;
  std::vector<cudaGraphConditionalHandle> handles(nh);
  std::vector<unsigned long long> hraw(nh);
  for (int h = 0; h < nh; ++h) {
    if (cudaGraphConditionalHandleCreate(&handles[h], g, kSkip, cudaGraphCondAssignDefault) != cudaSuccess)
      return bfail(b, RCCSDT_ERR_CUDA, "conditional handle creation failed");
    hraw[h] = (unsigned long long)handles[h];
  }
  if (cudaMemcpy(b->d_handles, hraw.data(), sizeof(unsigned long long) * nh, cudaMemcpyHostToDevice) != cudaSuccess)
    return bfail(b, RCCSDT_ERR_CUDA, "handle upload failed");
  // control kernel: every SWITCH takes its instance's code
  cudaGraphNode_t nctrl;
  {
    cudaKernelNodeParams kp = {};
    const unsigned long long* hp = (const unsigned long long*)b->d_handles;
    const int* cp = (const int*)b->d_codes;
    int nn = n, nnh = nh;
    void* args[] = {&hp, &cp, &nn, &nnh};
    kp.func = (void*)k_batch_switch;
    kp.gridDim = dim3((unsigned)((nh + 127) / 128));
    kp.blockDim = dim3(128);
    kp.kernelParams = args;
    if (cudaGraphAddKernelNode(&nctrl, g, nullptr, 0, &kp) != cudaSuccess)
      return bfail(b, RCCSDT_ERR_CUDA, "control node failed");
  }
  std::fill(b->body_launches.begin(), b->body_launches.end(), 0);
  std::vector<cudaGraphNode_t> last;
  if (!b->bgemm) {
    // one SWITCH per instance, bodies captured from the instance's own launch sequence
    const int st = add_switch_row(b, g, handles, 0, &nctrl, 1, -1, &last);
    if (st) return st;
  } else {
    cudaGraphNode_t ntab;
    {
      cudaKernelNodeParams kp = {};
      rcc::GProblem* pp = (rcc::GProblem*)b->d_probs;
      const int* pi = (const int*)b->d_pinst;
      const int* pt = (const int*)b->d_ptiles;
      int np = b->bg_nprob;
      const int* cp = (const int*)b->d_codes;
      const int* gc = (const int*)b->d_gcode;
      int* tot = (int*)b->d_total;
      void* args[] = {&pp, &pi, &pt, &np, &cp, &gc, &tot};
      kp.func = (void*)k_batch_table;
      kp.gridDim = dim3(1);
      kp.blockDim = dim3(32);
      kp.kernelParams = args;
      if (cudaGraphAddKernelNode(&ntab, g, &nctrl, 1, &kp) != cudaSuccess)
        return bfail(b, RCCSDT_ERR_CUDA, "table node failed");
    }
    std::vector<cudaGraphNode_t> rowA;
    int st = add_switch_row(b, g, handles, 0, &ntab, 1, 0, &rowA);
    if (st) return st;
    // the batch-wide grouped GEMM, captured into a child graph
    cudaGraph_t gg = nullptr;
    if (cudaStreamBeginCapture(b->run, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return bfail(b, RCCSDT_ERR_CUDA, "capture start failed");
    st = launch_batch_gemm(b, b->run);
    const cudaError_t ce = cudaStreamEndCapture(b->run, &gg);
    if (st) return st;
    if (ce != cudaSuccess) return bfail(b, RCCSDT_ERR_CUDA, "batch GEMM capture failed");
    cudaGraphNode_t ngemm;
    const cudaError_t ae = cudaGraphAddChildGraphNode(&ngemm, g, rowA.data(), (size_t)n, gg);
    cudaGraphDestroy(gg);
    if (ae != cudaSuccess) return bfail(b, RCCSDT_ERR_CUDA, "batch GEMM node failed");
    st = add_switch_row(b, g, handles, n, &ngemm, 1, 1, &last);
    if (st) return st;
  }
  // gather kernel after every SWITCH
  {
    cudaGraphNode_t ng;
    cudaKernelNodeParams kp = {};
    const double* const* sp = (const double* const*)b->d_scal;
    int nn = n;
    const int* bf = (const int*)b->d_bflag;
    double* op = (double*)b->d_out;
    void* args[] = {&sp, &nn, &bf, &op};
    kp.func = (void*)k_batch_gather;
    kp.gridDim = dim3((unsigned)((n + 127) / 128));
    kp.blockDim = dim3(128);
    kp.kernelParams = args;
    if (cudaGraphAddKernelNode(&ng, g, last.data(), (size_t)n, &kp) != cudaSuccess)
      return bfail(b, RCCSDT_ERR_CUDA, "gather node failed");
  }
  b->capture_ms = ms_since(t0);
  size_t nodes = 0;
  cudaGraphGetNodes(g, nullptr, &nodes);
  b->graph_nodes = (long long)nodes;
  t0 = std::chrono::steady_clock::now();
  const cudaError_t ie = cudaGraphInstantiate(&b->exec, g, 0);
  if (ie != cudaSuccess) return bfail(b, RCCSDT_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(ie));
  if (cudaGraphUpload(b->exec, b->run) != cudaSuccess || cudaStreamSynchronize(b->run) != cudaSuccess)
    return bfail(b, RCCSDT_ERR_CUDA, "graph upload failed");
  b->instantiate_ms = ms_since(t0);
  b->built = 1;
  return 0;
}
#endif

// Runs the bodies selected by h_codes for one iteration of the batch and leaves
// every instance's scalars in h_out.
int run_once(rccsdt_batch* b) {
  const int n = b->n;
#ifdef RCC_HOSTSIM
  // the graph's order with the bodies run directly: every part-0 body, the grouped
  // GEMMs of the instances on the grouped path, every part-1 body
  for (int part = 0; part < 3; ++part)
    for (int i = 0; i < n; ++i) {
      const int code = b->h_codes[i];
      if (code >= kSkip) continue;
      rccsdt_ctx* c = b->inst[i];
      const bool grouped = b->bgemm && b->gcode[(size_t)i * kBodies + code];
      int st = 0;
      rcc::ctx_begin_capture(c);
      if (!b->bgemm) {
        if (part == 0) st = rcc::ctx_enqueue_code(c, code);
      } else if (part == 0) {
        st = rcc::ctx_enqueue_part(c, code, 0);
      } else if (part == 1 && grouped) {
        st = rcc::ctx_run_grouped_gemm(c);
      } else if (part == 2 && grouped) {
        st = rcc::ctx_enqueue_part(c, code, 1);
      }
      rcc::ctx_reset_precision(c);
      if (!st && part == 2) st = rcc::ctx_read_scalars(c, b->h_out + (size_t)i * kOutStride);
      if (st) return bfail(b, st, std::string("instance ") + std::to_string(i) + ": " + rccsdt_last_error(c));
    }
  return 0;
#else
  if (!b->built) {
    const int st = build_graph(b);
    if (st) return st;
  }
  if (cudaMemcpyAsync(b->d_codes, b->h_codes, sizeof(int) * n, cudaMemcpyHostToDevice, b->run) != cudaSuccess)
    return bfail(b, RCCSDT_ERR_CUDA, "code upload failed");
  cudaEventRecord(b->ev0, b->run);
  const cudaError_t le = cudaGraphLaunch(b->exec, b->run);
  cudaEventRecord(b->ev1, b->run);
  if (le != cudaSuccess) return bfail(b, RCCSDT_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(le));
  if (cudaMemcpyAsync(b->h_out, b->d_out, sizeof(double) * kOutStride * n, cudaMemcpyDeviceToHost, b->run) !=
          cudaSuccess ||
      cudaStreamSynchronize(b->run) != cudaSuccess)
    return bfail(b, RCCSDT_ERR_CUDA, std::string("batch iteration failed: ") + cudaGetErrorString(cudaGetLastError()));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->ev0, b->ev1);
  b->launch_ms.push_back(ms);
  b->device_ms += ms;
  return 0;
#endif
}

}  // namespace

#define RCC_API extern "C" __attribute__((visibility("default")))

RCC_API int rccsdt_batch_create(int n, const int* o, const int* v, const int* naux, const rccsdt_options* opt,
                                void* stream, rccsdt_batch** out) {
  if (!out) return RCCSDT_ERR_ARG;
  *out = nullptr;
  if (n < 1 || !o || !v || !naux) return RCCSDT_ERR_ARG;
  rccsdt_options def;
  rccsdt_options_default(&def);
  auto* b = new rccsdt_batch();
  b->n = n;
  b->opt = opt ? *opt : def;
  b->stream = (cudaStream_t)stream;
  b->state.assign(n, SolveState());
  b->body_launches.assign((size_t)n * kBodies, 0);
  int st = 0;
  for (int i = 0; i < n && !st; ++i) {
    rccsdt_ctx* c = nullptr;
    st = rccsdt_create(o[i], v[i], naux[i], &b->opt, stream, &c);
    if (!st) {
      if (n > 1) rcc::ctx_set_concurrent(c, 1);
      b->inst.push_back(c);
    }
  }
  // batch-wide grouped GEMM when the instances share a split precision and at least
  // one of them takes the grouped path
  if (!st && rcc::split_opt(b->opt)) {
    b->gcode.assign((size_t)n * kBodies, 0);
    for (int i = 0; i < n; ++i) {
      const int kind = rcc::ctx_grouped_kind(b->inst[i]);
      if (kind < 0) continue;
      b->bgemm = 1;
      b->bg_kind = kind;
      rcc::ctx_set_batch_gemm(b->inst[i], 1);
      for (int code = 0; code < kBodies; ++code)
        b->gcode[(size_t)i * kBodies + code] = rcc::ctx_body_grouped(b->inst[i], code);
    }
  }
#ifdef RCC_HOSTSIM
  if (!st) {
    b->h_codes = (int*)calloc(n, sizeof(int));
    b->h_out = (double*)calloc((size_t)n * kOutStride, sizeof(double));
  }
#else
  if (!st) {
    if (cudaStreamCreateWithFlags(&b->run, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess ||
        cudaMalloc(&b->d_handles, sizeof(unsigned long long) * 2 * n) != cudaSuccess ||
        cudaMalloc(&b->d_codes, sizeof(int) * n) != cudaSuccess ||
        cudaMalloc(&b->d_scal, sizeof(void*) * n) != cudaSuccess ||
        cudaMalloc(&b->d_out, sizeof(double) * kOutStride * n) != cudaSuccess ||
        cudaHostAlloc((void**)&b->h_codes, sizeof(int) * n, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void**)&b->h_out, sizeof(double) * kOutStride * n, cudaHostAllocDefault) != cudaSuccess)
      st = RCCSDT_ERR_OOM;
    if (!st) {
      std::vector<const double*> sp(n);
      for (int i = 0; i < n; ++i) sp[i] = rcc::ctx_scalars(b->inst[i]);
      if (cudaMemcpy(b->d_scal, sp.data(), sizeof(void*) * n, cudaMemcpyHostToDevice) != cudaSuccess)
        st = RCCSDT_ERR_CUDA;
    }
    if (!st && cudaMalloc(&b->d_bflag, sizeof(int)) == cudaSuccess) {
      cudaMemset(b->d_bflag, 0, sizeof(int));
    } else if (!st) {
      st = RCCSDT_ERR_OOM;
    }
    if (!st && b->bgemm) {
      size_t np = 0;
      for (int i = 0; i < n; ++i) {
        std::vector<rcc::GProblem> pr;
        if (rcc::ctx_grouped_kind(b->inst[i]) >= 0 && !rcc::ctx_grouped_problems(b->inst[i], 256, &pr))
          np += pr.size();
      }
      if (cudaMalloc(&b->d_probs, sizeof(rcc::GProblem) * (np + 1)) != cudaSuccess ||
          cudaMalloc(&b->d_pinst, sizeof(int) * (np + 1)) != cudaSuccess ||
          cudaMalloc(&b->d_ptiles, sizeof(int) * (np + 1)) != cudaSuccess ||
          cudaMalloc(&b->d_total, sizeof(int)) != cudaSuccess ||
          cudaMalloc(&b->d_gcode, sizeof(int) * b->gcode.size()) != cudaSuccess ||
          cudaMemcpy(b->d_gcode, b->gcode.data(), sizeof(int) * b->gcode.size(), cudaMemcpyHostToDevice) !=
              cudaSuccess)
        st = RCCSDT_ERR_OOM;
    }
  }
#endif
  if (st) {
    rccsdt_batch_destroy(b);
    return st;
  }
  *out = b;
  return RCCSDT_OK;
}

RCC_API rccsdt_ctx* rccsdt_batch_instance(rccsdt_batch* b, int i) {
  if (!b || i < 0 || i >= b->n) return nullptr;
  return b->inst[i];
}

RCC_API int rccsdt_batch_solve(rccsdt_batch* b, double* e_corr, int* iterations, double* final_norm, int* status) {
  if (!b) return RCCSDT_ERR_ARG;
  const int n = b->n;
  for (int i = 0; i < n; ++i) {
    const int st = rcc::ctx_ready(b->inst[i]);
    if (st) return bfail(b, st, std::string("instance ") + std::to_string(i) + ": " + rccsdt_last_error(b->inst[i]));
  }
  if (!b->built)
    for (int i = 0; i < n; ++i) {
      const int st = rcc::ctx_prepare(b->inst[i]);
      if (st) return bfail(b, st, std::string("instance ") + std::to_string(i) + ": " + rccsdt_last_error(b->inst[i]));
    }
  b->state.assign(n, SolveState());
  b->launches = b->kernels = 0;
  b->device_ms = b->flop = 0.0;
  b->launch_ms.clear();
  for (;;) {
    int active = 0;
    for (int i = 0; i < n; ++i) {
      b->h_codes[i] = rcc::next_code(b->opt, b->state[i]);
      if (b->h_codes[i] < kSkip) ++active;
    }
    if (!active) break;
    const int st = run_once(b);
    if (st) return st;
    b->launches += 1;
    b->kernels += b->bgemm ? 4 : 2;  // control, gather (and the table kernel and batch GEMM)
    for (int i = 0; i < n; ++i) {
      const int code = b->h_codes[i];
      if (code >= kSkip) continue;
      b->kernels += b->body_launches[(size_t)i * kBodies + code];
      int o = 0, v = 0;
      rcc::ctx_dims(b->inst[i], &o, &v);
      b->flop += 2.0 * rccsdt_iteration_fma(o, v);
      rcc::take_result(b->opt, b->state[i], code, b->h_out + (size_t)i * kOutStride);
    }
  }
#ifndef RCC_HOSTSIM
  rcc::g_launch_count += b->kernels;
#endif
  int worst = RCCSDT_OK;
  for (int i = 0; i < n; ++i) {
    const SolveState& s = b->state[i];
    if (e_corr) e_corr[i] = s.e;
    if (iterations) iterations[i] = s.it;
    if (final_norm) final_norm[i] = s.norm;
    if (status) status[i] = s.status;
    if (s.status < 0 && (worst >= 0 || s.status < worst)) worst = s.status;
    else if (s.status > 0 && worst == RCCSDT_OK) worst = s.status;
  }
  if (worst < 0) b->err = "an instance failed (see the per-instance status)";
  return worst;
}

RCC_API int rccsdt_batch_stats(const rccsdt_batch* b, double* out, int cap) {
  if (!b || !out) return RCCSDT_ERR_ARG;
  const double v[14] = {(double)b->launches, b->device_ms, b->flop, (double)b->kernels,
                        (double)b->graph_nodes, b->capture_ms, b->instantiate_ms,
                        b->launch_ms.empty() ? 0.0 : b->launch_ms.front(), (double)b->bgemm,
                        (double)b->bg_nprob, (double)b->bg_maxtiles, (double)b->bg_bn, b->bg_ms, b->bg_fixed_ms};
  const int k = cap < 14 ? cap : 14;
  for (int q = 0; q < k; ++q) out[q] = v[q];
  return k;
}

RCC_API int rccsdt_batch_launch_times(const rccsdt_batch* b, double* ms, int cap) {
  if (!b || !ms) return RCCSDT_ERR_ARG;
  const int k = (int)b->launch_ms.size() < cap ? (int)b->launch_ms.size() : cap;
  for (int q = 0; q < k; ++q) ms[q] = b->launch_ms[q];
  return k;
}

RCC_API const char* rccsdt_batch_last_error(const rccsdt_batch* b) { return b ? b->err.c_str() : "null batch"; }

RCC_API void rccsdt_batch_destroy(rccsdt_batch* b) {
  if (!b) return;
#ifdef RCC_HOSTSIM
  free(b->h_codes);
  free(b->h_out);
#else
  if (b->run) cudaStreamSynchronize(b->run);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  cudaFree(b->d_handles);
  cudaFree(b->d_probs);
  cudaFree(b->d_pinst);
  cudaFree(b->d_ptiles);
  cudaFree(b->d_total);
  cudaFree(b->d_gcode);
  cudaFree(b->d_bflag);
  cudaFree(b->d_codes);
  cudaFree(b->d_scal);
  cudaFree(b->d_out);
  if (b->h_codes) cudaFreeHost(b->h_codes);
  if (b->h_out) cudaFreeHost(b->h_out);
  if (b->run) cudaStreamDestroy(b->run);
#endif
  for (rccsdt_ctx* c : b->inst) rccsdt_destroy(c);
  delete b;
}
