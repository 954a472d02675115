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
__global__ void k_batch_switch(const unsigned long long* __restrict__ handles, const int* __restrict__ codes, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cudaGraphSetConditional((cudaGraphConditionalHandle)handles[i], (unsigned)codes[i]);
}

__global__ void k_batch_gather(const double* const* __restrict__ scal, int n, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* s = scal[i];
  double* o = out + (size_t)i * kOutStride;
  o[0] = s[0];
  o[1] = s[1];
  o[2] = s[2];
  o[3] = 0.0;
  o[4] = s[4];
  o[5] = (double)((const int*)(s + 1000))[0];
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

// Builds and instantiates the batch graph (once per batch).
int build_graph(rccsdt_batch* b) {
  auto t0 = std::chrono::steady_clock::now();
  const int n = b->n;
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return bfail(b, RCCSDT_ERR_CUDA, "cudaGraphCreate failed");
  b->graph = g;
  std::vector<unsigned long long> handles(n);
  for (int i = 0; i < n; ++i) {
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, kSkip, cudaGraphCondAssignDefault) != cudaSuccess)
      return bfail(b, RCCSDT_ERR_CUDA, "conditional handle creation failed");
    handles[i] = (unsigned long long)h;
  }
  if (cudaMemcpy(b->d_handles, handles.data(), sizeof(unsigned long long) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return bfail(b, RCCSDT_ERR_CUDA, "handle upload failed");
  // control kernel
  cudaGraphNode_t nctrl;
  {
    cudaKernelNodeParams kp = {};
    const unsigned long long* hp = (const unsigned long long*)b->d_handles;
    const int* cp = (const int*)b->d_codes;
    int nn = n;
    void* args[] = {&hp, &cp, &nn};
    kp.func = (void*)k_batch_switch;
    kp.gridDim = dim3((unsigned)((n + 127) / 128));
    kp.blockDim = dim3(128);
    kp.kernelParams = args;
    if (cudaGraphAddKernelNode(&nctrl, g, nullptr, 0, &kp) != cudaSuccess)
      return bfail(b, RCCSDT_ERR_CUDA, "control node failed");
  }
  // one SWITCH per instance, bodies captured from the instance's own launch sequence
  std::vector<cudaGraphNode_t> sw(n);
  const bool split = rcc::split_opt(b->opt);
  for (int i = 0; i < n; ++i) {
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = (cudaGraphConditionalHandle)handles[i];
    p.conditional.type = cudaGraphCondTypeSwitch;
    p.conditional.size = kBodies;
    if (cudaGraphAddNode(&sw[i], g, &nctrl, nullptr, 1, &p) != cudaSuccess)
      return bfail(b, RCCSDT_ERR_CUDA, "conditional node failed");
    cudaGraph_t* bodies = p.conditional.phGraph_out;
    rccsdt_ctx* c = b->inst[i];
    for (int code = 0; code < kBodies; ++code) {
      const bool unused = (!split && (code == rcc::kEvalF64 || code == rcc::kStepF64 || code == rcc::kStepMid)) ||
                          (code == rcc::kStepMid && !rcc::has_mid(b->opt));
      if (unused) {
        cudaGraphNode_t e;
        cudaGraphAddEmptyNode(&e, bodies[code], nullptr, 0);
        b->body_launches[(size_t)i * kBodies + code] = 0;
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
      const int st = rcc::ctx_enqueue_code(c, code);
      cudaGraph_t out = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(b->run, &out);
      b->body_launches[(size_t)i * kBodies + code] = rcc::g_launch_count - l0;
      rcc::g_launch_count = l0;  // captured, not run: counted when a launch executes them
      rcc::ctx_set_stream(c, b->stream);
      rcc::ctx_reset_precision(c);
      if (st) return bfail(b, st, std::string("instance ") + std::to_string(i) + ": " + rccsdt_last_error(c));
      if (ce != cudaSuccess)
        return bfail(b, RCCSDT_ERR_CUDA, std::string("capture failed: ") + cudaGetErrorString(ce));
    }
  }
  // gather kernel after every SWITCH
  {
    cudaGraphNode_t ng;
    cudaKernelNodeParams kp = {};
    const double* const* sp = (const double* const*)b->d_scal;
    int nn = n;
    double* op = (double*)b->d_out;
    void* args[] = {&sp, &nn, &op};
    kp.func = (void*)k_batch_gather;
    kp.gridDim = dim3((unsigned)((n + 127) / 128));
    kp.blockDim = dim3(128);
    kp.kernelParams = args;
    if (cudaGraphAddKernelNode(&ng, g, sw.data(), (size_t)n, &kp) != cudaSuccess)
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
  for (int i = 0; i < n; ++i) {
    const int code = b->h_codes[i];
    if (code >= kSkip) continue;
    rccsdt_ctx* c = b->inst[i];
    rcc::ctx_begin_capture(c);
    int st = rcc::ctx_enqueue_code(c, code);
    rcc::ctx_reset_precision(c);
    if (!st) st = rcc::ctx_read_scalars(c, b->h_out + (size_t)i * kOutStride);
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
#ifdef RCC_HOSTSIM
  if (!st) {
    b->h_codes = (int*)calloc(n, sizeof(int));
    b->h_out = (double*)calloc((size_t)n * kOutStride, sizeof(double));
  }
#else
  if (!st) {
    if (cudaStreamCreateWithFlags(&b->run, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess ||
        cudaMalloc(&b->d_handles, sizeof(unsigned long long) * n) != cudaSuccess ||
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
    b->kernels += 2;
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
  const double v[8] = {(double)b->launches, b->device_ms, b->flop, (double)b->kernels,
                       (double)b->graph_nodes, b->capture_ms, b->instantiate_ms,
                       b->launch_ms.empty() ? 0.0 : b->launch_ms.front()};
  const int k = cap < 8 ? cap : 8;
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
