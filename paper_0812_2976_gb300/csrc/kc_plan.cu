// kc_plan.cu -- the ragged-batch plan: host-side runtime around the
// persistent kernel of kc_ragged.cu (descriptor upload, longest-first
// ordering, observation conversion, work queue, CUDA graph capture and
// replay, launch-shape autotuning).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <numeric>
#include <vector>

#include "kc_internal.h"
#include "kc_ragged.h"

using kc::cuda_status;
using kc::fail;
using kc::ok;

// Streams a plan can run on, each with its own work queue and graph.
constexpr int kPlanMaxStreams = 64;

// What one stream needs to run the plan: its work-queue counter (so that
// runs on different streams do not take each other's systems) and the graph
// captured with that counter, pointed at the last run's arrays.
struct PlanStream {
  cudaStream_t stream = nullptr;
  unsigned long long *queue = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t kernel_node = nullptr;
  const double *g_params = nullptr;
  void *g_chi2 = nullptr, *g_grad = nullptr;
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    kernel_node = nullptr;
  }
};

struct kc_plan {
  int device = 0;
  int mode = KC_MIXED;
  bool grad = false;
  double t0 = 0.0, jitter = 0.0;
  int64_t n_sys = 0, n_obs = 0, n_par = 0;
  int64_t *d_obs_off = nullptr, *d_par_off = nullptr, *d_order = nullptr;
  int32_t *d_n_pl = nullptr;
  double *d_t_ref = nullptr;
  void *d_obs_a = nullptr, *d_obs_b = nullptr;
  unsigned long long *d_queue = nullptr;  // kPlanMaxStreams counters
  bool obs_ready = false;
  int grid = 0, block = 256;
  std::vector<PlanStream> streams;       // the streams the plan has run on
  cudaStream_t cap_stream = nullptr;      // private stream graphs are captured on
  std::mutex mu;

  kc::RaggedDev dev() const {
    return kc::RaggedDev{d_obs_off, d_par_off, d_n_pl, d_order, d_t_ref, n_sys, t0,
                         kc::invalid_counter(), n_obs, n_par};
  }
  void drop_graph() {
    for (PlanStream &ps : streams) ps.drop_graph();
  }
  // The entry of stream st (created on first use, with the next free
  // counter); NULL when kPlanMaxStreams streams already have one.
  PlanStream *stream_for(cudaStream_t st) {
    for (PlanStream &ps : streams)
      if (ps.stream == st) return &ps;
    if ((int)streams.size() >= kPlanMaxStreams) return nullptr;
    streams.emplace_back();
    streams.back().stream = st;
    streams.back().queue = d_queue + streams.size() - 1;
    return &streams.back();
  }
  void release() {
    drop_graph();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
    for (void *p : {(void *)d_obs_off, (void *)d_par_off, (void *)d_order, (void *)d_n_pl,
                    (void *)d_t_ref, d_obs_a, d_obs_b, (void *)d_queue})
      if (p) cudaFree(p);
  }
};

namespace {

kc_status too_many_streams() {
  return fail(KC_ERR_UNSUPPORTED, "kc_plan_run: the plan has run on %d streams already",
              kPlanMaxStreams);
}

kc_status launch_direct(kc_plan *p, PlanStream *ps, const double *params, void *chi2, void *grad,
                        cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ps->queue, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess)
    e = kc::ragged_launch(p->dev(), p->mode, p->grad, p->d_obs_a, p->d_obs_b, params, chi2, grad,
                          ps->queue, p->grid, p->block, st);
  return cuda_status(e, "kc_plan_run");
}

// Records the queue reset and the kernel into a graph on the plan's private
// stream (the caller's stream may be the legacy default stream, which cannot
// be captured); the graph is then launched on whatever stream runs the plan.
kc_status capture(kc_plan *p, PlanStream *ps, const double *params, void *chi2, void *grad) {
  ps->drop_graph();
  cudaStream_t st = p->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status(e, "kc_plan_run: begin capture");
  cudaError_t e1 = cudaMemsetAsync(ps->queue, 0, sizeof(unsigned long long), st);
  cudaError_t e2 = kc::ragged_launch(p->dev(), p->mode, p->grad, p->d_obs_a, p->d_obs_b, params,
                                     chi2, grad, ps->queue, p->grid, p->block, st);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(st, &g);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_status(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e),
                       "kc_plan_run: capture");
  }
  size_t n = 0;
  cudaGraphGetNodes(g, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  cudaGraphGetNodes(g, nodes.data(), &n);
  cudaGraphNode_t kn = nullptr;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    cudaGraphNodeGetType(nd, &ty);
    if (ty == cudaGraphNodeTypeKernel) kn = nd;
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess || !kn) {
    cudaGraphDestroy(g);
    return cuda_status(e != cudaSuccess ? e : cudaErrorUnknown, "kc_plan_run: instantiate");
  }
  ps->graph = g;
  ps->exec = ex;
  ps->kernel_node = kn;
  ps->g_params = params;
  ps->g_chi2 = chi2;
  ps->g_grad = grad;
  return ok();
}

// Point the captured kernel at new parameter / output arrays.
kc_status retarget(kc_plan *p, PlanStream *ps, const double *params, void *chi2, void *grad) {
  cudaKernelNodeParams kp;
  cudaError_t e = cudaGraphKernelNodeGetParams(ps->kernel_node, &kp);
  if (e != cudaSuccess) return cuda_status(e, "kc_plan_run: node params");
  kc::RaggedDev d = p->dev();
  const void *oa = p->d_obs_a, *ob = p->d_obs_b;
  unsigned long long *q = ps->queue;
  void *args_mixed[] = {&d, (void *)&oa, (void *)&ob, (void *)&params, &chi2, &grad, &q};
  void *args_f64[] = {&d, (void *)&oa, (void *)&params, &chi2, &grad, &q};
  kp.kernelParams = p->mode == KC_MIXED ? args_mixed : args_f64;
  kp.extra = nullptr;
  e = cudaGraphExecKernelNodeSetParams(ps->exec, ps->kernel_node, &kp);
  if (e != cudaSuccess) return cuda_status(e, "kc_plan_run: update node");
  ps->g_params = params;
  ps->g_chi2 = chi2;
  ps->g_grad = grad;
  return ok();
}

int sm_count(int device) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
  return n > 0 ? n : 1;
}

}  // namespace

extern "C" {

kc_status kc_plan_create_ragged(kc_plan **plan, const int64_t *obs_off, const int32_t *n_pl,
                                int64_t n_sys, double t0, double jitter, kc_mode mode,
                                int want_grad) {
  if (!plan) return fail(KC_ERR_ARG, "kc_plan_create_ragged: plan is NULL");
  *plan = nullptr;
  if (n_sys < 1 || !obs_off || !n_pl)
    return fail(KC_ERR_ARG, "kc_plan_create_ragged: need n_sys >= 1, obs_off and n_pl");
  if (n_sys > (int64_t(1) << 40)) return fail(KC_ERR_ARG, "kc_plan_create_ragged: n_sys too large");
  if (mode != KC_FP64 && mode != KC_MIXED)
    return fail(KC_ERR_ARG, "kc_plan_create_ragged: bad mode");
  if (!std::isfinite(t0) || !std::isfinite(jitter))
    return fail(KC_ERR_ARG, "kc_plan_create_ragged: t0 and jitter must be finite");
  if (obs_off[0] != 0) return fail(KC_ERR_ARG, "kc_plan_create_ragged: obs_off[0] != 0");
  std::vector<int64_t> par_off(n_sys + 1, 0);
  std::vector<int64_t> work(n_sys);
  for (int64_t s = 0; s < n_sys; ++s) {
    // ordered first, so that the difference cannot overflow
    if (obs_off[s + 1] < obs_off[s])
      return fail(KC_ERR_ARG, "kc_plan_create_ragged: obs_off decreases at system %lld",
                  (long long)s);
    const int64_t n = obs_off[s + 1] - obs_off[s];
    if (n > KC_MAX_OBS)
      return fail(KC_ERR_ARG, "kc_plan_create_ragged: system %lld has %lld observations",
                  (long long)s, (long long)n);
    if (n_pl[s] < 1 || n_pl[s] > KC_MAX_PLANETS)
      return fail(KC_ERR_ARG, "kc_plan_create_ragged: system %lld has n_pl = %d", (long long)s,
                  n_pl[s]);
    par_off[s + 1] = par_off[s] + 5 * (int64_t)n_pl[s] + 1;
    work[s] = (int64_t)n_pl[s] * std::max<int64_t>(n, 1);
  }
  // Planet count first (descending), then work (descending): warps running
  // at the same time mostly execute the same unrolled body (one per planet
  // count), and the queue still ends with the smallest systems (1 planet,
  // few observations), which fill the tail.
  std::vector<int64_t> order(n_sys);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    if (n_pl[a] != n_pl[b]) return n_pl[a] > n_pl[b];
    return work[a] > work[b];
  });

  if (obs_off[n_sys] > (int64_t(1) << 40))
    return fail(KC_ERR_ARG, "kc_plan_create_ragged: more than 2^40 observations");
  kc_plan *p = new kc_plan();
  cudaGetDevice(&p->device);
  p->mode = mode;
  p->grad = want_grad != 0;
  p->t0 = t0;
  p->jitter = jitter;
  p->n_sys = n_sys;
  p->n_obs = obs_off[n_sys];
  p->n_par = par_off[n_sys];
  const size_t obs_bytes_a = p->n_obs * (mode == KC_MIXED ? sizeof(float4) : sizeof(kc::ObsR64));
  const size_t obs_bytes_b = mode == KC_MIXED ? p->n_obs * sizeof(float2) : 0;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes > 0 ? bytes : 16);
  };
  alloc((void **)&p->d_obs_off, sizeof(int64_t) * (n_sys + 1));
  alloc((void **)&p->d_par_off, sizeof(int64_t) * (n_sys + 1));
  alloc((void **)&p->d_order, sizeof(int64_t) * n_sys);
  alloc((void **)&p->d_n_pl, sizeof(int32_t) * n_sys);
  alloc((void **)&p->d_t_ref, sizeof(double) * n_sys);
  alloc(&p->d_obs_a, obs_bytes_a);
  alloc(&p->d_obs_b, obs_bytes_b);
  alloc((void **)&p->d_queue, sizeof(unsigned long long) * kPlanMaxStreams);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p->release();
    delete p;
    return fail(e == cudaErrorMemoryAllocation ? KC_ERR_NOMEM : KC_ERR_CUDA,
                "kc_plan_create_ragged: %s", cudaGetErrorString(e));
  }
  e = cudaMemcpy(p->d_obs_off, obs_off, sizeof(int64_t) * (n_sys + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_par_off, par_off.data(), sizeof(int64_t) * (n_sys + 1),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_order, order.data(), sizeof(int64_t) * n_sys, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_n_pl, n_pl, sizeof(int32_t) * n_sys, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    p->release();
    delete p;
    return cuda_status(e, "kc_plan_create_ragged: upload");
  }
  p->block = 256;
  const int per_sm = kc::ragged_max_blocks_per_sm(mode, p->grad, p->block);
  p->grid = sm_count(p->device) * (per_sm > 0 ? per_sm : 1);
  *plan = p;
  return ok();
}

kc_status kc_plan_sizes(const kc_plan *plan, int64_t *n_params, int64_t *n_obs) {
  if (!plan) return fail(KC_ERR_ARG, "kc_plan_sizes: plan is NULL");
  if (n_params) *n_params = plan->n_par;
  if (n_obs) *n_obs = plan->n_obs;
  return ok();
}

kc_status kc_plan_set_observations(kc_plan *plan, const double *t, const double *v_obs,
                                   const double *sigma, kc_stream stream) {
  if (!plan) return fail(KC_ERR_ARG, "kc_plan_set_observations: plan is NULL");
  if (plan->n_obs > 0 && (!t || !v_obs || !sigma))
    return fail(KC_ERR_ARG, "kc_plan_set_observations: NULL observation array");
  if (((uintptr_t)t | (uintptr_t)v_obs | (uintptr_t)sigma) & 7)
    return fail(KC_ERR_ARG, "kc_plan_set_observations: pointer not 8-byte aligned");
  std::lock_guard<std::mutex> lk(plan->mu);
  cudaError_t e = kc::ragged_prep(plan->dev(), plan->mode, t, v_obs, sigma,
                                  plan->jitter * plan->jitter, plan->d_obs_a, plan->d_obs_b,
                                  plan->d_t_ref, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_status(e, "kc_plan_set_observations");
  plan->obs_ready = true;
  return ok();
}

kc_status kc_plan_run(kc_plan *plan, const double *params, void *chi2_out, void *grad_out,
                      kc_stream stream) {
  if (!plan) return fail(KC_ERR_ARG, "kc_plan_run: plan is NULL");
  if (!params || !chi2_out) return fail(KC_ERR_ARG, "kc_plan_run: NULL params or chi2_out");
  if (plan->grad != (grad_out != nullptr))
    return fail(KC_ERR_ARG, "kc_plan_run: grad_out must be given exactly when the plan "
                            "was created with want_grad");
  if ((uintptr_t)params & 7) return fail(KC_ERR_ARG, "kc_plan_run: params not aligned");
  std::lock_guard<std::mutex> lk(plan->mu);
  if (!plan->obs_ready)
    return fail(KC_ERR_ARG, "kc_plan_run: kc_plan_set_observations has not been called");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  PlanStream *ps = plan->stream_for(st);
  if (!ps) return too_many_streams();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return cuda_status(e, "kc_plan_run: stream");
  if (cap != cudaStreamCaptureStatusNone)
    return launch_direct(plan, ps, params, chi2_out, grad_out, st);
  if (!ps->exec) {
    kc_status s = capture(plan, ps, params, chi2_out, grad_out);
    if (s != KC_OK) return s;
  } else if (ps->g_params != params || ps->g_chi2 != chi2_out || ps->g_grad != grad_out) {
    kc_status s = retarget(plan, ps, params, chi2_out, grad_out);
    if (s != KC_OK) return s;
  }
  return cuda_status(cudaGraphLaunch(ps->exec, st), "kc_plan_run: graph launch");
}

kc_status kc_plan_autotune(kc_plan *plan, const double *params, void *chi2_out, void *grad_out,
                           int32_t *block, int32_t *ctas_per_sm, kc_stream stream) {
  if (!plan) return fail(KC_ERR_ARG, "kc_plan_autotune: plan is NULL");
  if (!params || !chi2_out || plan->grad != (grad_out != nullptr))
    return fail(KC_ERR_ARG, "kc_plan_autotune: bad params / outputs");
  std::lock_guard<std::mutex> lk(plan->mu);
  if (!plan->obs_ready)
    return fail(KC_ERR_ARG, "kc_plan_autotune: kc_plan_set_observations has not been called");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  PlanStream *ps = plan->stream_for(st);
  if (!ps) return too_many_streams();
  const int sms = sm_count(plan->device);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_block = plan->block, best_k = std::max(1, plan->grid / sms);
  const char *env = getenv("KC_AUTOTUNE_VERBOSE");     // candidate timings to stderr
  const bool verbose = env && env[0] == '1';
  kc_status status = KC_OK;
  for (int b : {64, 128, 256}) {
    const int kmax = kc::ragged_max_blocks_per_sm(plan->mode, plan->grad, b);
    for (int k = 1; k <= kmax && status == KC_OK; ++k) {
      plan->block = b;
      plan->grid = sms * k;
      status = launch_direct(plan, ps, params, chi2_out, grad_out, st);   // warm-up
      float tmin = 1e30f;
      for (int rep = 0; rep < 2 && status == KC_OK; ++rep) {
        cudaEventRecord(e0, st);
        status = launch_direct(plan, ps, params, chi2_out, grad_out, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        tmin = std::min(tmin, ms);
      }
      if (verbose)
        fprintf(stderr, "kc_plan_autotune: block %3d ctas/SM %d: %9.2f us\n", b, k, 1e3 * tmin);
      if (status == KC_OK && tmin < best) {
        best = tmin;
        best_block = b;
        best_k = k;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan->block = best_block;
  plan->grid = sms * best_k;
  plan->drop_graph();
  if (status != KC_OK) return status;
  if (block) *block = best_block;
  if (ctas_per_sm) *ctas_per_sm = best_k;
  return ok();
}

void kc_plan_destroy(kc_plan *plan) {
  if (!plan) return;
  {
    std::lock_guard<std::mutex> lk(plan->mu);
    plan->release();
  }
  delete plan;
}

}  // extern "C"
