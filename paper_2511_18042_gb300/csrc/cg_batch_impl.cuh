// Batched advance of many independent grids (included by cg_api.cu).
// cg_multi_step forks the caller's stream into a pool of internal streams,
// runs each member's CFL time step and RK3 step on one of them (members are
// independent: each solver owns its scratch), and joins back.  cg_batch
// captures one such call into a CUDA graph and replays it, so a step of a
// whole batch of uneven grids costs one graph launch on the host;
// cg_batch_autotune picks the members' tile shapes and the pool width.

namespace {

constexpr int kPoolStreams = 16;     // default width
constexpr int kMaxPoolStreams = 32;  // streams created per thread and device

struct StreamPool {
  int dev = -1;
  cudaStream_t s[kMaxPoolStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kMaxPoolStreams] = {};
};
thread_local StreamPool g_pool;

int pool_ready() {
  int dev = 0;
  CG_CUDA(cudaGetDevice(&dev));
  if (g_pool.dev == dev) return CG_OK;
  for (int i = 0; i < kMaxPoolStreams; ++i) {
    CG_CUDA(cudaStreamCreateWithFlags(&g_pool.s[i], cudaStreamNonBlocking));
    CG_CUDA(cudaEventCreateWithFlags(&g_pool.join[i], cudaEventDisableTiming));
  }
  CG_CUDA(cudaEventCreateWithFlags(&g_pool.fork, cudaEventDisableTiming));
  g_pool.dev = dev;
  return CG_OK;
}

int multi_step(cg_solver* const* solvers, double* const* states, int count, cudaStream_t st,
               int width = kPoolStreams) {
  int rc = pool_ready();
  if (rc) return rc;
  if (width < 1) width = 1;
  if (width > kMaxPoolStreams) width = kMaxPoolStreams;
  int ns = count < width ? count : width;
  CG_CUDA(cudaEventRecord(g_pool.fork, st));
  for (int i = 0; i < ns; ++i) CG_CUDA(cudaStreamWaitEvent(g_pool.s[i], g_pool.fork, 0));
  // largest members first, round robin over the streams
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return solvers[a]->N > solvers[b]->N; });
  for (int k = 0; k < count; ++k) {
    int i = order[k];
    cg_solver* s = solvers[i];
    cudaStream_t si = g_pool.s[k % ns];
    DISPATCH_ND(s, cfl_launch, s, states[i], s->dt, nullptr, 0.0, si);
    rc = DISPATCH_ND(s, rk3, s, states[i], si);
    if (rc) return rc;
  }
  for (int i = 0; i < ns; ++i) {
    CG_CUDA(cudaEventRecord(g_pool.join[i], g_pool.s[i]));
    CG_CUDA(cudaStreamWaitEvent(st, g_pool.join[i], 0));
  }
  return CG_OK;
}

}  // namespace

struct cg_batch {
  std::vector<cg_solver*> solvers;
  std::vector<double*> states;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int warm = 0;
  int width = kPoolStreams;  // streams the members are spread over
};

extern "C" {

CG_API int cg_multi_step(cg_solver* const* solvers, double* const* states, int count, void* stream) {
  if (!solvers || !states || count < 1) return fail(CG_ERR_INVALID_ARG, "need at least one solver");
  for (int i = 0; i < count; ++i)
    if (!solvers[i] || !states[i]) return fail(CG_ERR_INVALID_ARG, "null solver or state %d", i);
  int rc = multi_step(solvers, states, count, (cudaStream_t)stream);
  if (rc) return rc;
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}

CG_API int cg_batch_create(int count, cg_solver* const* solvers, double* const* states, cg_batch** out) {
  if (!solvers || !states || !out || count < 1) return fail(CG_ERR_INVALID_ARG, "bad arguments");
  cg_batch* b = new (std::nothrow) cg_batch();
  if (!b) return fail(CG_ERR_OOM, "host allocation failed");
  b->solvers.assign(solvers, solvers + count);
  b->states.assign(states, states + count);
  for (int i = 0; i < count; ++i)
    if (!solvers[i] || !states[i]) {
      delete b;
      return fail(CG_ERR_INVALID_ARG, "null solver or state %d", i);
    }
  *out = b;
  return CG_OK;
}

CG_API int cg_batch_step(cg_batch* b, void* stream) {
  if (!b) return fail(CG_ERR_INVALID_ARG, "null batch");
  cudaStream_t st = (cudaStream_t)stream;
  int count = (int)b->solvers.size();
  if (!b->warm) {
    // first step runs eagerly: one-time kernel attributes and stream pool set-up
    int rc = multi_step(b->solvers.data(), b->states.data(), count, st, b->width);
    if (rc) return rc;
    b->warm = 1;
    return CG_OK;
  }
  if (!b->exec) {
    // capture one batch step; later calls replay it
    if (st == nullptr) return fail(CG_ERR_INVALID_ARG, "graph replay needs a non-default stream");
    CG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = multi_step(b->solvers.data(), b->states.data(), count, st, b->width);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fail(CG_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    b->graph = g;
    CG_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
  }
  CG_CUDA(cudaGraphLaunch(b->exec, st));
  return CG_OK;
}

// Autotunes every member's tile shape (equal shapes share one measurement),
// then the pool width: each candidate width times two batch steps from a
// saved copy of the states, which are restored afterwards (the call leaves
// the members' states as it found them).  A captured graph is dropped and
// recaptured at the next step.
CG_API int cg_batch_autotune(cg_batch* b, void* stream, int* width_out) {
  if (!b) return fail(CG_ERR_INVALID_ARG, "null batch");
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CG_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return fail(CG_ERR_INVALID_ARG, "cg_batch_autotune times kernels: not during capture");
  int count = (int)b->solvers.size();
  for (int i = 0; i < count; ++i) {
    int rc = autotune_solver(b->solvers[i], b->states[i], false, st);
    if (rc) return rc;
  }
  size_t total = 0;
  std::vector<size_t> off(count);
  for (int i = 0; i < count; ++i) {
    off[i] = total;
    total += (size_t)b->solvers[i]->nv * b->solvers[i]->N;
  }
  double* save = nullptr;
  int rc = dalloc(&save, total);
  if (rc) return rc;
  auto copy_states = [&](bool to_save) -> int {
    for (int i = 0; i < count; ++i) {
      size_t bytes = sizeof(double) * b->solvers[i]->nv * b->solvers[i]->N;
      cudaError_t e = to_save ? cudaMemcpyAsync(save + off[i], b->states[i], bytes, cudaMemcpyDeviceToDevice, st)
                              : cudaMemcpyAsync(b->states[i], save + off[i], bytes, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return fail(CG_ERR_CUDA, "state copy: %s", cudaGetErrorString(e));
    }
    return CG_OK;
  };
  const int cands[] = {1, 4, 8, 16, 32};
  int best = b->width;
  float best_ms = 1e30f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((rc = copy_states(true)) == CG_OK && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    for (int w : cands) {
      if ((rc = multi_step(b->solvers.data(), b->states.data(), count, st, w))) break;  // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < 2 && rc == CG_OK; ++r) rc = multi_step(b->solvers.data(), b->states.data(), count, st, w);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (rc || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        if (!rc) rc = fail(CG_ERR_CUDA, "batch autotune timing failed");
        break;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = w;
      }
      if ((rc = copy_states(false))) break;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  int rc2 = copy_states(false);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(save);
  if (rc) return rc;
  if (rc2) return rc2;
  if (e != cudaSuccess) return fail(CG_ERR_CUDA, "batch autotune: %s", cudaGetErrorString(e));
  b->width = best;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  if (width_out) *width_out = best;
  return CG_OK;
}

CG_API void cg_batch_destroy(cg_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
}

}  // extern "C"
