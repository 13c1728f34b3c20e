// Batched advance of many independent grids (included by cg_api.cu).
// cg_multi_step forks the caller's stream into a pool of internal streams,
// runs each member's CFL time step and RK3 step on one of them (members are
// independent: each solver owns its scratch), and joins back.  cg_batch
// captures one such call into a CUDA graph and replays it, so a step of a
// whole batch of uneven grids costs one graph launch on the host.

namespace {

constexpr int kPoolStreams = 16;

struct StreamPool {
  int dev = -1;
  cudaStream_t s[kPoolStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kPoolStreams] = {};
};
thread_local StreamPool g_pool;

int pool_ready() {
  int dev = 0;
  CG_CUDA(cudaGetDevice(&dev));
  if (g_pool.dev == dev) return CG_OK;
  for (int i = 0; i < kPoolStreams; ++i) {
    CG_CUDA(cudaStreamCreateWithFlags(&g_pool.s[i], cudaStreamNonBlocking));
    CG_CUDA(cudaEventCreateWithFlags(&g_pool.join[i], cudaEventDisableTiming));
  }
  CG_CUDA(cudaEventCreateWithFlags(&g_pool.fork, cudaEventDisableTiming));
  g_pool.dev = dev;
  return CG_OK;
}

int multi_step(cg_solver* const* solvers, double* const* states, int count, cudaStream_t st) {
  int rc = pool_ready();
  if (rc) return rc;
  int ns = count < kPoolStreams ? count : kPoolStreams;
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
    int rc = multi_step(b->solvers.data(), b->states.data(), count, st);
    if (rc) return rc;
    b->warm = 1;
    return CG_OK;
  }
  if (!b->exec) {
    // capture one batch step; later calls replay it
    if (st == nullptr) return fail(CG_ERR_INVALID_ARG, "graph replay needs a non-default stream");
    CG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = multi_step(b->solvers.data(), b->states.data(), count, st);
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

CG_API void cg_batch_destroy(cg_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
}

}  // extern "C"
