// Batched advance of many independent grids (included by cg_api.cu).
// cg_multi_step forks the caller's stream into a pool of internal streams,
// runs each member's CFL time step and RK3 step on one of them (members are
// independent: each solver owns its scratch), and joins back.  cg_batch
// captures one step into a CUDA graph and replays it, so a step of a whole
// batch of uneven grids costs one graph launch on the host.  A batch of 2D
// Cartesian per-interface hybrids steps through a work table instead (one
// launch per phase for every member, below); cg_batch_autotune picks the tile
// shapes, the pool width, the number of table groups and the faster path.

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
  for (int k = 0; k < count && !rc; ++k) {
    int i = order[k];
    cg_solver* s = solvers[i];
    cudaStream_t si = g_pool.s[k % ns];
    DISPATCH_ND(s, cfl_launch, s, states[i], s->dt, nullptr, 0.0, si);
    rc = DISPATCH_ND(s, rk3, s, states[i], si);
  }
  // join every forked stream back, also after an error: later work on the
  // caller's stream stays ordered after the members already enqueued, and a
  // stream capture is not left with an unjoined fork
  for (int i = 0; i < ns; ++i) {
    cudaError_t e = cudaEventRecord(g_pool.join[i], g_pool.s[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, g_pool.join[i], 0);
    if (e != cudaSuccess && !rc) rc = fail(CG_ERR_CUDA, "stream join: %s", cudaGetErrorString(e));
  }
  return rc;
}

// ---------------------------------------------------------------- work-table path
// A batch of 2D Cartesian per-interface hybrids (inviscid, one tile shape)
// advances phase by phase: each launch runs one phase of the RK stage for
// every member (cg_batch_jobs.cuh), 15 launches for the first stage of a step
// and 13 for the others, whatever the number of members.  The job arrays and
// block offsets are built once on the host and kept in one device buffer.

// one phase: device job array, block offsets (nm + 1), the member of every
// block, and the total blocks
struct TKind {
  const void* jobs = nullptr;
  const long long* off = nullptr;
  const int* mem = nullptr;
  long long total = 0;
};

struct BatchTable {
  int state = 0;  // 0: not built, 1: built, -1: the batch does not qualify
  int mixed = 0;
  int lw[2] = {0, 0};
  int nm = 0;
  void* dmem = nullptr;
  void* xmem = nullptr;      // per-member buffers of the table (second Gaussian pass, second node fluxes)
  unsigned* bar = nullptr;   // persistent stage: barrier words [2], then the error flag
  int blocks = 0;            // persistent stage: co-resident blocks (0: not available)
  TKind zero1, zero23, cfl, fin, prim[3], omega, field, troubled, grad, coef, gauss[2], nodeflux[2], hflux[2];
  TKind sweep[3][2];
  PersistentStage pst[3];
};

static bool table_member_ok(const cg_solver* s, const cg_solver* s0, bool same_tiles = true) {
  return s->nd == 2 && !s->dg.curv && s->p.scheme == CG_HYBRID && s->p.hybrid_mode == CG_HYBRID_CELL &&
         !s->p.viscous && !s->iface_out && s->p.precision == s0->p.precision &&
         (!same_tiles || (s->sweep_lw[0] == s0->sweep_lw[0] && s->sweep_lw[1] == s0->sweep_lw[1])) && s->lad.fb &&
         s->lad.tr && s->hflux[0] && s->hflux[1];
}

// host staging of the job arrays and offsets, copied to the device at once
struct TableBlob {
  std::vector<char> bytes;
  struct Rec { TKind* k; size_t jobs_at, off_at, mem_at; long long total; };
  std::vector<Rec> recs;
  template <class Job>
  void add(TKind* k, const std::vector<Job>& jobs, const std::vector<long long>& off) {
    auto put = [&](const void* p, size_t n) {
      size_t at = (bytes.size() + 255) / 256 * 256;
      bytes.resize(at + n);
      memcpy(bytes.data() + at, p, n);
      return at;
    };
    std::vector<int> mem((size_t)off.back());
    for (size_t m = 0; m + 1 < off.size(); ++m)
      for (long long b = off[m]; b < off[m + 1]; ++b) mem[(size_t)b] = (int)m;
    Rec r{k, put(jobs.data(), sizeof(Job) * jobs.size()), put(off.data(), sizeof(long long) * off.size()),
          put(mem.data(), sizeof(int) * mem.size()), off.back()};
    recs.push_back(r);
  }
};

// virtual blocks of a grid-stride body: each thread takes up to kTableItems
// items, so that a block's set-up (member lookup, job fields) is shared
constexpr int kTableItems = 16;
static long long table_blocks(long long work) {
  const long long per = (long long)BATCH_THREADS * kTableItems;
  return work < 1 ? 1 : (work + per - 1) / per;
}

template <typename T>
static int table_build_t(BatchTable& tb, cg_solver* const* sv, double* const* states, int nm) {
  TableBlob blob;
  auto offsets = [&](auto nblk) {
    std::vector<long long> off(nm + 1, 0);
    for (int m = 0; m < nm; ++m) off[m + 1] = off[m] + nblk(m);
    return off;
  };
  auto one = [](int) { return 1LL; };
  std::vector<JobZero> z1(nm), z23(nm);
  std::vector<JobFinish> fin(nm);
  std::vector<JobCfl<T>> cfl(nm);
  for (int m = 0; m < nm; ++m) {
    cg_solver* s = sv[m];
    z1[m] = JobZero{s->cflmax, s->hyb_flag, s->hyb_count};
    z23[m] = JobZero{nullptr, s->hyb_flag, s->hyb_count};
    fin[m] = JobFinish{s->cflmax, s->p.cfl, s->dt};
    cfl[m] = JobCfl<T>{s->dg, states[m], s->cflmax, (unsigned)table_blocks(s->N)};
  }
  blob.add(&tb.zero1, z1, offsets(one));
  blob.add(&tb.zero23, z23, offsets(one));
  blob.add(&tb.fin, fin, offsets(one));
  blob.add(&tb.cfl, cfl, offsets([&](int m) { return (long long)cfl[m].nb; }));
  for (int k = 0; k < 3; ++k) {
    std::vector<JobPrim<T>> pr(nm);
    for (int m = 0; m < nm; ++m) {
      cg_solver* s = sv[m];
      const double* Uc = k == 0 ? states[m] : (k == 1 ? s->U1 : s->U2);
      pr[m] = JobPrim<T>{s->dg, Uc, reinterpret_cast<T*>(s->W), (unsigned)table_blocks(s->N)};
    }
    blob.add(&tb.prim[k], pr, offsets([&](int m) { return (long long)pr[m].nb; }));
  }
  std::vector<JobOmega<T>> om(nm);
  std::vector<JobField<T>> fd(nm);
  std::vector<JobTroubled<T>> tr(nm);
  std::vector<JobGrad<T>> gr(nm);
  std::vector<JobCoef<T>> co(nm);
  std::vector<JobGauss<T>> ga[2] = {std::vector<JobGauss<T>>(nm), std::vector<JobGauss<T>>(nm)};
  std::vector<JobNodeflux<T>> nf[2] = {std::vector<JobNodeflux<T>>(nm), std::vector<JobNodeflux<T>>(nm)};
  std::vector<JobHflux<T>> hf[2] = {std::vector<JobHflux<T>>(nm), std::vector<JobHflux<T>>(nm)};
  // buffers of the table's own: the Gaussian's second pass writes bt2/kp2
  // (not the coefficient planes its first pass read) and the y node fluxes go
  // to Fn1 (not the x node fluxes' buffer), so that within a stage no buffer is
  // written after a phase read it (what a persistent stage needs); the
  // arithmetic is the members' own
  std::vector<size_t> xoff(nm + 1, 0);
  for (int m = 0; m < nm; ++m) {
    const cg_solver* s = sv[m];
    size_t b = (2 * (size_t)s->N + (size_t)s->nv * s->lad.fbox[1].size()) * sizeof(T);
    xoff[m + 1] = xoff[m] + (b + 255) / 256 * 256;
  }
  {
    int rc = dalloc((char**)&tb.xmem, xoff[nm]);
    if (rc) return rc;
  }
  for (int m = 0; m < nm; ++m) {
    cg_solver* s = sv[m];
    LadBuffers& L = s->lad;
    const T* W = reinterpret_cast<const T*>(s->W);
    T* fb = reinterpret_cast<T*>(L.fb);
    T* g = reinterpret_cast<T*>(L.gr);
    T* dv = reinterpret_cast<T*>(L.dv);
    T* xm = reinterpret_cast<T*>(static_cast<char*>(tb.xmem) + xoff[m]);
    T* bt[3] = {reinterpret_cast<T*>(L.bt[0]), reinterpret_cast<T*>(L.bt[1]), xm};
    T* kp[3] = {reinterpret_cast<T*>(L.kp[0]), reinterpret_cast<T*>(L.kp[1]), xm + s->N};
    T* Fn[2] = {reinterpret_cast<T*>(L.Fn), xm + 2 * s->N};
    JobOmega<T> o;
    o.g = s->dg;
    o.W = W;
    for (int d = 0; d < 3; ++d) {
      o.G[d] = reinterpret_cast<const T*>(s->G[d]);
      o.gb[d] = s->gdLB[d];
    }
    o.om = reinterpret_cast<T*>(s->om);
    o.ob = s->omBox;
    o.nb = (unsigned)table_blocks(s->omBox.size());
    om[m] = o;
    fd[m] = JobField<T>{s->dg, W, fb, L.fbx, (unsigned)table_blocks(L.fbx.size())};
    tr[m] = JobTroubled<T>{s->dg, W, s->p.hyb_rho, s->p.hyb_p, s->p.hybrid_sensor ? reinterpret_cast<const T*>(s->om) : nullptr, s->omBox,
                           s->p.sensor_thresh, L.tr, L.tbox, s->hyb_flag, s->hyb_count,
                           (unsigned)table_blocks(L.tbox.size()), s->p.hybrid_buffer};
    JobGrad<T> j;
    j.g = s->dg;
    j.fb = fb;
    j.fbx = L.fbx;
    for (int d = 0; d < 3; ++d) j.lb[d] = L.dfLB[d];
    j.gr = g;
    j.dv = dv;
    j.b3 = L.b3;
    j.nb = (unsigned)table_blocks(L.b3.size());
    gr[m] = j;
    co[m] = JobCoef<T>{s->dg, W, fb, L.fbx, g, dv, L.b3, s->p.c_beta, s->p.c_kappa, bt[0], kp[0],
                       (unsigned)table_blocks(s->N)};
    // the overbar along x then y: bt/kp 0 -> 1 -> 2
    ga[0][m] = JobGauss<T>{s->dg, 0, bt[0], kp[0], bt[1], kp[1], (unsigned)table_blocks(s->N)};
    ga[1][m] = JobGauss<T>{s->dg, 1, bt[1], kp[1], bt[2], kp[2], (unsigned)table_blocks(s->N)};
    for (int l = 0; l < 2; ++l) {
      nf[l][m] = JobNodeflux<T>{s->dg, l, W, bt[2], kp[2], g, dv, L.b3, Fn[l], L.fbox[l],
                                (unsigned)table_blocks(L.fbox[l].size())};
      hf[l][m] = JobHflux<T>{s->dg, l, Fn[l], L.fbox[l], reinterpret_cast<T*>(s->hflux[l]), L.hbox[l],
                             (unsigned)table_blocks(L.hbox[l].size())};
    }
  }
  blob.add(&tb.omega, om, offsets([&](int m) { return (long long)om[m].nb; }));
  blob.add(&tb.field, fd, offsets([&](int m) { return (long long)fd[m].nb; }));
  blob.add(&tb.troubled, tr, offsets([&](int m) { return (long long)tr[m].nb; }));
  blob.add(&tb.grad, gr, offsets([&](int m) { return (long long)gr[m].nb; }));
  blob.add(&tb.coef, co, offsets([&](int m) { return (long long)co[m].nb; }));
  for (int l = 0; l < 2; ++l) {
    blob.add(&tb.gauss[l], ga[l], offsets([&](int m) { return (long long)ga[l][m].nb; }));
    blob.add(&tb.nodeflux[l], nf[l], offsets([&](int m) { return (long long)nf[l][m].nb; }));
    blob.add(&tb.hflux[l], hf[l], offsets([&](int m) { return (long long)hf[l][m].nb; }));
  }
  // sweeps: the stage arguments of the per-interface hybrid stage
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 2; ++d) {
      std::vector<SweepJob> sj(nm);
      for (int m = 0; m < nm; ++m) {
        cg_solver* s = sv[m];
        double* U = states[m];
        const double* Uc = k == 0 ? U : (k == 1 ? s->U1 : s->U2);
        double* out = k == 0 ? s->U1 : (k == 1 ? s->U2 : U);
        StageArgs A = base_args(s);
        A.rk = 1;
        A.stage = k + 1;
        A.R = out;
        A.Un = U;
        A.Uc = Uc;
        A.Uout = out;
        A.mask = s->lad.tr;
        A.tBox = s->lad.tbox;
        A.first = d == 0;
        A.last = d == 1;
        A.hflux = s->hflux[d];
        A.hBox = s->lad.hbox[d];
        A.Gd = nullptr;
        A.gdLB = s->gdLB[d];
        A.iface_out = nullptr;
        dim3 gd = sweep_grid_dims(d, s->sweep_lw[d], s->dg);
        sj[m] = SweepJob{s->dg, gbr_cfg(s), A, gd.x, gd.y, gd.z};
      }
      blob.add(&tb.sweep[k][d], sj, offsets([&](int m) { return (long long)sj[m].gx * sj[m].gy * sj[m].gz; }));
    }
  void* dm = nullptr;
  int rc = dalloc((char**)&dm, blob.bytes.size());
  if (rc) return rc;
  CG_CUDA(cudaMemcpy(dm, blob.bytes.data(), blob.bytes.size(), cudaMemcpyHostToDevice));
  for (auto& r : blob.recs) {
    r.k->jobs = (const char*)dm + r.jobs_at;
    r.k->off = reinterpret_cast<const long long*>((const char*)dm + r.off_at);
    r.k->mem = reinterpret_cast<const int*>((const char*)dm + r.mem_at);
    r.k->total = r.total;
  }
  tb.dmem = dm;
  // the three persistent stages: the same phases as the table's launches
  if ((rc = dalloc(&tb.bar, 4))) return rc;
  CG_CUDA(cudaMemset(tb.bar, 0, 4 * sizeof(unsigned)));
  tb.blocks = tb.mixed ? persistent_blocks_f32_2(tb.lw[0], tb.lw[1]) : persistent_blocks_f64_2(tb.lw[0], tb.lw[1]);
  auto ref = [](const TKind& k) { return PhaseRef{k.jobs, k.off, k.mem, k.total}; };
  for (int k = 0; k < 3; ++k) {
    PersistentStage& P = tb.pst[k];
    P.zero = ref(k == 0 ? tb.zero1 : tb.zero23);
    P.cfl = ref(tb.cfl);
    P.fin = ref(tb.fin);
    P.prim = ref(tb.prim[k]);
    P.omega = ref(tb.omega);
    P.field = ref(tb.field);
    P.troubled = ref(tb.troubled);
    P.grad = ref(tb.grad);
    P.coef = ref(tb.coef);
    for (int l = 0; l < 2; ++l) {
      P.gauss[l] = ref(tb.gauss[l]);
      P.nodeflux[l] = ref(tb.nodeflux[l]);
      P.hflux[l] = ref(tb.hflux[l]);
      P.sweep[l] = ref(tb.sweep[k][l]);
    }
    P.with_cfl = k == 0;
    P.bar = tb.bar;
    P.err = reinterpret_cast<int*>(tb.bar + 2);
    P.expect = (unsigned)tb.blocks;
  }
  return CG_OK;
}

static void table_free(BatchTable& tb) {
  if (tb.dmem) cudaFree(tb.dmem);
  if (tb.xmem) cudaFree(tb.xmem);
  if (tb.bar) cudaFree(tb.bar);
  tb = BatchTable();
}

// One RK3 step of every member in three cooperative launches (one per stage).
static int table_step_persistent(const BatchTable& tb, cudaStream_t st) {
  if (tb.blocks < 1) return fail(CG_ERR_UNSUPPORTED, "no persistent stage for this tile shape");
  for (int k = 0; k < 3; ++k) {
    int e = tb.mixed ? launch_persistent_f32_2(tb.lw[0], tb.lw[1], tb.pst[k], tb.blocks, st)
                     : launch_persistent_f64_2(tb.lw[0], tb.lw[1], tb.pst[k], tb.blocks, st);
    if (e) return fail(CG_ERR_CUDA, "persistent stage %d: %s", k + 1, cudaGetErrorString((cudaError_t)e));
  }
  return CG_OK;
}

// Builds the table if the batch qualifies (state 1), else marks it (-1).
static int table_build(BatchTable& tb, const std::vector<cg_solver*>& sv, const std::vector<double*>& states) {
  table_free(tb);
  const int nm = (int)sv.size();
  for (int m = 0; m < nm; ++m)
    if (!table_member_ok(sv[m], sv[0])) {
      tb.state = -1;
      return CG_OK;
    }
  tb.nm = nm;
  tb.mixed = sv[0]->p.precision == CG_MIXED;
  tb.lw[0] = sv[0]->sweep_lw[0];
  tb.lw[1] = sv[0]->sweep_lw[1];
  int rc = tb.mixed ? table_build_t<float>(tb, sv.data(), states.data(), nm)
                    : table_build_t<double>(tb, sv.data(), states.data(), nm);
  if (rc) {
    table_free(tb);
    return rc;
  }
  tb.state = 1;
  return CG_OK;
}

template <class Job>
static void table_launch(const TKind& k, int, cudaStream_t st) {
  k_batched<Job><<<(unsigned)k.total, BATCH_THREADS, 0, st>>>(static_cast<const Job*>(k.jobs), k.off, k.mem);
}

template <class J1, class J2>
static void table_launch2(const TKind& a, const TKind& b, int, cudaStream_t st) {
  k_batched2<J1, J2><<<(unsigned)(a.total + b.total), BATCH_THREADS, 0, st>>>(
      static_cast<const J1*>(a.jobs), a.off, a.mem, a.total, static_cast<const J2*>(b.jobs), b.off, b.mem);
}

// One RK3 step (with each member's CFL dt) of every member.
template <typename T>
static int table_step_t(const BatchTable& tb, cudaStream_t st) {
  const int nm = tb.nm;
  auto sweep = [&](int k, int d) -> int {
    const TKind& K = tb.sweep[k][d];
    const SweepJob* J = static_cast<const SweepJob*>(K.jobs);
    int e = tb.mixed ? launch_sweep_batched_f32_2(d, tb.lw[d], J, K.off, K.mem, K.total, st)
                     : launch_sweep_batched_f64_2(d, tb.lw[d], J, K.off, K.mem, K.total, st);
    if (e) return fail(CG_ERR_CUDA, "batched sweep (dir %d): %s", d, cudaGetErrorString((cudaError_t)e));
    return CG_OK;
  };
  for (int k = 0; k < 3; ++k) {
    if (k == 0) {
      table_launch<JobZero>(tb.zero1, nm, st);
      table_launch<JobCfl<T>>(tb.cfl, nm, st);
      table_launch<JobFinish>(tb.fin, nm, st);
    } else {
      table_launch<JobZero>(tb.zero23, nm, st);
    }
    table_launch<JobPrim<T>>(tb.prim[k], nm, st);
    table_launch2<JobOmega<T>, JobField<T>>(tb.omega, tb.field, nm, st);
    table_launch2<JobTroubled<T>, JobGrad<T>>(tb.troubled, tb.grad, nm, st);
    table_launch<JobCoef<T>>(tb.coef, nm, st);
    table_launch<JobGauss<T>>(tb.gauss[0], nm, st);
    table_launch<JobGauss<T>>(tb.gauss[1], nm, st);
    for (int l = 0; l < 2; ++l) {
      table_launch<JobNodeflux<T>>(tb.nodeflux[l], nm, st);
      table_launch<JobHflux<T>>(tb.hflux[l], nm, st);
    }
    int rc;
    if ((rc = sweep(k, 0))) return rc;
    if ((rc = sweep(k, 1))) return rc;
  }
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}

static int table_step(const BatchTable& tb, cudaStream_t st) {
  return tb.mixed ? table_step_t<float>(tb, st) : table_step_t<double>(tb, st);
}

// launches of one table step
static int table_launches(const BatchTable&) { return 3 * 13 + 2; }

// The members split into groups (largest first, dealt round robin), one table
// per group; the groups run concurrently on the stream pool, so that phases
// of different groups (FP64-bound recovery, FP32 sweeps, memory-bound
// stencils) overlap on the device.
struct TableSet {
  int state = 0;  // 0: not built, 1: built, -1: the batch does not qualify
  int persistent = 0;  // one group stepped by the persistent stages
  std::vector<BatchTable> t;
};

static void tables_free(TableSet& ts) {
  for (auto& t : ts.t) table_free(t);
  ts.t.clear();
  ts.state = 0;
  ts.persistent = 0;
}

static int tables_build(TableSet& ts, const std::vector<cg_solver*>& sv, const std::vector<double*>& states,
                        int groups) {
  tables_free(ts);
  const int nm = (int)sv.size();
  for (int m = 0; m < nm; ++m)
    if (!table_member_ok(sv[m], sv[0])) {
      ts.state = -1;
      return CG_OK;
    }
  groups = std::max(1, std::min(groups, std::min(nm, kMaxPoolStreams)));
  std::vector<int> order(nm);
  for (int m = 0; m < nm; ++m) order[m] = m;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sv[a]->N > sv[b]->N; });
  std::vector<std::vector<cg_solver*>> gs(groups);
  std::vector<std::vector<double*>> gu(groups);
  for (int i = 0; i < nm; ++i) {
    gs[i % groups].push_back(sv[order[i]]);
    gu[i % groups].push_back(states[order[i]]);
  }
  ts.t.resize(groups);
  for (int g = 0; g < groups; ++g) {
    int rc = table_build(ts.t[g], gs[g], gu[g]);
    if (rc || ts.t[g].state != 1) {
      tables_free(ts);
      if (rc) return rc;
      ts.state = -1;
      return CG_OK;
    }
  }
  ts.state = 1;
  return CG_OK;
}

static int tables_step(const TableSet& ts, cudaStream_t st) {
  const int ng = (int)ts.t.size();
  if (ng == 1 && ts.persistent) return table_step_persistent(ts.t[0], st);
  if (ng == 1) return table_step(ts.t[0], st);
  int rc = pool_ready();
  if (rc) return rc;
  CG_CUDA(cudaEventRecord(g_pool.fork, st));
  for (int g = 0; g < ng; ++g) {
    CG_CUDA(cudaStreamWaitEvent(g_pool.s[g], g_pool.fork, 0));
    if ((rc = table_step(ts.t[g], g_pool.s[g]))) return rc;
    CG_CUDA(cudaEventRecord(g_pool.join[g], g_pool.s[g]));
    CG_CUDA(cudaStreamWaitEvent(st, g_pool.join[g], 0));
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
  TableSet tables;           // work-table path (qualifying batches)
  int groups = 1;            // member groups of the work table, run concurrently
  int use_table = 1;         // 0: the stream pool even where the table qualifies
  int persistent = 0;        // work table stepped by one persistent launch per stage
};

// the table set of the batch's current choice (built on first use)
static int batch_tables(cg_batch* b) {
  if (b->tables.state == 0) {
    int rc = tables_build(b->tables, b->solvers, b->states, b->persistent ? 1 : b->groups);
    if (rc) return rc;
  }
  if (b->tables.state == 1) b->tables.persistent = b->persistent && b->tables.t.size() == 1 && b->tables.t[0].blocks > 0;
  return CG_OK;
}

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

// one eager step of the batch by its current path
static int batch_once(cg_batch* b, cudaStream_t st) {
  if (b->use_table && b->tables.state == 1) return tables_step(b->tables, st);
  return multi_step(b->solvers.data(), b->states.data(), (int)b->solvers.size(), st, b->width);
}

CG_API int cg_batch_step(cg_batch* b, void* stream) {
  if (!b) return fail(CG_ERR_INVALID_ARG, "null batch");
  cudaStream_t st = (cudaStream_t)stream;
  if (!b->warm) {
    // first step runs eagerly: the work table, one-time kernel attributes and
    // the stream pool are set up here
    int rc = batch_tables(b);
    if (rc) return rc;
    rc = batch_once(b, st);
    if (rc) return rc;
    b->warm = 1;
    return CG_OK;
  }
  if (!b->exec) {
    // capture one batch step; later calls replay it
    if (st == nullptr) return fail(CG_ERR_INVALID_ARG, "graph replay needs a non-default stream");
    CG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = batch_once(b, st);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if ((rc || e != cudaSuccess) && b->tables.persistent) {
      // a cooperative launch this stream cannot capture: step by the table's launches
      if (g) cudaGraphDestroy(g);
      g = nullptr;
      cudaGetLastError();
      b->persistent = 0;
      b->tables.persistent = 0;
      CG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      rc = batch_once(b, st);
      e = cudaStreamEndCapture(st, &g);
    }
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
// then the pool width: each candidate width times two batch steps (replays of
// a captured step where the stream allows) from a saved copy of the states,
// which are restored afterwards (the call leaves the members' states as it
// found them).  A batch that qualifies for the work
// table also times the table with each common tile shape and keeps whichever
// path is faster.  A captured graph is dropped and recaptured at the next step.
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
  // device time of two batch steps of fn: one eager step first (kernel
  // attributes, stream pool), then, on a stream that can be captured, two
  // replays of a captured step after one warm-up replay, as cg_batch_step runs
  // them from its third call on; on the legacy stream, two eager steps
  auto time_steps = [&](auto&& fn, float* ms) -> int {
    int r = fn();
    if (r) return r;
    if (st != nullptr) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t x = nullptr;
      CG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      r = fn();
      cudaError_t e = cudaStreamEndCapture(st, &g);
      if (r) {
        if (g) cudaGraphDestroy(g);
        return r;
      }
      if (e != cudaSuccess) return fail(CG_ERR_CUDA, "batch autotune capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&x, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(CG_ERR_CUDA, "batch autotune graph: %s", cudaGetErrorString(e));
      e = cudaGraphLaunch(x, st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaGraphLaunch(x, st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      cudaGraphExecDestroy(x);
      if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
      if (e != cudaSuccess) return fail(CG_ERR_CUDA, "batch autotune timing: %s", cudaGetErrorString(e));
      return CG_OK;
    }
    CG_CUDA(cudaEventRecord(e0, st));
    for (int k = 0; k < 2 && r == CG_OK; ++k) r = fn();
    if (r) return r;
    CG_CUDA(cudaEventRecord(e1, st));
    CG_CUDA(cudaEventSynchronize(e1));
    CG_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return CG_OK;
  };
  if ((rc = copy_states(true)) == CG_OK && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    for (int w : cands) {
      float ms = 0.f;
      rc = time_steps([&]() { return multi_step(b->solvers.data(), b->states.data(), count, st, w); }, &ms);
      if (rc) break;
      if (ms < best_ms) {
        best_ms = ms;
        best = w;
      }
      if ((rc = copy_states(false))) break;
    }
  }
  // the work table, where the batch qualifies: one tile shape for all members,
  // each candidate timed the same way; it replaces the stream pool if faster
  bool table_ok = rc == CG_OK && e0 && e1;
  for (int i = 0; table_ok && i < count; ++i) table_ok = table_member_ok(b->solvers[i], b->solvers[0], false);
  b->use_table = 0;
  if (table_ok) {
    std::vector<std::array<int, 3>> keep(count);
    for (int i = 0; i < count; ++i)
      keep[i] = {b->solvers[i]->sweep_lw[0], b->solvers[i]->sweep_lw[1], b->solvers[i]->sweep_lw[2]};
    int tbest[3] = {0, 0, 1};  // lines per x tile, per y tile, groups
    float tbest_ms = 1e30f;
    auto try_table = [&](int lx, int ly, int ng) -> int {
      for (cg_solver* s : b->solvers) {
        s->sweep_lw[0] = lx;
        s->sweep_lw[1] = ly;
      }
      int r = tables_build(b->tables, b->solvers, b->states, ng);
      if (r || b->tables.state != 1) return r;
      float ms = 0.f;
      if ((r = time_steps([&]() { return tables_step(b->tables, st); }, &ms))) return r;
      if (ms < tbest_ms) {
        tbest_ms = ms;
        tbest[0] = lx;
        tbest[1] = ly;
        tbest[2] = ng;
      }
      return copy_states(false);
    };
    // the tile shape with one group, then the number of groups with that shape
    for (int lx : kSweepLwCands0)
      for (int ly : kSweepLwCands1)
        if (rc == CG_OK) rc = try_table(lx, ly, 1);
    const int lx = tbest[0], ly = tbest[1];
    for (int ng : {2, 4, 8})
      if (rc == CG_OK && lx && ng <= count) rc = try_table(lx, ly, ng);
    // one persistent launch per stage (one group, the chosen tile shape)
    int pbest = 0;
    if (rc == CG_OK && lx) {
      for (cg_solver* s : b->solvers) {
        s->sweep_lw[0] = lx;
        s->sweep_lw[1] = ly;
      }
      rc = tables_build(b->tables, b->solvers, b->states, 1);
      if (rc == CG_OK && b->tables.state == 1 && b->tables.t[0].blocks > 0) {
        b->tables.persistent = 1;
        float ms = 0.f;
        int r = time_steps([&]() { return tables_step(b->tables, st); }, &ms);
        if (r == CG_OK) {
          if (ms < tbest_ms) {
            tbest_ms = ms;
            tbest[2] = 1;
            pbest = 1;
          }
          rc = copy_states(false);
        } else {
          cudaGetLastError();  // a persistent stage that cannot be captured or launched: not a candidate
          rc = copy_states(false);
        }
      }
    }
    if (rc == CG_OK && tbest[0] && tbest_ms < best_ms) {
      for (cg_solver* s : b->solvers) {
        s->sweep_lw[0] = tbest[0];
        s->sweep_lw[1] = tbest[1];
      }
      b->groups = tbest[2];
      b->persistent = pbest;
      rc = tables_build(b->tables, b->solvers, b->states, b->groups);
      if (rc == CG_OK) rc = batch_tables(b);
      b->use_table = 1;
    } else {
      for (int i = 0; i < count; ++i)
        for (int d = 0; d < 3; ++d) b->solvers[i]->sweep_lw[d] = keep[i][d];
      tables_free(b->tables);
      b->persistent = 0;
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
  if (!b->use_table) b->tables.state = -1;  // stays on the stream pool
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  if (width_out) *width_out = best;
  return CG_OK;
}

CG_API void cg_batch_destroy(cg_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  tables_free(b->tables);
  delete b;
}

CG_API int cg_batch_path(const cg_batch* b, int* path_out, int* launches_out) {
  if (!b || !path_out) return fail(CG_ERR_INVALID_ARG, "null argument");
  const bool table = b->use_table && b->tables.state == 1;
  const bool pers = table && b->tables.persistent;
  *path_out = pers ? 2 : (table ? 1 : 0);
  int n = 0;
  if (table)
    for (const BatchTable& t : b->tables.t) n += table_launches(t);
  if (launches_out) *launches_out = pers ? 3 : (table ? n : -1);  // -1: per member, counted by the members
  return CG_OK;
}

CG_API int cg_batch_set_path(cg_batch* b, int path, int groups) {
  if (!b || path < 0 || path > 2 || groups < 1) return fail(CG_ERR_INVALID_ARG, "bad arguments");
  tables_free(b->tables);
  b->use_table = path > 0;
  b->persistent = path == 2;
  b->groups = path == 1 ? groups : 1;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  b->warm = 0;
  if (path > 0) {
    int rc = batch_tables(b);
    if (rc) return rc;
    if (b->tables.state != 1) return fail(CG_ERR_UNSUPPORTED, "the batch does not qualify for the work table");
    if (path == 2 && !b->tables.persistent)
      return fail(CG_ERR_UNSUPPORTED, "no persistent stage for this batch's tile shape");
  }
  return CG_OK;
}

CG_API int cg_batch_debug_barrier(cg_batch* b, int extra) {
  if (!b || extra < 0) return fail(CG_ERR_INVALID_ARG, "bad arguments");
  if (!(b->tables.state == 1 && b->tables.persistent)) return fail(CG_ERR_UNSUPPORTED, "not on the persistent path");
  for (BatchTable& t : b->tables.t)
    for (int k = 0; k < 3; ++k) t.pst[k].expect = (unsigned)(t.blocks + extra);
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  b->warm = 0;
  return CG_OK;
}

CG_API int cg_batch_sync(cg_batch* b, void* stream) {
  if (!b) return fail(CG_ERR_INVALID_ARG, "null batch");
  cudaStream_t st = (cudaStream_t)stream;
  CG_CUDA(cudaStreamSynchronize(st));
  for (BatchTable& t : b->tables.t) {
    if (!t.bar) continue;
    unsigned w[4];
    CG_CUDA(cudaMemcpy(w, t.bar, sizeof w, cudaMemcpyDeviceToHost));
    if (w[2]) {
      CG_CUDA(cudaMemset(t.bar, 0, sizeof w));
      return fail(CG_ERR_TIMEOUT, "a persistent stage's grid barrier gave up waiting");
    }
  }
  return CG_OK;
}

}  // extern "C"
