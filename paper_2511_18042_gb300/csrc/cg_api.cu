// C ABI of the cgflow library (include/cgflow.h): handles, scratch, the
// orchestration of one RK stage per scheme, RK3, CFL and diagnostics.
// Host arithmetic that must reproduce the method's rounding (interface frames
// of Cartesian grids, Thomas pivots) is compiled with contraction disabled.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <tuple>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/cgflow.h"
#include "cg_kernels.cuh"
#include "cg_lad.cuh"
#include "cg_batch_jobs.cuh"
#include "cg_lines.cuh"
#include "cg_metrics.cuh"
#include "cg_sweep.h"

using namespace cgk;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CG_CUDA(call)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(CG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int grid_blocks(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152LL * 32) b = 152LL * 32;
  return (int)b;
}

// host copy of the oracle-independent Thomas pivots for a constant-coefficient
// system (unit diagonal, off-diagonal a); closure rows 0 and m-1 decoupled
// (non-periodic) or cyclic with the Sherman-Morrison modification.
struct HostLine {
  std::vector<double> cp, den, z;
  double fden = 0.0, gam = -1.0;
};
// the tridiagonal rows (A x_{i-1} + B x_i + C x_{i+1}) actually eliminated:
// non-periodic lines with identity closure rows, cyclic lines with the
// Sherman-Morrison modification (gam = -1)
void line_rows(int m, double a, bool cyclic, std::vector<double>& A, std::vector<double>& B, std::vector<double>& C,
               double* gam_out) {
  A.assign(m, a);
  B.assign(m, 1.0);
  C.assign(m, a);
  if (!cyclic) {
    A[0] = 0.0; C[0] = 0.0; A[m - 1] = 0.0; C[m - 1] = 0.0;
  } else {
    double gam = -B[0];
    *gam_out = gam;
    B[0] = B[0] - gam;
    B[m - 1] = B[m - 1] - a * a / gam;
    A[0] = 0.0;
    C[m - 1] = 0.0;
  }
}

HostLine make_line(int m, double a, bool cyclic) {
  HostLine L;
  L.cp.assign(m, 0.0);
  L.den.assign(m, 1.0);
  std::vector<double> A, B, C;
  line_rows(m, a, cyclic, A, B, C, &L.gam);
  L.cp[0] = C[0] / B[0];
  L.den[0] = B[0];
  for (int i = 1; i < m; ++i) {
    double den = B[i] - A[i] * L.cp[i - 1];
    L.den[i] = den;
    L.cp[i] = C[i] / den;
  }
  if (cyclic) {
    std::vector<double> u(m, 0.0), dp(m);
    u[0] = L.gam;
    u[m - 1] = a;
    dp[0] = u[0] / B[0];
    for (int i = 1; i < m; ++i) dp[i] = (u[i] - A[i] * dp[i - 1]) / L.den[i];
    L.z.assign(m, 0.0);
    L.z[m - 1] = dp[m - 1];
    for (int i = m - 2; i >= 0; --i) L.z[i] = dp[i] - L.cp[i] * L.z[i + 1];
    L.fden = 1.0 + L.z[0] + a * L.z[m - 1] / L.gam;
  }
  return L;
}

// Partition of a line system into P chunks (see k_tri_part): local pivots,
// responses to the neighbouring chunks' boundary unknowns, and the factors of
// the boundary recursion, all in FP64 on the host.
struct HostPart {
  std::vector<double> aL, cp, rd, V, W, ch;
  int q = 0, P = 0;
};

HostPart make_part(const std::vector<double>& A, const std::vector<double>& B, const std::vector<double>& C, int P) {
  int m = (int)B.size();
  HostPart h;
  h.q = (m + P - 1) / P;
  h.P = (m + h.q - 1) / h.q;
  h.aL.assign(m, 0.0);
  h.cp.assign(m, 0.0);
  h.rd.assign(m, 0.0);
  h.V.assign(m, 0.0);
  h.W.assign(m, 0.0);
  h.ch.assign(5 * (size_t)h.P, 0.0);
  double beta_prev = 0.0;
  for (int k = 0; k < h.P; ++k) {
    int s = k * h.q, e = std::min(m, s + h.q), n = e - s;
    std::vector<double> den(n), cpl(n);
    den[0] = B[s];
    cpl[0] = n > 1 ? C[s] / den[0] : 0.0;
    for (int r = 1; r < n; ++r) {
      den[r] = B[s + r] - A[s + r] * cpl[r - 1];
      cpl[r] = r < n - 1 ? C[s + r] / den[r] : 0.0;
    }
    for (int r = 0; r < n; ++r) {
      h.aL[s + r] = r == 0 ? 0.0 : A[s + r];
      h.cp[s + r] = cpl[r];
      h.rd[s + r] = 1.0 / den[r];
    }
    // responses to A_s x_{s-1} (row s) and C_{e-1} x_e (row e-1)
    auto solve = [&](int row, double val, double* out) {
      std::vector<double> y(n);
      for (int r = 0; r < n; ++r) {
        double rhs = r == row ? val : 0.0;
        y[r] = (rhs - (r > 0 ? A[s + r] * y[r - 1] : 0.0)) / den[r];
      }
      for (int r = n - 2; r >= 0; --r) y[r] = y[r] - cpl[r] * y[r + 1];
      for (int r = 0; r < n; ++r) out[s + r] = y[r];
    };
    solve(0, A[s], h.V.data());
    solve(n - 1, C[e - 1], h.W.data());
    double VF = h.V[s], VL = h.V[e - 1], WF = h.W[s], WL = h.W[e - 1];
    double rF = 1.0 / (1.0 + VF * beta_prev);
    double qF = -WF * rF;
    double beta = -VL * beta_prev * qF - WL;
    double* c = &h.ch[5 * (size_t)k];
    c[0] = rF; c[1] = qF; c[2] = beta; c[3] = VF; c[4] = VL;
    beta_prev = beta;
  }
  return h;
}

// chunks per column for a launch of `columns` columns of m rows: enough
// threads to fill the GPU (152 SMs x 2048), at least 8 rows per chunk
int choose_parts(int m, long long columns) {
  int P = 1;
  while (P < kPartMax && columns * 2LL * P <= 152LL * 2048 && m / (2 * P) >= 8) P *= 2;
  return P;
}

struct DevLine {
  LineCoef lc{};
  double* buf = nullptr;
  PartCoef pc{};        // pc.P >= 4: the partitioned solver is used
  double* pbuf = nullptr;
  // FP32 mirrors of the same factors (the mixed form's gradient solves)
  LineCoefT<float> lcf{};
  float* fbuf = nullptr;
  PartCoefT<float> pcf{};
  float* fpbuf = nullptr;
};

template <typename T>
static const LineCoefT<T>& line_coef(const DevLine& L);
template <>
const LineCoefT<double>& line_coef<double>(const DevLine& L) { return L.lc; }
template <>
const LineCoefT<float>& line_coef<float>(const DevLine& L) { return L.lcf; }
template <typename T>
static const PartCoefT<T>& part_coef(const DevLine& L);
template <>
const PartCoefT<double>& part_coef<double>(const DevLine& L) { return L.pc; }
template <>
const PartCoefT<float>& part_coef<float>(const DevLine& L) { return L.pcf; }

}  // namespace

struct cg_grid {
  int nd;
  int n[3];
  double h[3];
  int bc[3][2];
  int curv;
  double* xyz = nullptr;  // device copy of the coordinates
  double period[3][3];
};

struct cg_solver {
  size_t dev_bytes = 0;  // device memory this solver holds (cg_solver_device_bytes)
  const cg_grid* grid;
  cg_params p;
  DevGrid dg;
  int nd, nv;
  long long N;
  // metric planes (curvilinear)
  double* metric = nullptr;
  // stage scratch
  double *W = nullptr, *acc = nullptr, *om = nullptr, *U1 = nullptr, *U2 = nullptr, *Rtmp = nullptr;
  double* G[3] = {nullptr, nullptr, nullptr};
  Box omBox;
  LineBuf gdLB[3];
  DevLine mig4[3];
  // LAD scratch
  LadBuffers lad;
  // hybrid
  unsigned char* mask = nullptr;
  double* hflux[3] = {nullptr, nullptr, nullptr};
  Box hBox[3];
  int* hyb_flag = nullptr;          // device: decision of the last stage
  unsigned long long* hyb_count = nullptr;
  // scalars
  double* dt = nullptr;             // device dt
  double* t = nullptr;              // device time
  unsigned long long* cflmax = nullptr;
  // set by rk3 with a fused CFL step: the next primitive launch (stage 1's)
  // also reduces the CFL maximum and writes dt (and t) here
  bool prim_cfl = false;
  double* prim_cfl_dt = nullptr;
  double* prim_cfl_t = nullptr;
  // set by the mixed form's deferred stage update: W already holds the
  // primitives of the next stage's state, so its primitive launch is skipped
  bool prim_ready = false;
  // cg_step_graph: the captured CFL + RK3 step and what it was captured for
  cudaGraphExec_t gexec = nullptr;
  double* g_U = nullptr;
  double* g_dt = nullptr;
  int g_lw[3] = {0, 0, 0};
  bool g_warm = false;  // an eager step ran (lazy allocations are made outside any capture)
  unsigned int* bad_flag = nullptr;
  unsigned long long* bad_idx = nullptr;
  long long launches = 0;
  long long last_bad = -1;
  double* host_stage = nullptr;     // device state for cg_advance_host
  int iface_dir = -1;               // diagnostics: direction whose interface fluxes are written
  double* iface_out = nullptr;
  DevLine c6grad[3], c6flux[3], filt[3];  // LAD-C6 line systems
  int sweep_lw[3] = {cgk::sweep_lw(0), cgk::sweep_lw(1), cgk::sweep_lw(2)};  // lines per sweep tile (autotuned or default)
  double* prof[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};  // inflow profiles
  // kernel timing (cg_timing_enable): CUDA events around the sweep launches
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_open;
};

static void fill_devgrid(const cg_grid* g, const cg_params* p, DevGrid& d) {
  memset(&d, 0, sizeof d);
  d.nd = g->nd;
  d.nv = g->nd + 2;
  d.N = 1;
  d.NP = 1;
  for (int k = 0; k < 3; ++k) {
    d.n[k] = g->n[k];
    d.N *= g->n[k];
    d.P[k] = g->n[k] + (k < g->nd ? 2 * PM : 0);
    d.NP *= d.P[k];
    d.bc[k][0] = g->bc[k][0];
    d.bc[k][1] = g->bc[k][1];
    for (int s = 0; s < 2; ++s) {
      double W[5] = {0, 0, 0, 0, 0}, Q[5];
      for (int v = 0; v < d.nv; ++v) W[v] = p->inflow[k][s][v];
      // conserved form of the inflow state (ideal gas)
      double q = 0.0;
      Q[0] = W[0];
      for (int m = 0; m < g->nd; ++m) {
        Q[1 + m] = W[0] * W[1 + m];
        q += W[1 + m] * W[1 + m];
      }
      Q[g->nd + 1] = W[g->nd + 1] / (p->gamma - 1.0) + 0.5 * W[0] * q;
      for (int v = 0; v < 5; ++v) {
        d.inflowW[k][s][v] = W[v];
        d.inflowQ[k][s][v] = v < d.nv ? Q[v] : 0.0;
      }
    }
  }
  d.gamma = p->gamma;
  d.gm1 = p->gamma - 1.0;
  d.gm2 = p->gamma * p->minf * p->minf;
  d.curv = g->curv;
  int nd = g->nd;
  if (!g->curv) {
    double h0 = g->h[0], h1 = g->h[1], h2 = g->h[2];
    if (nd == 1) { d.cxh[0] = 1.0; d.cjac = 1.0 / h0; }
    if (nd == 2) { d.cxh[0] = h1; d.cxh[1] = h0; d.cjac = 1.0 / (h0 * h1); }
    if (nd == 3) { d.cxh[0] = h1 * h2; d.cxh[1] = h0 * h2; d.cxh[2] = h0 * h1; d.cjac = 1.0 / (h0 * h1 * h2); }
    for (int k = 0; k < 3; ++k) d.ch[k] = g->h[k];
    // interface frame of each direction: the metric vector is (0..xi_dd..0)
    for (int dir = 0; dir < nd; ++dir) {
      double xi[3] = {0, 0, 0};
      xi[dir] = d.cxh[dir];
      double g2 = 0.0;
      for (int m = 0; m < nd; ++m) g2 += xi[m] * xi[m];
      double ig = 1.0 / sqrt(g2);
      double n[3] = {0, 0, 0}, t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0};
      for (int m = 0; m < nd; ++m) n[m] = xi[m] * ig;
      if (nd == 2) { t1[0] = -n[1]; t1[1] = n[0]; }
      if (nd == 3) {
        int s = 0;
        if (fabs(n[1]) < fabs(n[s])) s = 1;
        if (fabs(n[2]) < fabs(n[s])) s = 2;
        int a = (s + 1) % 3, b = (s + 2) % 3;
        double r = 1.0 / sqrt(n[a] * n[a] + n[b] * n[b]);
        t1[s] = 0.0;
        t1[a] = -n[b] * r;
        t1[b] = n[a] * r;
        t2[0] = n[1] * t1[2] - n[2] * t1[1];
        t2[1] = n[2] * t1[0] - n[0] * t1[2];
        t2[2] = n[0] * t1[1] - n[1] * t1[0];
      }
      d.cg2[dir] = g2;
      d.cg[dir] = sqrt(g2);
      d.cig[dir] = ig;
      d.cig2[dir] = 1.0 / g2;
      for (int m = 0; m < 3; ++m) { d.cn[dir][m] = n[m]; d.ct1[dir][m] = t1[m]; d.ct2[dir][m] = t2[m]; }
    }
  }
  d.twall = p->twall;
  d.visc = p->viscous ? 1 : 0;
  d.re = p->re;
  d.suth = p->suth;
  d.kc = (p->gamma - 1.0) * p->pr * p->minf * p->minf;
  for (int k = 0; k < 3; ++k) d.pf[k] = d.N / d.n[k];
  d.f_gamma = (float)d.gamma;
  d.f_gm1 = (float)d.gm1;
  d.f_gm2 = (float)d.gm2;
  d.f_cjac = (float)d.cjac;
  for (int k = 0; k < 3; ++k) {
    d.cjxh[k] = d.cjac * d.cxh[k];
    d.f_cjxh[k] = (float)d.cjxh[k];
    d.f_cxh[k] = (float)d.cxh[k];
    d.f_ch[k] = (float)d.ch[k];
    d.f_cg2[k] = (float)d.cg2[k];
    d.f_cg[k] = (float)d.cg[k];
    d.f_cig2[k] = (float)d.cig2[k];
    for (int m = 0; m < 3; ++m) {
      d.f_cn[k][m] = (float)d.cn[k][m];
      d.f_ct1[k][m] = (float)d.ct1[k][m];
      d.f_ct2[k][m] = (float)d.ct2[k][m];
    }
  }
}

static Box make_box(const cg_solver* s, int grow_all, int dir, int grow_dir) {
  Box b;
  for (int k = 0; k < 3; ++k) {
    int gr = k < s->nd ? (k == dir ? grow_dir : grow_all) : 0;
    b.off[k] = gr;
    b.ext[k] = s->dg.n[k] + 2 * gr;
  }
  return b;
}

// Line buffer along d: rows [lo, lo+m) (periodic: the n nodes), lines over
// the other active directions grown by `grow`.
static LineBuf make_lines(const cg_solver* s, int d, int lo, int m_nonper, int grow) {
  LineBuf lb;
  lb.d = d;
  lb.n = s->dg.n[d];
  lb.periodic = s->grid->bc[d][0] == CG_BC_PERIODIC;
  lb.lo = lb.periodic ? 0 : lo;
  lb.m = lb.periodic ? lb.n : m_nonper;
  lb.nl = 1;
  for (int k = 0; k < 3; ++k) {
    int gr = (k < s->nd && k != d) ? grow : 0;
    lb.off[k] = gr;
    lb.ext[k] = k == d ? 1 : s->dg.n[k] + 2 * gr;
    if (k != d) lb.nl *= lb.ext[k];
  }
  return lb;
}

// bytes this thread has allocated through dalloc (a solver's device footprint
// is the difference across its creation plus its lazily allocated buffers)
static thread_local size_t t_dalloc_bytes = 0;

template <typename T>
static int dalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(CG_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
  }
  t_dalloc_bytes += count * sizeof(T);
  return CG_OK;
}

static int upload_line(DevLine& L, int m, double a, bool cyclic, int lo, long long launch_columns) {
  HostLine h = make_line(m, a, cyclic);
  int rc = dalloc(&L.buf, (size_t)3 * m);
  if (rc) return rc;
  std::vector<double> all(3 * (size_t)m, 0.0);
  for (int i = 0; i < m; ++i) {
    all[i] = h.cp[i];
    all[m + i] = 1.0 / h.den[i];  // the recurrence multiplies by the reciprocal pivot
    all[2 * m + i] = cyclic ? h.z[i] : 0.0;
  }
  CG_CUDA(cudaMemcpy(L.buf, all.data(), all.size() * sizeof(double), cudaMemcpyHostToDevice));
  L.lc.cp = L.buf;
  L.lc.den = L.buf + m;
  L.lc.z = L.buf + 2 * m;
  L.lc.a = a;
  L.lc.gam = h.gam;
  L.lc.fden = h.fden;
  L.lc.m = m;
  L.lc.lo = lo;
  L.lc.periodic = cyclic ? 1 : 0;
  int P = choose_parts(m, launch_columns);
  if (P >= 4) {
    std::vector<double> A, B, C;
    double gam = -1.0;
    line_rows(m, a, cyclic, A, B, C, &gam);
    HostPart hp = make_part(A, B, C, P);
    size_t cnt = 5 * (size_t)m + hp.ch.size();
    rc = dalloc(&L.pbuf, cnt);
    if (rc) return rc;
    std::vector<double> pk;
    pk.reserve(cnt);
    for (auto* v : {&hp.aL, &hp.cp, &hp.rd, &hp.V, &hp.W, &hp.ch}) pk.insert(pk.end(), v->begin(), v->end());
    CG_CUDA(cudaMemcpy(L.pbuf, pk.data(), cnt * sizeof(double), cudaMemcpyHostToDevice));
    L.pc.aL = L.pbuf;
    L.pc.cp = L.pbuf + m;
    L.pc.rd = L.pbuf + 2 * (size_t)m;
    L.pc.V = L.pbuf + 3 * (size_t)m;
    L.pc.W = L.pbuf + 4 * (size_t)m;
    L.pc.ch = L.pbuf + 5 * (size_t)m;
    L.pc.z = cyclic ? L.lc.z : nullptr;
    L.pc.a = a;
    L.pc.gam = h.gam;
    L.pc.fden = h.fden;
    L.pc.m = m;
    L.pc.q = hp.q;
    L.pc.P = hp.P;
    L.pc.periodic = cyclic ? 1 : 0;
    std::vector<float> pf(pk.begin(), pk.end());
    rc = dalloc(&L.fpbuf, cnt);
    if (rc) return rc;
    CG_CUDA(cudaMemcpy(L.fpbuf, pf.data(), cnt * sizeof(float), cudaMemcpyHostToDevice));
    L.pcf = PartCoefT<float>{L.fpbuf, L.fpbuf + m, L.fpbuf + 2 * (size_t)m, L.fpbuf + 3 * (size_t)m,
                             L.fpbuf + 4 * (size_t)m, nullptr, L.fpbuf + 5 * (size_t)m, (float)a, (float)h.gam,
                             (float)h.fden, m, hp.q, hp.P, cyclic ? 1 : 0};
  }
  // FP32 mirror of the Thomas factors (and of z, which the partitioned form shares)
  {
    std::vector<float> af(all.begin(), all.end());
    rc = dalloc(&L.fbuf, af.size());
    if (rc) return rc;
    CG_CUDA(cudaMemcpy(L.fbuf, af.data(), af.size() * sizeof(float), cudaMemcpyHostToDevice));
    L.lcf = LineCoefT<float>{L.fbuf, L.fbuf + m, L.fbuf + 2 * (size_t)m, (float)a, (float)h.gam, (float)h.fden,
                             m, lo, cyclic ? 1 : 0};
    if (L.pcf.P) L.pcf.z = cyclic ? L.lcf.z : nullptr;
  }
  return CG_OK;
}

// ---------------------------------------------------------------- metrics
static int compute_metrics(cg_solver* s, cudaStream_t st) {
  const cg_grid* g = s->grid;
  int nd = g->nd;
  EBox eb;
  eb.nd = nd;
  eb.NE = 1;
  for (int d = 0; d < 3; ++d) {
    eb.n[d] = g->n[d];
    eb.ge[d] = d < nd ? MGC : 0;
    eb.PE[d] = eb.n[d] + 2 * eb.ge[d];
    eb.NE *= eb.PE[d];
  }
  int six = (s->p.scheme == CG_MEG6 || s->p.scheme == CG_MIG4) ? 1 : 0;
  const bool c6 = s->p.scheme == CG_LAD_C6;
  std::vector<double*> tmp;
  size_t tmp_bytes = 0;
  auto alloc = [&](double** p) -> int {
    int rc = dalloc(p, (size_t)eb.NE);
    if (!rc) { tmp.push_back(*p); tmp_bytes += (size_t)eb.NE * sizeof(double); }
    return rc;
  };
  int threads = 256, blocks = grid_blocks(eb.NE, threads);
  int per[3] = {0, 0, 0};
  for (int d = 0; d < nd; ++d) per[d] = g->bc[d][0] == CG_BC_PERIODIC;
  // LAD-C6: line scratch of the compact metric operator (4 (n + 4) doubles a line)
  double* c6scr = nullptr;
  if (c6) {
    size_t mx = 0;
    for (int d = 0; d < nd; ++d) mx = std::max(mx, (size_t)(eb.NE / eb.PE[d]) * 4 * (size_t)(eb.n[d] + 4));
    if (dalloc(&c6scr, mx)) return CG_ERR_OOM;
    tmp.push_back(c6scr);
    tmp_bytes += mx * sizeof(double);
  }
  // derivative of f along d with the scheme's metric operator into o
  auto mop = [&](const double* f, int d, int detrend, double* o) {
    km_op<<<blocks, threads, 0, st>>>(eb, f, d, 0, c6 ? 0 : six, o);
    if (c6)
      km_c6<<<grid_blocks(eb.NE / eb.PE[d], 128), 128, 0, st>>>(eb, f, d, per[d], detrend, o, c6scr);
  };
  double* X[3] = {nullptr, nullptr, nullptr};
  for (int m = 0; m < nd; ++m) {
    if (alloc(&X[m])) return CG_ERR_OOM;
    km_load<<<blocks, threads, 0, st>>>(eb, g->xyz, s->N, m, X[m]);
    for (int d = 0; d < nd; ++d) {
      int per = g->bc[d][0] == CG_BC_PERIODIC;
      km_extend<<<blocks, threads, 0, st>>>(eb, d, per, g->period[d][m], X[m]);
    }
  }
  double* dX[3][3] = {};
  for (int l = 0; l < nd; ++l)
    for (int m = 0; m < nd; ++m) {
      if (alloc(&dX[l][m])) return CG_ERR_OOM;
      mop(X[m], l, 1, dX[l][m]);
    }
  double* node[3][3] = {};
  double* vol;
  if (alloc(&vol)) return CG_ERR_OOM;
  for (int l = 0; l < nd; ++l)
    for (int m = 0; m < nd; ++m)
      if (alloc(&node[l][m])) return CG_ERR_OOM;
  if (nd == 1) {
    std::vector<double> ones(eb.NE, 1.0);
    CG_CUDA(cudaMemcpyAsync(node[0][0], ones.data(), eb.NE * sizeof(double), cudaMemcpyHostToDevice, st));
    CG_CUDA(cudaStreamSynchronize(st));
  } else if (nd == 2) {
    km_lin<<<blocks, threads, 0, st>>>(eb, dX[1][1], nullptr, 0, node[0][0]);
    km_lin<<<blocks, threads, 0, st>>>(eb, dX[1][0], nullptr, 2, node[0][1]);
    km_lin<<<blocks, threads, 0, st>>>(eb, dX[0][1], nullptr, 2, node[1][0]);
    km_lin<<<blocks, threads, 0, st>>>(eb, dX[0][0], nullptr, 0, node[1][1]);
  } else {
    // Thomas-Lombard form; LAD-C6 (cyclic compact operator) splits the
    // undifferentiated coordinate into its periodic part and linear trend,
    // whose terms (D_{l1} x_a) s[l2][b] - (D_{l2} x_a) s[l1][b] are added exactly
    double slope[3][3] = {};
    double* Xp[3] = {X[0], X[1], X[2]};
    if (c6) {
      for (int d = 0; d < 3; ++d)
        for (int b = 0; b < 3; ++b) slope[d][b] = per[d] ? g->period[d][b] / (double)g->n[d] : 0.0;
      for (int b = 0; b < 3; ++b) {
        if (alloc(&Xp[b])) return CG_ERR_OOM;
        km_detrend<<<blocks, threads, 0, st>>>(eb, X[b], slope[0][b], slope[1][b], slope[2][b], Xp[b]);
      }
    }
    double* P[3][3];
    for (int lp = 0; lp < 3; ++lp)
      for (int m = 0; m < 3; ++m) {
        if (alloc(&P[lp][m])) return CG_ERR_OOM;
        km_lin<<<blocks, threads, 0, st>>>(eb, dX[lp][(m + 1) % 3], Xp[(m + 2) % 3], 1, P[lp][m]);
      }
    double *A, *B;
    if (alloc(&A) || alloc(&B)) return CG_ERR_OOM;
    for (int l = 0; l < 3; ++l) {
      int l1 = (l + 1) % 3, l2 = (l + 2) % 3;
      for (int m = 0; m < 3; ++m) {
        mop(P[l1][m], l2, 0, A);
        mop(P[l2][m], l1, 0, B);
        km_lin<<<blocks, threads, 0, st>>>(eb, A, B, 3, node[l][m]);
        if (c6) {
          int a = (m + 1) % 3, b = (m + 2) % 3;
          km_trend<<<blocks, threads, 0, st>>>(eb, dX[l1][a], slope[l2][b], dX[l2][a], slope[l1][b], node[l][m]);
        }
      }
    }
  }
  km_vol<<<blocks, threads, 0, st>>>(eb, nd, dX[0][0], nd > 1 ? dX[0][1] : nullptr, nd > 2 ? dX[0][2] : nullptr,
                                     nd > 1 ? dX[1][0] : nullptr, nd > 1 ? dX[1][1] : nullptr,
                                     nd > 2 ? dX[1][2] : nullptr, nd > 2 ? dX[2][0] : nullptr,
                                     nd > 2 ? dX[2][1] : nullptr, nd > 2 ? dX[2][2] : nullptr, vol);
  double* ifc;
  if (alloc(&ifc)) return CG_ERR_OOM;
  // planes: xh (nd*nd), xt (nd*nd), jac (1), dxl (nd*nd)
  long long NP = s->dg.NP;
  int pb = grid_blocks(NP, threads);
  double* xh = s->metric;
  double* xt = xh + (size_t)nd * nd * NP;
  double* jac = xt + (size_t)nd * nd * NP;
  double* dxl = jac + NP;
  for (int l = 0; l < nd; ++l)
    for (int m = 0; m < nd; ++m) {
      km_store<<<pb, threads, 0, st>>>(eb, s->dg, node[l][m], 0, xh + (size_t)(l * nd + m) * NP);
      km_op<<<blocks, threads, 0, st>>>(eb, node[l][m], l, 1, six, ifc);
      km_store<<<pb, threads, 0, st>>>(eb, s->dg, ifc, 0, xt + (size_t)(l * nd + m) * NP);
      km_disp<<<pb, threads, 0, st>>>(eb, s->dg, X[m], l, dxl + (size_t)(l * nd + m) * NP);
    }
  km_store<<<pb, threads, 0, st>>>(eb, s->dg, vol, 1, jac);
  CG_CUDA(cudaGetLastError());
  CG_CUDA(cudaStreamSynchronize(st));
  for (double* p : tmp) cudaFree(p);
  t_dalloc_bytes -= tmp_bytes;  // set-up buffers: not held by the solver
  s->dg.xh = xh;
  s->dg.xt = xt;
  s->dg.jac = jac;
  s->dg.dxl = dxl;
  return CG_OK;
}


// ---------------------------------------------------------------- timing
static cudaEvent_t timing_event(cg_solver* s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
struct TimedRegion {
  cg_solver* s;
  int cls;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  TimedRegion(cg_solver* s_, int c, cudaStream_t st_) : s(s_), cls(c), st(st_) {
    if (s->timing) {
      a = timing_event(s);
      cudaEventRecord(a, st);
    }
  }
  ~TimedRegion() {
    if (s->timing) {
      cudaEvent_t b = timing_event(s);
      cudaEventRecord(b, st);
      s->ev_open.push_back({cls, {a, b}});
    }
  }
};

// ---------------------------------------------------------------- launches
template <int ND, bool CART, bool COMPACT>
static void launch_omega(cg_solver* s, cudaStream_t st, const int* guard, int want) {
  long long tot = s->omBox.size();
  if constexpr (ND >= 2 && !COMPACT) {
    const Box& ob = s->omBox;
    dim3 grid((unsigned)((ob.ext[0] + OMT_X - 1) / OMT_X), (unsigned)((ob.ext[1] + OMT_Y - 1) / OMT_Y),
              ND == 3 ? (unsigned)ob.ext[2] : 1u);
    if (s->p.precision == CG_MIXED)
      k_omega_tile<ND, CART, float><<<grid, dim3(OMT_X, OMT_Y), 0, st>>>(
          s->dg, reinterpret_cast<const float*>(s->W), reinterpret_cast<float*>(s->om), ob, guard, want);
    else
      k_omega_tile<ND, CART, double><<<grid, dim3(OMT_X, OMT_Y), 0, st>>>(s->dg, s->W, s->om, ob, guard, want);
    s->launches++;
    return;
  }
  if (s->p.precision == CG_MIXED)
    k_omega<ND, CART, COMPACT, float><<<grid_blocks(tot, 128), 128, 0, st>>>(
        s->dg, reinterpret_cast<const float*>(s->W), reinterpret_cast<const float*>(s->G[0]),
        reinterpret_cast<const float*>(s->G[1]), reinterpret_cast<const float*>(s->G[2]), s->gdLB[0], s->gdLB[1],
        s->gdLB[2], reinterpret_cast<float*>(s->om), s->omBox, guard, want);
  else
    k_omega<ND, CART, COMPACT, double><<<grid_blocks(tot, 128), 128, 0, st>>>(
        s->dg, s->W, s->G[0], s->G[1], s->G[2], s->gdLB[0], s->gdLB[1], s->gdLB[2], s->om, s->omBox, guard, want);
  s->launches++;
}

static GbrCfg gbr_cfg(const cg_solver* s) {
  GbrCfg q;
  q.gamma = s->p.gamma;
  q.gm1 = s->p.gamma - 1.0;
  q.thr = s->p.sensor_thresh;
  q.eps = s->p.mp_eps;
  q.alpha = s->p.mp_alpha;
  q.window = s->p.omega_window;
  q.f_gamma = (float)q.gamma;
  q.f_gm1 = (float)q.gm1;
  q.f_thr = (float)q.thr;
  q.f_eps = (float)q.eps;
  q.f_alpha = (float)q.alpha;
  return q;
}

template <int ND, int DIR, bool CART, bool COMPACT>
static int launch_sweep(cg_solver* s, const StageArgs& A, cudaStream_t st) {
  TimedRegion tr(s, CG_TIMING_SWEEP, st);
  int form = s->p.precision == CG_MIXED ? kSweepFP32 : (s->p.fma_sweep ? kSweepContracted : kSweepExact);
  int e = launch_sweep_any(form, ND, DIR, s->sweep_lw[DIR], CART, COMPACT, s->dg, gbr_cfg(s), A, st);
  if (e) return fail(CG_ERR_CUDA, "sweep launch (dir %d, %d lines per tile): %s", DIR, s->sweep_lw[DIR],
                     cudaGetErrorString((cudaError_t)e));
  s->launches++;
  return CG_OK;
}

template <int ND, bool CART, bool COMPACT>
static int sweep_dir(cg_solver* s, int dir, const StageArgs& A, cudaStream_t st) {
  if (dir == 0) return launch_sweep<ND, 0, CART, COMPACT>(s, A, st);
  if (ND >= 2 && dir == 1) return launch_sweep<ND, (ND >= 2 ? 1 : 0), CART, COMPACT>(s, A, st);
  if (ND >= 3 && dir == 2) return launch_sweep<ND, (ND >= 3 ? 2 : 0), CART, COMPACT>(s, A, st);
  return fail(CG_ERR_INVALID_ARG, "bad direction");
}

// Line solves of up to three systems in one launch.  Many columns: one thread
// per column in 32-thread blocks, so the long recurrences spread over as many
// SMs as possible.  Few columns (every system partitioned at set-up): the
// partitioned solver, 32 columns times the chunks per block.
template <typename T = double>
struct LineJob {
  const DevLine* L;
  T* x;
  long long nl;
  int ncomp;
  C6Src<T> src{};  // f set: the solver forms the C6 right-hand sides itself
};

// Whether launch_lines takes the partitioned solver for these jobs.
template <typename T>
static bool lines_partitioned(const LineJob<T>* jobs, int n) {
  bool part = true;
  for (int j = 0; j < n; ++j) part = part && jobs[j].L->pc.P >= 4;
  return part;
}

// Whether the solver should form the C6 right-hand sides itself: always on
// the one-thread-per-line path (taken when lines are many), and on the
// partitioned path with columns enough (32 an SM) that the longer chunk
// prologue (the window and its look-ahead loads) is hidden; a latency-bound
// launch of a few columns (a 1D tube) keeps the separate right-hand-side pass.
template <typename T>
static bool rhs_in_solver(const LineJob<T>* jobs, int n) {
  long long cols = 0;
  for (int j = 0; j < n; ++j) cols += jobs[j].nl * jobs[j].ncomp;
  return !lines_partitioned(jobs, n) || cols >= 152LL * 32;
}

template <typename T>
static void launch_lines(const LineJob<T>* jobs, int n, cudaStream_t st) {
  bool part = true;
  for (int j = 0; j < n; ++j) part = part && jobs[j].L->pc.P >= 4;
  if (part) {
    PartJobsT<T> J;
    J.njobs = n;
    J.start[0] = 0;
    int Pmax = 1;
    for (int j = 0; j < n; ++j) {
      J.pc[j] = part_coef<T>(*jobs[j].L);
      J.src[j] = jobs[j].src;
      J.x[j] = jobs[j].x;
      J.nl[j] = jobs[j].nl;
      J.ncomp[j] = jobs[j].ncomp;
      J.start[j + 1] = J.start[j] + (jobs[j].nl * jobs[j].ncomp + 31) / 32 * 32;
      Pmax = std::max(Pmax, J.pc[j].P);
    }
    k_tri_part<T><<<(unsigned)(J.start[n] / 32), dim3(32, Pmax), 0, st>>>(J);
    return;
  }
  ThomasJobsT<T> J;
  J.njobs = n;
  J.start[0] = 0;
  for (int j = 0; j < n; ++j) {
    J.lc[j] = line_coef<T>(*jobs[j].L);
    J.src[j] = jobs[j].src;
    J.x[j] = jobs[j].x;
    J.nl[j] = jobs[j].nl;
    J.ncomp[j] = jobs[j].ncomp;
    J.start[j + 1] = J.start[j] + jobs[j].nl * jobs[j].ncomp;
  }
  long long cols = J.start[n];
  k_thomas_jobs<T><<<(unsigned)((cols + 31) / 32), 32, 0, st>>>(J);
}

// Right-hand sides of the compact line systems: staged through shared memory
// (k_rhs_tile), or by the per-row kernels when there are too few lines.
template <int ND, typename T>
static void launch_rhs_c6(const T* f, Box fb, int nc, const LineBuf& lb, T* r, cudaStream_t st) {
  if (use_tile(lb)) {
    using Tl = XTileC6<T, ND + 3>;
    k_rhs_tile<T, ND + 3, 2, Tl><<<tile_grid(lb), XT_THREADS, 0, st>>>(lb, Tl{f, fb, fb.size(), nc}, r);
  } else {
    k_rhs_c6<T><<<grid_blocks((long long)lb.m * lb.nl, 256), 256, 0, st>>>(f, fb, nc, lb, r);
  }
}

template <int ND, typename TW, typename TR>
static void launch_rhs_mig4(const DevGrid& g, const TW* W, const LineBuf& lb, TR* r, cudaStream_t st) {
  if (use_tile(lb)) {
    using Tl = XTileMig4<ND, TW, TR>;
    k_rhs_tile<TR, ND + 2, 1, Tl><<<tile_grid(lb), XT_THREADS, 0, st>>>(lb, Tl{g, W, ND + 2}, r);
  } else {
    k_rhs_mig4<ND, TW, TR><<<grid_blocks((long long)lb.m * lb.nl, 256), 256, 0, st>>>(g, W, lb, r);
  }
}

template <int ND>
static void launch_rhs_filter(const DevGrid& g, const double* U, const LineBuf& lb, const double b[5], double* r,
                              cudaStream_t st) {
  if (use_tile(lb)) {
    using Tl = XTileFilter<ND>;
    k_rhs_tile<double, ND + 2, 4, Tl><<<tile_grid(lb), XT_THREADS, 0, st>>>(
        lb, Tl{g, U, b[0], b[1], b[2], b[3], b[4], ND + 2}, r);
  } else {
    k_rhs_filter<ND><<<grid_blocks((long long)lb.m * lb.nl, 256), 256, 0, st>>>(g, U, lb, b[0], b[1], b[2], b[3],
                                                                              b[4], r);
  }
}

// Primitives of Uc into W: FP64 storage, or FP32 for the mixed form (the
// recovery itself is FP64 in both).
// With a fused CFL step pending (rk3_cfl), the launch also reduces the CFL
// maximum of Uc and the step size follows from it before anything reads dt.
template <int ND>
static void launch_prim(cg_solver* s, const double* Uc, cudaStream_t st) {
  const bool mixed = s->p.precision == CG_MIXED;
  if (s->prim_ready) {
    s->prim_ready = false;
    return;
  }
  if (s->prim_cfl) {
    s->prim_cfl = false;
    cudaMemsetAsync(s->cflmax, 0, sizeof(unsigned long long), st);
    const int nb = grid_blocks(s->N, 256);
    if (s->dg.curv) {
      if (mixed) k_prim_cfl<ND, false, float><<<nb, 256, 0, st>>>(s->dg, Uc, reinterpret_cast<float*>(s->W), s->cflmax);
      else k_prim_cfl<ND, false, double><<<nb, 256, 0, st>>>(s->dg, Uc, s->W, s->cflmax);
    } else {
      if (mixed) k_prim_cfl<ND, true, float><<<nb, 256, 0, st>>>(s->dg, Uc, reinterpret_cast<float*>(s->W), s->cflmax);
      else k_prim_cfl<ND, true, double><<<nb, 256, 0, st>>>(s->dg, Uc, s->W, s->cflmax);
    }
    k_cfl_finish<<<1, 1, 0, st>>>(s->cflmax, s->p.cfl, s->prim_cfl_dt, s->prim_cfl_t, 0.0);
    s->launches += 3;
    return;
  }
  if (mixed)
    k_prim<ND, float><<<grid_blocks(s->N, 256), 256, 0, st>>>(s->dg, Uc, reinterpret_cast<float*>(s->W));
  else
    k_prim<ND, double><<<grid_blocks(s->N, 256), 256, 0, st>>>(s->dg, Uc, s->W);
  s->launches++;
}

// Primitives, sensor (and compact gradients) of the state Uc into W, om, G.
template <int ND>
static int stage_prep_gbr(cg_solver* s, const double* Uc, bool compact, cudaStream_t st, bool prim = true,
                          const int* guard = nullptr, int want = 0) {
  if (prim) {
    launch_prim<ND>(s, Uc, st);
  }
  if (compact) {
    if (s->p.precision == CG_MIXED) {  // the mixed form's gradients: FP32 right-hand sides and solves
      LineJob<float> jobs[3];
      for (int d = 0; d < ND; ++d) {
        const LineBuf& lb = s->gdLB[d];
        float* G = reinterpret_cast<float*>(s->G[d]);
        launch_rhs_mig4<ND, float, float>(s->dg, reinterpret_cast<const float*>(s->W), lb, G, st);
        s->launches++;
        jobs[d] = LineJob<float>{&s->mig4[d], G, lb.nl, ND + 2};
      }
      launch_lines(jobs, ND, st);
    } else {
      LineJob<double> jobs[3];
      for (int d = 0; d < ND; ++d) {
        const LineBuf& lb = s->gdLB[d];
        launch_rhs_mig4<ND, double, double>(s->dg, s->W, lb, s->G[d], st);
        s->launches++;
        jobs[d] = LineJob<double>{&s->mig4[d], s->G[d], lb.nl, ND + 2};
      }
      launch_lines(jobs, ND, st);
    }
    s->launches++;
  }
  if (s->dg.curv) {
    if (compact) launch_omega<ND, false, true>(s, st, guard, want);
    else launch_omega<ND, false, false>(s, st, guard, want);
  } else {
    if (compact) launch_omega<ND, true, true>(s, st, guard, want);
    else launch_omega<ND, true, false>(s, st, guard, want);
  }
  return CG_OK;
}

template <int ND>
static int stage_prep_prim(cg_solver* s, const double* Uc, cudaStream_t st) {
  launch_prim<ND>(s, Uc, st);
  return CG_OK;
}

static StageArgs base_args(cg_solver* s) {
  StageArgs A;
  memset(&A, 0, sizeof A);
  A.W = s->W;
  A.Wf = reinterpret_cast<const float*>(s->W);
  A.om = s->om;
  A.omBox = s->omBox;
  A.acc = s->acc;
  A.bad_flag = s->bad_flag;
  A.bad_idx = s->bad_idx;
  A.dt = s->dt;
  return A;
}

// One evaluation of the C-GBR fluxes over all directions with the epilogue of A.
template <int ND>
static int gbr_sweeps(cg_solver* s, bool compact, StageArgs A, cudaStream_t st, bool fresh = true) {
  for (int d = 0; d < ND; ++d) {
    A.first = fresh && d == 0;
    A.last = d == ND - 1;
    A.Gd = s->G[d];
    A.Gdf = reinterpret_cast<const float*>(s->G[d]);
    A.gdLB = s->gdLB[d];
    A.iface_out = (s->iface_out && s->iface_dir == d) ? s->iface_out : nullptr;
    int rc;
    if (s->dg.curv) rc = compact ? sweep_dir<ND, false, true>(s, d, A, st) : sweep_dir<ND, false, false>(s, d, A, st);
    else rc = compact ? sweep_dir<ND, true, true>(s, d, A, st) : sweep_dir<ND, true, false>(s, d, A, st);
    if (rc) return rc;
  }
  return CG_OK;
}

template <int ND>
static int lad_stage(cg_solver* s, const double* Uc, StageArgs A, cudaStream_t st);
template <int ND>
static void visc_pass_any(cg_solver* s, StageArgs A, cudaStream_t st, bool have_grad, const int* guard, int want);
template <int ND>
static int lad_filter(cg_solver* s, double* U, cudaStream_t st);
static int lad_alloc(cg_solver* s);
static void lad_free(LadBuffers& b);

// The mixed form's deferred update of stage stage_no (k_stage_update, the
// increment form of TVD-RK3, its FP32 increment sum in the U1 buffer); before
// stage 3 it writes the next stage's primitives into W instead of a state.
template <int ND>
static void launch_update(cg_solver* s, const StageArgs& A, int stage_no, cudaStream_t st) {
  const bool next = stage_no < 3;
  float* Z = reinterpret_cast<float*>(s->U1);
  float* Wn = reinterpret_cast<float*>(s->W);
  const int nb = grid_blocks(s->N, 256);
  auto go = [&](auto cart) {
    constexpr bool C = decltype(cart)::value;
    if (stage_no == 1) k_stage_update<ND, C, 1><<<nb, 256, 0, st>>>(s->dg, A, Z, Wn);
    else if (stage_no == 2) k_stage_update<ND, C, 2><<<nb, 256, 0, st>>>(s->dg, A, Z, Wn);
    else k_stage_update<ND, C, 3><<<nb, 256, 0, st>>>(s->dg, A, Z, Wn);
  };
  if (s->dg.curv) go(std::false_type{});
  else go(std::true_type{});
  s->launches++;
  s->prim_ready = next;
}

// RHS or RK stage: out = R (rk = 0) or the stage combination (rk = 1).  In the
// mixed form an RK stage's fluxes only sum into acc, and k_stage_update
// applies the FP64 residual and update as a pass of its own.
template <int ND>
static int stage(cg_solver* s, const double* Uc, const double* Un, double* out, int rk, int stage_no,
                 cudaStream_t st) {
  int sch = s->p.scheme;
  StageArgs A = base_args(s);
  A.rk = rk;
  A.stage = stage_no;
  A.R = out;
  A.Un = Un;
  A.Uc = Uc;
  A.Uout = out;
  A.defer = (rk && s->p.precision == CG_MIXED) ? 1 : 0;
  // the deferred stages 2 and 3 start from the primitives the previous update wrote
  if (A.defer && stage_no > 1 && !s->prim_ready) return fail(CG_ERR_UNSUPPORTED, "stage %d has no primitives", stage_no);
  int rc;
  if (sch == CG_MEG6 || sch == CG_MIG4) {
    bool compact = sch == CG_MIG4;
    stage_prep_gbr<ND>(s, Uc, compact, st);
    if (s->p.viscous) visc_pass_any<ND>(s, A, st, false, nullptr, 0);
    rc = gbr_sweeps<ND>(s, compact, A, st, !s->p.viscous);
  } else {
    rc = lad_stage<ND>(s, Uc, A, st);
  }
  if (rc) return rc;
  if (A.defer) launch_update<ND>(s, A, stage_no, st);
  return CG_OK;
}

// In the mixed form the stage states u1, u2 are not stored (k_stage_update
// hands their primitives on in W), so stages 2 and 3 name U as their state.
template <int ND>
static int rk3_stages(cg_solver* s, double* U, cudaStream_t st) {
  int rc;
  if (s->p.precision == CG_MIXED) {
    if ((rc = stage<ND>(s, U, U, U, 1, 1, st))) return rc;
    if ((rc = stage<ND>(s, U, U, U, 1, 2, st))) return rc;
    if ((rc = stage<ND>(s, U, U, U, 1, 3, st))) return rc;
    if (s->p.scheme == CG_LAD_C6 && s->p.filter_on) return lad_filter<ND>(s, U, st);
    return CG_OK;
  }
  if ((rc = stage<ND>(s, U, U, s->U1, 1, 1, st))) return rc;
  if ((rc = stage<ND>(s, s->U1, U, s->U2, 1, 2, st))) return rc;
  if ((rc = stage<ND>(s, s->U2, U, U, 1, 3, st))) return rc;
  if (s->p.scheme == CG_LAD_C6 && s->p.filter_on) return lad_filter<ND>(s, U, st);
  return CG_OK;
}

template <int ND>
static int rk3(cg_solver* s, double* U, cudaStream_t st) {
  s->prim_ready = false;
  int rc = rk3_stages<ND>(s, U, st);
  s->prim_ready = false;
  return rc;
}

// The CFL step and one RK3 step with its dt: stage 1's primitive launch
// reduces the CFL maximum of U (every stage path starts with that launch), so
// the state is read once for both.  Results are bitwise those of cfl_launch
// followed by rk3.
template <int ND>
static int rk3_cfl(cg_solver* s, double* U, double* dt_dev, double* t_dev, cudaStream_t st) {
  s->prim_ready = false;
  s->prim_cfl = true;
  s->prim_cfl_dt = dt_dev;
  s->prim_cfl_t = t_dev;
  const bool mixed = s->p.precision == CG_MIXED;
  int rc = stage<ND>(s, U, U, mixed ? U : s->U1, 1, 1, st);
  const bool unused = s->prim_cfl;
  s->prim_cfl = false;
  if (!rc && unused) rc = fail(CG_ERR_UNSUPPORTED, "stage 1 launched no primitive kernel");
  if (!rc) rc = stage<ND>(s, mixed ? U : s->U1, U, mixed ? U : s->U2, 1, 2, st);
  if (!rc) rc = stage<ND>(s, mixed ? U : s->U2, U, U, 1, 3, st);
  if (!rc && s->p.scheme == CG_LAD_C6 && s->p.filter_on) rc = lad_filter<ND>(s, U, st);
  s->prim_ready = false;
  return rc;
}

template <int ND>
static void cfl_launch(cg_solver* s, const double* U, double* dt_dev, double* t_dev, double t_end, cudaStream_t st) {
  cudaMemsetAsync(s->cflmax, 0, sizeof(unsigned long long), st);
  const bool mixed = s->p.precision == CG_MIXED;
  if (s->dg.curv) {
    if (mixed) k_cfl_max<ND, false, float><<<grid_blocks(s->N, 256), 256, 0, st>>>(s->dg, U, s->cflmax);
    else k_cfl_max<ND, false, double><<<grid_blocks(s->N, 256), 256, 0, st>>>(s->dg, U, s->cflmax);
  } else {
    if (mixed) k_cfl_max<ND, true, float><<<grid_blocks(s->N, 256), 256, 0, st>>>(s->dg, U, s->cflmax);
    else k_cfl_max<ND, true, double><<<grid_blocks(s->N, 256), 256, 0, st>>>(s->dg, U, s->cflmax);
  }
  k_cfl_finish<<<1, 1, 0, st>>>(s->cflmax, s->p.cfl, dt_dev, t_dev, t_end);
  s->launches += 2;
}

#define DISPATCH_ND(s, fn, ...)                      \
  ((s)->nd == 1 ? fn<1>(__VA_ARGS__)                 \
   : (s)->nd == 2 ? fn<2>(__VA_ARGS__)               \
                  : fn<3>(__VA_ARGS__))

#include "cg_lad_impl.cuh"

// ---------------------------------------------------------------- autotuner
// Lines per sweep tile, chosen per direction by timing the right-hand side of
// the caller's state with each candidate (one direction at a time, the others
// at their current choice).  Results are kept for the process, keyed by the
// grid's shape and kind and the scheme, so equal-sized grids (a batch) are
// timed once.
namespace {
using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, std::array<int, 3>> g_tune;

TuneKey tune_key(const cg_solver* s) {
  return TuneKey(s->nd, s->dg.n[0], s->dg.n[1], s->dg.n[2], s->p.scheme, s->p.precision, s->dg.curv,
                 s->p.hybrid_mode, s->p.viscous);
}
}  // namespace

static bool uses_sweep(const cg_solver* s) {
  return s->p.scheme == CG_MEG6 || s->p.scheme == CG_MIG4 || s->p.scheme == CG_HYBRID;
}

// ms of one right-hand side of U with the current tile choices (median of reps)
static int time_rhs(cg_solver* s, const double* U, double* R, cudaStream_t st, int reps, float* ms) {
  cudaEvent_t a, b;
  CG_CUDA(cudaEventCreate(&a));
  CG_CUDA(cudaEventCreate(&b));
  std::vector<float> t;
  int rc = DISPATCH_ND(s, stage, s, U, U, R, 0, 1, st);  // warm-up (first launch of a shape)
  for (int r = 0; r < reps && rc == CG_OK; ++r) {
    cudaEventRecord(a, st);
    rc = DISPATCH_ND(s, stage, s, U, U, R, 0, 1, st);
    cudaEventRecord(b, st);
    cudaError_t e = cudaEventSynchronize(b);
    float x = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&x, a, b);
    if (e != cudaSuccess && rc == CG_OK) rc = fail(CG_ERR_CUDA, "autotune timing: %s", cudaGetErrorString(e));
    t.push_back(x);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return CG_OK;
}

static int autotune_solver(cg_solver* s, const double* U, bool force, cudaStream_t st) {
  if (!uses_sweep(s)) return CG_OK;
  TuneKey key = tune_key(s);
  if (!force) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      for (int d = 0; d < 3; ++d) s->sweep_lw[d] = it->second[d];
      return CG_OK;
    }
  }
  double* R = nullptr;
  int rc = dalloc(&R, (size_t)s->nv * s->N);
  if (rc) return rc;
  for (int d = 0; d < s->nd && rc == CG_OK; ++d) {
    const int* cands = d == 0 ? kSweepLwCands0 : kSweepLwCands1;
    int nc = d == 0 ? (int)(sizeof kSweepLwCands0 / sizeof(int)) : (int)(sizeof kSweepLwCands1 / sizeof(int));
    int best = s->sweep_lw[d];
    float best_ms = 1e30f;
    for (int k = 0; k < nc && rc == CG_OK; ++k) {
      s->sweep_lw[d] = cands[k];
      float ms = 0.f;
      rc = time_rhs(s, U, R, st, 3, &ms);
      if (rc == CG_OK && ms < best_ms) {
        best_ms = ms;
        best = cands[k];
      }
    }
    s->sweep_lw[d] = best;
  }
  cudaFree(R);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = {s->sweep_lw[0], s->sweep_lw[1], s->sweep_lw[2]};
  return CG_OK;
}

#include "cg_batch_impl.cuh"

// ======================================================================
extern "C" {

CG_API void cg_params_default(cg_params* p) {
  memset(p, 0, sizeof *p);
  p->gamma = 1.4;
  p->minf = 1.0;
  p->scheme = CG_MEG6;
  p->precision = CG_FP64;
  p->hybrid_mode = CG_HYBRID_GLOBAL;
  p->hybrid_sensor = 0;
  p->hyb_rho = -HUGE_VAL;
  p->hyb_p = -HUGE_VAL;
  p->cfl = 0.2;
  p->c_beta = 1.75;
  p->c_kappa = 0.01;
  p->alpha_f = 0.45;
  p->sensor_thresh = 0.01;
  p->mp_eps = 1e-20;
  p->mp_alpha = 4.0;
  p->filter_on = 1;
  p->omega_window = 4;
  p->viscous = 0;
  p->re = 1.0;
  p->pr = 0.72;
  p->suth = 0.0;
  p->twall = 1.0;
  p->fma_sweep = 0;
  p->hybrid_buffer = 0;
}

CG_API int cg_solver_set_inflow_profile(cg_solver* s, int dir, int side, const double* W_host) {
  if (!s || !W_host) return fail(CG_ERR_INVALID_ARG, "null argument");
  if (dir < 0 || dir >= s->nd || side < 0 || side > 1 || s->grid->bc[dir][side] != CG_BC_INFLOW)
    return fail(CG_ERR_INVALID_ARG, "face (%d, %d) is not an inflow face", dir, side);
  size_t count = (size_t)s->nv * (size_t)s->dg.pf[dir];
  if (!s->prof[dir][side]) {
    size_t b0 = t_dalloc_bytes;
    int rc = dalloc(&s->prof[dir][side], count);
    if (rc) return rc;
    s->dev_bytes += t_dalloc_bytes - b0;
  }
  CG_CUDA(cudaMemcpy(s->prof[dir][side], W_host, count * sizeof(double), cudaMemcpyHostToDevice));
  s->dg.prof[dir][side] = s->prof[dir][side];
  return CG_OK;
}

CG_API const char* cg_last_error(void) { return g_err.c_str(); }

static int check_grid_args(int ndim, const int64_t n[3], const int bc[6]) {
  if (ndim < 1 || ndim > 3) return fail(CG_ERR_INVALID_ARG, "ndim must be 1, 2 or 3");
  for (int d = 0; d < 3; ++d) {
    if (d >= ndim) {
      if (n[d] != 1) return fail(CG_ERR_INVALID_ARG, "unused direction %d must have n = 1", d);
      continue;
    }
    if (n[d] < 1 || n[d] > (1 << 24)) return fail(CG_ERR_INVALID_ARG, "n[%d] out of range", d);
    for (int s = 0; s < 2; ++s)
      if (bc[2 * d + s] < CG_BC_PERIODIC || bc[2 * d + s] > CG_BC_WALL)
        return fail(CG_ERR_INVALID_ARG, "bad boundary type");
    if ((bc[2 * d] == CG_BC_PERIODIC) != (bc[2 * d + 1] == CG_BC_PERIODIC))
      return fail(CG_ERR_INVALID_ARG, "periodic direction %d needs both sides periodic", d);
    if (bc[2 * d] != CG_BC_PERIODIC && n[d] < 8)
      return fail(CG_ERR_INVALID_ARG, "non-periodic direction %d needs n >= 8", d);
  }
  return CG_OK;
}

CG_API int cg_grid_create_cartesian(int ndim, const int64_t n[3], const double h[3], const int bc[6], cg_grid** out) {
  if (!n || !h || !bc || !out) return fail(CG_ERR_INVALID_ARG, "null argument");
  int rc = check_grid_args(ndim, n, bc);
  if (rc) return rc;
  for (int d = 0; d < ndim; ++d)
    if (!(h[d] > 0.0)) return fail(CG_ERR_INVALID_ARG, "spacing must be positive");
  cg_grid* g = new (std::nothrow) cg_grid();
  if (!g) return fail(CG_ERR_OOM, "host allocation failed");
  g->nd = ndim;
  g->curv = 0;
  for (int d = 0; d < 3; ++d) {
    g->n[d] = (int)n[d];
    g->h[d] = d < ndim ? h[d] : 1.0;
    g->bc[d][0] = d < ndim ? bc[2 * d] : CG_BC_PERIODIC;
    g->bc[d][1] = d < ndim ? bc[2 * d + 1] : CG_BC_PERIODIC;
    for (int m = 0; m < 3; ++m) g->period[d][m] = 0.0;
  }
  *out = g;
  return CG_OK;
}

CG_API int cg_grid_create_curvilinear(int ndim, const int64_t n[3], const double* xyz_dev, const double period[9],
                                      const int bc[6], cg_grid** out) {
  if (!n || !xyz_dev || !bc || !out) return fail(CG_ERR_INVALID_ARG, "null argument");
  int rc = check_grid_args(ndim, n, bc);
  if (rc) return rc;
  for (int d = 0; d < ndim; ++d)
    if (bc[2 * d] != CG_BC_PERIODIC && n[d] < 2) return fail(CG_ERR_INVALID_ARG, "need two nodes per line");
  cg_grid* g = new (std::nothrow) cg_grid();
  if (!g) return fail(CG_ERR_OOM, "host allocation failed");
  g->nd = ndim;
  g->curv = 1;
  long long N = 1;
  for (int d = 0; d < 3; ++d) {
    g->n[d] = (int)n[d];
    N *= n[d];
    g->h[d] = 1.0;
    g->bc[d][0] = d < ndim ? bc[2 * d] : CG_BC_PERIODIC;
    g->bc[d][1] = d < ndim ? bc[2 * d + 1] : CG_BC_PERIODIC;
    for (int m = 0; m < 3; ++m) g->period[d][m] = (period && d < ndim && m < ndim) ? period[3 * d + m] : 0.0;
  }
  if (dalloc(&g->xyz, (size_t)ndim * N)) { delete g; return CG_ERR_OOM; }
  cudaError_t e = cudaMemcpy(g->xyz, xyz_dev, sizeof(double) * ndim * N, cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) {
    cudaFree(g->xyz);
    delete g;
    return fail(CG_ERR_CUDA, "coordinate copy failed: %s", cudaGetErrorString(e));
  }
  *out = g;
  return CG_OK;
}

CG_API void cg_grid_destroy(cg_grid* g) {
  if (!g) return;
  if (g->xyz) cudaFree(g->xyz);
  delete g;
}

CG_API void cg_solver_destroy(cg_solver* s) {
  if (!s) return;
  double* bufs[] = {s->metric, s->W, s->acc, s->om, s->U1, s->U2, s->Rtmp, s->G[0], s->G[1], s->G[2],
                    s->hflux[0], s->hflux[1], s->hflux[2], s->dt, s->t, s->host_stage};
  for (double* b : bufs)
    if (b) cudaFree(b);
  for (auto& o : s->ev_open) { cudaEventDestroy(o.second.first); cudaEventDestroy(o.second.second); }
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  for (int d = 0; d < 3; ++d) {
    DevLine* ls[4] = {&s->mig4[d], &s->c6grad[d], &s->c6flux[d], &s->filt[d]};
    for (DevLine* l : ls) {
      if (l->buf) cudaFree(l->buf);
      if (l->pbuf) cudaFree(l->pbuf);
      if (l->fbuf) cudaFree(l->fbuf);
      if (l->fpbuf) cudaFree(l->fpbuf);
    }
  }
  lad_free(s->lad);
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side)
      if (s->prof[d][side]) cudaFree(s->prof[d][side]);
  if (s->mask) cudaFree(s->mask);
  if (s->hyb_flag) cudaFree(s->hyb_flag);
  if (s->hyb_count) cudaFree(s->hyb_count);
  if (s->cflmax) cudaFree(s->cflmax);
  if (s->bad_flag) cudaFree(s->bad_flag);
  if (s->bad_idx) cudaFree(s->bad_idx);
  delete s;
}

// Parameter checks of a solver on grid g, shared by cg_solver_create and
// cg_rhs_meg6_noalloc so that both reject the same inputs.
static int check_params(const cg_grid* g, const cg_params* p) {
  if (p->scheme < CG_MEG6 || p->scheme > CG_HYBRID) return fail(CG_ERR_INVALID_ARG, "bad scheme");
  if (p->precision != CG_FP64 && p->precision != CG_MIXED) return fail(CG_ERR_INVALID_ARG, "bad precision");
  if (!(p->gamma > 1.0) || !(p->cfl > 0.0)) return fail(CG_ERR_INVALID_ARG, "gamma > 1 and cfl > 0 required");
  if (!(p->minf > 0.0)) return fail(CG_ERR_INVALID_ARG, "minf > 0 required");
  if (p->omega_window < 1 || p->omega_window > 4) return fail(CG_ERR_INVALID_ARG, "omega_window must be 1..4");
  if (p->hybrid_buffer < 0 || p->hybrid_buffer > 2) return fail(CG_ERR_INVALID_ARG, "hybrid_buffer must be 0..2");
  if (p->viscous && (!(p->re > 0.0) || !(p->pr > 0.0) || !(p->suth >= 0.0)))
    return fail(CG_ERR_INVALID_ARG, "viscous: re > 0, pr > 0 and suth >= 0 required");
  for (int d = 0; d < g->nd; ++d)
    for (int side = 0; side < 2; ++side)
      if (g->bc[d][side] == CG_BC_WALL && !(p->twall > 0.0))
        return fail(CG_ERR_INVALID_ARG, "isothermal walls need twall > 0");
  return CG_OK;
}

CG_API int cg_solver_create(const cg_grid* g, const cg_params* p, cg_solver** out) {
  if (!g || !p || !out) return fail(CG_ERR_INVALID_ARG, "null argument");
  int prc = check_params(g, p);
  if (prc) return prc;
  cg_solver* s = new (std::nothrow) cg_solver();
  if (!s) return fail(CG_ERR_OOM, "host allocation failed");
  size_t bytes0 = t_dalloc_bytes;
  s->grid = g;
  s->p = *p;
  s->nd = g->nd;
  s->nv = g->nd + 2;
  fill_devgrid(g, p, s->dg);
  s->N = s->dg.N;
  int rc = CG_OK;
  size_t NV = (size_t)s->nv * s->N;
  s->omBox = make_box(s, 4, -1, 4);
  if ((rc = dalloc(&s->W, NV)) || (rc = dalloc(&s->acc, NV)) || (rc = dalloc(&s->U1, NV)) ||
      (rc = dalloc(&s->U2, NV)) || (rc = dalloc(&s->om, (size_t)s->omBox.size())) || (rc = dalloc(&s->dt, 2)) ||
      (rc = dalloc(&s->t, 2)) || (rc = dalloc(&s->cflmax, 1)) || (rc = dalloc(&s->bad_flag, 1)) ||
      (rc = dalloc(&s->bad_idx, 1)) || (rc = dalloc(&s->hyb_flag, 2)) || (rc = dalloc(&s->hyb_count, 1))) {
    cg_solver_destroy(s);
    return rc;
  }
  cudaMemset(s->bad_flag, 0, sizeof(unsigned int));
  cudaMemset(s->bad_idx, 0xff, sizeof(unsigned long long));
  cudaMemset(s->hyb_flag, 0, 2 * sizeof(int));
  cudaMemset(s->hyb_count, 0, sizeof(unsigned long long));
  bool compact = p->scheme == CG_MIG4;
  long long mig4_cols = 0;
  for (int d = 0; d < s->nd; ++d) {
    s->gdLB[d] = make_lines(s, d, -6, g->n[d] + 12, 4);
    mig4_cols += s->gdLB[d].nl * s->nv;
  }
  for (int d = 0; d < s->nd; ++d) {
    if (compact) {
      if ((rc = dalloc(&s->G[d], (size_t)s->nv * s->gdLB[d].m * s->gdLB[d].nl))) { cg_solver_destroy(s); return rc; }
      bool cyc = g->bc[d][0] == CG_BC_PERIODIC;
      int m = cyc ? g->n[d] : g->n[d] + 12;
      if (cyc && m < 3) { cg_solver_destroy(s); return fail(CG_ERR_INVALID_ARG, "periodic compact lines need n >= 3"); }
      if ((rc = upload_line(s->mig4[d], m, 0.25, cyc, -6, mig4_cols))) { cg_solver_destroy(s); return rc; }
    }
  }
  if (g->curv) {
    size_t planes = (size_t)3 * s->nd * s->nd + 1;
    if ((rc = dalloc(&s->metric, planes * (size_t)s->dg.NP))) { cg_solver_destroy(s); return rc; }
    if ((rc = compute_metrics(s, 0))) { cg_solver_destroy(s); return rc; }
  }
  if ((rc = lad_alloc(s))) { cg_solver_destroy(s); return rc; }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { cg_solver_destroy(s); return fail(CG_ERR_CUDA, "setup: %s", cudaGetErrorString(e)); }
  s->dev_bytes = t_dalloc_bytes - bytes0;
  *out = s;
  return CG_OK;
}

CG_API int64_t cg_solver_device_bytes(const cg_solver* s) { return s ? (int64_t)s->dev_bytes : -1; }

CG_API int cg_metrics(cg_solver* s, double* node_dev, double* iface_dev, void* stream) {
  if (!s || !node_dev) return fail(CG_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  int nd = s->nd;
  long long N = s->N;
  std::vector<double> node((size_t)(nd * nd + 1) * N), ifc((size_t)nd * nd * N);
  std::vector<double> xh, xt, jac;
  if (s->dg.curv) {
    long long NP = s->dg.NP;
    std::vector<double> all((size_t)(3 * nd * nd + 1) * NP);
    CG_CUDA(cudaMemcpy(all.data(), s->metric, all.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int k = 0; k < s->dg.n[2]; ++k)
      for (int j = 0; j < s->dg.n[1]; ++j)
        for (int i = 0; i < s->dg.n[0]; ++i) {
          long long q = i + (long long)s->dg.n[0] * (j + (long long)s->dg.n[1] * k);
          long long pq = (i + (nd > 0 ? PM : 0)) +
                         (long long)s->dg.P[0] * ((j + (nd > 1 ? PM : 0)) + (long long)s->dg.P[1] * (k + (nd > 2 ? PM : 0)));
          for (int a = 0; a < nd * nd; ++a) {
            node[(size_t)a * N + q] = all[(size_t)a * NP + pq];
            ifc[(size_t)a * N + q] = all[(size_t)(nd * nd + a) * NP + pq];
          }
          node[(size_t)nd * nd * N + q] = all[(size_t)2 * nd * nd * NP + pq];
        }
  } else {
    for (long long q = 0; q < N; ++q) {
      for (int l = 0; l < nd; ++l)
        for (int m = 0; m < nd; ++m) {
          node[(size_t)(l * nd + m) * N + q] = l == m ? s->dg.cxh[l] : 0.0;
          ifc[(size_t)(l * nd + m) * N + q] = l == m ? s->dg.cxh[l] : 0.0;
        }
      node[(size_t)nd * nd * N + q] = s->dg.cjac;
    }
  }
  CG_CUDA(cudaMemcpyAsync(node_dev, node.data(), node.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  if (iface_dev)
    CG_CUDA(cudaMemcpyAsync(iface_dev, ifc.data(), ifc.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  CG_CUDA(cudaStreamSynchronize(st));
  return CG_OK;
}

CG_API int cg_rhs(cg_solver* s, const double* U, double* R, void* stream) {
  if (!s || !U || !R) return fail(CG_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = DISPATCH_ND(s, stage, s, U, U, R, 0, 1, st);
  if (rc) return rc;
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}

CG_API int cg_autotune(cg_solver* s, const double* U, int force, void* stream) {
  if (!s || !U) return fail(CG_ERR_INVALID_ARG, "null argument");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CG_CUDA(cudaStreamIsCapturing((cudaStream_t)stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return fail(CG_ERR_INVALID_ARG, "cg_autotune times kernels: not during capture");
  int rc = autotune_solver(s, U, force != 0, (cudaStream_t)stream);
  if (rc) return rc;
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}

CG_API int cg_tile_shape(const cg_solver* s, int lines_per_tile[3]) {
  if (!s || !lines_per_tile) return fail(CG_ERR_INVALID_ARG, "null argument");
  for (int d = 0; d < 3; ++d) lines_per_tile[d] = d < s->nd ? s->sweep_lw[d] : 0;
  return CG_OK;
}

CG_API int cg_set_tile_shape(cg_solver* s, const int lines_per_tile[3]) {
  if (!s || !lines_per_tile) return fail(CG_ERR_INVALID_ARG, "null argument");
  for (int d = 0; d < s->nd; ++d) {
    const int* cands = d == 0 ? kSweepLwCands0 : kSweepLwCands1;
    int nc = d == 0 ? (int)(sizeof kSweepLwCands0 / sizeof(int)) : (int)(sizeof kSweepLwCands1 / sizeof(int));
    bool ok = false;
    for (int k = 0; k < nc; ++k) ok = ok || cands[k] == lines_per_tile[d];
    if (!ok) return fail(CG_ERR_INVALID_ARG, "%d lines per tile is not a candidate along direction %d", lines_per_tile[d], d);
  }
  for (int d = 0; d < s->nd; ++d) s->sweep_lw[d] = lines_per_tile[d];
  return CG_OK;
}

CG_API int cg_rk3_step_dev(cg_solver* s, double* U, const double* dt_dev, void* stream) {
  if (!s || !U || !dt_dev) return fail(CG_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const double* keep = s->dt;
  s->dt = const_cast<double*>(dt_dev);
  int rc = DISPATCH_ND(s, rk3, s, U, st);
  s->dt = const_cast<double*>(keep);
  if (rc) return rc;
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}

static __global__ void k_convert_check(const double* d_in, float* f_out, const float* f_in, double* d_out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    f_out[i] = d2f_int(d_in[i]);
    d_out[i] = f2d_int(f_in[i]);
  }
}

CG_API int cg_convert_check(const double* d_in, float* f_out, const float* f_in, double* d_out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!d_in || !f_out || !f_in || !d_out))) return fail(CG_ERR_INVALID_ARG, "null argument");
  if (n == 0) return CG_OK;
  k_convert_check<<<grid_blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(d_in, f_out, f_in, d_out, (long long)n);
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}

CG_API int cg_step_dev(cg_solver* s, double* U, double* dt_dev, void* stream) {
  if (!s || !U || !dt_dev) return fail(CG_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  double* keep = s->dt;
  s->dt = dt_dev;
  int rc = DISPATCH_ND(s, rk3_cfl, s, U, dt_dev, nullptr, st);
  s->dt = keep;
  if (rc) return rc;
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}

CG_API int cg_step_graph(cg_solver* s, double* U, double* dt_dev, void* stream) {
  if (!s || !U || !dt_dev) return fail(CG_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (st == nullptr) return fail(CG_ERR_INVALID_ARG, "graph replay needs a non-default stream");
  if (s->timing) return cg_step_dev(s, U, dt_dev, stream);  // per-launch events: step eagerly
  if (!s->g_warm) {  // the first step runs eagerly: buffers a scheme allocates on first use exist before capture
    int rc = cg_step_dev(s, U, dt_dev, stream);
    if (rc) return rc;
    s->g_warm = true;
    return CG_OK;
  }
  bool same = s->gexec && s->g_U == U && s->g_dt == dt_dev;
  for (int d = 0; d < 3; ++d) same = same && s->g_lw[d] == s->sweep_lw[d];
  if (!same) {
    if (s->gexec) {
      cudaGraphExecDestroy(s->gexec);
      s->gexec = nullptr;
    }
    CG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    double* keep = s->dt;
    s->dt = dt_dev;
    int rc = DISPATCH_ND(s, rk3_cfl, s, U, dt_dev, nullptr, st);
    s->dt = keep;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fail(CG_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&s->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      s->gexec = nullptr;
      return fail(CG_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(e));
    }
    s->g_U = U;
    s->g_dt = dt_dev;
    for (int d = 0; d < 3; ++d) s->g_lw[d] = s->sweep_lw[d];
  }
  CG_CUDA(cudaGraphLaunch(s->gexec, st));
  return CG_OK;
}

CG_API int cg_rk3_step(cg_solver* s, double* U, double dt, void* stream) {
  if (!s || !U) return fail(CG_ERR_INVALID_ARG, "null argument");
  if (!(dt >= 0.0)) return fail(CG_ERR_INVALID_ARG, "dt must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  CG_CUDA(cudaMemcpyAsync(s->dt + 1, &dt, sizeof(double), cudaMemcpyHostToDevice, st));
  CG_CUDA(cudaStreamSynchronize(st));  // dt is pageable host memory
  return cg_rk3_step_dev(s, U, s->dt + 1, stream);
}

CG_API int cg_cfl_dt(cg_solver* s, const double* U, double* dt_out, int dt_on_device, void* stream) {
  if (!s || !U || !dt_out) return fail(CG_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  double* target = dt_on_device ? dt_out : s->dt;
  DISPATCH_ND(s, cfl_launch, s, U, target, nullptr, 0.0, st);
  CG_CUDA(cudaGetLastError());
  if (!dt_on_device) {
    CG_CUDA(cudaMemcpyAsync(dt_out, s->dt, sizeof(double), cudaMemcpyDeviceToHost, st));
    CG_CUDA(cudaStreamSynchronize(st));
  }
  return CG_OK;
}

CG_API int cg_sync_status(cg_solver* s, void* stream) {
  if (!s) return fail(CG_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned int flag = 0;
  unsigned long long idx = 0;
  CG_CUDA(cudaMemcpyAsync(&flag, s->bad_flag, sizeof flag, cudaMemcpyDeviceToHost, st));
  CG_CUDA(cudaMemcpyAsync(&idx, s->bad_idx, sizeof idx, cudaMemcpyDeviceToHost, st));
  CG_CUDA(cudaStreamSynchronize(st));
  if (flag) {
    s->last_bad = (long long)idx;
    CG_CUDA(cudaMemsetAsync(s->bad_flag, 0, sizeof(unsigned int), st));
    CG_CUDA(cudaMemsetAsync(s->bad_idx, 0xff, sizeof(unsigned long long), st));
    CG_CUDA(cudaStreamSynchronize(st));
    return fail(CG_ERR_NONPHYSICAL, "non-physical state (rho or p <= 0 or NaN) at node %lld", (long long)idx);
  }
  return CG_OK;
}

CG_API int64_t cg_last_bad_index(const cg_solver* s) { return s ? s->last_bad : -1; }
CG_API int64_t cg_launch_count(const cg_solver* s) { return s ? s->launches : 0; }

CG_API int cg_advance(cg_solver* s, double* U, int64_t nsteps, double t_end, double* t_out, int64_t* steps_out,
                      void* stream) {
  if (!s || !U) return fail(CG_ERR_INVALID_ARG, "null argument");
  if (nsteps <= 0 && !(t_end > 0.0)) return fail(CG_ERR_INVALID_ARG, "need nsteps > 0 or t_end > 0");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t k = 0;
  double t = 0.0;
  CG_CUDA(cudaMemsetAsync(s->t, 0, sizeof(double), st));
  while (nsteps <= 0 || k < nsteps) {
    if (t_end > 0.0) {
      // final time: the step size comes back to the host to clip the last step
      if (t >= t_end - 1e-14) break;
      DISPATCH_ND(s, cfl_launch, s, U, s->dt, nullptr, 0.0, st);
      double dt;
      CG_CUDA(cudaMemcpyAsync(&dt, s->dt, sizeof(double), cudaMemcpyDeviceToHost, st));
      CG_CUDA(cudaStreamSynchronize(st));
      if (t + dt > t_end) {
        dt = t_end - t;
        CG_CUDA(cudaMemcpyAsync(s->dt, &dt, sizeof(double), cudaMemcpyHostToDevice, st));
        CG_CUDA(cudaStreamSynchronize(st));
      }
      int rc = DISPATCH_ND(s, rk3, s, U, st);
      if (rc) return rc;
      t += dt;
    } else {
      int rc = DISPATCH_ND(s, rk3_cfl, s, U, s->dt, s->t, st);
      if (rc) return rc;
    }
    ++k;
  }
  if (!(t_end > 0.0)) {
    CG_CUDA(cudaMemcpyAsync(&t, s->t, sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CG_CUDA(cudaStreamSynchronize(st));
  if (t_out) *t_out = t;
  if (steps_out) *steps_out = k;
  return cg_sync_status(s, stream);
}

CG_API int cg_advance_host(cg_solver* s, double* U_host, int64_t nsteps, double t_end, double* t_out, void* stream) {
  if (!s || !U_host) return fail(CG_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  size_t bytes = sizeof(double) * s->nv * s->N;
  if (!s->host_stage) {
    size_t b0 = t_dalloc_bytes;
    if (dalloc(&s->host_stage, (size_t)s->nv * s->N)) return CG_ERR_OOM;
    s->dev_bytes += t_dalloc_bytes - b0;
  }
  CG_CUDA(cudaMemcpyAsync(s->host_stage, U_host, bytes, cudaMemcpyHostToDevice, st));
  int rc = cg_advance(s, s->host_stage, nsteps, t_end, t_out, nullptr, stream);
  CG_CUDA(cudaMemcpyAsync(U_host, s->host_stage, bytes, cudaMemcpyDeviceToHost, st));
  CG_CUDA(cudaStreamSynchronize(st));
  return rc;
}

CG_API int cg_omega(cg_solver* s, const double* U, double* omega, void* stream) {
  if (!s || !U || !omega) return fail(CG_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  bool compact = s->p.scheme == CG_MIG4;
  DISPATCH_ND(s, stage_prep_gbr, s, U, compact, st);
  // interior part of the sensor box
  Box ob = s->omBox;
  std::vector<double> box((size_t)ob.size()), in((size_t)s->N);
  if (s->p.precision == CG_MIXED) {  // the mixed form keeps the sensor in FP32
    std::vector<float> boxf(box.size());
    CG_CUDA(cudaMemcpyAsync(boxf.data(), s->om, boxf.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
    CG_CUDA(cudaStreamSynchronize(st));
    for (size_t i = 0; i < box.size(); ++i) box[i] = boxf[i];
  } else {
    CG_CUDA(cudaMemcpyAsync(box.data(), s->om, box.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CG_CUDA(cudaStreamSynchronize(st));
  }
  for (int k = 0; k < s->dg.n[2]; ++k)
    for (int j = 0; j < s->dg.n[1]; ++j)
      for (int i = 0; i < s->dg.n[0]; ++i)
        in[i + (size_t)s->dg.n[0] * (j + (size_t)s->dg.n[1] * k)] = box[(size_t)ob.at(i, j, k)];
  CG_CUDA(cudaMemcpyAsync(omega, in.data(), in.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  CG_CUDA(cudaStreamSynchronize(st));
  return CG_OK;
}

CG_API int cg_iface_flux(cg_solver* s, const double* U, int dir, double* F, void* stream) {
  if (!s || !U || !F) return fail(CG_ERR_INVALID_ARG, "null argument");
  if (dir < 0 || dir >= s->nd) return fail(CG_ERR_INVALID_ARG, "bad direction");
  int sch = s->p.scheme;
  if (sch != CG_MEG6 && sch != CG_MIG4 && !(sch == CG_HYBRID && s->p.hybrid_mode == CG_HYBRID_CELL))
    return fail(CG_ERR_UNSUPPORTED, "interface fluxes exist for the C-GBR and per-interface hybrid schemes");
  cudaStream_t st = (cudaStream_t)stream;
  if (!s->Rtmp) {
    size_t b0 = t_dalloc_bytes;
    if (dalloc(&s->Rtmp, (size_t)s->nv * s->N)) return CG_ERR_OOM;
    s->dev_bytes += t_dalloc_bytes - b0;
  }
  s->iface_dir = dir;
  s->iface_out = F;
  int rc = DISPATCH_ND(s, stage, s, U, U, s->Rtmp, 0, 1, st);
  s->iface_out = nullptr;
  if (rc) return rc;
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}

CG_API int cg_timing_enable(cg_solver* s, int on) {
  if (!s) return fail(CG_ERR_INVALID_ARG, "null argument");
  s->timing = on != 0;
  return CG_OK;
}

CG_API int cg_timing_query(cg_solver* s, int kernel_class, double* total_ms, int64_t* count) {
  if (!s || !total_ms || !count) return fail(CG_ERR_INVALID_ARG, "null argument");
  double tot = 0.0;
  int64_t n = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> keep;
  for (auto& o : s->ev_open) {
    if (o.first != kernel_class) { keep.push_back(o); continue; }
    CG_CUDA(cudaEventSynchronize(o.second.second));
    float ms = 0.0f;
    CG_CUDA(cudaEventElapsedTime(&ms, o.second.first, o.second.second));
    tot += ms;
    ++n;
    s->ev_pool.push_back(o.second.first);
    s->ev_pool.push_back(o.second.second);
  }
  s->ev_open.swap(keep);
  *total_ms = tot;
  *count = n;
  return CG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- no-allocation RHS
// Some callers must not allocate device memory: code that runs while a CUDA
// stream is being captured into a graph, plug-ins whose host application owns
// every device allocation through its own pool, and real-time loops that cannot
// afford the device-wide synchronisation a cudaMalloc/cudaFree may cause.
// cg_rhs_meg6_noalloc serves them: its working arrays (primitives, sensor,
// flux-difference accumulator) live in the fixed array below, which every GPU
// that loads this library holds until the process exits.
static constexpr long long kNoAllocDoubles = 1LL << 20;  // 8 MiB per device
static constexpr long long kNoAllocMaxCells = 1LL << 16;
static constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];
static std::mutex g_noalloc_mu;
static double* g_noalloc_addr[kNoAllocMaxDevices] = {};

extern "C" CG_API int cg_rhs_meg6_noalloc(int ndim, const int64_t n[3], const double h[3], const int bc[6],
                                          const cg_params* p, const double* U, double* R, void* stream) {
  if (!n || !h || !bc || !p || !U || !R) return fail(CG_ERR_INVALID_ARG, "null argument");
  int rc = check_grid_args(ndim, n, bc);
  if (rc) return rc;
  for (int d = 0; d < ndim; ++d)
    if (!(h[d] > 0.0)) return fail(CG_ERR_INVALID_ARG, "spacing must be positive");
  // grid descriptor on the stack (nothing allocated)
  cg_grid gr;
  gr.nd = ndim;
  gr.curv = 0;
  gr.xyz = nullptr;
  for (int d = 0; d < 3; ++d) {
    gr.n[d] = (int)n[d];
    gr.h[d] = d < ndim ? h[d] : 1.0;
    gr.bc[d][0] = d < ndim ? bc[2 * d] : CG_BC_PERIODIC;
    gr.bc[d][1] = d < ndim ? bc[2 * d + 1] : CG_BC_PERIODIC;
    for (int m = 0; m < 3; ++m) gr.period[d][m] = 0.0;
  }
  rc = check_params(&gr, p);
  if (rc) return rc;
  if (p->scheme != CG_MEG6) return fail(CG_ERR_UNSUPPORTED, "the no-allocation RHS evaluates the MEG6 scheme only");
  if (p->precision != CG_FP64) return fail(CG_ERR_UNSUPPORTED, "the no-allocation RHS supports CG_FP64 only");
  if (p->viscous)
    return fail(CG_ERR_UNSUPPORTED, "the no-allocation RHS is inviscid only (viscous needs the solver's scratch)");
  long long N = 1, box = 1;
  for (int d = 0; d < 3; ++d) {
    N *= n[d];
    box *= d < ndim ? n[d] + 8 : 1;
  }
  int nv = ndim + 2;
  long long need = 2LL * nv * N + box;
  if (N > kNoAllocMaxCells || need > kNoAllocDoubles)
    return fail(CG_ERR_INVALID_ARG,
                "grid too large for the no-allocation RHS: %lld cells need %lld scratch doubles; the limit is %lld "
                "cells and %lld doubles (use cg_solver_create / cg_rhs)",
                N, need, kNoAllocMaxCells, kNoAllocDoubles);
  // once per device, with that device current: device address of the array
  int dev = 0;
  CG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(CG_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
  double* base;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr)
        return fail(CG_ERR_CUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
      g_noalloc_addr[dev] = static_cast<double*>(ptr);
    }
    base = g_noalloc_addr[dev];
  }
  // solver descriptor on the stack; every scratch pointer is carved out of
  // the fixed array (W, accumulator, sensor), each written before read
  cg_solver s;
  s.grid = &gr;
  s.p = *p;
  s.nd = ndim;
  s.nv = nv;
  fill_devgrid(&gr, p, s.dg);
  s.N = s.dg.N;
  s.omBox = make_box(&s, 4, -1, 4);
  s.W = base;
  s.acc = base + (size_t)nv * N;
  s.om = base + (size_t)2 * nv * N;
  cudaStream_t st = (cudaStream_t)stream;
  rc = DISPATCH_ND((&s), stage, &s, U, U, R, 0, 1, st);
  if (rc) return rc;
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}
