// Batched tridiagonal line solves of the compact schemes and the implicit
// filter.  A parallel kernel builds every right-hand side into a line-major
// buffer ([component][row][line], lines contiguous, so a warp of 32 lines
// reads and writes 32 consecutive values); k_thomas_jobs then runs only the
// recurrence, one thread per (line, component), with the pivots precomputed
// on the host: dp_i = (r_i - a dp_{i-1}) rden_i, x_i = dp_i - cp_i x_{i+1}
// (cyclic lines add the Sherman-Morrison correction).  rden_i = 1/den_i is
// taken once on the host and every update is one fused multiply-add: on a
// GPU whose FP64 rate is the limit, a division per row would cost several
// times the rest of the row.  The result agrees with the plain elimination to
// a few units in the last place (the systems are diagonally dominant).
#pragma once
#include "cg_kernels.cuh"

namespace cgk {

// The source of a C6 line family whose right-hand sides the solver forms
// itself: nc planes of fs values of a node field on box fb, differenced along
// lb.  f = null: the right-hand sides are already in x.
template <typename T>
struct C6Src {
  const T* f = nullptr;
  Box fb{};
  long long fs = 0;
  LineBuf lb{};
};

// Up to three independent families of lines solved by one launch (e.g. the x
// and y lines of a stage): job j covers columns [start_j, start_j + nl_j * ncomp_j).
// T = double: the FP64 solves; T = float: the mixed form's FP32 gradient solves
// (coefficients mirrored in FP32).
template <typename T>
struct ThomasJobsT {
  LineCoefT<T> lc[3];
  C6Src<T> src[3];
  T* x[3];
  long long nl[3];
  int ncomp[3];
  long long start[4];
  int njobs;
};

template <typename T>
__device__ __forceinline__ void thomas_column(const LineCoefT<T>& lc, T* __restrict__ x, long long nl, long long t);
template <typename T>
__device__ __forceinline__ void thomas_column_c6(const LineCoefT<T>& lc, T* __restrict__ x, long long nl, long long t,
                                                 const C6Src<T>& sr);

// Thomas recurrence over every column (line x component) of x (in place).
template <typename T>
__global__ void k_thomas_jobs(ThomasJobsT<T> J) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int j = 0;
  while (j + 1 < J.njobs && t >= J.start[j + 1]) ++j;
  if (t >= J.start[J.njobs]) return;
  if (J.src[j].f) thomas_column_c6<T>(J.lc[j], J.x[j], J.nl[j], t - J.start[j], J.src[j]);
  else thomas_column<T>(J.lc[j], J.x[j], J.nl[j], t - J.start[j]);
}

// The recurrences below read row i+B..i+2B-1 (forward) or i-B..i-2B+1
// (backward) before they store rows i..i+B-1: loads of rows not yet written
// do not wait for the stores of the previous rows, so memory latency is paid
// once per batch of B rows instead of once per row.  The arithmetic of every
// row is the plain recurrence, in the same order.
constexpr int kRowBatch = 8;

// dp_i = (r_i - a dp_{i-1}) rden_i for i in [i0, i1), in place; returns dp_{i1-1}.
template <typename T>
__device__ __forceinline__ T thomas_forward(T* __restrict__ col, long long nl, const T* __restrict__ den,
                                            T a, int i0, int i1, T dp) {
  constexpr int B = kRowBatch;
  const int nfull = (i1 - i0) / B;
  T v[B], dn[B];
  if (nfull > 0) {
#pragma unroll
    for (int k = 0; k < B; ++k) {
      v[k] = col[(long long)(i0 + k) * nl];
      dn[k] = den[i0 + k];
    }
  }
  for (int b = 0; b < nfull; ++b) {
    const int base = i0 + b * B;
    const bool more = b + 1 < nfull;
    T nv[B], nd[B];
    if (more) {
#pragma unroll
      for (int k = 0; k < B; ++k) {
        nv[k] = col[(long long)(base + B + k) * nl];
        nd[k] = den[base + B + k];
      }
    }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      dp = fma_t(-a, dp, v[k]) * dn[k];
      col[(long long)(base + k) * nl] = dp;
    }
    if (more) {
#pragma unroll
      for (int k = 0; k < B; ++k) {
        v[k] = nv[k];
        dn[k] = nd[k];
      }
    }
  }
  for (int i = i0 + nfull * B; i < i1; ++i) {
    dp = fma_t(-a, dp, col[(long long)i * nl]) * den[i];
    col[(long long)i * nl] = dp;
  }
  return dp;
}

// x_i = dp_i - cp_i x_{i+1} for i = i1, i1-1, ..., i0, in place; returns x_{i0}.
template <typename T, int B = kRowBatch>
__device__ __forceinline__ T thomas_backward(T* __restrict__ col, long long nl, const T* __restrict__ cp,
                                             int i0, int i1, T xv) {
  const int nfull = (i1 - i0 + 1) / B;
  T v[B], c[B];
  if (nfull > 0) {
#pragma unroll
    for (int k = 0; k < B; ++k) {
      v[k] = col[(long long)(i1 - k) * nl];
      c[k] = cp[i1 - k];
    }
  }
  for (int b = 0; b < nfull; ++b) {
    const int top = i1 - b * B;
    const bool more = b + 1 < nfull;
    T nv[B], nc[B];
    if (more) {
#pragma unroll
      for (int k = 0; k < B; ++k) {
        nv[k] = col[(long long)(top - B - k) * nl];
        nc[k] = cp[top - B - k];
      }
    }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      xv = fma_t(-c[k], xv, v[k]);
      col[(long long)(top - k) * nl] = xv;
    }
    if (more) {
#pragma unroll
      for (int k = 0; k < B; ++k) {
        v[k] = nv[k];
        c[k] = nc[k];
      }
    }
  }
  for (int i = i1 - nfull * B; i >= i0; --i) {
    xv = fma_t(-cp[i], xv, col[(long long)i * nl]);
    col[(long long)i * nl] = xv;
  }
  return xv;
}

// x_i -= f z_i for i in [0, m), in place.
template <typename T>
__device__ __forceinline__ void thomas_correct(T* __restrict__ col, long long nl, const T* __restrict__ z,
                                               int m, T f) {
  constexpr int B = kRowBatch;
  int i = 0;
  for (; i + B <= m; i += B) {
    T v[B];
#pragma unroll
    for (int k = 0; k < B; ++k) v[k] = col[(long long)(i + k) * nl];
#pragma unroll
    for (int k = 0; k < B; ++k) col[(long long)(i + k) * nl] = fma_t(-f, z[i + k], v[k]);
  }
  for (; i < m; ++i) col[(long long)i * nl] = fma_t(-f, z[i], col[(long long)i * nl]);
}

template <typename T>
__device__ __forceinline__ void thomas_column(const LineCoefT<T>& lc, T* __restrict__ x, long long nl, long long t) {
  long long comp = t / nl, L = t % nl;
  T* col = x + comp * lc.m * nl + L;
  const T a = lc.a;
  const int m = lc.m;
  if (!lc.periodic) {
    // rows 0 and m-1 are identity rows (x = r there)
    thomas_forward(col, nl, lc.den, a, 1, m - 1, col[0]);
    thomas_backward(col, nl, lc.cp, 0, m - 2, col[(long long)(m - 1) * nl]);
  } else {
    T dp = col[0] * lc.den[0];
    col[0] = dp;
    const T xlast = thomas_forward(col, nl, lc.den, a, 1, m, dp);
    const T x0 = thomas_backward(col, nl, lc.cp, 0, m - 2, xlast);
    const T fact = (x0 + a * xlast / lc.gam) / lc.fden;
    thomas_correct(col, nl, lc.z, m, fact);
  }
}

// thomas_column of a C6 line family whose right-hand sides are formed on the
// way from the source field (c6_forward; the end rows of a non-periodic line
// take the E4 closure, as XTileC6 does).  Same recurrences and results.
template <typename T, int B>
__device__ __forceinline__ T c6_forward(T* __restrict__ col, long long nl, const T* __restrict__ aL, T a,
                                        const T* __restrict__ rd, int i0, int i1, T y, const T* __restrict__ fp,
                                        long long st, int lo, int m, bool periodic);

template <typename T>
__device__ __forceinline__ void thomas_column_c6(const LineCoefT<T>& lc, T* __restrict__ x, long long nl, long long t,
                                                 const C6Src<T>& sr) {
  const long long comp = t / nl, L = t % nl;
  T* col = x + comp * lc.m * nl + L;
  int cc[3] = {0, 0, 0};
  sr.lb.coords(L, cc);
  cc[sr.lb.d] = 0;
  const int d = sr.lb.d;
  const long long st = d == 0 ? 1 : (d == 1 ? (long long)sr.fb.ext[0] : (long long)sr.fb.ext[0] * sr.fb.ext[1]);
  const T* fp = sr.f + comp * sr.fs + sr.fb.at(cc[0], cc[1], cc[2]);
  auto F = [&](int pos) { return fp[(long long)pos * st]; };
  const T a = lc.a;
  const int m = lc.m, lo = sr.lb.lo;
  if (!lc.periodic) {
    // rows 0 and m-1 are identity rows holding the E4 closure values
    const T r0 = d4(F(lo - 2), F(lo - 1), F(lo + 1), F(lo + 2));
    col[0] = r0;
    c6_forward<T, 4>(col, nl, nullptr, a, lc.den, 1, m - 1, r0, fp, st, lo, m, false);
    const int pl = lo + m - 1;
    const T rl = d4(F(pl - 2), F(pl - 1), F(pl + 1), F(pl + 2));
    col[(long long)(m - 1) * nl] = rl;
    thomas_backward(col, nl, lc.cp, 0, m - 2, rl);
  } else {
    const T r0 = T(7.0 / 9.0) * (F(1) - F(-1)) + T(1.0 / 36.0) * (F(2) - F(-2));
    T dp = r0 * lc.den[0];
    col[0] = dp;
    const T xlast = c6_forward<T, 4>(col, nl, nullptr, a, lc.den, 1, m, dp, fp, st, 0, m, true);
    const T x0 = thomas_backward(col, nl, lc.cp, 0, m - 2, xlast);
    const T fact = (x0 + a * xlast / lc.gam) / lc.fden;
    thomas_correct(col, nl, lc.z, m, fact);
  }
}

// ---------------------------------------------------------------- partitioned solves
// For few columns (a 1D grid, few lines) one thread per column leaves the GPU
// idle: each column is split into P chunks of q rows solved concurrently.
// Chunk k solves its own block T_k (local pivots), giving y = T_k^{-1} r and,
// precomputed on the host, the responses V = T_k^{-1}(A_s e_s) and
// W = T_k^{-1}(C_{e-1} e_{e-1}) to the unknowns just outside it, so that
// x_i = y_i - V_i x_{s-1} - W_i x_e.  The 2P chunk-boundary unknowns then
// satisfy a block-bidiagonal recursion (host-computed factors rF, qF, beta),
// solved by one thread per column; a last pass applies the correction (and,
// for cyclic lines, the Sherman-Morrison term).  A block holds 32 columns
// (lanes, coalesced) times the chunks.
template <typename T>
struct PartCoefT {
  const T* aL;   // sub-diagonal of row i inside its chunk (0 at chunk starts)
  const T* cp;   // local elimination: super-diagonal / pivot (0 at chunk ends)
  const T* rd;   // reciprocal local pivots
  const T* V;    // response to the unknown before the chunk
  const T* W;    // response to the unknown after the chunk
  const T* z;    // cyclic: Sherman-Morrison vector, else null
  const T* ch;   // per chunk: rF, qF, beta, VF (= V at its first row), VL (= V at its last row)
  T a, gam, fden;
  int m, q, P, periodic;
};
using PartCoef = PartCoefT<double>;

template <typename T>
struct PartJobsT {
  PartCoefT<T> pc[3];
  C6Src<T> src[3];
  T* x[3];
  long long nl[3];
  int ncomp[3];
  long long start[4];  // first 32-column group of each job, in columns (multiples of 32)
  int njobs;
};

// Partitioned forward elimination inside one chunk: y_i = (r_i - aL_i y_{i-1})
// rd_i for i in [i0, i1), y_{i0-1} = 0 (aL is 0 at the chunk start), in place;
// returns y_{i1-1}.  Batched like thomas_forward (the column values only: the
// coefficients are shared by the block's columns and stay in cache).
template <typename T, int B>
__device__ __forceinline__ T part_forward(T* __restrict__ col, long long nl, const T* __restrict__ aL,
                                          const T* __restrict__ rd, int i0, int i1) {
  const int nfull = (i1 - i0) / B;
  T y = T(0);
  T v[B];
  if (nfull > 0) {
#pragma unroll
    for (int k = 0; k < B; ++k) v[k] = col[(long long)(i0 + k) * nl];
  }
  for (int b = 0; b < nfull; ++b) {
    const int base = i0 + b * B;
    const bool more = b + 1 < nfull;
    T nv[B];
    if (more) {
#pragma unroll
      for (int k = 0; k < B; ++k) nv[k] = col[(long long)(base + B + k) * nl];
    }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      y = fma_t(-aL[base + k], y, v[k]) * rd[base + k];
      col[(long long)(base + k) * nl] = y;
    }
    if (more) {
#pragma unroll
      for (int k = 0; k < B; ++k) v[k] = nv[k];
    }
  }
  for (int i = i0 + nfull * B; i < i1; ++i) {
    y = fma_t(-aL[i], y, col[(long long)i * nl]) * rd[i];
    col[(long long)i * nl] = y;
  }
  return y;
}

// The forward elimination (part_forward with sub-diagonal aL, or thomas_forward
// with the constant a when aL is null; y: the value before row i0) with the
// C6 right-hand side of each row formed on the way from
// the source field along the line (fp: the column's component at position 0,
// st: the stride between positions): r_i = 7/9 (f_{p+1} - f_{p-1}) +
// 1/36 (f_{p+2} - f_{p-2}), or the E4 closure d4 on the end rows of a
// non-periodic line, the expressions of k_rhs_c6 / XTileC6.  A window of the
// five positions around the row slides along; the values entering it are
// loaded B rows ahead.  The right-hand sides are never stored.
template <typename T, int B>
__device__ __forceinline__ T c6_forward(T* __restrict__ col, long long nl, const T* __restrict__ aL, T a,
                                        const T* __restrict__ rd, int i0, int i1, T y, const T* __restrict__ fp,
                                        long long st, int lo, int m, bool periodic) {
  const int p0 = periodic ? i0 : lo + i0;
  auto F = [&](int pos) { return fp[(long long)pos * st]; };
  T w0 = F(p0 - 2), w1 = F(p0 - 1), w2 = F(p0), w3 = F(p0 + 1), w4 = F(p0 + 2);
  T pre[B];
#pragma unroll
  for (int k = 0; k < B; ++k) pre[k] = (i0 + k + 1 < i1) ? F(p0 + 3 + k) : T(0);
  for (int base = i0; base < i1; base += B) {
    const int pb = p0 + (base - i0);
    T nxt[B];
#pragma unroll
    for (int k = 0; k < B; ++k) nxt[k] = (base + B + k + 1 < i1) ? F(pb + B + 3 + k) : T(0);
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int i = base + k;
      if (i < i1) {
        const bool closure = !periodic && (i == 0 || i == m - 1);
        const T r = closure ? d4(w0, w1, w3, w4) : T(7.0 / 9.0) * (w3 - w1) + T(1.0 / 36.0) * (w4 - w0);
        y = fma_t(-(aL ? aL[i] : a), y, r) * rd[i];
        col[(long long)i * nl] = y;
        w0 = w1;
        w1 = w2;
        w2 = w3;
        w3 = w4;
        w4 = pre[k];
      }
    }
#pragma unroll
    for (int k = 0; k < B; ++k) pre[k] = nxt[k];
  }
  return y;
}

// Partitioned update inside one chunk: x_i = y_i - V_i L_prev - W_i F_next
// (- f z_i on a cyclic line) for i in [i0, i1), in place, B rows per batch.
template <typename T, int B>
__device__ __forceinline__ void part_update(T* __restrict__ col, long long nl, const PartCoefT<T>& pc, int i0,
                                            int i1, T Lp, T Fn, T f) {
  int i = i0;
  for (; i + B <= i1; i += B) {
    T v[B];
#pragma unroll
    for (int k = 0; k < B; ++k) v[k] = col[(long long)(i + k) * nl];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      T x = fma_t(-pc.V[i + k], Lp, v[k]);
      x = fma_t(-pc.W[i + k], Fn, x);
      if (pc.periodic) x = fma_t(-f, pc.z[i + k], x);
      col[(long long)(i + k) * nl] = x;
    }
  }
  for (; i < i1; ++i) {
    T x = fma_t(-pc.V[i], Lp, col[(long long)i * nl]);
    x = fma_t(-pc.W[i], Fn, x);
    if (pc.periodic) x = fma_t(-f, pc.z[i], x);
    col[(long long)i * nl] = x;
  }
}

constexpr int kPartMax = 32;

template <typename T>
__global__ void __launch_bounds__(1024) k_tri_part(PartJobsT<T> J) {
  __shared__ T sYF[kPartMax][32], sYL[kPartMax][32], sF[kPartMax][32], sL[kPartMax][32];
  __shared__ T sFact[32];
  // rows per batch: up to 1024 threads leave 64 registers a thread
  constexpr int PB = 4;
  const int lane = threadIdx.x, k = threadIdx.y;
  const long long g0 = (long long)blockIdx.x * 32;
  int j = 0;
  while (j + 1 < J.njobs && g0 >= J.start[j + 1]) ++j;
  const PartCoefT<T>& pc = J.pc[j];
  const long long nl = J.nl[j];
  const long long c = g0 - J.start[j] + lane;
  const bool active = c < nl * J.ncomp[j];
  T* col = J.x[j] + (active ? (c / nl) * pc.m * nl + c % nl : 0);
  const int s = k * pc.q, e = min(pc.m, s + pc.q);
  const bool mine = active && k < pc.P && s < e;
  if (mine) {
    const C6Src<T>& sr = J.src[j];
    T y;
    if (sr.f) {  // form the C6 right-hand sides on the way
      int cc[3] = {0, 0, 0};
      sr.lb.coords(c % nl, cc);
      cc[sr.lb.d] = 0;
      const int d = sr.lb.d;
      const long long st = d == 0 ? 1 : (d == 1 ? (long long)sr.fb.ext[0] : (long long)sr.fb.ext[0] * sr.fb.ext[1]);
      const T* fp = sr.f + (c / nl) * sr.fs + sr.fb.at(cc[0], cc[1], cc[2]);
      y = c6_forward<T, PB>(col, nl, pc.aL, T(0), pc.rd, s, e, T(0), fp, st, sr.lb.lo, pc.m, pc.periodic != 0);
    } else {
      y = part_forward<T, PB>(col, nl, pc.aL, pc.rd, s, e);
    }
    sYL[k][lane] = y;
    y = thomas_backward<T, PB>(col, nl, pc.cp, s, e - 2, y);
    sYF[k][lane] = y;
  }
  __syncthreads();
  if (k == 0 && active) {
    // forward: F_k = pF_k + qF_k F_{k+1},  L_k = alpha_k + beta_k F_{k+1}
    T alpha = T(0), beta_prev = T(0);
    for (int kk = 0; kk < pc.P; ++kk) {
      const T* h = pc.ch + 5 * kk;
      T pF = fma_t(-h[3], alpha, sYF[kk][lane]) * h[0];
      alpha = fma_t(-h[4], fma_t(beta_prev, pF, alpha), sYL[kk][lane]);
      sF[kk][lane] = pF;
      sL[kk][lane] = alpha;
      beta_prev = h[2];
    }
    T Fn = T(0);
    for (int kk = pc.P - 1; kk >= 0; --kk) {
      const T* h = pc.ch + 5 * kk;
      T F = fma_t(h[1], Fn, sF[kk][lane]);
      T L = fma_t(h[2], Fn, sL[kk][lane]);
      sF[kk][lane] = F;
      sL[kk][lane] = L;
      Fn = F;
    }
    if (pc.periodic) sFact[lane] = (sF[0][lane] + pc.a * sL[pc.P - 1][lane] / pc.gam) / pc.fden;
  }
  __syncthreads();
  if (mine) {
    const T Lp = k > 0 ? sL[k - 1][lane] : T(0);
    const T Fn = k + 1 < pc.P ? sF[k + 1][lane] : T(0);
    const T f = pc.periodic ? sFact[lane] : T(0);
    part_update<T, PB>(col, nl, pc, s, e, Lp, Fn, f);
  }
}

#define LB_LOOP(lb, e) \
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)(lb).m * (lb).nl; \
       e += (long long)gridDim.x * blockDim.x)

// MIG4 right-hand sides of the primitives along lb.d: 3/4 (W_{i+1} - W_{i-1}),
// E4 closure rows at both ends of a non-periodic line.
template <int ND, typename TW = double, typename TR = double>
__global__ void k_rhs_mig4(DevGrid g, const TW* __restrict__ W, LineBuf lb, TR* __restrict__ r) {
  constexpr int NV = ND + 2;
  LB_LOOP(lb, e) {
    int i = (int)(e / lb.nl);
    long long L = e % lb.nl;
    int c[3] = {0, 0, 0};
    lb.coords(L, c);
    int pos = lb.periodic ? i : lb.lo + i;
    bool closure = !lb.periodic && (i == 0 || i == lb.m - 1);
    TR wp1[NV], wm1[NV];
    int cc[3] = {c[0], c[1], c[2]};
    cc[lb.d] = pos + 1; load_state<ND, false, TW, TR>(g, W, cc[0], cc[1], cc[2], wp1);
    cc[lb.d] = pos - 1; load_state<ND, false, TW, TR>(g, W, cc[0], cc[1], cc[2], wm1);
    if (closure) {
      TR wp2[NV], wm2[NV];
      cc[lb.d] = pos + 2; load_state<ND, false, TW, TR>(g, W, cc[0], cc[1], cc[2], wp2);
      cc[lb.d] = pos - 2; load_state<ND, false, TW, TR>(g, W, cc[0], cc[1], cc[2], wm2);
#pragma unroll
      for (int v = 0; v < NV; ++v) r[((long long)v * lb.m + i) * lb.nl + L] = d4(wm2[v], wm1[v], wp1[v], wp2[v]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) r[((long long)v * lb.m + i) * lb.nl + L] = TR(0.75) * (wp1[v] - wm1[v]);
    }
  }
}

// C6 right-hand sides of nc components of a field held on box fb (values at
// positions up to two past the rows): 7/9 (f_{i+1} - f_{i-1}) + 1/36 (f_{i+2} - f_{i-2}),
// E4 closure rows at both ends of a non-periodic line.  Periodic rows read the
// field at wrapped positions through the box (fb covers the wrap).
template <typename T = double>
__global__ void k_rhs_c6(const T* __restrict__ f, Box fb, int nc, LineBuf lb, T* __restrict__ r) {
  long long fs = fb.size();
  long long st = lb.d == 0 ? 1 : (lb.d == 1 ? (long long)fb.ext[0] : (long long)fb.ext[0] * fb.ext[1]);
  LB_LOOP(lb, e) {
    int i = (int)(e / lb.nl);
    long long L = e % lb.nl;
    int c[3] = {0, 0, 0};
    lb.coords(L, c);
    c[lb.d] = lb.periodic ? i : lb.lo + i;
    long long q = fb.at(c[0], c[1], c[2]);
    bool closure = !lb.periodic && (i == 0 || i == lb.m - 1);
    for (int v = 0; v < nc; ++v) {
      const T* p = f + v * fs + q;
      T rv = closure ? d4(p[-2 * st], p[-st], p[st], p[2 * st])
                     : T(7.0 / 9.0) * (p[st] - p[-st]) + T(1.0 / 36.0) * (p[2 * st] - p[-2 * st]);
      r[((long long)v * lb.m + i) * lb.nl + L] = rv;
    }
  }
}

// The filtered quantity at a (possibly ghost) node: the conserved state, or,
// on a curvilinear grid, the transformed conserved state Q/J that the
// discrete conservation law advances (J from the padded metric planes).
template <int ND>
__device__ __forceinline__ void load_filtered(const DevGrid& g, const double* __restrict__ U, const int* c,
                                              double* w) {
  load_state<ND, true>(g, U, c[0], c[1], c[2], w);
  if (g.curv) {
    const double J = g.jac[plin(g, c[0], c[1], c[2])];
#pragma unroll
    for (int v = 0; v < ND + 2; ++v) w[v] = w[v] / J;
  }
}

// Implicit-filter right-hand sides of the conserved state along lb.d:
// non-periodic rows 0 and m-1 hold the ghost values at -1 and n; rows 1..n
// hold sum_{m=0}^{4} (a_m/2)(f_{i+m} + f_{i-m}) of positions 0..n-1.
template <int ND>
__global__ void k_rhs_filter(DevGrid g, const double* __restrict__ U, LineBuf lb, double b0, double b1, double b2,
                             double b3, double b4, double* __restrict__ r) {
  constexpr int NV = ND + 2;
  LB_LOOP(lb, e) {
    int i = (int)(e / lb.nl);
    long long L = e % lb.nl;
    int c[3] = {0, 0, 0};
    lb.coords(L, c);
    int pos = lb.periodic ? i : lb.lo + i;
    bool closure = !lb.periodic && (i == 0 || i == lb.m - 1);
    double w[9][NV];
    int cc[3] = {c[0], c[1], c[2]};
    if (closure) {
      cc[lb.d] = pos;
      load_filtered<ND>(g, U, cc, w[4]);
#pragma unroll
      for (int v = 0; v < NV; ++v) r[((long long)v * lb.m + i) * lb.nl + L] = w[4][v];
      continue;
    }
#pragma unroll
    for (int t = -4; t <= 4; ++t) {
      cc[lb.d] = pos + t;
      load_filtered<ND>(g, U, cc, w[t + 4]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
      r[((long long)v * lb.m + i) * lb.nl + L] = b0 * w[4][v] + b1 * (w[5][v] + w[3][v]) + b2 * (w[6][v] + w[2][v]) +
                                                 b3 * (w[7][v] + w[1][v]) + b4 * (w[8][v] + w[0][v]);
  }
}

// ---------------------------------------------------------------- staged right-hand sides
// The kernels above load every stencil point of every row from memory, and
// along x (d = 0) consecutive threads take consecutive lines, i.e. grid rows
// nx apart, so that each load touches its own 32-byte sector.  k_rhs_tile
// stages a tile of XT_L lines x XT_R rows through shared memory instead: the
// stencil window of each line (the tile's rows plus the reach of their
// stencils) is read once, coalesced (along x for x lines, across the lines,
// which run along x, otherwise), and the right-hand sides are written
// line-fastest, coalesced in the line buffer.  Each Tile type supplies the
// loads (ghosts resolved as in the kernels above) and the row formula, the
// same expression as its per-row kernel.
constexpr int XT_L = 16, XT_R = 32, XT_THREADS = 256;

// H: reach of the interior rows' stencil, Tile::HC: reach of the closure rows.
// TS: the staged type (the right-hand side's type T unless the tile stages
// something else, e.g. the hi/lo pairs of the mixed filter).
template <typename T, int NC, int H, class Tile, typename TS = T>
__global__ void __launch_bounds__(XT_THREADS) k_rhs_tile(LineBuf lb, Tile tl, T* __restrict__ r) {
  constexpr int HM = H > Tile::HC ? H : Tile::HC;
  constexpr int W = XT_R + 2 * HM + 1;  // +1: spreads lines over banks
  __shared__ TS sw[NC][XT_L][W];
  const long long L0 = (long long)blockIdx.x * XT_L;
  const int i0 = blockIdx.y * XT_R;
  const int i1 = min(lb.m, i0 + XT_R);
  const int nlin = (int)min((long long)XT_L, lb.nl - L0);
  // window of positions the tile's rows read
  int ws = 0x7fffffff, we = -0x7fffffff;
  for (int i = i0; i < i1; ++i) {
    const bool closure = !lb.periodic && (i == 0 || i == lb.m - 1);
    const int pos = lb.periodic ? i : lb.lo + i;
    const int h = closure ? Tile::HC : H;
    ws = min(ws, pos - h);
    we = max(we, pos + h);
  }
  const int wn = we - ws + 1;
  const bool along = lb.d == 0;  // window positions contiguous in memory
  for (int e = threadIdx.x; e < nlin * wn; e += XT_THREADS) {
    const int l = along ? e / wn : e % nlin;
    const int p = along ? e - l * wn : e / nlin;
    int c[3] = {0, 0, 0};
    lb.coords(L0 + l, c);
    c[lb.d] = ws + p;
    TS w[NC];
    tl.load(c, w);
#pragma unroll
    for (int v = 0; v < NC; ++v) sw[v][l][p] = w[v];
  }
  __syncthreads();
  const int l = threadIdx.x % XT_L;
  if (l >= nlin) return;
  for (int i = i0 + threadIdx.x / XT_L; i < i1; i += XT_THREADS / XT_L) {
    const bool closure = !lb.periodic && (i == 0 || i == lb.m - 1);
    const int p = (lb.periodic ? i : lb.lo + i) - ws;
#pragma unroll
    for (int v = 0; v < NC; ++v)
      if (v < tl.nc) r[((long long)v * lb.m + i) * lb.nl + L0 + l] = tl.row(&sw[v][l][0], p, closure);
  }
}

// Implicit filter of the conserved state (the formula of k_rhs_filter).
template <int ND>
struct XTileFilter {
  DevGrid g;
  const double* U;
  double b0, b1, b2, b3, b4;
  int nc;
  static constexpr int HC = 0;
  __device__ void load(const int* c, double* w) const { load_filtered<ND>(g, U, c, w); }
  __device__ double row(const double* w, int p, bool closure) const {
    if (closure) return w[p];
    return b0 * w[p] + b1 * (w[p + 1] + w[p - 1]) + b2 * (w[p + 2] + w[p - 2]) + b3 * (w[p + 3] + w[p - 3]) +
           b4 * (w[p + 4] + w[p - 4]);
  }
};

// ---------------------------------------------------------------- mixed filter
// The mixed form's implicit filter in increment form: D = Qf - Q solves
// alpha D_{i-1} + D_i + alpha D_{i+1} = sum_n c_n (Q_{i+n} + Q_{i-n} - 2 Q_i),
// n = 1..4, with c_1 = b_1 - alpha and c_n = b_n otherwise (the filter's row
// minus its left-hand side applied to Q; the b_n keep constants, so the
// right-hand side is a sum of second differences), and D = 0 on the identity
// rows of non-periodic lines.  Each FP64 value is split once into a float
// pair hi + lo (hi its FP32 image, lo the FP32 image of the rest); the second
// differences are formed from the pairs in FP32, hi differences first (exact
// between values within a factor two, so a smooth field keeps the relative
// precision of the difference itself), and the line systems are solved in
// FP32.  The state update Q + D is FP64 (k_filter_store_inc).
__device__ __forceinline__ float2 split_hilo(double x) {
  const float hi = d2f_int(x);
  return make_float2(hi, d2f_int(x - f2d_int(hi)));
}

// The filtered variable of the mixed filter: Q, or Q/J on a curvilinear grid
// formed as Q times the refined reciprocal of J (relative error below 2e-14,
// far under the hi/lo pair's 48 bits) instead of five IEEE FP64 divisions.
template <int ND>
__device__ __forceinline__ void load_filtered_mixed(const DevGrid& g, const double* __restrict__ U, const int* c,
                                                    double* w) {
  load_state<ND, true>(g, U, c[0], c[1], c[2], w);
  if (g.curv) {
    const double r = recip_refined(g.jac[plin(g, c[0], c[1], c[2])]);
#pragma unroll
    for (int v = 0; v < ND + 2; ++v) w[v] = w[v] * r;
  }
}

struct FilterInc {
  float c1, c2, c3, c4;
  // w: the pairs at offsets -4..4 of the row's position, w[4] the centre
  __device__ __forceinline__ float row(const float2* w) const {
    const float2 o = w[4];
    auto d2 = [&](int k) {
      const float2 a = w[4 + k], b = w[4 - k];
      return ((a.x - o.x) + (b.x - o.x)) + ((a.y + b.y) - 2.0f * o.y);
    };
    return c1 * d2(1) + c2 * d2(2) + c3 * d2(3) + c4 * d2(4);
  }
};

template <int ND>
struct XTileFilterInc {
  DevGrid g;
  const double* U;
  FilterInc fc;
  int nc;
  static constexpr int HC = 0;
  __device__ void load(const int* c, float2* w) const {
    double q[ND + 2];
    load_filtered_mixed<ND>(g, U, c, q);
#pragma unroll
    for (int v = 0; v < ND + 2; ++v) w[v] = split_hilo(q[v]);
  }
  __device__ float row(const float2* w, int p, bool closure) const { return closure ? 0.0f : fc.row(w + p - 4); }
};

// Per-row form of the same right-hand sides (line families of fewer lines than a tile).
template <int ND>
__global__ void k_rhs_filter_inc(DevGrid g, const double* __restrict__ U, LineBuf lb, FilterInc fc,
                                 float* __restrict__ r) {
  constexpr int NV = ND + 2;
  LB_LOOP(lb, e) {
    int i = (int)(e / lb.nl);
    long long L = e % lb.nl;
    int c[3] = {0, 0, 0};
    lb.coords(L, c);
    int pos = lb.periodic ? i : lb.lo + i;
    if (!lb.periodic && (i == 0 || i == lb.m - 1)) {
#pragma unroll
      for (int v = 0; v < NV; ++v) r[((long long)v * lb.m + i) * lb.nl + L] = 0.0f;
      continue;
    }
    float2 w[NV][9];
    int cc[3] = {c[0], c[1], c[2]};
#pragma unroll
    for (int t = -4; t <= 4; ++t) {
      cc[lb.d] = pos + t;
      double q[NV];
      load_filtered_mixed<ND>(g, U, cc, q);
#pragma unroll
      for (int v = 0; v < NV; ++v) w[v][t + 4] = split_hilo(q[v]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) r[((long long)v * lb.m + i) * lb.nl + L] = fc.row(w[v]);
  }
}

// MIG4 gradients of the primitives (the formula of k_rhs_mig4).
template <int ND, typename TW, typename TR>
struct XTileMig4 {
  DevGrid g;
  const TW* W;
  int nc;
  static constexpr int HC = 2;
  __device__ void load(const int* c, TR* w) const { load_state<ND, false, TW, TR>(g, W, c[0], c[1], c[2], w); }
  __device__ TR row(const TR* w, int p, bool closure) const {
    if (closure) return d4(w[p - 2], w[p - 1], w[p + 1], w[p + 2]);
    return TR(0.75) * (w[p + 1] - w[p - 1]);
  }
};

// C6 derivatives of nc components held on a box (the formula of k_rhs_c6).
template <typename T, int NC>
struct XTileC6 {
  const T* f;
  Box fb;
  long long fs;
  int nc;
  static constexpr int HC = 2;
  __device__ void load(const int* c, T* w) const {
    const long long q = fb.at(c[0], c[1], c[2]);
#pragma unroll
    for (int v = 0; v < NC; ++v) w[v] = v < nc ? f[v * fs + q] : T(0);
  }
  __device__ T row(const T* w, int p, bool closure) const {
    if (closure) return d4(w[p - 2], w[p - 1], w[p + 1], w[p + 2]);
    return T(7.0 / 9.0) * (w[p + 1] - w[p - 1]) + T(1.0 / 36.0) * (w[p + 2] - w[p - 2]);
  }
};

// The staged form when a tile's lines are all there to share it.
__host__ __forceinline__ bool use_tile(const LineBuf& lb) { return lb.nl >= XT_L; }

__host__ __forceinline__ dim3 tile_grid(const LineBuf& lb) {
  return dim3((unsigned)((lb.nl + XT_L - 1) / XT_L), (unsigned)((lb.m + XT_R - 1) / XT_R));
}

// Filtered line values back into the interior of the state.
template <int ND>
__global__ void k_filter_store(DevGrid g, const double* __restrict__ x, LineBuf lb, double* __restrict__ U) {
  constexpr int NV = ND + 2;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.N; q += (long long)gridDim.x * blockDim.x) {
    int c[3];
    node_coords(g, q, c);
    const double J = g.curv ? g.jac[plin(g, c[0], c[1], c[2])] : 1.0;
#pragma unroll
    for (int v = 0; v < NV; ++v) U[v * g.N + q] = g.curv ? x[lb.at(v, c[lb.d], c)] * J : x[lb.at(v, c[lb.d], c)];
  }
}

// The mixed filter's increments into the interior of the state:
// Q += D (Q/J += D on a curvilinear grid: Q += J D), the sum in FP64.
template <int ND>
__global__ void k_filter_store_inc(DevGrid g, const float* __restrict__ x, LineBuf lb, double* __restrict__ U) {
  constexpr int NV = ND + 2;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.N; q += (long long)gridDim.x * blockDim.x) {
    int c[3];
    node_coords(g, q, c);
    const float J = g.curv ? d2f_int(g.jac[plin(g, c[0], c[1], c[2])]) : 1.0f;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float d = x[lb.at(v, c[lb.d], c)];
      U[v * g.N + q] = U[v * g.N + q] + f2d_int(g.curv ? J * d : d);
    }
  }
}

// k_filter_store_inc for lines along x on tiles of 32 positions x 8 lines:
// the tile's increments are staged with consecutive threads on consecutive
// lines (the x-line buffer keeps a line's positions a line count apart),
// then each thread updates one node.
constexpr int FST_X = 32, FST_Y = 8;
template <int ND>
__global__ void __launch_bounds__(FST_X * FST_Y) k_filter_store_inc_xt(DevGrid g, const float* __restrict__ x,
                                                                       LineBuf lb, double* __restrict__ U) {
  constexpr int NV = ND + 2;
  __shared__ float sD[NV][FST_Y][FST_X + 1];
  const int x0 = (int)blockIdx.x * FST_X;
  const long long L0 = (long long)blockIdx.y * FST_Y + (long long)blockIdx.z * gridDim.y * FST_Y;
  const int tid = threadIdx.y * FST_X + threadIdx.x;
  {
    const int ly = tid % FST_Y, lx = tid / FST_Y;
    if (x0 + lx < g.n[0] && L0 + ly < lb.nl) {
      int c[3] = {0, 0, 0};
      lb.coords(L0 + ly, c);
#pragma unroll
      for (int v = 0; v < NV; ++v) sD[v][ly][lx] = x[lb.at(v, x0 + lx, c)];
    }
  }
  __syncthreads();
  const int xi = x0 + (int)threadIdx.x;
  const long long L = L0 + threadIdx.y;
  if (xi >= g.n[0] || L >= lb.nl) return;
  int c[3] = {0, 0, 0};
  lb.coords(L, c);
  c[0] = xi;
  const long long q = lin(g, c[0], c[1], c[2]);
  const float J = g.curv ? d2f_int(g.jac[plin(g, c[0], c[1], c[2])]) : 1.0f;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float d = sD[v][threadIdx.y][threadIdx.x];
    U[v * g.N + q] = U[v * g.N + q] + f2d_int(g.curv ? J * d : d);
  }
}

}  // namespace cgk
