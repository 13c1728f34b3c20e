// Device building blocks of the FP64 RHS (parity form).
//
// Every floating-point expression here is written in the same operation order
// as the method's definition it implements (the paper's equations and the
// published methods it cites), and this translation unit is compiled with
// -fmad=false, so each a*b+c rounds twice: results are reproducible on any
// IEEE FP64 machine.  Zero metric components of Cartesian grids are dropped
// at compile time (x + 0*y == x for the finite values that occur here; only
// the sign of an exact zero can differ, and no sign-sensitive operation
// consumes one).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cgk {

constexpr int BC_PERIODIC = 0, BC_EXTRAP = 1, BC_REFLECT = 2, BC_INFLOW = 3, BC_WALL = 4;
constexpr int PM = 8;  // ghost layers stored with curvilinear metric planes

// Grid as seen by the kernels (passed by value).
struct DevGrid {
  int nd, nv;
  int n[3];
  long long N;
  int bc[3][2];
  double inflowW[3][2][5];  // primitive state held on inflow faces
  double inflowQ[3][2][5];  // the same state in conserved variables
  double gamma, gm1, gm2;   // gamma, gamma-1, gamma*minf^2
  int curv;
  // Cartesian constants
  double cxh[3];    // node metric xi_hat[l][l]
  double cjac;      // J
  double cjxh[3];   // J xi_hat[l][l] (the product, as the sensor forms it)
  double ch[3];     // spacing (LAD displacement |Delta x_l|)
  // per-direction interface frame of a Cartesian grid (computed on the host
  // with the same operations as the per-interface frame of a curvilinear one)
  double cg2[3], cg[3], cig[3], cig2[3];
  double cn[3][3], ct1[3][3], ct2[3][3];
  // curvilinear metrics: planes on the box padded by PM in active directions
  int P[3];
  long long NP;
  const double* xh;   // nd*nd planes, xi_hat[l][m]
  const double* xt;   // nd*nd planes, interface metrics of l-interface i+1/2 at node i
  const double* jac;  // J
  const double* dxl;  // nd*nd planes, LAD displacement vectors
  // isothermal no-slip walls and physical viscosity (Sutherland)
  double twall;       // wall temperature (units of T_inf)
  int visc;           // physical viscous terms on
  double re, suth, kc;  // Re, S / T_inf, (gamma-1) Pr minf^2
  // per-node inflow profiles (primitive, nv planes over the face), or null
  const double* prof[3][2];
  long long pf[3];    // nodes of a face normal to d
  // FP32 copies of the constants the mixed form's kernels use, rounded once on
  // the host: a conversion in the kernel would run on the FP64 pipe
  float f_gamma, f_gm1, f_gm2;
  float f_cxh[3], f_cjac, f_ch[3], f_cjxh[3];
  float f_cg2[3], f_cg[3], f_cig2[3];
  float f_cn[3][3], f_ct1[3][3], f_ct2[3][3];
};

// A grid constant in the arithmetic type T: the FP64 value, or its FP32 copy
// (the same float the conversion would give).
template <typename T>
__device__ __forceinline__ T gconst(double d, float f) {
  if constexpr (sizeof(T) == 4) return f;
  else return d;
}

// Node coordinates of the linear index q (32-bit division when the grid has
// fewer than 2^31 nodes: a 64-bit division by a variable costs several times more).
__device__ __forceinline__ void node_coords(const DevGrid& g, long long q, int* c) {
  if (g.N <= 0x7fffffffLL) {
    const unsigned r = (unsigned)q, n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
    const unsigned t = r / n0;
    c[0] = (int)(r - t * n0);
    c[1] = (int)(t % n1);
    c[2] = (int)(t / n1);
  } else {
    c[0] = (int)(q % g.n[0]);
    c[1] = (int)((q / g.n[0]) % g.n[1]);
    c[2] = (int)(q / ((long long)g.n[0] * g.n[1]));
  }
}

__device__ __forceinline__ long long lin(const DevGrid& g, int i, int j, int k) {
  return (long long)i + (long long)g.n[0] * ((long long)j + (long long)g.n[1] * (long long)k);
}
__device__ __forceinline__ long long plin(const DevGrid& g, int i, int j, int k) {
  int gi = i + (g.nd > 0 ? PM : 0), gj = j + (g.nd > 1 ? PM : 0), gk = k + (g.nd > 2 ? PM : 0);
  return (long long)gi + (long long)g.P[0] * ((long long)gj + (long long)g.P[1] * (long long)gk);
}

// Boundary resolution of a possibly-ghost node.  Ghost values are defined as
// if the ghost layers were filled direction by direction (x, then y over the
// x-extended range, then z), so the outermost direction is resolved first.
struct Src {
  long long idx;  // interior linear index (valid when face < 0)
  int flip;       // bit d set: negate velocity component d
  int face;       // >= 0: inflow face 2*d + side (state held fixed)
  long long pidx; // >= 0: node of the face's inflow profile
  int walls;      // isothermal-wall images applied (one per wall crossed)
};

__device__ __forceinline__ Src resolve(const DevGrid& g, int c0, int c1, int c2) {
  int c[3] = {c0, c1, c2};
  Src s;
  s.flip = 0;
  s.face = -1;
  s.pidx = -1;
  s.walls = 0;
#pragma unroll
  for (int d = 2; d >= 0; --d) {
    if (d >= g.nd) continue;
    int n = g.n[d];
    int x = c[d];
    if (x >= 0 && x < n) continue;
    int side = x < 0 ? 0 : 1;
    int bc = g.bc[d][side];
    if (bc == BC_INFLOW) {
      s.face = 2 * d + side;
      s.idx = 0;
      if (g.prof[d][side]) {
        // transverse position on the face, clamped to it (directions not yet
        // resolved may still point at ghosts)
        long long pi = 0, mul = 1;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          if (e >= g.nd || e == d) continue;
          int y = c[e] < 0 ? 0 : (c[e] >= g.n[e] ? g.n[e] - 1 : c[e]);
          pi += (long long)y * mul;
          mul *= g.n[e];
        }
        s.pidx = pi;
      }
      return s;
    } else if (bc == BC_PERIODIC) {
      x %= n;
      if (x < 0) x += n;
    } else if (bc == BC_REFLECT) {
      x = side == 0 ? -x - 1 : 2 * n - 1 - x;
      s.flip ^= (1 << d);
    } else if (bc == BC_WALL) {
      x = side == 0 ? -x - 1 : 2 * n - 1 - x;
      s.walls++;
    } else {
      x = side == 0 ? 0 : n - 1;
    }
    // positions deeper than one mirror image never feed a used value; keep them in range
    x = x < 0 ? 0 : (x >= n ? n - 1 : x);
    c[d] = x;
  }
  s.idx = lin(g, c[0], c[1], c[2]);
  return s;
}

// Primitive state (or conserved: cons = true) at a possibly-ghost node from
// nv planes F of N values.
template <int ND>
__device__ __forceinline__ void prim_to_cons(const DevGrid& g, const double* W, double* Q) {
  double q = 0.0;
  Q[0] = W[0];
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    Q[1 + k] = W[0] * W[1 + k];
    q = q + W[1 + k] * W[1 + k];
  }
  Q[ND + 1] = W[ND + 1] / g.gm1 + 0.5 * W[0] * q;
}

template <int ND>
__device__ __forceinline__ void cons_to_prim_g(const DevGrid& g, const double* Q, double* W) {
  double rho = Q[0];
  double irho = 1.0 / rho;
  double ke = 0.0;
  W[0] = rho;
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    W[1 + k] = Q[1 + k] * irho;
    ke = ke + Q[1 + k] * W[1 + k];
  }
  W[ND + 1] = g.gm1 * (Q[ND + 1] - 0.5 * ke);
}

// ---------------------------------------------------------------- binary64 <-> binary32
// Format conversions on the integer pipes.  On this part a hardware conversion
// between FP64 and FP32 issues on the FP64 pipe, which runs at 2 instructions
// per clock per SM against 64 for the integer pipes, so the mixed form's
// FP64-bound kernels (recovery, RK update) convert with integer operations.
// Both follow the IEEE 754 interchange formats (binary64: 1 sign, 11 exponent
// bits with bias 1023, 52 fraction bits; binary32: 1, 8 with bias 127, 23)
// and round to nearest, ties to even, so they return exactly what the
// hardware conversion returns; inputs whose result is not a normal number or
// zero (subnormal results, infinities, NaN, overflow) take the hardware
// conversion through a call the compiler cannot predicate into the fast path.
static __device__ __noinline__ float d2f_slow(double x) { return (float)x; }
static __device__ __noinline__ double f2d_slow(float x) { return (double)x; }

__device__ __forceinline__ float d2f_int(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  const unsigned sign = hi & 0x80000000u;
  if (e >= 897u && e <= 1150u) {  // binary32 exponents -126..127: a normal result
    // exponent rebiased (1023 -> 127) with the top 23 fraction bits below it
    unsigned f = (((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;  // the 29 dropped fraction bits
    f += (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) ? 1u : 0u;  // a carry may reach the
    return __uint_as_float(sign | f);                                        // exponent (and infinity)
  }
  if (e <= 872u) return __uint_as_float(sign);  // |x| < 2^-150: rounds to a signed zero
  return d2f_slow(x);
}

__device__ __forceinline__ double f2d_int(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xffu;
  if (e != 0u && e != 0xffu)  // normal: rebias the exponent (127 -> 1023), widen the fraction
    return __hiloint2double((int)((b & 0x80000000u) | (((b >> 3) & 0x0fffffffu) + (896u << 20))), (int)(b << 29));
  if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  return f2d_slow(x);
}

// A stored FP64 value in the arithmetic type T (the FP32 image through d2f_int).
template <typename T>
__device__ __forceinline__ T to_t(double x) {
  if constexpr (sizeof(T) == 4) return d2f_int(x);
  else return x;
}

// The mixed form's recovery: FP64 arithmetic for the cancellation in
// E - rho|u|^2/2, with 1/rho from the FP32 reciprocal refined by one Newton
// step in FP64 (r1 = r0 + r0 (1 - rho r0): relative error below 2e-14, far
// under what the FP32 result keeps) instead of an IEEE FP64 division, which
// on this part costs more FP64-pipe issue than the rest of the recovery.
// Densities outside the FP32 normal range take the division.
// Densities whose FP32 image or reciprocal would not be a normal float take
// the division.  Conversions on the integer pipes (d2f_int, f2d_int).
__device__ __forceinline__ double recip_refined(double x) {
  const float xf = d2f_int(x);
  if (!(fabsf(xf) >= 1e-37f && fabsf(xf) <= 1e37f)) return 1.0 / x;
  const double r = f2d_int(__frcp_rn(xf));
  return __fma_rn(r, __fma_rn(-x, r, 1.0), r);
}

template <int ND>
__device__ __forceinline__ void cons_to_prim_mixed(double gm1, const double* Q, float* W) {
  const double rho = Q[0];
  const double r = recip_refined(rho);
  double ke = 0.0;
  W[0] = d2f_int(rho);
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    const double u = Q[1 + k] * r;
    W[1 + k] = d2f_int(u);
    ke = __fma_rn(Q[1 + k], u, ke);
  }
  W[ND + 1] = d2f_int(gm1 * __fma_rn(-0.5, ke, Q[ND + 1]));
}

// Image of a state across an isothermal no-slip wall: velocity negated,
// pressure kept, temperature reflected about the wall value
// (T_ghost = 2 T_w - T), density from the equation of state.
template <int ND, typename T = double>
__device__ __forceinline__ void wall_image(const DevGrid& g, T* w) {
  constexpr int IP = ND + 1;
  T Tm = T(g.gm2) * w[IP] / w[0];
  T Tg = T(2.0) * T(g.twall) - Tm;
  w[0] = T(g.gm2) * w[IP] / Tg;
#pragma unroll
  for (int m = 0; m < ND; ++m) w[1 + m] = -w[1 + m];
}

// TW: the type the planes are stored in (double; float for the mixed form's
// primitives); TO: the type the state is returned (and its ghost images
// formed) in.  The conserved form (CONS) is FP64 only.
template <int ND, bool CONS = false, typename TW = double, typename TO = double>
__device__ __forceinline__ void load_state(const DevGrid& g, const TW* __restrict__ F, int c0,
                                           int c1, int c2, TO* w) {
  static_assert(!CONS || sizeof(TO) == 8, "conserved ghosts are FP64");
  Src s = resolve(g, c0, c1, c2);
  if (s.face >= 0) {
    if (s.pidx >= 0) {
      const double* P = g.prof[s.face >> 1][s.face & 1];
      long long fn = g.pf[s.face >> 1];
      double wp[ND + 2];
#pragma unroll
      for (int v = 0; v < ND + 2; ++v) wp[v] = P[(long long)v * fn + s.pidx];
      if (CONS) prim_to_cons<ND>(g, wp, reinterpret_cast<double*>(w));
      else {
#pragma unroll
        for (int v = 0; v < ND + 2; ++v) w[v] = TO(wp[v]);
      }
    } else {
      const double* st = CONS ? g.inflowQ[s.face >> 1][s.face & 1] : g.inflowW[s.face >> 1][s.face & 1];
#pragma unroll
      for (int v = 0; v < ND + 2; ++v) w[v] = TO(st[v]);
    }
  } else {
#pragma unroll
    for (int v = 0; v < ND + 2; ++v) w[v] = TO(F[(long long)v * g.N + s.idx]);
  }
#pragma unroll
  for (int d = 0; d < ND; ++d)
    if (s.flip & (1 << d)) w[1 + d] = -w[1 + d];
  for (int k = 0; k < s.walls; ++k) {
    if (CONS) {
      double wp[ND + 2];
      cons_to_prim_g<ND>(g, reinterpret_cast<const double*>(w), wp);
      wall_image<ND>(g, wp);
      prim_to_cons<ND>(g, wp, reinterpret_cast<double*>(w));
    } else {
      wall_image<ND, TO>(g, w);
    }
  }
}

// Scalar field at a possibly-ghost node: periodic wraps, a wall mirrors,
// anything else copies the boundary node.
__device__ __forceinline__ long long scalar_src(const DevGrid& g, int c0, int c1, int c2) {
  int c[3] = {c0, c1, c2};
#pragma unroll
  for (int d = 2; d >= 0; --d) {
    if (d >= g.nd) continue;
    int n = g.n[d], x = c[d];
    if (x >= 0 && x < n) continue;
    int side = x < 0 ? 0 : 1;
    int bc = g.bc[d][side];
    if (bc == BC_PERIODIC) { x %= n; if (x < 0) x += n; }
    else if (bc == BC_REFLECT || bc == BC_WALL) x = side == 0 ? -x - 1 : 2 * n - 1 - x;
    else x = side == 0 ? 0 : n - 1;
    x = x < 0 ? 0 : (x >= n ? n - 1 : x);
    c[d] = x;
  }
  return lin(g, c[0], c[1], c[2]);
}

// ---------------------------------------------------------------- line buffers
// Rows [lo, lo + m) along direction d (periodic: rows 0..n-1, positions wrap);
// lines over the other directions on the box (off, ext).
struct LineBuf {
  int d, lo, m, n, periodic;
  int off[3], ext[3];  // box of the other directions (entry d unused)
  long long nl;        // lines
  // lines ordered with the lower other direction fastest (x where it is one)
  __host__ __device__ long long line(const int* c) const {
    int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
    return (long long)(c[o1] + off[o1]) + (long long)ext[o1] * (long long)(c[o2] + off[o2]);
  }
  __device__ long long at(int comp, int pos, const int* c) const {
    int row;
    if (periodic) {
      row = pos % n;
      if (row < 0) row += n;
    } else {
      row = pos - lo;
    }
    return ((long long)comp * m + row) * nl + line(c);
  }
  __device__ void coords(long long L, int* c) const {
    int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
    c[o1] = (int)(L % ext[o1]) - off[o1];
    c[o2] = (int)(L / ext[o1]) - off[o2];
  }
};

// ---------------------------------------------------------------- state
// primitive from conserved: rho, u = m / rho, p = (gamma-1)(E - (m.u)/2)
template <int ND>
__device__ __forceinline__ void cons_to_prim(double gm1, const double* Q, double* W) {
  double rho = Q[0];
  double irho = 1.0 / rho;
  W[0] = rho;
  double ke = 0.0;
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    W[1 + k] = Q[1 + k] * irho;
    ke = (k == 0) ? Q[1] * W[1] : ke + Q[1 + k] * W[1 + k];
  }
  W[ND + 1] = gm1 * (Q[ND + 1] - 0.5 * ke);
}

// fused multiply-add in the arithmetic type
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// ---------------------------------------------------------------- stencils
// T = double: the FP64 parity form; T = float: the mixed form's flux arithmetic.
// explicit sixth-order central first derivative (MEG6 gradients)
template <typename T = double>
__device__ __forceinline__ T d6(T m3, T m2, T m1, T p1, T p2, T p3) {
  return T(0.75) * (p1 - m1) - T(3.0 / 20.0) * (p2 - m2) + T(1.0 / 60.0) * (p3 - m3);
}
// explicit fourth-order central first derivative (E4)
template <typename T = double>
__device__ __forceinline__ T d4(T m2, T m1, T p1, T p2) {
  return T(2.0 / 3.0) * (p1 - m1) - T(1.0 / 12.0) * (p2 - m2);
}
// second derivative from values and first derivatives (gradient-based)
template <typename T = double>
__device__ __forceinline__ T d2_from_grad(T wm, T w0, T wp, T dm, T dp) {
  return T(2.0) * (wp - T(2.0) * w0 + wm) - T(0.5) * (dp - dm);
}

// ---------------------------------------------------------------- MP5
template <typename T>
__device__ __forceinline__ T dmin(T a, T b) { return a < b ? a : b; }
template <typename T>
__device__ __forceinline__ T dmax(T a, T b) { return a > b ? a : b; }
template <typename T>
__device__ __forceinline__ T minmod2(T a, T b) {
  if (a > T(0) && b > T(0)) return dmin(a, b);
  if (a < T(0) && b < T(0)) return dmax(a, b);
  return T(0);
}
template <typename T>
__device__ __forceinline__ T minmod4(T a, T b, T c, T d) {
  if (a > T(0) && b > T(0) && c > T(0) && d > T(0)) return dmin(dmin(a, b), dmin(c, d));
  if (a < T(0) && b < T(0) && c < T(0) && d < T(0)) return dmax(dmax(a, b), dmax(c, d));
  return T(0);
}
// Suresh & Huynh (1997) monotonicity-preserving fifth-order interface value
// from u_{i-2} .. u_{i+2} (left state at i+1/2).
template <typename T>
__device__ __forceinline__ T mp5(T um2, T um1, T u0, T up1, T up2, T alpha, T eps) {
  T ul = (T(2.0) * um2 - T(13.0) * um1 + T(47.0) * u0 + T(27.0) * up1 - T(3.0) * up2) / T(60.0);
  T ump = u0 + minmod2(up1 - u0, alpha * (u0 - um1));
  if ((ul - u0) * (ul - ump) <= eps) return ul;
  T dm1 = um2 - T(2.0) * um1 + u0;
  T d0 = um1 - T(2.0) * u0 + up1;
  T dp1 = u0 - T(2.0) * up1 + up2;
  T dm4p = minmod4(T(4.0) * d0 - dp1, T(4.0) * dp1 - d0, d0, dp1);
  T dm4m = minmod4(T(4.0) * d0 - dm1, T(4.0) * dm1 - d0, d0, dm1);
  T uul = u0 + alpha * (u0 - um1);
  T uav = T(0.5) * (u0 + up1);
  T umd = uav - T(0.5) * dm4p;
  T ulc = u0 + T(0.5) * (u0 - um1) + T(4.0 / 3.0) * dm4m;
  T umin = dmax(dmin(dmin(u0, up1), umd), dmin(dmin(u0, uul), ulc));
  T umax = dmin(dmax(dmax(u0, up1), umd), dmax(dmax(u0, uul), ulc));
  return ul + minmod2(umin - ul, umax - ul);
}

// ---------------------------------------------------------------- frames
// Structural sparsity of the interface frame on a Cartesian grid (normal n,
// tangents t1, t2 along the axes); a curvilinear frame is dense.
__host__ __device__ constexpr bool frame_nz(bool cart, int nd, int dir, int vec, int m) {
  return !cart ? true
               : (vec == 0 ? m == dir
                           : (vec == 1 ? (nd == 2 ? m == 1 - dir : (dir == 2 ? m == 1 : m == 2))
                                       : (dir == 0 ? m == 1 : m == 0)));
}

// sum_m a[m] * u[m] over the structurally non-zero a[m], in index order
template <int ND, bool CART, int DIR, int VEC, typename T = double>
__device__ __forceinline__ T sdot(const T* a, const T* u) {
  T s = T(0);
  bool first = true;
#pragma unroll
  for (int m = 0; m < ND; ++m) {
    if (!frame_nz(CART, ND, DIR, VEC, m)) continue;
    if (first) { s = a[m] * u[m]; first = false; }
    else s = s + a[m] * u[m];
  }
  return s;
}

}  // namespace cgk
