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

constexpr int BC_PERIODIC = 0, BC_EXTRAP = 1, BC_REFLECT = 2, BC_INFLOW = 3;
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
};

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
};

__device__ __forceinline__ Src resolve(const DevGrid& g, int c0, int c1, int c2) {
  int c[3] = {c0, c1, c2};
  Src s;
  s.flip = 0;
  s.face = -1;
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
      return s;
    } else if (bc == BC_PERIODIC) {
      x %= n;
      if (x < 0) x += n;
    } else if (bc == BC_REFLECT) {
      x = side == 0 ? -x - 1 : 2 * n - 1 - x;
      s.flip ^= (1 << d);
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
template <int ND, bool CONS = false>
__device__ __forceinline__ void load_state(const DevGrid& g, const double* __restrict__ F, int c0,
                                           int c1, int c2, double* w) {
  Src s = resolve(g, c0, c1, c2);
  if (s.face >= 0) {
    const double* st = CONS ? g.inflowQ[s.face >> 1][s.face & 1] : g.inflowW[s.face >> 1][s.face & 1];
#pragma unroll
    for (int v = 0; v < ND + 2; ++v) w[v] = st[v];
  } else {
#pragma unroll
    for (int v = 0; v < ND + 2; ++v) w[v] = F[(long long)v * g.N + s.idx];
  }
#pragma unroll
  for (int d = 0; d < ND; ++d)
    if (s.flip & (1 << d)) w[1 + d] = -w[1 + d];
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
    else if (bc == BC_REFLECT) x = side == 0 ? -x - 1 : 2 * n - 1 - x;
    else x = side == 0 ? 0 : n - 1;
    x = x < 0 ? 0 : (x >= n ? n - 1 : x);
    c[d] = x;
  }
  return lin(g, c[0], c[1], c[2]);
}

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

// ---------------------------------------------------------------- stencils
// explicit sixth-order central first derivative (MEG6 gradients)
__device__ __forceinline__ double d6(double m3, double m2, double m1, double p1, double p2, double p3) {
  return 0.75 * (p1 - m1) - (3.0 / 20.0) * (p2 - m2) + (1.0 / 60.0) * (p3 - m3);
}
// explicit fourth-order central first derivative (E4)
__device__ __forceinline__ double d4(double m2, double m1, double p1, double p2) {
  return (2.0 / 3.0) * (p1 - m1) - (1.0 / 12.0) * (p2 - m2);
}
// second derivative from values and first derivatives (gradient-based)
__device__ __forceinline__ double d2_from_grad(double wm, double w0, double wp, double dm, double dp) {
  return 2.0 * (wp - 2.0 * w0 + wm) - 0.5 * (dp - dm);
}

// ---------------------------------------------------------------- MP5
__device__ __forceinline__ double dmin(double a, double b) { return a < b ? a : b; }
__device__ __forceinline__ double dmax(double a, double b) { return a > b ? a : b; }
__device__ __forceinline__ double minmod2(double a, double b) {
  if (a > 0.0 && b > 0.0) return dmin(a, b);
  if (a < 0.0 && b < 0.0) return dmax(a, b);
  return 0.0;
}
__device__ __forceinline__ double minmod4(double a, double b, double c, double d) {
  if (a > 0.0 && b > 0.0 && c > 0.0 && d > 0.0) return dmin(dmin(a, b), dmin(c, d));
  if (a < 0.0 && b < 0.0 && c < 0.0 && d < 0.0) return dmax(dmax(a, b), dmax(c, d));
  return 0.0;
}
// Suresh & Huynh (1997) monotonicity-preserving fifth-order interface value
// from u_{i-2} .. u_{i+2} (left state at i+1/2).
__device__ __forceinline__ double mp5(double um2, double um1, double u0, double up1, double up2,
                                      double alpha, double eps) {
  double ul = (2.0 * um2 - 13.0 * um1 + 47.0 * u0 + 27.0 * up1 - 3.0 * up2) / 60.0;
  double ump = u0 + minmod2(up1 - u0, alpha * (u0 - um1));
  if ((ul - u0) * (ul - ump) <= eps) return ul;
  double dm1 = um2 - 2.0 * um1 + u0;
  double d0 = um1 - 2.0 * u0 + up1;
  double dp1 = u0 - 2.0 * up1 + up2;
  double dm4p = minmod4(4.0 * d0 - dp1, 4.0 * dp1 - d0, d0, dp1);
  double dm4m = minmod4(4.0 * d0 - dm1, 4.0 * dm1 - d0, d0, dm1);
  double uul = u0 + alpha * (u0 - um1);
  double uav = 0.5 * (u0 + up1);
  double umd = uav - 0.5 * dm4p;
  double ulc = u0 + 0.5 * (u0 - um1) + (4.0 / 3.0) * dm4m;
  double umin = dmax(dmin(dmin(u0, up1), umd), dmin(dmin(u0, uul), ulc));
  double umax = dmin(dmax(dmax(u0, up1), umd), dmax(dmax(u0, uul), ulc));
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
template <int ND, bool CART, int DIR, int VEC>
__device__ __forceinline__ double sdot(const double* a, const double* u) {
  double s = 0.0;
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
