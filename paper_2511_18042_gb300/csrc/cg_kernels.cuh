// Kernels of one RK stage of the FP64 RHS: primitives, sensor, compact
// (tridiagonal) gradients, the fused C-GBR interface sweep with the residual
// and RK epilogue, and the CFL reduction.
#pragma once
#include <type_traits>
#include "cg_gbr.cuh"

namespace cgk {

// A box of node positions: index (i+off0) + ext0*((j+off1) + ext1*(k+off2)).
struct Box {
  int off[3], ext[3];
  __host__ __device__ long long size() const { return (long long)ext[0] * ext[1] * ext[2]; }
  __host__ __device__ long long at(int i, int j, int k) const {
    return (long long)(i + off[0]) + (long long)ext[0] * ((long long)(j + off[1]) + (long long)ext[1] * (long long)(k + off[2]));
  }
};

// Everything the stage kernels read and write besides the grid.
struct StageArgs {
  const double* W;     // primitives (nv planes, interior)
  const void* om;      // sensor on omBox, in the stage's arithmetic type
  Box omBox;
  const double* Gd;    // compact gradients along the sweep direction (line buffer gdLB)
  LineBuf gdLB;
  double* acc;         // flux-difference accumulator (nv planes)
  int first, last;     // first / last direction of the stage
  int defer;           // the last direction stores the total like the others; k_stage_update
                       // applies the residual and RK update afterwards
  int rk;              // last direction: 1 = RK update, 0 = write R
  int stage;           // 1, 2, 3
  double* R;
  const double* Un;    // state at the start of the step
  const double* Uc;    // state of the current stage
  double* Uout;
  const double* dt;    // device scalar
  unsigned int* bad_flag;
  unsigned long long* bad_idx;
  const unsigned char* mask;  // per-interface hybrid: troubled nodes on tBox (GBR where a neighbour is troubled)
  Box tBox;
  const int* guard;           // global hybrid: the kernel runs only if *guard == guard_want
  int guard_want;
  const void* hflux;          // per-interface hybrid: LAD flux-form interface fluxes (nv planes on hBox,
                              // in the sweep's arithmetic type)
  Box hBox;
  double* iface_out;          // diagnostics: interface fluxes [v][line][n+1] (NULL: none)
  const float* Wf;            // mixed form: the primitives stored in FP32
  const float* Gdf;           // mixed form: the compact gradients in FP32
};

// ---------------------------------------------------------------- stage epilogue
// Non-physical test of the mixed form: the sign of rho p / (gamma-1) =
// rho E - |m|^2/2 without a division.  An FP32 screen comes first: the float
// images carry a relative error of 2^-24 each, so rho E - |m|^2/2 evaluated
// in FP32 is within 4e-7 (rho E + |m|^2/2) of the exact value, and a margin of
// 1e-5 of that sum proves the sign; only nodes without that margin take the
// FP64 test.
template <int ND>
__device__ __forceinline__ bool mixed_nonphysical(const double* out) {
  constexpr int IP = ND + 1;
  const float r0 = d2f_int(out[0]), e0 = d2f_int(out[IP]);
  float m2f = 0.f;
#pragma unroll
  for (int m = 0; m < ND; ++m) {
    const float mm = d2f_int(out[1 + m]);
    m2f = m2f + mm * mm;
  }
  const float re = r0 * e0, hm = 0.5f * m2f;
  if (r0 > 0.f && re - hm > 1e-5f * (re + hm)) return false;
  double m2 = out[1] * out[1];
#pragma unroll
  for (int m = 1; m < ND; ++m) m2 = __fma_rn(out[1 + m], out[1 + m], m2);
  return !(out[0] > 0.0) || !(__fma_rn(out[0], out[IP], -0.5 * m2) > 0.0);
}

// The last direction's epilogue of one node from its stage totals tot[v] (the
// directions' flux differences; FP32 in the mixed form, MIX): R = -J tot
// (rk = 0) or the TVD-RK3 combination, and the non-physical test after stage
// 3.  Each stage has its own branch: a selection between the stages'
// formulas per value would issue all of them on the FP64 pipe.
// * FP64 form: the oracle's operation order, r = -(J tot), then
//   Un + dt r, or a Un + b (Uc + dt r).
// * mixed form: the stage increment z = -(b dt J) tot formed in FP32 (the
//   precision of the FP32 total itself: the factor adds a relative 2e-7),
//   widened on the integer pipes, and accumulated in FP64:
//   U = a Un + b Uc + z (Un + z in stage 1), one FP64 add or two fused
//   multiply-adds per variable.
template <int ND, bool MIX, typename TA>
__device__ __forceinline__ void stage_epilogue(const DevGrid& g, const StageArgs& A, long long qi, double J,
                                               const TA* tot, double (&out)[ND + 2]) {
  constexpr int NV = ND + 2, IP = ND + 1;
  auto wide = [](TA t) -> double {
    if constexpr (MIX) return f2d_int(t);
    else return double(t);
  };
  if (!A.rk) {
#pragma unroll
    for (int v = 0; v < NV; ++v) A.R[v * g.N + qi] = -(J * wide(tot[v]));
    return;
  }
  const double dt = *A.dt;
  if (A.stage == 1) {
    [[maybe_unused]] float cJf = 0.f;
    if constexpr (MIX) cJf = -(d2f_int(dt) * d2f_int(J));
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double un = A.Un[v * g.N + qi];
      if constexpr (MIX) {
        out[v] = un + f2d_int(cJf * tot[v]);
      } else {
        const double r = -(J * wide(tot[v]));
        out[v] = un + dt * r;
      }
      A.Uout[v * g.N + qi] = out[v];
    }
    return;
  }
  const double ca = A.stage == 2 ? 0.75 : (1.0 / 3.0), cb = A.stage == 2 ? 0.25 : (2.0 / 3.0);
  [[maybe_unused]] float cJf = 0.f;
  if constexpr (MIX) cJf = -((A.stage == 2 ? 0.25f : (2.0f / 3.0f)) * d2f_int(dt)) * d2f_int(J);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double un = A.Un[v * g.N + qi], uc = A.Uc[v * g.N + qi];
    if constexpr (MIX) {
      out[v] = __fma_rn(ca, un, __fma_rn(cb, uc, f2d_int(cJf * tot[v])));
    } else {
      const double r = -(J * wide(tot[v]));
      out[v] = ca * un + cb * (uc + dt * r);
    }
    A.Uout[v * g.N + qi] = out[v];
  }
  if (A.stage != 3) return;
  bool bad;
  if constexpr (MIX) {
    bad = mixed_nonphysical<ND>(out);
  } else {
    double ke = out[1] * (out[1] / out[0]);
#pragma unroll
    for (int m = 1; m < ND; ++m) ke = ke + out[1 + m] * (out[1 + m] / out[0]);
    double p = g.gm1 * (out[IP] - 0.5 * ke);
    bad = !(out[0] > 0.0) || !(p > 0.0);
  }
  if (bad) {
    atomicOr(A.bad_flag, 1u);
    atomicMin(A.bad_idx, (unsigned long long)qi);
  }
}

// ---------------------------------------------------------------- block coordinates
// Each stage kernel is a body over the coordinates of its block plus a thin
// __global__ wrapper that passes the hardware ones.  The batched stage
// (cg_batch_stage.cu) runs the same bodies with a member's share of one
// persistent grid instead.
struct VBlock {
  unsigned x, y, z;     // block index
  unsigned gx, gy, gz;  // grid size in blocks
};

__device__ __forceinline__ VBlock hw_block() {
  return VBlock{blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y, gridDim.z};
}

// ---------------------------------------------------------------- primitives
// Primitives recovered in FP64 (p = (gamma-1)(E - rho|u|^2/2)); stored as TW
// (float for the mixed form's FP32 consumers).
template <int ND, typename TW = double>
__device__ __forceinline__ void k_prim_body(const VBlock& vb, const DevGrid& g, const double* __restrict__ U, TW* __restrict__ W) {
  constexpr int NV = ND + 2;
  for (long long q = vb.x * (long long)blockDim.x + threadIdx.x; q < g.N;
       q += (long long)vb.gx * blockDim.x) {
    double Q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Q[v] = U[v * g.N + q];
    if constexpr (sizeof(TW) == 4) {
      float w[NV];
      cons_to_prim_mixed<ND>(g.gm1, Q, w);
#pragma unroll
      for (int v = 0; v < NV; ++v) W[v * g.N + q] = w[v];
    } else {
      double w[NV];
      cons_to_prim<ND>(g.gm1, Q, w);
#pragma unroll
      for (int v = 0; v < NV; ++v) W[v * g.N + q] = w[v];
    }
  }
}

template <int ND, typename TW = double>
__global__ void k_prim(DevGrid g, const double* __restrict__ U, TW* __restrict__ W) {
  k_prim_body<ND, TW>(hw_block(), g, U, W);
}

// ---------------------------------------------------------------- sensor
// Quotient of the sensor's ratios: IEEE division in FP64; in the mixed form's
// FP32 sensor the fast reciprocal-multiply (2 ulp, denominators below 2^126:
// sums of pressures and of squared velocity gradients).
template <typename T>
__device__ __forceinline__ T sensor_div(T a, T b) {
  if constexpr (sizeof(T) == 4) return __fdividef(a, b);
  else return a / b;
}

// Omega^d = phi * zeta on the box [-4, n+3]: phi the largest normalised
// pressure second difference over the directions, zeta a Ducros ratio of the
// dilatation (one in irrotational dilatation-free flow).
// T = double: FP64 parity form; T = float: the mixed form's FP32 sensor
// (FP64 primitives and gradients read, converted once).
// Ducros ratio zeta = (div^2 + eps) / (div^2 + |curl|^2 + eps) from the
// physical velocity gradients gu[k][m] = d u_k / d x_m.
template <int ND, typename T>
__device__ __forceinline__ T sensor_zeta(const T (&gu)[3][3]) {
  T div = gu[0][0];
#pragma unroll
  for (int k = 1; k < ND; ++k) div = div + gu[k][k];
  const T eps = T(1e-32);
  if (ND == 1) return sensor_div(div * div + eps, div * div + eps);
  if (ND == 2) {
    T w3 = gu[1][0] - gu[0][1];
    return sensor_div(div * div + eps, div * div + w3 * w3 + eps);
  }
  T w1 = gu[2][1] - gu[1][2], w2 = gu[0][2] - gu[2][0], w3 = gu[1][0] - gu[0][1];
  return sensor_div(div * div + eps, div * div + (w1 * w1 + w2 * w2 + w3 * w3) + eps);
}

// Physical velocity gradients gu[k][m] = sum_l (J xi_hat[l][m]) du[l][k] from
// the index-space ones du[l][k] = d u_k / d xi_l at node c.
template <int ND, bool CART, typename T>
__device__ __forceinline__ void sensor_gu(const DevGrid& g, const int* c, const T (&du)[3][3], T (&gu)[3][3]) {
  if (CART) {
#pragma unroll
    for (int k = 0; k < ND; ++k)
#pragma unroll
      for (int m = 0; m < ND; ++m) gu[k][m] = gconst<T>(g.cjxh[m], g.f_cjxh[m]) * du[m][k];
  } else {
    long long pq = plin(g, c[0], c[1], c[2]);
    // J xi_hat: in the mixed form each factor is rounded to FP32 (on the
    // integer pipes) and the product taken there
    const T J = to_t<T>(g.jac[pq]);
    T xm[3][3];
#pragma unroll
    for (int l = 0; l < ND; ++l)
#pragma unroll
      for (int m = 0; m < ND; ++m) xm[l][m] = J * to_t<T>(g.xh[(l * ND + m) * g.NP + pq]);
#pragma unroll
    for (int k = 0; k < ND; ++k)
#pragma unroll
      for (int m = 0; m < ND; ++m) {
        T s = xm[0][m] * du[0][k];
#pragma unroll
        for (int l = 1; l < ND; ++l) s = s + xm[l][m] * du[l][k];
        gu[k][m] = s;
      }
  }
}

template <int ND, bool CART, bool COMPACT, typename T = double>
__device__ __forceinline__ void k_omega_body(const VBlock& vb, const DevGrid& g, const T* __restrict__ W, const T* __restrict__ G0,
                        const T* __restrict__ G1, const T* __restrict__ G2, LineBuf gb0,
                        LineBuf gb1, LineBuf gb2, T* __restrict__ om, Box ob, const int* guard, int want) {
  constexpr int NV = ND + 2, IP = ND + 1;
  if (guard && *guard != want) return;
  long long tot = ob.size();
  for (long long e = vb.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)vb.gx * blockDim.x) {
    int c[3];
    if (tot <= 0x7fffffffLL) {  // 32-bit index arithmetic (a 64-bit division costs several times more)
      unsigned r = (unsigned)e;
      const unsigned x0 = (unsigned)ob.ext[0], x1 = (unsigned)ob.ext[1];
      c[0] = (int)(r % x0) - ob.off[0];
      r /= x0;
      c[1] = (int)(r % x1) - ob.off[1];
      c[2] = (int)(r / x1) - ob.off[2];
    } else {
      long long r = e;
      c[0] = (int)(r % ob.ext[0]) - ob.off[0];
      r /= ob.ext[0];
      c[1] = (int)(r % ob.ext[1]) - ob.off[1];
      c[2] = (int)(r / ob.ext[1]) - ob.off[2];
    }
    T phi = T(0);
    T du[3][3];  // du[l][k] = d u_k / d xi_l
    // nodes whose whole stencil is interior read the planes directly (the
    // same values the boundary mapping would give), and only the components
    // used: pressure at the neighbours, velocities on the gradient stencil
    bool inner = true;
#pragma unroll
    for (int d = 0; d < ND; ++d) inner = inner && c[d] >= 3 && c[d] < g.n[d] - 3;
    if (inner) {
      const long long q = lin(g, c[0], c[1], c[2]);
      const T p0 = T(W[IP * g.N + q]);
#pragma unroll
      for (int l = 0; l < ND; ++l) {
        const long long st = l == 0 ? 1 : (l == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1]);
        const T* P = W + IP * g.N + q;
        const T pm = T(P[-st]), pp = T(P[st]);
        T a = sensor_div(fabs(pp - T(2.0) * p0 + pm), pp + T(2.0) * p0 + pm);
        if (a > phi) phi = a;
        if (!COMPACT) {
#pragma unroll
          for (int k = 0; k < ND; ++k) {
            const T* V = W + (1 + k) * g.N + q;
            du[l][k] = d6<T>(T(V[-3 * st]), T(V[-2 * st]), T(V[-st]), T(V[st]), T(V[2 * st]), T(V[3 * st]));
          }
        } else {
          const T* G = l == 0 ? G0 : (l == 1 ? G1 : G2);
          const LineBuf& gb = l == 0 ? gb0 : (l == 1 ? gb1 : gb2);
#pragma unroll
          for (int k = 0; k < ND; ++k) du[l][k] = T(G[gb.at(1 + k, c[l], c)]);
        }
      }
    } else {
    T w0d[NV];
    load_state<ND, false, T, T>(g, W, c[0], c[1], c[2], w0d);
    const T p0 = T(w0d[IP]);
#pragma unroll
    for (int l = 0; l < ND; ++l) {
      // neighbours c-3..c-1, c+1..c+3 along l (c-1, c+1 only with compact
      // gradients) from one load site: the boundary resolution is inlined once
      // per direction instead of once per neighbour, which kept the 3D kernel's
      // code out of the instruction cache
      T s[6][NV];
      const int t0 = COMPACT ? 2 : 0, t1 = COMPACT ? 4 : 6;
#pragma unroll 1
      for (int t = t0; t < t1; ++t) {
        int a[3] = {c[0], c[1], c[2]};
        a[l] += t < 3 ? t - 3 : t - 2;
        load_state<ND, false, T, T>(g, W, a[0], a[1], a[2], s[t]);
      }
      const T pm = T(s[2][IP]), pp = T(s[3][IP]);
      T a = sensor_div(fabs(pp - T(2.0) * p0 + pm), pp + T(2.0) * p0 + pm);
      if (a > phi) phi = a;
      if (!COMPACT) {
#pragma unroll
        for (int k = 0; k < ND; ++k)
          du[l][k] = d6<T>(T(s[0][1 + k]), T(s[1][1 + k]), T(s[2][1 + k]), T(s[3][1 + k]), T(s[4][1 + k]),
                           T(s[5][1 + k]));
      } else {
        const T* G = l == 0 ? G0 : (l == 1 ? G1 : G2);
        const LineBuf& gb = l == 0 ? gb0 : (l == 1 ? gb1 : gb2);
#pragma unroll
        for (int k = 0; k < ND; ++k) du[l][k] = T(G[gb.at(1 + k, c[l], c)]);
      }
    }
    }
    T gu[3][3];
    sensor_gu<ND, CART, T>(g, c, du, gu);
    om[ob.at(c[0], c[1], c[2])] = phi * sensor_zeta<ND, T>(gu);
  }
}

template <int ND, bool CART, bool COMPACT, typename T = double>
__global__ void k_omega(DevGrid g, const T* __restrict__ W, const T* __restrict__ G0,
                        const T* __restrict__ G1, const T* __restrict__ G2, LineBuf gb0,
                        LineBuf gb1, LineBuf gb2, T* __restrict__ om, Box ob, const int* guard, int want) {
  k_omega_body<ND, CART, COMPACT, T>(hw_block(), g, W, G0, G1, G2, gb0, gb1, gb2, om, ob, guard, want);
}

// The sensor of explicit gradients (MEG6) in 2D and 3D on tiles of 32 x 8
// nodes of the box (one z plane per block in 3D): pressure and velocities of
// the tile and a halo of three nodes in x and y staged once in shared memory
// (ghost positions through the boundary mapping, as load_state gives them),
// the z neighbours read directly.  The same values and the same arithmetic in
// the same order as k_omega_body, with one global load per staged value
// instead of one per stencil point.
constexpr int OMT_X = 32, OMT_Y = 8, OMT_H = 3;
template <int ND, bool CART, typename T>
__global__ void __launch_bounds__(OMT_X * OMT_Y) k_omega_tile(DevGrid g, const T* __restrict__ W, T* __restrict__ om, Box ob,
                                                             const int* guard, int want) {
  static_assert(ND >= 2, "tiles of x and y");
  constexpr int NV = ND + 2, IP = ND + 1;
  constexpr int SX = OMT_X + 2 * OMT_H, SY = OMT_Y + 2 * OMT_H;
  __shared__ T sP[SY][SX];
  __shared__ T sU[ND][SY][SX];
  if (guard && *guard != want) return;
  const int x0 = (int)blockIdx.x * OMT_X - ob.off[0], y0 = (int)blockIdx.y * OMT_Y - ob.off[1];
  const int cz = ND == 3 ? (int)blockIdx.z - ob.off[2] : 0;
  const bool zin = cz >= 0 && cz < (ND == 3 ? g.n[2] : 1);
  const int tid = threadIdx.y * OMT_X + threadIdx.x;
  for (int e = tid; e < SX * SY; e += OMT_X * OMT_Y) {
    const int sy = e / SX, sx = e - sy * SX;
    const int x = x0 - OMT_H + sx, y = y0 - OMT_H + sy;
    T w[NV];
    if (zin && x >= 0 && x < g.n[0] && y >= 0 && y < g.n[1]) {
      const long long q = lin(g, x, y, cz);
#pragma unroll
      for (int v = 1; v < NV; ++v) w[v] = W[v * g.N + q];
    } else {
      load_state<ND, false, T, T>(g, W, x, y, cz, w);
    }
    sP[sy][sx] = w[IP];
#pragma unroll
    for (int k = 0; k < ND; ++k) sU[k][sy][sx] = w[1 + k];
  }
  __syncthreads();
  const int ex = (int)blockIdx.x * OMT_X + threadIdx.x, ey = (int)blockIdx.y * OMT_Y + threadIdx.y;
  if (ex >= ob.ext[0] || ey >= ob.ext[1]) return;
  int c[3] = {x0 + (int)threadIdx.x, y0 + (int)threadIdx.y, cz};
  const int tx = threadIdx.x + OMT_H, ty = threadIdx.y + OMT_H;
  const T p0 = sP[ty][tx];
  T phi = T(0);
  T du[3][3];
  {  // x
    const T pm = sP[ty][tx - 1], pp = sP[ty][tx + 1];
    T a = sensor_div(fabs(pp - T(2.0) * p0 + pm), pp + T(2.0) * p0 + pm);
    if (a > phi) phi = a;
#pragma unroll
    for (int k = 0; k < ND; ++k)
      du[0][k] = d6<T>(sU[k][ty][tx - 3], sU[k][ty][tx - 2], sU[k][ty][tx - 1], sU[k][ty][tx + 1], sU[k][ty][tx + 2],
                       sU[k][ty][tx + 3]);
  }
  {  // y
    const T pm = sP[ty - 1][tx], pp = sP[ty + 1][tx];
    T a = sensor_div(fabs(pp - T(2.0) * p0 + pm), pp + T(2.0) * p0 + pm);
    if (a > phi) phi = a;
#pragma unroll
    for (int k = 0; k < ND; ++k)
      du[1][k] = d6<T>(sU[k][ty - 3][tx], sU[k][ty - 2][tx], sU[k][ty - 1][tx], sU[k][ty + 1][tx], sU[k][ty + 2][tx],
                       sU[k][ty + 3][tx]);
  }
  if constexpr (ND == 3) {  // z: direct loads in the interior, the boundary mapping elsewhere
    T s[6][NV];
    const bool inner = c[0] >= 0 && c[0] < g.n[0] && c[1] >= 0 && c[1] < g.n[1] && c[2] >= 3 && c[2] < g.n[2] - 3;
    if (inner) {
      const long long q = lin(g, c[0], c[1], c[2]), st = (long long)g.n[0] * g.n[1];
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        const long long qt = q + (long long)(t < 3 ? t - 3 : t - 2) * st;
#pragma unroll
        for (int v = 1; v < NV; ++v) s[t][v] = W[v * g.N + qt];
      }
    } else {
#pragma unroll 1
      for (int t = 0; t < 6; ++t) load_state<ND, false, T, T>(g, W, c[0], c[1], c[2] + (t < 3 ? t - 3 : t - 2), s[t]);
    }
    const T pm = s[2][IP], pp = s[3][IP];
    T a = sensor_div(fabs(pp - T(2.0) * p0 + pm), pp + T(2.0) * p0 + pm);
    if (a > phi) phi = a;
#pragma unroll
    for (int k = 0; k < ND; ++k)
      du[2][k] = d6<T>(s[0][1 + k], s[1][1 + k], s[2][1 + k], s[3][1 + k], s[4][1 + k], s[5][1 + k]);
  }
  T gu[3][3];
  sensor_gu<ND, CART, T>(g, c, du, gu);
  om[ob.at(c[0], c[1], c[2])] = phi * sensor_zeta<ND, T>(gu);
}

// ---------------------------------------------------------------- compact gradients
// Tridiagonal (MIG4: 1/4, 1, 1/4) first derivative of the primitives along d,
// one thread per (line, variable), Thomas elimination with the line-independent
// pivots cp[] and reciprocal pivots 1/den[] precomputed on the host.  Non-periodic lines span the
// positions [-6, n+5] with E4 closure rows at both ends; periodic lines are
// cyclic on [0, n-1] (Sherman-Morrison with the correction vector z[]) and
// the ghost positions copy the wrapped values.  Lines exist for every
// position of the other directions in [-4, n+3].
template <typename T>
struct LineCoefT {
  const T* cp;   // Thomas pivots of the line system
  const T* den;  // reciprocals of the elimination pivots, 1/den_i
  const T* z;    // cyclic: solution of the correction system
  T a;           // off-diagonal
  T gam;         // cyclic: -1
  T fden;        // cyclic: 1 + z[0] + a z[m-1] / gam
  int m;         // unknowns
  int lo;        // first position of the system (non-periodic)
  int periodic;
};
using LineCoef = LineCoefT<double>;

// ---------------------------------------------------------------- C-GBR sweep
constexpr int SWEEP_TL = 64;
// lines per tile: the default, and the candidates an autotuner may choose from
// (LW * SWEEP_TL must be a multiple of the 256 threads of a block)
__host__ __device__ constexpr int sweep_lw(int dir) { return dir == 0 ? 4 : 8; }
template <int ND, int LW>
__host__ __device__ constexpr int sweep_smem_doubles() {
  return (ND + 2) * (SWEEP_TL + 9 + SWEEP_TL + 3 + SWEEP_TL + 1 + SWEEP_TL) * LW + (SWEEP_TL + 7) * LW;
}

// Blocks per SM the register budget is sized for (256 threads a block):
// * FP64: two (128 registers).  The 3D curvilinear sweep, with its frame and
//   metric terms, spills about 300 bytes a thread there, to L1; at one block
//   (8 warps an SM) it did not spill but ran 9-12 % slower on the 3D ramp.
// * 1D/2D FP32: four (64 registers; up to 40 bytes a thread spill).  The
//   kernel is latency-bound at two blocks, 16 warps an SM: four took the
//   triple point's mixed MEG6 step from 1.24 to 1.02 ms.
// * 3D FP32: three (85 registers; up to 112 bytes a thread spill): on the 3D
//   ramp 10-15 % faster than two.
template <int ND, bool CART, typename T>
__host__ __device__ constexpr int sweep_min_blocks() {
  return sizeof(T) == 8 ? 2 : (ND <= 2 ? 4 : 3);
}

// T = double: FP64 form; T = float: mixed form (FP32 reconstruction and
// fluxes from FP64 primitives; FP64 flux differences, residual and RK update).
// UNIT tags the translation unit that compiles the kernel (0: FP64 without
// contraction, the oracle's operation order; 1: FP64 with fused multiply-add;
// 2: FP32): the code is the same, the compilation flags differ, and distinct
// instantiations keep the units' kernels apart.
template <int ND, int DIR, bool CART, bool COMPACT, typename T, int LW, int UNIT>
__device__ __forceinline__ void k_gbr_sweep_body(const VBlock& vb, const DevGrid& g, const GbrCfg& q, const StageArgs& A) {
  static_assert((SWEEP_TL * LW) % 256 == 0, "a tile must hold a multiple of the block's threads");
  constexpr int NV = ND + 2;
  constexpr bool MIX = sizeof(T) == 4;
  constexpr int TL = SWEEP_TL;
  constexpr int RW = TL + 9, RD = TL + 3, RDD = TL + 1, RO = TL + 7;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  T* sW = sm;
  T* sD = sW + NV * RW * LW;
  T* sDD = sD + NV * RD * LW;
  T* sF = sDD + NV * RDD * LW;
  T* sO = sF + NV * TL * LW;
  auto IX = [](int v, int r, int l, int rows) {
    return DIR == 0 ? (v * LW + l) * rows + r : (v * rows + r) * LW + l;
  };
  // The mixed form in 2D (four FP32 components, 16 bytes a node) keeps the
  // staged arrays node-major and moves a node's components with one 16-byte
  // shared-memory access (consecutive threads take consecutive nodes, so the
  // accesses stay free of bank conflicts); the other forms keep one plane per
  // component.
  constexpr bool VEC = MIX && NV == 4;
  auto NX = [](int r, int l, int rows) { return DIR == 0 ? l * rows + r : r * LW + l; };
  auto ldn = [&](const T* arr, int r, int l, int rows, T* w) {
    if constexpr (VEC) {
      const float4 f = reinterpret_cast<const float4*>(arr)[NX(r, l, rows)];
      w[0] = f.x;
      w[1] = f.y;
      w[2] = f.z;
      w[3] = f.w;
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) w[v] = arr[IX(v, r, l, rows)];
    }
  };
  auto stn = [&](T* arr, int r, int l, int rows, const T* w) {
    if constexpr (VEC) {
      reinterpret_cast<float4*>(arr)[NX(r, l, rows)] = make_float4(w[0], w[1], w[2], w[3]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) arr[IX(v, r, l, rows)] = w[v];
    }
  };
  if (A.guard && *A.guard != A.guard_want) return;
  const int tid = threadIdx.x;
  const int n = g.n[DIR];
  // tile origin along DIR and line coordinates
  int i0;
  long long nlines;
  if (DIR == 0) {
    i0 = vb.x * (TL - 1);
    nlines = (long long)g.n[1] * g.n[2];
  } else {
    i0 = vb.y * (TL - 1);
    nlines = 0;
  }
  // The tile's lines, computed once per block (the integer divisions and
  // index products would otherwise be repeated for every staged value):
  // coordinates of the two other directions (-1 in entry 0: no such line),
  // the linear index of the line's node 0 in the state planes and in the
  // sensor box; node x of the line is at base + x * stride.
  __shared__ int s_lc[LW][3];
  __shared__ long long s_lq[LW], s_lo[LW];
  if (tid < LW) {
    const int l = tid;
    int c[3] = {0, 0, 0};
    bool ok;
    if (DIR == 0) {
      long long L = (long long)vb.y * LW + l;
      ok = L < nlines;
      if (ok) {
        c[1] = (int)(L % g.n[1]);
        c[2] = (int)(L / g.n[1]);
      }
    } else {
      int x = vb.x * LW + l;
      ok = x < g.n[0];
      if (ok) {
        c[0] = x;
        c[DIR == 1 ? 2 : 1] = vb.z;
      }
    }
    s_lc[l][0] = ok ? c[0] : -1;
    s_lc[l][1] = c[1];
    s_lc[l][2] = c[2];
    c[DIR] = 0;
    s_lq[l] = ok ? lin(g, c[0], c[1], c[2]) : 0;
    s_lo[l] = ok ? A.omBox.at(c[0], c[1], c[2]) : 0;
  }
  __syncthreads();
  const long long qs = DIR == 0 ? 1 : (DIR == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1]);
  const long long os = DIR == 0 ? 1 : (DIR == 1 ? (long long)A.omBox.ext[0] : (long long)A.omBox.ext[0] * A.omBox.ext[1]);
  // coordinates of line l (the two other directions)
  auto line_coords = [&](int l, int* c) -> bool {
    if (s_lc[l][0] < 0) return false;
    c[0] = s_lc[l][0];
    c[1] = s_lc[l][1];
    c[2] = s_lc[l][2];
    return true;
  };
  // Per-interface hybrid: a tile none of whose interfaces takes the GBR flux
  // (no troubled node on either side of any of them) skips steps 1-3, whose
  // staged primitives, derivatives and sensor values only the GBR fluxes read.
  bool stage_tile = true;
  if (A.mask) {
    int any = 0;
#pragma unroll 1
    for (int e = tid; e < TL * LW; e += blockDim.x) {
      int a = DIR == 0 ? e % TL : e / LW;
      int l = DIR == 0 ? e / TL : e % LW;
      int i = i0 - 1 + a;
      int c[3] = {0, 0, 0};
      if (!line_coords(l, c) || i > n - 1) continue;
      c[DIR] = i;
      int cn[3] = {c[0], c[1], c[2]};
      cn[DIR] = i + 1;
      if (A.mask[A.tBox.at(c[0], c[1], c[2])] != 0 || A.mask[A.tBox.at(cn[0], cn[1], cn[2])] != 0) any = 1;
    }
    stage_tile = __syncthreads_or(any) != 0;
  }
  if (stage_tile) {
    // 1. primitives of the tile (ghosts resolved by the boundary conditions;
    // interior nodes read directly, the same values)
    for (int e = tid; e < RW * LW; e += blockDim.x) {
      int r = DIR == 0 ? e % RW : e / LW;
      int l = DIR == 0 ? e / RW : e % LW;
      int c[3] = {0, 0, 0};
      T w[NV];
      const int x = i0 - 5 + r;
      if (line_coords(l, c) && x >= 0 && x < n) {
        const long long q0 = s_lq[l] + (long long)x * qs;
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = MIX ? T(A.Wf[(long long)v * g.N + q0]) : T(A.W[(long long)v * g.N + q0]);
      } else if (line_coords(l, c)) {
        c[DIR] = x;
        if (MIX) load_state<ND, false, float, T>(g, A.Wf, c[0], c[1], c[2], w);
        else load_state<ND, false, double, T>(g, A.W, c[0], c[1], c[2], w);
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = T(1);
      }
      stn(sW, r, l, RW, w);
    }
    // sensor window values
    for (int e = tid; e < RO * LW; e += blockDim.x) {
      int r = DIR == 0 ? e % RO : e / LW;
      int l = DIR == 0 ? e / RO : e % LW;
      T o = T(0);
      int x = i0 - 4 + r;
      if (s_lc[l][0] >= 0 && x <= n + 3) o = static_cast<const T*>(A.om)[s_lo[l] + (long long)x * os];
      sO[(DIR == 0) ? l * RO + r : r * LW + l] = o;
    }
    __syncthreads();
    // 2. first derivatives along DIR on nodes i0-2 .. i0+TL
    for (int e = tid; e < RD * LW; e += blockDim.x) {
      int r = DIR == 0 ? e % RD : e / LW;
      int l = DIR == 0 ? e / RD : e % LW;
      T d[NV];
      if (!COMPACT) {
        T m3[NV], m2[NV], m1[NV], p1[NV], p2[NV], p3[NV];
        ldn(sW, r, l, RW, m3);
        ldn(sW, r + 1, l, RW, m2);
        ldn(sW, r + 2, l, RW, m1);
        ldn(sW, r + 4, l, RW, p1);
        ldn(sW, r + 5, l, RW, p2);
        ldn(sW, r + 6, l, RW, p3);
#pragma unroll
        for (int v = 0; v < NV; ++v) d[v] = d6(m3[v], m2[v], m1[v], p1[v], p2[v], p3[v]);
      } else {
        int c[3] = {0, 0, 0};
        int x = i0 - 2 + r;
        bool ok = line_coords(l, c) && x <= n + 5;
#pragma unroll
        for (int v = 0; v < NV; ++v)
          d[v] = ok ? (MIX ? T(A.Gdf[A.gdLB.at(v, x, c)]) : T(A.Gd[A.gdLB.at(v, x, c)])) : T(0);
      }
      stn(sD, r, l, RD, d);
    }
    __syncthreads();
    // 3. second derivatives on nodes i0-1 .. i0+TL-1
    for (int e = tid; e < RDD * LW; e += blockDim.x) {
      int r = DIR == 0 ? e % RDD : e / LW;
      int l = DIR == 0 ? e / RDD : e % LW;
      T wm[NV], w0[NV], wp[NV], dm[NV], dp[NV], dd[NV];
      ldn(sW, r + 3, l, RW, wm);
      ldn(sW, r + 4, l, RW, w0);
      ldn(sW, r + 5, l, RW, wp);
      ldn(sD, r, l, RD, dm);
      ldn(sD, r + 2, l, RD, dp);
#pragma unroll
      for (int v = 0; v < NV; ++v) dd[v] = d2_from_grad(wm[v], w0[v], wp[v], dm[v], dp[v]);
      stn(sDD, r, l, RDD, dd);
    }
    __syncthreads();
  }
  // 4. interface fluxes i+1/2, i = i0-1+a
  constexpr int PER = (TL * LW) / 256;
#pragma unroll 1
  for (int k = 0; k < PER; ++k) {
    int e = tid + k * 256;
    int a = DIR == 0 ? e % TL : e / LW;
    int l = DIR == 0 ? e / TL : e % LW;
    int i = i0 - 1 + a;
    int c[3] = {0, 0, 0};
    T F[NV];
    bool ok = line_coords(l, c) && i <= n - 1;
    c[DIR] = i;
    bool use_gbr = ok;
    if (ok && A.mask) {
      int cn[3] = {c[0], c[1], c[2]};
      cn[DIR] = i + 1;
      use_gbr = A.mask[A.tBox.at(c[0], c[1], c[2])] != 0 || A.mask[A.tBox.at(cn[0], cn[1], cn[2])] != 0;
    }
    if (use_gbr) {
      T Wst[6][NV], Wd[2][NV], Wdd[2][NV];
#pragma unroll
      for (int j = 0; j < 6; ++j) ldn(sW, a + 2 + j, l, RW, Wst[j]);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        ldn(sD, a + 1 + j, l, RD, Wd[j]);
        ldn(sDD, a + j, l, RDD, Wdd[j]);
      }
      T omb = sO[(DIR == 0) ? l * RO + a + 3 : (a + 3) * LW + l];
      for (int jj = 1 - q.window; jj <= q.window; ++jj) {
        T o = sO[(DIR == 0) ? l * RO + a + 3 + jj : (a + 3 + jj) * LW + l];
        omb = dmax(omb, o);
      }
      T xi[3] = {T(0), T(0), T(0)};
      if (!CART) {
        long long pq = plin(g, c[0], c[1], c[2]);
#pragma unroll
        for (int m = 0; m < ND; ++m) xi[m] = to_t<T>(g.xt[(DIR * ND + m) * g.NP + pq]);
      }
      gbr_flux<ND, CART, DIR, T>(q, g, Wst, Wd, Wdd, omb, xi, F);
    } else if (ok) {
      long long hi = A.hBox.at(c[0], c[1], c[2]);
      long long hs = A.hBox.size();
#pragma unroll
      for (int v = 0; v < NV; ++v) F[v] = static_cast<const T*>(A.hflux)[v * hs + hi];
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) F[v] = T(0);
    }
    stn(sF, a, l, TL, F);
    if (A.iface_out && ok) {
      long long line = DIR == 0 ? (long long)c[1] + (long long)g.n[1] * c[2]
                                : (DIR == 1 ? (long long)c[0] + (long long)g.n[0] * c[2]
                                            : (long long)c[0] + (long long)g.n[0] * c[1]);
      long long nlin = g.N / n;
#pragma unroll
      for (int v = 0; v < NV; ++v) A.iface_out[((long long)v * nlin + line) * (n + 1) + (i + 1)] = (double)F[v];
    }
  }
  __syncthreads();
  // 5. flux differences of cells i0 .. i0+TL-2, residual and RK epilogue
  for (int e = tid; e < (TL - 1) * LW; e += blockDim.x) {
    int a = DIR == 0 ? e % (TL - 1) : e / LW;
    int l = DIR == 0 ? e / (TL - 1) : e % LW;
    int c[3] = {0, 0, 0};
    int x = i0 + a;
    if (!line_coords(l, c) || x >= n) continue;
    c[DIR] = x;
    long long qi = s_lq[l] + (long long)x * qs;
    // mixed form: the FP32 fluxes differenced and summed over the directions in
    // FP32 (acc read as float), the stage total carried into the FP64 update
    using TA = typename std::conditional<MIX, float, double>::type;
    TA* acc = reinterpret_cast<TA*>(A.acc);
    TA tot[NV];
    T f0[NV], f1[NV];
    ldn(sF, a, l, TL, f0);
    ldn(sF, a + 1, l, TL, f1);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const TA diff = TA(f1[v] - f0[v]);
      tot[v] = A.first ? diff : acc[v * g.N + qi] + diff;
    }
    if (!A.last || A.defer) {
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v * g.N + qi] = tot[v];
      continue;
    }
    const double J = CART ? g.cjac : g.jac[plin(g, c[0], c[1], c[2])];
    double out[NV];
    stage_epilogue<ND, MIX, TA>(g, A, qi, J, tot, out);
  }
}

template <int ND, int DIR, bool CART, bool COMPACT, typename T, int LW, int UNIT>
__global__ void __launch_bounds__(256, sweep_min_blocks<ND, CART, T>()) k_gbr_sweep(DevGrid g, GbrCfg q, StageArgs A) {
  k_gbr_sweep_body<ND, DIR, CART, COMPACT, T, LW, UNIT>(hw_block(), g, q, A);
}

// ---------------------------------------------------------------- deferred stage update
// The mixed form's last step of an RK stage as one streaming pass, in the
// increment form of the TVD-RK3 scheme: with k_s = dt L(u^(s-1)) the stage
// increments (here -dt J times the stage total of the directions' FP32 flux
// differences summed in acc, formed in FP32),
//   u1 = un + k1,   u2 = un + (k1 + k2) / 4,   u^(n+1) = un + (k1 + k2) / 6 + 2 k3 / 3,
// which is the Shu-Osher form u2 = 3/4 un + 1/4 (u1 + k2), u^(n+1) =
// 1/3 un + 2/3 (u2 + k3) rearranged.  The increments and their running sum Z
// = k1 (+ k2) stay FP32 (the precision of the fluxes they come from); each
// stage state is un plus one widened increment, one FP64 add per variable.
// Stages 1 and 2 store no state: the primitives of u1 and u2 (the recovery
// of k_prim) go straight to Wn for the next stage, whose primitive launch is
// skipped; stage 3 writes u^(n+1) and takes the non-physical test.
template <int ND, bool CART, int STAGE>
__global__ void __launch_bounds__(256, 6) k_stage_update(DevGrid g, StageArgs A, float* __restrict__ Z,
                                                         float* __restrict__ Wn) {
  constexpr int NV = ND + 2;
  const float* acc = reinterpret_cast<const float*>(A.acc);
  const float dtf = d2f_int(*A.dt);
  constexpr int stage = STAGE;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.N;
       q += (long long)gridDim.x * blockDim.x) {
    double J;
    if (CART) {
      J = g.cjac;
    } else {
      int c[3];
      node_coords(g, q, c);
      J = g.jac[plin(g, c[0], c[1], c[2])];
    }
    const float cJ = -(dtf * d2f_int(J));
    double out[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const long long i = v * g.N + q;
      const float k = cJ * acc[i];
      float inc;
      if constexpr (stage == 1) {
        Z[i] = k;
        inc = k;
      } else if constexpr (stage == 2) {
        const float z = Z[i] + k;
        Z[i] = z;
        inc = 0.25f * z;
      } else {
        inc = (1.0f / 6.0f) * Z[i] + (2.0f / 3.0f) * k;
      }
      out[v] = A.Un[i] + f2d_int(inc);
    }
    if constexpr (stage == 3) {
#pragma unroll
      for (int v = 0; v < NV; ++v) A.Uout[v * g.N + q] = out[v];
      if (mixed_nonphysical<ND>(out)) {
        atomicOr(A.bad_flag, 1u);
        atomicMin(A.bad_idx, (unsigned long long)q);
      }
    } else {
      float w[NV];
      cons_to_prim_mixed<ND>(g.gm1, out, w);
#pragma unroll
      for (int v = 0; v < NV; ++v) Wn[v * g.N + q] = w[v];
    }
  }
}

// ---------------------------------------------------------------- CFL
// T = double: the exact FP64 rate.  T = float (mixed form): the primitives
// (pressure recovery) in FP64, the sound speed and the spectral radii in FP32.
// The rate of node q from its primitives w: J sum_l (|xi_hat_l . u| + c |xi_hat_l|).
template <int ND, bool CART, typename T>
__device__ __forceinline__ T cfl_rate(const DevGrid& g, long long q, const T* w) {
  constexpr int IP = ND + 1;
  T cs = sqrt(gconst<T>(g.gamma, g.f_gamma) * T(w[IP]) / T(w[0]));
  T s = T(0);
  T J;
  if (CART) {
    J = gconst<T>(g.cjac, g.f_cjac);
#pragma unroll
    for (int l = 0; l < ND; ++l) {
      const T xh = gconst<T>(g.cxh[l], g.f_cxh[l]);
      T t = fabs(xh * T(w[1 + l])) + cs * sqrt(xh * xh);
      s = (l == 0) ? t : s + t;
    }
  } else {
    int c[3];
    node_coords(g, q, c);
    long long pq = plin(g, c[0], c[1], c[2]);
    J = to_t<T>(g.jac[pq]);
#pragma unroll
    for (int l = 0; l < ND; ++l) {
      T dot = T(0), mag = T(0);
#pragma unroll
      for (int m = 0; m < ND; ++m) {
        T x = to_t<T>(g.xh[(l * ND + m) * g.NP + pq]);
        dot = (m == 0) ? x * T(w[1 + m]) : dot + x * T(w[1 + m]);
        mag = (m == 0) ? x * x : mag + x * x;
      }
      T t = fabs(dot) + cs * sqrt(mag);
      s = (l == 0) ? t : s + t;
    }
  }
  return J * s;
}

// Block maximum of the threads' rates, then one atomic (non-negative doubles
// order like their bits).  The running maximum is kept in T: the largest
// float converted once equals the largest of the converted floats.
template <typename T>
__device__ __forceinline__ void cfl_block_max(T best, unsigned long long* __restrict__ mx) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) best = dmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  const double bestd = double(best);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bestd;
  __syncthreads();
  if (threadIdx.x < 32) {
    double b = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) b = dmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    if (threadIdx.x == 0) atomicMax(mx, (unsigned long long)__double_as_longlong(b));
  }
}

template <int ND, bool CART, typename T = double>
__device__ __forceinline__ void k_cfl_max_body(const VBlock& vb, const DevGrid& g, const double* __restrict__ U, unsigned long long* __restrict__ mx) {
  constexpr int NV = ND + 2;
  T best = T(0);
  for (long long q = vb.x * (long long)blockDim.x + threadIdx.x; q < g.N;
       q += (long long)vb.gx * blockDim.x) {
    double Q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Q[v] = U[v * g.N + q];
    T w[NV];
    if constexpr (sizeof(T) == 4) {
      cons_to_prim_mixed<ND>(g.gm1, Q, w);
    } else {
      cons_to_prim<ND>(g.gm1, Q, w);
    }
    T r = cfl_rate<ND, CART, T>(g, q, w);
    if (r > best) best = r;
  }
  cfl_block_max<T>(best, mx);
}

// The first stage's primitives and the step's CFL maximum from one pass over
// the state: the same recovery and the same rate as k_prim and k_cfl_max, so
// the stored primitives and the step size are bitwise those of the two kernels.
template <int ND, bool CART, typename TW = double>
__global__ void k_prim_cfl(DevGrid g, const double* __restrict__ U, TW* __restrict__ W, unsigned long long* __restrict__ mx) {
  constexpr int NV = ND + 2;
  TW best = TW(0);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.N;
       q += (long long)gridDim.x * blockDim.x) {
    double Q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Q[v] = U[v * g.N + q];
    TW w[NV];
    if constexpr (sizeof(TW) == 4) {
      cons_to_prim_mixed<ND>(g.gm1, Q, w);
    } else {
      cons_to_prim<ND>(g.gm1, Q, w);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) W[v * g.N + q] = w[v];
    TW r = cfl_rate<ND, CART, TW>(g, q, w);
    if (r > best) best = r;
  }
  cfl_block_max<TW>(best, mx);
}

template <int ND, bool CART, typename T = double>
__global__ void k_cfl_max(DevGrid g, const double* __restrict__ U, unsigned long long* __restrict__ mx) {
  k_cfl_max_body<ND, CART, T>(hw_block(), g, U, mx);
}

// dt = cfl / max rate; with a final time: clip to t_end - t and advance t.
static __device__ __forceinline__ void k_cfl_finish_body(const VBlock& vb, const unsigned long long* mx, double cfl, double* dt, double* t, double t_end) {
  double m = __longlong_as_double((long long)*mx);
  double d = cfl / m;
  if (t) {
    double tt = *t;
    if (t_end > 0.0 && tt + d > t_end) d = t_end - tt;
    if (d < 0.0) d = 0.0;
    *t = tt + d;
  }
  *dt = d;
}

static __global__ void k_cfl_finish(const unsigned long long* mx, double cfl, double* dt, double* t, double t_end) {
  k_cfl_finish_body(hw_block(), mx, cfl, dt, t, t_end);
}

}  // namespace cgk
