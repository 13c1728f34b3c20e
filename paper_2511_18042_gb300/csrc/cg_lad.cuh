// LAD (Sec. 2.2): artificial bulk viscosity beta* and conductivity kappa*
// (Eq. 4-6) smoothed by the truncated-Gaussian overbar, central node fluxes
// F^c + F^v (Eq. 2-3 with mu = 0, beta = beta*, kappa = kappa*) and their
// E4 / C6 divergence; the eighth-order implicit filter of LAD-C6; the
// troubled-node flags of the hybrid (Sec. 5).
#pragma once
#include <type_traits>
#include "cg_kernels.cuh"

namespace cgk {

struct LadBuffers {
  double* fb = nullptr;     // LAD fields (u_k, T, rho, e) on fbx ([-8, n+7]^nd)
  double* gr = nullptr;     // physical gradients of the fields: nf*nd planes on b3 ([-3, n+2]^nd)
  double* dv = nullptr;     // dilatation on b3
  double* bt[2] = {nullptr, nullptr};  // beta* (ping-pong, interior)
  double* kp[2] = {nullptr, nullptr};  // kappa*
  double* Fn = nullptr;     // node fluxes: nv planes on fbox (positions [-2, n+1]) per direction,
                            // every direction's held at once (slices fstride apart)
  double* D = nullptr;      // C6 flux derivatives, one line buffer DLB per direction
  Box ubx{};                // [-2, n+1] in every direction: the union of the node-flux boxes
  size_t fstride = 0;       // values between the directions' node-flux slices of Fn
  size_t dstride = 0;       // values between the directions' slices of D
  double* df[3] = {nullptr, nullptr, nullptr};  // C6 computational derivatives of the fields (line buffers)
  double* lines = nullptr;  // right-hand sides / solutions of the filter lines
  double* vco = nullptr;    // physical viscosity: mu, lambda, kappa at the nodes of vbx (3 planes)
  Box vbx;                  // [-2, n+1]^nd: every node a node flux is taken at
  unsigned char* tr = nullptr;  // hybrid: troubled nodes on tbox ([-1, n]^nd)
  Box fbx, b3, tbox, fbox[3], hbox[3];
  LineBuf dfLB[3], DLB[3], filtLB[3];
};

// fields differentiated by LAD: velocities, T = gamma M^2 p / rho, rho, e = p / (rho (gamma-1))
// (T = double: FP64 parity form; T = float: mixed form, fields, gradients,
// coefficients and fluxes in FP32 from FP64 primitives)
template <int ND, typename T = double>
__device__ __forceinline__ void lad_fields(const DevGrid& g, const T* w, T* f) {
  constexpr int IP = ND + 1;
  T rho = w[0], p = w[IP];
#pragma unroll
  for (int k = 0; k < ND; ++k) f[k] = w[1 + k];
  f[ND] = gconst<T>(g.gm2, g.f_gm2) * p / rho;
  f[ND + 1] = rho;
  f[ND + 2] = p / (rho * gconst<T>(g.gm1, g.f_gm1));
}

__device__ __forceinline__ void box_coords(const Box& b, long long e, int* c) {
  if (b.size() <= 0x7fffffffLL) {  // 32-bit division, as node_coords
    const unsigned r = (unsigned)e, x0 = (unsigned)b.ext[0], x1 = (unsigned)b.ext[1];
    const unsigned t = r / x0;
    c[0] = (int)(r - t * x0) - b.off[0];
    c[1] = (int)(t % x1) - b.off[1];
    c[2] = (int)(t / x1) - b.off[2];
    return;
  }
  c[0] = (int)(e % b.ext[0]) - b.off[0];
  long long r = e / b.ext[0];
  c[1] = (int)(r % b.ext[1]) - b.off[1];
  c[2] = (int)(r / b.ext[1]) - b.off[2];
}

// grid-stride loop over a box (in a kernel body: vb is the block's coordinates)
#define BOX_LOOP(b, e) \
  for (long long e = vb.x * (long long)blockDim.x + threadIdx.x; e < (b).size(); e += (long long)vb.gx * blockDim.x)

// the LAD fields at every node of the box fbx (ghosts by the boundary rule)
template <int ND, typename T = double>
__device__ __forceinline__ void k_lad_fieldbuf_body(const VBlock& vb, const DevGrid& g, const T* __restrict__ W, T* __restrict__ f, Box fbx) {
  constexpr int NV = ND + 2, NF = ND + 3;
  long long fs = fbx.size();
  BOX_LOOP(fbx, e) {
    int c[3];
    box_coords(fbx, e, c);
    T w[NV], fl[NF];
    load_state<ND, false, T, T>(g, W, c[0], c[1], c[2], w);
    lad_fields<ND, T>(g, w, fl);
#pragma unroll
    for (int v = 0; v < NF; ++v) f[v * fs + e] = fl[v];
  }
}

template <int ND, typename T = double>
__global__ void k_lad_fieldbuf(DevGrid g, const T* __restrict__ W, T* __restrict__ f, Box fbx) {
  k_lad_fieldbuf_body<ND, T>(hw_block(), g, W, f, fbx);
}

// Physical gradients and dilatation at node c (index e of b3) from the
// index-space derivatives d[l][f] = d f / d xi_l.
template <int ND, bool CART, typename T>
__device__ __forceinline__ void lad_grad_out(const DevGrid& g, const int* c, long long e, long long bs,
                                             const T (&d)[3][ND + 3], T* __restrict__ gr, T* __restrict__ dv) {
  constexpr int NF = ND + 3;
  T div = T(0);
  if (CART) {
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int m = 0; m < ND; ++m) {
        T v = gconst<T>(g.cjxh[m], g.f_cjxh[m]) * d[m][f];
        gr[(f * ND + m) * bs + e] = v;
        if (f < ND && m == f) div = (f == 0) ? v : div + v;
      }
  } else {
    long long pq = plin(g, c[0], c[1], c[2]);
    double J = g.jac[pq];
    T xm[3][3];
#pragma unroll
    for (int l = 0; l < ND; ++l)
#pragma unroll
      for (int m = 0; m < ND; ++m) xm[l][m] = to_t<T>(J * g.xh[(l * ND + m) * g.NP + pq]);
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int m = 0; m < ND; ++m) {
        T sm = xm[0][m] * d[0][f];
#pragma unroll
        for (int l = 1; l < ND; ++l) sm = sm + xm[l][m] * d[l][f];
        gr[(f * ND + m) * bs + e] = sm;
        if (f < ND && m == f) div = (f == 0) ? sm : div + sm;
      }
  }
  dv[e] = div;
}

// Physical gradients and dilatation on b3.  E4 differences the field buffer;
// C6 reads the compact derivatives from the line buffers df.
template <int ND, bool CART, bool C6, typename T = double>
__device__ __forceinline__ void k_lad_grad_body(const VBlock& vb, const DevGrid& g, const T* __restrict__ fb, Box fbx, const T* __restrict__ df0,
                           const T* __restrict__ df1, const T* __restrict__ df2, LineBuf lb0, LineBuf lb1,
                           LineBuf lb2, T* __restrict__ gr, T* __restrict__ dv, Box b3, const int* guard,
                           int want) {
  constexpr int NF = ND + 3;
  if (guard && *guard != want) return;
  long long bs = b3.size(), fs = fbx.size();
  BOX_LOOP(b3, e) {
    int c[3];
    box_coords(b3, e, c);
    T d[3][NF];  // d[l][f] = d f / d xi_l
    long long q = fbx.at(c[0], c[1], c[2]);
#pragma unroll
    for (int l = 0; l < ND; ++l) {
      if (C6) {
        const T* df = l == 0 ? df0 : (l == 1 ? df1 : df2);
        const LineBuf& lb = l == 0 ? lb0 : (l == 1 ? lb1 : lb2);
#pragma unroll
        for (int f = 0; f < NF; ++f) d[l][f] = T(df[lb.at(f, c[l], c)]);
      } else {
        long long st = l == 0 ? 1 : (l == 1 ? (long long)fbx.ext[0] : (long long)fbx.ext[0] * fbx.ext[1]);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const T* p = fb + f * fs + q;
          d[l][f] = d4(p[-2 * st], p[-st], p[st], p[2 * st]);
        }
      }
    }
    lad_grad_out<ND, CART, T>(g, c, e, bs, d, gr, dv);
  }
}

// The C6 form of k_lad_grad in 2D and 3D on tiles of 32 (x) x 8 (y) nodes of
// b3, one z plane per block.  The x-line buffer holds a line's positions a
// line count apart, so reading it node by node along x would touch one
// sector per value; the tile stages its x derivatives with consecutive
// threads on consecutive lines (consecutive y), then reads them from shared
// memory.  The y and z buffers are read directly (consecutive x are
// consecutive lines there).  Same values and arithmetic as k_lad_grad.
constexpr int LGT_X = 32, LGT_Y = 8;
template <int ND, bool CART, typename T>
__global__ void __launch_bounds__(LGT_X * LGT_Y) k_lad_grad_xt(DevGrid g, const T* __restrict__ df0, const T* __restrict__ df1,
                                                             const T* __restrict__ df2, LineBuf lb0, LineBuf lb1,
                                                             LineBuf lb2, T* __restrict__ gr, T* __restrict__ dv, Box b3,
                                                             const int* guard, int want) {
  static_assert(ND >= 2, "tiles of x and y");
  constexpr int NF = ND + 3;
  __shared__ T sD[NF][LGT_Y][LGT_X + 1];
  if (guard && *guard != want) return;
  const int bx0 = (int)blockIdx.x * LGT_X, by0 = (int)blockIdx.y * LGT_Y;
  const int cz = ND == 3 ? (int)blockIdx.z - b3.off[2] : 0;
  const int tid = threadIdx.y * LGT_X + threadIdx.x;
  {
    const int ly = tid % LGT_Y, lx = tid / LGT_Y;  // consecutive threads: consecutive lines
    if (bx0 + lx < b3.ext[0] && by0 + ly < b3.ext[1]) {
      int c[3] = {bx0 + lx - b3.off[0], by0 + ly - b3.off[1], cz};
#pragma unroll
      for (int f = 0; f < NF; ++f) sD[f][ly][lx] = df0[lb0.at(f, c[0], c)];
    }
  }
  __syncthreads();
  const int ex = bx0 + (int)threadIdx.x, ey = by0 + (int)threadIdx.y;
  if (ex >= b3.ext[0] || ey >= b3.ext[1]) return;
  int c[3] = {ex - b3.off[0], ey - b3.off[1], cz};
  T d[3][NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    d[0][f] = sD[f][threadIdx.y][threadIdx.x];
    d[1][f] = df1[lb1.at(f, c[1], c)];
    if (ND == 3) d[2][f] = df2[lb2.at(f, c[2], c)];
  }
  lad_grad_out<ND, CART, T>(g, c, b3.at(c[0], c[1], c[2]), b3.size(), d, gr, dv);
}

template <int ND, bool CART, bool C6, typename T = double>
__global__ void k_lad_grad(DevGrid g, const T* __restrict__ fb, Box fbx, const T* __restrict__ df0,
                           const T* __restrict__ df1, const T* __restrict__ df2, LineBuf lb0, LineBuf lb1,
                           LineBuf lb2, T* __restrict__ gr, T* __restrict__ dv, Box b3, const int* guard,
                           int want) {
  k_lad_grad_body<ND, CART, C6, T>(hw_block(), g, fb, fbx, df0, df1, df2, lb0, lb1, lb2, gr, dv, b3, guard, want);
}

// Euclidean norm of an FP32 gradient (ND components), overflow- and
// underflow-safe through the CUDA library's hypot forms.
template <int ND>
__device__ __forceinline__ float grad_norm(float a, float b, float c) {
  if constexpr (ND == 1) return fabsf(a);
  else if constexpr (ND == 2) return hypotf(a, b);
  else return norm3df(a, b, c);
}

// Raw coefficients at interior nodes, Eq. (4)-(6):
// beta* = C_beta rho f_sw |sum_l d4(div)_l Delta_{l,beta}^2|,
// kappa* = C_kappa (rho c / T) |sum_l d4(e)_l Delta_{l,kappa}|.
template <int ND, bool CART, typename T = double>
__device__ __forceinline__ void k_lad_coef_body(const VBlock& vb, const DevGrid& g, const T* __restrict__ W, const T* __restrict__ fb, Box fbx,
                           const T* __restrict__ gr, const T* __restrict__ dv, Box b3, double c_beta_d,
                           double c_kappa_d, T* __restrict__ bt, T* __restrict__ kp, const int* guard, int want) {
  const T c_beta = T(c_beta_d), c_kappa = T(c_kappa_d);
  constexpr int NV = ND + 2, IP = ND + 1;
  if (guard && *guard != want) return;
  long long bs = b3.size(), fs = fbx.size();
  for (long long q = vb.x * (long long)blockDim.x + threadIdx.x; q < g.N; q += (long long)vb.gx * blockDim.x) {
    int c[3];
    node_coords(g, q, c);
    long long e0 = b3.at(c[0], c[1], c[2]);
    T w[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = T(W[v * g.N + q]);
    T rho = w[0], p = w[IP];
    long long fq = fbx.at(c[0], c[1], c[2]);
    T Tt = fb[ND * fs + fq];
    T cs = sqrt(gconst<T>(g.gamma, g.f_gamma) * p / rho);
    T div = dv[e0];
    T curl2 = T(0);
    auto G = [&](int f, int m) { return gr[(f * ND + m) * bs + e0]; };
    if (ND == 2) {
      T w3 = G(1, 0) - G(0, 1);
      curl2 = w3 * w3;
    } else if (ND == 3) {
      T w1 = G(2, 1) - G(1, 2), w2 = G(0, 2) - G(2, 0), w3 = G(1, 0) - G(0, 1);
      curl2 = w1 * w1 + w2 * w2 + w3 * w3;
    }
    // The switch of Eq. (4) is zero where the flow expands (div >= 0): there
    // beta* is +0 whatever its other factors, so the switch's ratio, |grad rho|
    // and the spacings Delta_beta (divisions and a square root, on the FP64
    // pipe) are formed only where div < 0, each as in the full product.
    const bool comp = div < T(0);
    T fsw = T(0), gmr = T(0), gme;
    if (comp) fsw = (div * div) / (div * div + curl2 + T(1e-32));
    if constexpr (sizeof(T) == 4) {
      // |grad rho| and |grad e| without squaring: in FP32 a square under
      // ~1e-38 flushes, and |x . grad| / (0 + 1e-32) would then inflate the
      // length scales Delta_beta, Delta_kappa far beyond the grid spacing
      if (comp) gmr = grad_norm<ND>(G(ND + 1, 0), G(ND + 1, ND > 1 ? 1 : 0), G(ND + 1, ND > 2 ? 2 : 0));
      gme = grad_norm<ND>(G(ND + 2, 0), G(ND + 2, ND > 1 ? 1 : 0), G(ND + 2, ND > 2 ? 2 : 0));
    } else {
      gme = G(ND + 2, 0) * G(ND + 2, 0);
#pragma unroll
      for (int m = 1; m < ND; ++m) gme = gme + G(ND + 2, m) * G(ND + 2, m);
      gme = sqrt(gme);
      if (comp) {
        gmr = G(ND + 1, 0) * G(ND + 1, 0);
#pragma unroll
        for (int m = 1; m < ND; ++m) gmr = gmr + G(ND + 1, m) * G(ND + 1, m);
        gmr = sqrt(gmr);
      }
    }
    T sb = T(0), sk = T(0);
#pragma unroll
    for (int l = 0; l < ND; ++l) {
      long long st = l == 0 ? 1 : (l == 1 ? (long long)b3.ext[0] : (long long)b3.ext[0] * b3.ext[1]);
      long long fst = l == 0 ? 1 : (l == 1 ? (long long)fbx.ext[0] : (long long)fbx.ext[0] * fbx.ext[1]);
      const T* ev = fb + (ND + 2) * fs + fq;
      T d4e = (ev[-2 * fst] + ev[2 * fst]) - T(4.0) * (ev[-fst] + ev[fst]) + T(6.0) * ev[0];
      // projections x_l . grad of rho (pr) and e (pe), x_l = dx/dxi_l
      T pr = T(0), pe;
      if (CART) {
        if (comp) pr = gconst<T>(g.ch[l], g.f_ch[l]) * G(ND + 1, l);
        pe = gconst<T>(g.ch[l], g.f_ch[l]) * G(ND + 2, l);
      } else {
        long long pq = plin(g, c[0], c[1], c[2]);
        pe = to_t<T>(g.dxl[(l * ND + 0) * g.NP + pq]) * G(ND + 2, 0);
#pragma unroll
        for (int m = 1; m < ND; ++m) pe = pe + to_t<T>(g.dxl[(l * ND + m) * g.NP + pq]) * G(ND + 2, m);
        if (comp) {
          pr = to_t<T>(g.dxl[(l * ND + 0) * g.NP + pq]) * G(ND + 1, 0);
#pragma unroll
          for (int m = 1; m < ND; ++m) pr = pr + to_t<T>(g.dxl[(l * ND + m) * g.NP + pq]) * G(ND + 1, m);
        }
      }
      T Dk = fabs(pe) / (gme + T(1e-32));
      T tk = d4e * Dk;
      sk = (l == 0) ? tk : sk + tk;
      if (comp) {
        T d4d = (dv[e0 - 2 * st] + dv[e0 + 2 * st]) - T(4.0) * (dv[e0 - st] + dv[e0 + st]) + T(6.0) * div;
        T Db = fabs(pr) / (gmr + T(1e-32));
        T tb = d4d * Db * Db;
        sb = (l == 0) ? tb : sb + tb;
      }
    }
    bt[q] = c_beta * rho * fsw * fabs(sb);
    kp[q] = c_kappa * (rho * cs / Tt) * fabs(sk);
  }
}

template <int ND, bool CART, typename T = double>
__global__ void k_lad_coef(DevGrid g, const T* __restrict__ W, const T* __restrict__ fb, Box fbx,
                           const T* __restrict__ gr, const T* __restrict__ dv, Box b3, double c_beta_d,
                           double c_kappa_d, T* __restrict__ bt, T* __restrict__ kp, const int* guard, int want) {
  k_lad_coef_body<ND, CART, T>(hw_block(), g, W, fb, fbx, gr, dv, b3, c_beta_d, c_kappa_d, bt, kp, guard, want);
}

// truncated-Gaussian overbar along l (nine points, Cook & Cabot), two fields;
// ghost values: periodic wrap, wall mirror, otherwise the boundary node.
template <int ND, typename T = double>
__device__ __forceinline__ void k_gauss_body(const VBlock& vb, const DevGrid& g, int l, const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ ao,
                        T* __restrict__ bo, const int* guard, int want) {
  if (guard && *guard != want) return;
  const T A0 = T(3565.0 / 10368.0), A1 = T(3091.0 / 12960.0), A2 = T(1997.0 / 25920.0), A3 = T(149.0 / 12960.0),
          A4 = T(107.0 / 103680.0);
  for (long long q = vb.x * (long long)blockDim.x + threadIdx.x; q < g.N; q += (long long)vb.gx * blockDim.x) {
    int c[3];
    node_coords(g, q, c);
    long long s[9];
    if (c[l] >= 4 && c[l] < g.n[l] - 4) {  // interior stencil: the nodes themselves
      const long long st = l == 0 ? 1 : (l == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1]);
#pragma unroll
      for (int t = -4; t <= 4; ++t) s[t + 4] = q + t * st;
    } else {
#pragma unroll
      for (int t = -4; t <= 4; ++t) {
        int cc[3] = {c[0], c[1], c[2]};
        cc[l] += t;
        s[t + 4] = scalar_src(g, cc[0], cc[1], cc[2]);
      }
    }
    ao[q] = A0 * a[s[4]] + A1 * (a[s[3]] + a[s[5]]) + A2 * (a[s[2]] + a[s[6]]) + A3 * (a[s[1]] + a[s[7]]) +
            A4 * (a[s[0]] + a[s[8]]);
    bo[q] = A0 * b[s[4]] + A1 * (b[s[3]] + b[s[5]]) + A2 * (b[s[2]] + b[s[6]]) + A3 * (b[s[1]] + b[s[7]]) +
            A4 * (b[s[0]] + b[s[8]]);
  }
}

template <int ND, typename T = double>
__global__ void k_gauss(DevGrid g, int l, const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ ao,
                        T* __restrict__ bo, const int* guard, int want) {
  k_gauss_body<ND, T>(hw_block(), g, l, a, b, ao, bo, guard, want);
}

// Node fluxes along l at positions [-2, n+1] (interior lines).
// MODE 0 (LAD, inviscid case): F = F^c(W; xi_hat_l) - [0, xi_hat_l tau,
//   xi_hat_l . phi], tau = beta* div, phi_m = u_m tau + kappa* dT/dx_m.
// MODE 1 (LAD with physical viscosity) and MODE 2 (the physical viscous flux
// alone, -F^v): Eq. (3) with Stokes' hypothesis,
//   tau_ma = mu (du_a/dx_m + du_m/dx_a) + delta_ma (beta* - 2/3 mu) div,
//   phi_m = sum_a u_a tau_ma + (kappa* + kappa_hat) dT/dx_m,
//   mu = T^{3/2} (1 + S) / (T + S) / Re, kappa_hat = mu / ((gamma-1) Pr M^2)
// (MODE 2: no convective flux, beta* = kappa* = 0).
constexpr int NF_LAD = 0, NF_LAD_VISC = 1, NF_VISC = 2;

// node flux along l at node c (the body of k_lad_nodeflux; F: nv values)
template <int ND, bool CART, int MODE, typename T>
__device__ __forceinline__ void nodeflux_at(const DevGrid& g, int l, const T* __restrict__ W, const T* __restrict__ bt,
                                            const T* __restrict__ kp, const T* __restrict__ gr,
                                            const T* __restrict__ dv, const Box& b3, const T* __restrict__ vco,
                                            const Box& vbx, const int* c, T* F) {
  constexpr int NV = ND + 2, IP = ND + 1;
  constexpr bool CONV = MODE != NF_VISC, PHYS = MODE != NF_LAD;
  const long long bs = b3.size();
  {
    T w[NV];
    load_state<ND, false, T, T>(g, W, c[0], c[1], c[2], w);
    T xi[3];
    if (CART) {
#pragma unroll
      for (int m = 0; m < ND; ++m) xi[m] = (m == l) ? gconst<T>(g.cxh[l], g.f_cxh[l]) : T(0);
    } else {
      long long pq = plin(g, c[0], c[1], c[2]);
#pragma unroll
      for (int m = 0; m < ND; ++m) xi[m] = to_t<T>(g.xh[(l * ND + m) * g.NP + pq]);
    }
    T rho = w[0], p = w[IP];
    T fc[NV];
    if (CONV) {
      T U, q2;
      if (CART) U = xi[l] * w[1 + l];
      else {
        U = xi[0] * w[1];
#pragma unroll
        for (int m = 1; m < ND; ++m) U = U + xi[m] * w[1 + m];
      }
      q2 = w[1] * w[1];
#pragma unroll
      for (int m = 1; m < ND; ++m) q2 = q2 + w[1 + m] * w[1 + m];
      T E = p / gconst<T>(g.gm1, g.f_gm1) + T(0.5) * rho * q2;
      fc[0] = rho * U;
#pragma unroll
      for (int m = 0; m < ND; ++m) fc[1 + m] = (CART && m != l) ? rho * w[1 + m] * U : rho * w[1 + m] * U + xi[m] * p;
      fc[IP] = (E + p) * U;
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) fc[v] = T(0);
    }
    long long sq = scalar_src(g, c[0], c[1], c[2]);
    long long be = b3.at(c[0], c[1], c[2]);
    if (!PHYS) {
      T tau = bt[sq] * dv[be];
      T kap = kp[sq];
      T fe = T(0);
      bool first = true;
#pragma unroll
      for (int m = 0; m < ND; ++m) {
        if (CART && m != l) continue;
        T phi = w[1 + m] * tau + kap * gr[(ND * ND + m) * bs + be];
        fe = first ? xi[m] * phi : fe + xi[m] * phi;
        first = false;
      }
      F[0] = fc[0];
#pragma unroll
      for (int m = 0; m < ND; ++m) F[1 + m] = (CART && m != l) ? fc[1 + m] : fc[1 + m] - xi[m] * tau;
      F[IP] = fc[IP] - fe;
    } else {
      // mu, lambda = beta* - 2/3 mu and kappa* + mu / ((gamma-1) Pr M^2) of
      // the node, formed once per stage by k_lad_viscoef
      const long long vq = vbx.at(c[0], c[1], c[2]), vs = vbx.size();
      T mu = vco[vq];
      T lam = vco[vs + vq];
      T kap = vco[2 * vs + vq];
      T div = dv[be];
      T tau[ND][ND];
#pragma unroll
      for (int m = 0; m < ND; ++m)
#pragma unroll
        for (int a = 0; a < ND; ++a) {
          T sm = gr[(a * ND + m) * bs + be] + gr[(m * ND + a) * bs + be];
          tau[m][a] = mu * sm;
          if (m == a) tau[m][a] = tau[m][a] + lam * div;
        }
      T fe = T(0);
      bool first = true;
#pragma unroll
      for (int m = 0; m < ND; ++m) {
        if (CART && m != l) continue;
        T phi = w[1] * tau[m][0];
#pragma unroll
        for (int a = 1; a < ND; ++a) phi = phi + w[1 + a] * tau[m][a];
        phi = phi + kap * gr[(ND * ND + m) * bs + be];
        fe = first ? xi[m] * phi : fe + xi[m] * phi;
        first = false;
      }
      F[0] = fc[0];
#pragma unroll
      for (int a = 0; a < ND; ++a) {
        T fv;
        if (CART) fv = xi[l] * tau[l][a];
        else {
          fv = xi[0] * tau[0][a];
#pragma unroll
          for (int m = 1; m < ND; ++m) fv = fv + xi[m] * tau[m][a];
        }
        F[1 + a] = fc[1 + a] + (-fv);
      }
      F[IP] = fc[IP] + (-fe);
    }
  }
}

template <int ND, bool CART, int MODE, typename T = double>
__device__ __forceinline__ void k_lad_nodeflux_body(const VBlock& vb, const DevGrid& g, int l, const T* __restrict__ W, const T* __restrict__ bt,
                               const T* __restrict__ kp, const T* __restrict__ gr, const T* __restrict__ dv, Box b3,
                               const T* __restrict__ vco, Box vbx, T* __restrict__ Fn, Box fb, const int* guard,
                               int want) {
  constexpr int NV = ND + 2;
  if (guard && *guard != want) return;
  long long fs = fb.size();
  BOX_LOOP(fb, e) {
    int c[3];
    box_coords(fb, e, c);
    T F[NV];
    nodeflux_at<ND, CART, MODE, T>(g, l, W, bt, kp, gr, dv, b3, vco, vbx, c, F);
#pragma unroll
    for (int v = 0; v < NV; ++v) Fn[v * fs + e] = F[v];
  }
}

// The node fluxes of every direction in one pass over ub (the union of the
// directions' boxes, positions [-2, n+1] in every direction): each node forms
// all directions' fluxes (the loads they share, issued once) and stores those
// whose box holds it; the values are those of k_lad_nodeflux.
__device__ __forceinline__ bool box_holds(const Box& b, const int* c) {
  return c[0] + b.off[0] >= 0 && c[0] + b.off[0] < b.ext[0] && c[1] + b.off[1] >= 0 && c[1] + b.off[1] < b.ext[1] &&
         c[2] + b.off[2] >= 0 && c[2] + b.off[2] < b.ext[2];
}

template <int ND, bool CART, int MODE, typename T>
__global__ void k_lad_nodeflux_all(DevGrid g, const T* __restrict__ W, const T* __restrict__ bt,
                                   const T* __restrict__ kp, const T* __restrict__ gr, const T* __restrict__ dv, Box b3,
                                   const T* __restrict__ vco, Box vbx, T* __restrict__ F0, Box fb0, T* __restrict__ F1,
                                   Box fb1, T* __restrict__ F2, Box fb2, Box ub, const int* guard, int want) {
  constexpr int NV = ND + 2;
  if (guard && *guard != want) return;
  const VBlock vb = hw_block();
  BOX_LOOP(ub, e) {
    int c[3];
    box_coords(ub, e, c);
    T F[3][NV];
#pragma unroll
    for (int l = 0; l < ND; ++l) nodeflux_at<ND, CART, MODE, T>(g, l, W, bt, kp, gr, dv, b3, vco, vbx, c, F[l]);
#pragma unroll
    for (int l = 0; l < ND; ++l) {
      const Box& fb = l == 0 ? fb0 : (l == 1 ? fb1 : fb2);
      T* Fo = l == 0 ? F0 : (l == 1 ? F1 : F2);
      if (!box_holds(fb, c)) continue;
      const long long fs = fb.size(), q = fb.at(c[0], c[1], c[2]);
#pragma unroll
      for (int v = 0; v < NV; ++v) Fo[v * fs + q] = F[l][v];
    }
  }
}

template <int ND, bool CART, int MODE, typename T = double>
__global__ void k_lad_nodeflux(DevGrid g, int l, const T* __restrict__ W, const T* __restrict__ bt,
                               const T* __restrict__ kp, const T* __restrict__ gr, const T* __restrict__ dv, Box b3,
                               const T* __restrict__ vco, Box vbx, T* __restrict__ Fn, Box fb, const int* guard,
                               int want) {
  k_lad_nodeflux_body<ND, CART, MODE, T>(hw_block(), g, l, W, bt, kp, gr, dv, b3, vco, vbx, Fn, fb, guard, want);
}

// Physical viscosity of Eq. (3) with Sutherland's law at every node of vbx,
// for the node fluxes of all directions: mu, lambda = beta* - 2/3 mu (beta*
// added when ART, the LAD scheme with physical viscosity) and the
// conductivity kappa* + mu / ((gamma-1) Pr M^2), each formed as the node
// fluxes formed them.
template <int ND, bool ART, typename T = double>
__device__ __forceinline__ void k_lad_viscoef_body(const VBlock& vb, const DevGrid& g, const T* __restrict__ W,
                                                   const T* __restrict__ bt, const T* __restrict__ kp,
                                                   T* __restrict__ vco, Box vbx, const int* guard, int want) {
  constexpr int NV = ND + 2, IP = ND + 1;
  if (guard && *guard != want) return;
  const long long vs = vbx.size();
  BOX_LOOP(vbx, e) {
    int c[3];
    box_coords(vbx, e, c);
    T w[NV];
    load_state<ND, false, T, T>(g, W, c[0], c[1], c[2], w);
    T rho = w[0], p = w[IP];
    long long sq = scalar_src(g, c[0], c[1], c[2]);
    T Tt = T(g.gm2) * p / rho;
    T S = T(g.suth);
    T mu = Tt * sqrt(Tt) * (T(1.0) + S) / (Tt + S) / T(g.re);
    T kth = mu / T(g.kc);
    T lam = (ART ? bt[sq] : T(0)) - T(2.0 / 3.0) * mu;
    T kap = (ART ? kp[sq] : T(0)) + kth;
    vco[e] = mu;
    vco[vs + e] = lam;
    vco[2 * vs + e] = kap;
  }
}

template <int ND, bool ART, typename T = double>
__global__ void k_lad_viscoef(DevGrid g, const T* __restrict__ W, const T* __restrict__ bt, const T* __restrict__ kp,
                              T* __restrict__ vco, Box vbx, const int* guard, int want) {
  k_lad_viscoef_body<ND, ART, T>(hw_block(), g, W, bt, kp, vco, vbx, guard, want);
}

// Stage epilogue shared by the LAD divergence kernels: tot = acc + D (or D),
// then store acc, R = -J tot, or the RK combination.
// FUSED (mixed form): stage_epilogue's mixed update; otherwise the oracle's
// operation order.  FUSED also sums the directions' flux differences in FP32:
// acc then holds FP32 values (the buffer read as float), and only the stage
// total enters the FP64 residual and update.
template <int ND, bool FUSED = false, typename TD = double>
__device__ __forceinline__ void lad_epilogue(const DevGrid& g, const StageArgs& A, long long qi, const int* c,
                                             const TD* Dv) {
  constexpr int NV = ND + 2;
  static_assert(FUSED || sizeof(TD) == 8, "the FP64 form accumulates in FP64");
  using TA = typename std::conditional<FUSED, float, double>::type;
  TA* acc = reinterpret_cast<TA*>(A.acc);
  TA tot[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) tot[v] = A.first ? TA(Dv[v]) : acc[v * g.N + qi] + TA(Dv[v]);
  if (!A.last || A.defer) {
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v * g.N + qi] = tot[v];
    return;
  }
  const double J = g.curv ? g.jac[plin(g, c[0], c[1], c[2])] : g.cjac;
  double out[NV];
  stage_epilogue<ND, FUSED, TA>(g, A, qi, J, tot, out);
}

// E4 divergence of the node fluxes along l (explicit) or the compact result D.
template <int ND, typename T = double>
__global__ void k_lad_div(DevGrid g, int l, const T* __restrict__ Fn, Box fb, const T* __restrict__ D,
                          LineBuf DL, StageArgs A, const int* guard, int want) {
  constexpr int NV = ND + 2;
  if (guard && *guard != want) return;
  long long fs = fb.size();
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.N; q += (long long)gridDim.x * blockDim.x) {
    int c[3];
    node_coords(g, q, c);
    T Dv[NV];
    if (D) {
#pragma unroll
      for (int v = 0; v < NV; ++v) Dv[v] = D[DL.at(v, c[l], c)];
    } else {
      long long e = fb.at(c[0], c[1], c[2]);
      long long st = l == 0 ? 1 : (l == 1 ? (long long)fb.ext[0] : (long long)fb.ext[0] * fb.ext[1]);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T* f = Fn + v * fs;
        Dv[v] = d4(f[e - 2 * st], f[e - st], f[e + st], f[e + 2 * st]);
      }
    }
    lad_epilogue<ND, sizeof(T) == 4, T>(g, A, q, c, Dv);
  }
}

// The C6 divergence along x (D from the x-line buffer) on tiles of 32 (x) x
// 8 lines: the tile's D values are staged with consecutive threads on
// consecutive lines, then each thread takes one node, as k_lad_div.
template <int ND, typename T>
__global__ void __launch_bounds__(LGT_X * LGT_Y) k_lad_div_xt(DevGrid g, const T* __restrict__ D, LineBuf DL, StageArgs A,
                                                            const int* guard, int want) {
  constexpr int NV = ND + 2;
  __shared__ T sD[NV][LGT_Y][LGT_X + 1];
  if (guard && *guard != want) return;
  const int x0 = (int)blockIdx.x * LGT_X;
  const long long L0 = (long long)blockIdx.y * LGT_Y + (long long)blockIdx.z * gridDim.y * LGT_Y;
  const int tid = threadIdx.y * LGT_X + threadIdx.x;
  {
    const int ly = tid % LGT_Y, lx = tid / LGT_Y;
    if (x0 + lx < g.n[0] && L0 + ly < DL.nl) {
      int c[3] = {0, 0, 0};
      DL.coords(L0 + ly, c);
#pragma unroll
      for (int v = 0; v < NV; ++v) sD[v][ly][lx] = D[DL.at(v, x0 + lx, c)];
    }
  }
  __syncthreads();
  const int x = x0 + (int)threadIdx.x;
  const long long L = L0 + threadIdx.y;
  if (x >= g.n[0] || L >= DL.nl) return;
  int c[3] = {0, 0, 0};
  DL.coords(L, c);
  c[0] = x;
  T Dv[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Dv[v] = sD[v][threadIdx.y][threadIdx.x];
  lad_epilogue<ND, sizeof(T) == 4, T>(g, A, lin(g, c[0], c[1], c[2]), c, Dv);
}

// The C6 divergences of all directions in one pass on the tiles of
// k_lad_div_xt: the x derivatives staged through shared memory, the y (and z)
// derivatives read directly, summed in the order of the per-direction
// launches (x, then y, then z, in the accumulator's type), then one epilogue.
template <int ND, typename T>
__global__ void __launch_bounds__(LGT_X * LGT_Y) k_lad_div_all_xt(DevGrid g, const T* __restrict__ D0, LineBuf DL0,
                                                                const T* __restrict__ D1, LineBuf DL1,
                                                                const T* __restrict__ D2, LineBuf DL2, StageArgs A,
                                                                const int* guard, int want) {
  constexpr int NV = ND + 2;
  using TA = typename std::conditional<sizeof(T) == 4, float, double>::type;
  __shared__ T sD[NV][LGT_Y][LGT_X + 1];
  if (guard && *guard != want) return;
  const int x0 = (int)blockIdx.x * LGT_X;
  const long long L0 = (long long)blockIdx.y * LGT_Y + (long long)blockIdx.z * gridDim.y * LGT_Y;
  const int tid = threadIdx.y * LGT_X + threadIdx.x;
  {
    const int ly = tid % LGT_Y, lx = tid / LGT_Y;
    if (x0 + lx < g.n[0] && L0 + ly < DL0.nl) {
      int c[3] = {0, 0, 0};
      DL0.coords(L0 + ly, c);
#pragma unroll
      for (int v = 0; v < NV; ++v) sD[v][ly][lx] = D0[DL0.at(v, x0 + lx, c)];
    }
  }
  __syncthreads();
  const int x = x0 + (int)threadIdx.x;
  const long long L = L0 + threadIdx.y;
  if (x >= g.n[0] || L >= DL0.nl) return;
  int c[3] = {0, 0, 0};
  DL0.coords(L, c);
  c[0] = x;
  T Dv[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    TA t = TA(sD[v][threadIdx.y][threadIdx.x]);
    t = t + TA(D1[DL1.at(v, c[1], c)]);
    if (ND == 3) t = t + TA(D2[DL2.at(v, c[2], c)]);
    Dv[v] = T(t);
  }
  StageArgs B = A;
  B.first = 1;
  B.last = 1;
  lad_epilogue<ND, sizeof(T) == 4, T>(g, B, lin(g, c[0], c[1], c[2]), c, Dv);
}

// Troubled-node criterion of Sec. 5 at node (x, y, z) (ghost-resolved):
// rho < hyb_rho or p < hyb_p, or (with the sensor) Omega > threshold.
// The criterion's thresholds in the stored type TW.  For FP32 storage they are
// rounded outward (rho, p: up; Omega: down), so that for every float w,
// w < hr holds exactly when w < hr_f and om > thr exactly when om > thr_f:
// the FP32 comparisons take the FP64 decisions, without widening each
// neighbour's state on the FP64 pipe.
template <typename TW>
struct TroubleThr {
  TW hr, hp, thr;
  TroubleThr() = default;
  __device__ explicit TroubleThr(double r, double p, double t) {
    if constexpr (sizeof(TW) == 4) {
      hr = f32_up(r);
      hp = f32_up(p);
      thr = f32_down(t);
    } else {
      hr = r;
      hp = p;
      thr = t;
    }
  }
  __device__ static float f32_up(double x) {
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
  }
  __device__ static float f32_down(double x) {
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return f;
  }
};

template <int ND, typename TW>
__device__ __forceinline__ bool troubled_at(const DevGrid& g, const TW* __restrict__ W, const TroubleThr<TW>& th,
                                            const TW* __restrict__ om, const Box& ob, int x, int y, int z) {
  constexpr int NV = ND + 2, IP = ND + 1;
  TW w[NV];
  load_state<ND, false, TW, TW>(g, W, x, y, z, w);
  bool t = w[0] < th.hr || w[IP] < th.hp;
  if (om && om[ob.at(x, y, z)] > th.thr) t = true;
  return t;
}

// Hybrid: troubled nodes on tbox ([-1, n]^nd); counts troubled interior nodes
// and sets flag[0] = 1 if any (the global decision of Algorithm 3).  With a
// buffer buf > 0 the mask tr marks a node when any node within buf of it in
// each direction is troubled (the sensor box [-4, n+3] covers buf <= 2).
template <int ND, typename TW = double>
__device__ __forceinline__ void k_troubled_body(const VBlock& vb, const DevGrid& g, const TW* __restrict__ W, double hr, double hp, const TW* __restrict__ om,
                           Box ob, double thr, unsigned char* __restrict__ tr, Box tb, int* flag,
                           unsigned long long* count, int buf = 0) {
  unsigned long long local = 0;
  // the thresholds in TW, rounded once per block (FP64 work) and shared
  __shared__ TW s_th[3];
  __syncthreads();  // a block running several members' jobs: the previous member's reads are done
  if (threadIdx.x == 0) {
    const TroubleThr<TW> t0(hr, hp, thr);
    s_th[0] = t0.hr;
    s_th[1] = t0.hp;
    s_th[2] = t0.thr;
  }
  __syncthreads();
  TroubleThr<TW> th;
  th.hr = s_th[0];
  th.hp = s_th[1];
  th.thr = s_th[2];
  BOX_LOOP(tb, e) {
    int c[3];
    box_coords(tb, e, c);
    bool own = troubled_at<ND, TW>(g, W, th, om, ob, c[0], c[1], c[2]);
    bool t = own;
    if (buf > 0 && tr) {
      const int bz = ND > 2 ? buf : 0, by = ND > 1 ? buf : 0;
      for (int dz = -bz; dz <= bz && !t; ++dz)
        for (int dy = -by; dy <= by && !t; ++dy)
          for (int dx = -buf; dx <= buf && !t; ++dx)
            if (dx || dy || dz) t = troubled_at<ND, TW>(g, W, th, om, ob, c[0] + dx, c[1] + dy, c[2] + dz);
    }
    if (tr) tr[e] = t ? 1 : 0;
    bool interior = true;
#pragma unroll
    for (int d = 0; d < ND; ++d) interior = interior && c[d] >= 0 && c[d] < g.n[d];
    if (own && interior) ++local;
  }
  if (local) {
    atomicAdd(count, local);
    atomicOr(flag, 1);
  }
}

template <int ND, typename TW = double>
__global__ void k_troubled(DevGrid g, const TW* __restrict__ W, double hr, double hp, const TW* __restrict__ om,
                           Box ob, double thr, unsigned char* __restrict__ tr, Box tb, int* flag,
                           unsigned long long* count, int buf) {
  k_troubled_body<ND, TW>(hw_block(), g, W, hr, hp, om, ob, thr, tr, tb, flag, count, buf);
}

// Per-interface hybrid: LAD flux at interfaces i+1/2 (i in [-1, n-1]) in the
// conservative E4 flux form h = 7/12 (F_i + F_{i+1}) - 1/12 (F_{i-1} + F_{i+2}).
template <int ND, typename T = double>
__device__ __forceinline__ void k_lad_hflux_body(const VBlock& vb, const DevGrid& g, int l, const T* __restrict__ Fn, Box fb, T* __restrict__ H, Box hb) {
  constexpr int NV = ND + 2;
  long long fs = fb.size(), hs = hb.size();
  long long st = l == 0 ? 1 : (l == 1 ? (long long)fb.ext[0] : (long long)fb.ext[0] * fb.ext[1]);
  BOX_LOOP(hb, e) {
    int c[3];
    box_coords(hb, e, c);
    long long q = fb.at(c[0], c[1], c[2]);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T* f = Fn + v * fs;
      H[v * hs + e] = T(7.0 / 12.0) * (f[q] + f[q + st]) - T(1.0 / 12.0) * (f[q - st] + f[q + 2 * st]);
    }
  }
}

template <int ND, typename T = double>
__global__ void k_lad_hflux(DevGrid g, int l, const T* __restrict__ Fn, Box fb, T* __restrict__ H, Box hb) {
  k_lad_hflux_body<ND, T>(hw_block(), g, l, Fn, fb, H, hb);
}

}  // namespace cgk
