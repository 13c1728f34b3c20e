// C-GBR (Sec. 2.3): characteristic gradient-based reconstruction with MP5
// limiting and the wave-appropriate selection of Eq. (8), HLLC flux of
// Eq. (9)-(10), and the kernels of one RK stage.
#pragma once
#include "cg_device.cuh"

namespace cgk {

struct GbrCfg {
  double gamma, gm1, thr, eps, alpha;
  int window;  // interface sensor window half-width
  float f_gamma, f_gm1, f_thr, f_eps, f_alpha;  // FP32 copies for the mixed form
};

// interface frame: unit normal, tangents, averaged state and its sound speed
template <int ND, typename T = double>
struct Frame {
  T n[3], t1[3], t2[3];
  T ha, hb, ic2, cb, cr;
};

// orthonormal tangents of a curvilinear frame (2D: (-n_y, n_x); 3D: t1 from
// the two largest components of n, t2 = n x t1)
template <int ND, typename T = double>
__device__ __forceinline__ void tangents(const T* n, T* t1, T* t2) {
  if (ND == 2) {
    t1[0] = -n[1];
    t1[1] = n[0];
  } else if (ND == 3) {
    int s = 0;
    if (fabs(n[1]) < fabs(n[s])) s = 1;
    if (fabs(n[2]) < fabs(n[s])) s = 2;
    int a = (s + 1) % 3, b = (s + 2) % 3;
    T r = T(1.0) / sqrt(n[a] * n[a] + n[b] * n[b]);
    t1[s] = T(0);
    t1[a] = -n[b] * r;
    t1[b] = n[a] * r;
    t2[0] = n[1] * t1[2] - n[2] * t1[1];
    t2[1] = n[2] * t1[0] - n[0] * t1[2];
    t2[2] = n[0] * t1[1] - n[1] * t1[0];
  }
}

template <int ND, bool CART, int DIR, typename T = double>
__device__ __forceinline__ void to_char(const Frame<ND, T>& f, const T* w, T* c) {
  constexpr int IP = ND + 1;
  T un = sdot<ND, CART, DIR, 0, T>(f.n, w + 1);
  c[0] = f.ha * w[IP] - f.hb * un;
  c[1] = w[0] - f.ic2 * w[IP];
  if (ND >= 2) c[2] = sdot<ND, CART, DIR, 1, T>(f.t1, w + 1);
  if (ND == 3) c[3] = sdot<ND, CART, DIR, 2, T>(f.t2, w + 1);
  c[IP] = f.ha * w[IP] + f.hb * un;
}

template <int ND, bool CART, int DIR, typename T = double>
__device__ __forceinline__ void from_char(const Frame<ND, T>& f, const T* c, T* w) {
  constexpr int IP = ND + 1;
  T s = c[0] + c[IP];
  T un = (c[IP] - c[0]) * f.cr;
  w[0] = c[1] + s;
  w[IP] = (f.cb * f.cb) * s;
#pragma unroll
  for (int m = 0; m < ND; ++m) {
    // u_m = u_n n_m + C3 t1_m + C4 t2_m, structurally zero terms dropped
    T u = T(0);
    bool any = false;
    if (frame_nz(CART, ND, DIR, 0, m)) { u = un * f.n[m]; any = true; }
    if (ND >= 2 && frame_nz(CART, ND, DIR, 1, m)) { u = any ? u + c[2] * f.t1[m] : c[2] * f.t1[m]; any = true; }
    if (ND == 3 && frame_nz(CART, ND, DIR, 2, m)) { u = any ? u + c[3] * f.t2[m] : c[3] * f.t2[m]; any = true; }
    w[1 + m] = u;
  }
}

// HLLC flux (Eq. 9-10) with interface metrics xi (not normalised);
// g2 = |xi|^2, g = |xi|, ig2 = 1/|xi|^2 supplied by the caller.
template <int ND, bool CART, int DIR, typename T = double>
__device__ __forceinline__ void hllc(T gamma, T gm1, const T* WL, const T* WR, const T* xi, T g2, T g, T ig2, T* F) {
  constexpr int IP = ND + 1;
  T rL = WL[0], pL = WL[IP], rR = WR[0], pR = WR[IP];
  T UL = sdot<ND, CART, DIR, 0, T>(xi, WL + 1);
  T UR = sdot<ND, CART, DIR, 0, T>(xi, WR + 1);
  T qL = WL[1] * WL[1], qR = WR[1] * WR[1];
#pragma unroll
  for (int m = 1; m < ND; ++m) {
    qL = qL + WL[1 + m] * WL[1 + m];
    qR = qR + WR[1 + m] * WR[1 + m];
  }
  T EL = pL / gm1 + T(0.5) * rL * qL;
  T ER = pR / gm1 + T(0.5) * rR * qR;
  T cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
  T sL = sqrt(rL), sR = sqrt(rR);
  T iden = T(1.0) / (sL + sR);
  T uh[3];
#pragma unroll
  for (int m = 0; m < ND; ++m) uh[m] = (sL * WL[1 + m] + sR * WR[1 + m]) * iden;
  T qh = uh[0] * uh[0];
#pragma unroll
  for (int m = 1; m < ND; ++m) qh = qh + uh[m] * uh[m];
  T Uh = sdot<ND, CART, DIR, 0, T>(xi, uh);
  T HL = (EL + pL) / rL, HR = (ER + pR) / rR;
  T Hh = (sL * HL + sR * HR) * iden;
  T ch = sqrt(gm1 * (Hh - T(0.5) * qh));
  T SL = dmin(UL - cL * g, Uh - ch * g);
  T SR = dmax(UR + cR * g, Uh + ch * g);
  T Ss = (rR * UR * (SR - UR) - rL * UL * (SL - UL) + (pL - pR) * g2) / (rR * (SR - UR) - rL * (SL - UL));
  const T* W;
  T S, U, E, r, p;
  bool star;
  if (T(0) <= SL) { W = WL; S = T(0); U = UL; E = EL; r = rL; p = pL; star = false; }
  else if (T(0) <= Ss) { W = WL; S = SL; U = UL; E = EL; r = rL; p = pL; star = true; }
  else if (T(0) <= SR) { W = WR; S = SR; U = UR; E = ER; r = rR; p = pR; star = true; }
  else { W = WR; S = T(0); U = UR; E = ER; r = rR; p = pR; star = false; }
  // convective flux of the chosen side (Eq. 2)
  T FK[ND + 2];
  FK[0] = r * U;
#pragma unroll
  for (int m = 0; m < ND; ++m)
    FK[1 + m] = frame_nz(CART, ND, DIR, 0, m) ? r * W[1 + m] * U + xi[m] * p : r * W[1 + m] * U;
  FK[IP] = (E + p) * U;
  if (!star) {
#pragma unroll
    for (int v = 0; v < ND + 2; ++v) F[v] = FK[v];
    return;
  }
  T fac = r * (S - U) / (S - Ss);
  T d = Ss - U;
  F[0] = FK[0] + S * (fac - r);
#pragma unroll
  for (int m = 0; m < ND; ++m) {
    T qs = frame_nz(CART, ND, DIR, 0, m) ? fac * (W[1 + m] + xi[m] * d * ig2) : fac * W[1 + m];
    F[1 + m] = FK[1 + m] + S * (qs - r * W[1 + m]);
  }
  T qe = fac * (E / r + d * (Ss * ig2 + p / (r * (S - U))));
  F[IP] = FK[IP] + S * (qe - E);
}

// Flux at one interface i+1/2 from the stencil W_{i-2..i+3}, the gradients
// W'_{i,i+1}, second derivatives W''_{i,i+1}, the interface sensor and the
// interface metrics.  Wave order: 0 = u_n - c, 1 = entropy, 2.. = shear,
// last = u_n + c.
template <int ND, bool CART, int DIR, typename T = double>
__device__ __forceinline__ void gbr_flux(const GbrCfg& q, const DevGrid& g, const T (&Wst)[6][ND + 2],
                                         const T (&Wd)[2][ND + 2], const T (&Wdd)[2][ND + 2], T omb,
                                         const T* xi, T* F) {
  constexpr int NV = ND + 2, IP = ND + 1;
  const T c12 = T(1.0 / 12.0);
  const T gamma = gconst<T>(q.gamma, q.f_gamma), gm1 = gconst<T>(q.gm1, q.f_gm1),
          alpha = gconst<T>(q.alpha, q.f_alpha), eps = gconst<T>(q.eps, q.f_eps), thr = gconst<T>(q.thr, q.f_thr);
  Frame<ND, T> fr;
  T g2, gg, ig2;
  if (CART) {
    g2 = gconst<T>(g.cg2[DIR], g.f_cg2[DIR]);
    gg = gconst<T>(g.cg[DIR], g.f_cg[DIR]);
    ig2 = gconst<T>(g.cig2[DIR], g.f_cig2[DIR]);
#pragma unroll
    for (int m = 0; m < ND; ++m) {
      fr.n[m] = gconst<T>(g.cn[DIR][m], g.f_cn[DIR][m]);
      fr.t1[m] = gconst<T>(g.ct1[DIR][m], g.f_ct1[DIR][m]);
      fr.t2[m] = gconst<T>(g.ct2[DIR][m], g.f_ct2[DIR][m]);
    }
  } else {
    g2 = xi[0] * xi[0];
#pragma unroll
    for (int m = 1; m < ND; ++m) g2 = g2 + xi[m] * xi[m];
    gg = sqrt(g2);
    T ig = T(1.0) / gg;
    ig2 = T(1.0) / g2;
#pragma unroll
    for (int m = 0; m < ND; ++m) fr.n[m] = xi[m] * ig;
    tangents<ND, T>(fr.n, fr.t1, fr.t2);
  }
  T rb = T(0.5) * (Wst[2][0] + Wst[3][0]);
  T pb = T(0.5) * (Wst[2][IP] + Wst[3][IP]);
  fr.cb = sqrt(gamma * pb / rb);
  T ic = T(1.0) / fr.cb;
  fr.ic2 = ic * ic;
  fr.ha = T(0.5) * fr.ic2;
  fr.hb = T(0.5) * rb * ic;
  fr.cr = fr.cb / rb;

  T C[6][NV], Cd[2][NV], Cdd[2][NV];
#pragma unroll
  for (int j = 0; j < 6; ++j) to_char<ND, CART, DIR, T>(fr, Wst[j], C[j]);
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    to_char<ND, CART, DIR, T>(fr, Wd[j], Cd[j]);
    to_char<ND, CART, DIR, T>(fr, Wdd[j], Cdd[j]);
  }
  const bool disc = omb > thr;
  T CL[NV], CR[NV];
#pragma unroll
  for (int b = 0; b < NV; ++b) {
    T v0 = C[0][b], v1 = C[1][b], v2 = C[2][b], v3 = C[3][b], v4 = C[4][b], v5 = C[5][b];
    T cl = v2 + T(0.5) * Cd[0][b] + Cdd[0][b] * c12;
    T cr = v3 - T(0.5) * Cd[1][b] + Cdd[1][b] * c12;
    if (b == 0 || b == IP) {  // acoustic: sensor
      if (disc) {
        CL[b] = mp5(v0, v1, v2, v3, v4, alpha, eps);
        CR[b] = mp5(v5, v4, v3, v2, v1, alpha, eps);
      } else {
        CL[b] = cl;
        CR[b] = cr;
      }
    } else if (b == 1) {      // entropy: MP criterion
      T cc = T(0.5) * (cl + cr);
      T umpL = v2 + minmod2(v3 - v2, alpha * (v2 - v1));
      CL[b] = ((cl - v2) * (cl - umpL) > eps) ? mp5(v0, v1, v2, v3, v4, alpha, eps) : cc;
      T umpR = v3 + minmod2(v2 - v3, alpha * (v3 - v4));
      CR[b] = ((cr - v3) * (cr - umpR) > eps) ? mp5(v5, v4, v3, v2, v1, alpha, eps) : cc;
    } else {                  // shear: sensor
      if (disc) {
        CL[b] = mp5(v0, v1, v2, v3, v4, alpha, eps);
        CR[b] = mp5(v5, v4, v3, v2, v1, alpha, eps);
      } else {
        T cc = T(0.5) * (cl + cr);
        CL[b] = cc;
        CR[b] = cc;
      }
    }
  }
  T WL[NV], WR[NV];
  from_char<ND, CART, DIR, T>(fr, CL, WL);
  from_char<ND, CART, DIR, T>(fr, CR, WR);
  if (WL[0] <= T(0) || WL[IP] <= T(0) || WR[0] <= T(0) || WR[IP] <= T(0)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) { WL[v] = Wst[2][v]; WR[v] = Wst[3][v]; }
  }
  T xl[3];
  if (CART) {
#pragma unroll
    for (int m = 0; m < ND; ++m) xl[m] = (m == DIR) ? gconst<T>(g.cxh[DIR], g.f_cxh[DIR]) : T(0);
  } else {
#pragma unroll
    for (int m = 0; m < ND; ++m) xl[m] = xi[m];
  }
  hllc<ND, CART, DIR, T>(gamma, gm1, WL, WR, xl, g2, gg, ig2, F);
}

}  // namespace cgk
