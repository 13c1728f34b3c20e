// LAD (Sec. 2.2): artificial bulk viscosity beta* and conductivity kappa*
// (Eq. 4-6) smoothed by the truncated-Gaussian overbar, central node fluxes
// F^c + F^v (Eq. 2-3 with mu = 0, beta = beta*, kappa = kappa*) and their
// E4 / C6 divergence; the eighth-order implicit filter of LAD-C6; the
// troubled-node flags of the hybrid (Sec. 5).
#pragma once
#include "cg_kernels.cuh"

namespace cgk {

struct LadBuffers {
  double* gr = nullptr;     // physical gradients of (u_k, T, rho, e): nf*nd planes on b3 ([-3, n+2]^nd)
  double* dv = nullptr;     // dilatation on b3
  double* bt[2] = {nullptr, nullptr};  // beta* (ping-pong, interior)
  double* kp[2] = {nullptr, nullptr};  // kappa*
  double* Fn = nullptr;     // node fluxes along one direction: nv planes on fbox (positions [-2, n+1])
  double* D = nullptr;      // compact flux derivative (nv planes, interior)
  double* df[3] = {nullptr, nullptr, nullptr};  // C6: computational derivatives of the fields on b3
  double* tmp = nullptr;    // filter ping-pong state
  unsigned char* tr = nullptr;  // hybrid: troubled nodes on tbox ([-1, n]^nd)
  Box b3, tbox, fbox[3], hbox[3];
};

// fields differentiated by LAD: velocities, T = gamma M^2 p / rho, rho, e = p / (rho (gamma-1))
template <int ND>
__device__ __forceinline__ void lad_fields(const DevGrid& g, const double* w, double* f) {
  constexpr int IP = ND + 1;
  double rho = w[0], p = w[IP];
#pragma unroll
  for (int k = 0; k < ND; ++k) f[k] = w[1 + k];
  f[ND] = g.gm2 * p / rho;
  f[ND + 1] = rho;
  f[ND + 2] = p / (rho * g.gm1);
}

__device__ __forceinline__ void box_coords(const Box& b, long long e, int* c) {
  c[0] = (int)(e % b.ext[0]) - b.off[0];
  long long r = e / b.ext[0];
  c[1] = (int)(r % b.ext[1]) - b.off[1];
  c[2] = (int)(r / b.ext[1]) - b.off[2];
}

#define BOX_LOOP(b, e) \
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (b).size(); e += (long long)gridDim.x * blockDim.x)

// Physical gradients and dilatation on b3.  E4 computes the computational
// derivatives in place; C6 reads them from the compact line solves (df).
template <int ND, bool CART, bool C6>
__global__ void k_lad_grad(DevGrid g, const double* __restrict__ W, const double* __restrict__ df0,
                           const double* __restrict__ df1, const double* __restrict__ df2, double* __restrict__ gr,
                           double* __restrict__ dv, Box b3, const int* guard, int want) {
  constexpr int NV = ND + 2, NF = ND + 3;
  if (guard && *guard != want) return;
  long long bs = b3.size();
  BOX_LOOP(b3, e) {
    int c[3];
    box_coords(b3, e, c);
    double d[3][NF];  // d[l][f] = d f / d xi_l
#pragma unroll
    for (int l = 0; l < ND; ++l) {
      if (C6) {
        const double* df = l == 0 ? df0 : (l == 1 ? df1 : df2);
#pragma unroll
        for (int f = 0; f < NF; ++f) d[l][f] = df[f * bs + e];
      } else {
        double fm2[NF], fm1[NF], fp1[NF], fp2[NF], w[NV];
        int cc[3] = {c[0], c[1], c[2]};
        cc[l] = c[l] - 2; load_state<ND>(g, W, cc[0], cc[1], cc[2], w); lad_fields<ND>(g, w, fm2);
        cc[l] = c[l] - 1; load_state<ND>(g, W, cc[0], cc[1], cc[2], w); lad_fields<ND>(g, w, fm1);
        cc[l] = c[l] + 1; load_state<ND>(g, W, cc[0], cc[1], cc[2], w); lad_fields<ND>(g, w, fp1);
        cc[l] = c[l] + 2; load_state<ND>(g, W, cc[0], cc[1], cc[2], w); lad_fields<ND>(g, w, fp2);
#pragma unroll
        for (int f = 0; f < NF; ++f) d[l][f] = d4(fm2[f], fm1[f], fp1[f], fp2[f]);
      }
    }
    double div = 0.0;
    if (CART) {
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int m = 0; m < ND; ++m) {
          double v = (g.cjac * g.cxh[m]) * d[m][f];
          gr[(f * ND + m) * bs + e] = v;
          if (f < ND && m == f) div = (f == 0) ? v : div + v;
        }
    } else {
      long long pq = plin(g, c[0], c[1], c[2]);
      double J = g.jac[pq];
      double xm[3][3];
#pragma unroll
      for (int l = 0; l < ND; ++l)
#pragma unroll
        for (int m = 0; m < ND; ++m) xm[l][m] = J * g.xh[(l * ND + m) * g.NP + pq];
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int m = 0; m < ND; ++m) {
          double s = xm[0][m] * d[0][f];
#pragma unroll
          for (int l = 1; l < ND; ++l) s = s + xm[l][m] * d[l][f];
          gr[(f * ND + m) * bs + e] = s;
          if (f < ND && m == f) div = (f == 0) ? s : div + s;
        }
    }
    dv[e] = div;
  }
}

// Raw coefficients at interior nodes, Eq. (4)-(6):
// beta* = C_beta rho f_sw |sum_l d4(div)_l Delta_{l,beta}^2|,
// kappa* = C_kappa (rho c / T) |sum_l d4(e)_l Delta_{l,kappa}|.
template <int ND, bool CART>
__global__ void k_lad_coef(DevGrid g, const double* __restrict__ W, const double* __restrict__ gr,
                           const double* __restrict__ dv, Box b3, double c_beta, double c_kappa,
                           double* __restrict__ bt, double* __restrict__ kp, const int* guard, int want) {
  constexpr int NV = ND + 2, IP = ND + 1;
  if (guard && *guard != want) return;
  long long bs = b3.size();
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.N; q += (long long)gridDim.x * blockDim.x) {
    int c[3];
    c[0] = (int)(q % g.n[0]);
    c[1] = (int)((q / g.n[0]) % g.n[1]);
    c[2] = (int)(q / ((long long)g.n[0] * g.n[1]));
    long long e0 = b3.at(c[0], c[1], c[2]);
    double w[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = W[v * g.N + q];
    double rho = w[0], p = w[IP];
    double T = g.gm2 * p / rho;
    double cs = sqrt(g.gamma * p / rho);
    double div = dv[e0];
    double curl2 = 0.0;
    auto G = [&](int f, int m) { return gr[(f * ND + m) * bs + e0]; };
    if (ND == 2) {
      double w3 = G(1, 0) - G(0, 1);
      curl2 = w3 * w3;
    } else if (ND == 3) {
      double w1 = G(2, 1) - G(1, 2), w2 = G(0, 2) - G(2, 0), w3 = G(1, 0) - G(0, 1);
      curl2 = w1 * w1 + w2 * w2 + w3 * w3;
    }
    double heav = div < 0.0 ? 1.0 : 0.0;
    double fsw = heav * (div * div) / (div * div + curl2 + 1e-32);
    double gmr = G(ND + 1, 0) * G(ND + 1, 0), gme = G(ND + 2, 0) * G(ND + 2, 0);
#pragma unroll
    for (int m = 1; m < ND; ++m) {
      gmr = gmr + G(ND + 1, m) * G(ND + 1, m);
      gme = gme + G(ND + 2, m) * G(ND + 2, m);
    }
    gmr = sqrt(gmr);
    gme = sqrt(gme);
    double sb = 0.0, sk = 0.0;
#pragma unroll
    for (int l = 0; l < ND; ++l) {
      long long st = l == 0 ? 1 : (l == 1 ? (long long)b3.ext[0] : (long long)b3.ext[0] * b3.ext[1]);
      double d4d = (dv[e0 - 2 * st] + dv[e0 + 2 * st]) - 4.0 * (dv[e0 - st] + dv[e0 + st]) + 6.0 * div;
      double ev[5];
#pragma unroll
      for (int t = -2; t <= 2; ++t) {
        int cc[3] = {c[0], c[1], c[2]};
        cc[l] += t;
        double ww[NV];
        load_state<ND>(g, W, cc[0], cc[1], cc[2], ww);
        ev[t + 2] = ww[IP] / (ww[0] * g.gm1);
      }
      double d4e = (ev[0] + ev[4]) - 4.0 * (ev[1] + ev[3]) + 6.0 * ev[2];
      double pr, pe;
      if (CART) {
        pr = g.ch[l] * G(ND + 1, l);
        pe = g.ch[l] * G(ND + 2, l);
      } else {
        long long pq = plin(g, c[0], c[1], c[2]);
        pr = g.dxl[(l * ND + 0) * g.NP + pq] * G(ND + 1, 0);
        pe = g.dxl[(l * ND + 0) * g.NP + pq] * G(ND + 2, 0);
#pragma unroll
        for (int m = 1; m < ND; ++m) {
          double x = g.dxl[(l * ND + m) * g.NP + pq];
          pr = pr + x * G(ND + 1, m);
          pe = pe + x * G(ND + 2, m);
        }
      }
      double Db = fabs(pr) / (gmr + 1e-32);
      double Dk = fabs(pe) / (gme + 1e-32);
      double tb = d4d * Db * Db, tk = d4e * Dk;
      sb = (l == 0) ? tb : sb + tb;
      sk = (l == 0) ? tk : sk + tk;
    }
    bt[q] = c_beta * rho * fsw * fabs(sb);
    kp[q] = c_kappa * (rho * cs / T) * fabs(sk);
  }
}

// truncated-Gaussian overbar along l (nine points, Cook & Cabot), two fields;
// ghost values: periodic wrap, wall mirror, otherwise the boundary node.
template <int ND>
__global__ void k_gauss(DevGrid g, int l, const double* __restrict__ a, const double* __restrict__ b,
                        double* __restrict__ ao, double* __restrict__ bo, const int* guard, int want) {
  if (guard && *guard != want) return;
  const double A0 = 3565.0 / 10368.0, A1 = 3091.0 / 12960.0, A2 = 1997.0 / 25920.0, A3 = 149.0 / 12960.0,
               A4 = 107.0 / 103680.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.N; q += (long long)gridDim.x * blockDim.x) {
    int c[3];
    c[0] = (int)(q % g.n[0]);
    c[1] = (int)((q / g.n[0]) % g.n[1]);
    c[2] = (int)(q / ((long long)g.n[0] * g.n[1]));
    long long s[9];
#pragma unroll
    for (int t = -4; t <= 4; ++t) {
      int cc[3] = {c[0], c[1], c[2]};
      cc[l] += t;
      s[t + 4] = scalar_src(g, cc[0], cc[1], cc[2]);
    }
    ao[q] = A0 * a[s[4]] + A1 * (a[s[3]] + a[s[5]]) + A2 * (a[s[2]] + a[s[6]]) + A3 * (a[s[1]] + a[s[7]]) +
            A4 * (a[s[0]] + a[s[8]]);
    bo[q] = A0 * b[s[4]] + A1 * (b[s[3]] + b[s[5]]) + A2 * (b[s[2]] + b[s[6]]) + A3 * (b[s[1]] + b[s[7]]) +
            A4 * (b[s[0]] + b[s[8]]);
  }
}

// Node fluxes along l at positions [-2, n+1] (interior lines):
// F = F^c(W; xi_hat_l) - [0, xi_hat_l tau, xi_hat_l . phi], tau = beta* div,
// phi_m = u_m tau + kappa* dT/dx_m.
template <int ND, bool CART>
__global__ void k_lad_nodeflux(DevGrid g, int l, const double* __restrict__ W, const double* __restrict__ bt,
                               const double* __restrict__ kp, const double* __restrict__ gr,
                               const double* __restrict__ dv, Box b3, double* __restrict__ Fn, Box fb,
                               const int* guard, int want) {
  constexpr int NV = ND + 2, IP = ND + 1;
  if (guard && *guard != want) return;
  long long fs = fb.size(), bs = b3.size();
  BOX_LOOP(fb, e) {
    int c[3];
    box_coords(fb, e, c);
    double w[NV];
    load_state<ND>(g, W, c[0], c[1], c[2], w);
    double xi[3];
    if (CART) {
#pragma unroll
      for (int m = 0; m < ND; ++m) xi[m] = (m == l) ? g.cxh[l] : 0.0;
    } else {
      long long pq = plin(g, c[0], c[1], c[2]);
#pragma unroll
      for (int m = 0; m < ND; ++m) xi[m] = g.xh[(l * ND + m) * g.NP + pq];
    }
    double U, q2;
    if (CART) U = xi[l] * w[1 + l];
    else {
      U = xi[0] * w[1];
#pragma unroll
      for (int m = 1; m < ND; ++m) U = U + xi[m] * w[1 + m];
    }
    q2 = w[1] * w[1];
#pragma unroll
    for (int m = 1; m < ND; ++m) q2 = q2 + w[1 + m] * w[1 + m];
    double rho = w[0], p = w[IP];
    double E = p / g.gm1 + 0.5 * rho * q2;
    long long sq = scalar_src(g, c[0], c[1], c[2]);
    long long be = b3.at(c[0], c[1], c[2]);
    double tau = bt[sq] * dv[be];
    double kap = kp[sq];
    double fe = 0.0;
    bool first = true;
#pragma unroll
    for (int m = 0; m < ND; ++m) {
      if (CART && m != l) continue;
      double phi = w[1 + m] * tau + kap * gr[(ND * ND + m) * bs + be];
      fe = first ? xi[m] * phi : fe + xi[m] * phi;
      first = false;
    }
    Fn[0 * fs + e] = rho * U;
#pragma unroll
    for (int m = 0; m < ND; ++m) {
      double fc = (CART && m != l) ? rho * w[1 + m] * U : rho * w[1 + m] * U + xi[m] * p;
      Fn[(1 + m) * fs + e] = (CART && m != l) ? fc : fc - xi[m] * tau;
    }
    Fn[IP * fs + e] = (E + p) * U - fe;
  }
}

// Stage epilogue shared by the LAD divergence kernels: tot = acc + D (or D),
// then store acc, R = -J tot, or the RK combination.
template <int ND>
__device__ __forceinline__ void lad_epilogue(const DevGrid& g, const StageArgs& A, long long qi, const int* c,
                                             const double* Dv) {
  constexpr int NV = ND + 2, IP = ND + 1;
  double J = g.curv ? g.jac[plin(g, c[0], c[1], c[2])] : g.cjac;
  double out[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double tot = A.first ? Dv[v] : A.acc[v * g.N + qi] + Dv[v];
    if (!A.last) {
      A.acc[v * g.N + qi] = tot;
      continue;
    }
    double r = -(J * tot);
    if (!A.rk) {
      A.R[v * g.N + qi] = r;
      continue;
    }
    double dt = *A.dt;
    double un = A.Un[v * g.N + qi];
    double o;
    if (A.stage == 1) o = un + dt * r;
    else if (A.stage == 2) o = 0.75 * un + 0.25 * (A.Uc[v * g.N + qi] + dt * r);
    else o = (1.0 / 3.0) * un + (2.0 / 3.0) * (A.Uc[v * g.N + qi] + dt * r);
    out[v] = o;
    A.Uout[v * g.N + qi] = o;
  }
  if (A.last && A.rk && A.stage == 3) {
    double ke = out[1] * (out[1] / out[0]);
#pragma unroll
    for (int m = 1; m < ND; ++m) ke = ke + out[1 + m] * (out[1 + m] / out[0]);
    double p = g.gm1 * (out[IP] - 0.5 * ke);
    if (!(out[0] > 0.0) || !(p > 0.0)) {
      atomicOr(A.bad_flag, 1u);
      atomicMin(A.bad_idx, (unsigned long long)qi);
    }
  }
}

// E4 divergence of the node fluxes along l (explicit) or the compact result D.
template <int ND>
__global__ void k_lad_div(DevGrid g, int l, const double* __restrict__ Fn, Box fb, const double* __restrict__ D,
                          StageArgs A, const int* guard, int want) {
  constexpr int NV = ND + 2;
  if (guard && *guard != want) return;
  long long fs = fb.size();
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.N; q += (long long)gridDim.x * blockDim.x) {
    int c[3];
    c[0] = (int)(q % g.n[0]);
    c[1] = (int)((q / g.n[0]) % g.n[1]);
    c[2] = (int)(q / ((long long)g.n[0] * g.n[1]));
    double Dv[NV];
    if (D) {
#pragma unroll
      for (int v = 0; v < NV; ++v) Dv[v] = D[v * g.N + q];
    } else {
      long long e = fb.at(c[0], c[1], c[2]);
      long long st = l == 0 ? 1 : (l == 1 ? (long long)fb.ext[0] : (long long)fb.ext[0] * fb.ext[1]);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double* f = Fn + v * fs;
        Dv[v] = d4(f[e - 2 * st], f[e - st], f[e + st], f[e + 2 * st]);
      }
    }
    lad_epilogue<ND>(g, A, q, c, Dv);
  }
}

// Compact (Thomas) solve of one line: rows [0, m-1] <-> positions lo .. lo+m-1
// (non-periodic: explicit E4 closure rows 0 and m-1; periodic: cyclic on
// [0, n-1]).  rhsfn(x) gives the interior right-hand side at position x,
// e4fn(x) the closure value, out(x) the result slot.
template <typename RHS, typename E4F, typename OUT>
__device__ __forceinline__ void thomas_line(const LineCoef& lc, RHS rhsfn, E4F e4fn, OUT out) {
  const double a = lc.a;
  int m = lc.m;
  if (!lc.periodic) {
    int lo = lc.lo;
    double dp = e4fn(lo);
    out(lo) = dp;
    for (int i = 1; i < m - 1; ++i) {
      dp = (rhsfn(lo + i) - a * dp) / lc.den[i];
      out(lo + i) = dp;
    }
    double x = e4fn(lo + m - 1);
    out(lo + m - 1) = x;
    for (int i = m - 2; i >= 0; --i) {
      double& o = out(lo + i);
      x = o - lc.cp[i] * x;
      o = x;
    }
  } else {
    double dp = rhsfn(0) / 2.0;
    out(0) = dp;
    for (int i = 1; i < m; ++i) {
      dp = (rhsfn(i) - a * dp) / lc.den[i];
      out(i) = dp;
    }
    const double xlast = dp;
    double x = dp;
    for (int i = m - 2; i >= 0; --i) {
      double& o = out(i);
      x = o - lc.cp[i] * x;
      o = x;
    }
    double fact = (out(0) + a * xlast / lc.gam) / lc.fden;
    for (int i = 0; i < m; ++i) {
      double& o = out(i);
      o = o - fact * lc.z[i];
    }
  }
}

// C6 computational derivatives of the LAD fields along l for lines on b3 in
// the other directions; the system spans [-6, n+5] (or is cyclic); results
// at positions [-3, n+2] are kept (df on b3).
template <int ND>
__global__ void k_lad_c6_fields(DevGrid g, int l, const double* __restrict__ W, LineCoef lc, double* __restrict__ work,
                                long long wstride, double* __restrict__ df, Box b3) {
  constexpr int NV = ND + 2, NF = ND + 3;
  int o1 = (l + 1) % 3, o2 = (l + 2) % 3;
  int e1 = b3.ext[o1], e2 = b3.ext[o2];
  long long nl = (long long)e1 * e2 * NF;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nl) return;
  int f = (int)(t % NF);
  long long r = t / NF;
  int c[3];
  c[o1] = (int)(r % e1) - b3.off[o1];
  c[o2] = (int)(r / e1) - b3.off[o2];
  int n = g.n[l];
  double* wk = work + (t / NF) * wstride * NF + (long long)f * wstride;  // scratch line of length n + 16
  auto fv = [&](int x) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[l] = x;
    double w[NV], fl[NF];
    load_state<ND>(g, W, cc[0], cc[1], cc[2], w);
    lad_fields<ND>(g, w, fl);
    return fl[f];
  };
  auto rhs = [&](int x) {
    return (7.0 / 9.0) * (fv(x + 1) - fv(x - 1)) + (1.0 / 36.0) * (fv(x + 2) - fv(x - 2));
  };
  auto e4 = [&](int x) { return d4(fv(x - 2), fv(x - 1), fv(x + 1), fv(x + 2)); };
  auto out = [&](int x) -> double& { return wk[x + 8]; };
  thomas_line(lc, rhs, e4, out);
  long long bs = b3.size();
  for (int x = -3; x <= n + 2; ++x) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[l] = x;
    double v = lc.periodic ? wk[((x % n) + n) % n + 8] : wk[x + 8];
    df[f * bs + b3.at(cc[0], cc[1], cc[2])] = v;
  }
}

// C6 derivative of the node fluxes along l on interior lines: system on
// [0, n-1] with E4 closure rows (or cyclic); D gets the interior values.
template <int ND>
__global__ void k_lad_c6_flux(DevGrid g, int l, const double* __restrict__ Fn, Box fb, LineCoef lc,
                              double* __restrict__ D) {
  constexpr int NV = ND + 2;
  int o1 = (l + 1) % 3, o2 = (l + 2) % 3;
  int e1 = g.n[o1], e2 = g.n[o2];
  long long nl = (long long)e1 * e2 * NV;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nl) return;
  int v = (int)(t % NV);
  long long r = t / NV;
  int c[3];
  c[o1] = (int)(r % e1);
  c[o2] = (int)(r / e1);
  long long fs = fb.size();
  auto f = [&](int x) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[l] = x;
    return Fn[v * fs + fb.at(cc[0], cc[1], cc[2])];
  };
  auto rhs = [&](int x) { return (7.0 / 9.0) * (f(x + 1) - f(x - 1)) + (1.0 / 36.0) * (f(x + 2) - f(x - 2)); };
  auto e4 = [&](int x) { return d4(f(x - 2), f(x - 1), f(x + 1), f(x + 2)); };
  auto out = [&](int x) -> double& {
    int cc[3] = {c[0], c[1], c[2]};
    cc[l] = x;
    return D[v * g.N + (cc[0] + (long long)g.n[0] * (cc[1] + (long long)g.n[1] * cc[2]))];
  };
  thomas_line(lc, rhs, e4, out);
}

// Eighth-order implicit filter of the conserved state along l (LAD-C6, after
// the last stage): non-periodic system on [-1, n] whose end rows keep the
// ghost values, periodic cyclic on [0, n-1].  Reads Uin (ghosts by the
// conserved-variable boundary rule), writes Uout on interior lines.
template <int ND>
__global__ void k_filter(DevGrid g, int l, const double* __restrict__ Uin, LineCoef lc, double b0, double b1,
                         double b2, double b3c, double b4, double* __restrict__ work, double* __restrict__ Uout) {
  constexpr int NV = ND + 2;
  int o1 = (l + 1) % 3, o2 = (l + 2) % 3;
  int e1 = g.n[o1], e2 = g.n[o2];
  long long nl = (long long)e1 * e2 * NV;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nl) return;
  int v = (int)(t % NV);
  long long r = t / NV;
  int c[3];
  c[o1] = (int)(r % e1);
  c[o2] = (int)(r / e1);
  int n = g.n[l];
  auto f = [&](int x) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[l] = x;
    double w[NV];
    load_state<ND, true>(g, Uin, cc[0], cc[1], cc[2], w);
    return w[v];
  };
  auto rhs = [&](int x) {
    int y = x;
    return b0 * f(y) + b1 * (f(y + 1) + f(y - 1)) + b2 * (f(y + 2) + f(y - 2)) + b3c * (f(y + 3) + f(y - 3)) +
           b4 * (f(y + 4) + f(y - 4));
  };
  auto ends = [&](int x) { return x == lc.lo ? f(-1) : f(n); };
  double* wk = work + t * (long long)(n + 2);
  auto out = [&](int x) -> double& { return wk[lc.periodic ? x : x - lc.lo]; };
  thomas_line(lc, rhs, ends, out);
  for (int x = 0; x < n; ++x) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[l] = x;
    Uout[v * g.N + (cc[0] + (long long)g.n[0] * (cc[1] + (long long)g.n[1] * cc[2]))] = wk[lc.periodic ? x : x + 1];
  }
}

// Hybrid: troubled nodes on tbox ([-1, n]^nd): rho < hyb_rho or p < hyb_p, or
// (with the sensor) Omega > threshold; counts troubled interior nodes and
// sets flag[0] = 1 if any (the global decision of Algorithm 3).
template <int ND>
__global__ void k_troubled(DevGrid g, const double* __restrict__ W, double hr, double hp, const double* __restrict__ om,
                           Box ob, double thr, unsigned char* __restrict__ tr, Box tb, int* flag,
                           unsigned long long* count) {
  constexpr int NV = ND + 2, IP = ND + 1;
  unsigned long long local = 0;
  BOX_LOOP(tb, e) {
    int c[3];
    box_coords(tb, e, c);
    double w[NV];
    load_state<ND>(g, W, c[0], c[1], c[2], w);
    bool t = w[0] < hr || w[IP] < hp;
    if (om && om[ob.at(c[0], c[1], c[2])] > thr) t = true;
    if (tr) tr[e] = t ? 1 : 0;
    bool interior = true;
#pragma unroll
    for (int d = 0; d < ND; ++d) interior = interior && c[d] >= 0 && c[d] < g.n[d];
    if (t && interior) ++local;
  }
  if (local) {
    atomicAdd(count, local);
    atomicOr(flag, 1);
  }
}

// Per-interface hybrid: LAD flux at interfaces i+1/2 (i in [-1, n-1]) in the
// conservative E4 flux form h = 7/12 (F_i + F_{i+1}) - 1/12 (F_{i-1} + F_{i+2}).
template <int ND>
__global__ void k_lad_hflux(DevGrid g, int l, const double* __restrict__ Fn, Box fb, double* __restrict__ H, Box hb) {
  constexpr int NV = ND + 2;
  long long fs = fb.size(), hs = hb.size();
  long long st = l == 0 ? 1 : (l == 1 ? (long long)fb.ext[0] : (long long)fb.ext[0] * fb.ext[1]);
  BOX_LOOP(hb, e) {
    int c[3];
    box_coords(hb, e, c);
    long long q = fb.at(c[0], c[1], c[2]);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double* f = Fn + v * fs;
      H[v * hs + e] = (7.0 / 12.0) * (f[q] + f[q + st]) - (1.0 / 12.0) * (f[q - st] + f[q + 2 * st]);
    }
  }
}

}  // namespace cgk
