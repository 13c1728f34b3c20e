// Grid metrics on the device (once per solver), Sec. 2.1: xi_hat = xi_x / J.
//
// Node metrics come from derivatives D of the node coordinates, D being the
// scheme's own first derivative (explicit sixth order for C-GBR, E4 for LAD-E4
// and the hybrid, the compact sixth-order C6 of the LAD-C6 flux divergence)
// so that the discrete metric identities hold for the flux divergence
// actually used (freestream preservation).  2D: xi_x = y_eta,
// xi_y = -x_eta, eta_x = -y_xi, eta_y = x_xi.  3D: conservative
// (Thomas-Lombard) form xi_x = (y_eta z)_zeta - (y_zeta z)_eta and its cyclic
// permutations.  Interface metrics: the flux-form interpolant H of the node
// metrics along the interface direction (D = difference of H).  Coordinates
// are extended 14 layers past the grid: linear extrapolation at ends,
// translation by the period across periodic directions.
#pragma once
#include "cg_device.cuh"

namespace cgk {

constexpr int MGC = 14;

struct EBox {
  int nd, n[3], ge[3], PE[3];
  long long NE;
  __host__ __device__ long long at(int i, int j, int k) const {
    return (long long)(i + ge[0]) + (long long)PE[0] * ((long long)(j + ge[1]) + (long long)PE[1] * (long long)(k + ge[2]));
  }
  __host__ __device__ long long stride(int d) const {
    return d == 0 ? 1 : (d == 1 ? (long long)PE[0] : (long long)PE[0] * PE[1]);
  }
  __device__ void coords(long long e, int* c) const {
    c[0] = (int)(e % PE[0]) - ge[0];
    long long r = e / PE[0];
    c[1] = (int)(r % PE[1]) - ge[1];
    c[2] = (int)(r / PE[1]) - ge[2];
  }
};

#define EB_LOOP(eb, e) \
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (eb).NE; e += (long long)gridDim.x * blockDim.x)

// interior coordinates -> extended box (NaN elsewhere)
__global__ void km_load(EBox eb, const double* __restrict__ xyz, long long N, int m, double* __restrict__ X) {
  EB_LOOP(eb, e) {
    int c[3];
    eb.coords(e, c);
    bool in = true;
    for (int d = 0; d < 3; ++d) in = in && c[d] >= 0 && c[d] < eb.n[d];
    X[e] = in ? xyz[(long long)m * N + (c[0] + (long long)eb.n[0] * (c[1] + (long long)eb.n[1] * c[2]))]
              : __longlong_as_double(0x7ff8000000000000LL);
  }
}

// ghost layers along d: directions before d over their extended range, after d interior
__global__ void km_extend(EBox eb, int d, int periodic, double period, double* __restrict__ X) {
  EB_LOOP(eb, e) {
    int c[3];
    eb.coords(e, c);
    bool ok = true;
    for (int a = d + 1; a < 3; ++a) ok = ok && c[a] >= 0 && c[a] < eb.n[a];
    int n = eb.n[d], t = c[d];
    if (!ok || (t >= 0 && t < n)) continue;
    long long s = eb.stride(d);
    long long q0 = e - (long long)t * s;  // node 0 of this line
    double v;
    if (periodic) {
      int r = t % n;
      if (r < 0) r += n;
      int fl = (t - r) / n;
      v = X[q0 + (long long)r * s] + (double)fl * period;
    } else if (t < 0) {
      double x0 = X[q0], x1 = X[q0 + s];
      v = x0 + (double)(-t) * (x0 - x1);
    } else {
      double xa = X[q0 + (long long)(n - 1) * s], xb = X[q0 + (long long)(n - 2) * s];
      v = xa + (double)(t - (n - 1)) * (xa - xb);
    }
    X[e] = v;
  }
}

// op 0: derivative D, op 1: interpolant H (at i+1/2 stored at i); six: order pair
__global__ void km_op(EBox eb, const double* __restrict__ f, int d, int op, int six, double* __restrict__ o) {
  EB_LOOP(eb, e) {
    int c[3];
    eb.coords(e, c);
    int lo = -eb.ge[d], hi = eb.n[d] + eb.ge[d], t = c[d];
    long long s = eb.stride(d);
    int r = six ? 3 : 2;
    double nan = __longlong_as_double(0x7ff8000000000000LL);
    double v = nan;
    if (op == 0) {
      if (t - r >= lo && t + r < hi && !isnan(f[e - r * s]) && !isnan(f[e + r * s]))
        v = six ? d6(f[e - 3 * s], f[e - 2 * s], f[e - s], f[e + s], f[e + 2 * s], f[e + 3 * s])
                : d4(f[e - 2 * s], f[e - s], f[e + s], f[e + 2 * s]);
    } else {
      if (t - r + 1 >= lo && t + r < hi && !isnan(f[e - (r - 1) * s]) && !isnan(f[e + r * s])) {
        if (six)
          v = (37.0 / 60.0) * (f[e] + f[e + s]) - (8.0 / 60.0) * (f[e - s] + f[e + 2 * s]) +
              (1.0 / 60.0) * (f[e - 2 * s] + f[e + 3 * s]);
        else
          v = (7.0 / 12.0) * (f[e] + f[e + s]) - (1.0 / 12.0) * (f[e - s] + f[e + 2 * s]);
      }
    }
    o[e] = v;
  }
}

// o = sa*a (+ sb*b) elementwise with sa, sb in {+1, -1, 0}; kind 1: o = a*b
__global__ void km_lin(EBox eb, const double* __restrict__ a, const double* __restrict__ b, int kind, double* __restrict__ o) {
  EB_LOOP(eb, e) {
    double v;
    if (kind == 0) v = a[e];
    else if (kind == 1) v = a[e] * b[e];
    else if (kind == 2) v = -a[e];
    else v = a[e] - b[e];
    o[e] = v;
  }
}

// volume 1/J: 2D determinant or 3D rule of Sarrus on D_l x_m (dX[l*3+m])
__global__ void km_vol(EBox eb, int nd, const double* __restrict__ d00, const double* __restrict__ d01,
                       const double* __restrict__ d02, const double* __restrict__ d10, const double* __restrict__ d11,
                       const double* __restrict__ d12, const double* __restrict__ d20, const double* __restrict__ d21,
                       const double* __restrict__ d22, double* __restrict__ vol) {
  EB_LOOP(eb, e) {
    double v;
    if (nd == 1) v = d00[e];
    else if (nd == 2) v = d00[e] * d11[e] - d10[e] * d01[e];
    else {
      // a_mn = d x_m / d xi_n
      double a11 = d00[e], a12 = d10[e], a13 = d20[e];
      double a21 = d01[e], a22 = d11[e], a23 = d21[e];
      double a31 = d02[e], a32 = d12[e], a33 = d22[e];
      v = a11 * (a22 * a33 - a23 * a32) - a12 * (a21 * a33 - a23 * a31) + a13 * (a21 * a32 - a22 * a31);
    }
    vol[e] = v;
  }
}

// copy onto the padded metric box of the kernels (PM layers): field -> plane
__global__ void km_store(EBox eb, DevGrid g, const double* __restrict__ f, int recip, double* __restrict__ plane) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.NP; e += (long long)gridDim.x * blockDim.x) {
    int c[3];
    c[0] = (int)(e % g.P[0]);
    long long r = e / g.P[0];
    c[1] = (int)(r % g.P[1]);
    c[2] = (int)(r / g.P[1]);
    for (int d = 0; d < 3; ++d) c[d] -= (d < g.nd ? PM : 0);
    double v = f[eb.at(c[0], c[1], c[2])];
    plane[e] = recip ? 1.0 / v : v;
  }
}
// LAD displacement 0.5 (x_{+1} - x_{-1}) along l, component m
__global__ void km_disp(EBox eb, DevGrid g, const double* __restrict__ X, int l, double* __restrict__ plane) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.NP; e += (long long)gridDim.x * blockDim.x) {
    int c[3];
    c[0] = (int)(e % g.P[0]);
    long long r = e / g.P[0];
    c[1] = (int)(r % g.P[1]);
    c[2] = (int)(r / g.P[1]);
    for (int d = 0; d < 3; ++d) c[d] -= (d < g.nd ? PM : 0);
    long long q = eb.at(c[0], c[1], c[2]);
    long long s = eb.stride(l);
    plane[e] = 0.5 * (X[q + s] - X[q - s]);
  }
}

// C6 compact derivative along d (the operator of the LAD-C6 flux divergence),
// one thread per line of the extended box, written over the E4 values km_op
// left in o.  Non-periodic d: rows [0, n-1], explicit E4 rows at both ends
// (reading -2 .. n+1), interior rows (1/3, 1, 1/3) with the C6 right-hand
// side; Thomas elimination.  Periodic d: the cyclic system (Sherman-Morrison)
// on f minus its linear trend along the line (detrend = 1, a coordinate:
// T = f_n - f_0), plus T/n; the extended nodes by wrapping.  A line with a
// NaN in -2 .. n+1 is left as it is.  scr: 4 (n + 4) doubles per line.
__global__ void km_c6(EBox eb, const double* __restrict__ f, int d, int periodic, int detrend,
                      double* __restrict__ o, double* __restrict__ scr) {
  const int n = eb.n[d], g = eb.ge[d];
  const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;  // transverse directions
  const long long nl = (long long)eb.PE[a1] * eb.PE[a2];
  const long long s = eb.stride(d);
  const double a = 1.0 / 3.0;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < nl; L += (long long)gridDim.x * blockDim.x) {
    int c[3];
    c[d] = 0;
    c[a1] = (int)(L % eb.PE[a1]) - eb.ge[a1];
    c[a2] = (int)(L / eb.PE[a1]) - eb.ge[a2];
    const long long q0 = eb.at(c[0], c[1], c[2]);
    bool ok = true;
    for (int t = -2; t <= n + 1; ++t) ok = ok && !isnan(f[q0 + (long long)t * s]);
    if (!ok) continue;
    const int m = n;
    double* r = scr + L * 4 * (long long)(n + 4);
    double* cp = r + (n + 4);
    double* dp = cp + (n + 4);
    double* z = dp + (n + 4);
    if (!periodic) {
      const double* fl = f + q0;
      r[0] = d4(fl[-2 * s], fl[-s], fl[s], fl[2 * s]);
      r[m - 1] = d4(fl[(m - 3) * s], fl[(m - 2) * s], fl[m * s], fl[(m + 1) * s]);
      for (int i = 1; i < m - 1; ++i) {
        const double* p = fl + (long long)i * s;
        r[i] = (7.0 / 9.0) * (p[s] - p[-s]) + (1.0 / 36.0) * (p[2 * s] - p[-2 * s]);
      }
      // Thomas: closure rows decoupled (a = 0 there), unit diagonal
      cp[0] = 0.0 / 1.0;
      dp[0] = r[0] / 1.0;
      for (int i = 1; i < m; ++i) {
        const double ai = i == m - 1 ? 0.0 : a, ci = i == m - 1 ? 0.0 : a;
        const double den = 1.0 - ai * cp[i - 1];
        cp[i] = ci / den;
        dp[i] = (r[i] - ai * dp[i - 1]) / den;
      }
      double x = dp[m - 1];
      o[q0 + (long long)(m - 1) * s] = x;
      for (int i = m - 2; i >= 0; --i) {
        x = dp[i] - cp[i] * x;
        o[q0 + (long long)i * s] = x;
      }
      continue;
    }
    const double T = detrend ? f[q0 + (long long)n * s] - f[q0] : 0.0;
    // detrended values at -2 .. n+1 in z (z[t + 2])
    for (int t = -2; t <= n + 1; ++t) z[t + 2] = f[q0 + (long long)t * s] - T * (double)t / (double)n;
    for (int i = 0; i < m; ++i) {
      const double* p = z + i + 2;
      r[i] = (7.0 / 9.0) * (p[1] - p[-1]) + (1.0 / 36.0) * (p[2] - p[-2]);
    }
    // Sherman-Morrison: T + u v^T, u = (gam, 0 .. 0, a), v = (1, 0 .. 0, a / gam)
    const double gam = -1.0;
    auto diag = [&](int i) { return i == 0 ? 1.0 - gam : (i == m - 1 ? 1.0 - a * a / gam : 1.0); };
    auto sub = [&](int i) { return i == 0 ? 0.0 : a; };
    auto sup = [&](int i) { return i == m - 1 ? 0.0 : a; };
    cp[0] = sup(0) / diag(0);
    dp[0] = r[0] / diag(0);
    for (int i = 1; i < m; ++i) {
      const double den = diag(i) - sub(i) * cp[i - 1];
      cp[i] = sup(i) / den;
      dp[i] = (r[i] - sub(i) * dp[i - 1]) / den;
    }
    // x in r (overwrites the right-hand side), then z = T^{-1} u with the same cp
    r[m - 1] = dp[m - 1];
    for (int i = m - 2; i >= 0; --i) r[i] = dp[i] - cp[i] * r[i + 1];
    {
      const double u0 = gam;
      dp[0] = u0 / diag(0);
      for (int i = 1; i < m; ++i) {
        const double den = diag(i) - sub(i) * cp[i - 1];
        const double ui = i == m - 1 ? a : 0.0;
        dp[i] = (ui - sub(i) * dp[i - 1]) / den;
      }
      z[m - 1] = dp[m - 1];
      for (int i = m - 2; i >= 0; --i) z[i] = dp[i] - cp[i] * z[i + 1];
    }
    const double fact = (r[0] + a * r[m - 1] / gam) / (1.0 + z[0] + a * z[m - 1] / gam);
    for (int i = 0; i < m; ++i) o[q0 + (long long)i * s] = (r[i] - fact * z[i]) + T / (double)n;
    for (int t = 1; t <= g; ++t) {
      int w0 = (-t) % n;
      if (w0 < 0) w0 += n;
      o[q0 - (long long)t * s] = o[q0 + (long long)w0 * s];
      o[q0 + (long long)(n - 1 + t) * s] = o[q0 + (long long)((n - 1 + t) % n) * s];
    }
  }
}

// X - s0 i - s1 j - s2 k: the periodic part of a coordinate (its linear trends
// across the periodic directions removed)
__global__ void km_detrend(EBox eb, const double* __restrict__ X, double s0, double s1, double s2,
                           double* __restrict__ o) {
  EB_LOOP(eb, e) {
    int c[3];
    eb.coords(e, c);
    o[e] = ((X[e] - s0 * (double)c[0]) - s1 * (double)c[1]) - s2 * (double)c[2];
  }
}

// o = (o + d1 * s1) - d2 * s2: the trend terms of the Thomas-Lombard metrics
__global__ void km_trend(EBox eb, const double* __restrict__ d1, double s1, const double* __restrict__ d2, double s2,
                         double* __restrict__ o) {
  EB_LOOP(eb, e) { o[e] = (o[e] + d1[e] * s1) - d2[e] * s2; }
}

}  // namespace cgk
