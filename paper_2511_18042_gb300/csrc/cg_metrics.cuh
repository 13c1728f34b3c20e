// Grid metrics on the device (once per solver), Sec. 2.1: xi_hat = xi_x / J.
//
// Node metrics come from derivatives D of the node coordinates, D being the
// scheme's own explicit first derivative (sixth order for C-GBR, E4 for LAD-E4
// and the hybrid) so that the discrete metric identities hold for the flux
// divergence actually used (freestream preservation).  2D: xi_x = y_eta,
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

}  // namespace cgk
