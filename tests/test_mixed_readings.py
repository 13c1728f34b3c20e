"""The two rearrangements the mixed form's FP64 accumulation rests on, checked on
the CPU against the paper's forms (the oracle's filter, the Shu-Osher stages).

* TVD-RK3 (Sec. 2.1) in increment form: with k_s = dt L(u^(s-1)),
  u1 = un + k1, u2 = un + (k1 + k2)/4, u^(n+1) = un + (k1 + k2)/6 + 2 k3/3
  equals the Shu-Osher stages u2 = 3/4 un + 1/4 (u1 + k2),
  u^(n+1) = 1/3 un + 2/3 (u2 + k3).
* The implicit filter of LAD-C6 (Algorithm 1) in increment form: D = Qf - Q
  solves the filter's tridiagonal system with the right-hand side
  sum_n c_n (Q_{i+n} + Q_{i-n} - 2 Q_i), c_1 = a_1/2 - alpha, c_n = a_n/2,
  because the filter keeps constants (a_0 + a_1 + ... + a_4 = 1 + 2 alpha).
  Formed in FP32 from a hi/lo split of each FP64 value (hi differences
  first), D is accurate to about 1e-11 of the field or better; from the FP32
  images alone only to about 1e-8."""
import numpy as np

import oracle


def test_rk3_increment_form_is_the_shu_osher_form():
    rng = np.random.default_rng(3)
    un = rng.uniform(0.5, 2.0, 1000)
    k1, k2, k3 = (rng.normal(0, 1e-2, 1000) for _ in range(3))
    u1 = un + k1
    u2_so = 0.75 * un + 0.25 * (u1 + k2)
    u3_so = (1.0 / 3.0) * un + (2.0 / 3.0) * (u2_so + k3)
    u2_inc = un + (k1 + k2) / 4.0
    u3_inc = un + (k1 + k2) / 6.0 + 2.0 * k3 / 3.0
    assert np.abs(u2_inc - u2_so).max() <= 4e-16 * np.abs(un).max()
    assert np.abs(u3_inc - u3_so).max() <= 4e-16 * np.abs(un).max()


def _filter_coefficients(alpha):
    # the eighth-order filter's right-hand coefficients a_0..a_4 (Gaitonde & Visbal form)
    return np.array([(93 + 70 * alpha) / 128, (7 + 18 * alpha) / 16, (-7 + 14 * alpha) / 32,
                     (1 - 2 * alpha) / 16, (-1 + 2 * alpha) / 128])


def _increment_rhs(f, alpha, n):
    a = _filter_coefficients(alpha)
    c = np.array([a[1] / 2 - alpha, a[2] / 2, a[3] / 2, a[4] / 2])
    idx = np.arange(n)
    r = np.zeros(n)
    for k in range(1, 5):
        r += c[k - 1] * (f[(idx + k) % n] + f[(idx - k) % n] - 2 * f[idx])
    return r


def test_filter_coefficients_keep_constants():
    for alpha in (0.3, 0.45, 0.49):
        a = _filter_coefficients(alpha)
        assert abs(a[0] + a[1:].sum() - (1 + 2 * alpha)) <= 1e-15


def test_filter_increment_form_equals_the_oracle_filter():
    n, alpha = 96, 0.45
    rng = np.random.default_rng(7)
    x = np.arange(n) / n
    f = 1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.05 * rng.standard_normal(n)
    fpad = np.concatenate([f[-4:], f, f[:4]])
    ref = oracle.line_op("FILTER", fpad, 4, periodic=True, alpha_f=alpha)[4:4 + n]
    D = oracle.tridiag(alpha, _increment_rhs(f, alpha, n), True)
    assert np.abs(f + D - ref).max() <= 1e-14 * np.abs(f).max()


def test_filter_increment_from_a_hi_lo_split_keeps_its_precision():
    """Smooth fields (one on a large mean): the increment formed in FP32 from
    hi/lo pairs is within 1e-10 of the field's size of the FP64 increment;
    formed from the FP32 images alone it is off by more than 1e-9."""
    n, alpha = 128, 0.45
    x = np.arange(n) / n
    a = _filter_coefficients(alpha)
    c = np.array([a[1] / 2 - alpha, a[2] / 2, a[3] / 2, a[4] / 2], dtype=np.float32)
    idx = np.arange(n)
    for f in (100.0 + 1e-2 * np.sin(2 * np.pi * 3 * x) + 1e-4 * np.sin(2 * np.pi * 29 * x),
              1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.02 * np.sin(2 * np.pi * 13 * x)):
        exact = oracle.tridiag(alpha, _increment_rhs(f, alpha, n), True)
        hi = f.astype(np.float32)
        lo = (f - hi.astype(np.float64)).astype(np.float32)

        def rhs32(use_lo):
            r = np.zeros(n, dtype=np.float32)
            for k in range(1, 5):
                p, m = (idx + k) % n, (idx - k) % n
                d = (hi[p] - hi[idx]) + (hi[m] - hi[idx])
                if use_lo:
                    d = d + ((lo[p] + lo[m]) - np.float32(2) * lo[idx])
                r = r + c[k - 1] * d
            return r.astype(np.float64)

        size = np.abs(f).max()
        split = oracle.tridiag(alpha, rhs32(True), True)
        plain = oracle.tridiag(alpha, rhs32(False), True)
        assert np.abs(split - exact).max() <= 1e-10 * size
        assert np.abs(plain - exact).max() >= 1e-9 * size
