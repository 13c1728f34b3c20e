"""The mixed form converts between binary64 and binary32 with integer
operations (round to nearest, ties to even, from the IEEE 754 formats) instead
of the hardware conversion.  Both directions must return exactly what the
hardware conversion returns, for every class of input: random bit patterns
over all exponents, the ties and near-ties of the rounding, the ends of the
binary32 normal range, subnormal results, signed zeros, infinities and NaN.
numpy's conversions (round to nearest even) are checked alongside."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18042_gb300 import _native as nat
    return nat


def _doubles(rng):
    out = [rng.integers(0, 2 ** 64, size=400000, dtype=np.uint64).view(np.float64)]
    # every binary64 exponent that lands near the binary32 range, random fractions
    e = rng.integers(800, 1250, size=400000, dtype=np.uint64)
    frac = rng.integers(0, 2 ** 52, size=400000, dtype=np.uint64)
    sign = rng.integers(0, 2, size=400000, dtype=np.uint64) << np.uint64(63)
    out.append((sign | (e << np.uint64(52)) | frac).view(np.float64))
    # ties and neighbours of ties: a float plus half its ulp, +-1 binary64 ulp
    f = rng.integers(0, 2 ** 32, size=100000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    f = f[np.isfinite(f)].astype(np.float64)
    half = np.abs(f) * 2.0 ** -24
    for t in (f + half, f - half):
        out += [t, np.nextafter(t, np.inf), np.nextafter(t, -np.inf)]
    fmax = float(np.finfo(np.float32).max)
    specials = [0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, fmax, -fmax,
                fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -24), np.nextafter(fmax * (1 + 2.0 ** -24), 0),
                2.0 ** -126, 2.0 ** -127, 2.0 ** -149, 2.0 ** -150, 3 * 2.0 ** -151, 2.0 ** -151,
                np.nextafter(2.0 ** -150, 1), np.nextafter(2.0 ** -126, 0), 1e-300, -1e-300, 1e300, 5e-324]
    out.append(np.array(specials + [-x for x in specials]))
    return np.concatenate(out)


def _floats(rng, n):
    r = rng.integers(0, 2 ** 32, size=n - 10, dtype=np.uint64).astype(np.uint32)
    specials = np.array([0x00000000, 0x80000000, 0x00000001, 0x807fffff, 0x00800000, 0x7f7fffff,
                         0x7f800000, 0xff800000, 0x7fc00000, 0x3f800000], dtype=np.uint32)
    return np.concatenate([r, specials]).view(np.float32)


def test_integer_pipe_conversions_equal_the_hardware(lib):
    rng = np.random.default_rng(11)
    d = _doubles(rng)
    n = d.size
    f = _floats(rng, n)
    d_in = torch.as_tensor(d, device="cuda")
    f_in = torch.as_tensor(f, device="cuda")
    f_out = torch.empty(n, dtype=torch.float32, device="cuda")
    d_out = torch.empty(n, dtype=torch.float64, device="cuda")
    lib.check(lib.lib().cg_convert_check(d_in.data_ptr(), f_out.data_ptr(), f_in.data_ptr(), d_out.data_ptr(), n,
                                         None))
    torch.cuda.synchronize()
    hw_f = d_in.to(torch.float32)
    hw_d = f_in.to(torch.float64)
    got_f, got_d = f_out.cpu().numpy(), d_out.cpu().numpy()
    nan_f, nan_d = np.isnan(got_f), np.isnan(got_d)
    assert np.array_equal(nan_f, np.isnan(d)) and np.array_equal(nan_d, np.isnan(f))
    assert np.array_equal(got_f.view(np.uint32)[~nan_f], hw_f.cpu().numpy().view(np.uint32)[~nan_f])
    assert np.array_equal(got_d.view(np.uint64)[~nan_d], hw_d.cpu().numpy().view(np.uint64)[~nan_d])
    with np.errstate(over="ignore", invalid="ignore"):
        ref_f = d.astype(np.float32)
        ref_d = f.astype(np.float64)
    assert np.array_equal(got_f.view(np.uint32)[~nan_f], ref_f.view(np.uint32)[~nan_f])
    assert np.array_equal(got_d.view(np.uint64)[~nan_d], ref_d.view(np.uint64)[~nan_d])


def test_zero_length_and_null_arguments(lib):
    assert lib.lib().cg_convert_check(None, None, None, None, 0, None) == 0
    assert lib.lib().cg_convert_check(None, None, None, None, 4, None) == -1
