"""The integer-pipe FP64 <-> FP32 conversions of the FP32 forms (numa_convert_f64_f32,
numa_convert_f32_f64) against IEEE-754 conversion: numpy's on the host (round to nearest,
ties to even; exact widening) and the GPU's own conversion instructions (torch casts), bit
for bit, on seeded bit patterns that cover every exponent, the rounding ties, FP32
subnormals and underflow, overflow to infinity, zeros, infinities and NaN."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _f64_patterns(n=1 << 20):
    rng = np.random.Generator(np.random.PCG64(77))
    b = rng.integers(0, 2 ** 64, n, dtype=np.uint64)
    k = n // 8
    sign_frac = b & np.uint64(0x800FFFFFFFFFFFFF)
    # exponents across FP32's whole range and beyond (subnormal results, overflow)
    e = rng.integers(1023 - 160, 1023 + 140, n, dtype=np.uint64)
    b[k:4 * k] = sign_frac[k:4 * k] | (e[k:4 * k] << np.uint64(52))
    # exact ties and near-ties of the 29 dropped bits
    tie = (sign_frac & ~np.uint64(0x1FFFFFFF)) | np.uint64(0x10000000)
    b[4 * k:5 * k] = tie[4 * k:5 * k] | (e[4 * k:5 * k] << np.uint64(52))
    b[5 * k:6 * k] = b[4 * k:5 * k] + rng.integers(-2, 3, k).astype(np.int64).view(np.uint64)
    x = b.view(np.float64)
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0,
                         float(np.finfo(np.float32).max), float(np.finfo(np.float32).max) * (1 + 2 ** -25),
                         float(np.finfo(np.float32).max) * (1 + 2 ** -24), 2.0 ** -126, 2.0 ** -149,
                         2.0 ** -150, 2.0 ** -150 * (1 + 2 ** -40), 3 * 2.0 ** -151, 2.0 ** -1074,
                         5e-324, 1e-320, 1e300, -1e300, 0.1, 1.0 / 3.0])
    return np.concatenate([specials, x])


def _same_bits(a, b):
    nan = np.isnan(a) & np.isnan(b)
    return np.all(nan | (a.view(np.uint32 if a.dtype == np.float32 else np.uint64)
                         == b.view(np.uint32 if b.dtype == np.float32 else np.uint64)))


def test_f64_to_f32_is_ieee_round_to_nearest_even():
    import torch
    import paper_1702_04316_gb300 as pkg
    x = _f64_patterns()
    xd = torch.from_numpy(x).cuda()
    got = pkg.convert(xd).cpu().numpy()
    with np.errstate(over="ignore", invalid="ignore"):
        ref = x.astype(np.float32)
    assert np.array_equal(np.isnan(got), np.isnan(x))
    assert _same_bits(got, ref)
    assert _same_bits(got, xd.float().cpu().numpy())


def test_f32_to_f64_is_exact():
    import torch
    import paper_1702_04316_gb300 as pkg
    rng = np.random.Generator(np.random.PCG64(78))
    u = rng.integers(0, 2 ** 32, 1 << 20, dtype=np.uint64).astype(np.uint32)
    u[:4096] &= np.uint32(0x807FFFFF)          # subnormals and zeros
    u[4096:4200] |= np.uint32(0x7F800000)       # infinities and NaN
    x = np.concatenate([np.array([0.0, -0.0, np.inf, -np.inf, np.nan], np.float32), u.view(np.float32)])
    xd = torch.from_numpy(x).cuda()
    got = pkg.convert(xd).cpu().numpy()
    assert got.dtype == np.float64
    with np.errstate(invalid="ignore"):
        assert _same_bits(got, x.astype(np.float64))
    assert _same_bits(got, xd.double().cpu().numpy())


def test_convert_rejects_bad_arguments():
    import torch
    import paper_1702_04316_gb300 as pkg
    with pytest.raises(ValueError):
        pkg.convert(torch.zeros(4, dtype=torch.float16, device="cuda"))
    assert pkg.convert(torch.zeros(0, dtype=torch.float64, device="cuda")).numel() == 0


def test_reciprocal_within_one_ulp_of_division():
    """The right-hand side's 1 / rho (Newton's method from an FP32 seed with a third-order
    step) against the IEEE quotient (numpy on the host, and the GPU's own division): at most
    one unit in the last place apart over densities and over every FP32-normal exponent, and
    the quotient itself outside that range."""
    import torch
    import paper_1702_04316_gb300 as pkg
    rng = np.random.Generator(np.random.PCG64(79))
    dens = rng.uniform(0.01, 2.0, 1 << 20)                 # densities, kg / m^3
    b = rng.integers(0, 2 ** 64, 1 << 20, dtype=np.uint64)
    e = rng.integers(1023 - 126, 1023 + 127, b.size, dtype=np.uint64)
    wide = ((b & np.uint64(0x800FFFFFFFFFFFFF)) | (e << np.uint64(52))).view(np.float64)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 2.0 ** -126, 2.0 ** -127,
                        2.0 ** 126, 2.0 ** 127, 2.0 ** 128, 1e-300, 1e300, 5e-324, 3.0, 0.1])
    x = np.concatenate([special, dens, wide])
    xd = torch.from_numpy(x).cuda()
    got = pkg.reciprocal(xd).cpu().numpy()
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        ref = 1.0 / x
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    fin = np.isfinite(ref) & (ref != 0)
    ulp = np.abs(got[fin].view(np.int64) - ref[fin].view(np.int64))
    assert ulp.max() <= 1
    assert np.array_equal(got[~fin & ~np.isnan(ref)], ref[~fin & ~np.isnan(ref)])
    hw = (1.0 / xd).cpu().numpy()
    assert np.abs(got[fin].view(np.int64) - hw[fin].view(np.int64)).max() <= 1
    assert (ulp == 0).mean() > 0.5                          # mostly the correctly rounded value
