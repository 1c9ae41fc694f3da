"""The library's own FP64 elementary functions (nsfr_math_eval) against numpy's
(host libm) values and against CUDA's own log/exp on the same GPU.

log and exp are table-driven (Tang's method) and the reciprocals start from an
FP32 seed; the kernels compute the entropy variables, the face states and the
two-point fluxes with them, so their error bounds are checked here directly:
  log   |y - ln x| <= 2 ulp(max(|ln x|, 1/2))  (absolute accuracy near x = 1)
  exp   |y - e^x|  <= 2 ulp(e^x)
  rcp   |y - 1/x|  <= 1 ulp(1/x)
  rcp1  |y x - 1|  <= 2^-43
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(20231207)


def _eval(fn, x):
    from paper_2312_07725_gb300 import nsfr
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    y = nsfr.math_eval(fn, xd)
    torch.cuda.synchronize()
    return y.cpu().numpy(), xd


def _log_inputs():
    m = RNG.uniform(1.0, 2.0, 200_000)
    k = RNG.integers(-1020, 1020, 200_000)
    near1 = 1.0 + RNG.uniform(-0.05, 0.05, 50_000)
    physical = np.concatenate([RNG.uniform(0.5, 3.0, 50_000), RNG.uniform(50.0, 100.0, 50_000),
                               RNG.uniform(1e-3, 1e-1, 50_000)])
    edges = np.array([1.0, 2.0, 0.5, np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0), 2.0 ** -1022, 1.7e308])
    return np.concatenate([np.ldexp(m, k), near1, physical, edges])


def test_log_within_two_ulp_of_libm_and_cuda():
    x = _log_inputs()
    y, xd = _eval("log", x)
    ref = np.log(x)
    scale = np.spacing(np.maximum(np.abs(ref), 0.5))
    assert np.max(np.abs(y - ref) / scale) <= 2.0
    cuda = torch.log(xd).cpu().numpy()
    assert np.max(np.abs(y - cuda) / scale) <= 3.0


def test_log_special_arguments_follow_the_ieee_results():
    x = np.array([0.0, -0.0, -1.0, np.inf, np.nan, 5e-324, 1e-310])
    y, _ = _eval("log", x)
    with np.errstate(divide="ignore", invalid="ignore"):
        ref = np.log(x)
    assert np.array_equal(np.isnan(y), np.isnan(ref))
    fin = np.isfinite(ref)
    assert np.all(y[~np.isnan(ref) & ~fin] == ref[~np.isnan(ref) & ~fin])
    assert np.allclose(y[fin], ref[fin], rtol=1e-15, atol=0)


def test_exp_within_two_ulp_of_libm_and_cuda():
    x = np.concatenate([RNG.uniform(-699.0, 699.0, 200_000), RNG.uniform(-1.0, 1.0, 100_000),
                        RNG.uniform(-10.0, 10.0, 100_000), np.array([0.0, -0.0, 1.0, -1.0, 1e-20, 699.9])])
    y, xd = _eval("exp", x)
    ref = np.exp(x)
    assert np.max(np.abs(y - ref) / np.spacing(ref)) <= 2.0
    cuda = torch.exp(xd).cpu().numpy()
    assert np.max(np.abs(y - cuda) / np.spacing(ref)) <= 3.0


def test_exp_special_arguments_follow_the_ieee_results():
    x = np.array([750.0, -750.0, np.inf, -np.inf, np.nan, 709.0, -708.0])
    y, _ = _eval("exp", x)
    with np.errstate(over="ignore"):
        ref = np.exp(x)
    assert np.array_equal(np.isnan(y), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert np.allclose(y[ok], ref[ok], rtol=1e-15, atol=0)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_reciprocals_meet_their_bounds(sign):
    m = RNG.uniform(1.0, 2.0, 300_000)
    k = RNG.integers(-1000, 1000, 300_000)
    x = sign * np.concatenate([np.ldexp(m, k), RNG.uniform(0.01, 100.0, 100_000), np.array([1.0, 2.0, 3.0, 71.4])])
    y, _ = _eval("rcp", x)
    ref = 1.0 / x
    assert np.max(np.abs(y - ref) / np.spacing(np.abs(ref))) <= 1.0
    y1, _ = _eval("rcp1", x)
    assert np.max(np.abs(y1 * x - 1.0)) <= 2.0 ** -43


def test_math_eval_rejects_host_buffers_and_unknown_functions():
    from paper_2312_07725_gb300 import NSFRError, nsfr
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(NSFRError):
        nsfr.math_eval("log", x.cpu(), torch.empty(4, dtype=torch.float64))
    with pytest.raises(KeyError):
        nsfr.math_eval("sin", x)


def _ff_round(x):
    """The float-float value the library's functions see: x split into the nearest
    float and the nearest float of the remainder, summed back exactly."""
    hi = x.astype(np.float32).astype(np.float64)
    lo = (x - hi).astype(np.float32).astype(np.float64)
    return hi + lo


def test_float_float_log_within_2_pow_minus_44_of_libm():
    """ff_log (FP32-bulk kernels): |y - ln x| <= 2^-44 max(|ln x|, 0.7) over the
    float-normal range the kernels use (densities, pressures, 2 beta)."""
    m = RNG.uniform(1.0, 2.0, 200_000)
    k = RNG.integers(-60, 60, 200_000)
    near1 = 1.0 + RNG.uniform(-0.02, 0.02, 100_000)
    physical = np.concatenate([RNG.uniform(0.5, 3.0, 50_000), RNG.uniform(50.0, 100.0, 50_000),
                               RNG.uniform(1e-3, 1e-1, 50_000)])
    x = _ff_round(np.concatenate([np.ldexp(m, k), near1, physical, [1.0, 2.0, 0.5, 0.75]]))
    y, _ = _eval("log_ff", x)
    ref = np.log(x)
    err = np.abs(y - ref) / np.maximum(np.abs(ref), 0.7)
    assert err.max() <= 2.0 ** -44, err.max()
    assert abs(y[-4]) < 2.0 ** -48  # ln 1: the float r^3 q term leaves ~2^-51


def test_float_float_exp_within_2_pow_minus_44_of_libm():
    # down to -60: below about -64 the trailing float of e^x is subnormal
    x = _ff_round(np.concatenate([RNG.uniform(-60.0, 80.0, 200_000), RNG.uniform(-1.0, 1.0, 100_000),
                                  [0.0, 1.0, -1.0, np.log(2.0)]]))
    y, _ = _eval("exp_ff", x)
    ref = np.exp(x)
    err = np.abs(y - ref) / ref
    assert err.max() <= 2.0 ** -44, err.max()
    assert y[-4] == 1.0


def _pack_pairs(hi, lo):
    """float32 pairs as the 64 bits of float64 values (hi in the high word)."""
    bits = (hi.astype(np.float32).view(np.uint32).astype(np.uint64) << np.uint64(32)) | \
        lo.astype(np.float32).view(np.uint32).astype(np.uint64)
    return bits.view(np.float64)


def test_join_of_float_pairs_is_their_exact_sum():
    """ff_join_i (integer-pipe join of a float-float pair, used by the FP64 volume
    kernels): y equals hi + lo exactly whenever that sum fits a double, and is
    within 2^-52 of it otherwise, including the borrow below a power of two and the
    carry past an all-ones significand."""
    from fractions import Fraction
    n = 6000
    e = RNG.integers(-60, 100, n)
    hi = np.ldexp(RNG.uniform(1.0, 2.0, n), e).astype(np.float32) * RNG.choice([-1.0, 1.0], n).astype(np.float32)
    k = RNG.integers(0, 45, n)
    lo = (hi.astype(np.float64) * RNG.uniform(-0.49, 0.49, n) * np.ldexp(1.0, -k)).astype(np.float32)
    lo[np.abs(lo) < np.float32(2.0 ** -126)] = 0.0  # subnormal floats count as zero: not tested here
    pw = np.ldexp(1.0, RNG.integers(-60, 60, 2000)).astype(np.float32)  # borrow: hi = 2^e, lo < 0
    lo_pw = (-pw.astype(np.float64) * RNG.uniform(1e-9, 0.49, 2000)).astype(np.float32)
    ones = (np.ldexp(2.0 - 2.0 ** -23, RNG.integers(-60, 60, 2000))).astype(np.float32)  # carry
    lo_ones = (ones.astype(np.float64) * RNG.uniform(1e-9, 0.49, 2000)).astype(np.float32)
    special_hi = np.array([1.0, -1.0, 0.0, 3.0, 1.5, -2.0], np.float32)
    special_lo = np.array([0.0, 0.0, 0.0, 2.0 ** -30, -2.0 ** -40, 2.0 ** -80], np.float32)
    H = np.concatenate([hi, pw, ones, special_hi])
    L = np.concatenate([lo, lo_pw, lo_ones, special_lo])
    y, _ = _eval("join", _pack_pairs(H, L))
    for h, l, v in zip(H.astype(np.float64), L.astype(np.float64), y):
        exact = Fraction(h) + Fraction(l)
        if float(exact) == exact:
            assert v == float(exact), (h, l, v)
        else:
            assert abs(Fraction(v) - exact) <= abs(exact) * Fraction(1, 2 ** 52), (h, l, v)


def _logmean1_ref(x):
    from decimal import Decimal, getcontext
    getcontext().prec = 50
    out = np.empty_like(x)
    for i, v in enumerate(x):
        d = Decimal(float(v))
        out[i] = 1.0 if d == 1 else float((d - 1) / d.ln())
    return out


def test_logmean_series_branch_within_two_ulp():
    """The volume kernels' logarithmic mean (x - 1)/ln x of x and 1 against its
    closed form in 50-digit decimal arithmetic.  On the series branch
    (u = ((x-1)/(x+1))^2 < 1e-4, the float-float tail plus one FP64 FMA) it is
    within 2 ulp; on the log branch, (x - 1)/ln x with the library's log, within
    the log's absolute accuracy divided by |ln x| (1e-14 relative near the
    threshold)."""
    near = 1.0 + np.concatenate([RNG.uniform(-0.021, 0.021, 4000), RNG.uniform(-1e-6, 1e-6, 500),
                                 np.array([0.0, 2.0 ** -52, -2.0 ** -53, 0.0198, 0.0202, -0.0198, -0.0194])])
    far = np.concatenate([RNG.uniform(0.1, 0.97, 500), RNG.uniform(1.03, 10.0, 500)])
    x = np.concatenate([near, far])
    y, _ = _eval("logmean1", x)
    ref = _logmean1_ref(x)
    u = ((x - 1.0) / (x + 1.0)) ** 2
    series = u < 0.99e-4
    logb = u > 1.01e-4
    assert series.sum() > 3000 and logb.sum() > 1000
    ulps = np.abs(y - ref) / np.spacing(np.abs(ref))
    assert np.max(ulps[series]) <= 2.0, np.max(ulps[series])
    assert np.max(np.abs(y - ref)[logb] / ref[logb]) <= 1e-14


def _unpack_pairs(y):
    bits = y.view(np.uint64)
    hi = (bits >> np.uint64(32)).astype(np.uint32).view(np.float32)
    lo = (bits & np.uint64(0xffffffff)).astype(np.uint32).view(np.float32)
    return hi, lo


def test_split_into_nearest_float_and_truncated_remainder():
    """ff_split_i (integer-pipe split of a double, used by the log, exp and all float-float
    paths): hi is the float nearest x (ties away from zero), lo the leading 24 bits of the
    exact remainder x - hi (truncated toward zero), so |x - hi - lo| < 2^-48 |x|; a remainder
    below the FP32 normal range gives lo = 0."""
    from fractions import Fraction
    import math
    n = 4000
    x = np.ldexp(RNG.uniform(1.0, 2.0, n), RNG.integers(-90, 90, n)) * RNG.choice([-1.0, 1.0], n)
    f = np.float32(RNG.uniform(1.0, 2.0, 200)).astype(np.float64)
    half_ulp = np.ldexp(1.0, np.frexp(f)[1] - 25)     # exact ties between two floats
    x = np.concatenate([x, f, -f, f + half_ulp, -(f + half_ulp), np.array([1.0, -3.0, 1e-30, 7e29])])
    y, _ = _eval("split", x)
    hi, lo = _unpack_pairs(y)
    for xv, h, l in zip(x, hi.astype(np.float64), lo.astype(np.float64)):
        X = Fraction(xv)
        f0 = np.float32(xv)                      # nearest float, ties to even
        want = Fraction(float(f0))
        if want != X:                            # the float on X's other side
            f1 = np.nextafter(f0, np.float32(-np.inf) if want > X else np.float32(np.inf))
            other = Fraction(float(f1))
            if abs(X - other) == abs(X - want) and abs(other) > abs(want):
                want = other                     # a tie goes away from zero
        assert Fraction(h) == want, (xv, h)
        R = X - want
        if R == 0:
            assert l == 0.0
        else:
            e = math.floor(math.log2(abs(float(R))))
            if Fraction(2) ** e > abs(R):
                e -= 1
            q = math.floor(abs(R) * Fraction(2) ** (23 - e))
            if e < -126:                         # below the FP32 normal range: flushed
                assert l == 0.0, (xv, l)
                continue
            assert Fraction(l) == (1 if R > 0 else -1) * Fraction(q) / Fraction(2) ** (23 - e), (xv, l)
        assert abs(X - Fraction(h) - Fraction(l)) < abs(X) * Fraction(1, 2 ** 48)


def test_int_to_double_is_exact():
    """i2d_i (integer-pipe int-to-double conversion, used by the log's and exp's
    reductions): exact for every 32-bit int."""
    ints = np.concatenate([RNG.integers(-2 ** 31, 2 ** 31, 20000), np.array([0, 1, -1, 2 ** 31 - 1, -2 ** 31, 1023,
                                                                            -1022, 32316, -32316])])
    bits = (np.uint64(0x3ff00000) << np.uint64(32)) | (ints.astype(np.int64) & 0xffffffff).astype(np.uint64)
    y, _ = _eval("i2d", bits.view(np.float64))
    assert np.array_equal(y, ints.astype(np.float64))
