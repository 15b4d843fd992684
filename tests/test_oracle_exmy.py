"""Pins of the oracle's ExMy emulator (Sec. IV-A formats, Sec. V-B
round-to-nearest-even conversion) against facts fixed outside it:
exhaustive code-point round trips, tie-to-even midpoints, the known maxima
of IEEE/OCP formats, library casts (numpy, torch, ml_dtypes) and a
brute-force nearest-code search."""
import numpy as np
import pytest

from paper_2310_07854_gb300 import formats as F

EXTRAS = [F.fmt(5, 9), F.fmt(6, 8), F.fmt(6, 6)]  # Table II per-tensor results
ALL = [f for f in F.search_set() if f != F.FP32] + EXTRAS


def _finite_codes(f, orc):
    codes = np.arange(1 << f.bits, dtype=np.uint32)
    vals = orc.decode(codes, f.E, f.M, f.flags)
    keep = np.isfinite(vals)
    return codes[keep], vals[keep]


@pytest.mark.parametrize("f", ALL, ids=str)
def test_code_points_roundtrip(f, orc):
    """Every finite code decodes to a value that encodes back to itself."""
    codes, vals = _finite_codes(f, orc)
    assert np.all(vals.astype(np.float32).astype(np.float64) == vals)
    back = orc.encode(vals.astype(np.float32), f.E, f.M, f.flags)
    assert np.array_equal(back, codes)
    # magnitudes are strictly increasing in the code (sign-magnitude order)
    pos = codes < (1 << (f.bits - 1))
    assert np.all(np.diff(vals[pos]) > 0)


@pytest.mark.parametrize("f", ALL, ids=str)
def test_midpoints_round_to_even(f, orc):
    codes, vals = _finite_codes(f, orc)
    pos = codes < (1 << (f.bits - 1))
    c, v = codes[pos], vals[pos]
    mid = (v[:-1] + v[1:]) / 2
    m32 = mid.astype(np.float32)
    exact = m32.astype(np.float64) == mid
    assert exact.all()
    got = orc.encode(m32, f.E, f.M, f.flags)
    even = np.where(c[:-1] % 2 == 0, c[:-1], c[1:])
    assert np.array_equal(got, even)
    # one float32 step either side of a midpoint goes to the nearer code
    lo = np.nextafter(m32, np.float32(-np.inf))
    hi = np.nextafter(m32, np.float32(np.inf))
    assert np.array_equal(orc.encode(lo, f.E, f.M, f.flags), c[:-1])
    assert np.array_equal(orc.encode(hi, f.E, f.M, f.flags), c[1:])
    # and negatives mirror positives
    assert np.array_equal(orc.encode(-m32, f.E, f.M, f.flags),
                          even | np.uint32(1 << (f.bits - 1)))


def test_known_maxima(orc):
    known = {(2, 1): 6.0, (3, 2): 28.0, (2, 3): 7.5, (4, 3): 448.0,
             (5, 2): 57344.0, (5, 10): 65504.0,
             (8, 7): float(np.float32(3.3895313892515355e38))}
    for (E, M), v in known.items():
        assert orc.max_finite(E, M) == v, (E, M)
    # smallest subnormals: 2^(2 - 2^(E-1) - M)
    for f in ALL:
        tiny = orc.decode(np.array([1], np.uint32), f.E, f.M, f.flags)[0]
        assert tiny == 2.0 ** (2 - 2 ** (f.E - 1) - f.M)


def test_special_values(orc):
    x = np.array([np.inf, -np.inf, np.nan, 0.0, -0.0, 1e30, -1e30], np.float32)
    # half: IEEE, overflow to Inf, canonical NaN 0x7fff
    h = orc.encode(x, 5, 10)
    assert list(h) == [0x7C00, 0xFC00, 0x7FFF, 0, 0x8000, 0x7C00, 0xFC00]
    # E4M3 (fn, saturating): Inf -> 448, NaN -> 0x7f
    e = orc.encode(x, 4, 3)
    assert list(e) == [0x7E, 0xFE, 0x7F, 0, 0x80, 0x7E, 0xFE]
    # E5M2 saturates: Inf -> 57344 (0x7b)
    assert list(orc.encode(x, 5, 2)) == [0x7B, 0xFB, 0x7F, 0, 0x80, 0x7B, 0xFB]
    # finite-only E2M1: Inf clamps to 6, NaN -> +max (reading)
    assert list(orc.encode(x, 2, 1)) == [0x7, 0xF, 0x7, 0, 0x8, 0x7, 0xF]
    # FP32 is the identity on bits
    bits = np.array([0x7FC00001, 0x00000001, 0x80000000], np.uint32)
    assert np.array_equal(orc.encode(bits.view(np.float32), 8, 23), bits)


def _random_f32(rng, n, lo_exp=-30, hi_exp=20):
    mant = rng.uniform(1, 2, n)
    ex = rng.integers(lo_exp, hi_exp, n)
    s = rng.choice([-1.0, 1.0], n)
    return (s * mant * 2.0 ** ex).astype(np.float32)


def test_half_matches_numpy(orc):
    rng = np.random.default_rng(1)
    x = np.concatenate([_random_f32(rng, 200000, -30, 17),
                        rng.integers(0, 2**32, 200000, dtype=np.uint64)
                        .astype(np.uint32).view(np.float32)])
    x = x[np.isfinite(x)]
    got = orc.encode(x, 5, 10)
    with np.errstate(over="ignore"):  # out-of-range inputs round to +-Inf, as intended
        want = x.astype(np.float16).view(np.uint16).astype(np.uint32)
    assert np.array_equal(got, want)


def test_bf16_and_fp8_match_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = _random_f32(rng, 200000, -140, 127)
    got = orc.encode(x, 8, 7)
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy()
    assert np.array_equal(got, want.astype(np.uint16).astype(np.uint32))
    for (E, M), dt in (((4, 3), torch.float8_e4m3fn), ((5, 2), torch.float8_e5m2)):
        lim = orc.max_finite(E, M)
        xr = x[np.abs(x) <= lim]  # out of range, torch gives NaN/Inf instead of clamping
        got = orc.encode(xr, E, M)
        want = torch.from_numpy(xr).to(dt).view(torch.uint8).numpy().astype(np.uint32)
        assert np.array_equal(got, want), (E, M)


def test_bf16_overflow_matches_torch(orc):
    """At the top of the float32 range bfloat16 rounds to nearest even and
    everything from the midpoint above its maximum up goes to Inf, as torch's
    float32 -> bfloat16 cast does; Inf stays Inf."""
    torch = pytest.importorskip("torch")
    top = np.append(np.arange(0x7F7F0000, 0x7F800000, 7, dtype=np.uint32), np.uint32(0x7F800000))
    x = np.concatenate([top, top | np.uint32(0x80000000)]).view(np.float32)
    got = orc.encode(x, 8, 7)
    want = torch.from_numpy(x.copy()).to(torch.bfloat16).view(torch.int16).numpy()
    assert np.array_equal(got, want.astype(np.uint16).astype(np.uint32))
    assert (got == 0x7F80).sum() > 100 and (got == 0x7F7F).sum() > 100


def test_sub_byte_formats_match_ml_dtypes(orc):
    mld = pytest.importorskip("ml_dtypes")
    rng = np.random.default_rng(3)
    cases = [((2, 1), mld.float4_e2m1fn), ((3, 2), mld.float6_e3m2fn),
             ((2, 3), mld.float6_e2m3fn), ((4, 3), mld.float8_e4m3fn),
             ((5, 2), mld.float8_e5m2)]
    for (E, M), dt in cases:
        lim = orc.max_finite(E, M)
        x = _random_f32(rng, 100000, -12, 8)
        x = x[np.abs(x) <= lim]
        got = orc.encode(x, E, M)
        want = x.astype(dt).view(np.uint8).astype(np.uint32)
        assert np.array_equal(got, want), (E, M)


@pytest.mark.parametrize("f", [f for f in ALL if f.bits <= 8], ids=str)
def test_brute_force_nearest_code(f, orc):
    """Search every code for the nearest value; ties go to the even code;
    beyond the largest finite value the format saturates (or gives Inf)."""
    codes, vals = _finite_codes(f, orc)
    order = np.argsort(vals, kind="stable")
    rng = np.random.default_rng(f.bits * 100 + f.E)
    vmax = vals.max()
    x = np.concatenate([
        rng.uniform(-1.2 * vmax, 1.2 * vmax, 4000),
        rng.uniform(-4, 4, 4000) * vals[vals > 0].min(),
    ]).astype(np.float32)
    got = orc.encode(x, f.E, f.M, f.flags)
    for xi, gi in zip(x.astype(np.float64), got):
        if abs(xi) > vmax:
            want_mag = vmax
            cand = codes[(vals == np.copysign(want_mag, xi))]
            if (f.flags & F.IEEE) and not (f.flags & F.SAT):
                continue  # IEEE overflow: checked in test_special_values
            assert gi == cand[0]
            continue
        dist = np.abs(vals - xi)
        best = dist.min()
        tied = codes[dist == best]
        if len(tied) > 1 and best > 0:
            tied = tied[tied % 2 == 0]
        elif best == 0:
            # exact: keep the sign of zero
            sign = 1 << (f.bits - 1) if np.signbit(xi) else 0
            tied = tied[(tied & (1 << (f.bits - 1))) == sign] if xi == 0 else tied
        assert gi in tied, (xi, gi, tied)
    del order


def test_pack_layout_worked_example(orc):
    """Sec. IV-A register packing: value i of a row sits in word i // k at
    bit offset bits * (i % k), least significant first."""
    # E2M1 codes of 0.5, 1, 1.5, 2, 3, 4, 6, -0.5, then 1 (second word)
    x = np.array([[0.5, 1, 1.5, 2, 3, 4, 6, -0.5, 1]], np.float32)
    codes = orc.encode(x, 2, 1)
    assert list(codes[0]) == [1, 2, 3, 4, 5, 6, 7, 9, 2]
    packed = orc.pack_rows(codes, 4)
    words = packed.view(np.uint32)[0]
    assert words[0] == 0x97654321 and words[1] == 0x2 and words.size == 4
    assert np.array_equal(orc.unpack_rows(packed, 9, 4), codes)
    # FP6: five per word, top two bits zero
    c6 = np.arange(1, 7, dtype=np.uint32)[None, :]
    w6 = orc.pack_rows(c6, 6).view(np.uint32)[0]
    assert w6[0] == (1 | 2 << 6 | 3 << 12 | 4 << 18 | 5 << 24) and w6[1] == 6
