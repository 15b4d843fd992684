"""GPU converters (vapr_pack / vapr_unpack) against the oracle's ExMy
emulator: bit-exact codes, exact decodes, zero padding, ragged rows, and
every float32 bit pattern for the seven sweep formats."""
import numpy as np
import pytest

import oracle
from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import formats as F

pytestmark = pytest.mark.gpu

EXTRAS = [F.fmt(5, 9), F.fmt(6, 8), F.fmt(6, 6)]
ALL = F.search_set() + EXTRAS


def _inputs(rng, rows, row_len):
    n = rows * row_len
    x = np.concatenate([
        rng.uniform(-1, 1, n // 4) * 2.0 ** rng.integers(-30, 30, n // 4),
        rng.integers(0, 2**32, n // 4, dtype=np.uint64).astype(np.uint32).view(np.float32),
        rng.uniform(-8, 8, n // 4),
        rng.uniform(-1, 1, n - 3 * (n // 4)) * 2.0 ** rng.integers(-150, -120, n - 3 * (n // 4)),
    ]).astype(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 65504, 65520, 448, 464, 57344, 6.0,
                        7.5, 28.0, 3.4028235e38, 1e-45, -1e-45, 0.25, 0.75], np.float32)
    x[:special.size] = special
    rng.shuffle(x[special.size:])
    return x.reshape(rows, row_len)


@pytest.mark.parametrize("f", ALL, ids=str)
def test_pack_matches_emulator(f):
    import torch
    rng = np.random.default_rng(f.bits * 31 + f.E)
    rows, row_len = 300, 37  # ragged: 37 is not a multiple of any k > 1
    x = _inputs(rng, rows, row_len)
    dst = B.alloc_packed(rows, row_len, f)
    dst.fill_(0xAB)  # padding must be overwritten with zeros
    B.vapr_pack(torch.as_tensor(x, device="cuda"), rows, row_len, f, dst)
    got = dst.cpu().numpy()
    codes = oracle.encode(x, f.E, f.M, f.flags)
    want = oracle.pack_rows(codes, f.bits)
    assert got.shape == want.shape
    mism = np.flatnonzero((got != want).any(1))
    assert mism.size == 0, f"{f}: rows {mism[:5]} differ"


@pytest.mark.parametrize("f", ALL, ids=str)
def test_unpack_decodes_every_code(f):
    import torch
    if f == F.FP32:
        codes = np.random.default_rng(1).integers(0, 2**32, 1 << 16, dtype=np.uint64).astype(np.uint32)
    else:
        codes = np.arange(1 << f.bits, dtype=np.uint32)
    row_len = 61
    total = -(-codes.size // row_len) * row_len
    codes = np.resize(codes, total).reshape(-1, row_len)  # repeats codes to fill the rows
    packed = oracle.pack_rows(codes, f.bits)
    out = torch.empty(codes.shape, dtype=torch.float32, device="cuda")
    B.vapr_unpack(torch.as_tensor(packed, device="cuda"), codes.shape[0], row_len, f, out)
    got = out.cpu().numpy().astype(np.float64)
    want = oracle.decode(codes, f.E, f.M, f.flags)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], want[~nan])
    # signed zeros keep their sign
    assert np.array_equal(np.signbit(got[~nan]), np.signbit(want[~nan]))


# generic formats whose encoder takes the one-multiply fast path (finite,
# E < 8), two of them the searched table's G and J formats
FAST_GENERIC = (F.fmt(6, 3), F.fmt(3, 4), F.fmt(2, 2), F.fmt(5, 4))


@pytest.mark.slow
@pytest.mark.parametrize("f", F.SWEEP + FAST_GENERIC, ids=str)
def test_pack_all_float32_bit_patterns(f):
    """Every one of the 2^32 float32 inputs (65 chunks of 16448 rows x 4080;
    4080 is a multiple of every pack factor, the last chunk wraps around).
    Expected codes come from the oracle; only the comparison runs on the GPU."""
    import torch
    row_len, rows = 4080, 16448
    chunk = row_len * rows
    k, bits = f.per_word, f.bits
    W = row_len // k
    mask = (1 << bits) - 1 if bits < 32 else 0xFFFFFFFF
    shifts = torch.arange(k, device="cuda", dtype=torch.int64) * bits
    idx = torch.arange(chunk, device="cuda", dtype=torch.int64)
    dst = B.alloc_packed(rows, row_len, f)
    for start in range(0, 1 << 32, chunk):
        bits32 = (idx + start) & 0xFFFFFFFF
        x = torch.where(bits32 >= 2**31, bits32 - 2**32, bits32).to(torch.int32).view(torch.float32)
        B.vapr_pack(x, rows, row_len, f, dst)
        words = dst.view(torch.int32)[:, :W].to(torch.int64)
        got = ((words.unsqueeze(-1) >> shifts) & mask).reshape(rows, row_len)
        want = oracle.encode_bits_range(start, chunk, f.E, f.M, f.flags)
        want = torch.as_tensor(want.astype(np.int64), device="cuda").reshape(rows, row_len)
        bad = (got != want).reshape(-1).nonzero()
        if bad.numel():
            i0 = int(bad[0])
            raise AssertionError(f"{f}: input bits {(start + i0) & 0xFFFFFFFF:#010x} -> "
                                 f"{int(got.reshape(-1)[i0]):#x}, want {int(want.reshape(-1)[i0]):#x}"
                                 f" ({bad.numel()} mismatches in this chunk)")
