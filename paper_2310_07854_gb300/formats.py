"""ExMy storage formats: the 21-format search set, per-tensor tables, parsing.

Sec. IV-A: a reduced-precision format has one sign bit, E exponent bits and
M mantissa bits; FP4, FP5, FP6, FP8, FP10, FP16 and FP32 are the candidate
widths, and one 32-bit register holds floor(32 / bits) values.  The paper
counts 21 formats, 21^5 = 4,084,101 combinations over five tensors, and
three formats of at least 16 bits (E5M10, E8M7, E8M23).  The enumeration
below reproduces those counts: for bits in {4, 5, 6, 8, 10} every split with
E >= 2 and M >= 1 (1 + 2 + 3 + 5 + 7 = 18 formats) plus the three 16/32-bit
IEEE-style formats.

Special values (the paper is silent; reading chosen to agree with IEEE half
and bfloat16 and with the OCP 8/6/4-bit formats):

* ``IEEE``: the all-ones exponent encodes Inf and NaN (E8M23, E8M7, E5M10,
  E5M2, and every other 8-exponent-bit format, so that no code lies beyond
  float32); overflow goes to Inf unless ``SAT`` is set (E5M2 and the
  sub-16-bit E8 formats saturate).
* ``FN``: no Inf; the all-ones exponent and mantissa is NaN (E4M3).
* neither: every code is finite (E2M1, E3M2, E2M3 and all others).
* ``SAT``: overflow and Inf clamp to the largest finite magnitude.
"""
from __future__ import annotations

import dataclasses
import itertools
import re

IEEE = 1
FN = 2
SAT = 4

TENSORS = ("pos", "dist", "grad", "jgrad", "xform")
# short names used in format-table strings: P, D, G, J, T
_SHORT = {"P": "pos", "D": "dist", "G": "grad", "J": "jgrad", "T": "xform"}


@dataclasses.dataclass(frozen=True)
class Fmt:
    E: int
    M: int
    flags: int

    @property
    def bits(self) -> int:
        return 1 + self.E + self.M

    @property
    def per_word(self) -> int:
        """Values per 32-bit word (Sec. IV-A register packing)."""
        return 32 // self.bits

    @property
    def name(self) -> str:
        return f"E{self.E}M{self.M}"

    def row_bytes(self, row_len: int) -> int:
        """Bytes of one packed row, padded to 16 bytes."""
        words = -(-row_len // self.per_word)
        return -(-4 * words // 16) * 16

    def row_bytes_unpadded(self, row_len: int) -> int:
        return 4 * -(-row_len // self.per_word)

    def __str__(self) -> str:
        return self.name


def default_flags(E: int, M: int) -> int:
    if (E, M) in ((8, 23), (8, 7), (5, 10)):
        return IEEE
    if (E, M) == (5, 2):
        return IEEE | SAT
    if (E, M) == (4, 3):
        return FN | SAT
    if E == 8:
        # the all-ones exponent stays reserved, so no code exceeds float32
        return IEEE | SAT
    return SAT


def fmt(E: int, M: int, flags: int | None = None) -> Fmt:
    if not (2 <= E <= 8 and 1 <= M <= 23 and 1 + E + M <= 32):
        raise ValueError(f"unsupported format E{E}M{M}")
    if E == 8 and flags is not None and not flags & IEEE:
        raise ValueError("8-exponent-bit formats must reserve Inf/NaN")
    if 1 + E + M > 16 and (E, M) != (8, 23):
        raise ValueError(f"unsupported format E{E}M{M}: widths above 16 bits "
                         "other than E8M23 are not storage formats here")
    return Fmt(E, M, default_flags(E, M) if flags is None else flags)


def parse(name: str) -> Fmt:
    """'E5M10' / 'fp16' / 'bf16' / 'fp32' / 'e4m3' -> Fmt."""
    alias = {"FP32": (8, 23), "F32": (8, 23), "FP16": (5, 10), "HALF": (5, 10),
             "F16": (5, 10), "BF16": (8, 7)}
    key = name.strip().upper()
    if key in alias:
        return fmt(*alias[key])
    m = re.fullmatch(r"E(\d+)M(\d+)", key)
    if not m:
        raise ValueError(f"cannot parse format {name!r}")
    return fmt(int(m.group(1)), int(m.group(2)))


FP32 = fmt(8, 23)
BF16 = fmt(8, 7)
FP16 = fmt(5, 10)
E4M3 = fmt(4, 3)
E5M2 = fmt(5, 2)
E3M2 = fmt(3, 2)
E2M3 = fmt(2, 3)
E2M1 = fmt(2, 1)

# The seven formats of the per-tensor sweep.
SWEEP = (FP32, BF16, FP16, E4M3, E5M2, E3M2, E2M1)


def search_set() -> list[Fmt]:
    """The 21 candidate formats of Sec. IV-A, narrowest first."""
    out = []
    for bits in (4, 5, 6, 8, 10):
        for E in range(2, bits - 1):
            out.append(fmt(E, bits - 1 - E))
    out += [FP16, BF16, FP32]
    return out


def hardware_formats() -> list[Fmt]:
    """Members of the search set that sm_103a converts with one cvt
    instruction (FP32, FP16, BF16, E4M3, E5M2, E3M2, E2M3, E2M1); the rest
    use the generic integer converter."""
    hw = {(2, 1), (2, 3), (3, 2), (4, 3), (5, 2), (5, 10), (8, 7), (8, 23)}
    return [f for f in search_set() if (f.E, f.M) in hw]


def formats_at_least(bits: int) -> list[Fmt]:
    """Candidates a per-tensor search result of ``bits`` leaves (Sec. V-A)."""
    return [f for f in search_set() if f.bits >= bits]


@dataclasses.dataclass(frozen=True)
class FormatTable:
    """Storage format of each large tensor: sphere positions (P), per-sphere
    distances (D), distance gradients (G), joint gradients (J) and link
    transforms (T)."""

    pos: Fmt = FP32
    dist: Fmt = FP32
    grad: Fmt = FP32
    jgrad: Fmt = FP32
    xform: Fmt = FP32

    @classmethod
    def parse(cls, spec: str) -> "FormatTable":
        """'P=E5M10,D=E2M1,G=E2M1,J=E4M3,T=E8M23' (missing tensors: FP32)."""
        kw = {}
        for part in filter(None, (p.strip() for p in spec.split(","))):
            key, val = part.split("=")
            key = key.strip().upper()
            if key not in _SHORT:
                raise ValueError(f"unknown tensor {key!r}")
            kw[_SHORT[key]] = parse(val)
        return cls(**kw)

    def __str__(self) -> str:
        return ",".join(f"{s}={getattr(self, t).name}" for s, t in _SHORT.items())

    @property
    def total_bits(self) -> int:
        return sum(getattr(self, t).bits for t in TENSORS)


FP32_TABLE = FormatTable()


def sweep_tables(tensors=("pos", "dist", "grad", "jgrad"), formats=SWEEP):
    """All per-tensor combinations of ``formats`` over ``tensors``."""
    for combo in itertools.product(formats, repeat=len(tensors)):
        yield FormatTable(**dict(zip(tensors, combo)))
