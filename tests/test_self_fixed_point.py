"""The self terms' fixed point (collision stage): a sphere named by at most d
pairs sums at most d terms u * 2^e rounded to integers, |u| <= 1 up to the
hardware reciprocal square root's error, with e = 30 - floor(log2 d) (the
device takes it as clz(d) - 1).  Checks over every degree the robot limits
allow (a pair (i, i) names its sphere twice) that no sum, and no single
term, reaches 2^31, and that the particle arm's degrees give e = 25."""
import numpy as np

from paper_2310_07854_gb300 import synth

VAPR_MAX_PAIRS = 8128
RSQRT_REL = 2.0 ** -22  # a generous bound on rsqrtf's relative error


def exponent(d: int) -> int:
    clz = 32 - int(d).bit_length()
    return clz - 1


def test_no_overflow_for_any_degree():
    for d in range(1, 2 * VAPR_MAX_PAIRS + 1):
        e = exponent(d)
        term = np.floor(2.0 ** e * (1.0 + RSQRT_REL) + 0.5)
        assert term < 2 ** 31
        assert d * term < 2 ** 31, (d, e)


def test_exponent_is_the_finest_that_fits():
    for d in range(1, 2 * VAPR_MAX_PAIRS + 1):
        e = exponent(d)
        assert d * 2.0 ** (e + 1) >= 2 ** 31 or e == 30, (d, e)


def test_particle_arm_exponent():
    r = synth.make_workload("particle_32768").robot
    deg = np.bincount(np.asarray(r.pairs).ravel(), minlength=r.n_spheres)
    assert exponent(int(deg.max())) == 25
