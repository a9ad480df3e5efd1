"""The FP64 particle kernels take u = z / dz without a division: q = RN(z y) with y = RN(1/dz)
from the host, then twice q <- RN(q + RN(z - q dz) y), each remainder formed exactly by one
fused multiply-add (Markstein, IBM J. Res. Dev. 34, 1990: with a correctly rounded
reciprocal and a faithful q, the corrected quotient is the correctly rounded one).  The
shape weights need the quotient correctly rounded (one ulp of u is ~Nz ulps of a weight),
so this pins the step sequence in exact rational arithmetic against the IEEE quotient over
the workloads' cell sizes and z ranges, with cell boundaries and binade edges included,
and shows why the first correction is needed."""
import random
from fractions import Fraction as Fr

import pytest


def rn(f):
    return float(f)   # exact rational -> nearest double, ties to even


def fma(a, b, c):
    return rn(Fr(a) * Fr(b) + Fr(c))


def quotient(z, dz, corrections):
    y = rn(Fr(1) / Fr(dz))
    q = rn(Fr(z) * Fr(y))
    for _ in range(corrections):
        r = fma(-q, dz, z)
        q = fma(r, y, q)
    return q


def samples(n, seed):
    rng = random.Random(seed)
    out = []
    for t in range(n):
        dz = rng.choice([0.05e-6, 1e-6 / 3, 0.1e-6 * (1 + rng.random()), rng.uniform(1e-9, 1e-3)])
        Nz = rng.choice([64, 256, 525, 2048, 8192])
        kind = t % 4
        if kind == 0:
            z = rng.uniform(0, Nz * dz)
        elif kind == 1:   # a few ulps around a cell boundary
            z = rng.randrange(0, Nz) * dz * (1 + rng.choice([-1, 1]) * 2.0**-52 * rng.randrange(0, 4))
        elif kind == 2:   # quotients just below a power of two (the top of a binade)
            k = rng.randrange(0, 13)
            z = (2.0**k) * dz * (1 - 2.0**-52 * rng.randrange(1, 64))
        else:
            z = rng.uniform(0, dz)
        out.append((z, dz))
    return out


@pytest.mark.parametrize("seed", [1, 2])
def test_two_corrections_give_the_correctly_rounded_quotient(seed):
    for z, dz in samples(4000, seed):
        assert quotient(z, dz, 2) == rn(Fr(z) / Fr(dz)), (z, dz)


def test_each_remainder_is_exact_after_the_first_correction():
    for z, dz in samples(2000, 3):
        y = rn(Fr(1) / Fr(dz))
        q = fma(fma(-rn(Fr(z) * Fr(y)), dz, z), y, rn(Fr(z) * Fr(y)))
        assert Fr(fma(-q, dz, z)) == Fr(z) - Fr(q) * Fr(dz)


def test_the_product_alone_can_leave_an_inexact_remainder():
    """Why the first correction is there: RN(z y) is not always a faithful quotient, and then
    z - q dz is not representable, so Markstein's premise for a single correction fails
    (about 0.2 % of these samples)."""
    inexact = 0
    for z, dz in samples(20000, 4):
        q = rn(Fr(z) * Fr(rn(Fr(1) / Fr(dz))))
        inexact += Fr(fma(-q, dz, z)) != Fr(z) - Fr(q) * Fr(dz)
    assert inexact > 0
