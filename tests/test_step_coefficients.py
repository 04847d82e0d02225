"""The identity behind the subtree solver's table of step coefficients (host arithmetic).

Algorithm hhs-fsi halves the pivot step at every level, and each level's kicks use h/6, 2h/3
and h^2/48 of its step h (Alg. fsi, Eq. time-evolution-operator-hhs-fsi).  Rounding to nearest
commutes with scaling by a power of two (absent underflow and overflow), so the rounded
coefficients of h = tau0 2^-r are those of tau0 times 2^-r (times 2^-2r for h^2/48).  The
solver builds its table K[r], r = 0..64, that way, with 2^-r assembled from the exponent field,
and takes no FP64 division per frame.  This test checks, in IEEE double arithmetic, that the
table gives the bits the divisions give: at the pivots of the benchmark configurations and
at random ones, for every level down to r = 65 (a frame's fsi(S) uses the level below it).
"""

import struct

import numpy as np


def pow2_neg(r):
    # 2^-r from the biased exponent field, as the kernel builds it
    return struct.unpack("<d", struct.pack("<q", (1023 - r) << 52))[0]


def test_power_of_two_from_the_exponent_field():
    for r in range(0, 200):
        assert pow2_neg(r) == 2.0 ** -r


def test_level_coefficients_are_exact_scalings_of_the_first_level():
    rng = np.random.default_rng(2011)
    pivots = [2.0 ** -7, 2.0 ** -10, 0.005, 0.0625 / 8, 1.0, 1.0 / 3.0, 0.1]
    pivots += [float(t) for t in rng.uniform(2.0 ** -12, 1.0, 3000)]
    for tau0 in pivots:
        k6, k23, k48 = tau0 / 6.0, 2.0 * tau0 / 3.0, tau0 * tau0 / 48.0
        h = tau0
        for r in range(0, 66):
            s = pow2_neg(r)
            assert h == tau0 * s
            # the divisions a frame at level r would take, and the table's products
            assert h / 6.0 == k6 * s
            assert 2.0 * h / 3.0 == k23 * s
            assert h * h / 48.0 == k48 * (s * s)
            h = 0.5 * h
