"""Products with different coefficient sizes in f and g (ks_mul_bits),
exact against the Python big-integer twin of the oracle: the operands are
decoded with their own bit sizes, multiplied as integer polynomials, and the
result is encoded with the output limbs of the larger size."""
import numpy as np
import pytest

import ks_inputs as gen
import oracle
from oracle import pyref
from tests._gpu import assert_same, to_dev, to_host

pytestmark = pytest.mark.gpu

CASES = [(300, 48, 200, 16), (200, 16, 300, 48), (100, 130, 150, 20), (64, 64, 64, 65),
         (1, 5, 700, 200), (500, 3, 1, 1), (257, 70, 129, 64)]


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    return ks


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("signed", [False, True])
def test_unequal_bit_sizes(ks, variant, signed):
    import torch
    for i, (lf, bf, lg, bg) in enumerate(CASES):
        f = gen.random_poly(lf, bf, signed, 1000 + i)
        g = gen.random_poly(lg, bg, signed, 2000 + i)
        B = max(bf, bg)
        ol = ks.out_limbs(lf, lg, B, signed)
        h = torch.empty((lf + lg - 1, ol), dtype=torch.int64, device="cuda")
        ks.ks_mul_bits(h, to_dev(f), bf, to_dev(g), bg, signed, variant)
        ks.status_sync()
        want = pyref.poly_mul(gen.to_ints(f, signed), gen.to_ints(g, signed))
        assert_same(to_host(h), gen.from_ints(want, 64 * ol),
                    "bits %d x %d, variant %d, signed %s" % (bf, bg, variant, signed))


def test_equal_limbs_matches_ks_mul(ks):
    # 48-bit and 16-bit coefficients share the one-limb layout: the same call as ks_mul
    f = gen.random_poly(4000, 48, True, 5)
    g = gen.random_poly(3000, 16, True, 6)
    import torch
    ol = ks.out_limbs(4000, 3000, 48, True)
    h = torch.empty((6999, ol), dtype=torch.int64, device="cuda")
    ks.ks_mul_bits(h, to_dev(f), 48, to_dev(g), 16, True)
    ks.status_sync()
    assert_same(to_host(h), oracle.mul(f, g, 48, True), "48 x 16 bits")
