"""(Z/pZ)[x, y] products by the polynomial-ring substitutions of Sec. 2
(KS_1 standard, KS_2 negated, KS_3 reciprocal, KS_4 four-point, KS_C the
complex points of Sec. 2.5), through the C ABI, exact against the bivariate
oracle."""
import numpy as np
import pytest

import ks_inputs as gen
import oracle
from tests._gpu import to_dev, to_host

pytestmark = pytest.mark.gpu

P61 = (1 << 61) - 1
VARIANTS = [0, 1, 2, 3, 4, 5]


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    return ks


def rand_biv(lx, ly, p, seed):
    return gen.random_residues(lx * ly, p, seed).reshape(ly, lx)


def biv_gpu(ks, f, g, p, variant):
    import torch
    ly, lx = f.shape
    h = torch.full((2 * ly - 1, 2 * lx - 1), -1, dtype=torch.int64, device="cuda")
    ks.ks_mul_bivariate_mod(h, to_dev(f), to_dev(g), p, variant)
    ks.status_sync()
    return to_host(h)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("p", [3, 5, 65537, 998244353, 2147483647, P61])
def test_bivariate_exact(ks, variant, p):
    for lx, ly in ((1, 1), (1, 7), (6, 1), (2, 2), (3, 4), (5, 5), (17, 9), (40, 33), (64, 3)):
        f, g = rand_biv(lx, ly, p, 11 * lx + ly), rand_biv(lx, ly, p, 11 * lx + ly + 5)
        got = biv_gpu(ks, f, g, p, variant)
        want = oracle.mul_biv_mod(f, g, p)
        assert np.array_equal(got, want), (variant, p, lx, ly)


@pytest.mark.parametrize("variant", VARIANTS)
def test_bivariate_extremes(ks, variant):
    p = P61
    lx, ly = 23, 19
    f = np.full((ly, lx), p - 1, dtype=np.uint64)  # every coefficient -1
    assert np.array_equal(biv_gpu(ks, f, f, p, variant), oracle.mul_biv_mod(f, f, p))
    z = np.zeros((ly, lx), dtype=np.uint64)
    assert np.array_equal(biv_gpu(ks, z, f, p, variant), oracle.mul_biv_mod(z, f, p))


@pytest.mark.parametrize("variant", VARIANTS)
def test_bivariate_larger(ks, variant):
    # a size whose univariate products take the library's large-product engines;
    # checked at points (h(r, s) = f(r, s) g(r, s)) and on sampled rows
    p = P61
    lx, ly = 200, 150
    f, g = rand_biv(lx, ly, p, 91), rand_biv(lx, ly, p, 92)
    h = biv_gpu(ks, f, g, p, variant)
    rng = np.random.default_rng(variant)

    def ev(a, r, s):
        xs = [pow(r, j, p) for j in range(a.shape[1])]
        tot, sp = 0, 1
        for row in a.tolist():
            tot = (tot + sp * (sum(int(c) * x for c, x in zip(row, xs)) % p)) % p
            sp = sp * s % p
        return tot
    for _ in range(2):
        r, s = int(rng.integers(2, p)), int(rng.integers(2, p))
        assert ev(h, r, s) == ev(f, r, s) * ev(g, r, s) % p
    for k in (0, 1, ly - 1, 2 * ly - 2):
        lo, hi = max(0, k - ly + 1), min(k, ly - 1)
        row = np.zeros(2 * lx - 1, dtype=object)
        for i in range(lo, hi + 1):
            row += np.convolve(f[i].astype(object), g[k - i].astype(object))
        assert [int(c) % p for c in row] == [int(c) for c in h[k]], k


def test_bivariate_errors(ks):
    import torch
    f = to_dev(np.zeros((3, 4), dtype=np.uint64))
    h = torch.zeros((5, 7), dtype=torch.int64, device="cuda")
    for variant in (2, 4, 5):  # halving needs an odd modulus
        with pytest.raises(ks.KSError):
            ks.ks_mul_bivariate_mod(h, f, f, 1 << 20, variant)
    for variant in (1, 3, 0):  # the other variants take any modulus
        ks.ks_mul_bivariate_mod(h, f, f, 1 << 20, variant)
    with pytest.raises(ks.KSError):
        ks.ks_mul_bivariate_mod(h, f, f, 1 << 63, 1)
    ks.status_sync()
