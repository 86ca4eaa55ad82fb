"""Pins of the bivariate oracle (the plain product in (Z/pZ)[x, y], the
setting of Sec. 2) against facts that do not re-use it: reductions to the
univariate (Z/pZ)[x] product, evaluation at points, closed forms, and the
pure-Python twin on tiny inputs."""
import itertools

import numpy as np
import pytest

import ks_inputs as gen
import oracle
from oracle import pyref

P61 = (1 << 61) - 1
PRIMES = [3, 65537, 2147483647, P61]


def rand_biv(lx, ly, p, seed):
    return gen.random_residues(lx * ly, p, seed).reshape(ly, lx)


def ev(a, r, s, p):
    """a(r, s) mod p by direct summation over the coefficients a[i][j] r^j s^i."""
    tot = 0
    for i, row in enumerate(a.tolist()):
        for j, c in enumerate(row):
            tot = (tot + int(c) * pow(r, j, p) * pow(s, i, p)) % p
    return tot


@pytest.mark.parametrize("p", PRIMES)
def test_single_row_is_the_univariate_product(p):
    # ly = 1: h(x, y) = f_0(x) g_0(x), the (Z/pZ)[x] product
    f, g = rand_biv(37, 1, p, 1), rand_biv(37, 1, p, 2)
    want = oracle.mul_mod(f.reshape(-1), g.reshape(-1), p).reshape(1, -1)
    assert np.array_equal(oracle.mul_biv_mod(f, g, p), want)


@pytest.mark.parametrize("p", PRIMES)
def test_single_column_is_the_univariate_product_in_y(p):
    # lx = 1: h is a polynomial in y only
    f, g = rand_biv(1, 29, p, 3), rand_biv(1, 29, p, 4)
    want = oracle.mul_mod(f.reshape(-1), g.reshape(-1), p).reshape(-1, 1)
    assert np.array_equal(oracle.mul_biv_mod(f, g, p), want)


@pytest.mark.parametrize("p", PRIMES)
def test_evaluation_at_points(p):
    # h(r, s) = f(r, s) g(r, s) mod p
    rng = np.random.default_rng(p % 1000)
    for lx, ly in ((7, 5), (16, 16), (3, 40)):
        f, g = rand_biv(lx, ly, p, lx + 10 * ly), rand_biv(lx, ly, p, lx + 10 * ly + 1)
        h = oracle.mul_biv_mod(f, g, p)
        for _ in range(3):
            r, s = int(rng.integers(0, p)), int(rng.integers(0, p))
            assert ev(h, r, s, p) == ev(f, r, s, p) * ev(g, r, s, p) % p


def test_closed_forms():
    p = 1000003
    lx, ly = 6, 4
    # all coefficients -1: h[k][m] = (pairs i + i' = k) (pairs j + j' = m)
    f = np.full((ly, lx), p - 1, dtype=np.uint64)
    h = oracle.mul_biv_mod(f, f, p)
    for k in range(2 * ly - 1):
        for m in range(2 * lx - 1):
            cy = min(k, ly - 1) - max(0, k - ly + 1) + 1
            cx = min(m, lx - 1) - max(0, m - lx + 1) + 1
            assert int(h[k][m]) == cy * cx % p
    # monomials: x^a y^b times x^c y^d is x^(a+c) y^(b+d)
    for a, b, c, d in ((0, 0, 5, 3), (2, 1, 3, 2), (5, 3, 5, 3)):
        f = np.zeros((ly, lx), dtype=np.uint64)
        g = np.zeros((ly, lx), dtype=np.uint64)
        f[b][a] = 7
        g[d][c] = 11
        h = oracle.mul_biv_mod(f, g, p)
        assert int(h[b + d][a + c]) == 77 and int(h.sum()) == 77


def test_bruteforce_against_the_python_twin():
    p = 5
    for lx, ly in ((1, 1), (2, 1), (1, 2), (2, 2)):
        for vals in itertools.product(range(p), repeat=lx * ly):
            f = np.array(vals, dtype=np.uint64).reshape(ly, lx)
            g = np.array(vals[::-1], dtype=np.uint64).reshape(ly, lx)
            want = np.array(pyref.biv_mul_mod(f.tolist(), g.tolist(), p), dtype=np.uint64)
            assert np.array_equal(oracle.mul_biv_mod(f, g, p), want)
    rng = np.random.default_rng(9)
    for _ in range(20):
        lx, ly = int(rng.integers(1, 6)), int(rng.integers(1, 6))
        f = rand_biv(lx, ly, P61, int(rng.integers(1 << 30)))
        g = rand_biv(lx, ly, P61, int(rng.integers(1 << 30)))
        want = np.array(pyref.biv_mul_mod(f.tolist(), g.tolist(), P61), dtype=np.uint64)
        assert np.array_equal(oracle.mul_biv_mod(f, g, P61), want)


def test_rejects_bad_inputs():
    f = np.zeros((2, 3), dtype=np.uint64)
    with pytest.raises(ValueError):
        oracle.mul_biv_mod(f, np.zeros((3, 2), dtype=np.uint64), 7)
    f[0][0] = 7
    with pytest.raises(ValueError):
        oracle.mul_biv_mod(f, f, 7)
