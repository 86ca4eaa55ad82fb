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


# ---- the complex evaluation points of Sec. 2.5 (step model)
from oracle import ks_steps  # noqa: E402


@pytest.mark.parametrize("p", [3, 5, 13, 65537, 998244353, P61])
def test_complex_points_equal_the_plain_product(p):
    # p = 1 (mod 4) and p = 3 (mod 4): R[i] = R[t]/(t^2 + 1) either way
    rng = np.random.default_rng(p % 1000)
    for lx, ly in ((1, 1), (1, 5), (4, 1), (2, 2), (3, 4), (5, 5), (8, 7), (9, 6)):
        f = [[int(x) for x in rng.integers(0, p, lx)] for _ in range(ly)]
        g = [[int(x) for x in rng.integers(0, p, lx)] for _ in range(ly)]
        run = ks_steps.biv_complex_points(f, g, p)
        assert run["h"] == pyref.biv_mul_mod(f, g, p), (p, lx, ly)
        assert run["products"] == 5


def test_complex_points_combinations():
    # H1 = A0 + A1 + A2 + A3, H2 = A0 - A1 + A2 - A3, Re = A0 - A2, Im = A1 - A3,
    # each A_r holding the rows k = r (mod 4) at x^(kM) without overlap
    p, lx, ly = 65537, 7, 9
    rng = np.random.default_rng(5)
    f = [[int(x) for x in rng.integers(0, p, lx)] for _ in range(ly)]
    g = [[int(x) for x in rng.integers(0, p, lx)] for _ in range(ly)]
    run = ks_steps.biv_complex_points(f, g, p)
    A, M, h = run["A"], run["M"], pyref.biv_mul_mod(f, g, p)
    n = len(run["H1"])
    for r in range(4):
        want = [0] * n
        for k in range(r, 2 * ly - 1, 4):
            for j, c in enumerate(h[k]):
                assert want[k * M + j] == 0 or c == 0  # no two rows of A_r meet
                want[k * M + j] = (want[k * M + j] + c) % p
        assert A[r][:n] == want
    assert run["H1"] == [(a + b + c + d) % p for a, b, c, d in zip(*A)]
    assert run["H2"] == [(a - b + c - d) % p for a, b, c, d in zip(*A)]
    assert run["Re"] == [(a - c) % p for a, _, c, _ in zip(*A)]
    assert run["Im"] == [(b - d) % p for _, b, _, d in zip(*A)]


def test_complex_points_planted_slips_fail():
    # a combination without the factor 2 on Re, or with Im's sign flipped,
    # does not give the product
    p, lx, ly = 998244353, 5, 6
    rng = np.random.default_rng(6)
    f = [[int(x) for x in rng.integers(0, p, lx)] for _ in range(ly)]
    g = [[int(x) for x in rng.integers(0, p, lx)] for _ in range(ly)]
    run = ks_steps.biv_complex_points(f, g, p)
    want, M, inv4 = pyref.biv_mul_mod(f, g, p), run["M"], pow(4, -1, p)
    H1, H2, Re, Im = run["H1"], run["H2"], run["Re"], run["Im"]
    slip0 = [(a + b + r) * inv4 % p for a, b, r in zip(H1, H2, Re)]
    assert [slip0[0 * M + j] for j in range(2 * lx - 1)] != want[0]
    slip1 = [(a - b - 2 * m) * inv4 % p for a, b, m in zip(H1, H2, Im)]
    assert [slip1[1 * M + j] for j in range(2 * lx - 1)] != want[1]


def test_complex_points_need_an_odd_modulus():
    with pytest.raises(ValueError):
        ks_steps.biv_complex_points([[1, 2]], [[3, 4]], 1 << 20)
