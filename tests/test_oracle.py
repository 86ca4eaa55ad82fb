"""Pins the schoolbook oracle to facts that do not come from the oracle itself.

* the worked example of Harvey Sec. 1 (printed product and coefficients);
* brute force over every tiny input, against numpy's polynomial convolution on
  Python integers and against the pure-Python twin;
* evaluation identities h(1) = f(1) g(1), h(-1) = f(-1) g(-1) and
  h(r) = f(r) g(r) mod q at random points r and primes q;
* closed forms: all-maximal coefficients (the equality case of the bound
  h_i <= L (2^b - 1)^2 of Sec. 3), signed extremes, monomials;
* the (Z/pZ)[x] product of Sec. 4 against the same identities mod p.
"""
import itertools
import random

import numpy as np
import pytest

import ks_inputs as gen
import oracle
from oracle import pyref
from tests._golden import load


def _h_ints(f_int, g_int, b, signed, ol=None):
    f = gen.from_ints(f_int, b)
    g = gen.from_ints(g_int, b)
    h = oracle.mul(f, g, b, signed, n_limbs_out=ol, threads=2)
    return gen.to_ints(h, True if signed else False)


def test_intro_example():
    ex = load("intro_example.txt")
    f, g, h = ex["f"], ex["g"], ex["h"]
    assert pyref.poly_eval(f, 10 ** 7) == ex["f(10^7)"]
    assert pyref.poly_eval(g, 10 ** 7) == ex["g(10^7)"]
    assert ex["f(10^7)"] * ex["g(10^7)"] == ex["h(10^7)"]
    assert _h_ints(f, g, 10, False) == h
    assert pyref.poly_mul(f, g) == h
    # the printed coefficients are the base-10^7 digits of the printed product
    assert sum(c * 10 ** (7 * i) for i, c in enumerate(h)) == ex["h(10^7)"]


def _convolve_objects(f, g):
    return [int(x) for x in np.convolve(np.array(f, dtype=object), np.array(g, dtype=object))]


@pytest.mark.parametrize("b,signed", [(1, False), (2, False), (2, True), (3, True)])
def test_bruteforce_tiny(b, signed):
    vals = range(-(1 << (b - 1)), 1 << (b - 1)) if signed else range(0, 1 << b)
    vals = list(vals)
    n = 0
    for lf in (1, 2, 3):
        for lg in (1, 2, 3):
            if signed and b == 3 and lf + lg > 4:
                continue
            for f in itertools.product(vals, repeat=lf):
                for g in itertools.product(vals, repeat=lg):
                    want = _convolve_objects(list(f), list(g))
                    assert pyref.poly_mul(list(f), list(g)) == want
                    assert _h_ints(list(f), list(g), b, signed) == want, (f, g)
                    n += 1
    assert n > 100


def _rand_case(rng, lf, lg, b, signed):
    f = gen.random_poly(lf, b, signed, rng.getrandbits(64))
    g = gen.random_poly(lg, b, signed, rng.getrandbits(64))
    return f, g


@pytest.mark.parametrize("b", [1, 7, 48, 63, 64, 65, 128, 200, 256, 513])
@pytest.mark.parametrize("signed", [False, True])
def test_evaluation_identities(b, signed):
    rng = random.Random(1000 * b + signed)
    for lf, lg in [(1, 1), (1, 9), (17, 5), (33, 33), (40, 71)]:
        f, g = _rand_case(rng, lf, lg, b, signed)
        fi, gi = gen.to_ints(f, signed), gen.to_ints(g, signed)
        h = gen.to_ints(oracle.mul(f, g, b, signed, threads=3), signed)
        assert len(h) == lf + lg - 1
        for x in (1, -1):
            assert pyref.poly_eval(h, x) == pyref.poly_eval(fi, x) * pyref.poly_eval(gi, x)
        for q in (2 ** 61 - 1, 2 ** 89 - 1, 1000003):
            r = rng.randrange(q)
            assert (pyref.poly_eval(h, r) - pyref.poly_eval(fi, r) * pyref.poly_eval(gi, r)) % q == 0


@pytest.mark.parametrize("b", [1, 5, 64, 100, 257])
def test_all_max_equality_case(b):
    """h_k = count_k (2^b - 1)^2: the bound of Sec. 3 with equality."""
    for lf, lg in [(1, 1), (8, 8), (9, 4), (16, 17)]:
        m = (1 << b) - 1
        h = _h_ints([m] * lf, [m] * lg, b, False)
        for k, hk in enumerate(h):
            cnt = min(k, lf - 1) - max(0, k - lg + 1) + 1
            assert hk == cnt * m * m
        e = oracle.ceil_log2(min(lf, lg))
        assert max(h) < 1 << (2 * b + e)


@pytest.mark.parametrize("b", [2, 8, 48, 64, 65, 130])
def test_signed_extremes(b):
    lo, hi = -(1 << (b - 1)), (1 << (b - 1)) - 1
    for lf, lg in [(1, 1), (7, 3), (16, 16), (17, 16)]:
        cnt = [min(k, lf - 1) - max(0, k - lg + 1) + 1 for k in range(lf + lg - 1)]
        assert _h_ints([lo] * lf, [lo] * lg, b, True) == [c * lo * lo for c in cnt]
        assert _h_ints([lo] * lf, [hi] * lg, b, True) == [c * lo * hi for c in cnt]
        assert _h_ints([hi] * lf, [lo] * lg, b, True) == [c * lo * hi for c in cnt]


def test_monomials_shift():
    rng = random.Random(7)
    b = 70
    g = [rng.randrange(1 << b) for _ in range(11)]
    for a in range(5):
        f = [0] * a + [1]
        assert _h_ints(f, g, b, False) == [0] * a + g
    # a negative monomial negates
    assert _h_ints([0, -1], [5, -7, 3], 8, True) == [0, -5, 7, -3]


def test_selected_coefficients_match_full():
    f = gen.random_poly(300, 130, True, 11)
    g = gen.random_poly(200, 130, True, 12)
    full = oracle.mul(f, g, 130, True, threads=4)
    ks = np.array([0, 1, 5, 199, 200, 298, 299, 300, 498], dtype=np.int64)
    part = oracle.coeffs(ks, f, g, 130, True, threads=3)
    assert np.array_equal(part, full[ks])


def test_out_limbs_bound_is_tight_enough():
    # all-max unsigned at L = 2^e and signed all-min both fit the stated width
    for b in (32, 64, 96):
        for L in (4, 5, 8):
            ol = oracle.out_limbs(L, L, b, False)
            m = (1 << b) - 1
            assert L * m * m < 1 << (64 * ol)
            ol = oracle.out_limbs(L, L, b, True)
            assert L * (1 << (2 * b - 2)) < 1 << (64 * ol - 1)


@pytest.mark.parametrize("p", [2 ** 61 - 1, 1000003, 2 ** 64 - 59])
def test_mul_mod(p):
    rng = random.Random(p % 1000)
    for lf, lg in [(1, 1), (13, 29), (64, 64)]:
        f = gen.random_residues(lf, p, rng.getrandbits(64))
        g = gen.random_residues(lg, p, rng.getrandbits(64))
        h = [int(x) for x in oracle.mul_mod(f, g, p, threads=2).reshape(-1)]
        fi = [int(x) for x in f.reshape(-1)]
        gi = [int(x) for x in g.reshape(-1)]
        assert h == pyref.poly_mul_mod(fi, gi, p)
        r = rng.randrange(p)
        assert pyref.poly_eval(h, r) % p == pyref.poly_eval(fi, r) * pyref.poly_eval(gi, r) % p


def test_threads_do_not_change_result():
    f = gen.random_poly(100, 200, True, 1)
    g = gen.random_poly(90, 200, True, 2)
    a = oracle.mul(f, g, 200, True, threads=1)
    b = oracle.mul(f, g, 200, True, threads=7)
    assert np.array_equal(a, b)


def test_rejects_bad_arguments():
    f = gen.random_poly(3, 8, False, 1)
    with pytest.raises(ValueError):
        oracle.mul_mod(np.array([[5]], dtype=np.uint64), np.array([[1]], dtype=np.uint64), 5)
    with pytest.raises(ValueError):
        oracle.mul(f, f, 0, False)


def test_stored_config5b_digests_are_the_oracles():
    # the golden digests of the 64 products mod 2^61 - 1 were written by
    # tests/golden/make_config5b_hash.py from the oracle alone; two of them are
    # recomputed here (a few seconds each), and the file lists all 64
    import hashlib
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "config5b_products.txt")
    digests = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            i, d = line.split()
            digests[int(i)] = d
    assert sorted(digests) == list(range(64))
    p, L = (1 << 61) - 1, 1 << 16
    for i in (0, 63):
        h = oracle.mul_mod(gen.random_residues(L, p, 900 + 2 * i),
                           gen.random_residues(L, p, 901 + 2 * i), p)
        assert hashlib.sha256(np.ascontiguousarray(h, dtype=np.uint64).tobytes()).hexdigest() \
            == digests[i], i


def test_stored_config5a_digest_format():
    # the full 2^20 x 256-bit product takes the oracle about 1.5 hours, so only
    # the stored record's shape is checked here: 2^21 - 1 coefficients of the
    # library's output limb count, and a SHA-256
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "config5a_product.txt")
    kv = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    L = 1 << 20
    assert tuple(int(x) for x in kv["shape"].split()) == (2 * L - 1, oracle.out_limbs(L, L, 256,
                                                                                    False))
    assert len(kv["sha256"]) == 64 and int(kv["sha256"], 16) >= 0
