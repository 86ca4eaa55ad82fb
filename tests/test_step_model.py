"""Pins the step model of the four variants to the paper's worked examples and to
the schoolbook product; checks the invariants the paper states along the way.

Fixtures: Sec. 1 (intro), Sec. 3.2 (reciprocal, base ten, N = 4), Sec. 3.3
(negated, base ten), Sec. 3.4 (four points, base ten, N = 2).
"""
import random

import pytest

from oracle import ks_steps as S
from oracle import pyref
from tests._golden import load

F = [274, 610, 887, 621]
G = [553, 298, 424, 790]
H = [151522, 418982, 788467, 1082839, 1043046, 964034, 490590]


def test_decimal_N_matches_paper():
    # b = 3 decimal digits, e = ceil(log10 4) = 1: N = 7, 4, 4, 2 (Sec. 1, 3.2-3.4)
    e = S.ceil_log(4, 10)
    assert e == 1
    assert [S.variant_N(v, 3, e) for v in (1, 2, 3, 4)] == [7, 4, 4, 2]


def test_ks1_intro_replay():
    ex = load("intro_example.txt")
    r = S.ks_mul_unsigned(F, G, 3, 1, base=10)
    assert r.X == 10 ** 7
    assert r.evals["F"] == ex["f(10^7)"] and r.evals["G"] == ex["g(10^7)"]
    assert r.products["P"] == ex["h(10^7)"]
    assert r.h == ex["h"] == H


def test_ks3_example_replay():
    ex = load("ks3_example.txt")
    r = S.ks_mul_unsigned(F, G, 3, 3, base=10)
    assert r.X == 10 ** ex["N"]
    assert r.evals["F"] == ex["f(10^4)"]
    assert r.evals["Fr"] == ex["10^12 f(10^-4)"]
    assert r.evals["G"] == ex["g(10^4)"]
    assert r.evals["Gr"] == ex["10^12 g(10^-4)"]
    assert r.products["P"] == ex["h(10^4)"]
    assert r.products["R"] == ex["10^24 h(10^-4)"]
    rec = r.recoveries[0]
    assert rec.u[0] == ex["u_0"] == rec.alpha[0]
    assert rec.w[1] == ex["w_1"]
    assert rec.eps[0] == ex["eps_0"]
    assert rec.beta[0] == ex["beta_0"]
    assert rec.h[0] == ex["h_0"]
    assert r.products["P"] - rec.h[0] == ex["h(10^4) - h_0"]
    assert r.products["R"] - 10 ** 24 * rec.h[0] == ex["10^24 h(10^-4) - 10^24 h_0"]
    assert rec.h[1] == ex["h_1"]
    assert r.h == H


def test_ks2_example_replay():
    ex = load("ks2_example.txt")
    r = S.ks_mul_unsigned(F, G, 3, 2, base=10)
    assert r.X == 10 ** ex["N"]
    assert r.evals["F+"] == ex["f(10^4)"] and r.evals["F-"] == ex["f(-10^4)"]
    assert r.evals["G+"] == ex["g(10^4)"] and r.evals["G-"] == ex["g(-10^4)"]
    assert r.products["P+"] == ex["h(10^4)"] and r.products["P-"] == ex["h(-10^4)"]
    assert r.halves["E"] == ex["h0(10^8)"]
    assert r.halves["XO"] == ex["10^4 h1(10^8)"]
    assert r.h == H


def test_ks4_example_replay():
    ex = load("ks4_example.txt")
    r = S.ks_mul_unsigned(F, G, 3, 4, base=10)
    assert r.X == 10 ** ex["N"]
    sign = (-1) ** (len(F) - 1)  # rev f(-X) = (-1)^(L-1) X^(L-1) f(-1/X)
    assert r.evals["F+"] == ex["f(10^2)"] and r.evals["F-"] == ex["f(-10^2)"]
    assert r.evals["Fr+"] == ex["10^6 f(10^-2)"]
    assert r.evals["Fr-"] == sign * ex["10^6 f(-10^-2)"]
    assert r.evals["G+"] == ex["g(10^2)"] and r.evals["G-"] == ex["g(-10^2)"]
    assert r.evals["Gr+"] == ex["10^6 g(10^-2)"]
    assert r.evals["Gr-"] == sign * ex["10^6 g(-10^-2)"]
    assert r.products["P+"] == ex["h(10^2)"] and r.products["P-"] == ex["h(-10^2)"]
    assert r.products["R+"] == ex["10^12 h(10^-2)"]
    assert r.products["R-"] == ex["10^12 h(-10^-2)"]
    assert r.halves["E"] == ex["h0(10^4)"]
    assert r.halves["ER"] == ex["10^12 h0(10^-4)"]
    assert r.halves["XO"] == ex["10^2 h1(10^4)"]
    assert r.halves["XOR"] == ex["10^10 h1(10^-4)"]
    assert r.h == H


def _check_recovery_invariants(rec, X):
    assert all(d in (0, 1) for d in rec.delta)          # carries of eq. (carry-1)
    assert all(e in (0, 1) for e in rec.eps)            # carries of eq. (carry-2)
    assert all(0 <= a < X for a in rec.alpha)
    assert all(0 <= bb < X - 1 for bb in rec.beta)      # eq. (beta-range)


SHAPES = [(1, 1), (1, 2), (2, 1), (2, 2), (3, 2), (5, 5), (6, 3), (8, 8), (9, 16), (17, 4),
          (16, 16), (31, 33)]


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
@pytest.mark.parametrize("b", [1, 2, 5, 16, 47, 64, 65, 130])
def test_variants_match_schoolbook(variant, b):
    rng = random.Random(variant * 1000 + b)
    for lf, lg in SHAPES:
        f = [rng.randrange(1 << b) for _ in range(lf)]
        g = [rng.randrange(1 << b) for _ in range(lg)]
        r = S.ks_mul_unsigned(f, g, b, variant)
        assert r.h == pyref.poly_mul(f, g), (lf, lg)
        Xrec = r.X if variant == 3 else r.X * r.X
        for rec in r.recoveries:
            _check_recovery_invariants(rec, Xrec)


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_variants_all_max(variant):
    """Maximal coefficients meet the bound of Sec. 3 with equality; the
    reconstruction must still see beta_i < 2^N - 1."""
    for b in (1, 3, 8, 33):
        for L in (1, 2, 3, 4, 7, 8, 9):
            m = (1 << b) - 1
            r = S.ks_mul_unsigned([m] * L, [m] * (L + 1), b, variant)
            assert r.h == pyref.poly_mul([m] * L, [m] * (L + 1))


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
@pytest.mark.parametrize("b", [1, 2, 8, 48, 64])
def test_signed_bias_reading(variant, b):
    rng = random.Random(b * 7 + variant)
    lo, hi = -(1 << (b - 1)), 1 << (b - 1)
    for lf, lg in SHAPES:
        f = [rng.randrange(lo, hi) for _ in range(lf)]
        g = [rng.randrange(lo, hi) for _ in range(lg)]
        assert S.ks_mul_signed(f, g, b, variant) == pyref.poly_mul(f, g)
    for lf, lg in [(4, 4), (5, 3)]:
        assert S.ks_mul_signed([lo] * lf, [lo] * lg, b, variant) == pyref.poly_mul([lo] * lf, [lo] * lg)


@pytest.mark.parametrize("b,L", [(8, 16), (48, 64), (64, 33), (5, 100)])
def test_operand_lengths_match_propositions(b, L):
    """Bit lengths of the evaluated operands against the Propositions of Sec. 3."""
    m = (1 << b) - 1
    f = [m] * L
    e = S.ceil_log(L, 2)
    N1, N2, N4 = S.variant_N(1, b, e), S.variant_N(2, b, e), S.variant_N(4, b, e)
    assert S.evaluate(f, 2 ** N1).bit_length() == N1 * (L - 1) + b
    Fp, Fm = S.eval_pm(f, 2 ** N2)
    assert Fp.bit_length() == N2 * (L - 1) + b
    assert abs(Fm).bit_length() <= N2 * (L - 1) + b
    Fp4, _ = S.eval_pm(f, 2 ** N4)
    # the overlapping sum may carry one bit beyond the Proposition's length
    assert N4 * (L - 1) + b <= Fp4.bit_length() <= N4 * (L - 1) + b + 1


def test_planted_mistakes_fail_the_pins(monkeypatch):
    """A plausible slip in the reconstruction (dropping the epsilon carry) or in
    the negated evaluation (odd part without its factor X) breaks a pin."""
    good = S.recover

    def no_eps(fwd, rev, n, X):
        u = [S.digit(fwd, i, X) for i in range(n + 1)]
        w = [S.digit(rev, n - j, X) for j in range(n + 1)]
        alpha, beta, delta = [0] * n, [0] * n, [0] * n
        alpha[0], a_prev = u[0], 0
        for j in range(n - 1):
            beta[j] = (w[j] - a_prev) % X
            alpha[j + 1] = (u[j + 1] - beta[j] - delta[j]) % X
            delta[j + 1] = (beta[j] + alpha[j + 1] + delta[j] - u[j + 1]) // X
            a_prev = alpha[j]
        beta[n - 1] = (w[n - 1] - a_prev) % X
        return S.Recovery([alpha[i] + X * beta[i] for i in range(n)], alpha, beta, delta,
                          [0] * n, u, w)

    monkeypatch.setattr(S, "recover", no_eps)
    rng = random.Random(3)
    bad = 0
    for _ in range(50):
        f = [rng.randrange(1 << 16) for _ in range(9)]
        g = [rng.randrange(1 << 16) for _ in range(9)]
        bad += S.ks_mul_unsigned(f, g, 16, 3).h != pyref.poly_mul(f, g)
    assert bad > 0
    monkeypatch.setattr(S, "recover", good)

    def wrong_pm(coeffs, X):  # odd part packed without its factor X
        f0, f1 = S.even_odd(coeffs)
        e = S.evaluate(f0, X * X)
        o = S.evaluate(f1, X * X)
        return e + o, e - o

    monkeypatch.setattr(S, "eval_pm", wrong_pm)
    with pytest.raises(AssertionError):
        test_ks2_example_replay()


def _rand_recoverable(n, X, rng):
    """Coefficients 0 <= c_i < X (X - 1) (the range Sec. 3.2 recovers) and their fwd, rev."""
    c = [rng.randrange(X * (X - 1)) for _ in range(n)]
    fwd = sum(ci * X ** i for i, ci in enumerate(c))
    rev = sum(ci * X ** i for i, ci in enumerate(reversed(c)))
    return c, fwd, rev


@pytest.mark.parametrize("X", [10, 16, 2 ** 7, 2 ** 20])
def test_recover_runs_downward_on_the_reversed_problem(X):
    # x^(n-1) h(1/x) has coefficients c_(n-1-i): its fwd is rev and its rev is fwd,
    # so the same recurrence with the two swapped yields the c_i from the top down
    rng = random.Random(X)
    for n in (1, 2, 3, 17, 64):
        c, fwd, rev = _rand_recoverable(n, X, rng)
        assert S.recover(fwd, rev, n, X).h == c
        assert S.recover(rev, fwd, n, X).h == c[::-1]


def _seeded_chain(fwd, rev, n, X, s, length, seed_prev, seed_cur):
    """Sec. 3.2's recurrence started at index s >= 1 from the exact values
    c_(s-1), c_s instead of from index 0: alpha_(s-1), beta_(s-1), alpha_s follow
    from the seeds, delta_(s-1) = u_s - beta_(s-1) - alpha_s (mod X) is 0 or 1, and
    the steps j = s .. s + length - 1 give c_j."""
    u = [S.digit(fwd, i, X) for i in range(n + 1)]
    w = [S.digit(rev, n - j, X) for j in range(n + 1)]
    a_prev, b_prev = seed_prev % X, seed_prev // X
    a_cur = seed_cur % X
    d_prev = (u[s] - b_prev - a_cur) % X
    assert d_prev in (0, 1)
    delta = (b_prev + a_cur + d_prev - u[s]) // X
    out = []
    for j in range(s, min(s + length, n)):
        if j <= n - 2:
            eps = 1 if a_cur > w[j + 1] else 0
            beta = (w[j] - a_prev - eps) % X
            a_next = (u[j + 1] - beta - delta) % X
            t = beta + a_next + delta - u[j + 1]
            assert t % X == 0 and t // X in (0, 1)
            out.append(a_cur + X * beta)
            a_prev, a_cur, delta = a_cur, a_next, t // X
        else:
            out.append(a_cur + X * ((w[j] - a_prev) % X))
    return out


@pytest.mark.parametrize("X", [10, 2 ** 7, 2 ** 31])
def test_one_seed_pair_starts_a_chain_each_way(X):
    # the exact pair (c_(s-1), c_s) starts the chain [s, s + m) upward and, on the
    # reversed problem, the chain [s - m, s) downward: every other seed pair suffices
    rng = random.Random(X + 1)
    n, m = 96, 16
    c, fwd, rev = _rand_recoverable(n, X, rng)
    for s in range(m, n, 2 * m):
        up = _seeded_chain(fwd, rev, n, X, s, m, c[s - 1], c[s])
        assert up == c[s:s + m]
        # reversed index r = n - 1 - i: the pair becomes (c~_(n-s-1), c~_(n-s)) = (c_s, c_(s-1))
        down = _seeded_chain(rev, fwd, n, X, n - s, m, c[s], c[s - 1])
        assert down == c[s - m:s][::-1]


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
@pytest.mark.parametrize("bf,bg", [(1, 30), (7, 64), (40, 3), (33, 33)])
def test_unequal_bit_sizes_match_schoolbook(variant, bf, bg):
    # N from bf + bg in place of 2b: random, all-ones-maximal and signed operands
    rng = random.Random(97 * bf + bg + variant)
    for lf, lg in ((1, 1), (5, 3), (17, 40), (64, 64)):
        f = [rng.randrange(1 << bf) for _ in range(lf)]
        g = [rng.randrange(1 << bg) for _ in range(lg)]
        assert S.ks_mul_unsigned_bits(f, g, bf, bg, variant).h == pyref.poly_mul(f, g)
        fm, gm = [(1 << bf) - 1] * lf, [(1 << bg) - 1] * lg
        assert S.ks_mul_unsigned_bits(fm, gm, bf, bg, variant).h == pyref.poly_mul(fm, gm)
        fs = [rng.randrange(-(1 << (bf - 1)), 1 << (bf - 1)) for _ in range(lf)]
        gs = [rng.randrange(-(1 << (bg - 1)), 1 << (bg - 1)) for _ in range(lg)]
        assert S.ks_mul_signed_bits(fs, gs, bf, bg, variant) == pyref.poly_mul(fs, gs)


def test_unequal_bit_sizes_N_is_tight_for_ks1():
    # one bit less than bf + bg + e and the all-maximal product no longer fits its fields
    bf, bg, L = 9, 21, 8
    f, g = [(1 << bf) - 1] * L, [(1 << bg) - 1] * L
    e = S.ceil_log(L, 2)
    N = S.variant_N_bits(1, bf, bg, e)
    assert N == bf + bg + e == S.variant_N(1, 15, e)
    assert S.ks1(f, g, 2 ** N).h == pyref.poly_mul(f, g)
    assert S.ks1(f, g, 2 ** (N - 1)).h != pyref.poly_mul(f, g)
    # and the unequal-size N is smaller than the equal-size one at max(bf, bg)
    assert N < S.variant_N(1, max(bf, bg), e)


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
@pytest.mark.parametrize("bf,bg", [(1, 1), (2, 2), (8, 8), (48, 48), (64, 64), (5, 17), (1, 30)])
def test_signed_offset_reading(variant, bf, bg):
    # signed evaluations, K U(Y) added to the integers read, K subtracted: the schoolbook
    # product on random operands and on the extremes (the largest positive h_k is
    # min(Lf, Lg) 2^(bf-1) 2^(bg-1) = K exactly when every pair is (-2^(bf-1), -2^(bg-1)))
    rng = random.Random(31 * bf + bg + 7 * variant)
    lo_f, hi_f = -(1 << (bf - 1)), (1 << (bf - 1)) - 1
    lo_g, hi_g = -(1 << (bg - 1)), (1 << (bg - 1)) - 1
    for lf, lg in SHAPES:
        f = [rng.randint(lo_f, hi_f) for _ in range(lf)]
        g = [rng.randint(lo_g, hi_g) for _ in range(lg)]
        r = S.ks_mul_signed_offset(f, g, bf, bg, variant)
        assert r.h == pyref.poly_mul(f, g), (lf, lg)
        for rec in r.recoveries:
            _check_recovery_invariants(rec, r.X if variant == 3 else r.X * r.X)
        for a, c in [(lo_f, lo_g), (lo_f, hi_g), (hi_f, lo_g), (hi_f, hi_g)]:
            fe, ge = [a] * lf, [c] * lg
            assert S.ks_mul_signed_offset(fe, ge, bf, bg, variant).h == pyref.poly_mul(fe, ge)


def test_signed_offset_range_fits_every_read():
    # the shifted coefficients lie in [0, 2K]; the top is reached by the all-minimum
    # product, and it must fit what each variant reads: a field of N (Sec. 3.1) or 2N
    # (Sec. 3.3) bits, and c < X (X - 1) for the reconstruction (Sec. 3.2: beta < X - 1)
    r = S.ks_mul_signed_offset([-1], [-1, -1, -1], 1, 1, 3)
    assert r.h == [1, 1, 1]
    for bf in range(1, 9):
        for bg in range(1, 9):
            for e in range(0, 7):
                top = 2 << (bf + bg - 2 + e)          # 2K
                N = [S.signed_N(v, bf, bg, e) for v in (1, 2, 3, 4)]
                assert top < 1 << N[0]
                assert top < 1 << (2 * N[1])
                X3, Y4 = 1 << N[2], 1 << (2 * N[3])
                assert top < X3 * (X3 - 1), (bf, bg, e)
                assert top < Y4 * (Y4 - 1)
    # at bf = bg = 1, e = 0 the reciprocal variant's own N = 1 gives X (X - 1) = 2 = 2K
    assert S.variant_N_bits(3, 1, 1, 0) == 1 and S.signed_N(3, 1, 1, 0) == 2


@pytest.mark.parametrize("X", [10, 2 ** 7, 2 ** 28, 2 ** 56])
@pytest.mark.parametrize("n,m", [(1, 4), (3, 4), (4, 4), (5, 4), (8, 4), (9, 4), (12, 4),
                                 (13, 4), (64, 8), (100, 16), (97, 32)])
def test_chains_alternate_down_and_up(X, n, m):
    # chain c covers [c m, (c+1) m): odd chains upward, even chains downward, one exact
    # pair (c_(s-1), c_s) at every s = m (2j + 1) starting two chains; the top chain
    # runs down from n without a seed
    rng = random.Random(X + 13 * n + m)
    c, fwd, rev = _rand_recoverable(n, X, rng)
    assert S.recover_chains(fwd, rev, n, X, m, c) == c
    # the chains read the exact values only at the pair positions
    used = {s + d for s in range(m, n, 2 * m) for d in (-1, 0)}
    masked = [c[i] if i in used else None for i in range(n)]
    assert S.recover_chains(fwd, rev, n, X, m, masked) == c


def test_chains_fail_with_a_wrong_seed():
    rng = random.Random(5)
    X, n, m = 2 ** 20, 64, 8
    c, fwd, rev = _rand_recoverable(n, X, rng)
    bad = list(c)
    bad[m] += 1                          # the first pair's c_s off by one
    try:
        out = S.recover_chains(fwd, rev, n, X, m, bad)
    except AssertionError:
        return                           # a carry check caught it
    assert out != c


def test_planted_offset_slip_fails(monkeypatch):
    # shifting one coefficient too few (U_(n-1) for U_n) breaks the pins
    good = S.ones
    monkeypatch.setattr(S, "ones", lambda n, Y: good(max(n - 1, 0), Y))
    rng = random.Random(11)
    f = [rng.randint(-128, 127) for _ in range(9)]
    g = [rng.randint(-128, 127) for _ in range(7)]
    for v in (1, 2, 3, 4):
        try:
            bad = S.ks_mul_signed_offset(f, g, 8, 8, v).h != pyref.poly_mul(f, g)
        except AssertionError:
            bad = True
        assert bad, v
