"""Step model of the four Kronecker-substitution variants -- TEST INFRASTRUCTURE ONLY.

Each variant is run on Python integers, following the steps of Harvey's
Sec. 3 in the paper's order and notation, in any base: the evaluation point is
X = base^N, so base 2 gives the method itself and base 10 replays the paper's
worked examples (Sec. 1, and the examples of Sec. 3.2, 3.3 and 3.4).  Every
intermediate (evaluations, products, combined halves, the digits u_i and
w_i, and the reconstruction's alpha_i, beta_i, delta_i, epsilon_i) is returned
so that tests can pin it.

Readings of the paper used here (the paper is silent or garbled on them):

* Unequal lengths: Lh = Lf + Lg - 1 replaces 2L - 1, and
  e = ceil(log_base min(Lf, Lg)) bounds the number of terms per h_k.
* Reversal: rev f(x) = x^(Lf-1) f(1/x), i.e. the coefficient list reversed.
  The four-point variant's reversed pair is taken as rev f(+-X) rev g(+-X) =
  rev h(+-X); this reproduces the printed values of the Sec. 3.4 example,
  whose sign of 10^6 f(-10^-2) differs from the displayed sum formula of
  Sec. 2.4 by (-1)^(L-1).
* Four-point pairing: when Lh is even, the even-index half of rev h holds the
  odd coefficients of h, so the even coefficients come from (E, OR) and the
  odd ones from (O, ER).
* Signed coefficients (the paper treats non-negative ones only), two readings:
  - bias: bias each coefficient by c = 2^(b-1) to make it non-negative,
    multiply, and subtract c (f U_g + U_f g) + c^2 U_f U_g, with U the
    all-ones polynomial;
  - offset: evaluate the signed coefficients as they are (the evaluations of
    Sec. 3.3 are signed anyway), then add K U_h(Y) to every integer that the
    coefficients are read from (K = 2^(bf + bg - 2 + e), Y the digit base of
    that integer), which shifts every coefficient into [0, 2K] -- the
    non-negative range the read-off and the reconstruction of Sec. 3 need --
    and subtract K from each coefficient read.  |h_k| <= min(Lf, Lg)
    2^(bf - 1) 2^(bg - 1) <= K.
"""
from __future__ import annotations

from dataclasses import dataclass, field


def ceil_log(n: int, base: int) -> int:
    """Smallest e >= 0 with base^e >= n."""
    e, p = 0, 1
    while p < n:
        p *= base
        e += 1
    return e


def variant_N(variant: int, b: int, e: int) -> int:
    """The evaluation exponent N of each variant (Sec. 3.1-3.4)."""
    if variant == 1:
        return 2 * b + e                      # Sec. 3.1
    if variant in (2, 3):
        return b + (e + 1) // 2               # Sec. 3.3 and Sec. 3.2
    if variant == 4:
        return (2 * b + e + 3) // 4           # Sec. 3.4
    raise ValueError("variant must be 1..4")


def evaluate(coeffs: list[int], X: int) -> int:
    """sum_i c_i X^i (Horner), for any integer X, positive or negative."""
    v = 0
    for c in reversed(coeffs):
        v = v * X + c
    return v


def digit(v: int, i: int, X: int) -> int:
    """The i-th base-X digit of the non-negative integer v."""
    return (v // X ** i) % X


def even_odd(coeffs: list[int]) -> tuple[list[int], list[int]]:
    return coeffs[0::2], coeffs[1::2]


def eval_pm(coeffs: list[int], X: int) -> tuple[int, int]:
    """f(X) and f(-X) from the even and odd parts, as Sec. 3.3 describes:
    f(+-X) = f0(X^2) +- X f1(X^2), each part packed at spacing 2N without overlap."""
    f0, f1 = even_odd(coeffs)
    e = evaluate(f0, X * X)
    o = X * evaluate(f1, X * X)
    return e + o, e - o


@dataclass
class Recovery:
    h: list[int]
    alpha: list[int]
    beta: list[int]
    delta: list[int]
    eps: list[int]
    u: list[int]
    w: list[int]


def recover(fwd: int, rev: int, n: int, X: int) -> Recovery:
    """Reciprocal reconstruction of Sec. 3.2 (eqs. for digits u_i, w_i and carries).

    fwd = sum_{i<n} c_i X^i and rev = sum_{i<n} c_{n-1-i} X^i, with
    0 <= c_i < X (X - 1).  Returns c_0..c_{n-1} and the intermediates.
    Digits: fwd = sum_{i=0}^{n} u_i X^i;  rev = sum_{i=0}^{n} w_{n-i} X^i.
    """
    if n < 1:
        raise ValueError("need at least one coefficient")
    u = [digit(fwd, i, X) for i in range(n + 1)]
    w = [digit(rev, n - j, X) for j in range(n + 1)]
    alpha = [0] * n
    beta = [0] * n
    delta = [0] * n
    eps = [0] * n
    alpha[0] = u[0]
    a_prev = 0                                # alpha_{-1}
    for j in range(n - 1):
        # epsilon_j: carry out of alpha_j + beta_{j+1} + eps_{j+1} in rev
        eps[j] = 1 if alpha[j] > w[j + 1] else 0
        beta[j] = (w[j] - a_prev - eps[j]) % X
        alpha[j + 1] = (u[j + 1] - beta[j] - delta[j]) % X
        t = beta[j] + alpha[j + 1] + delta[j] - u[j + 1]
        assert t % X == 0
        delta[j + 1] = t // X
        a_prev = alpha[j]
    beta[n - 1] = (w[n - 1] - a_prev - 0) % X   # eps_{n-1} = 0
    h = [alpha[i] + X * beta[i] for i in range(n)]
    return Recovery(h, alpha, beta, delta, eps, u, w)


@dataclass
class Run:
    variant: int
    X: int
    h: list[int]
    evals: dict = field(default_factory=dict)
    products: dict = field(default_factory=dict)
    halves: dict = field(default_factory=dict)
    recoveries: list = field(default_factory=list)


def ks1(f: list[int], g: list[int], X: int) -> Run:
    """Standard substitution (Sec. 3.1): one product at X, coefficients read off base X."""
    F, G = evaluate(f, X), evaluate(g, X)
    P = F * G
    lh = len(f) + len(g) - 1
    h = [digit(P, k, X) for k in range(lh)]
    return Run(1, X, h, {"F": F, "G": G}, {"P": P})


def ks2(f: list[int], g: list[int], X: int) -> Run:
    """Negated points (Sec. 3.3): products at +X and -X; even coefficients from
    (P+ + P-)/2 = h0(X^2), odd ones from (P+ - P-)/2 = X h1(X^2)."""
    Fp, Fm = eval_pm(f, X)
    Gp, Gm = eval_pm(g, X)
    Pp, Pm = Fp * Gp, Fm * Gm
    assert (Pp + Pm) % 2 == 0 and (Pp - Pm) % (2 * X) == 0
    E = (Pp + Pm) // 2
    Oh = (Pp - Pm) // 2
    lh = len(f) + len(g) - 1
    Y = X * X
    h = [0] * lh
    for k in range(lh):
        h[k] = digit(E, k // 2, Y) if k % 2 == 0 else digit(Oh // X, k // 2, Y)
    return Run(2, X, h, {"F+": Fp, "F-": Fm, "G+": Gp, "G-": Gm},
               {"P+": Pp, "P-": Pm}, {"E": E, "XO": Oh})


def ks3(f: list[int], g: list[int], X: int) -> Run:
    """Reciprocal points (Sec. 3.2): P = f(X) g(X) and R = rev f(X) rev g(X)
    = X^(Lh-1) h(1/X); the coefficients come from the reconstruction."""
    F, G = evaluate(f, X), evaluate(g, X)
    Fr, Gr = evaluate(f[::-1], X), evaluate(g[::-1], X)
    P, R = F * G, Fr * Gr
    lh = len(f) + len(g) - 1
    rec = recover(P, R, lh, X)
    return Run(3, X, rec.h, {"F": F, "G": G, "Fr": Fr, "Gr": Gr}, {"P": P, "R": R},
               recoveries=[rec])


def ks4(f: list[int], g: list[int], X: int) -> Run:
    """Four points (Sec. 3.4): products at +-X and, reversed, at +-1/X; the
    combined halves at Y = X^2 feed two runs of the Sec. 3.2 reconstruction,
    one for the even-index and one for the odd-index coefficients."""
    Fp, Fm = eval_pm(f, X)
    Gp, Gm = eval_pm(g, X)
    Frp, Frm = eval_pm(f[::-1], X)
    Grp, Grm = eval_pm(g[::-1], X)
    Pp, Pm, Rp, Rm = Fp * Gp, Fm * Gm, Frp * Grp, Frm * Grm
    for a, b in ((Pp, Pm), (Rp, Rm)):
        assert (a + b) % 2 == 0 and (a - b) % (2 * X) == 0
    E, O = (Pp + Pm) // 2, (Pp - Pm) // (2 * X)
    ER, OR = (Rp + Rm) // 2, (Rp - Rm) // (2 * X)
    lh = len(f) + len(g) - 1
    n0, n1 = (lh + 1) // 2, lh // 2
    Y = X * X
    even_pair = (E, ER) if lh % 2 == 1 else (E, OR)
    odd_pair = (O, OR) if lh % 2 == 1 else (O, ER)
    rec0 = recover(even_pair[0], even_pair[1], n0, Y)
    recs = [rec0]
    h = [0] * lh
    h[0::2] = rec0.h
    if n1 > 0:
        rec1 = recover(odd_pair[0], odd_pair[1], n1, Y)
        recs.append(rec1)
        h[1::2] = rec1.h
    return Run(4, X, h,
               {"F+": Fp, "F-": Fm, "Fr+": Frp, "Fr-": Frm,
                "G+": Gp, "G-": Gm, "Gr+": Grp, "Gr-": Grm},
               {"P+": Pp, "P-": Pm, "R+": Rp, "R-": Rm},
               {"E": E, "O": O, "ER": ER, "OR": OR,
                "XO": (Pp - Pm) // 2, "XOR": (Rp - Rm) // 2},
               recs)


VARIANTS = {1: ks1, 2: ks2, 3: ks3, 4: ks4}


def ks_mul_unsigned(f: list[int], g: list[int], b: int, variant: int, base: int = 2) -> Run:
    """Runs one variant with the paper's N for coefficients of at most b base-digits."""
    if min(f) < 0 or min(g) < 0:
        raise ValueError("the paper's variants take non-negative coefficients")
    e = ceil_log(min(len(f), len(g)), base)
    N = variant_N(variant, b, e)
    return VARIANTS[variant](f, g, base ** N)


def variant_N_bits(variant: int, bf: int, bg: int, e: int) -> int:
    """N for coefficient sizes bf (f) and bg (g).  The coefficients of h are below
    min(Lf, Lg) 2^(bf + bg), so bf + bg takes the place of 2b in Sec. 3.1-3.4."""
    s = bf + bg + e
    if variant == 1:
        return s
    if variant in (2, 3):
        return (s + 1) // 2
    if variant == 4:
        return (s + 3) // 4
    raise ValueError("variant must be 1..4")


def ks_mul_unsigned_bits(f: list[int], g: list[int], bf: int, bg: int, variant: int,
                         base: int = 2) -> Run:
    """One variant for coefficients of at most bf (f) and bg (g) base-digits."""
    if min(f) < 0 or min(g) < 0:
        raise ValueError("the paper's variants take non-negative coefficients")
    e = ceil_log(min(len(f), len(g)), base)
    return VARIANTS[variant](f, g, base ** variant_N_bits(variant, bf, bg, e))


def ks_mul_signed_bits(f: list[int], g: list[int], bf: int, bg: int, variant: int) -> list[int]:
    """Signed coefficients, f in [-2^(bf-1), 2^(bf-1)) and g in [-2^(bg-1), 2^(bg-1)):
    the bias reading with one bias per operand, cf = 2^(bf-1) and cg = 2^(bg-1);
    h = h' - cg (f U_g) - cf (U_f g) - cf cg (U_f U_g)."""
    cf, cg = 1 << (bf - 1), 1 << (bg - 1)
    hb = ks_mul_unsigned_bits([x + cf for x in f], [x + cg for x in g], bf, bg, variant).h
    lf, lg = len(f), len(g)
    out = []
    for k in range(lf + lg - 1):
        lo, hi = max(0, k - lg + 1), min(k, lf - 1)
        lo2, hi2 = max(0, k - lf + 1), min(k, lg - 1)
        out.append(hb[k] - cg * sum(f[lo:hi + 1]) - cf * sum(g[lo2:hi2 + 1])
                   - cf * cg * (hi - lo + 1))
    return out


def ks_mul_signed(f: list[int], g: list[int], b: int, variant: int) -> list[int]:
    """Signed coefficients in [-2^(b-1), 2^(b-1)) by the bias reading (see module doc)."""
    c = 1 << (b - 1)
    fb = [x + c for x in f]
    gb = [x + c for x in g]
    hb = ks_mul_unsigned(fb, gb, b, variant).h
    lf, lg = len(f), len(g)
    out = []
    for k in range(lf + lg - 1):
        lo, hi = max(0, k - lg + 1), min(k, lf - 1)
        wf = sum(f[lo:hi + 1])                       # (f * U_g)_k
        lo2, hi2 = max(0, k - lf + 1), min(k, lg - 1)
        wg = sum(g[lo2:hi2 + 1])                     # (U_f * g)_k
        cnt = hi - lo + 1                            # (U_f * U_g)_k
        out.append(hb[k] - c * (wf + wg) - c * c * cnt)
    return out


def signed_N(variant: int, bf: int, bg: int, e: int) -> int:
    """N of the offset reading.  The shifted coefficients lie in [0, 2^(s-1)],
    s = bf + bg + e, one bit below the unsigned bound 2^s, so the Propositions'
    N still holds, except for the reciprocal variant at s = 2 (bf = bg = 1,
    e = 0), where X (X - 1) = 2 is not above 2^(s-1) = 2: there N = 2."""
    N = variant_N_bits(variant, bf, bg, e)
    if variant == 3 and bf + bg + e <= 2:
        N = 2
    return N


def ones(n: int, Y: int) -> int:
    """U_n(Y) = 1 + Y + ... + Y^(n-1)."""
    return sum(Y ** i for i in range(n))


def ks_mul_signed_offset(f: list[int], g: list[int], bf: int, bg: int, variant: int) -> Run:
    """Signed coefficients, f in [-2^(bf-1), 2^(bf-1)), g in [-2^(bg-1), 2^(bg-1)),
    by the offset reading (module doc): the variant's evaluations and products
    on the signed values, K U(Y) added to what the coefficients are read from,
    the unsigned read-off or reconstruction, K subtracted.  Returns the Run with
    h the signed coefficients and `halves` holding the shifted integers."""
    lf, lg = len(f), len(g)
    lh = lf + lg - 1
    e = ceil_log(min(lf, lg), 2)
    N = signed_N(variant, bf, bg, e)
    K = 1 << (bf + bg - 2 + e)
    X = 1 << N
    if variant == 1:
        P = evaluate(f, X) * evaluate(g, X)
        Ps = P + K * ones(lh, X)
        hs = [digit(Ps, k, X) for k in range(lh)]
        return Run(1, X, [c - K for c in hs], {}, {"P": P}, {"P'": Ps})
    Y = X * X
    n0, n1 = (lh + 1) // 2, lh // 2
    if variant == 2:
        Fp, Fm = eval_pm(f, X)
        Gp, Gm = eval_pm(g, X)
        Pp, Pm = Fp * Gp, Fm * Gm
        E, O = (Pp + Pm) // 2, (Pp - Pm) // (2 * X)
        Es, Os = E + K * ones(n0, Y), O + K * ones(n1, Y)
        hs = [digit(Es, k // 2, Y) if k % 2 == 0 else digit(Os, k // 2, Y) for k in range(lh)]
        return Run(2, X, [c - K for c in hs], {}, {"P+": Pp, "P-": Pm}, {"E'": Es, "O'": Os})
    if variant == 3:
        P = evaluate(f, X) * evaluate(g, X)
        R = evaluate(f[::-1], X) * evaluate(g[::-1], X)
        Ps, Rs = P + K * ones(lh, X), R + K * ones(lh, X)
        rec = recover(Ps, Rs, lh, X)
        return Run(3, X, [c - K for c in rec.h], {}, {"P": P, "R": R}, {"P'": Ps, "R'": Rs},
                   [rec])
    Fp, Fm = eval_pm(f, X)
    Gp, Gm = eval_pm(g, X)
    Frp, Frm = eval_pm(f[::-1], X)
    Grp, Grm = eval_pm(g[::-1], X)
    Pp, Pm, Rp, Rm = Fp * Gp, Fm * Gm, Frp * Grp, Frm * Grm
    E, O = (Pp + Pm) // 2, (Pp - Pm) // (2 * X)
    ER, OR = (Rp + Rm) // 2, (Rp - Rm) // (2 * X)
    # each holds the coefficients of one parity class of h or of rev h
    Es, Os = E + K * ones(n0, Y), O + K * ones(n1, Y)
    ERs, ORs = ER + K * ones(n0, Y), OR + K * ones(n1, Y)
    even_pair = (Es, ERs) if lh % 2 == 1 else (Es, ORs)
    odd_pair = (Os, ORs) if lh % 2 == 1 else (Os, ERs)
    hs = [0] * lh
    recs = [recover(even_pair[0], even_pair[1], n0, Y)]
    hs[0::2] = recs[0].h
    if n1 > 0:
        recs.append(recover(odd_pair[0], odd_pair[1], n1, Y))
        hs[1::2] = recs[1].h
    return Run(4, X, [c - K for c in hs], {},
               {"P+": Pp, "P-": Pm, "R+": Rp, "R-": Rm},
               {"E'": Es, "O'": Os, "ER'": ERs, "OR'": ORs}, recs)


def recover_chains(fwd: int, rev: int, n: int, X: int, m: int, exact: list[int]) -> list[int]:
    """The reconstruction of Sec. 3.2 split into chains of m coefficients that
    need no predecessor: chain c covers [c m, (c + 1) m).  An odd chain runs
    upward from s = c m, an even one downward from s = (c + 1) m, both started
    by the exact pair (c_(s-1), c_s) taken from `exact` (a downward chain is the
    same recurrence on the reversed problem x^(n-1) h(1/x), whose fwd is rev and
    whose rev is fwd).  An even chain whose s would reach n runs downward from
    n without a seed (the reversed problem's start at index 0).  Each pair of
    exact values therefore starts two chains."""
    u = [digit(fwd, i, X) for i in range(n + 1)]
    w = [digit(rev, n - j, X) for j in range(n + 1)]
    out = [None] * n

    def chain(du, dw, length, seed, last_at):
        # du[t], dw[t]: the chain's own digits u, w at step t (t = 0 .. length)
        if seed is None:
            a_prev, a_cur, delta = 0, du[0], 0
        else:
            sp, sc = seed
            a_prev, b_prev, a_cur = sp % X, sp // X, sc % X
            d_prev = (du[0] - b_prev - a_cur) % X
            assert d_prev in (0, 1)
            delta = (b_prev + a_cur + d_prev - du[0]) // X
        w_cur = dw[0]
        res = []
        for t in range(length):
            if t != last_at:
                eps = 1 if a_cur > dw[t + 1] else 0
                beta = (w_cur - a_prev - eps) % X
                a_next = (du[t + 1] - beta - delta) % X
                d_next = (beta + a_next + delta - du[t + 1]) // X
                assert d_next in (0, 1)
                res.append(a_cur + X * beta)
                a_prev, a_cur, delta, w_cur = a_cur, a_next, d_next, dw[t + 1]
            else:
                res.append(a_cur + X * ((w_cur - a_prev) % X))
        return res

    nch = (n + m - 1) // m
    for c in range(nch):
        lo, hi = c * m, min((c + 1) * m, n)
        if c % 2 == 1:                       # upward from s = c m
            s = lo
            du = [u[s + t] for t in range(hi - s + 1)]
            dw = [w[s + t] for t in range(hi - s + 1)]
            vals = chain(du, dw, hi - s, (exact[s - 1], exact[s]),
                         (n - 1 - s) if hi == n else -1)
            for t, v in enumerate(vals):
                out[s + t] = v
        else:                                # downward from s = (c + 1) m, or from n
            s = hi
            seeded = s <= n - 1
            du = [w[s - t] for t in range(s - lo + 1)]
            dw = [u[s - t] for t in range(s - lo + 1)]
            seed = (exact[s], exact[s - 1]) if seeded else None
            vals = chain(du, dw, s - lo, seed, (s - 1) if lo == 0 else -1)
            for t, v in enumerate(vals):
                out[s - 1 - t] = v
    return out


# ---------------------------------------------------------------- Sec. 2.5
def _pmul(a: list[int], b: list[int], p: int) -> list[int]:
    """a b in (Z/pZ)[x] by the plain convolution."""
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] = (out[i + j] + x * y) % p
    return out


def biv_complex_points(f: list[list[int]], g: list[list[int]], p: int) -> dict:
    """h = f g in (Z/pZ)[x, y] (f[i][j]: the coefficient of x^j y^i) by the
    complex evaluation points of Sec. 2.5, p odd.

    M = ceil(lx / 2); S = R[i] with i^2 = -1 (pairs re + i im, so any odd p).
    The three points y = x^M, -x^M, i x^M give H1 = h(x, x^M), H2 = h(x, -x^M)
    (two products in R[x]) and h(x, i x^M) = F G with F = f(x, i x^M) =
    F_re + i F_im: a complex product, done with three products in R[x]
    (F_re G_re, F_im G_im, (F_re + F_im)(G_re + G_im)) -- five in all.

    The reading of "appropriate linear combinations": with A_r the sum of the
    terms h_k(x) x^(kM) whose rows k are r (mod 4),
      H1 = A0 + A1 + A2 + A3,  H2 = A0 - A1 + A2 - A3,
      Re h(x, i x^M) = A0 - A2,  Im h(x, i x^M) = A1 - A3,
    so A0 = (H1 + H2 + 2 Re) / 4, A2 = (H1 + H2 - 2 Re) / 4,
       A1 = (H1 - H2 + 2 Im) / 4, A3 = (H1 - H2 - 2 Im) / 4,
    and, as h_k has length 2 lx - 1 <= 4M - 1, the rows of one A_r do not
    overlap: h_k is read off A_(k mod 4) at x^(kM).  Returns h and the
    intermediates."""
    if p % 2 == 0:
        raise ValueError("Sec. 2.5's combinations halve: p must be odd")
    ly, lx = len(f), len(f[0])
    M = (lx + 1) // 2
    LF = M * (ly - 1) + lx

    def ev(a, sign_of_row, rows):
        out = [0] * LF
        for r in rows:
            s = sign_of_row(r)
            for j, c in enumerate(a[r]):
                out[r * M + j] = (out[r * M + j] + s * c) % p
        return out

    allr = range(ly)
    # f(x, +-x^M), and f(x, i x^M) = F_re + i F_im (i^r = (-1)^(r/2) or i (-1)^((r-1)/2))
    Fp = ev(f, lambda r: 1, allr)
    Fm = ev(f, lambda r: -1 if r % 2 else 1, allr)
    Fre = ev(f, lambda r: -1 if (r // 2) % 2 else 1, range(0, ly, 2))
    Fim = ev(f, lambda r: -1 if (r // 2) % 2 else 1, range(1, ly, 2))
    Gp = ev(g, lambda r: 1, allr)
    Gm = ev(g, lambda r: -1 if r % 2 else 1, allr)
    Gre = ev(g, lambda r: -1 if (r // 2) % 2 else 1, range(0, ly, 2))
    Gim = ev(g, lambda r: -1 if (r // 2) % 2 else 1, range(1, ly, 2))
    H1, H2 = _pmul(Fp, Gp, p), _pmul(Fm, Gm, p)
    P3, P4 = _pmul(Fre, Gre, p), _pmul(Fim, Gim, p)
    P5 = _pmul([(x + y) % p for x, y in zip(Fre, Fim)], [(x + y) % p for x, y in zip(Gre, Gim)], p)
    Re = [(x - y) % p for x, y in zip(P3, P4)]
    Im = [(z - x - y) % p for x, y, z in zip(P3, P4, P5)]
    inv4 = pow(4, -1, p)
    A = [[(x + y + 2 * r) * inv4 % p for x, y, r in zip(H1, H2, Re)],
         [(x - y + 2 * m) * inv4 % p for x, y, m in zip(H1, H2, Im)],
         [(x + y - 2 * r) * inv4 % p for x, y, r in zip(H1, H2, Re)],
         [(x - y - 2 * m) * inv4 % p for x, y, m in zip(H1, H2, Im)]]
    hx = 2 * lx - 1
    h = [[A[k % 4][k * M + j] for j in range(hx)] for k in range(2 * ly - 1)]
    return {"h": h, "M": M, "H1": H1, "H2": H2, "Re": Re, "Im": Im, "A": A,
            "products": 5}
