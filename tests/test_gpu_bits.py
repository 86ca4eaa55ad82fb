"""Products with different coefficient sizes in f and g (ks_mul_bits, and
batch problems with coeff_bits_g), planned with N from bf + bg (Sec. 3.1-3.4
with bf + bg in place of 2b), exact against the oracle: the plain product of
the integer polynomials, written with ks_out_limbs_bits limbs."""
import numpy as np
import pytest

import ks_inputs as gen
import oracle
from oracle import pyref
from tests._gpu import assert_same, to_dev, to_host

pytestmark = pytest.mark.gpu

# (len_f, bits_f, len_g, bits_g): ragged lengths, limb counts that differ, the
# 1- and 4-bit regimes against wide partners
CASES = [(300, 48, 200, 16), (200, 16, 300, 48), (100, 130, 150, 20), (64, 64, 64, 65),
         (1, 5, 700, 200), (500, 3, 1, 1), (257, 70, 129, 64), (333, 4, 222, 61),
         (97, 1, 131, 128)]
# larger shapes that reach the tensor-core and transform engines under KS_AUTO
LARGE = [(4000, 4, 3000, 60), (3000, 1, 2000, 64), (2500, 4, 2501, 4), (1800, 200, 1700, 40)]


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    return ks


def widen(a: np.ndarray, il: int, signed: bool) -> np.ndarray:
    """The same coefficients with il >= a.shape[1] limbs (sign- or zero-extended)."""
    out = np.zeros((a.shape[0], il), dtype=np.uint64)
    out[:, :a.shape[1]] = a
    if signed and il > a.shape[1]:
        neg = (a[:, -1] >> np.uint64(63)) == 1
        out[neg, a.shape[1]:] = np.uint64(0xFFFFFFFFFFFFFFFF)
    return out


def want_product(ks, f, bf, g, bg, signed):
    """The oracle's product at max(bf, bg) bits, written with the unequal-size limbs
    (the high limbs it drops are the sign- or zero-extension of the value)."""
    B = max(bf, bg)
    il = (B + 63) // 64
    ol = ks.out_limbs_bits(f.shape[0], g.shape[0], bf, bg, signed)
    full = oracle.mul(widen(f, il, signed), widen(g, il, signed), B, signed)
    return np.ascontiguousarray(full[:, :ol]), full


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("signed", [False, True])
def test_unequal_bit_sizes(ks, variant, signed):
    import torch
    for i, (lf, bf, lg, bg) in enumerate(CASES):
        f = gen.random_poly(lf, bf, signed, 1000 + i)
        g = gen.random_poly(lg, bg, signed, 2000 + i)
        ol = ks.out_limbs_bits(lf, lg, bf, bg, signed)
        h = torch.empty((lf + lg - 1, ol), dtype=torch.int64, device="cuda")
        ks.ks_mul_bits(h, to_dev(f), bf, to_dev(g), bg, signed, variant)
        ks.status_sync()
        want = pyref.poly_mul(gen.to_ints(f, signed), gen.to_ints(g, signed))
        assert_same(to_host(h), gen.from_ints(want, 64 * ol),
                    "bits %d x %d, variant %d, signed %s" % (bf, bg, variant, signed))


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("signed", [False, True])
def test_unequal_bit_sizes_large(ks, variant, signed):
    import torch
    for i, (lf, bf, lg, bg) in enumerate(LARGE):
        f = gen.random_poly(lf, bf, signed, 3000 + i)
        g = gen.random_poly(lg, bg, signed, 4000 + i)
        want, full = want_product(ks, f, bf, g, bg, signed)
        # the dropped limbs are the extension of what is kept
        top = want[:, -1].view(np.int64) < 0 if signed else np.zeros(want.shape[0], bool)
        ext = np.where(top, np.uint64(0xFFFFFFFFFFFFFFFF), np.uint64(0))
        for l in range(want.shape[1], full.shape[1]):
            assert np.array_equal(full[:, l], ext)
        h = torch.empty(want.shape, dtype=torch.int64, device="cuda")
        ks.ks_mul_bits(h, to_dev(f), bf, to_dev(g), bg, signed, variant)
        ks.status_sync()
        assert_same(to_host(h), want, "bits %d x %d (L %d, %d), variant %d, signed %s"
                    % (bf, bg, lf, lg, variant, signed))


@pytest.mark.parametrize("engine", ["ENGINE_SCHOOLBOOK", "ENGINE_TC", "ENGINE_NTT"])
def test_unequal_bit_sizes_in_plans(ks, engine):
    # every engine and variant, as batch problems with coeff_bits_g, in one plan
    import torch
    jobs, wants = [], []
    for i, (lf, bf, lg, bg, sg) in enumerate(
            [(900, 4, 700, 60, True), (600, 64, 650, 1, False), (400, 130, 300, 20, True),
             (1000, 4, 1000, 4, False), (257, 48, 129, 16, True)]):
        for variant in (1, 2, 3, 4):
            f = gen.random_poly(lf, bf, sg, 5000 + 10 * i + variant)
            g = gen.random_poly(lg, bg, sg, 6000 + 10 * i + variant)
            want, _ = want_product(ks, f, bf, g, bg, sg)
            h = torch.zeros(want.shape, dtype=torch.int64, device="cuda")
            jobs.append(dict(h=h, f=to_dev(f), g=to_dev(g), coeff_bits=bf, coeff_bits_g=bg,
                             is_signed=sg, variant=variant, engine=getattr(ks, engine)))
            wants.append(want)
    plan = ks.Plan(jobs)
    plan.execute()
    plan.status()
    for j, want in zip(jobs, wants):
        assert_same(to_host(j["h"]), want, "%s %d x %d variant %d"
                    % (engine, j["coeff_bits"], j["coeff_bits_g"], j["variant"]))
    plan.close()


def test_plan_info_matches_the_product(ks):
    # the N the plan reports is the one of bf + bg (KS_1: bf + bg + e), below that of
    # two max(bf, bg)-bit operands
    info = ks.plan_info(3000, 2000, 1, False, 1, ks.ENGINE_TC, bits_g=64)
    assert info["N"] == 1 + 64 + 11
    assert info["N"] < ks.plan_info(3000, 2000, 64, False, 1, ks.ENGINE_TC)["N"]


def test_equal_limbs_matches_ks_mul(ks):
    # equal sizes through ks_mul_bits: the same plan and result as ks_mul
    f = gen.random_poly(4000, 48, True, 5)
    g = gen.random_poly(3000, 48, True, 6)
    import torch
    ol = ks.out_limbs(4000, 3000, 48, True)
    assert ol == ks.out_limbs_bits(4000, 3000, 48, 48, True)
    h = torch.empty((6999, ol), dtype=torch.int64, device="cuda")
    ks.ks_mul_bits(h, to_dev(f), 48, to_dev(g), 48, True)
    ks.status_sync()
    assert_same(to_host(h), oracle.mul(f, g, 48, True), "48 x 48 bits")
