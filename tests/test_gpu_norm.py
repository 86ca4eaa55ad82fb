"""The two forms of the carry normalization give the same words: the single
pass with look-back (used up to 2048 tile CTAs) and the tile pass plus carry
pass (used above), each forced on the same products, below and above the
size where the library switches, are bit-identical and match the oracle."""
import numpy as np
import pytest

import oracle
from tests._gpu import (assert_same, fingerprint_check, random_case, sampled_check, to_dev,
                        to_host)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    yield ks
    ks.lib.ks_debug_norm_form(0)


def _both_forms(ks, f, g, b, sg, v, e):
    out = []
    for form in (1, 2):
        ks.lib.ks_debug_norm_form(form)
        try:
            h = ks.mul(to_dev(f), to_dev(g), b, sg, v, e)
            ks.status_sync()
            out.append(to_host(h))
        finally:
            ks.lib.ks_debug_norm_form(0)
    return out


@pytest.mark.parametrize("case", [(3000, 2800, 48, True, 4, "ENGINE_TC"),
                                  (2500, 2400, 64, False, 1, "ENGINE_NTT"),
                                  (1900, 2100, 30, True, 2, "ENGINE_SCHOOLBOOK"),
                                  (2000, 1999, 40, False, 3, "ENGINE_TC")])
def test_forms_agree_small(ks, case):
    lf, lg, b, sg, v, eng = case
    f, g = random_case(lf, lg, b, sg, 7100 + lf)
    one, two = _both_forms(ks, f, g, b, sg, v, getattr(ks, eng))
    want = oracle.mul(f, g, b, sg)
    assert_same(one, want, "single pass %s" % (case,))
    assert_same(two, want, "two passes %s" % (case,))


@pytest.mark.parametrize("L", [32768, 65536])
def test_forms_agree_around_the_switch(ks, L):
    # KS1 on the transform, 64-bit: about 1150 tiles at L = 2^15, 2300 at 2^16
    f, g = random_case(L, L, 64, False, 7300 + L)
    info = ks.plan_info(L, L, 64, False, 1, ks.ENGINE_NTT)
    assert (info["nwords"] + 255) // 256 in range(1000, 2500)
    one, two = _both_forms(ks, f, g, 64, False, 1, ks.ENGINE_NTT)
    assert np.array_equal(one, two), "the two forms differ"
    sampled_check(one, f, g, 64, False, 24, 7400 + L)
    fingerprint_check(one, f, g, False, 7500 + L)
