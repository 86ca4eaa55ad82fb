"""Squaring (f = g, the same device buffer and length) on every engine and
variant, bit-exact against the oracle.  The int32-digit engines pack each
evaluation once and, on the transform engine, transform it once; the result
must be the same exact product.  A buffer passed on both sides with different
lengths is not a square and must still give f * g."""
import numpy as np
import pytest

import oracle
from tests._gpu import (assert_same, fingerprint_check, random_case, sampled_check, to_dev,
                        to_host)

pytestmark = pytest.mark.gpu

ENGINES = [1, 2, 3]
VARIANTS = [1, 2, 3, 4]


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    return ks


def _square(ks, f, b, signed, variant, engine):
    tf = to_dev(f)
    h = ks.mul(tf, tf, b, signed, variant, engine)
    ks.status_sync()
    return to_host(h)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("variant", VARIANTS)
def test_square_small(ks, engine, variant):
    for L, b, signed in ((1, 5, False), (2, 3, True), (300, 40, True), (2048, 64, False)):
        f, _ = random_case(L, 1, b, signed, 31 * L + b)
        assert_same(_square(ks, f, b, signed, variant, engine), oracle.mul(f, f, b, signed),
                    "square L=%d b=%d variant %d engine %d" % (L, b, variant, engine))


@pytest.mark.parametrize("variant", VARIANTS)
def test_square_transform_regime(ks, variant):
    # transform engine at a size where its forward transforms dominate
    L, b = 65536, 64
    f, _ = random_case(L, 1, b, False, 4242)
    got = _square(ks, f, b, False, variant, 2)
    fingerprint_check(got, f, f, False, variant, nchecks=2)
    sampled_check(got, f, f, b, False, 8, variant)


def test_same_buffer_different_lengths_is_not_a_square(ks):
    import torch
    b = 48
    f, _ = random_case(700, 1, b, True, 77)
    tf = to_dev(f)
    for engine in ENGINES:
        for variant in VARIANTS:
            # g is the first 300 coefficients of the same buffer
            g = tf[:300]
            ol = ks.out_limbs(700, 300, b, True)
            h = torch.empty((999, ol), dtype=torch.int64, device="cuda")
            ws = torch.empty(ks.workspace_bytes(700, 300, b, True, variant, engine) // 8 + 32,
                             dtype=torch.int64, device="cuda")
            ks.ks_mul_ex(h, tf, g, b, True, variant, engine, ws)
            ks.status_sync()
            assert_same(to_host(h), oracle.mul(f, f[:300], b, True),
                        "prefix of the same buffer, variant %d engine %d" % (variant, engine))


def test_square_in_a_batch(ks):
    import torch
    probs, want = [], []
    for i, (L, b, signed, variant, engine) in enumerate(
            [(500, 30, True, 4, 1), (500, 30, True, 2, 2), (1000, 64, False, 1, 2),
             (800, 20, False, 3, 3), (257, 47, True, 4, 2)]):
        f, g = random_case(L, L, b, signed, 600 + i)
        tf = to_dev(f)
        ol = ks.out_limbs(L, L, b, signed)
        for square in (True, False):
            h = torch.empty((2 * L - 1, ol), dtype=torch.int64, device="cuda")
            tg = tf if square else to_dev(g)
            probs.append(dict(h=h, f=tf, g=tg, coeff_bits=b, is_signed=signed, variant=variant,
                              engine=engine))
            want.append(oracle.mul(f, f if square else g, b, signed))
    plan = ks.Plan(probs)
    for _ in range(2):  # twice: the plan is reusable
        plan.execute()
        ks.status_sync()
        for i, (q, w) in enumerate(zip(probs, want)):
            assert_same(to_host(q["h"]), w, "batch product %d" % i)
    plan.close()
