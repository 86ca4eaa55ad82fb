"""Launch overlap (programmatic dependent launch) changes no result: every
variant and engine, by direct calls and by a captured plan of several
products, is exact against the oracle with the overlap on and off."""
import numpy as np
import pytest

import oracle
from tests._gpu import assert_same, gpu_mul, random_case, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    yield ks
    ks.set_pdl(False)


CASES = [  # (len_f, len_g, bits, signed, variant, engine name)
    (2500, 2300, 48, True, 4, "ENGINE_TC"),
    (2500, 2300, 48, True, 3, "ENGINE_TC"),
    (1800, 1700, 64, False, 1, "ENGINE_NTT"),
    (1800, 1700, 64, False, 2, "ENGINE_NTT"),
    (900, 1000, 20, True, 4, "ENGINE_SCHOOLBOOK"),
    (700, 650, 200, False, 4, "ENGINE_NTT"),
]


@pytest.mark.parametrize("pdl", [True, False])
@pytest.mark.parametrize("case", CASES)
def test_direct_calls_exact(ks, pdl, case):
    lf, lg, b, sg, variant, eng = case
    f, g = random_case(lf, lg, b, sg, 900 + lf + b)
    want = oracle.mul(f, g, b, sg)
    ks.set_pdl(pdl)
    try:
        for _ in range(2):  # back to back: the second call overlaps the first's tail
            got = gpu_mul(ks, f, g, b, sg, variant, getattr(ks, eng))
            assert_same(got, want, "pdl=%s %s" % (pdl, case))
    finally:
        ks.set_pdl(False)


@pytest.mark.parametrize("pdl", [True, False])
def test_plan_replays_exact(ks, pdl):
    import torch
    ks.set_pdl(pdl)
    try:
        jobs, wants, outs = [], [], []
        for i, (lf, lg, b, sg, variant) in enumerate(
                [(3000, 2900, 48, True, 4), (1200, 1300, 64, False, 1),
                 (2000, 1999, 30, True, 3), (500, 480, 300, False, 2)]):
            f, g = random_case(lf, lg, b, sg, 950 + i)
            wants.append(oracle.mul(f, g, b, sg))
            h = torch.zeros((lf + lg - 1, ks.out_limbs(lf, lg, b, sg)), dtype=torch.int64,
                            device="cuda")
            outs.append(h)
            jobs.append(dict(h=h, f=to_dev(f), g=to_dev(g), coeff_bits=b, is_signed=sg,
                             variant=variant))
        plan = ks.Plan(jobs)
        stream = torch.cuda.Stream()  # graph capture needs a stream of its own
        torch.cuda.synchronize()
        plan.capture(stream)
        for rep in range(3):
            with torch.cuda.stream(stream):
                for h in outs:
                    h.zero_()
            plan.execute(stream)
            plan.status()
            for h, want in zip(outs, wants):
                assert_same(to_host(h), want, "plan replay %d pdl=%s" % (rep, pdl))
        plan.close()
    finally:
        ks.set_pdl(False)
