"""The batched plan: many uneven products (all variants and engines, signed and
unsigned) in one launch sequence, checked bit-exact against the oracle;
re-execution with new inputs in the same buffers; CUDA-graph capture and
replay; and a launch count that does not grow with the batch."""
import numpy as np
import pytest

import ks_inputs as gen
import oracle
from tests._gpu import assert_same, random_case, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    return ks


def _batch(ks, n, seed, len_hi=700, bits_hi=300, forced=True):
    import torch
    lf, lg, cb, sg = gen.uneven_batch(n, seed, 1, len_hi, 1, bits_hi)
    probs, host = [], []
    for i in range(n):
        f, g = random_case(int(lf[i]), int(lg[i]), int(cb[i]), bool(sg[i]), seed + 31 * i)
        ol = ks.out_limbs(int(lf[i]), int(lg[i]), int(cb[i]), bool(sg[i]))
        h = torch.full((int(lf[i] + lg[i] - 1), ol), -1, dtype=torch.int64, device="cuda")
        q = dict(h=h, f=to_dev(f), g=to_dev(g), coeff_bits=int(cb[i]), is_signed=bool(sg[i]))
        if forced:
            q["variant"] = [0, 1, 2, 3, 4][i % 5]
            q["engine"] = [0, 1, 2, 3][(i // 5) % 4]
        probs.append(q)
        host.append((f, g))
    return probs, host


def _check(ks, probs, host):
    for i, (q, (f, g)) in enumerate(zip(probs, host)):
        assert_same(to_host(q["h"]), oracle.mul(f, g, q["coeff_bits"], q["is_signed"]),
                    "batch item %d (len %d x %d, b=%d)" % (i, f.shape[0], g.shape[0],
                                                          q["coeff_bits"]))


def test_plan_mixed_batch(ks):
    probs, host = _batch(ks, 160, 11)
    plan = ks.Plan(probs)
    plan.execute()
    ks.status_sync()
    _check(ks, probs, host)
    # every variant and engine occurs
    choices = {plan.choice(i) for i in range(len(probs))}
    assert {v for v, _ in choices} == {1, 2, 3, 4}
    assert {e for _, e in choices} == {1, 2, 3}
    plan.close()


def test_plan_launches_do_not_grow_with_batch(ks):
    counts = []
    for n in (20, 400):
        probs, _ = _batch(ks, n, 5, len_hi=300, bits_hi=100, forced=False)
        plan = ks.Plan(probs)
        plan.execute()
        ks.status_sync()
        counts.append(plan.launches())
        plan.close()
    assert counts[1] <= 30, counts
    assert counts[1] <= counts[0] + 6, counts


def test_plan_reexecute_with_new_inputs(ks):
    import torch
    probs, host = _batch(ks, 60, 23)
    plan = ks.Plan(probs)
    plan.execute()
    # new coefficients in the same buffers
    new_host = []
    for i, q in enumerate(probs):
        f, g = random_case(q["f"].shape[0], q["g"].shape[0], q["coeff_bits"], q["is_signed"],
                           777 + i)
        q["f"].copy_(to_dev(f))
        q["g"].copy_(to_dev(g))
        new_host.append((f, g))
    torch.cuda.synchronize()
    plan.execute()
    ks.status_sync()
    _check(ks, probs, new_host)
    plan.close()


def test_plan_graph_capture_and_replay(ks):
    import torch
    probs, host = _batch(ks, 80, 41, forced=False)
    s = torch.cuda.Stream()
    plan = ks.Plan(probs, ks.DISPATCH_AUTO)
    plan.capture(s)
    for q in probs:
        q["h"].fill_(-1)
    torch.cuda.synchronize()
    for _ in range(3):
        plan.execute(s)
    s.synchronize()
    ks.status_sync(s)
    _check(ks, probs, host)
    plan.close()


def test_plan_dispatch_ks1(ks):
    probs, host = _batch(ks, 40, 3, forced=False)
    plan = ks.Plan(probs, ks.DISPATCH_KS1)
    plan.execute()
    ks.status_sync()
    assert all(plan.choice(i)[0] == 1 for i in range(len(probs)))
    _check(ks, probs, host)
    plan.close()
