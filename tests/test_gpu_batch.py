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


def test_plan_batches_transform_products(ks):
    # transform-engine products of a few lengths (several per length, squarings among
    # them, all four variants): one launch sequence per transform length and kind,
    # not one per product, and every result exact
    import torch
    probs, host = [], []
    for i in range(48):
        L = [200, 700, 1500, 3000][i % 4]
        lf, lg, b, sg = L + (i % 7), L - (i % 5), [16, 64, 130][i % 3], bool(i & 1)
        f, g = random_case(lf, lg, b, sg, 4400 + i)
        square = i % 8 == 0
        if square:
            g, lg = f, lf
        ol = ks.out_limbs(lf, lg, b, sg)
        df = to_dev(f)
        h = torch.full((lf + lg - 1, ol), -1, dtype=torch.int64, device="cuda")
        probs.append(dict(h=h, f=df, g=df if square else to_dev(g), coeff_bits=b, is_signed=sg,
                          variant=1 + i % 4, engine=ks.ENGINE_NTT))
        host.append((f, g))
    plan = ks.Plan(probs)
    plan.execute()
    plan.status()
    _check(ks, probs, host)
    few = plan.launches()
    plan.close()
    # the same products one per plan launch their transforms separately
    single = 0
    for q in probs[:8]:
        p1 = ks.Plan([q])
        p1.execute()
        p1.status()
        single += p1.launches()
        p1.close()
    _check(ks, probs[:8], host[:8])
    assert few < 0.5 * single * len(probs) / 8, (few, single)
