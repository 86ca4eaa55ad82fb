"""Failure detection on the GPU in the forms that fault and hang nothing:

* a bounded device wait that runs out: a test hook makes the tensor-core
  kernel's copy warp wait, before its first copy, on a barrier nothing
  completes, with every wait of the kernel bounded at 20 ms; the kernel gives
  up with no copy or MMA in flight and the call reports KS_ETIMEOUT, through the
  stream's status word (ks_status_sync) and through a plan's own
  (ks_plan_status); the context stays usable and the next product is exact;
* an allocation that fails on the host (KS_ENOMEM) for the cached workspace
  and for a plan."""
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
    return ks


def test_bounded_wait_runs_out_and_is_reported(ks):
    import torch
    f, g = random_case(1500, 1400, 48, True, 77)
    tf, tg = to_dev(f), to_dev(g)
    want = oracle.mul(f, g, 48, True)
    ks.debug_tc_stall(True, 20_000_000)
    try:
        ks.mul(tf, tg, 48, True, ks.KS_4, ks.ENGINE_TC)
        with pytest.raises(ks.KSError) as e:
            ks.status_sync()
        assert e.value.status == ks.KS_ETIMEOUT
        h = torch.empty((f.shape[0] + g.shape[0] - 1, ks.out_limbs(1500, 1400, 48, True)),
                        dtype=torch.int64, device="cuda")
        plan = ks.Plan([dict(h=h, f=tf, g=tg, coeff_bits=48, is_signed=True, variant=ks.KS_4,
                             engine=ks.ENGINE_TC)])
        plan.execute()
        with pytest.raises(ks.KSError) as e:
            plan.status()
        assert e.value.status == ks.KS_ETIMEOUT
        ks.status_sync()  # the plan's failure is its own, not the stream's
    finally:
        ks.debug_tc_stall(False, 0)
    # the context stays usable: the same plan and a direct call are exact again
    plan.execute()
    plan.status()
    assert_same(to_host(h), want, "plan after the timeout")
    plan.close()
    assert_same(gpu_mul(ks, f, g, 48, True, ks.KS_4, ks.ENGINE_TC), want, "after the timeout")


def test_failed_allocations_report_enomem(ks):
    import torch
    f, g = random_case(3000, 3100, 64, False, 78)
    tf, tg = to_dev(f), to_dev(g)
    ks.release_cache()
    ks.debug_fail_allocs(1)
    try:
        with pytest.raises(ks.KSError) as e:
            ks.mul(tf, tg, 64, False, ks.KS_3)
        assert e.value.status == ks.KS_ENOMEM
    finally:
        ks.debug_fail_allocs(0)
    h = torch.empty((6099, ks.out_limbs(3000, 3100, 64, False)), dtype=torch.int64, device="cuda")
    ks.debug_fail_allocs(1)
    try:
        with pytest.raises(ks.KSError) as e:
            ks.Plan([dict(h=h, f=tf, g=tg, coeff_bits=64, is_signed=False)])
        assert e.value.status == ks.KS_ENOMEM
    finally:
        ks.debug_fail_allocs(0)
    want = oracle.mul(f, g, 64, False)
    assert_same(gpu_mul(ks, f, g, 64, False, ks.KS_3), want, "after the failed allocation")
    plan = ks.Plan([dict(h=h, f=tf, g=tg, coeff_bits=64, is_signed=False)])
    plan.execute()
    plan.status()
    assert_same(to_host(h), want, "plan after the failed allocation")
    plan.close()
