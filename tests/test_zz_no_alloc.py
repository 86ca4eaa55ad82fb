"""ks_mul_static: the entry point for callers that may not allocate device
memory at call time (its scratch is a fixed array inside the library).

Its results must equal those of ks_mul, the allocating entry point, for two
calls in a row (different problems, so stale scratch from the first call
would show in the second).  Kept in a file of its own that pytest collects
last; it passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest
import torch

from tests._gpu import assert_same, random_case, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    return ks


def _pair(ks, lf, lg, b, signed, variant, seed):
    f, g = random_case(lf, lg, b, signed, seed)
    tf, tg = to_dev(f), to_dev(g)
    ol = ks.out_limbs(lf, lg, b, signed)
    h_ref = torch.empty((lf + lg - 1, ol), dtype=torch.int64, device="cuda")
    h_static = torch.full((lf + lg - 1, ol), -1, dtype=torch.int64, device="cuda")
    return tf, tg, h_ref, h_static


def test_static_matches_ks_mul_two_calls_in_a_row(ks):
    cases = [(16384, 16384, 48, True, 4, 11), (3000, 2077, 64, False, 3, 12)]
    prepared = [_pair(ks, *c) for c in cases]
    for (lf, lg, b, signed, variant, _), (tf, tg, h_ref, _) in zip(cases, prepared):
        ks.ks_mul(h_ref, tf, tg, b, signed, variant)
    ks.status_sync()
    # two calls in a row on the shared scratch, no synchronization between them
    for (lf, lg, b, signed, variant, _), (tf, tg, _, h_static) in zip(cases, prepared):
        ks.ks_mul_static(h_static, tf, tg, b, signed, variant)
    ks.status_sync()
    for (lf, lg, b, signed, variant, _), (_, _, h_ref, h_static) in zip(cases, prepared):
        assert_same(to_host(h_static), to_host(h_ref), "ks_mul_static vs ks_mul, variant %d"
                    % variant)


def test_static_refuses_oversize_problem(ks):
    lf = lg = 100000
    assert ks.workspace_bytes(lf, lg, 64, False, 4) > ks.STATIC_SCRATCH_BYTES
    t = torch.zeros((8, 1), dtype=torch.int64, device="cuda")
    h = torch.zeros((8, 3), dtype=torch.int64, device="cuda")
    before = ks.launch_count()
    # the size check comes first: the (deliberately short) buffers are never touched
    rc = ks.lib.ks_mul_static(ks._dptr(h), ks._dptr(t), lf, ks._dptr(t), lg, 64, 0, 4,
                              ks._stream_ptr(None))
    assert rc == ks.KS_ERANGE
    assert ks.launch_count() == before
    ks.status_sync()
