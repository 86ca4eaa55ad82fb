"""The host-buffer entry point (ks_mul_host) replays its captured launches:
repeated calls with new inputs in the same host buffers, alternating problems
(each change captures afresh) and a launch-overlap toggle between calls, on a
stream of its own and on the default stream, are exact against the oracle."""
import numpy as np
import pytest

import oracle
from tests._gpu import assert_same, random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    yield ks
    ks.set_pdl(False)


def _pinned(shape):
    import torch
    return torch.empty(shape, dtype=torch.int64).pin_memory().numpy().view(np.uint64)


PROBLEMS = [(3000, 2900, 48, True, 4, 0), (3000, 2900, 48, True, 1, 0),
            (1500, 1700, 64, False, 3, 0), (900, 800, 200, True, 2, 0),
            (3000, 2900, 48, True, 4, 0)]


@pytest.mark.parametrize("own_stream", [True, False])
def test_repeated_host_calls_exact(ks, own_stream):
    import torch
    stream = torch.cuda.Stream() if own_stream else None
    for i, (lf, lg, b, sg, v, e) in enumerate(PROBLEMS):
        ol = ks.out_limbs(lf, lg, b, sg)
        il = (b + 63) // 64
        fh, gh, hh = _pinned((lf, il)), _pinned((lg, il)), _pinned((lf + lg - 1, ol))
        for rep in range(3):  # the first call captures, the next ones replay
            f, g = random_case(lf, lg, b, sg, 600 + 10 * i + rep)
            fh[:] = f
            gh[:] = g
            if rep == 2:
                ks.set_pdl(True)  # a setting the capture baked in: captured afresh
            try:
                ks.ks_mul_host(hh, fh, gh, b, sg, v, e, stream)
            finally:
                ks.set_pdl(False)
            assert_same(hh.copy(), oracle.mul(f, g, b, sg),
                        "problem %d call %d, own stream %s" % (i, rep, own_stream))
