"""Direct calls captured into a CUDA graph: after one call outside the
capture (which loads the transform's twiddle tables and creates the helper
stream), ks_mul_ex records into a caller's graph, and replays are exact
against the oracle for new inputs written into the same buffers."""
import numpy as np
import pytest

import oracle
from tests._gpu import assert_same, random_case, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    return ks


@pytest.mark.parametrize("variant,engine", [(1, "ENGINE_NTT"), (4, "ENGINE_NTT"),
                                            (4, "ENGINE_TC"), (3, "ENGINE_SCHOOLBOOK")])
def test_captured_ks_mul_ex_replays_exact(ks, variant, engine):
    import torch
    lf, lg, b, sg = 3000, 2800, 64, True
    eng = getattr(ks, engine)
    nbytes = ks.workspace_bytes(lf, lg, b, sg, variant, eng)
    ws = torch.empty(nbytes // 8 + 64, dtype=torch.int64, device="cuda")
    ol = ks.out_limbs(lf, lg, b, sg)
    df = torch.zeros((lf, 1), dtype=torch.int64, device="cuda")
    dg = torch.zeros((lg, 1), dtype=torch.int64, device="cuda")
    h = torch.zeros((lf + lg - 1, ol), dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):  # the call outside the capture
        ks.ks_mul_ex(h, df, dg, b, sg, variant, eng, ws, stream=s)
    s.synchronize()
    ks.status_sync()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        h.zero_()
        ks.ks_mul_ex(h, df, dg, b, sg, variant, eng, ws, stream=s)
    for rep in range(2):
        f, g = random_case(lf, lg, b, sg, 700 + 10 * variant + rep)
        df.copy_(to_dev(f))
        dg.copy_(to_dev(g))
        graph.replay()
        torch.cuda.synchronize()
        ks.status_sync()
        assert_same(to_host(h), oracle.mul(f, g, b, sg),
                    "replay %d, variant %d, %s" % (rep, variant, engine))
