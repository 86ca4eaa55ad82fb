"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Sizes run from single coefficients to several engine and normalization tiles
with ragged tails; all four variants (Sec. 3.1-3.4), unsigned and signed,
equal and unequal lengths, odd and even Lh, and the degenerate cases (L = 1,
zero polynomials, f aliasing g, extreme coefficients meeting the bound of
Sec. 3 with equality)."""
import numpy as np
import pytest

import ks_inputs as gen
import oracle
from tests._gpu import assert_same, gpu_mul, random_case, to_dev, to_host

pytestmark = pytest.mark.gpu

VARIANTS = [1, 2, 3, 4]
ENGINES = [1, 2, 3]  # INT32 schoolbook, NTT, tensor cores


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    return ks


SHAPES = [(1, 1), (1, 5), (5, 1), (2, 2), (3, 4), (7, 7), (16, 15), (33, 64), (100, 101),
          (257, 300), (1000, 999), (2048, 1500)]


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("signed", [False, True])
@pytest.mark.parametrize("b", [1, 2, 7, 31, 48, 63, 64, 65, 100, 128])
def test_random_shapes(ks, engine, variant, signed, b):
    for i, (lf, lg) in enumerate(SHAPES):
        if b >= 100 and lf * lg > 300000:
            continue
        f, g = random_case(lf, lg, b, signed, 1000 * b + 10 * i + variant)
        want = oracle.mul(f, g, b, signed)
        got = gpu_mul(ks, f, g, b, signed, variant, engine)
        assert_same(got, want, "engine %d variant %d b=%d signed=%d shape=%s"
                    % (engine, variant, b, signed, (lf, lg)))


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("b", [200, 256, 511, 1024])
def test_wide_coefficients(ks, engine, variant, b):
    for signed in (False, True):
        for lf, lg in [(1, 1), (9, 4), (40, 41)]:
            f, g = random_case(lf, lg, b, signed, b + lf + 3 * variant + signed)
            want = oracle.mul(f, g, b, signed)
            got = gpu_mul(ks, f, g, b, signed, variant, engine)
            assert_same(got, want, "engine %d variant %d b=%d signed=%d"
                        % (engine, variant, b, signed))


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("variant", VARIANTS)
def test_extremes(ks, engine, variant):
    """All-maximal digits drive every exact accumulation to its bound (for the
    tensor cores: fp32 partial sums of 16,516,096 < 2^24 per chunk)."""
    for b in (1, 8, 48, 64, 65):
        for lf, lg in [(1, 1), (4, 4), (8, 9), (64, 64), (513, 200), (1500, 1500)]:
            m = (1 << b) - 1
            f, g = gen.const_poly(lf, b, m), gen.const_poly(lg, b, m)
            assert_same(gpu_mul(ks, f, g, b, False, variant, engine), oracle.mul(f, g, b, False),
                        "all-max b=%d engine %d" % (b, engine))
            lo, hi = -(1 << (b - 1)), (1 << (b - 1)) - 1
            for a, c in [(lo, lo), (lo, hi), (hi, hi)]:
                f, g = gen.const_poly(lf, b, a), gen.const_poly(lg, b, c)
                assert_same(gpu_mul(ks, f, g, b, True, variant, engine),
                            oracle.mul(f, g, b, True), "signed extremes b=%d engine %d"
                            % (b, engine))


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("variant", VARIANTS)
def test_zero_and_aliasing(ks, engine, variant):
    b = 40
    z = np.zeros((50, 1), dtype=np.uint64)
    f, _ = random_case(50, 1, b, True, 5)
    for signed in (False, True):
        assert_same(gpu_mul(ks, z, f, b, signed, variant, engine), oracle.mul(z, f, b, signed),
                    "zero")
    # f aliasing g: the same device buffer on both sides
    tf = to_dev(f)
    h = ks.mul(tf, tf, b, True, variant)
    ks.status_sync()
    assert_same(to_host(h), oracle.mul(f, f, b, True), "square")


def test_explicit_workspace_and_errors(ks):
    import torch
    f, g = random_case(300, 200, 33, False, 9)
    want = oracle.mul(f, g, 33, False)
    for v in VARIANTS:
        n = ks.workspace_bytes(300, 200, 33, False, v, ks.ENGINE_SCHOOLBOOK)
        ws = torch.empty(n // 8 + 1, dtype=torch.int64, device="cuda")
        h = torch.empty((499, ks.out_limbs(300, 200, 33, False)), dtype=torch.int64,
                        device="cuda")
        ks.ks_mul_ex(h, to_dev(f), to_dev(g), 33, False, v, ks.ENGINE_SCHOOLBOOK, ws)
        ks.status_sync()
        assert_same(to_host(h), want, "ks_mul_ex variant %d" % v)
        # too small a workspace is refused
        small = torch.empty(8, dtype=torch.int64, device="cuda")
        with pytest.raises(ks.KSError) as ei:
            ks.ks_mul_ex(h, to_dev(f), to_dev(g), 33, False, v, ks.ENGINE_SCHOOLBOOK, small)
        assert ei.value.status == ks.KS_EINVAL
    # h overlapping f is refused
    tf = to_dev(np.zeros((600, 1), dtype=np.uint64))
    with pytest.raises(ks.KSError):
        ks.ks_mul(tf[:499], tf[100:400], tf[100:300], 8, False, 1)
    with pytest.raises(ks.KSError):
        ks.ks_mul(tf[:10], tf[100:105], tf[200:206], 8, False, 9)


def test_host_buffers(ks):
    for v in VARIANTS:
        f, g = random_case(700, 650, 61, True, 77 + v)
        want = oracle.mul(f, g, 61, True)
        h = np.zeros_like(want)
        ks.ks_mul_host(h, f, g, 61, True, v, ks.ENGINE_SCHOOLBOOK)
        assert_same(h, want, "host variant %d" % v)


@pytest.mark.parametrize("p", [2 ** 61 - 1, 1000003, 7, 2 ** 62 + 135])
def test_mul_mod(ks, p):
    import torch
    for v in VARIANTS:
        f = gen.random_residues(900, p, 11 + v)
        g = gen.random_residues(1100, p, 12 + v)
        h = torch.empty((1999, 1), dtype=torch.int64, device="cuda")
        ks.ks_mul_mod(h, to_dev(f), to_dev(g), p, v)
        ks.status_sync()
        assert_same(to_host(h), oracle.mul_mod(f, g, p), "mod %d variant %d" % (p, v))


def test_batch(ks):
    import torch
    lf, lg, cb, sg = gen.uneven_batch(24, 4242, 8, 700, 4, 130)
    probs, wants = [], []
    for i in range(24):
        f, g = random_case(int(lf[i]), int(lg[i]), int(cb[i]), bool(sg[i]), 300 + i)
        ol = ks.out_limbs(int(lf[i]), int(lg[i]), int(cb[i]), bool(sg[i]))
        h = torch.empty((int(lf[i] + lg[i] - 1), ol), dtype=torch.int64, device="cuda")
        probs.append(dict(h=h, f=to_dev(f), g=to_dev(g), coeff_bits=int(cb[i]),
                          is_signed=bool(sg[i]), variant=(i % 5), engine=0))
        wants.append(oracle.mul(f, g, int(cb[i]), bool(sg[i])))
    ks.ks_mul_batch(probs)
    ks.status_sync()
    for i, (q, w) in enumerate(zip(probs, wants)):
        assert_same(to_host(q["h"]), w, "batch item %d" % i)
