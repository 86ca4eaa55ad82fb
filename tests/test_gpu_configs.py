"""The five workload configurations at full size, through the C ABI.

Where the CPU oracle finishes in seconds (the 4096-product batch included) the
comparison is exact and complete.  The long sweep points are checked by
modular fingerprints h(r) = f(r) g(r) mod q at random points, and sampled
coefficients are compared exactly with the oracle's dot products.  The
2^20 x 256-bit product and the 64 products mod 2^61 - 1 are compared in full
with the oracle's complete products, run once offline: their SHA-256 digests
are in tests/golden/ (written by the make_config5*_hash.py scripts there)."""
import hashlib
import os

import numpy as np
import pytest

import ks_inputs as gen
import oracle
from tests._gpu import (assert_same, fingerprint_check, gpu_mul, random_case, sampled_check,
                        to_dev, to_host)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    return ks


def test_config1_1024_u64(ks):
    f, g = random_case(1024, 1024, 64, False, 101)
    want = oracle.mul(f, g, 64, False)
    assert want.shape == (2047, 3)  # up to 138 bits
    for engine in (0, 2, 3):
        for variant in (1, 2, 3, 4):
            assert_same(gpu_mul(ks, f, g, 64, False, variant, engine), want,
                        "config 1 variant %d engine %d" % (variant, engine))


@pytest.fixture(scope="module")
def config2():
    f = gen.random_poly(16384, 48, True, 20071229)
    g = gen.random_poly(16384, 48, True, 20071230)
    return f, g, oracle.mul(f, g, 48, True)


@pytest.mark.parametrize("engine", [0, 2, 3])
def test_config2_16384_s48(ks, config2, engine):
    f, g, want = config2
    for variant in (1, 2, 3, 4):
        assert_same(gpu_mul(ks, f, g, 48, True, variant, engine), want,
                    "config 2 variant %d engine %d" % (variant, engine))


SWEEP_L = [16, 64, 256, 1024, 4096, 16384]
SWEEP_B = [8, 64, 256, 1024]


@pytest.mark.parametrize("b", SWEEP_B)
def test_config3_sweep(ks, b):
    for L in SWEEP_L:
        for signed in (False, True):
            f, g = random_case(L, L, b, signed, 7 * L + b + signed)
            nl = (b + 63) // 64
            exact = L * L * nl * nl <= 4e8
            want = oracle.mul(f, g, b, signed) if exact else None
            for variant in (1, 2, 3, 4):
                got = gpu_mul(ks, f, g, b, signed, variant)
                if exact:
                    assert_same(got, want, "sweep L=%d b=%d variant %d" % (L, b, variant))
                else:
                    fingerprint_check(got, f, g, signed, L + variant, nchecks=2)
                    sampled_check(got, f, g, b, signed, 6, L * variant)


@pytest.mark.parametrize("L,b", [(65536, 8), (65536, 64), (262144, 8), (262144, 64)])
def test_config3_long(ks, L, b):
    f, g = random_case(L, L, b, False, L + b)
    for variant in (1, 4):
        got = gpu_mul(ks, f, g, b, False, variant)
        fingerprint_check(got, f, g, False, variant, nchecks=2)
        sampled_check(got, f, g, b, False, 8, variant)


def test_config4_uneven_batch(ks):
    import torch
    lf, lg, cb, sg = gen.uneven_batch(4096, 20071231)
    probs, inputs = [], []
    for i in range(4096):
        f, g = random_case(int(lf[i]), int(lg[i]), int(cb[i]), bool(sg[i]), 5000 + i)
        ol = ks.out_limbs(int(lf[i]), int(lg[i]), int(cb[i]), bool(sg[i]))
        h = torch.empty((int(lf[i] + lg[i] - 1), ol), dtype=torch.int64, device="cuda")
        probs.append(dict(h=h, f=to_dev(f), g=to_dev(g), coeff_bits=int(cb[i]),
                          is_signed=bool(sg[i])))
        inputs.append((f, g))
    ks.ks_mul_batch(probs)
    ks.status_sync()
    # every product exact (the oracle's 4096 products take about half a minute)
    for i, (q, (f, g)) in enumerate(zip(probs, inputs)):
        assert_same(to_host(q["h"]), oracle.mul(f, g, q["coeff_bits"], q["is_signed"]),
                    "batch %d" % i)


def _golden_5a():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "config5a_product.txt")
    kv = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    return tuple(int(x) for x in kv["shape"].split()), kv["sha256"]


def test_config5a_2pow20_u256(ks):
    L, b = 1 << 20, 256
    f, g = random_case(L, L, b, False, 55)
    shape, digest = _golden_5a()
    for variant in (1, 4):
        got = gpu_mul(ks, f, g, b, False, variant)
        # every coefficient, against the oracle's full product
        assert got.shape == shape
        assert hashlib.sha256(np.ascontiguousarray(got).tobytes()).hexdigest() == digest, variant
        fingerprint_check(got, f, g, False, variant, nchecks=2)
        sampled_check(got, f, g, b, False, 12, variant)


def _golden_5b():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "config5b_products.txt")
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            i, digest = line.split()
            out[int(i)] = digest
    return out


def test_config5b_64_products_mod_mersenne61(ks):
    import torch
    p = (1 << 61) - 1
    L = 1 << 16
    rng = np.random.default_rng(61)
    digests = _golden_5b()
    assert sorted(digests) == list(range(64))
    for i in range(64):
        f = gen.random_residues(L, p, 900 + 2 * i)
        g = gen.random_residues(L, p, 901 + 2 * i)
        h = torch.empty((2 * L - 1, 1), dtype=torch.int64, device="cuda")
        ks.ks_mul_mod(h, to_dev(f), to_dev(g), p, 4 if i % 2 else 1)
        hh = to_host(h)
        # every residue, against the oracle's full product
        assert hashlib.sha256(np.ascontiguousarray(hh).tobytes()).hexdigest() == digests[i], i
        got = [int(x) for x in hh.reshape(-1)]
        fi = [int(x) for x in f.reshape(-1)]
        gi = [int(x) for x in g.reshape(-1)]
        assert all(0 <= x < p for x in got)
        if i < 4:
            r = int(rng.integers(2, p - 1))
            hv = 0
            for c in reversed(got):
                hv = (hv * r + c) % p
            fv = gv = 0
            for c in reversed(fi):
                fv = (fv * r + c) % p
            for c in reversed(gi):
                gv = (gv * r + c) % p
            assert hv == fv * gv % p
            for k in [0, 1, L - 1, L, 2 * L - 2] + [int(x) for x in rng.integers(0, 2 * L - 1, 4)]:
                lo, hi = max(0, k - L + 1), min(k, L - 1)
                want = sum(fi[t] * gi[k - t] for t in range(lo, hi + 1)) % p
                assert got[k] == want, (i, k)
    ks.status_sync()


@pytest.mark.parametrize("variant,L,b,signed,engine", [
    (3, 300000, 8, False, 2),   # chains of 256: one CTA per seed, 64-bit coefficients
    (4, 300000, 20, True, 2),   # chains of 128 in both runs of Sec. 3.4
    (4, 524288, 48, False, 3),  # tensor-core products, chains of 128
    (3, 524288, 100, True, 2),  # multi-word seeds, chains of 256
])
def test_long_reconstruction_chains(ks, variant, L, b, signed, engine):
    # runs of more than 2^18 coefficients take longer chains, whose seeds no
    # longer fit the blocked seed kernel's window
    f, g = random_case(L, L, b, signed, L + 3 * b + variant)
    got = gpu_mul(ks, f, g, b, signed, variant, engine)
    fingerprint_check(got, f, g, signed, variant + b, nchecks=2)
    sampled_check(got, f, g, b, signed, 8, L + variant)
