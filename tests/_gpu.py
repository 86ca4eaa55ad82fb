"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and
compare it with the CPU oracle (exact limb equality), or, at sizes the
oracle cannot finish quickly, with sampled exact coefficients and modular
fingerprints h(r) = f(r) g(r) mod q."""
from __future__ import annotations

import numpy as np

import ks_inputs as gen
import oracle


def to_dev(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def to_host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def gpu_mul(ks, f: np.ndarray, g: np.ndarray, b: int, signed: bool, variant: int,
            engine: int = 0) -> np.ndarray:
    h = ks.mul(to_dev(f), to_dev(g), b, signed, variant, engine)
    ks.status_sync()
    return to_host(h)


def assert_same(got: np.ndarray, want: np.ndarray, what: str = "") -> None:
    assert got.shape == want.shape, (what, got.shape, want.shape)
    if not np.array_equal(got, want):
        bad = np.nonzero((got != want).any(axis=1))[0]
        k = int(bad[0])
        raise AssertionError("%s: %d of %d coefficients differ, first k=%d got=%s want=%s"
                             % (what, bad.size, got.shape[0], k, got[k].tolist(),
                                want[k].tolist()))


def residues(limbs: np.ndarray, signed: bool, q: int) -> np.ndarray:
    """Each multi-limb coefficient modulo a prime q < 2^31, as int64."""
    limbs = np.asarray(limbs, dtype=np.uint64)
    nl = limbs.shape[1]
    acc = np.zeros(limbs.shape[0], dtype=np.uint64)
    qq = np.uint64(q)
    for l in range(nl):
        w = np.uint64(pow(2, 64 * l, q))
        acc = (acc + (limbs[:, l] % qq) * w) % qq
    if signed:
        neg = (limbs[:, nl - 1] >> np.uint64(63)) == 1
        corr = np.uint64(pow(2, 64 * nl, q))
        acc = np.where(neg, (acc + qq - corr) % qq, acc)
    return acc.astype(np.int64)


def eval_mod(coeff_res: np.ndarray, r: int, q: int) -> int:
    """sum_k c_k r^k mod q for residues c_k (vectorized by blocks of powers)."""
    n = coeff_res.size
    B = 1024
    small = np.empty(B, dtype=np.uint64)
    p = 1
    for i in range(B):
        small[i] = p
        p = p * r % q
    rb = pow(r, B, q)
    total, scale = 0, 1
    qq = np.uint64(q)
    for s in range(0, n, B):
        blk = coeff_res[s:s + B].astype(np.uint64)
        part = int(((blk * small[:blk.size]) % qq).sum() % qq)
        total = (total + part * scale) % q
        scale = scale * rb % q
    return total


def fingerprint_check(h: np.ndarray, f: np.ndarray, g: np.ndarray, signed: bool, seed: int,
                      nchecks: int = 3) -> None:
    """h(r) = f(r) g(r) mod q at random r for a few primes q < 2^31."""
    rng = np.random.default_rng(seed)
    for q in (2147483629, 2147483587, 1000000007)[:nchecks]:
        r = int(rng.integers(2, q - 1))
        hv = eval_mod(residues(h, signed, q), r, q)
        fv = eval_mod(residues(f, signed, q), r, q)
        gv = eval_mod(residues(g, signed, q), r, q)
        assert hv == fv * gv % q, ("fingerprint mismatch", q, r)


def sampled_check(h: np.ndarray, f: np.ndarray, g: np.ndarray, b: int, signed: bool,
                  nsamples: int, seed: int) -> None:
    """Exact oracle values at the ends, the middle and random k."""
    lh = h.shape[0]
    rng = np.random.default_rng(seed)
    ks_ = {0, 1, lh - 1, lh - 2, lh // 2, f.shape[0] - 1, g.shape[0] - 1}
    ks_ |= set(int(x) for x in rng.integers(0, lh, size=nsamples))
    ks_ = np.array(sorted(k for k in ks_ if 0 <= k < lh), dtype=np.int64)
    want = oracle.coeffs(ks_, f, g, b, signed, n_limbs_out=h.shape[1])
    assert_same(h[ks_], want, "sampled coefficients")


def random_case(lf: int, lg: int, b: int, signed: bool, seed: int):
    return gen.random_poly(lf, b, signed, seed), gen.random_poly(lg, b, signed, seed + 7777)
