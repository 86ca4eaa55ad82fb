"""Writes config5b_products.txt: the SHA-256 of each of the 64 exact products
in (Z/pZ)[x], p = 2^61 - 1, of the seeded length-2^16 residue pairs of
tests/test_gpu_configs.py (product i: ks_inputs.random_residues(2^16, p,
900 + 2 i) and seed 901 + 2 i), computed by the oracle's mod-p schoolbook
product alone, each over its 2^17 - 1 residues as little-endian 64-bit
words.  About five minutes on eight cores.

    python tests/golden/make_config5b_hash.py
"""
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import ks_inputs  # noqa: E402
import oracle  # noqa: E402

P, L, N = (1 << 61) - 1, 1 << 16, 64


def main():
    t0 = time.time()
    lines = []
    for i in range(N):
        f = ks_inputs.random_residues(L, P, 900 + 2 * i)
        g = ks_inputs.random_residues(L, P, 901 + 2 * i)
        h = oracle.mul_mod(f, g, P)
        lines.append("%d %s" % (i, hashlib.sha256(
            np.ascontiguousarray(h, dtype=np.uint64).tobytes()).hexdigest()))
    with open(os.path.join(HERE, "config5b_products.txt"), "w") as fh:
        fh.write("# SHA-256 of each exact product mod p = 2^61 - 1 of\n")
        fh.write("# ks_inputs.random_residues(2^16, p, 900 + 2 i) and (.., 901 + 2 i),\n")
        fh.write("# i = 0 .. 63: the oracle's mod-p schoolbook product (oracle.mul_mod),\n")
        fh.write("# 2^17 - 1 residues as little-endian 64-bit words; written by\n")
        fh.write("# make_config5b_hash.py in %.0f s on %d threads.\n"
                 % (time.time() - t0, oracle.default_threads()))
        fh.write("\n".join(lines) + "\n")
    print("%d products, %.0f s" % (N, time.time() - t0))


if __name__ == "__main__":
    main()
