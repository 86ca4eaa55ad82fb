"""Writes config5a_product.txt: the SHA-256 of the exact product of the
2^20 x 2^20 unsigned 256-bit workload (the seeded inputs of
tests/test_gpu_configs.py: ks_inputs.random_poly(2^20, 256, False, 55) and
seed 55 + 7777), computed by the oracle's schoolbook product alone, over its
2^21 - 1 coefficients of out_limbs little-endian 64-bit limbs each, in
order.  About 1.8e13 limb products: one to two hours on eight cores.

    python tests/golden/make_config5a_hash.py
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

L, B, SEED = 1 << 20, 256, 55


def main():
    f = ks_inputs.random_poly(L, B, False, SEED)
    g = ks_inputs.random_poly(L, B, False, SEED + 7777)
    t0 = time.time()
    h = oracle.mul(f, g, B, False)
    secs = time.time() - t0
    digest = hashlib.sha256(np.ascontiguousarray(h, dtype=np.uint64).tobytes()).hexdigest()
    with open(os.path.join(HERE, "config5a_product.txt"), "w") as fh:
        fh.write("# SHA-256 of the exact product of ks_inputs.random_poly(2^20, 256, False, 55)\n")
        fh.write("# and ks_inputs.random_poly(2^20, 256, False, 55 + 7777): the oracle's\n")
        fh.write("# schoolbook product (oracle.mul), %d coefficients of %d 64-bit limbs,\n"
                 % h.shape)
        fh.write("# little-endian, in order; written by make_config5a_hash.py in %.0f s\n" % secs)
        fh.write("# on %d threads.\n" % oracle.default_threads())
        fh.write("shape = %d %d\n" % h.shape)
        fh.write("sha256 = %s\n" % digest)
    print(digest, h.shape, "%.0f s" % secs)


if __name__ == "__main__":
    main()
