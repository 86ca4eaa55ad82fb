"""Runs one product shape a few times through the library (for profilers).

    python -m paper_0712_4046_gb300.run_case --variant 4 --len 16384 --bits 48 --signed --reps 3

Inputs are the seeded synthetic coefficients of ``ks_inputs``.  Prints the
plan the library ran.  No timing: use ``bench.py`` for numbers.
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--variant", type=int, default=4)
    ap.add_argument("--engine", type=int, default=0)
    ap.add_argument("--len", type=int, default=16384)
    ap.add_argument("--len-g", type=int, default=0)
    ap.add_argument("--bits", type=int, default=48)
    ap.add_argument("--signed", action="store_true")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=20071229)
    ap.add_argument("--square", action="store_true", help="g = f (the same buffer)")
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import numpy as np
    import torch

    import ks_inputs
    import paper_0712_4046_gb300 as ks

    lf, lg = args.len, args.len_g or args.len
    f = ks_inputs.random_poly(lf, args.bits, args.signed, args.seed)
    g = ks_inputs.random_poly(lg, args.bits, args.signed, args.seed + 1)
    tf = torch.from_numpy(f.view(np.int64)).cuda()
    tg = tf if args.square else torch.from_numpy(g.view(np.int64)).cuda()
    if args.square:
        lg = lf
    for _ in range(args.reps):
        h = ks.mul(tf, tg, args.bits, args.signed, args.variant, args.engine)
    ks.status_sync()
    print(ks.plan_info(lf, lg, args.bits, args.signed, args.variant, args.engine), tuple(h.shape))
    return 0


if __name__ == "__main__":
    sys.exit(main())
