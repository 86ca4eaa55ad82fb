"""Reads the paper's worked-example fixtures in ``tests/golden/`` (``key = value`` lines)."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, value = line.partition(" = ")
            parts = value.split()
            out[key.strip()] = int(parts[0]) if len(parts) == 1 else [int(p) for p in parts]
    return out
