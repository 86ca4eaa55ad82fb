"""Autotuning and learned dispatch (no counterpart in the paper, which picks the
variant by hand per experiment; its Sec. 4 notes that small degrees favour the
standard substitution and moderate ones the four-point variant).

* ``measure``: times every (variant, engine) configuration the library can run
  on a grid of problem shapes, with the library's own timer (``tune_time``).
* ``build_table``: the exhaustive autotuned table -- the measured best
  configuration per shape; KS_AUTO then takes the nearest shape.
* ``train``: the MLP cost model (features -> predicted log2 microseconds per
  configuration), trained on those timings by the library's CUDA kernels.
* ``regret``: mean of t(chosen) / t(best) - 1 over measured shapes, for any
  chooser (fixed KS1, the heuristic, the table, the model).
* ``save_state`` / ``load_state``: the table, the model and the raw timings
  in one versioned JSON file with a SHA-256 checksum, keyed by device name,
  SM count and library version; ``install`` hands them to the library.

    python -m paper_0712_4046_gb300.dispatch --tune --out state.json
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import sys
import time

import numpy as np

FORMAT = 1
DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
STATE_FILE = os.path.join(DATA_DIR, "dispatch_state.json")
ENGINE_INDEX = {1: 0, 2: 1, 3: 2}      # schoolbook, NTT, tensor cores
INDEX_ENGINE = {0: 1, 1: 2, 2: 3}
CONFIGS = [(v, e) for v in (1, 2, 3, 4) for e in (1, 2, 3)]


def output_index(variant: int, engine: int) -> int:
    return 3 * (variant - 1) + ENGINE_INDEX[engine]


BATCH_BITS_SAT = 26.0  # log2 of the batch operand bits beyond which the GPU is full


def features(lf, lg, b, signed, batch):
    """The library's features of a product in a batch of `batch` equal ones:
    lengths, size, sign and the batch's operand bits W = batch (lf + lg) b,
    log-scaled and saturating at 2^26."""
    w = math.log2(max(1.0, float(batch) * (lf + lg) * b))
    return [math.log2(lf) / 20.0, math.log2(lg) / 20.0, math.log2(b) / 11.0,
            1.0 if signed else 0.0, min(w, BATCH_BITS_SAT) / BATCH_BITS_SAT]


def saturating_batch(lf, lg, b, cap=4096):
    """The smallest power-of-two batch of equal products whose operand bits reach
    2^26 (the saturated regime), at most `cap`."""
    B = 1
    while B < cap and B * (lf + lg) * b < (1 << int(BATCH_BITS_SAT)):
        B *= 2
    return B


def default_grid():
    """Config-3 sweep (equal lengths x bits, unsigned and signed; b = 4 is the
    small-modulus regime of Sec. 4, where packing dominates), uneven lengths,
    and batch sizes for the batched executor."""
    shapes = []
    for L in (16, 64, 256, 1024, 4096, 16384, 65536, 262144):
        for b in (4, 8, 64, 256, 1024):
            for s in (0, 1):
                if L >= 65536 and b >= 256 and s:
                    continue
                shapes.append((L, L, b, s, 1))
    for lf, lg in ((8, 8192), (64, 4096), (300, 5000), (1000, 100), (4096, 512), (2048, 8192)):
        for b in (4, 16, 48, 128, 512):
            shapes.append((lf, lg, b, b % 2, 1))
    for L, b in ((64, 16), (256, 48), (1024, 64), (4096, 32), (512, 256)):
        for batch in (16, 256):
            shapes.append((L, L, b, 0, batch))
    # the large batches of the batched executor
    for L, b, s in ((64, 16, 0), (256, 48, 1), (1024, 64, 0), (512, 256, 1)):
        for batch in (1024, 4096):
            shapes.append((L, L, b, s, batch))
    # saturated batches over the uneven-batch range (lengths 8 .. 8192, bits
    # 4 .. 512): what a product costs inside a batch that fills the GPU
    pairs = [(L, L) for L in (8, 32, 128, 512, 2048, 8192)]
    pairs += [(8, 2048), (64, 8192), (512, 32), (2048, 128), (8192, 1024)]
    for lf, lg in pairs:
        for b in (4, 16, 64, 256, 512):
            for s in (0, 1):
                shapes.append((lf, lg, b, s, saturating_batch(lf, lg, b)))
    return shapes


def measure(shapes, max_ms=60.0, reps=5, log=None):
    """Times each (variant, engine) of each shape; unplannable or slow ones are skipped."""
    import paper_0712_4046_gb300 as ks
    data = []
    for (lf, lg, b, s, batch) in shapes:
        times = {}
        for v, e in CONFIGS:
            if e == 1 and batch > 1 and lf * lg * b * b > 4e10:
                continue
            try:
                first = ks.tune_time(lf, lg, b, bool(s), v, e, batch, 1)
                if first * batch > max_ms:
                    t = first
                else:
                    r = reps if first * batch * reps < 200 else 2
                    t = ks.tune_time(lf, lg, b, bool(s), v, e, batch, r)
            except ks.KSError:
                continue
            times[str(output_index(v, e))] = t * 1000.0  # microseconds per product
        if times:
            data.append({"lf": lf, "lg": lg, "b": b, "signed": s, "batch": batch,
                         "us": times})
            if log:
                best = min(times, key=times.get)
                print("shape %s best %s %.1f us" % ((lf, lg, b, s, batch), best, times[best]),
                      file=log, flush=True)
    return data


def xy(data):
    X = np.array([features(d["lf"], d["lg"], d["b"], d["signed"], d["batch"]) for d in data],
                 dtype=np.float32)
    T = np.zeros((len(data), 12), dtype=np.float32)
    M = np.zeros((len(data), 12), dtype=np.float32)
    for i, d in enumerate(data):
        for k, us in d["us"].items():
            T[i, int(k)] = math.log2(max(us, 1e-3))
            M[i, int(k)] = 1.0
    return X, T, M


def build_table(data):
    rows = []
    for d in data:
        if d["batch"] != 1:
            continue
        k = int(min(d["us"], key=d["us"].get))
        rows.append([d["lf"], d["lg"], d["b"], d["signed"], k // 3 + 1, INDEX_ENGINE[k % 3]])
    return rows


def init_params(seed=0):
    import paper_0712_4046_gb300 as ks
    rng = np.random.default_rng(seed)
    shapes = [(32, 5), (32,), (32, 32), (32,), (12, 32), (12,)]
    parts = []
    for s in shapes:
        if len(s) == 2:
            parts.append(rng.normal(0.0, math.sqrt(2.0 / s[1]), size=s).reshape(-1))
        else:
            parts.append(np.zeros(s))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == ks.mlp_param_count()
    return p


def train(data, steps=4000, lr=3e-3, seed=0):
    import paper_0712_4046_gb300 as ks
    X, T, M = xy(data)
    p0 = init_params(seed)
    # output biases start at the mean measured log-time of each configuration
    b3 = np.array([T[M[:, j] > 0, j].mean() if (M[:, j] > 0).any() else 0.0 for j in range(12)])
    p0[-12:] = b3.astype(np.float32)
    return ks.mlp_train(p0, X, T, M, steps, lr)


# ------------------------------------------------------------------ choosers
def choose_table(rows):
    def pick(d):
        best, bd = None, 1e300
        for r in rows:
            if r[3] != d["signed"]:
                continue
            dist = ((math.log2(r[0]) - math.log2(d["lf"])) ** 2
                    + (math.log2(r[1]) - math.log2(d["lg"])) ** 2
                    + 2.0 * (math.log2(r[2]) - math.log2(d["b"])) ** 2)
            if dist < bd:
                bd, best = dist, output_index(r[4], r[5])
        return best
    return pick


def choose_mlp(params):
    import paper_0712_4046_gb300 as ks

    def pick_all(data):
        ks.mlp_set_params(params)
        X, _, _ = xy(data)
        return ks.mlp_predict(X)
    return pick_all


def regret(data, chosen):
    """chosen[i]: output index picked for data[i], or a list of indices in order of
    preference (the first measured one counts).  Mean of t(chosen)/t(best) - 1."""
    r = []
    for d, c in zip(data, chosen):
        us = {int(k): v for k, v in d["us"].items()}
        best = min(us.values())
        prefs = c if isinstance(c, (list, tuple)) else [c]
        t = next((us[k] for k in prefs if k is not None and k in us), max(us.values()))
        r.append(t / best - 1.0)
    return float(np.mean(r)) if r else float("nan")


def mlp_choices(params, data):
    y = choose_mlp(params)(data)
    return [list(np.argsort(y[i])) for i in range(len(data))]


def library_choices(data, variant=0):
    """The library's own choice (heuristic when nothing is installed)."""
    import paper_0712_4046_gb300 as ks
    out = []
    for d in data:
        info = ks.plan_info(d["lf"], d["lg"], d["b"], bool(d["signed"]), variant, 0)
        out.append(output_index(info["variant"], info["engine"]))
    return out


def split(data, frac=0.75, seed=7):
    rng = np.random.default_rng(seed)
    idx = rng.permutation(len(data))
    k = int(len(data) * frac)
    return [data[i] for i in idx[:k]], [data[i] for i in idx[k:]]


# ------------------------------------------------------------------ persistence
def device_key():
    import torch

    import paper_0712_4046_gb300 as ks
    prop = torch.cuda.get_device_properties(torch.cuda.current_device())
    return {"device": prop.name, "sms": prop.multi_processor_count,
            "library": int(ks.lib.ks_version())}


def _checksum(body) -> str:
    return hashlib.sha256(json.dumps(body, sort_keys=True).encode()).hexdigest()


def save_state(path, key, rows, params, data, report):
    body = {"format": FORMAT, "key": key, "table": rows,
            "mlp": [float(x) for x in params], "timings": data, "report": report}
    with open(path, "w") as fh:
        json.dump({"body": body, "sha256": _checksum(body)}, fh)


def load_state(path=STATE_FILE):
    """The verified state, or None (missing file, wrong format or checksum)."""
    try:
        with open(path) as fh:
            doc = json.load(fh)
        body = doc["body"]
        if body.get("format") != FORMAT or _checksum(body) != doc.get("sha256"):
            return None
        return body
    except (OSError, ValueError, KeyError):
        return None


def install(path=STATE_FILE, require_match=True) -> bool:
    """Installs the table and model of a saved state into the library when the
    state was measured on this kind of device (else leaves the heuristic)."""
    import paper_0712_4046_gb300 as ks
    body = load_state(path)
    if body is None:
        return False
    if require_match:
        try:
            key = device_key()
        except Exception:
            return False
        if {k: body["key"].get(k) for k in ("device", "sms")} != \
                {k: key[k] for k in ("device", "sms")}:
            return False
    ks.dispatch_set_table(body["table"])
    ks.mlp_set_params(np.array(body["mlp"], dtype=np.float32))
    return True


def uninstall():
    import paper_0712_4046_gb300 as ks
    ks.dispatch_set_table([])
    ks.mlp_set_params(None)


def tune(out_path, shapes=None, steps=4000, log=sys.stderr):
    t0 = time.time()
    uninstall()
    data = measure(shapes or default_grid(), log=log)
    train_set, test_set = split(data)
    params, loss = train(train_set, steps=steps)
    rows_train = build_table(train_set)
    report = {
        "shapes": len(data), "train": len(train_set), "test": len(test_set),
        "train_loss": loss,
        "regret_test": {
            "fixed_ks1": regret(test_set, library_choices(test_set, variant=1)),
            "heuristic": regret(test_set, library_choices(test_set)),
            "table": regret(test_set, [choose_table(rows_train)(d) for d in test_set]),
            "mlp": regret(test_set, mlp_choices(params, test_set)),
        },
        "seconds": time.time() - t0,
    }
    # the installed model and table use every measured shape
    params_all, loss_all = train(data, steps=steps)
    report["final_loss"] = loss_all
    save_state(out_path, device_key(), build_table(data), params_all, data, report)
    print(json.dumps(report), file=log, flush=True)
    return report


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--tune", action="store_true")
    ap.add_argument("--out", default=STATE_FILE)
    ap.add_argument("--steps", type=int, default=4000)
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    if args.tune:
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        tune(args.out, steps=args.steps)
    return 0


if __name__ == "__main__":
    sys.exit(main())
