#!/usr/bin/env python3
"""Benchmark: Z[x] products/s and output Gbit/s, KS4 vs KS1, bit-exact, one GB300.

Workload (the single-GPU configuration the metric is quoted on): one signed
product, len_f = len_g = 16384, coefficients uniform in [-2^47, 2^47) from a
fixed seed; all four variants (Sec. 3.1-3.4) run on the same inputs.  A step
is one whole product (pack, sub-products, normalize/combine, unpack or
reconstruction, signed correction) with inputs resident on the device; the
headline `value` is KS4's products/s, the other variants are reported beside
it under `variants`.

Each variant is timed twice: through a one-product plan (ks_plan_create)
captured once and replayed as a CUDA graph per step -- the headline -- and
through one ks_mul call per step (`ks_mul_*` keys).  Timing: W warm-up steps,
then K steps, each bracketed by CUDA events on the library's stream; between
steps a 256 MiB buffer is written to flush the 129 MB L2 (outside the
events).  A separate short pass with the library's per-phase CUDA events
gives the phase times and the dominant kernel's duration for the roofline.
`e2e` times the host-buffer entry point (ks_mul_host: H2D copy, product, D2H
copy) with pinned buffers.

`--impl reference` times the CPU oracle (plain schoolbook, all host cores) on
the same workload instead.  `--case V,L,B,SIGNED[,ENGINE[,REPS]]` runs one
product shape REPS times through ks_mul and prints its plan (no timing; a
fixed launch sequence for profilers).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import ks_inputs  # noqa: E402

WORKLOAD = {"workload": "zx_product_16384_s48", "len_f": 16384, "len_g": 16384,
            "coeff_bits": 48, "is_signed": True, "seed_f": 20071229, "seed_g": 20071230}
METRIC = "Z[x] products/s and output Gbit/s, KS4 vs KS1, bit-exact, 1 GB300"
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one tc_kernel
# launch on this workload's KS4 product, from an ncu capture of the current
# kernel (the tc_kernel summary under profiles/: 5.22 MB read, no DRAM
# writes); set to None whenever the kernel changes until it is captured again
TC_KERNEL_DRAM_BYTES = 5.22e6
TC_KERNEL_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch "
                            "(the tc_kernel capture of this workload under profiles/)")
# 32-bit IMAD issue rate per SM per clock (the INT32 multiply-add pipe), x2 ops per MAC
IMAD_PER_SM_CLK = 64
SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--case", default=None,
                    help="V,L,B,SIGNED[,ENGINE[,REPS]]: run one product shape, no timing")
    return ap.parse_args()


def run_case(spec: str) -> int:
    """One product shape REPS times through ks_mul (a fixed launch sequence for
    profilers); prints the plan the library ran."""
    import torch
    import paper_0712_4046_gb300 as ks
    parts = [int(x) for x in spec.split(",")]
    v, L, b, sg = parts[:4]
    engine = parts[4] if len(parts) > 4 else 0
    reps = parts[5] if len(parts) > 5 else 3
    f = ks_inputs.random_poly(L, b, bool(sg), WORKLOAD["seed_f"])
    g = ks_inputs.random_poly(L, b, bool(sg), WORKLOAD["seed_g"])
    tf = torch.from_numpy(f.view(np.int64)).cuda()
    tg = torch.from_numpy(g.view(np.int64)).cuda()
    for _ in range(reps):
        ks.mul(tf, tg, b, bool(sg), v, engine)
    torch.cuda.synchronize()
    ks.status_sync()
    print(json.dumps(ks.plan_info(L, L, b, bool(sg), v, engine)))
    return 0


def output_bits(lf, lg, b):
    e = (min(lf, lg) - 1).bit_length()
    return (lf + lg - 1) * (2 * b + e)


def inputs():
    w = WORKLOAD
    f = ks_inputs.random_poly(w["len_f"], w["coeff_bits"], w["is_signed"], w["seed_f"])
    g = ks_inputs.random_poly(w["len_g"], w["coeff_bits"], w["is_signed"], w["seed_g"])
    return f, g


BF16_TFLOPS = 1900.0
PEAK_KIND = "fallback"


def peaks():
    """HBM GB/s, max SM MHz, and the kind of figure (measured or fallback)."""
    global BF16_TFLOPS, PEAK_KIND
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        BF16_TFLOPS = float(p["bf16_tflops"])
        PEAK_KIND = "measured"
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        BF16_TFLOPS, PEAK_KIND = 1900.0, "fallback"
        return 6800.0, 2070.0, "fallback"


class Clocks:
    """nvidia-smi sampling (200 ms) while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples go to a scratch file (set KS_CLOCKS_DIR to keep them);
        # the JSON line carries their summary
        self.path = os.path.join(os.environ.get("KS_CLOCKS_DIR") or tempfile.gettempdir(),
                                 "ks_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                          "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        # wait (up to 5 s) for the first sample, so the timed work is covered
        t_end = time.time() + 5.0
        while self.proc is not None and time.time() < t_end:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                pass
            time.sleep(0.05)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup(backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
    return world, rank, local


def barrier_max(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle arm
def run_oracle(f, g, steps: int, warmup: int, budget_s: float):
    import oracle
    w = WORKLOAD
    cores = os.cpu_count() or 1
    for _ in range(max(0, min(warmup, 1))):
        oracle.mul(f, g, w["coeff_bits"], w["is_signed"], threads=cores)
    times = []
    t_end = time.perf_counter() + budget_s
    for i in range(steps):
        t0 = time.perf_counter()
        oracle.mul(f, g, w["coeff_bits"], w["is_signed"], threads=cores)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end and i + 1 >= 1:
            break
    return times, cores


def reference_main(args):
    world, rank, _ = dist_setup("gloo")
    if rank != 0:
        return 0
    f, g = inputs()
    w = WORKLOAD
    times, cores = run_oracle(f, g, args.steps, args.warmup, budget_s=240.0)
    ms = 1000.0 * statistics.mean(times)
    value = 1000.0 / ms
    obits = output_bits(w["len_f"], w["len_g"], w["coeff_bits"])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "products/s",
        "n_gpus": args.gpus, "steps": len(times), "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded splitmix64)",
        "config": dict(WORKLOAD, variant="schoolbook oracle", l2="n/a (host)"),
        "output_gbit_per_s": value * obits / 1e9,
        "cpu_baseline": {"value": value, "unit": "products/s", "cores": cores, "kind": "oracle",
                         "sample": "%d full products of the workload" % len(times)},
        "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
def main_ours(args):
    import torch
    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_0712_4046_gb300 as ks

    w = WORKLOAD
    f, g = inputs()
    lf, lg, b, sg = w["len_f"], w["len_g"], w["coeff_bits"], w["is_signed"]
    tf = torch.from_numpy(f.view(np.int64)).to(dev)
    tg = torch.from_numpy(g.view(np.int64)).to(dev)
    ol = ks.out_limbs(lf, lg, b, sg)
    lh = lf + lg - 1
    h = torch.empty((lh, ol), dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    # a dedicated stream (graph capture cannot use the legacy default stream); torch's
    # own work (the L2 flush) is issued on it too
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    obits = output_bits(lf, lg, b)
    hbm_gbs, sm_max_mhz, peak_kind = peaks()

    results = {}
    outputs = {}  # each variant's product, checked against the oracle in the CPU leg
    # (label, variant, engine): the library's choice for every variant, KS1 on the
    # tensor cores (the same engine as KS4's), and the INT32-pipe schoolbook engine
    # for KS1 and KS4 (the plain GPU baseline)
    runs = [("KS1", 1, 0), ("KS1_tc", 1, ks.ENGINE_TC), ("KS2", 2, 0), ("KS3", 3, 0),
            ("KS4", 4, 0), ("KS1_int32", 1, ks.ENGINE_SCHOOLBOOK),
            ("KS4_int32", 4, ks.ENGINE_SCHOOLBOOK)]
    ws = {}

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        ks.status_sync(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            evs[i][0].record(stream)
            fn()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        ks.status_sync(stream)
        return barrier_max(sum(a.elapsed_time(z) for a, z in evs), world, dev)

    with Clocks(local) as clk:
        for label, variant, engine in runs:
            if engine:
                n = ks.workspace_bytes(lf, lg, b, sg, variant, engine)
                ws[label] = torch.empty(n // 8 + 32, dtype=torch.int64, device=dev)

            def step():
                if engine:
                    ks.ks_mul_ex(h, tf, tg, b, sg, variant, engine, ws[label], stream)
                else:
                    ks.ks_mul(h, tf, tg, b, sg, variant, stream)
            # (1) one call per product, as timed (no profiling events)
            launches0 = ks.launch_count()
            total_ms = timed(step, args.steps)
            launches = (ks.launch_count() - launches0) // (args.steps + args.warmup)
            # (2) the same product through a one-product plan replayed as a CUDA graph
            h.zero_()
            plan = ks.Plan([dict(h=h, f=tf, g=tg, coeff_bits=b, is_signed=sg, variant=variant,
                                 engine=engine)])
            plan.capture(stream)
            graph_ms = timed(lambda: plan.execute(stream), args.steps)
            plan.status()
            graph_launches = plan.launches()
            plan.close()
            outputs[label] = h.cpu().numpy().view(np.uint64).copy()
            # (3) a short profiled pass for the per-phase times (events between phases)
            ks.profile_collect()
            ks.profile_enable(True)
            for _ in range(min(args.steps, 5)):
                flush.zero_()
                step()
            torch.cuda.synchronize()
            ks.profile_enable(False)
            phases = ks.profile_collect()
            results[label] = {"ms_per_step": total_ms / args.steps,
                              "graph_ms_per_step": graph_ms / args.steps,
                              "launches": launches, "graph_launches": graph_launches,
                              "phases": phases, "variant": variant, "engine": engine}
        # ---- KS1-KS4 across the moderate-size regime (Sec. 4's experiment)
        curve, curve_out = run_curve(ks, dev, stream, flush, args.steps, args.warmup, world)
        # ---- 64 products in (Z/pZ)[x], p = 2^61 - 1, L = 2^16 (the Sec. 4 application)
        modp, modp_out = run_modp(ks, dev, stream, flush, args.warmup, world)
        # ---- batched workload: 4096 uneven products, one plan per dispatch mode
        batched = run_batched(ks, dev, stream, flush, args.steps, args.warmup, world)
        # ---- HBM-bound phases (pack, normalize, unpack) where the arrays exceed L2
        hbm_phases = run_hbm_phases(ks, dev, stream, flush, hbm_gbs, peak_kind)
        # ---- the polynomial-ring variants of Sec. 2 on one (Z/pZ)[x, y] product
        bivariate = run_bivariate(ks, dev, stream, flush, args.steps, args.warmup)
    clocks = clk.summary()

    # ---- e2e through the host-buffer entry point (pinned buffers)
    fh = torch.from_numpy(f.view(np.int64)).pin_memory().numpy().view(np.uint64)
    gh = torch.from_numpy(g.view(np.int64)).pin_memory().numpy().view(np.uint64)
    hh = torch.empty((lh, ol), dtype=torch.int64).pin_memory().numpy().view(np.uint64)
    for _ in range(args.warmup):
        ks.ks_mul_host(hh, fh, gh, b, sg, 4, 0, stream)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ks.ks_mul_host(hh, fh, gh, b, sg, 4, 0, stream)
    e2e_s = barrier_max(time.perf_counter() - t0, world, dev)
    outputs["KS4_host"] = hh.copy()

    # ---- roofline of the dominant kernel of KS4: the tensor-core product
    # (the largest share of the serialised ncu launch list; the seeds run
    # concurrently on a helper stream, so their event spans overlap others)
    r4 = results["KS4"]
    info = ks.plan_info(lf, lg, b, sg, 4, ks.ENGINE_AUTO)
    ph = {k: v for k, v in r4["phases"].items() if v[1] > 0}
    dom = "product"
    dom_ms = ph[dom][0] / ph[dom][1]
    roof = roofline_for(dom, dom_ms, info, lf, lg, b, sg, hbm_gbs, sm_max_mhz, peak_kind)
    if info["engine"] == ks.ENGINE_TC:
        roof["traffic"] = TC_KERNEL_DRAM_BYTES
        roof["traffic_source"] = (TC_KERNEL_TRAFFIC_SOURCE if TC_KERNEL_DRAM_BYTES
                                  else "not captured for this kernel")
        roof["kernel"] = "tc_kernel"

    cpu, exact = None, None
    if rank == 0 and world == 1:
        cpu, exact = cpu_leg(f, g, outputs, curve_out, modp_out)

    if rank != 0:
        return 0
    # headline: KS4 through the plan API replayed as a CUDA graph, one product per step
    ms4 = r4["graph_ms_per_step"]
    value = world * 1000.0 / ms4
    variants = {}
    for v, r in results.items():
        pps = world * 1000.0 / r["graph_ms_per_step"]
        variants[v] = {"products_per_s": pps, "ms_per_step": r["graph_ms_per_step"],
                       "ks_mul_products_per_s": world * 1000.0 / r["ms_per_step"],
                       "ks_mul_ms_per_step": r["ms_per_step"],
                       "launches": r["graph_launches"],
                       "engine": ks.plan_info(lf, lg, b, sg, r["variant"],
                                              r["engine"])["engine"],
                       "output_gbit_per_s": pps * obits / 1e9,
                       "phases_ms": {k: round(x[0] / max(1, x[1]), 5)
                                     for k, x in r["phases"].items() if x[1] > 0}}
    best_ks1 = min(results[k]["graph_ms_per_step"] for k in ("KS1", "KS1_tc", "KS1_int32"))
    line = {
        "metric": METRIC, "value": value, "unit": "products/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms4,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded splitmix64)",
        "config": dict(WORKLOAD, variant="KS4", engine=info["engine"],
                       api="ks_plan (one product) replayed as a CUDA graph per step",
                       l2="flushed between steps (256 MiB write)",
                       parallelism="replicas" if world > 1 else "single"),
        "output_gbit_per_s": value * obits / 1e9,
        "bit_exact": exact,
        "ks4_over_ks1": best_ks1 / ms4,
        "ks4_over_ks1_same_engine": results["KS1_tc"]["graph_ms_per_step"] / ms4,
        "ks4_over_int32_ks1": results["KS1_int32"]["graph_ms_per_step"] / ms4,
        "ks_mul_products_per_s": world * 1000.0 / r4["ms_per_step"],
        "variants": variants,
        "gpu_launches": int(r4["graph_launches"]),
        "roofline": roof,
        "clocks": clocks,
        "e2e": {"value": world * args.steps / e2e_s, "unit": "products/s",
                "h2d_bytes_per_step": int(f.nbytes + g.nbytes),
                "d2h_bytes_per_step": int(lh * ol * 8)},
        "cpu_baseline": cpu,
        "ks4_over_ks1_curve": curve,
        "modp_batch": modp,
        "batched": batched,
        "hbm_phases": hbm_phases,
        "bivariate": bivariate,
    }
    print(json.dumps(line))
    return 0


def cpu_leg(f, g, outputs, curve_out, modp_out):
    """The CPU oracle timed on the host cores over full products of the
    workload (bounded), and the bit-exactness of every product the GPU arm
    computed: each variant's output on the workload, the curve's shapes and one
    product of the (Z/pZ)[x] batch."""
    import oracle
    w = WORKLOAD
    times, cores = run_oracle(f, g, 30, 1, budget_s=15.0)
    v = len(times) / sum(times)
    cpu = {"value": v, "unit": "products/s", "cores": cores, "kind": "oracle",
           "sample": "%d full products of the workload, all host threads" % len(times)}
    want = oracle.mul(f, g, w["coeff_bits"], w["is_signed"], threads=cores)
    exact = {k: bool(np.array_equal(o, want)) for k, o in outputs.items()}
    for key, (fc, gc, bc, hs) in curve_out.items():
        wc = oracle.mul(fc, gc, bc, False, threads=cores)
        exact["curve_" + key] = all(bool(np.array_equal(x, wc)) for x in hs)
    if modp_out is not None:
        fm, gm, p, hm = modp_out
        exact["modp_product0"] = bool(np.array_equal(hm, oracle.mul_mod(fm, gm, p, threads=cores)))
    exact["all"] = all(exact.values())
    return cpu, exact


CURVE = {"lens": [128, 512, 1024, 2048, 4096, 8192], "bits": [4, 48], "seed": 4046}


def run_curve(ks, dev, stream, flush, steps, warmup, world):
    """KS1-KS4 at degree {128 .. 8192} x {4, 48}-bit unsigned coefficients (the
    sizes and moduli of Sec. 4's experiments), each through a one-product plan
    replayed as a CUDA graph, L2 flushed between steps.  KS1 is timed on every
    engine and its best is the reference; KS2-KS4 use the library's engine."""
    import torch
    out, keep = {"config": dict(CURVE, l2="flushed between steps", api="ks_plan graph replay")}, {}
    cfgs = [("KS1", 1, 0), ("KS1_tc", 1, ks.ENGINE_TC), ("KS1_ntt", 1, ks.ENGINE_NTT),
            ("KS2", 2, 0), ("KS3", 3, 0), ("KS4", 4, 0), ("KS4_tc", 4, ks.ENGINE_TC)]
    for b in CURVE["bits"]:
        for L in CURVE["lens"]:
            f = ks_inputs.random_poly(L, b, False, CURVE["seed"] + L + b)
            g = ks_inputs.random_poly(L, b, False, CURVE["seed"] + L + b + 1)
            tf = torch.from_numpy(f.view(np.int64)).to(dev)
            tg = torch.from_numpy(g.view(np.int64)).to(dev)
            h = torch.empty((2 * L - 1, ks.out_limbs(L, L, b, False)), dtype=torch.int64,
                            device=dev)
            row, hs = {}, []
            for label, v, e in cfgs:
                try:
                    plan = ks.Plan([dict(h=h, f=tf, g=tg, coeff_bits=b, is_signed=False,
                                         variant=v, engine=e)])
                except ks.KSError:
                    continue  # engine not available at this size
                plan.capture(stream)
                for _ in range(max(warmup, 3)):
                    plan.execute(stream)
                torch.cuda.synchronize()
                evs = [(torch.cuda.Event(enable_timing=True),
                        torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
                for i in range(steps):
                    flush.zero_()
                    evs[i][0].record(stream)
                    plan.execute(stream)
                    evs[i][1].record(stream)
                torch.cuda.synchronize()
                plan.status()
                us = 1000.0 * barrier_max(sum(a.elapsed_time(z) for a, z in evs), world,
                                          dev) / steps
                row[label] = {"us": round(us, 2), "engine": plan.choice(0)[1]}
                plan.close()
                hs.append(h.cpu().numpy().view(np.uint64).copy())
            ks1 = min(row[k]["us"] for k in ("KS1", "KS1_tc", "KS1_ntt") if k in row)
            ks4 = min(row[k]["us"] for k in ("KS4", "KS4_tc") if k in row)
            row["ks4_over_best_ks1"] = round(ks1 / ks4, 3)
            row["ks2_over_best_ks1"] = round(ks1 / row["KS2"]["us"], 3)
            key = "L%d_b%d" % (L, b)
            out[key] = row
            keep[key] = (f, g, b, hs)
    return out, keep


MODP = {"workload": "modp_64x2pow16_p61", "n": 64, "len": 1 << 16, "p": (1 << 61) - 1,
        "seed": 5}


def run_modp(ks, dev, stream, flush, warmup, world, steps=3):
    """64 products in (Z/pZ)[x], p = 2^61 - 1, L = 2^16, uniform residues: one
    ks_mul_mod call per product (the library's variant and engine), a step is
    the whole batch, L2 flushed before each step."""
    import torch
    n, L, p = MODP["n"], MODP["len"], MODP["p"]
    fs, gs, hs = [], [], []
    for i in range(n):
        fs.append(torch.from_numpy(ks_inputs.random_residues(L, p, MODP["seed"] + 2 * i)
                                   .view(np.int64)).to(dev).reshape(L, 1))
        gs.append(torch.from_numpy(ks_inputs.random_residues(L, p, MODP["seed"] + 2 * i + 1)
                                   .view(np.int64)).to(dev).reshape(L, 1))
        hs.append(torch.empty((2 * L - 1, 1), dtype=torch.int64, device=dev))

    def step():
        for i in range(n):
            ks.ks_mul_mod(hs[i], fs[i], gs[i], p, 0, stream)
    for _ in range(max(1, warmup)):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    ks.status_sync(stream)
    ms = barrier_max(sum(a.elapsed_time(z) for a, z in evs), world, dev) / steps
    info = ks.plan_info(L, L, 61, False)
    res = {"config": dict(MODP, api="ks_mul_mod per product", l2="flushed before each step"),
           "products_per_s": world * n * 1000.0 / ms, "ms_per_batch": ms,
           "variant": info["variant"], "engine": info["engine"]}
    keep = (fs[0].cpu().numpy().view(np.uint64).reshape(-1),
            gs[0].cpu().numpy().view(np.uint64).reshape(-1), p,
            hs[0].cpu().numpy().view(np.uint64).reshape(-1, 1))
    del fs, gs, hs
    return res, keep


BIV_WORKLOAD = {"workload": "biv_mod_p61_256x256", "lx": 256, "ly": 256, "p": (1 << 61) - 1,
                "seed_f": 61, "seed_g": 62}


def run_bivariate(ks, dev, stream, flush, steps, warmup):
    """One product in (Z/pZ)[x, y] (l_x = l_y = 256, p = 2^61 - 1) by each of
    the four substitutions of Sec. 2, CUDA events on the bench stream, L2
    flushed before each product."""
    import torch
    w = BIV_WORKLOAD
    lx, ly, p = w["lx"], w["ly"], w["p"]
    f = ks_inputs.random_residues(lx * ly, p, w["seed_f"]).reshape(ly, lx)
    g = ks_inputs.random_residues(lx * ly, p, w["seed_g"]).reshape(ly, lx)
    tf = torch.from_numpy(f.view(np.int64)).to(dev)
    tg = torch.from_numpy(g.view(np.int64)).to(dev)
    h = torch.empty((2 * ly - 1, 2 * lx - 1), dtype=torch.int64, device=dev)
    out = {"config": dict(w, l2="flushed before each product (256 MiB write)")}
    ref = None
    for label, variant in (("KS1", 1), ("KS2", 2), ("KS3", 3), ("KS4", 4), ("KS_C", 5)):
        for _ in range(max(1, warmup)):
            ks.ks_mul_bivariate_mod(h, tf, tg, p, variant, stream)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            evs[i][0].record(stream)
            ks.ks_mul_bivariate_mod(h, tf, tg, p, variant, stream)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        ks.status_sync(stream)
        ms = sum(a.elapsed_time(z) for a, z in evs) / steps
        cur = h.cpu()
        same = True if ref is None else bool(torch.equal(cur, ref))
        ref = cur if ref is None else ref
        out[label] = {"ms": ms, "products_per_s": 1000.0 / ms, "same_as_KS1": same}
    return out


HBM_WORKLOAD = {"workload": "zx_product_2pow20_u256", "len_f": 1 << 20, "len_g": 1 << 20,
                "coeff_bits": 256, "is_signed": False, "seed_f": 55, "seed_g": 56}


def op_bits(info, lf, lg, b):
    """Bit lengths of the evaluated operands of one sub-product (the
    Propositions of Sec. 3.1-3.4: N (L - 1) + b)."""
    N = info["N"]
    return N * (lf - 1) + b, N * (lg - 1) + b


def phase_bytes(phase, info, lf, lg, b):
    """Algorithmic bytes of one memory-bound phase (every input read once, every
    output written once, in the most compact form the step has): pack reads the
    coefficients and writes the packed operands (N (L - 1) + b bits each);
    normalization reads the sub-products and writes the normalized values (each
    the size of a product of the operands); unpack reads the normalized values
    and writes the coefficients."""
    nprod, nnorm, ol, il = info["nprod"], info["nnorm"], info["out_limbs"], info["in_limbs"]
    fa, fb = op_bits(info, lf, lg, b)
    prod_bytes = (fa + fb + 7) // 8
    if phase == "pack":
        return (lf + lg) * il * 8 + nprod * ((fa + 7) // 8 + (fb + 7) // 8)
    if phase == "normalize":
        return (nprod + nnorm) * prod_bytes
    if phase == "unpack":
        return nnorm * prod_bytes + (lf + lg - 1) * ol * 8
    return None


def engine_bytes(phase, info, lf, lg):
    """Bytes the library's kernels move in that phase (its own storage formats:
    16-bit digits held in int32, int64 column sums), for comparison."""
    nprod, nA, nB, ncols = info["nprod"], info["nA"], info["nB"], info["ncols"]
    nw, nnorm, ol, il = info["nwords"], info["nnorm"], info["out_limbs"], info["in_limbs"]
    if phase == "pack":
        return (lf + lg) * il * 8 + nprod * (nA + nB) * 4
    if phase == "normalize":
        return nprod * ncols * 8 + nnorm * nw * 4
    if phase == "unpack":
        return nnorm * nw * 4 + (lf + lg - 1) * ol * 8
    return None


def run_hbm_phases(ks, dev, stream, flush, hbm_gbs, peak_kind, reps=3):
    """Per-phase achieved bandwidth of pack, normalize and unpack on one
    2^20 x 256-bit product (the transform regime; every array is larger than
    the 129 MB L2), from the library's per-phase CUDA events on the launching
    stream, L2 flushed before each product."""
    import torch
    w = HBM_WORKLOAD
    lf, lg, b = w["len_f"], w["len_g"], w["coeff_bits"]
    f = ks_inputs.random_poly(lf, b, False, w["seed_f"])
    g = ks_inputs.random_poly(lg, b, False, w["seed_g"])
    tf = torch.from_numpy(f.view(np.int64)).to(dev)
    tg = torch.from_numpy(g.view(np.int64)).to(dev)
    ol = ks.out_limbs(lf, lg, b, False)
    h = torch.empty((lf + lg - 1, ol), dtype=torch.int64, device=dev)
    out = {"config": dict(w, l2="flushed before each product (256 MiB write)", reps=reps),
           "peak_gbs": hbm_gbs, "peak_kind": peak_kind, "variants": {}}
    for label, variant in (("KS1", 1), ("KS2", 2)):
        info = ks.plan_info(lf, lg, b, False, variant, ks.ENGINE_AUTO)
        ks.ks_mul(h, tf, tg, b, False, variant, stream)  # warm-up (workspace, tables)
        torch.cuda.synchronize()
        ks.profile_collect()
        ks.profile_enable(True)
        t0 = time.perf_counter()
        for _ in range(reps):
            flush.zero_()
            ks.ks_mul(h, tf, tg, b, False, variant, stream)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / reps
        ks.profile_enable(False)
        ks.status_sync(stream)
        ph = ks.profile_collect()
        res = {"engine": info["engine"], "product_ms_wall": wall * 1000.0}
        for name in ("pack", "normalize", "unpack", "product"):
            tot, cnt = ph.get(name, (0.0, 0))
            if cnt == 0:
                continue
            ms = tot / cnt
            byts = phase_bytes(name, info, lf, lg, b)
            r = {"ms": ms}
            if byts is not None:
                gbs = byts / (ms / 1000.0) / 1e9
                eb = engine_bytes(name, info, lf, lg)
                r.update({"bytes": int(byts), "achieved_gbs": gbs, "frac": gbs / hbm_gbs,
                          "engine_bytes": int(eb), "engine_over_algorithmic": eb / byts})
            res[name] = r
        out["variants"][label] = res
    del tf, tg, h
    ks.release_cache()
    torch.cuda.empty_cache()
    return out


BATCH = {"workload": "uneven_batch_4096", "n": 4096, "seed": 20071231, "len": [8, 8192],
         "coeff_bits": [4, 512], "signed_fraction": 0.5}


def run_batched(ks, dev, stream, flush, steps, warmup, world):
    """4096 independent products (lengths log-uniform in [8, 8192] drawn
    independently, bits log-uniform in [4, 512], half signed) in one batched
    plan, replayed as a CUDA graph; fixed KS1 vs the autotuned table vs the
    learned model."""
    import torch
    lf, lg, cb, sg = ks_inputs.uneven_batch(BATCH["n"], BATCH["seed"])
    probs = []
    out_bits = 0
    for i in range(BATCH["n"]):
        f = ks_inputs.random_poly(int(lf[i]), int(cb[i]), bool(sg[i]), 7 * i + 1)
        g = ks_inputs.random_poly(int(lg[i]), int(cb[i]), bool(sg[i]), 7 * i + 2)
        ol = ks.out_limbs(int(lf[i]), int(lg[i]), int(cb[i]), bool(sg[i]))
        h = torch.empty((int(lf[i] + lg[i] - 1), ol), dtype=torch.int64, device=dev)
        probs.append(dict(h=h, f=torch.from_numpy(f.view(np.int64)).to(dev),
                          g=torch.from_numpy(g.view(np.int64)).to(dev),
                          coeff_bits=int(cb[i]), is_signed=bool(sg[i])))
        out_bits += output_bits(int(lf[i]), int(lg[i]), int(cb[i]))
    side = torch.cuda.Stream(device=dev)
    res = {}
    for name, mode in (("fixed_ks1", ks.DISPATCH_KS1), ("table", ks.DISPATCH_TABLE),
                       ("mlp", ks.DISPATCH_MLP)):
        plan = ks.Plan(probs, mode)
        plan.capture(side)
        for _ in range(warmup):
            plan.execute(side)
        side.synchronize()
        if world > 1:
            torch.distributed.barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for i in range(steps):
            with torch.cuda.stream(side):
                flush.zero_()
            evs[i][0].record(side)
            plan.execute(side)
            evs[i][1].record(side)
        side.synchronize()
        ks.status_sync(side)
        ms = barrier_max(sum(a.elapsed_time(z) for a, z in evs), world, dev) / steps
        choices = {}
        for i in range(len(probs)):
            v, e = plan.choice(i)
            key = "KS%d/%s" % (v, {1: "int32", 2: "ntt", 3: "tc"}[e])
            choices[key] = choices.get(key, 0) + 1
        res[name] = {"products_per_s": world * BATCH["n"] * 1000.0 / ms, "ms_per_batch": ms,
                     "output_gbit_per_s": world * out_bits / ms / 1e6,
                     "launches_per_batch": plan.launches(), "choices": choices}
        plan.close()
    res["config"] = dict(BATCH, graph=True, dispatch_state_installed=ks.DISPATCH_STATE_INSTALLED)
    res["mlp_over_fixed_ks1"] = res["mlp"]["products_per_s"] / res["fixed_ks1"]["products_per_s"]
    res["table_over_fixed_ks1"] = (res["table"]["products_per_s"]
                                   / res["fixed_ks1"]["products_per_s"])
    return res


def roofline_for(phase, ms, info, lf, lg, b, sg, hbm_gbs, sm_max_mhz, peak_kind):
    """Algorithmic work of one launch of the dominant phase over its event time.
    For the products: k ceil(opbits_f / 8) ceil(opbits_g / 8) 8-bit-digit
    multiply-adds (2 flops each) over the k sub-products, the Propositions'
    operand lengths; the engine's own digit work (7-bit digits on the tensor
    cores, 16-bit on the INT32 pipe) over that is `engine_overhead`."""
    nprod, nA, nB = info["nprod"], info["nA"], info["nB"]
    sec = ms / 1000.0
    fa, fb = op_bits(info, lf, lg, b)
    alg = 2.0 * nprod * ((fa + 7) // 8) * ((fb + 7) // 8)
    if phase == "product" and info["engine"] == 3:
        ach = alg / sec / 1e12
        return {"bound": "tensor", "phase": phase, "achieved": ach, "peak": BF16_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / BF16_TFLOPS, "traffic": None,
                "algorithmic_flops": alg, "engine_overhead": 2.0 * nprod * nA * nB / alg,
                "peak_kind": PEAK_KIND + " dense bf16 burst (fp16 runs at the bf16 rate)"}
    if phase == "product" and info["engine"] == 1:
        peak = SMS * IMAD_PER_SM_CLK * 2 * sm_max_mhz * 1e6 / 1e12
        ach = alg / sec / 1e12
        return {"bound": "alu", "phase": phase, "achieved": ach, "peak": peak,
                "unit": "TOP/s", "frac": ach / peak, "traffic": None,
                "algorithmic_flops": alg, "engine_overhead": 2.0 * nprod * nA * nB / alg,
                "peak_kind": "derived: 152 SMs x 64 IMAD/clk x 2 ops x max SM clock"}
    byts = phase_bytes(phase, info, lf, lg, b)
    ach = byts / sec / 1e9
    return {"bound": "hbm", "phase": phase, "achieved": ach, "peak": hbm_gbs, "unit": "GB/s",
            "frac": ach / hbm_gbs, "traffic": None, "peak_kind": peak_kind}


def main():
    args = parse()
    if args.case:
        return run_case(args.case)
    if args.impl == "reference":
        return reference_main(args)
    return main_ours(args)


if __name__ == "__main__":
    sys.exit(main())
