#!/usr/bin/env python3
"""Throughput of the GB300 speckle-masking path on TiO-shaped bursts.

One step = one whole burst through every stage (spectra, power/mean/noise,
modulus, bispectrum, phase recursion, inverse transform, mosaic) on a
synthetic 2560x2160x100 uint16 burst already resident in HBM.  ``value`` is
bursts/s over all ranks; ``e2e`` is the same metric through the serving API
(sm_submit_burst / sm_poll) from pinned host buffers, host<->device copies
inside the timed region.  Every input (1.1 GB of frames, 3.5 GB of spectra,
34 GB of bispectrum) is larger than the 129 MB L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank reconstructs its own bursts (replicas; the
path has no exchange step), a barrier brackets the timed region and the
slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (synth config, N, R)
    "tio2560": ("tio2560", 256, 24),
    "halpha1024": ("halpha1024", 128, 16),
    "subfield64": ("subfield64", 64, 8),
}
FP32_LANES_PER_SM = 128
FLOPS_PER_TRIPLE = 14          # two complex products + one complex add
METRIC = "bursts/sec and p99 latency, served vs plain, 2560x2160x100 at 1e-3 rel L2"
MODE_NAMES = {0: "submission", 1: "concurrent", 2: "pipelined"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tio2560", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--spectra", default="fp32", choices=["fp32", "fp16", "bf16"],
                    help="frame-spectra storage (precision sweep)")
    ap.add_argument("--acc", default="plain", choices=["plain", "kahan"], help="bispectrum sums")
    ap.add_argument("--phase", default="fp32", choices=["fp32", "fp64", "ff"], help="recursion arithmetic (ff: float-float)")
    ap.add_argument("--weight", default="bispec", choices=["bispec", "unit", "snr"], help="phase-term weighting")
    ap.add_argument("--iters", type=int, default=0, help="least-squares phase sweeps after the recursion")
    ap.add_argument("--inflight", type=int, default=2, help="bursts in flight on the served e2e path")
    ap.add_argument("--batch", type=int, default=4,
                    help="bursts per batched persistent launch in the batched record (0: skip it)")
    ap.add_argument("--batch-launch", default="tuned", choices=["tuned", "fused", "tiles", "grid"],
                    help="launch shape of the batched record's main part (tuned: the autotuned table's)")
    ap.add_argument("--mode", type=int, default=0, choices=[0, 1, 2],
                    help="served paths: 0 bursts' kernels in submission order, 1 concurrently, 2 pipelined (a "
                         "burst's phase/inverse/mosaic beside the next burst's transforms and bispectrum)")
    ap.add_argument("--layout", default="overlap50", choices=["overlap50", "paper"],
                    help="overlap50: stride N/2, ragged edges padded, blended mosaic; paper: stride N/4, "
                         "full tiles only, central-block mosaic (1110 cubes, 2368x1920 for TiO)")
    ap.add_argument("--size", default=None,
                    help="WxH override (profiling a smaller case of the same kernels)")
    return ap.parse_args()


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------- CPU oracle
def _oracle_subfield_task(task):
    """One host core's share of the CPU baseline: the FP64 oracle on one
    subfield at two frame counts and on one seeing cube at the same counts
    (seconds for each).  Runs in a spawned worker with one BLAS thread."""
    import time as _t
    from oracle import speckle_oracle as O
    path, sub, cube, N, R, frames_small, d_over_r0 = task
    frames = np.load(path, mmap_mode="r")
    stf = O.stf_model(N, 0.2885, d_over_r0)
    out = []
    for F in frames_small:
        fr = np.asarray(frames[:F])
        t0 = _t.perf_counter()
        O.reconstruct_subfield(fr, sub, N, 0.2885, R, N // 8, stf)
        t1 = _t.perf_counter()
        In, _, _ = O.frame_spectra(fr, cube, N, N // 8)
        P, M = O.power_mean(In)
        num, den = O.spectral_ratio(P, M, O.noise_floor(P, N, 0.2885), F, N, 0.2885)
        O.fit_d_over_r0(num, den, N, 0.2885)
        out.append((t1 - t0, _t.perf_counter() - t1))
    return out


def oracle_samples(workload: str, frames_small=(4, 8), reps: int = 1) -> list:
    """Time the FP64 oracle on all host cores (os.sched_getaffinity): a pool of
    one spawned worker per core, each reconstructing its own subfield (and
    fitting one seeing cube) at two frame counts, all at once; the per-core
    times are extrapolated linearly in F to the workload's frame count and
    over ceil(n_sub / cores) rounds of subfields plus ceil(n_cubes / cores)
    rounds of cubes.  One process runs `reps` timed samples (the synthetic
    burst is made once)."""
    cfg, N, R = WORKLOADS[workload]
    code = f"""
import json, math, multiprocessing as mp, os, sys, tempfile, time
sys.path.insert(0, {ROOT!r})
import numpy as np
from synth import CONFIGS, make_burst
from oracle import speckle_oracle as O
from bench import _oracle_subfield_task
spec = CONFIGS[{cfg!r}]
b = make_burst(spec, F={max(frames_small)}, burst=99)
subs = O.subfield_grid(spec.W, spec.H, {N}, {N} // 2)
cubes = O.seeing_cubes(spec.W, spec.H, {N}, {N} // 2)
cores = len(os.sched_getaffinity(0))
runs = []
with tempfile.TemporaryDirectory() as tmp:
    path = os.path.join(tmp, "frames.npy")
    np.save(path, b["frames"])
    tasks = [(path, subs[(len(subs) // 2 + 7 * k) % len(subs)], subs[cubes[(len(cubes) // 2 + k) % len(cubes)]],
              {N}, {R}, {tuple(frames_small)!r}, b["d_over_r0"]) for k in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        for _ in range({int(reps)}):
            t0 = time.perf_counter()
            per = pool.map(_oracle_subfield_task, tasks, chunksize=1)
            wall = time.perf_counter() - t0
            runs.append({{"per": per, "wall": wall}})
print(json.dumps({{"runs": runs, "n_sub": len(subs), "n_cubes": len(cubes), "F": spec.F, "cores": cores}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=900 + 60 * int(reps))
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    (f1, f2) = frames_small
    cores = d["cores"]

    def extrapolate(t1, t2):           # linear in F, to the workload's F
        per_frame = max((t2 - t1) / (f2 - f1), 0.0)
        return max(t1 - f1 * per_frame, 0.0) + d["F"] * per_frame

    out = []
    for run in d["runs"]:
        per = run["per"]                # per core: [(sub, cube) at f1, (sub, cube) at f2]
        a1 = statistics.mean(p[0][0] for p in per)
        a2 = statistics.mean(p[1][0] for p in per)
        s1 = statistics.mean(p[0][1] for p in per)
        s2 = statistics.mean(p[1][1] for p in per)
        rounds_sub = -(-d["n_sub"] // cores)
        rounds_cube = -(-d["n_cubes"] // cores)
        per_burst = rounds_sub * extrapolate(a1, a2) + rounds_cube * extrapolate(s1, s2)
        out.append({"value": 1.0 / per_burst, "unit": "bursts/s", "cores": cores, "kind": "oracle",
                    "sample": (f"FP64 numpy oracle on {cores} host cores (one spawned worker per core, one BLAS "
                               f"thread each): {cores} {N}x{N} subfields at once at F={f1} and F={f2} "
                               f"(mean {a1:.2f} s, {a2:.2f} s per subfield) and {cores} seeing cubes "
                               f"({s1:.2f} s, {s2:.2f} s), extrapolated linearly in F to {d['F']} frames and "
                               f"over {rounds_sub} rounds of subfields ({d['n_sub']}) + {rounds_cube} of cubes "
                               f"({d['n_cubes']}) = {per_burst:.0f} s per burst"),
                    "seconds": run["wall"]})
    return out


def oracle_sample(workload: str, frames_small=(4, 8)) -> dict:
    return oracle_samples(workload, frames_small, 1)[0]


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg, N, _ = WORKLOADS[args.workload]
    # one oracle process: W untimed samples, then K timed ones (each one
    # subfield per host core at F = 2 and 4 plus one seeing cube per core,
    # about 5 s)
    runs = oracle_samples(args.workload, (2, 4), args.warmup + args.steps)[args.warmup:]
    vals = [r["value"] for r in runs]
    s = runs[-1]
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "bursts/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"{args.workload} burst (FP64 oracle sample)"},
            "cpu_baseline": {"value": v, "unit": "bursts/s", "cores": s["cores"], "kind": "oracle",
                             "sample": s["sample"]},
            "e2e": {"value": v, "unit": "bursts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- ncu traffic
KERNEL_SOURCES = ("k_bispec.cu", "sm_bispec_tile.cuh")    # the bispectrum kernel and its tile body


def kernel_sha256() -> str:
    """SHA-256 over the bispectrum kernel's source files, in order."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1701_00581_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def kernel_traffic(units_per_launch: float, shape: dict):
    """DRAM bytes (read + write) per launch of the dominant kernel from the
    committed ncu summary, scaled from the captured case to this launch by
    the units processed; None when the kernel source changed since the
    counters were taken (the summary records the sources' SHA-256) or when
    this launch's subfield shape (N, R, F, spectra storage, sums) is not the
    captured one, since the bytes per subfield depend on all five."""
    path = os.path.join(ROOT, "profiles", "k_bispectrum_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("source_sha256") != kernel_sha256():
        return None
    if any(rec.get("shape", {}).get(k) != v for k, v in shape.items()):
        return None
    return rec["dram_bytes_per_unit"] * units_per_launch


# ---------------------------------------------------------------------------- serving
def serve_mixed(local, tio_burst, tio_ch, capacity, steps, mode=2):
    """Open-loop serving: Poisson arrivals of bursts from three NVST-shaped
    channels (TiO and G-band 2560x2160 with 256^2 subfields, H-alpha 1024^2
    with 128^2 subfields), admitted into the engine (120 GB budget) as slots
    free up.  Latency = arrival to mosaic on the host."""
    import torch
    from paper_1701_00581_gb300 import Channel, Engine
    from synth import CONFIGS, make_burst
    ha = CONFIGS["halpha1024"]
    hb = make_burst(ha, channel=2, burst=0, device=f"cuda:{local}")
    chans = [tio_ch, tio_ch, Channel(W=ha.W, H=ha.H, N=128, R=16, max_frames=ha.F)]
    frames = [torch.from_numpy(tio_burst["frames"]).pin_memory(), None,
              torch.from_numpy(hb["frames"]).pin_memory()]
    frames[1] = frames[0]
    eng = Engine(chans, hbm_budget_bytes=int(120e9), max_inflight=3, device=local, overlap_kernels=mode)
    outs = {c: [torch.empty((chans[c].H, chans[c].W), dtype=torch.float32).pin_memory() for _ in range(3)]
            for c in range(3)}
    # warm up every channel once
    for c in range(3):
        t = eng.submit(c, frames[c].numpy(), outs[c][0].numpy())        # seeing estimated per burst
        eng.poll(t, -1)
    n = max(30, 6 * steps)
    rate = 0.6 * capacity                      # offered load: 60 % of the measured capacity
    rng = np.random.default_rng(2017)
    arrive = np.cumsum(rng.exponential(1.0 / rate, n))
    chan = rng.integers(0, 3, n)
    queue, pending, lat, k, done = [], [], [], 0, 0
    t0 = time.perf_counter()
    while done < n:
        now = time.perf_counter() - t0
        while k < n and arrive[k] <= now:
            queue.append(k)
            k += 1
        while queue:
            i = queue[0]
            c = int(chan[i])
            tk = eng.try_submit(c, frames[c].numpy(), outs[c][i % 3].numpy())
            if tk is None:
                break
            pending.append((tk, i))
            queue.pop(0)
        still = []
        for tk, i in pending:
            st, _ = eng.poll(tk, 0)
            if st == 0:
                lat.append(time.perf_counter() - t0 - arrive[i])
                done += 1
            else:
                still.append((tk, i))
        pending = still
        time.sleep(0.0005)
    span = time.perf_counter() - t0
    eng.close()
    return {"offered_bursts_per_s": round(rate, 3), "achieved_bursts_per_s": round(n / span, 3),
            "arrival_span_s": round(float(arrive[-1]), 3), "makespan_s": round(span, 3),
            "realised_arrival_rate": round(n / float(arrive[-1]), 3), "bursts": n, "channels": "TiO 2560x2160, G-band 2560x2160, H-alpha 1024x1024 (uniform mix)",
            "latency_ms_p50": round(1000 * float(np.percentile(lat, 50)), 1),
            "latency_ms_p99": round(1000 * float(np.percentile(lat, 99)), 1),
            "nvst_rate_bursts_per_s": 0.3, "kernel_order": MODE_NAMES[mode],
            "note": "Poisson arrivals at 60% of the measured e2e capacity; latency = arrival to mosaic on host"}


# ---------------------------------------------------------------------------- batched
def run_batched(torch, plan, frames, spec, F, n_sub, info, args, stream, peak):
    """args.batch bursts (the same synthetic burst in separate workspaces) per
    step through sm_batch_reconstruct, captured once in a CUDA graph and
    replayed; also the batched spectra + bispectrum launch alone, and the
    same for the fused persistent launch shape; CUDA events on the launching
    stream."""
    from paper_1701_00581_gb300 import SM_U16, Batch
    nb = args.batch
    items = []
    for _ in range(nb):
        ws, lay = plan.workspace(F, n_sub)
        out = torch.empty((spec.H, spec.W), dtype=torch.float32, device=frames.device)
        items.append({"frames": frames, "ws": ws, "lay": lay, "out": out})
    from paper_1701_00581_gb300 import SM_BATCH_FUSED, SM_BATCH_GRID, SM_BATCH_TILES
    launch = {"tuned": 0, "fused": SM_BATCH_FUSED, "tiles": SM_BATCH_TILES, "grid": SM_BATCH_GRID}[args.batch_launch]
    bt = Batch([plan] * nb, [F] * nb, [SM_U16] * nb, launch=launch)

    def captured(batch):
        """The batch's whole reconstruction captured once in a CUDA graph (on
        a side stream), replayed on `stream` for every step."""
        batch.reconstruct(items, stream)                 # untimed: first launches, attribute setup
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            batch.reconstruct(items, side)
        torch.cuda.synchronize()
        return g

    graph = captured(bt)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            graph.replay()
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ok = bt.status() == 0
    del graph
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(args.steps):
        bt.spectra_bispectrum(items, stream)
    k1.record(stream)
    torch.cuda.synchronize()
    kms = k0.elapsed_time(k1) / args.steps
    ok = ok and bt.status() == 0
    opts = dict(bt.opts)
    bt.close()
    # the persistent fused launch itself (transforms and tiles from one
    # device queue), whatever the tuned shape is, timed the same way
    bf = Batch([plan] * nb, [F] * nb, [SM_U16] * nb, launch=SM_BATCH_FUSED)
    fgraph = captured(bf)
    f0, f1, f2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    with torch.cuda.stream(stream):
        f0.record(stream)
        for _ in range(args.steps):
            bf.spectra_bispectrum(items, stream)
        f1.record(stream)
        for _ in range(args.steps):
            fgraph.replay()
        f2.record(stream)
    torch.cuda.synchronize()
    del fgraph
    fused = {"launch_ms_per_burst": round(f0.elapsed_time(f1) / (args.steps * nb), 3),
             "bursts_per_s": round(nb * args.steps / (f1.elapsed_time(f2) / 1000.0), 4),
             "items": bf.info["n_items"], "ctas": bf.info["grid"], "opts": dict(bf.opts),
             "status_ok": bf.status() == 0,
             "note": "SM_BATCH_FUSED: every transform and tile of the batch from one device queue; the whole "
                     "batch captured in a CUDA graph and replayed per step"}
    bf.close()
    triples = info["n_pairs"] * F * n_sub * nb
    ach = FLOPS_PER_TRIPLE * triples / (kms / 1000.0) / 1e12
    rec = {"value": round(nb * args.steps / (ms / 1000.0), 4), "unit": "bursts/s", "bursts_per_launch": nb,
           "ms_per_burst": round(ms / (nb * args.steps), 3), "status_ok": ok,
           "launch": opts, "launch_ms": round(kms, 3), "launch_ms_per_burst": round(kms / nb, 3),
           "persistent_fused": fused,
           "launch_roofline": {"bound": "alu", "achieved": round(ach, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                               "frac": round(ach / peak, 4),
                               "note": "bispectrum flops only (14 x used triples); the launch also does every FFT"},
           "note": f"{nb} copies of the burst in separate workspaces per batched spectra + bispectrum launch "
                   "(the autotuned shape), then each burst's remaining stages, the whole batch captured once in a "
                   "CUDA graph and replayed per step; inputs resident in HBM"}
    del items
    return rec


def run_batched_small(torch, dev, args, stream, nb=8):
    """Small bursts, where batching pays: single-subfield bursts (64x64x100
    float32, |v| <= 8, seeing estimated from each burst), `nb` distinct
    bursts reconstructed one sm_reconstruct call each, then the same bursts
    through one batch (sm_batch_reconstruct: one batched spectra +
    bispectrum launch for all of them); inputs resident in HBM, CUDA events
    on the launching stream."""
    from paper_1701_00581_gb300 import SM_F32, Batch, Channel, Plan
    from synth import CONFIGS, make_burst
    spec = CONFIGS["subfield64"]
    F = spec.F
    plan = Plan(Channel(W=spec.W, H=spec.H, N=64, R=8, max_frames=F))
    n = plan.info["n_sub"]
    items = []
    for k in range(nb):
        bk = make_burst(spec, channel=40 + k, burst=0)
        ws, lay = plan.workspace(F, n)
        items.append({"frames": torch.from_numpy(bk["frames"]).to(dev), "ws": ws, "lay": lay,
                      "out": torch.empty((spec.H, spec.W), dtype=torch.float32, device=dev)})
    bt = Batch([plan] * nb, [F] * nb, [SM_F32] * nb)

    def one_by_one():
        for it in items:
            plan.reconstruct(it["frames"], F, None, n, it["ws"], it["lay"], it["out"], None, stream)

    def batched():
        bt.reconstruct(items, stream)

    res = {}
    for name, fn in (("one_by_one", one_by_one), ("batched", batched)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = nb * args.steps / (e0.elapsed_time(e1) / 1000.0)
    ok = bt.status() == 0
    opts = dict(bt.opts)
    bt.close()
    return {"value": round(res["batched"], 1), "unit": "bursts/s", "one_by_one": round(res["one_by_one"], 1),
            "speedup": round(res["batched"] / res["one_by_one"], 2), "bursts_per_launch": nb, "status_ok": ok,
            "launch": opts,
            "workload": "64x64x100 float32 single-subfield bursts (N = 64, |v| <= 8), seeing estimated per burst",
            "note": f"{nb} distinct bursts: one sm_reconstruct each vs one sm_batch_reconstruct; inputs resident in HBM"}


def serve_batched(torch, b, spec, ch, F, local, args, world, dev, nb=2):
    """The serving engine in batched mode: batches of `nb` bursts submitted
    together (one batched launch each), two batches in flight, frames from
    pinned host memory and mosaics copied back inside the timed region."""
    from paper_1701_00581_gb300 import Engine
    host_frames = torch.from_numpy(b["frames"]).pin_memory()
    fr_np = host_frames.numpy()
    n_in = 2 * nb
    outs = [torch.empty((spec.H, spec.W), dtype=torch.float32).pin_memory() for _ in range(n_in)]
    budget_gb = 160
    eng = Engine([ch], hbm_budget_bytes=int(budget_gb * 1e9), max_inflight=n_in, device=local, overlap_kernels=3)

    def run(nbatches):
        pending, lat, k = [], [], 0
        t_start = time.perf_counter()
        done = 0
        while done < nbatches:
            while k < nbatches and len(pending) < 2:
                items = [dict(channel=0, frames=fr_np, out=outs[(k % 2) * nb + i].numpy()) for i in range(nb)]
                tks = eng.try_submit_batch(items)
                if tks is None:
                    break
                pending.append((tks, time.perf_counter()))
                k += 1
            tks, ts = pending.pop(0)
            for t in tks:
                eng.poll(t, -1)
            lat.append(time.perf_counter() - ts)
            done += 1
        return time.perf_counter() - t_start, lat

    run(max(1, args.warmup // nb + 1))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    nbatches = max(2, args.steps // nb)
    el, lat = run(nbatches)
    el_max = max_over_ranks(el, dev)
    eng.close()
    return {"value": whole_job_rate(nbatches * nb, world, el_max), "unit": "bursts/s", "bursts_per_batch": nb,
            "batches_in_flight": 2, "h2d_bytes_per_step": int(b["frames"].nbytes),
            "d2h_bytes_per_step": int(spec.W * spec.H * 4),
            "latency_ms_p50": 1000 * float(np.percentile(lat, 50)),
            "latency_ms_p99": 1000 * float(np.percentile(lat, 99)), "hbm_budget_gb": budget_gb,
            "note": "engine in batched mode (overlap_kernels=3): batches of bursts through one batched launch, "
                    "latency per batch from submit to the last mosaic"}


# ---------------------------------------------------------------------------- ranks
def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (x itself when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, seconds_max: float) -> float:
    """Units all ranks processed divided by the slowest rank's time."""
    return units_per_rank * world / seconds_max


# ---------------------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1701_00581_gb300 import Channel, Engine, Plan, build
    build.build()
    from synth import CONFIGS, make_burst

    cfg, N, R = WORKLOADS[args.workload]
    spec = CONFIGS[cfg]
    if args.size:
        import dataclasses
        w, h = (int(x) for x in args.size.lower().split("x"))
        spec = dataclasses.replace(spec, W=w, H=h)
    b = make_burst(spec, channel=1, burst=rank, device=f"cuda:{local}")
    F = spec.F
    from paper_1701_00581_gb300 import (SM_ACC_KAHAN, SM_ACC_PLAIN, SM_BF16, SM_FP16, SM_FP32,
                                        SM_PHASE_FF, SM_PHASE_FP32, SM_PHASE_FP64, SM_W_BISPEC, SM_W_SNR, SM_W_UNIT,
                                        SM_EDGE_DROP, SM_MOSAIC_CENTRAL)
    modes = dict(spectra_prec={"fp32": SM_FP32, "fp16": SM_FP16, "bf16": SM_BF16}[args.spectra],
                 acc_mode={"plain": SM_ACC_PLAIN, "kahan": SM_ACC_KAHAN}[args.acc],
                 phase_prec={"fp32": SM_PHASE_FP32, "fp64": SM_PHASE_FP64, "ff": SM_PHASE_FF}[args.phase],
                 phase_weight={"bispec": SM_W_BISPEC, "unit": SM_W_UNIT, "snr": SM_W_SNR}[args.weight],
                 phase_iters=args.iters)
    if args.layout == "paper":
        modes.update(stride=N // 4, edge_mode=SM_EDGE_DROP, mosaic_mode=SM_MOSAIC_CENTRAL)
    ch = Channel(W=spec.W, H=spec.H, N=N, R=R, max_frames=F, **modes)
    plan = Plan(ch, device=local)
    info = plan.info
    n_sub = info["n_sub"]
    dev = torch.device("cuda", local)
    frames = torch.from_numpy(b["frames"]).to(dev)
    ws, lay = plan.workspace(F, n_sub)
    stf = plan.views(ws, lay, F, n_sub)["stf"]       # written by the seeing stage
    out = torch.empty((spec.H, spec.W), dtype=torch.float32, device=dev)
    valid = torch.empty((spec.H, spec.W), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        plan.stage_spectra(frames, F, 0, n_sub, ws, lay, stream)
        plan.stage_stats(F, n_sub, ws, lay, stream)
        plan.stage_seeing(F, 0, n_sub, ws, lay, stream)      # Sect. 3.1: r0 from the burst itself
        plan.stage_seeing_stf(ws, lay, stream)
        plan.stage_amplitude(n_sub, stf, ws, lay, stream)
        if ev is not None:
            ev[0].record(stream)
        plan.stage_bispectrum(F, n_sub, ws, lay, stream)
        if ev is not None:
            ev[1].record(stream)
        plan.stage_phase(n_sub, ws, lay, stream)
        plan.stage_inverse(F, 0, n_sub, ws, lay, stream)
        plan.stage_mosaic(ws, lay, out, valid, stream)

    launches_per_step = 9 + 2 * args.iters
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    bev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for i in range(args.steps):
        step(bev[i])
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = t0.elapsed_time(t1)
    bisp_ms = statistics.mean(a.elapsed_time(c) for a, c in bev)
    if world > 1:
        dist.barrier()
    ms_max = max_over_ranks(ms, dev)
    value = whole_job_rate(args.steps, world, ms_max / 1000.0)

    # roofline of the dominant kernel (bispectrum): FP32 ALU bound
    triples = info["n_pairs"] * F * n_sub
    achieved = FLOPS_PER_TRIPLE * triples / (bisp_ms / 1000.0) / 1e12
    props = torch.cuda.get_device_properties(local)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sm_max = 2070.0
    if os.path.exists(peaks_path):
        sm_max = float(json.load(open(peaks_path)).get("sm_max_mhz", sm_max))
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    traffic = kernel_traffic(n_sub, {"N": info["N"], "R": info["R"], "F": F, "spectra": args.spectra, "acc": args.acc})
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4),
                "traffic": None if traffic is None else int(traffic),
                "kernel": "k_bispectrum", "kernel_ms": round(bisp_ms, 3),
                "note": (f"{FLOPS_PER_TRIPLE} flops x {triples:.3e} used triples per launch; peak = "
                         f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                         f"{sm_max:.0f} MHz")}

    # plain end to end: one burst at a time through sm_reconstruct, the
    # frames copied in from pinned host memory and the mosaic copied out
    # inside the timed region, nothing overlapped (the served path's baseline)
    plain_e2e = None
    if not args.no_e2e:
        host_frames = torch.from_numpy(b["frames"]).pin_memory()
        host_out = torch.empty((spec.H, spec.W), dtype=torch.float32).pin_memory()
        dframes = torch.empty_like(frames)

        def plain_one():
            dframes.copy_(host_frames, non_blocking=True)
            plan.reconstruct(dframes, F, None, n_sub, ws, lay, out, None, stream)
            host_out.copy_(out, non_blocking=True)
            torch.cuda.current_stream().synchronize()

        for _ in range(max(1, args.warmup)):
            plain_one()
        if world > 1:
            dist.barrier()
        t_p = time.perf_counter()
        for _ in range(args.steps):
            plain_one()
        el_p = max_over_ranks(time.perf_counter() - t_p, dev)
        plain_e2e = {"value": whole_job_rate(args.steps, world, el_p), "unit": "bursts/s",
                     "h2d_bytes_per_step": int(b["frames"].nbytes), "d2h_bytes_per_step": int(spec.W * spec.H * 4),
                     "note": "sm_reconstruct one burst at a time, copies not overlapped"}
        del dframes, host_frames

    del ws, stf                              # the plain path's workspace (stf is a view of it)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    # batched: args.batch bursts per step through one persistent spectra +
    # bispectrum launch (sm_batch_reconstruct), inputs resident in HBM
    batched = None
    batched_small = None
    if args.batch > 0:
        batched = run_batched(torch, plan, frames, spec, F, n_sub, info, args, stream, peak)
        torch.cuda.empty_cache()
        batched_small = run_batched_small(torch, frames.device, args, stream)
        torch.cuda.empty_cache()

    # end to end through the serving API, host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        host_frames = torch.from_numpy(b["frames"]).pin_memory()
        K_IN = max(1, args.inflight)
        host_out = [torch.empty((spec.H, spec.W), dtype=torch.float32).pin_memory() for _ in range(K_IN)]
        host_valid = [torch.empty((spec.H, spec.W), dtype=torch.uint8).pin_memory() for _ in range(K_IN)]
        # the paper's layout needs a 123 GB workspace for one TiO burst
        budget_gb = 200 if args.layout == "paper" else 120
        eng = Engine([ch], hbm_budget_bytes=int(budget_gb * 1e9), max_inflight=K_IN, device=local,
                     overlap_kernels=args.mode)
        fr_np = host_frames.numpy()

        stages = []

        def serve(n):
            pending, lat = [], []
            submitted = done = 0
            t_start = time.perf_counter()
            while done < n:
                while submitted < n and len(pending) < K_IN:
                    k = submitted % K_IN
                    tk = eng.try_submit(0, fr_np, host_out[k].numpy(), host_valid[k].numpy())
                    if tk is None:
                        break
                    pending.append((tk, time.perf_counter()))
                    submitted += 1
                tk, ts = pending.pop(0)
                _, res = eng.poll(tk, -1)
                lat.append(time.perf_counter() - ts)
                stages.append(res["stage_ms"])
                done += 1
            return time.perf_counter() - t_start, lat

        serve(max(1, args.warmup))
        stages.clear()
        if world > 1:
            dist.barrier()
        el, lat = serve(args.steps)
        el_max = max_over_ranks(el, dev)
        eng.close()
        e2e = {"value": whole_job_rate(args.steps, world, el_max), "unit": "bursts/s",
               "h2d_bytes_per_step": int(b["frames"].nbytes),
               "d2h_bytes_per_step": int(spec.W * spec.H * 5),
               "latency_ms_p50": 1000 * float(np.percentile(lat, 50)),
               "latency_ms_p99": 1000 * float(np.percentile(lat, 99)),
               "max_inflight": K_IN, "hbm_budget_gb": budget_gb,
               "kernel_order": MODE_NAMES[args.mode],
               "stage_ms": {k: round(float(np.mean([st[k] for st in stages])), 3) for k in stages[0]}}

    # batched end to end: bursts submitted in batches of two (sm_submit_batch),
    # two batches in flight, host buffers, copies inside the timed region
    batched_e2e = None
    if not args.no_e2e and args.batch > 0:
        batched_e2e = serve_batched(torch, b, spec, ch, F, local, args, world, dev)

    serving = None
    if not args.no_serve and args.workload == "tio2560" and not args.size:
        serving = serve_mixed(local, b, ch, e2e["value"] if e2e else value, args.steps, args.mode)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            cpu = oracle_sample(args.workload)
            cpu.pop("seconds", None)
        except Exception as e:  # reported, never fatal
            cpu = {"value": None, "error": str(e)[-300:]}

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 4), "unit": "bursts/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.spectra == "fp32" else f"{args.spectra} spectra, f32 arithmetic",
                "data": "synthetic",
                "config": {"workload": f"{args.workload} burst: {spec.W}x{spec.H}x{F} uint16, "
                                       f"{n_sub} subfields of {N}^2 at "
                                       + ("50% overlap" if args.layout == "overlap50" else
                                          "75% overlap, full tiles, central-block mosaic (the paper's layout)")
                                       + f", |v|<={R}",
                           "path": "plain per-burst stages",
                           "precision": f"spectra {args.spectra}, bispectrum sums {args.acc} fp32, "
                                        f"recursion {args.phase}",
                           "phase": f"recursion weighted by {args.weight}"
                                    + (f", {args.iters} least-squares sweeps" if args.iters else ""),
                           "seeing": "estimated from each burst (spectral ratio over the non-overlapping "
                                     f"{N}^2 cubes, {info['n_cubes']} cubes)",
                           "l2": "inputs larger than L2 (no flush)",
                           "parallelism": f"replicas x{world}"},
                "gpu_launches": launches_per_step * args.steps,
                "roofline": roofline, "clocks": clocks, "e2e": e2e, "plain_e2e": plain_e2e, "batched": batched,
                "batched_small": batched_small, "batched_e2e": batched_e2e,
                "serving": serving,
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
