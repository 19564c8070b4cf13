"""Autotuner of the batched persistent launch (run on the GPU).

    python -m paper_1701_00581_gb300.autotune [--bursts 2] [--reps 3] [--write]

For each channel shape (N, R) of the NVST-shaped workloads it times the
persistent spectra + bispectrum launch (sm_batch_spectra_bispectrum) over a
synthetic burst of that shape, for every launch shape the library offers:

* lookahead: subfields whose transforms are queued ahead of their tiles;
* CTAs per SM: 4 (128 registers a thread) or 3 (168, no spilling);
* the launch: one persistent launch of transforms and tiles (fused); the
  per-stage transforms, then a persistent launch of the tiles; or the
  per-stage transforms, then one grid of CTAs over every burst's tiles.

The fastest options of each launch per (N, R) go into the table of
``csrc/sm_tune.h`` (with --write), which the library compiles in: a batch
built without options takes the fastest entry of its shape, one built with
a launch kind but no other options takes that launch's entry.  The timings are printed as a table and, with
--write, also saved to ``profiles/autotune_batch_launch.md``.  The tile
geometry itself (16 x 8 targets by 8 x 4 offsets per CTA) is fixed in the
kernel; its share of computed pairs that are used is reported per shape
(``used / computed`` from the plan), the quantity a different tile would
change.
"""
from __future__ import annotations

import argparse
import itertools
import os
import re
import statistics
import sys
import time

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
TUNE_H = os.path.join(PKG, "csrc", "sm_tune.h")
REPORT = os.path.join(ROOT, "profiles", "autotune_batch_launch.md")

# (workload name, synth config, N, R, bursts per launch: None = --bursts);
# single-subfield bursts are timed eight to a launch, the use batching has
# for them
SHAPES = [("tio2560", "tio2560", 256, 24, None), ("halpha1024", "halpha1024", 128, 16, None),
          ("subfield64", "subfield64", 64, 8, 8)]
LAUNCH_NAMES = {1: "fused persistent", 2: "stage FFT + persistent tiles", 3: "stage FFT + tile grid"}
GRID = {"lookahead": (2, 4), "ctas_per_sm": (3, 4), "launch": (1, 2, 3), "tile_order": (1, 2)}


def tune_shape(torch, cfg, N, R, bursts, reps, frames_n):
    from paper_1701_00581_gb300 import SM_F32, SM_U16, Batch, Channel, Plan
    from synth import CONFIGS, make_burst
    spec = CONFIGS[cfg]
    ftype = SM_U16 if spec.counts else SM_F32
    F = spec.F if frames_n is None else frames_n
    b = make_burst(spec, channel=3, burst=0, device="cuda:0", F=F)
    plan = Plan(Channel(W=spec.W, H=spec.H, N=N, R=R, max_frames=F))
    frames = torch.from_numpy(b["frames"]).to("cuda:0")
    n = plan.info["n_sub"]
    items = []
    for _ in range(bursts):
        ws, lay = plan.workspace(F, n)
        items.append({"frames": frames, "ws": ws, "lay": lay})
    stream = torch.cuda.current_stream()
    rows = []
    for la, cps, fuse, order in itertools.product(GRID["lookahead"], GRID["ctas_per_sm"], GRID["launch"],
                                                   GRID["tile_order"]):
        if fuse != 1 and la != GRID["lookahead"][0]:
            continue                     # lookahead only orders transform items
        if fuse == 3 and (cps != 4 or order != 1):
            continue                     # the grid launch has no queue: 4 CTAs per SM, the plan's order
        bt = Batch([plan] * bursts, [F] * bursts, [ftype] * bursts, lookahead=la, ctas_per_sm=cps, launch=fuse,
                   tile_order=order)
        bt.spectra_bispectrum(items, stream)
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bt.spectra_bispectrum(items, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / bursts)
        ok = bt.status() == 0
        rows.append({"lookahead": la, "ctas_per_sm": cps, "launch": fuse, "tile_order": order,
                     "ms_per_burst": statistics.median(times), "ok": ok, "ctas": bt.info["grid"]})
        bt.close()
    # reference: the per-stage spectra and bispectrum kernels, burst by burst
    times = []
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for it in items:
            plan.stage_spectra(it["frames"], F, 0, n, it["ws"], it["lay"], stream)
            plan.stage_bispectrum(F, n, it["ws"], it["lay"], stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if r:
            times.append(e0.elapsed_time(e1) / bursts)
    stage_ms = statistics.median(times)
    del items, frames
    torch.cuda.empty_cache()
    used = plan.info["n_pairs"] / (plan.info["n_tiles"] * plan.info["tile_pairs"])
    return rows, {"W": spec.W, "H": spec.H, "F": F, "n_sub": n, "n_tiles": plan.info["n_tiles"],
                  "used_over_slots": used, "stage_ms": stage_ms, "bursts": bursts}


def write_table(best):
    """best: (N, R) -> the timed rows; one table entry per (N, R) and launch
    kind, the fastest options of that launch."""
    src = open(TUNE_H).read()
    lines = ["constexpr TuneEntry kTune[] = {"]
    for (N, R), rows in sorted(best.items(), reverse=True):
        for launch in sorted({r["launch"] for r in rows}):
            r = min((r for r in rows if r["launch"] == launch), key=lambda r: r["ms_per_burst"])
            lines.append(f"    {{{N}, {R}, {r['lookahead']}, {r['ctas_per_sm']}, {r['launch']}, {r['tile_order']}, "
                         f"{r['ms_per_burst']:.4f}}},")
    lines.append("};")
    new = re.sub(r"// BEGIN TABLE \(autotune.py\)\n.*?// END TABLE",
                 "// BEGIN TABLE (autotune.py)\n" + "\n".join(lines) + "\n// END TABLE", src, flags=re.S)
    open(TUNE_H, "w").write(new)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--bursts", type=int, default=2, help="bursts per timed launch")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--frames", type=int, default=None, help="frames per burst (default: the workload's)")
    ap.add_argument("--write", action="store_true", help="write csrc/sm_tune.h and the profiles/ summary")
    args = ap.parse_args()
    sys.path.insert(0, ROOT)
    import torch
    from paper_1701_00581_gb300 import build
    build.build()
    best, report = {}, []
    t0 = time.time()
    for name, cfg, N, R, nb in SHAPES:
        rows, meta = tune_shape(torch, cfg, N, R, nb or args.bursts, args.reps, args.frames)
        ok = [r for r in rows if r["ok"]]
        win = min(ok, key=lambda r: r["ms_per_burst"])
        best[(N, R)] = ok
        report.append((name, N, R, meta, rows, win))
    out = [f"# Autotune of the batched persistent launch\n",
           f"Command: `python -m paper_1701_00581_gb300.autotune --bursts {args.bursts} --reps {args.reps}"
           + (f" --frames {args.frames}" if args.frames else "") + " --write`",
           f"(spectra + bispectrum launch time per burst, median of {args.reps}, {args.bursts} bursts per launch "
           f"unless stated; "
           f"{time.time() - t0:.0f} s)\n"]
    for name, N, R, meta, rows, win in report:
        out.append(f"## {name}: N = {N}, R = {R} ({meta['W']}x{meta['H']}x{meta['F']}, {meta['n_sub']} subfields, "
                   f"{meta['n_tiles']} tiles per subfield, used pairs / tile slots = {meta['used_over_slots']:.3f}; "
                   f"{meta['bursts']} bursts per launch)\n")
        out.append(f"Per-stage spectra + bispectrum kernels for comparison: {meta['stage_ms']:.4g} ms per burst.\n")
        out.append("| lookahead | CTAs/SM | launch | tile order | ms per burst |")
        out.append("|---|---|---|---|---|")
        for r in sorted(rows, key=lambda r: r["ms_per_burst"]):
            mark = " **(chosen)**" if r is win else ""
            out.append(f"| {r['lookahead']} | {r['ctas_per_sm']} | {LAUNCH_NAMES[r['launch']]} "
                       f"| {'plan' if r['tile_order'] == 1 else 'costliest first'} | {r['ms_per_burst']:.4g}{mark} |")
        out.append("")
    text = "\n".join(out)
    print(text)
    if args.write:
        write_table(best)
        os.makedirs(os.path.dirname(REPORT), exist_ok=True)
        open(REPORT, "w").write(text + "\n")


if __name__ == "__main__":
    main()
