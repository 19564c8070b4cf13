"""Host logic of the batched launch's tuning and of the bench's traffic
record (CPU): the autotuner writes one table entry per (N, R) and launch
kind, the library's lookup picks the nearest shape and the requested (or
fastest) launch from the compiled table, and the bench applies the
committed DRAM traffic only to the kernel sources and subfield shape it was
measured on."""
import json
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TUNE_H = os.path.join(ROOT, "paper_1701_00581_gb300", "csrc", "sm_tune.h")


def _table(path):
    src = open(path).read()
    body = re.search(r"constexpr TuneEntry kTune\[\] = \{(.*?)\};", src, flags=re.S).group(1)
    rows = []
    for m in re.finditer(r"\{([^{}]*)\}", body):
        v = [x.strip() for x in m.group(1).split(",")]
        rows.append(dict(N=int(v[0]), R=int(v[1]), lookahead=int(v[2]), ctas=int(v[3]), launch=int(v[4]),
                         order=int(v[5]), ms=float(v[6])))
    return rows


def test_autotune_writes_one_entry_per_launch_kind(tmp_path, monkeypatch):
    from paper_1701_00581_gb300 import autotune
    path = tmp_path / "sm_tune.h"
    shutil.copy(TUNE_H, path)
    monkeypatch.setattr(autotune, "TUNE_H", str(path))
    rows = [dict(lookahead=la, ctas_per_sm=c, launch=l, tile_order=o, ms_per_burst=ms, ok=True)
            for la, c, l, o, ms in [(2, 4, 1, 1, 10.5), (4, 4, 1, 2, 10.2), (2, 3, 2, 1, 11.0),
                                    (2, 4, 2, 2, 10.9), (2, 4, 3, 1, 10.4)]]
    autotune.write_table({(128, 16): rows, (64, 8): rows[:1]})
    got = _table(path)
    assert [(r["N"], r["R"], r["launch"]) for r in got] == [(128, 16, 1), (128, 16, 2), (128, 16, 3), (64, 8, 1)]
    fused = got[0]
    assert (fused["lookahead"], fused["order"], fused["ms"]) == (4, 2, 10.2)      # fastest of its launch kind
    tiles = got[1]
    assert (tiles["ctas"], tiles["order"], tiles["ms"]) == (4, 2, 10.9)
    # the rest of the header is kept
    assert open(path).read().split("// BEGIN TABLE")[0] == open(TUNE_H).read().split("// BEGIN TABLE")[0]


def test_tune_lookup_follows_the_table(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    cases = [(256, 24, 0), (256, 9, 0), (256, 24, 1), (256, 24, 2), (256, 24, 3), (128, 16, 0), (100, 8, 0),
             (64, 8, 0), (64, 8, 1), (512, 30, 2)]
    src = ['#include <cstdio>', f'#include "{TUNE_H}"', "int main() {"]
    for N, R, L in cases:
        src.append(f'  {{ auto t = smt::tune_for({N}, {R}, {L}); std::printf("%d %d %d %d %d %d\\n", t.N, t.R, '
                   f't.lookahead, t.ctas_per_sm, t.launch, t.tile_order); }}')
    src += ["  return 0;", "}"]
    f = tmp_path / "tune.cpp"
    f.write_text("\n".join(src) + "\n")
    exe = tmp_path / "tune"
    subprocess.run([cxx, "-std=c++17", str(f), "-o", str(exe)], check=True)
    out = [list(map(int, l.split())) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                             text=True).stdout.splitlines()]
    table = _table(TUNE_H)
    for (N, R, L), (n, r, la, c, l, o) in zip(cases, out):
        # the nearest N of the table, then its nearest R
        bn = min({e["N"] for e in table}, key=lambda x: abs(x - N))
        br = min({e["R"] for e in table if e["N"] == bn}, key=lambda x: abs(x - R))
        assert (n, r) == (bn, br), (N, R, L)
        shape = [e for e in table if e["N"] == bn and e["R"] == br]
        pick = [e for e in shape if L == 0 or e["launch"] == L] or shape
        best = min(pick, key=lambda e: e["ms"])
        assert (la, c, o) == (best["lookahead"], best["ctas"], best["order"]), (N, R, L)
        assert l == (L if L else best["launch"])


def test_bench_traffic_applies_only_to_the_captured_kernel_and_shape(monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "k_bispectrum_traffic.json")))
    shape = dict(rec["shape"])
    if rec["source_sha256"] != bench.kernel_sha256():
        pytest.skip("the committed traffic record is for other kernel sources")
    t = bench.kernel_traffic(304, shape)
    assert t == pytest.approx(rec["dram_bytes_per_unit"] * 304)
    assert bench.kernel_traffic(304, dict(shape, N=128)) is None
    assert bench.kernel_traffic(304, dict(shape, spectra="fp16")) is None
    monkeypatch.setattr(bench, "kernel_sha256", lambda: "0" * 64)
    assert bench.kernel_traffic(304, shape) is None
