"""Parity of the full-size TiO burst through the path bench.py times.

bench.py reconstructs a 2560 x 2160 x 100 uint16 burst (304 subfields of
256^2 at 50 % overlap, the bottom row 256 x 240, |v| <= 24) stage by stage,
every subfield in one chunk, with the seeing estimated from the burst itself
(Sect. 3.1) and the model STF at that estimate.  The same stage calls run
here, and the FP64 oracle is run independently on a fixed sample of 16
subfields -- two 2 x 2 blocks in the interior, the 2 x 2 block at the
origin and four consecutive 256 x 240 subfields of the bottom row -- with its
own seeing estimate over all 80 cubes:

* the burst's D/r0 against the oracle's;
* per sampled subfield: P, M at 1e-4, B at every used pair at 1e-4, the
  sub-image at 1e-3;
* the mosaic at 1e-3 over every pixel whose covering subfields are all in
  the sample (the interiors of the blocks and of the bottom strip).
"""
import os
import tempfile

import numpy as np
import pytest

from oracle import speckle_oracle as O

from . import _cases as CS
from . import _oracle_pool as OP

pytestmark = pytest.mark.gpu

SPEC_TOL = 1e-4
IMG_TOL = 1e-3
N, R, STRIDE, TAPER = 256, 24, 128, 32


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_00581_gb300 import build
    build.build()
    return t


def _sample(nsx, nsy):
    """Subfield indices of the sample: 2 x 2 blocks at grid (0, 0), (3, 3) and
    (12, 9), and four consecutive subfields of the bottom (ragged) row."""
    blocks = [(0, 0), (3, 3), (12, 9)]
    s = [(j + dj) * nsx + (i + di) for (i, j) in blocks for dj in (0, 1) for di in (0, 1)]
    s += [(nsy - 1) * nsx + i for i in (6, 7, 8, 9)]
    return s


@pytest.fixture(scope="module")
def run(torch):
    from paper_1701_00581_gb300 import Channel, Plan
    from synth import CONFIGS, make_burst
    spec = CONFIGS["tio2560"]
    b = make_burst(spec, channel=1, burst=0, device="cuda:0")
    F = spec.F
    plan = Plan(Channel(W=spec.W, H=spec.H, N=N, R=R, max_frames=F))
    n = plan.info["n_sub"]
    dev = "cuda:0"
    frames = torch.from_numpy(b["frames"]).to(dev)
    ws, lay = plan.workspace(F, n)
    views = plan.views(ws, lay, F, n)
    out = torch.zeros((spec.H, spec.W), device=dev)
    valid = torch.zeros((spec.H, spec.W), dtype=torch.uint8, device=dev)
    # the step bench.py times, call for call
    plan.stage_spectra(frames, F, 0, n, ws, lay)
    plan.stage_stats(F, n, ws, lay)
    plan.stage_seeing(F, 0, n, ws, lay)
    plan.stage_seeing_stf(ws, lay)
    plan.stage_amplitude(n, views["stf"], ws, lay)
    plan.stage_bispectrum(F, n, ws, lay)
    plan.stage_phase(n, ws, lay)
    plan.stage_inverse(F, 0, n, ws, lay)
    plan.stage_mosaic(ws, lay, out, valid)
    torch.cuda.synchronize()
    subs = [tuple(int(t) for t in q) for q in plan.subfields()]
    pick = _sample(plan.info["nsx"], plan.info["nsy"])
    assert sum(subs[s][3] == 240 for s in pick) == 4
    wv = OP.used_pairs(N, R, CS.FC)
    idx = plan.pair_index(wv)
    gpu = {s: {"P": views["P"][s].cpu().numpy(), "M": views["M"][s].cpu().numpy(),
               "B": views["B"][s].cpu().numpy()[idx], "rec": views["rec"][s].cpu().numpy()}
           for s in pick}
    seeing = views["seeing"].cpu().numpy().copy()
    res = {"gpu": gpu, "seeing": seeing, "out": out.cpu().numpy(), "valid": valid.cpu().numpy().astype(bool),
           "subs": subs, "pick": pick, "spec": spec, "K": plan.info["K"]}
    del ws, views, frames
    torch.cuda.empty_cache()
    # the oracle, on the host cores
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "frames.npy")
        np.save(path, b["frames"])
        cubes = O.seeing_cubes(spec.W, spec.H, N, STRIDE)
        xs = np.array(OP.pool_map(OP.cube_seeing, [(path, subs[c], N, CS.FC, TAPER) for c in cubes]))
        x_burst = float(1.0 / np.mean(1.0 / xs))
        stf = O.stf_model(N, CS.FC, [x_burst])
        orc = OP.pool_map(OP.subfield_whole,
                          [(path, s, subs[s], N, CS.FC, R, TAPER, stf, tmp) for s in pick])
        res["oracle"] = {o["s"]: o for o in orc}
        for s in pick:
            res["oracle"][s]["B"] = np.load(os.path.join(tmp, f"B_{s}.npy"))
    res["x_cubes"], res["x_burst"] = xs, x_burst
    return res


def _half_box(grid, K):
    return grid[N // 2:N // 2 + K + 1, N // 2 - K:N // 2 + K + 1]


def test_tio_seeing_estimate_matches_the_oracle(run):
    assert len(run["x_cubes"]) == 80
    assert np.allclose(run["seeing"][:80], run["x_cubes"], rtol=2e-3, atol=0)
    assert run["seeing"][80] == pytest.approx(run["x_burst"], rel=2e-3)


def test_tio_sampled_subfields_P_M_B(run):
    K = run["K"]
    for s in run["pick"]:
        g, o = run["gpu"][s], run["oracle"][s]
        assert CS.rel_l2(g["P"][:, :2 * K + 1], _half_box(o["P"], K)) < SPEC_TOL, s
        assert CS.rel_l2(g["M"][:, :2 * K + 1], _half_box(o["M"], K)) < SPEC_TOL, s
        assert CS.rel_l2(g["B"], o["B"]) < SPEC_TOL, s


def test_tio_sampled_sub_images(run):
    for s in run["pick"]:
        x0, y0, w, h = run["subs"][s]
        got = run["gpu"][s]["rec"][:h, :w]
        assert CS.rel_l2(got, run["oracle"][s]["rec"][:h, :w]) < IMG_TOL, s


def test_tio_mosaic_where_the_sample_covers_every_subfield(run):
    spec, subs, pick = run["spec"], run["subs"], run["pick"]
    cover_all = np.zeros((spec.H, spec.W), np.int32)
    cover_pick = np.zeros((spec.H, spec.W), np.int32)
    for s, (x0, y0, w, h) in enumerate(subs):
        cover_all[y0:y0 + h, x0:x0 + w] += 1
        if s in pick:
            cover_pick[y0:y0 + h, x0:x0 + w] += 1
    ref, ref_valid = O.mosaic([run["oracle"][s]["rec"] for s in pick], [subs[s] for s in pick],
                              spec.W, spec.H, TAPER)
    region = (cover_all == cover_pick) & (cover_pick > 0) & ref_valid
    # 256^2 at the origin block, 128^2 in each interior block, 512 x 112 of the strip
    assert region.sum() >= 256 * 256 + 2 * 128 * 128 + 256 * 112
    assert np.array_equal(run["valid"][region], ref_valid[region])
    assert CS.rel_l2(run["out"][region], ref[region]) < IMG_TOL
