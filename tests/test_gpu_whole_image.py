"""The whole TiO mosaic against a full oracle run (opt-in).

The 2560 x 2160 x 100 burst goes through the stage calls bench.py times
(304 subfields of 256^2, seeing estimated from the burst); the FP64 oracle
then reconstructs every one of the 304 subfields on the host cores, with its
own seeing estimate over the 80 cubes, and merges them.  The mosaic is
compared over the whole valid mask at 1e-3 rel L2, the mask exactly.

The oracle run takes about 40 s of one core per subfield (some 15 minutes
on 16 cores), so the test runs only with SPECKLE_WHOLE_IMAGE=1; the
sampled full-size tests cover the same path on every GPU run.
"""
import os
import tempfile

import numpy as np
import pytest

from oracle import speckle_oracle as O

from . import _cases as CS
from . import _oracle_pool as OP

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("SPECKLE_WHOLE_IMAGE") != "1",
                                 reason="full oracle run of a TiO burst; set SPECKLE_WHOLE_IMAGE=1")]

IMG_TOL = 1e-3
N, R, STRIDE, TAPER = 256, 24, 128, 32


def test_whole_tio_mosaic_matches_a_full_oracle_run():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_00581_gb300 import Channel, Plan, build
    from synth import CONFIGS, make_burst
    build.build()
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
    got, got_valid = out.cpu().numpy(), valid.cpu().numpy().astype(bool)
    subs = [tuple(int(t) for t in q) for q in plan.subfields()]
    del ws, views, frames
    torch.cuda.empty_cache()
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "frames.npy")
        np.save(path, b["frames"])
        cubes = O.seeing_cubes(spec.W, spec.H, N, STRIDE)
        xs = np.array(OP.pool_map(OP.cube_seeing, [(path, subs[c], N, CS.FC, TAPER) for c in cubes]))
        stf = O.stf_model(N, CS.FC, [float(1.0 / np.mean(1.0 / xs))])
        recs = dict(OP.pool_map(OP.subfield_image, [(path, s, subs[s], N, CS.FC, R, TAPER, stf)
                                                    for s in range(len(subs))]))
    ref, ref_valid = O.mosaic([recs[s] for s in range(len(subs))], subs, spec.W, spec.H, TAPER)
    err = CS.rel_l2(got[ref_valid], ref[ref_valid])
    report = os.environ.get("SPECKLE_REPORT_DIR")
    if report:
        with open(os.path.join(report, "whole_image_tio.txt"), "w") as f:
            f.write(f"TiO 2560x2160x100, 304 subfields: mosaic rel L2 against the full oracle run {err:.3e} over "
                    f"{int(ref_valid.sum())} valid pixels; masks equal: {bool(np.array_equal(got_valid, ref_valid))}\n")
    assert np.array_equal(got_valid, ref_valid)
    assert np.all(got[~ref_valid] == 0)
    assert err < IMG_TOL
