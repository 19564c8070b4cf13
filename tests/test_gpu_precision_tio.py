"""Precision sweep on the full-size TiO burst (2560 x 2160 x 100 uint16, 304
subfields of 256^2, |v| <= 24).

Every precision mode of the path -- frame spectra stored in FP32, FP16
(scaled by 2^14) or BF16; bispectrum sums plain or compensated (Kahan);
recursion arithmetic FP32, FP64 or float-float -- runs the whole burst on the GPU with
the same model STF, and is compared with the FP64 oracle on a fixed sample
of 16 subfields (two 2 x 2 blocks, the 2 x 2 block at the origin, four
ragged 256 x 240 subfields of the bottom row).  Per stage:

* power spectrum: rel L2 of P on the half box, worst subfield;
* bispectrum phase: RMS of arg(B_gpu conj B_oracle) over every used pair,
  weighted by |B_oracle|^2, worst subfield (radians);
* image: rel L2 of the sub-images, worst subfield, and of the mosaic over
  the pixels the sample covers alone.

The reconstructed image -- the mosaic -- is gated at 1e-3 in every mode
(the mixed-precision tolerance); the other figures are reported
(SPECKLE_REPORT_DIR) with gates that follow each storage type's mantissa:
BF16 spectra (8 significant bits) leave single sub-images at about 1.3e-3,
which the overlapping blend of the mosaic averages down to about 5e-4.
"""
import os
import tempfile

import numpy as np
import pytest

from oracle import speckle_oracle as O

from . import _cases as CS
from . import _oracle_pool as OP
from .test_gpu_fullsize_bench_path import _sample

pytestmark = pytest.mark.gpu

N, R, STRIDE, TAPER = 256, 24, 128, 32
IMG_TOL = 1e-3


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_00581_gb300 import build
    build.build()
    return t


@pytest.fixture(scope="module")
def tio(torch):
    from paper_1701_00581_gb300 import Channel, Plan
    from synth import CONFIGS, make_burst
    spec = CONFIGS["tio2560"]
    b = make_burst(spec, channel=1, burst=0, device="cuda:0")
    plan = Plan(Channel(W=spec.W, H=spec.H, N=N, R=R, max_frames=spec.F))
    subs = [tuple(int(t) for t in q) for q in plan.subfields()]
    pick = _sample(plan.info["nsx"], plan.info["nsy"])
    stf = O.stf_model(N, CS.FC, [float(np.mean(b["d_over_r0"]))])
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "frames.npy")
        np.save(path, b["frames"])
        orc = OP.pool_map(OP.subfield_whole, [(path, s, subs[s], N, CS.FC, R, TAPER, stf, tmp) for s in pick])
        oracle = {o["s"]: o for o in orc}
        for s in pick:
            oracle[s]["B"] = np.load(os.path.join(tmp, f"B_{s}.npy"))
    return {"spec": spec, "burst": b, "subs": subs, "pick": pick, "stf": stf, "oracle": oracle}


def _gpu(torch, tio, **modes):
    from paper_1701_00581_gb300 import Channel, Plan
    spec = tio["spec"]
    plan = Plan(Channel(W=spec.W, H=spec.H, N=N, R=R, max_frames=spec.F, **modes))
    n = plan.info["n_sub"]
    dev = "cuda:0"
    frames = torch.from_numpy(tio["burst"]["frames"]).to(dev)
    stf = torch.from_numpy(tio["stf"]).to(dev)
    ws, lay = plan.workspace(spec.F, n)
    out = torch.zeros((spec.H, spec.W), device=dev)
    valid = torch.zeros((spec.H, spec.W), dtype=torch.uint8, device=dev)
    plan.reconstruct(frames, spec.F, stf, n, ws, lay, out, valid)
    torch.cuda.synchronize()
    v = plan.views(ws, lay, spec.F, n)
    idx = plan.pair_index(OP.used_pairs(N, R, CS.FC))
    res = {s: {"P": v["P"][s].cpu().numpy(), "B": v["B"][s].cpu().numpy()[idx], "rec": v["rec"][s].cpu().numpy()}
           for s in tio["pick"]}
    res["out"] = out.cpu().numpy()
    res["K"] = plan.info["K"]
    del ws, v
    torch.cuda.empty_cache()
    return res


def _errors(tio, g):
    K = g["K"]
    eP = eB = eI = 0.0
    for s in tio["pick"]:
        o = tio["oracle"][s]
        Pref = o["P"][N // 2:N // 2 + K + 1, N // 2 - K:N // 2 + K + 1]
        eP = max(eP, CS.rel_l2(g[s]["P"][:, :2 * K + 1], Pref))
        w = np.abs(o["B"]) ** 2
        dphi = np.angle(g[s]["B"].astype(np.complex128) * np.conj(o["B"]))
        eB = max(eB, float(np.sqrt(np.sum(w * dphi ** 2) / np.sum(w))))
        x0, y0, ww, hh = tio["subs"][s]
        eI = max(eI, CS.rel_l2(g[s]["rec"][:hh, :ww], o["rec"][:hh, :ww]))
    spec, subs, pick = tio["spec"], tio["subs"], tio["pick"]
    cover_all = np.zeros((spec.H, spec.W), np.int32)
    cover_pick = np.zeros((spec.H, spec.W), np.int32)
    for s, (x0, y0, ww, hh) in enumerate(subs):
        cover_all[y0:y0 + hh, x0:x0 + ww] += 1
        if s in pick:
            cover_pick[y0:y0 + hh, x0:x0 + ww] += 1
    ref, ref_valid = O.mosaic([tio["oracle"][s]["rec"] for s in pick], [subs[s] for s in pick], spec.W, spec.H,
                              TAPER)
    region = (cover_all == cover_pick) & (cover_pick > 0) & ref_valid
    eM = CS.rel_l2(g["out"][region], ref[region])
    return eP, eB, eI, eM


def _mode_name(m):
    from paper_1701_00581_gb300 import SM_ACC_KAHAN, SM_BF16, SM_FP16, SM_PHASE_FF, SM_PHASE_FP64
    return (f"spectra {dict([(0, 'FP32'), (SM_FP16, 'FP16'), (SM_BF16, 'BF16')])[m.get('spectra_prec', 0)]}, "
            f"sums {'Kahan' if m.get('acc_mode') == SM_ACC_KAHAN else 'plain'}, "
            f"recursion {dict([(0, 'FP32'), (SM_PHASE_FP64, 'FP64'), (SM_PHASE_FF, 'float-float')])[m.get('phase_prec', 0)]}")


def _modes():
    from paper_1701_00581_gb300 import SM_ACC_KAHAN, SM_BF16, SM_FP16, SM_PHASE_FF, SM_PHASE_FP64
    # (modes, (P gate, bispectrum phase gate in rad, sub-image gate))
    return [({}, (1e-4, 1e-4, 1e-3)), (dict(spectra_prec=SM_FP16), (1e-3, 1e-3, 1e-3)),
            (dict(spectra_prec=SM_BF16), (1e-2, 1e-2, 2e-3)),
            (dict(acc_mode=SM_ACC_KAHAN), (1e-4, 1e-4, 1e-3)), (dict(phase_prec=SM_PHASE_FP64), (1e-4, 1e-4, 1e-3)),
            (dict(spectra_prec=SM_FP16, acc_mode=SM_ACC_KAHAN, phase_prec=SM_PHASE_FP64), (1e-3, 1e-3, 1e-3)),
            (dict(spectra_prec=SM_BF16, acc_mode=SM_ACC_KAHAN, phase_prec=SM_PHASE_FP64), (1e-2, 1e-2, 2e-3)),
            (dict(phase_prec=SM_PHASE_FF), (1e-4, 1e-4, 1e-3)),
            (dict(spectra_prec=SM_FP16, phase_prec=SM_PHASE_FF), (1e-3, 1e-3, 1e-3))]


@pytest.mark.parametrize("k", range(9))
def test_precision_mode_on_the_tio_burst(torch, tio, k):
    modes, (gP, gB, gI) = _modes()[k]
    eP, eB, eI, eM = _errors(tio, _gpu(torch, tio, **modes))
    line = (f"{_mode_name(modes)}: P rel L2 {eP:.3e}, bispectrum phase RMS {eB:.3e} rad, "
            f"sub-image rel L2 {eI:.3e}, mosaic rel L2 {eM:.3e}\n")
    report = os.environ.get("SPECKLE_REPORT_DIR")
    if report:
        with open(os.path.join(report, "precision_tio.txt"), "a") as f:
            f.write(line)
    print(line)
    assert eP < gP
    assert eB < gB
    assert eM < IMG_TOL
    assert eI < gI
