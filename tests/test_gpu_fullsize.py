"""Parity at the full workload sizes, in the launch configuration bench.py
times (every subfield of the burst in one chunk), on sampled outputs the
FP64 oracle computes one by one.

* 2560x2160x100 TiO-shaped burst, 304 subfields of 256^2 (19 of them
  256x240): spectra of sampled frames, P / M / noise and the modulus of
  sampled subfields, the bispectrum on seeded random pairs, and for one
  ragged edge subfield the whole recursion and sub-image; the valid mask of
  the whole mosaic.
* 1024x1024x100 H-alpha-shaped burst, 225 subfields of 128^2: two whole
  subfields end to end.
"""
import numpy as np
import pytest

from oracle import speckle_oracle as O

from . import _cases as CS

pytestmark = pytest.mark.gpu

SPEC_TOL = 1e-4
IMG_TOL = 1e-3


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_00581_gb300 import build
    build.build()
    return t


def _run(torch, name, N, R):
    """Generate the burst on the GPU, run every stage over all subfields in
    one chunk (as bench.py does); return device views plus host inputs."""
    from paper_1701_00581_gb300 import Channel, Plan
    from synth import CONFIGS, make_burst
    spec = CONFIGS[name]
    b = make_burst(spec, channel=1, burst=0, device="cuda:0")
    plan = Plan(Channel(W=spec.W, H=spec.H, N=N, R=R, max_frames=spec.F))
    n = plan.info["n_sub"]
    stf = plan.model_stf(b["d_over_r0"])
    dev = "cuda:0"
    frames = torch.from_numpy(b["frames"]).to(dev)
    stf_d = torch.from_numpy(stf).to(dev)
    ws, lay = plan.workspace(spec.F, n)
    out = torch.zeros((spec.H, spec.W), device=dev)
    valid = torch.zeros((spec.H, spec.W), dtype=torch.uint8, device=dev)
    plan.reconstruct(frames, spec.F, stf_d, n, ws, lay, out, valid)
    torch.cuda.synchronize()
    return {"plan": plan, "burst": b, "views": plan.views(ws, lay, spec.F, n), "out": out,
            "valid": valid, "ws": ws, "spec": spec}


def _half_box(plan, grid):
    N, K = plan.info["N"], plan.info["K"]
    return grid[N // 2:N // 2 + K + 1, N // 2 - K:N // 2 + K + 1]


@pytest.fixture(scope="module")
def tio(torch):
    return _run(torch, "tio2560", 256, 24)


def test_tio_spectra_and_statistics_sampled(tio):
    plan, b, v = tio["plan"], tio["burst"], tio["views"]
    N, K, R = 256, plan.info["K"], 24
    subs = plan.subfields()
    iy, ix = CS.box_to_grid_index(N, K, R)
    stf_o = O.stf_model(N, CS.FC, b["d_over_r0"])
    for s in (0, 150, 295, 303):
        sub = tuple(int(t) for t in subs[s])
        In, flux, mu = O.frame_spectra(b["frames"], sub, N, N // 8)
        for f in (0, 57, 99):
            got = v["spec"][s, f].cpu().numpy()[:, :2 * K + 1]
            assert CS.rel_l2(got, In[f][iy][:, ix]) < SPEC_TOL
        assert CS.rel_l2(v["flux"][s].cpu().numpy(), flux) < 1e-6
        P, M = O.power_mean(In)
        noise = O.noise_floor(P, N, CS.FC)
        assert CS.rel_l2(v["P"][s].cpu().numpy()[:, :2 * K + 1], _half_box(plan, P)) < SPEC_TOL
        assert CS.rel_l2(v["M"][s].cpu().numpy()[:, :2 * K + 1], _half_box(plan, M)) < SPEC_TOL
        assert abs(float(v["noise"][s]) - noise) <= SPEC_TOL * noise
        A = O.amplitude(P, noise, stf_o, N, CS.FC)
        assert CS.rel_l2(v["A"][s].cpu().numpy()[:, :2 * K + 1], _half_box(plan, A)) < SPEC_TOL


def test_tio_bispectrum_sampled_pairs(tio):
    plan, b, v = tio["plan"], tio["burst"], tio["views"]
    wv = CS.used_pairs(256, 24)
    rng = np.random.default_rng(2017)
    pick = wv[rng.choice(len(wv), 20000, replace=False)]
    idx = plan.pair_index(pick)
    assert np.all(idx >= 0)
    subs = plan.subfields()
    for s in (150, 303):
        In, _, _ = O.frame_spectra(b["frames"], tuple(int(t) for t in subs[s]), 256, 32)
        ref = CS.oracle_B_used(In, pick)
        got = v["B"][s].cpu().numpy()[idx]
        assert CS.rel_l2(got, ref) < SPEC_TOL


def test_tio_edge_subfield_end_to_end(tio):
    """Whole recursion and sub-image of the bottom-right 256x240 subfield."""
    plan, b, v = tio["plan"], tio["burst"], tio["views"]
    N, R, K = 256, 24, plan.info["K"]
    s = plan.info["n_sub"] - 1
    sub = tuple(int(t) for t in plan.subfields()[s])
    assert sub[3] == 240
    In, flux, mu = O.frame_spectra(b["frames"], sub, N, N // 8)
    P, M = O.power_mean(In)
    noise = O.noise_floor(P, N, CS.FC)
    A = O.amplitude(P, noise, O.stf_model(N, CS.FC, b["d_over_r0"]), N, CS.FC)
    # the recursion reads exactly the used pairs; give the oracle those, in
    # its own (u in the upper half plane) representation
    wv = CS.used_pairs(N, R)
    u = wv[:, :2] - wv[:, 2:]
    up = O.in_half_plane(u[:, 0], u[:, 1])
    pairs = np.where(up[:, None], np.concatenate([u, wv[:, 2:]], 1), -np.concatenate([u, wv[:, 2:]], 1))
    B = O.bispectrum(In, pairs)
    z = O.phase_recursion(B, pairs, M, N, CS.FC, R)
    rec = O.inverse(A, z, float(flux.mean()), float(mu.mean()), O.window2d(sub[2], sub[3], N // 8))
    Ah = _half_box(plan, A)
    zg = v["z"][s].cpu().numpy()[:, :2 * K + 1]
    m = Ah > 0
    assert CS.rel_l2((Ah * zg)[m], (Ah * _half_box(plan, z))[m]) < IMG_TOL
    got = v["rec"][s].cpu().numpy()[:sub[3], :sub[2]]
    assert CS.rel_l2(got, rec[:sub[3], :sub[2]]) < IMG_TOL


def test_tio_mosaic_valid_mask_and_values(tio):
    plan, spec = tio["plan"], tio["spec"]
    subs = [tuple(int(t) for t in s) for s in plan.subfields()]
    zeros = [np.zeros((256, 256))] * len(subs)
    _, valid_o = O.mosaic(zeros, subs, spec.W, spec.H, 32)
    valid_g = tio["valid"].cpu().numpy().astype(bool)
    assert np.array_equal(valid_g, valid_o)
    out = tio["out"].cpu().numpy()
    assert np.all(np.isfinite(out)) and np.all(out[~valid_g] == 0)
    # where one subfield alone covers a pixel, out = rec_s / window_s there
    rec0 = tio["views"]["rec"][0].cpu().numpy()
    win0 = O.window2d(256, 256, 32)
    y, x = 20, 20
    assert out[y, x] == pytest.approx(rec0[y, x] / win0[y, x], rel=1e-5)


def test_halpha_whole_subfields(torch):
    r = _run(torch, "halpha1024", 128, 16)
    plan, b, v = r["plan"], r["burst"], r["views"]
    N, R, K = 128, 16, plan.info["K"]
    stf_o = O.stf_model(N, CS.FC, b["d_over_r0"])
    wv = CS.used_pairs(N, R)
    idx = plan.pair_index(wv)
    subs = plan.subfields()
    for s in (0, 112):
        sub = tuple(int(t) for t in subs[s])
        o = O.reconstruct_subfield(b["frames"], sub, N, CS.FC, R, N // 8, stf_o)
        assert CS.rel_l2(v["P"][s].cpu().numpy()[:, :2 * K + 1], _half_box(plan, o["P"])) < SPEC_TOL
        Bg = v["B"][s].cpu().numpy()[idx]
        assert CS.rel_l2(Bg, CS.oracle_B_used(o["In"], wv)) < SPEC_TOL
        assert CS.rel_l2(v["rec"][s].cpu().numpy(), o["rec"]) < IMG_TOL


def test_tio_seeing_on_the_80_cubes(tio, torch):
    """Sect. 3.1: the 2560 x 2160 burst's 80 non-overlapping 256^2 cubes,
    each cube's fitted D/r0 against the oracle fit on the same statistics."""
    from oracle import speckle_oracle as O
    from .test_gpu_seeing import FIT_TOL, oracle_fit_on_gpu_stats
    plan, v, spec = tio["plan"], tio["views"], tio["spec"]
    n = plan.info["n_sub"]
    lay = plan.layout(spec.F, n)
    assert plan.info["n_cubes"] == 80
    assert plan.cubes().tolist() == O.seeing_cubes(spec.W, spec.H, 256, 128)
    plan.stage_seeing(spec.F, 0, n, tio["ws"], lay)
    plan.stage_seeing_stf(tio["ws"], lay)
    torch.cuda.synchronize()
    seeing = v["seeing"].cpu().numpy()
    xs = np.array([oracle_fit_on_gpu_stats(plan, v, spec.F, c, int(c)) for c in plan.cubes()])
    assert np.allclose(seeing[:80], xs, rtol=FIT_TOL, atol=0)
    assert seeing[80] == pytest.approx(1.0 / np.mean(1.0 / xs), rel=FIT_TOL)
    # the estimate tracks the burst's seeing (D/r0 drawn in 8..15 per frame)
    assert 5.0 < seeing[80] < 20.0
