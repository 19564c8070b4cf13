"""Front end on the GPU (Table 2: flat/dark preprocessing) against the oracle."""
import numpy as np
import pytest

from oracle import speckle_oracle as O

from . import _cases as CS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_00581_gb300 import build
    build.build()
    return t


def _detector(H, W, seed=31):
    rng = np.random.default_rng(seed)
    dark = rng.uniform(50.0, 80.0, (H, W)).astype(np.float32)
    g = rng.uniform(0.7, 1.3, (H, W))
    flat = (dark + 1500.0 * g).astype(np.float32)
    flat[5, 9] = dark[5, 9]                   # a dead pixel
    return dark, flat, g


@pytest.mark.parametrize("frame_type", ["u16", "f32"])
def test_flat_dark_matches_oracle_and_feeds_the_path(torch, frame_type):
    from paper_1701_00581_gb300 import Plan
    plan = Plan(CS.gpu_channel("ragged"))
    b = CS.burst("ragged")
    scene = b["frames"].astype(np.float64)
    F, H, W = scene.shape
    dark, flat, g = _detector(H, W)
    raw = dark[None] + scene * g[None]
    raw = np.clip(np.rint(raw), 0, 65535).astype(np.uint16) if frame_type == "u16" else raw.astype(np.float32)
    dev = "cuda:0"
    d_flat, d_dark = torch.from_numpy(flat).to(dev), torch.from_numpy(dark).to(dev)
    d_gain = torch.empty((H, W), dtype=torch.float32, device=dev)
    plan.stage_gain(d_flat, d_dark, d_gain)
    d_raw = torch.from_numpy(raw).to(dev)
    d_cal = torch.empty((F, H, W), dtype=torch.float32, device=dev)
    plan.stage_calibrate(d_raw, F, d_dark, d_gain, d_cal)
    torch.cuda.synchronize()
    gain = d_gain.cpu().numpy()
    gref = O.calib_gain(flat, dark)
    assert gain[5, 9] == 0.0
    assert np.allclose(gain, gref, rtol=2e-7, atol=0)
    cal = d_cal.cpu().numpy()
    cref = O.calibrate(raw, dark, gain.astype(np.float64))      # the kernel alone, on the GPU's gain
    assert np.allclose(cal, cref, rtol=1e-6, atol=1e-6 * np.abs(cref).max())
    assert np.all(cal[:, 5, 9] == 0.0)
    # calibrated frames through the whole path (F32 frames) against the oracle's
    gpu = CS.gpu_run(plan, cal, b["stf_emp"])
    c = CS.case("ragged")
    o = O.reconstruct_burst(cref, c["N"], c["stride"], CS.FC, c["R"], c["taper"], b["stf_emp"])
    v = o["valid"]
    assert np.array_equal(gpu["valid"], v)
    assert CS.rel_l2(gpu["out"][v], o["out"][v]) < 1e-3


def test_front_end_errors(torch):
    from paper_1701_00581_gb300 import Plan, SpeckleError
    plan = Plan(CS.gpu_channel("ragged"))
    H, W = plan.ch.H, plan.ch.W
    x = torch.zeros((2, H, W), dtype=torch.float32, device="cuda:0")
    d = torch.zeros((H, W), dtype=torch.float32, device="cuda:0")
    with pytest.raises(SpeckleError):
        plan.stage_calibrate(x, 2, d, d, x)            # out aliases raw


def test_photon_bias_removal_matches_oracle(torch):
    """photon_gain = 0.1 photons per count (~8e5 photons per 64^2 tile), so
    the correction moves B well beyond the parity tolerance; GPU against the
    oracle's corrected bispectrum and image."""
    from paper_1701_00581_gb300 import Plan
    gain = 0.1
    plan = Plan(CS.gpu_channel("ragged", photon_gain=gain))
    b = CS.burst("ragged")
    g = CS.gpu_run(plan, b["frames"], b["stf_emp"])
    c = CS.case("ragged")
    o = O.reconstruct_burst(b["frames"], c["N"], c["stride"], CS.FC, c["R"], c["taper"], b["stf_emp"],
                            photon_gain=gain)
    o0 = CS.oracle_run("ragged")
    wv = CS.used_pairs(64, 8)
    idx = plan.pair_index(wv)
    pairs_u = np.stack([wv[:, 0] - wv[:, 2], wv[:, 1] - wv[:, 3], wv[:, 2], wv[:, 3]], axis=1)
    for s in (0, plan.info["n_sub"] - 1):
        res = o["sub"][s]
        a1, a2 = O.photon_terms(res["flux"], gain)
        ref = O.bispectrum_unbiased(CS.oracle_B_used(res["In"], wv), pairs_u, res["P"], a1, a2)
        raw = CS.oracle_B_used(o0["sub"][s]["In"], wv)
        assert CS.rel_l2(ref, raw) > 1e-3                          # the correction matters here
        assert CS.rel_l2(g["B"][s][idx], ref) < 1e-4
    v = o["valid"]
    assert np.array_equal(g["valid"], v)
    assert CS.rel_l2(g["out"][v], o["out"][v]) < 1e-3


@pytest.mark.parametrize("frame_type", ["u16", "f32"])
def test_correlation_tracking_matches_oracle(torch, frame_type):
    """Frames cut from one scene at known integer offsets: the GPU finds the
    oracle's shifts (exactly), its correlation surface to 1e-3 of the peak,
    and shifts the frames to the oracle's aligned frames (exactly: copies of
    samples)."""
    from paper_1701_00581_gb300 import Channel, Plan
    from synth import burst as S
    rng = np.random.default_rng(52)
    big = S.make_object(360, 300, rng) * 2000.0
    H, W, G, Sr = 200, 256, 128, 12
    offs = [(0, 0), (5, -3), (-12, 7), (9, 12), (-7, -11), (12, -12), (0, 4), (-3, 0)]
    frames = np.stack([big[40 + dy:40 + dy + H, 40 + dx:40 + dx + W] for dx, dy in offs])
    frames = np.rint(frames).astype(np.uint16) if frame_type == "u16" else frames.astype(np.float32)
    F = len(offs)
    plan = Plan(Channel(W=W, H=H, N=64, R=8, max_frames=F))
    dev = "cuda:0"
    d_frames = torch.from_numpy(frames).to(dev)
    rwin = torch.empty((G, G), dtype=torch.float32, device=dev)
    cc = torch.empty((F, 2 * Sr + 1, 2 * Sr + 1), dtype=torch.float64, device=dev)
    shifts = torch.empty((F, 2), dtype=torch.int32, device=dev)
    plan.stage_track(d_frames, F, 0, G, Sr, rwin, cc, shifts)
    out = torch.empty((F, H, W), dtype=torch.float32, device=dev)
    plan.stage_shift(d_frames, F, shifts, out)
    torch.cuda.synchronize()
    sh_ref, C_ref = O.track_shifts(frames, 0, G, Sr)
    assert shifts.cpu().numpy().tolist() == sh_ref.tolist() == [[-dx, -dy] for dx, dy in offs]
    # FP32 products of ~2000-count samples with the zero-mean reference cancel
    # ~1600-fold in each sum, so the surface agrees to ~1e-4 of its peak; the
    # integer decision is exact because the peaks stand far above that
    assert np.allclose(cc.cpu().numpy(), C_ref, rtol=0, atol=1e-3 * np.abs(C_ref).max())
    al = O.apply_shifts(frames, sh_ref)
    assert np.array_equal(out.cpu().numpy().astype(np.float64), al)
    from paper_1701_00581_gb300 import SpeckleError
    with pytest.raises(SpeckleError):
        plan.stage_track(d_frames, F, 0, 240, Sr, rwin, cc, shifts)       # window + search exceed the frame
