"""GPU parity: every stage of the CUDA path, through the C ABI, against the
FP64 oracle on the same seeded inputs.

Tolerances: accumulated spectra (P, M, B) and the modulus within 1e-4
relative L2 per subfield; sub-images and the mosaic within 1e-3 relative L2
(over the valid mask); integer and index outputs (subfield grid, pair
positions, valid mask) exact.
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


@pytest.fixture(scope="module")
def ragged(torch):
    from paper_1701_00581_gb300 import Plan
    plan = Plan(CS.gpu_channel("ragged"))
    b = CS.burst("ragged")
    return plan, CS.gpu_run(plan, b["frames"], b["stf_emp"]), CS.oracle_run("ragged")


def _half_box(plan, grid):
    """Oracle centred grid -> half-box [K+1][2K+1] (ky = 0..K, kx = -K..K)."""
    N, K = plan.info["N"], plan.info["K"]
    return grid[N // 2:N // 2 + K + 1, N // 2 - K:N // 2 + K + 1]


def test_plan_matches_oracle_domains(torch):
    from paper_1701_00581_gb300 import Plan
    for name in ("ragged", "sub64"):
        c = CS.case(name)
        plan = Plan(CS.gpu_channel(name))
        sp = c["spec"]
        subs = O.subfield_grid(sp.W, sp.H, c["N"], c["stride"])
        assert plan.subfields().tolist() == [list(s) for s in subs]
        assert plan.info["n_U"] == len(O.domain_U(c["N"], CS.FC))
        assert plan.info["n_V"] == len(O.domain_V(c["R"]))
        assert plan.info["n_pairs"] == len(CS.used_pairs(c["N"], c["R"]))
        rings = O.recursion_rings(c["N"], CS.FC)
        assert plan.info["n_rings"] == len(rings)
        assert plan.info["n_points"] == sum(len(r) for r in rings)


def test_plan_full_size_domains(torch):
    from paper_1701_00581_gb300 import Channel, Plan
    for (W, H, N, R, nsub, npairs) in ((1024, 1024, 128, 16, 225, None), (2560, 2160, 256, 24, 304, None)):
        plan = Plan(Channel(W=W, H=H, N=N, R=R))
        assert plan.info["n_sub"] == nsub
        assert plan.info["n_pairs"] == len(CS.used_pairs(N, R))
        assert plan.info["n_rings"] == len(O.recursion_rings(N, CS.FC))
        assert plan.subfields().tolist() == [list(s) for s in O.subfield_grid(W, H, N, N // 2)]


def test_pair_index_is_a_bijection_on_used_pairs(ragged):
    plan, _, _ = ragged
    wv = CS.used_pairs(64, 8)
    idx = plan.pair_index(wv)
    assert np.all(idx >= 0)
    assert len(np.unique(idx)) == len(idx)
    assert idx.max() < plan.info["n_tiles"] * plan.info["tile_pairs"]
    bad = np.array([[3, 2, 0, 0], [5, 5, 9, 0], [-3, 0, 1, 0], [1, 1, 2, 0], [30, 30, 1, 1]])
    assert np.all(plan.pair_index(bad) == -1)


def test_spectra_parity(ragged):
    plan, g, o = ragged
    N, K, R = 64, plan.info["K"], 8
    iy, ix = CS.box_to_grid_index(N, K, R)
    for s, res in o["sub"].items():
        ref = res["In"][:, iy][:, :, ix]
        got = g["spec"][s][:, :, :2 * K + 1]
        assert CS.rel_l2(got, ref) < SPEC_TOL
        assert CS.rel_l2(g["flux"][s], res["flux"]) < 1e-6
        assert CS.rel_l2(g["mu"][s], res["mu"]) < 1e-6


def test_power_mean_noise_parity(ragged):
    plan, g, o = ragged
    K = plan.info["K"]
    for s, res in o["sub"].items():
        assert CS.rel_l2(g["P"][s][:, :2 * K + 1], _half_box(plan, res["P"])) < SPEC_TOL
        assert CS.rel_l2(g["M"][s][:, :2 * K + 1], _half_box(plan, res["M"])) < SPEC_TOL
        assert abs(g["noise"][s] - res["noise"]) <= SPEC_TOL * res["noise"]


def test_bispectrum_parity(ragged):
    plan, g, o = ragged
    wv = CS.used_pairs(64, 8)
    idx = plan.pair_index(wv)
    for s, res in o["sub"].items():
        ref = CS.oracle_B_used(res["In"], wv)
        assert CS.rel_l2(g["B"][s][idx], ref) < SPEC_TOL


def test_amplitude_parity(ragged):
    plan, g, o = ragged
    K = plan.info["K"]
    for s, res in o["sub"].items():
        assert CS.rel_l2(g["A"][s][:, :2 * K + 1], _half_box(plan, res["A"])) < SPEC_TOL


def test_phase_parity_weighted_by_modulus(ragged):
    plan, g, o = ragged
    K = plan.info["K"]
    for s, res in o["sub"].items():
        A = _half_box(plan, res["A"])
        zo = _half_box(plan, res["z"])
        zg = g["z"][s][:, :2 * K + 1]
        m = A > 0
        assert CS.rel_l2((A * zg)[m], (A * zo)[m]) < IMG_TOL


def test_subimage_and_mosaic_parity(ragged):
    plan, g, o = ragged
    for s, res in o["sub"].items():
        x0, y0, w, h = o["subs"][s]
        assert CS.rel_l2(g["rec"][s][:h, :w], res["rec"][:h, :w]) < IMG_TOL
    assert np.array_equal(g["valid"], o["valid"])
    v = o["valid"]
    assert CS.rel_l2(g["out"][v], o["out"][v]) < IMG_TOL
    assert np.all(g["out"][~v] == 0)


def test_whole_path_entry_single_subfield(torch):
    """sm_reconstruct on the 64x64, 100-frame float32 workload."""
    from paper_1701_00581_gb300 import Plan
    plan = Plan(CS.gpu_channel("sub64"))
    b = CS.burst("sub64")
    o = CS.oracle_run("sub64")
    dev = "cuda:0"
    frames = torch.from_numpy(b["frames"]).to(dev)
    stf = torch.from_numpy(b["stf_emp"]).to(dev)
    ws, lay = plan.workspace(100, 1)
    out = torch.zeros((64, 64), device=dev)
    valid = torch.zeros((64, 64), dtype=torch.uint8, device=dev)
    plan.reconstruct(frames, 100, stf, 1, ws, lay, out, valid)
    torch.cuda.synchronize()
    v = o["valid"]
    assert np.array_equal(valid.cpu().numpy().astype(bool), v)
    assert CS.rel_l2(out.cpu().numpy()[v], o["out"][v]) < IMG_TOL
    # accumulated spectra of the same run
    K = plan.info["K"]
    vw = plan.views(ws, lay, 100, 1)
    res = o["sub"][0]
    assert CS.rel_l2(vw["P"][0].cpu().numpy()[:, :2 * K + 1], _half_box(plan, res["P"])) < SPEC_TOL
    wv = CS.used_pairs(64, 8)
    Bg = vw["B"][0].cpu().numpy()[plan.pair_index(wv)]
    assert CS.rel_l2(Bg, CS.oracle_B_used(res["In"], wv)) < SPEC_TOL


def test_chunking_and_repeat_are_bitwise_stable(torch, ragged):
    plan, g, _ = ragged
    b = CS.burst("ragged")
    g5 = CS.gpu_run(plan, b["frames"], b["stf_emp"], chunk=5)
    g5b = CS.gpu_run(plan, b["frames"], b["stf_emp"], chunk=5)
    assert np.array_equal(g5["out"], g["out"])
    assert np.array_equal(g5b["out"], g5["out"])
    assert np.array_equal(g5["rec"], g["rec"])


def test_constant_frames_degenerate(torch):
    """Flat frames: after the mean is removed every spectrum is (to rounding)
    zero off DC, so the modulus vanishes and the mosaic returns the constant."""
    from paper_1701_00581_gb300 import Plan
    plan = Plan(CS.gpu_channel("ragged"))
    frames = np.full((8, 110, 150), 1000, dtype=np.uint16)
    g = CS.gpu_run(plan, frames, CS.burst("ragged")["stf_emp"])
    v = g["valid"]
    assert v.mean() > 0.8
    assert np.max(np.abs(g["out"][v] - 1000.0)) < 1e-2
    K = plan.info["K"]
    A = g["A"][:, :, :2 * K + 1].copy()
    A[:, 0, K] = 0.0                  # DC is defined as 1
    assert np.max(A) < 1e-4
    assert np.all(np.isfinite(g["z"][:, :, :2 * K + 1][A > 0]))


def test_single_noise_free_frame_recovers_phases(torch):
    """One seeing-free, noise-free frame: the recursion returns the frame's own phases."""
    from paper_1701_00581_gb300 import Channel, Plan
    from synth import burst as S
    spec = S.BurstSpec(W=64, H=64, F=1, N=64, dr0=(1.0, 1.0), counts=False)
    b = S.make_burst(spec, channel=3, psf="diffraction", noise=False)
    plan = Plan(Channel(W=64, H=64, N=64, R=8, stride=32, taper=8, max_frames=1))
    g = CS.gpu_run(plan, b["frames"], np.ones((64, 64)))
    In, _, _ = O.frame_spectra(b["frames"].astype(np.float64), (0, 0, 64, 64), 64, 8)
    K = plan.info["K"]
    ref = _half_box(plan, In[0])
    zg = g["z"][0][:, :2 * K + 1]
    T0 = _half_box(plan, O.otf_t0(64, CS.FC))
    m = (T0 > 0) & (np.abs(ref) > 1e-4)
    m[0, :K + 1] = False
    assert np.max(np.abs(zg[m] - ref[m] / np.abs(ref[m]))) < 1e-3


def test_invalid_stage_arguments_fail_cleanly(ragged):
    from paper_1701_00581_gb300 import SpeckleError
    plan, _, _ = ragged
    ws, lay = plan.workspace(8, 2)
    with pytest.raises(SpeckleError):
        plan.stage_stats(8, plan.info["n_sub"] + 1, ws, lay)
    with pytest.raises(SpeckleError):
        plan.stage_inverse(8, plan.info["n_sub"] - 1, 2, ws, lay)
    with pytest.raises(SpeckleError):
        plan.layout(plan.ch.max_frames + 1, 1)
    with pytest.raises(SpeckleError):
        plan.stage_amplitude(1, None, ws, lay)


@pytest.mark.parametrize("name,kw", [("unit_weights", dict(phase_weight=1)),
                                     ("snr_weights", dict(phase_weight=2)),
                                     ("least_squares_5", dict(phase_iters=5)),
                                     ("least_squares_snr_3", dict(phase_weight=2, phase_iters=3)),
                                     ("overlap75", dict(stride=16)),
                                     ("chain_R1", dict(R=1))])
def test_method_variants_match_oracle(torch, name, kw):
    """Unit-modulus and SNR-weighted phase terms, least-squares sweeps after
    the recursion, a 75 % overlap grid (stride N/4, as in the paper's own
    1110-cube layout) and R = 1 (single-path recursion), each against the
    oracle run with the same parameters."""
    from paper_1701_00581_gb300 import Channel, Plan
    c = CS.case("ragged")
    sp = c["spec"]
    stride = kw.get("stride", c["stride"])
    R = kw.get("R", c["R"])
    weight = kw.get("phase_weight", O.W_BISPEC)
    iters = kw.get("phase_iters", 0)
    plan = Plan(Channel(W=sp.W, H=sp.H, N=c["N"], R=R, stride=stride, fc=CS.FC, taper=c["taper"],
                        phase_weight=weight, phase_iters=iters, max_frames=sp.F))
    b = CS.burst("ragged")
    g = CS.gpu_run(plan, b["frames"], b["stf_emp"])
    o = O.reconstruct_burst(b["frames"], c["N"], stride, CS.FC, R, c["taper"], b["stf_emp"], weight,
                            iters=iters)
    if iters:
        # the sweeps sum in a fixed order: a second run is bitwise equal
        g2 = CS.gpu_run(plan, b["frames"], b["stf_emp"])
        assert np.array_equal(g2["z"], g["z"]) and np.array_equal(g2["out"], g["out"])
    assert plan.info["n_sub"] == len(o["subs"])
    wv = CS.used_pairs(c["N"], R)
    idx = plan.pair_index(wv)
    for s in (0, len(o["subs"]) - 1):
        assert CS.rel_l2(g["B"][s][idx], CS.oracle_B_used(o["sub"][s]["In"], wv)) < SPEC_TOL
    v = o["valid"]
    assert np.array_equal(g["valid"], v)
    assert CS.rel_l2(g["out"][v], o["out"][v]) < IMG_TOL


def test_odd_R_at_256_matches_oracle(torch):
    """N = 256 with an odd offset radius (R = 9): the offset-block grid then
    starts at -R and the offsets move in 16-byte chunks (the box centre
    column K = 73 is odd), unlike the even-R and N = 64 cases above.  Two
    subfields, the second ragged (172 px wide), 4 uint16 frames."""
    from paper_1701_00581_gb300 import Channel, Plan
    from synth import burst as S
    spec = S.BurstSpec(W=300, H=256, F=4, N=256, dr0=(5.0, 9.0), counts=True)
    b = S.make_burst(spec, channel=11, burst=0)
    N, R, stride, taper = 256, 9, 128, 16
    plan = Plan(Channel(W=spec.W, H=spec.H, N=N, R=R, stride=stride, fc=CS.FC, taper=taper, max_frames=spec.F))
    g = CS.gpu_run(plan, b["frames"], b["stf_emp"])
    o = O.reconstruct_burst(b["frames"], N, stride, CS.FC, R, taper, b["stf_emp"])
    assert plan.info["n_sub"] == len(o["subs"]) == 2
    wv = CS.used_pairs(N, R)
    idx = plan.pair_index(wv)
    assert (idx >= 0).all()
    for s in range(2):
        assert CS.rel_l2(g["B"][s][idx], CS.oracle_B_used(o["sub"][s]["In"], wv)) < SPEC_TOL
    v = o["valid"]
    assert np.array_equal(g["valid"], v)
    assert CS.rel_l2(g["out"][v], o["out"][v]) < IMG_TOL


def test_paper_layout_matches_oracle(torch):
    """The paper's own layout: full tiles only at stride N/4, merged by
    their central stride x stride blocks (Sect. 3.2)."""
    from paper_1701_00581_gb300 import SM_EDGE_DROP, SM_MOSAIC_CENTRAL, Channel, Plan
    c = CS.case("ragged")
    sp = c["spec"]
    N, stride = c["N"], c["N"] // 4
    plan = Plan(Channel(W=sp.W, H=sp.H, N=N, R=c["R"], stride=stride, fc=CS.FC, taper=c["taper"],
                        max_frames=sp.F, edge_mode=SM_EDGE_DROP, mosaic_mode=SM_MOSAIC_CENTRAL))
    b = CS.burst("ragged")
    g = CS.gpu_run(plan, b["frames"], b["stf_emp"])
    o = O.reconstruct_burst(b["frames"], N, stride, CS.FC, c["R"], c["taper"], b["stf_emp"], paper_layout=True)
    assert plan.subfields().tolist() == [list(s) for s in o["subs"]]
    assert np.array_equal(g["valid"], o["valid"])
    v = o["valid"]
    assert v.sum() == (len(set(s[0] for s in o["subs"])) * stride) * (len(set(s[1] for s in o["subs"])) * stride)
    assert CS.rel_l2(g["out"][v], o["out"][v]) < IMG_TOL
    assert np.all(g["out"][~v] == 0)


def test_paper_layout_plan_of_the_tio_burst(torch):
    from paper_1701_00581_gb300 import SM_EDGE_DROP, SM_MOSAIC_CENTRAL, Channel, Plan, SpeckleError
    plan = Plan(Channel(W=2560, H=2160, N=256, R=24, stride=64, edge_mode=SM_EDGE_DROP,
                        mosaic_mode=SM_MOSAIC_CENTRAL))
    assert plan.info["n_sub"] == 1110 and plan.info["nsx"] == 37 and plan.info["nsy"] == 30
    assert plan.info["n_cubes"] == 80
    with pytest.raises(SpeckleError):          # the central mosaic needs full tiles
        Plan(Channel(W=2560, H=2160, N=256, R=24, stride=64, mosaic_mode=SM_MOSAIC_CENTRAL))
