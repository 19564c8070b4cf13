"""Batched persistent launch (sm_batch_*) on the GPU.

Four bursts of different channels -- subfields of 64^2 (ragged edges), 64^2
float32 frames, 256^2 with a ragged 172-px tile and 128^2 with ragged
edges; uint16 and float32 frames; the STF given or the seeing estimated --
share one persistent spectra + bispectrum launch.  Each burst's result is
bitwise the same as that burst alone in a batch, and matches the FP64
oracle: P, M and B at every used pair at 1e-4 per subfield, the image at
1e-3 over the valid mask.
"""
import numpy as np
import pytest

from oracle import speckle_oracle as O
from synth import burst as S

from . import _cases as CS

pytestmark = pytest.mark.gpu

SPEC_TOL = 1e-4
IMG_TOL = 1e-3

# name: (spec, N, R, STF given?)
CASES = {
    "ragged64": (S.BurstSpec(W=150, H=110, F=8, N=64, dr0=(5.0, 9.0), counts=True), 64, 8, True),
    "float64": (S.BurstSpec(W=64, H=64, F=12, N=64, dr0=(6.0, 6.0), counts=False), 64, 8, True),
    "wide256": (S.BurstSpec(W=300, H=256, F=6, N=256, dr0=(8.0, 12.0), counts=True), 256, 9, False),
    "ragged128": (S.BurstSpec(W=200, H=150, F=5, N=128, dr0=(5.0, 12.0), counts=True), 128, 16, False),
}
ORDER = ["ragged64", "float64", "wide256", "ragged128"]


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_00581_gb300 import build
    build.build()
    return t


@pytest.fixture(scope="module")
def bursts():
    out = {}
    for k, name in enumerate(ORDER):
        spec, N, R, given = CASES[name]
        out[name] = S.make_burst(spec, channel=20 + k, burst=0)
    return out


def _setup(torch, name, b, **modes):
    from paper_1701_00581_gb300 import Channel, Plan
    spec, N, R, given = CASES[name]
    plan = Plan(Channel(W=spec.W, H=spec.H, N=N, R=R, max_frames=spec.F, **modes))
    dev = "cuda:0"
    n = plan.info["n_sub"]
    ws, lay = plan.workspace(spec.F, n)
    ws.zero_()
    io = {"frames": torch.from_numpy(b["frames"]).to(dev), "ws": ws, "lay": lay,
          "out": torch.zeros((spec.H, spec.W), device=dev),
          "valid": torch.zeros((spec.H, spec.W), dtype=torch.uint8, device=dev)}
    if given:
        io["stf"] = torch.from_numpy(b["stf_emp"]).to(dev)
    return plan, io


def _run(torch, names, bursts, opts=None):
    """The bursts through one batch (options tuned for the batch, or given);
    returns every buffer and the options used."""
    from paper_1701_00581_gb300 import Batch, SM_F32, SM_U16
    setups = [_setup(torch, nm, bursts[nm]) for nm in names]
    plans = [p for p, _ in setups]
    ios = [io for _, io in setups]
    fts = [SM_U16 if CASES[nm][0].counts else SM_F32 for nm in names]
    bt = Batch(plans, [CASES[nm][0].F for nm in names], fts, **(opts or {}))
    bt.reconstruct(ios)
    torch.cuda.synchronize()
    assert bt.status() == 0
    res = {}
    for nm, plan, io in zip(names, plans, ios):
        F, n = CASES[nm][0].F, plan.info["n_sub"]
        v = plan.views(io["ws"], io["lay"], F, n)
        res[nm] = {"plan": plan, "out": io["out"].cpu().numpy(), "valid": io["valid"].cpu().numpy().astype(bool),
                   **{k: v[k].cpu().numpy().copy() for k in ("spec", "P", "M", "B", "rec", "flux")}}
    res["opts"] = dict(bt.opts)
    bt.close()
    return res


@pytest.fixture(scope="module")
def mixed(torch, bursts):
    return _run(torch, ORDER, bursts)


@pytest.fixture(scope="module")
def alone(torch, bursts, mixed):
    return {nm: _run(torch, [nm], bursts, mixed["opts"])[nm] for nm in ORDER}


def test_batch_info_counts_the_work(torch, bursts):
    from paper_1701_00581_gb300 import SM_BATCH_FUSED, SM_BATCH_GRID, SM_BATCH_TILES, SM_F32, SM_U16, Batch
    setups = [_setup(torch, nm, bursts[nm]) for nm in ORDER]
    fts = [SM_U16 if CASES[nm][0].counts else SM_F32 for nm in ORDER]
    n_fft = sum(CASES[nm][0].F * p.info["n_sub"] for nm, (p, _) in zip(ORDER, setups))
    n_bis = sum(p.info["n_tiles"] * p.info["n_sub"] for p, _ in setups)
    for launch, items in ((SM_BATCH_FUSED, n_fft + n_bis), (SM_BATCH_TILES, n_bis), (SM_BATCH_GRID, 0)):
        bt = Batch([p for p, _ in setups], [CASES[nm][0].F for nm in ORDER], fts, launch=launch)
        assert bt.opts["launch"] == launch
        assert bt.info["n_items"] == items
        assert (bt.info["grid"] > 0) == (launch != SM_BATCH_GRID) and bt.info["device_bytes"] > 0
        bt.close()


@pytest.mark.parametrize("name", ORDER)
def test_each_burst_is_the_same_alone_and_in_the_mix(mixed, alone, name):
    a, m = alone[name], mixed[name]
    for k in ("spec", "flux", "P", "M", "B", "rec", "out", "valid"):
        assert np.array_equal(a[k], m[k]), k


@pytest.mark.parametrize("name", ORDER)
def test_batched_burst_matches_the_oracle(mixed, bursts, name):
    spec, N, R, given = CASES[name]
    b = bursts[name]
    g = mixed[name]
    plan = g["plan"]
    K = plan.info["K"]
    ref = O.reconstruct_burst(b["frames"], N, N // 2, CS.FC, R, N // 8, b["stf_emp"] if given else None)
    wv = CS.used_pairs(N, R)
    idx = plan.pair_index(wv)
    iy, ix = CS.box_to_grid_index(N, K, R)
    for s, res in ref["sub"].items():
        assert CS.rel_l2(g["spec"][s][:, :, :2 * K + 1], res["In"][:, iy][:, :, ix]) < SPEC_TOL
        Pref = res["P"][N // 2:N // 2 + K + 1, N // 2 - K:N // 2 + K + 1]
        Mref = res["M"][N // 2:N // 2 + K + 1, N // 2 - K:N // 2 + K + 1]
        assert CS.rel_l2(g["P"][s][:, :2 * K + 1], Pref) < SPEC_TOL
        assert CS.rel_l2(g["M"][s][:, :2 * K + 1], Mref) < SPEC_TOL
        assert CS.rel_l2(g["B"][s][idx], CS.oracle_B_used(res["In"], wv)) < SPEC_TOL
    v = ref["valid"]
    assert np.array_equal(g["valid"], v)
    assert CS.rel_l2(g["out"][v], ref["out"][v]) < IMG_TOL
    assert np.all(g["out"][~v] == 0)


def test_batch_rejects_bad_compositions(torch, bursts):
    from paper_1701_00581_gb300 import SM_ACC_KAHAN, SM_FP16, Batch, Channel, Plan, SpeckleError, SM_U16, _lib
    p0 = Plan(Channel(W=150, H=110, N=64, R=8, max_frames=8))
    p16 = Plan(Channel(W=150, H=110, N=64, R=8, max_frames=8, spectra_prec=SM_FP16))
    pk = Plan(Channel(W=150, H=110, N=64, R=8, max_frames=8, acc_mode=SM_ACC_KAHAN))
    for plans, F in (([p0, p16], [8, 8]), ([pk], [8]), ([p0], [9]), ([p0] * 9, [8] * 9)):
        with pytest.raises(SpeckleError) as e:
            Batch(plans, F, [SM_U16] * len(plans))
        assert e.value.status == _lib.SM_EINVAL
    # a workspace not laid out for all subfields in one chunk
    bt = Batch([p0], [8], [SM_U16])
    ws, lay = p0.workspace(8, 2)
    frames = torch.zeros((8, 110, 150), dtype=torch.uint16, device="cuda:0")
    with pytest.raises(SpeckleError) as e:
        bt.spectra_bispectrum([{"frames": frames, "ws": ws, "lay": lay}])
    assert e.value.status == _lib.SM_EINVAL
    bt.close()


@pytest.mark.parametrize("opts", [dict(lookahead=1, ctas_per_sm=3, launch=1), dict(lookahead=4, ctas_per_sm=4, launch=1),
                                  dict(ctas_per_sm=4, launch=2, tile_order=2), dict(ctas_per_sm=3, launch=2),
                                  dict(launch=3)])
def test_every_launch_shape_gives_the_same_bursts(torch, bursts, mixed, opts):
    """The autotuner's choices change only the schedule: every lookahead, CTA
    count, tile order and launch gives bitwise the same result for the same
    placement of the transforms (items of the persistent launch, or the
    per-stage spectra kernel first), and the two placements agree to
    rounding (their windowed means are summed in different orders)."""
    from paper_1701_00581_gb300 import Batch, SM_BATCH_FUSED, SM_F32, SM_U16
    setups = [_setup(torch, nm, bursts[nm]) for nm in ORDER]
    fts = [SM_U16 if CASES[nm][0].counts else SM_F32 for nm in ORDER]
    bt = Batch([p for p, _ in setups], [CASES[nm][0].F for nm in ORDER], fts, **opts)
    ref_fused = mixed["opts"]["launch"] == SM_BATCH_FUSED
    bt.reconstruct([io for _, io in setups])
    torch.cuda.synchronize()
    assert bt.status() == 0
    for nm, (plan, io) in zip(ORDER, setups):
        v = plan.views(io["ws"], io["lay"], CASES[nm][0].F, plan.info["n_sub"])
        B, out = v["B"].cpu().numpy(), io["out"].cpu().numpy()
        if (opts["launch"] == SM_BATCH_FUSED) == ref_fused:
            assert np.array_equal(B, mixed[nm]["B"]) and np.array_equal(out, mixed[nm]["out"])
        else:
            assert CS.rel_l2(B, mixed[nm]["B"]) < 1e-5
            m = mixed[nm]["valid"]
            assert CS.rel_l2(out[m], mixed[nm]["out"][m]) < 1e-5
    bt.close()


@pytest.mark.parametrize("launch", ["grid", "tiles"])
def test_staged_launches_equal_the_stage_kernels(torch, bursts, launch):
    """With the transforms placed first (the per-stage spectra kernel), the
    batched tile grid and the persistent launch of the tiles give bitwise
    the bispectrum of the per-stage kernels, burst by burst."""
    from paper_1701_00581_gb300 import SM_BATCH_GRID, SM_BATCH_TILES
    opts = {"launch": {"grid": SM_BATCH_GRID, "tiles": SM_BATCH_TILES}[launch]}
    got = _run(torch, ORDER, bursts, opts)
    for nm in ORDER:
        spec, N, R, given = CASES[nm]
        plan, io = _setup(torch, nm, bursts[nm])
        n = plan.info["n_sub"]
        plan.stage_spectra(io["frames"], spec.F, 0, n, io["ws"], io["lay"])
        plan.stage_bispectrum(spec.F, n, io["ws"], io["lay"])
        torch.cuda.synchronize()
        v = plan.views(io["ws"], io["lay"], spec.F, n)
        assert np.array_equal(v["spec"].cpu().numpy(), got[nm]["spec"])
        assert np.array_equal(v["B"].cpu().numpy(), got[nm]["B"])


def test_batch_is_captured_in_a_cuda_graph(torch, bursts, mixed):
    """The whole batched reconstruction -- the queue reset, the batched
    launch, the status copy and every burst's remaining stages -- is captured
    once in a CUDA graph on a side stream and replayed twice: each replay
    gives bitwise the eager result."""
    from paper_1701_00581_gb300 import Batch, SM_F32, SM_U16
    setups = [_setup(torch, nm, bursts[nm]) for nm in ORDER]
    fts = [SM_U16 if CASES[nm][0].counts else SM_F32 for nm in ORDER]
    bt = Batch([p for p, _ in setups], [CASES[nm][0].F for nm in ORDER], fts, **mixed["opts"])
    ios = [io for _, io in setups]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        bt.reconstruct(ios, side)
    for _ in range(2):
        for io in ios:
            io["out"].zero_()
        g.replay()
        torch.cuda.synchronize()
        assert bt.status() == 0
        for nm, io in zip(ORDER, ios):
            assert np.array_equal(io["out"].cpu().numpy(), mixed[nm]["out"])
    bt.close()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_half_precision_batches_match_the_stage_kernels(torch, bursts, prec):
    """Spectra stored in FP16 or BF16: the batched launches stage the raw
    half-precision values, convert them a stage ahead and run the FP32 tile
    body, in every launch shape.  With the transforms placed first the
    bispectrum is bitwise that of the per-stage kernels; the fused launch's
    own transforms round the FP32 spectra differently before storage, which
    moves B by at most a half-precision rounding step."""
    from paper_1701_00581_gb300 import SM_BATCH_FUSED, SM_BATCH_GRID, SM_BATCH_TILES, SM_BF16, SM_F32, SM_FP16, \
        SM_U16, Batch
    mode = {"fp16": SM_FP16, "bf16": SM_BF16}[prec]
    tol = {"fp16": 2e-3, "bf16": 2e-2}[prec]
    fts = [SM_U16 if CASES[nm][0].counts else SM_F32 for nm in ORDER]
    ref = {}
    for nm in ORDER:
        spec = CASES[nm][0]
        plan, io = _setup(torch, nm, bursts[nm], spectra_prec=mode)
        n = plan.info["n_sub"]
        plan.stage_spectra(io["frames"], spec.F, 0, n, io["ws"], io["lay"])
        plan.stage_bispectrum(spec.F, n, io["ws"], io["lay"])
        torch.cuda.synchronize()
        ref[nm] = plan.views(io["ws"], io["lay"], spec.F, n)["B"].cpu().numpy()
    for launch in (SM_BATCH_FUSED, SM_BATCH_TILES, SM_BATCH_GRID):
        setups = [_setup(torch, nm, bursts[nm], spectra_prec=mode) for nm in ORDER]
        bt = Batch([p for p, _ in setups], [CASES[nm][0].F for nm in ORDER], fts, launch=launch)
        bt.spectra_bispectrum([io for _, io in setups])
        torch.cuda.synchronize()
        assert bt.status() == 0
        for nm, (plan, io) in zip(ORDER, setups):
            B = plan.views(io["ws"], io["lay"], CASES[nm][0].F, plan.info["n_sub"])["B"].cpu().numpy()
            if launch == SM_BATCH_FUSED:
                assert CS.rel_l2(B, ref[nm]) < tol, nm
            else:
                assert np.array_equal(B, ref[nm]), nm
        bt.close()
