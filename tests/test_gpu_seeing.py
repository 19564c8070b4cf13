"""Seeing estimate (Sect. 3.1, spectral ratio technique) on the GPU.

The stage is checked twice against the oracle: on the GPU's own P, M and
noise floor (the same inputs, so only summation order differs and the
fitted D/r0 agrees to 1e-9), and end to end from the frames (FP32 spectra
against FP64, the burst's D/r0 to 2e-3 and the image to the 1e-3 image
tolerance).  The chunked two-pass path and the serving engine give the same
result as one chunk.
"""
import numpy as np
import pytest

from oracle import speckle_oracle as O

from . import _cases as CS

pytestmark = pytest.mark.gpu

FIT_TOL = 1e-9       # same P, M, noise on both sides
SEEING_TOL = 2e-3    # FP32 spectra against the FP64 oracle
IMG_TOL = 1e-3


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_00581_gb300 import build
    build.build()
    return t


def centred(plan, hb):
    """Half box [ky = 0..K][kx + K] -> centred N x N grid (rows ky >= 0 only)."""
    N, K = plan.info["N"], plan.info["K"]
    g = np.zeros((N, N), dtype=hb.dtype)
    g[N // 2:N // 2 + K + 1, N // 2 - K:N // 2 + K + 1] = hb[:, :2 * K + 1]
    return g


def oracle_fit_on_gpu_stats(plan, v, F, c_sub, sl):
    P = centred(plan, v["P"][sl].cpu().numpy().astype(np.float64))
    M = centred(plan, v["M"][sl].cpu().numpy().astype(np.complex128))
    noise = float(v["noise"][sl].cpu().numpy())
    num, den = O.spectral_ratio(P, M, noise, F, plan.info["N"], CS.FC)
    return O.fit_d_over_r0(num, den, plan.info["N"], CS.FC, plan.ch.ck)


def test_cubes_match_oracle(torch):
    from paper_1701_00581_gb300 import Channel, Plan
    for W, H, N, stride in [(150, 110, 64, 32), (300, 256, 256, 128), (1024, 1024, 128, 64), (96, 80, 64, 32)]:
        plan = Plan(Channel(W=W, H=H, N=N, R=4, stride=stride, max_frames=4))
        assert plan.cubes().tolist() == O.seeing_cubes(W, H, N, stride)
    plan = Plan(Channel(W=150, H=50, N=64, R=4, max_frames=4))
    assert plan.info["n_cubes"] == 0 and plan.cubes().size == 0


def test_seeing_stage_matches_oracle_on_the_same_statistics(torch):
    from paper_1701_00581_gb300 import Plan
    plan = Plan(CS.gpu_channel("ragged"))
    b = CS.burst("ragged")
    F = b["frames"].shape[0]
    n = plan.info["n_sub"]
    dev = "cuda:0"
    frames = torch.from_numpy(b["frames"]).to(dev)
    ws, lay = plan.workspace(F, n)
    plan.stage_spectra(frames, F, 0, n, ws, lay)
    plan.stage_stats(F, n, ws, lay)
    plan.stage_seeing(F, 0, n, ws, lay)
    plan.stage_seeing_stf(ws, lay)
    torch.cuda.synchronize()
    v = plan.views(ws, lay, F, n)
    seeing = v["seeing"].cpu().numpy()
    cubes = plan.cubes()
    xs = np.array([oracle_fit_on_gpu_stats(plan, v, F, c, int(c)) for c in cubes])
    assert np.allclose(seeing[:len(cubes)], xs, rtol=FIT_TOL, atol=0)
    xb = 1.0 / np.mean(1.0 / xs)
    assert seeing[len(cubes)] == pytest.approx(xb, rel=FIT_TOL)
    stf = O.stf_model(plan.info["N"], CS.FC, [seeing[len(cubes)]], plan.ch.ck)
    assert np.allclose(v["stf"].cpu().numpy(), stf, rtol=1e-12, atol=1e-15)


def test_estimated_reconstruction_matches_oracle(torch):
    from paper_1701_00581_gb300 import Plan
    plan = Plan(CS.gpu_channel("ragged"))
    b = CS.burst("ragged")
    F = b["frames"].shape[0]
    c = CS.case("ragged")
    o = O.reconstruct_burst(b["frames"], c["N"], c["stride"], CS.FC, c["R"], c["taper"], None)
    n = plan.info["n_sub"]
    dev = "cuda:0"
    frames = torch.from_numpy(b["frames"]).to(dev)
    results = []
    for chunk in (n, 5):
        ws, lay = plan.workspace(F, chunk)
        out = torch.zeros((plan.ch.H, plan.ch.W), device=dev)
        valid = torch.zeros((plan.ch.H, plan.ch.W), dtype=torch.uint8, device=dev)
        plan.reconstruct(frames, F, None, chunk, ws, lay, out, valid)
        torch.cuda.synchronize()
        seeing = plan.views(ws, lay, F, chunk)["seeing"].cpu().numpy()
        results.append((out.cpu().numpy(), valid.cpu().numpy().astype(bool), seeing))
    (out1, valid1, s1), (out2, valid2, s2) = results
    ncub = plan.info["n_cubes"]
    assert np.allclose(s1[:ncub], o["seeing"][0], rtol=SEEING_TOL)
    assert s1[ncub] == pytest.approx(o["seeing"][1], rel=SEEING_TOL)
    assert np.array_equal(valid1, o["valid"])
    assert CS.rel_l2(out1[o["valid"]], o["out"][o["valid"]]) < IMG_TOL
    # the two-pass chunked path estimates from the same cube statistics
    assert np.array_equal(s1, s2)
    assert np.array_equal(valid1, valid2)
    assert np.array_equal(out1, out2)


def test_engine_estimates_seeing(torch):
    from paper_1701_00581_gb300 import Engine, Plan
    ch = CS.gpu_channel("ragged")
    b = CS.burst("ragged")
    F = b["frames"].shape[0]
    plan = Plan(ch)
    n = plan.info["n_sub"]
    dev = "cuda:0"
    frames = torch.from_numpy(b["frames"]).to(dev)
    ws, lay = plan.workspace(F, n)
    ref = torch.zeros((ch.H, ch.W), device=dev)
    plan.reconstruct(frames, F, None, n, ws, lay, ref)
    torch.cuda.synchronize()
    ref_seeing = plan.views(ws, lay, F, n)["seeing"].cpu().numpy()[plan.info["n_cubes"]]
    eng = Engine([ch], hbm_budget_bytes=1 << 30, max_inflight=2)
    outs = []
    for _ in range(2):        # the second burst replays the captured graph
        out = np.zeros((ch.H, ch.W), np.float32)
        t = eng.submit(0, b["frames"], out)
        st, res = eng.poll(t, -1)
        assert st == 0
        assert res["d_over_r0"] == ref_seeing
        outs.append(out)
    # with d_over_r0 given the result reports no estimate
    out = np.zeros((ch.H, ch.W), np.float32)
    st, res = eng.poll(eng.submit(0, b["frames"], out, d_over_r0=b["d_over_r0"]), -1)
    assert st == 0 and res["d_over_r0"] == 0.0
    eng.close()
    for o in outs:
        assert np.array_equal(o, ref.cpu().numpy())


def test_seeing_errors(torch):
    from paper_1701_00581_gb300 import Channel, Plan, SpeckleError
    from paper_1701_00581_gb300 import _lib
    plan = Plan(CS.gpu_channel("ragged"))
    ws, lay = plan.workspace(4, plan.info["n_sub"])
    with pytest.raises(SpeckleError) as e:
        plan.stage_seeing(1, 0, plan.info["n_sub"], ws, lay)          # one frame has no spectral ratio
    assert e.value.status == _lib.SM_EINVAL
    nocube = Plan(Channel(W=150, H=50, N=64, R=4, max_frames=4))
    ws2, lay2 = nocube.workspace(4, nocube.info["n_sub"])
    for call in (lambda: nocube.stage_seeing(4, 0, nocube.info["n_sub"], ws2, lay2),
                 lambda: nocube.stage_seeing_stf(ws2, lay2)):
        with pytest.raises(SpeckleError) as e:
            call()
        assert e.value.status == _lib.SM_EINVAL
    import torch as T
    frames = T.zeros((4, 50, 150), dtype=T.uint16, device="cuda:0")
    out = T.zeros((50, 150), device="cuda:0")
    with pytest.raises(SpeckleError) as e:
        nocube.reconstruct(frames, 4, None, nocube.info["n_sub"], ws2, lay2, out)
    assert e.value.status == _lib.SM_EINVAL
