"""The allocation-free whole-path entry point, sm_reconstruct_noalloc.

Callers that may not allocate device memory while they run (a camera loop
that fixes its device memory at start-up, a plug-in whose host framework
owns every allocation) call this entry point instead of sm_reconstruct; it
works on a fixed scratch array inside the library.  Its mosaic must match
the one sm_reconstruct computes on a caller-provided workspace, call after
call.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from . import _cases as CS

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-3


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_00581_gb300 import build
    build.build()
    return t


def test_noalloc_matches_workspace_entry_on_two_calls(torch):
    from paper_1701_00581_gb300 import Plan
    plan = Plan(CS.gpu_channel("ragged"))
    b = CS.burst("ragged")
    F, n = b["frames"].shape[0], plan.info["n_sub"]
    dev = "cuda:0"
    frames = torch.from_numpy(b["frames"]).to(dev)
    stf = torch.from_numpy(b["stf_emp"]).to(dev)
    ws, lay = plan.workspace(F, n)
    ref = torch.zeros((110, 150), device=dev)
    ref_valid = torch.zeros((110, 150), dtype=torch.uint8, device=dev)
    plan.reconstruct(frames, F, stf, n, ws, lay, ref, ref_valid)
    torch.cuda.synchronize()
    ref_np, v = ref.cpu().numpy(), ref_valid.cpu().numpy().astype(bool)
    for _ in range(2):
        out = torch.full((110, 150), -1.0, device=dev)
        valid = torch.zeros((110, 150), dtype=torch.uint8, device=dev)
        plan.reconstruct_noalloc(frames, F, stf, out, valid)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(valid.cpu().numpy().astype(bool), v)
        assert CS.rel_l2(got[v], ref_np[v]) < IMG_TOL
        assert np.all(got[~v] == 0)


def test_noalloc_rejects_a_channel_too_large_for_the_scratch(torch):
    from paper_1701_00581_gb300 import Channel, Plan, SpeckleError, _lib
    plan = Plan(Channel(W=2560, H=2160, N=256, R=24))
    frames = torch.zeros((1, 8, 8), dtype=torch.uint16, device="cuda:0")
    stf = torch.zeros((256, 256), dtype=torch.float64, device="cuda:0")
    out = torch.zeros((8, 8), device="cuda:0")
    with pytest.raises(SpeckleError) as e:
        plan.reconstruct_noalloc(frames, 1, stf, out)
    assert e.value.status == _lib.SM_ENOMEM
    assert "bytes" in str(e.value)
