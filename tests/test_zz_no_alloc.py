"""The allocation-free whole-path entry point, sm_reconstruct_noalloc.

Some callers may not allocate device memory once they are running: a camera
or telescope control loop that fixes its device memory at start-up (an
allocation can synchronise the device and stall frame acquisition), or a
plug-in whose host framework owns every device allocation.  They call this
entry point instead of sm_reconstruct; it works on a fixed scratch array
inside the library.  It runs the same kernels in the same order as
sm_reconstruct does with the same subfield chunk, so its mosaic must equal
that one bit for bit, call after call, whether the whole burst fits the
array at once, goes through it in chunks, or has its seeing estimated from
the burst.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from synth import burst as S

from . import _cases as CS

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 64 << 20          # SM_NOALLOC_SCRATCH_BYTES of speckle.h


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_00581_gb300 import build
    build.build()
    return t


def _largest_chunk(plan, F):
    """The chunk the entry point picks: the most subfields whose workspace fits."""
    best = 0
    for n in range(1, plan.info["n_sub"] + 1):
        if plan.layout(F, n).bytes <= SCRATCH_BYTES:
            best = n
        else:
            break
    return best


def _compare(torch, plan, frames_np, stf_np, calls=2):
    F, (H, W) = frames_np.shape[0], frames_np.shape[1:]
    dev = "cuda:0"
    frames = torch.from_numpy(frames_np).to(dev)
    stf = None if stf_np is None else torch.from_numpy(stf_np).to(dev)
    chunk = _largest_chunk(plan, F)
    assert chunk >= 1
    ws, lay = plan.workspace(F, chunk)
    ref = torch.zeros((H, W), device=dev)
    ref_valid = torch.zeros((H, W), dtype=torch.uint8, device=dev)
    plan.reconstruct(frames, F, stf, chunk, ws, lay, ref, ref_valid)
    torch.cuda.synchronize()
    ref_np, v = ref.cpu().numpy(), ref_valid.cpu().numpy()
    del ws
    for _ in range(calls):
        out = torch.full((H, W), -1.0, device=dev)
        valid = torch.full((H, W), 7, dtype=torch.uint8, device=dev)
        plan.reconstruct_noalloc(frames, F, stf, out, valid)
        torch.cuda.synchronize()
        assert np.array_equal(valid.cpu().numpy(), v)
        assert np.array_equal(out.cpu().numpy(), ref_np)
    return chunk, ref_np, v.astype(bool)


def test_noalloc_equals_workspace_entry_on_two_calls(torch):
    from paper_1701_00581_gb300 import Plan
    plan = Plan(CS.gpu_channel("ragged"))
    b = CS.burst("ragged")
    chunk, out, v = _compare(torch, plan, b["frames"], b["stf_emp"])
    assert chunk == plan.info["n_sub"]                # the whole burst fits at once
    o = CS.oracle_run("ragged")
    assert np.array_equal(v, o["valid"])
    assert CS.rel_l2(out[v], o["out"][v]) < 1e-3


def test_noalloc_estimates_the_seeing_without_an_stf(torch):
    from paper_1701_00581_gb300 import Plan
    plan = Plan(CS.gpu_channel("ragged"))
    b = CS.burst("ragged")
    _compare(torch, plan, b["frames"], None)


def test_noalloc_chunks_a_burst_larger_than_the_scratch(torch):
    """A 1024 x 1024 channel (225 subfields of 128^2, |v| <= 16): its whole
    workspace exceeds the array, one subfield fits, so the burst goes through
    in chunks -- with the STF given and with the seeing estimated (the
    two-pass schedule)."""
    from paper_1701_00581_gb300 import Channel, Plan
    spec = S.BurstSpec(W=1024, H=1024, F=4, N=128, dr0=(5.0, 12.0), counts=True)
    b = S.make_burst(spec, channel=13, burst=0)
    plan = Plan(Channel(W=1024, H=1024, N=128, R=16, max_frames=4))
    assert plan.layout(4, plan.info["n_sub"]).bytes > SCRATCH_BYTES
    stf = plan.model_stf(b["d_over_r0"])
    chunk, _, _ = _compare(torch, plan, b["frames"], stf, calls=1)
    assert 1 <= chunk < plan.info["n_sub"]
    _compare(torch, plan, b["frames"], None, calls=2)


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
