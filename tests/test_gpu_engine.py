"""Serving engine (sm_open / sm_submit_burst / sm_poll / sm_close) on the GPU.

A burst served by the engine gives the same mosaic as the plain stage path,
and the same mosaic alone as in a mix of concurrently admitted bursts; the
admission and error paths return their status codes without faulting.
"""
import numpy as np
import pytest

from synth import burst as S

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


def _bursts(n):
    spec = CS.RAGGED["spec"]
    return [S.make_burst(spec, channel=11, burst=i) for i in range(n)]


def _plain(torch, ch, b):
    from paper_1701_00581_gb300 import Plan
    plan = Plan(ch)
    stf = plan.model_stf(b["d_over_r0"])
    g = CS.gpu_run(plan, b["frames"], stf)
    return g["out"], g["valid"]


def _serve_one(eng, b, H, W):
    out = np.zeros((H, W), np.float32)
    valid = np.zeros((H, W), np.uint8)
    t = eng.submit(0, b["frames"], out, valid, d_over_r0=b["d_over_r0"])
    st, res = eng.poll(t, -1)
    assert st == 0 and res["gpu_ms"] > 0
    return out, valid.astype(bool)


@pytest.mark.parametrize("mode", [0, 2])
def test_engine_matches_plain_path(torch, mode):
    """Served in submission order or pipelined (the back half's 256-thread
    phase kernel gives bitwise the phasors of the stage path's 512-thread
    one), the mosaic is bitwise the plain stage path's."""
    from paper_1701_00581_gb300 import Engine
    ch = CS.gpu_channel("ragged")
    b = _bursts(1)[0]
    ref_out, ref_valid = _plain(torch, ch, b)
    eng = Engine([ch], hbm_budget_bytes=1 << 30, max_inflight=2, overlap_kernels=mode)
    out, valid = _serve_one(eng, b, 110, 150)
    eng.close()
    assert np.array_equal(valid, ref_valid)
    assert np.array_equal(out, ref_out)


@pytest.mark.parametrize("overlap", [0, 1, 2])
def test_alone_equals_in_the_mix(torch, overlap):
    """Bursts admitted while others are on the device give the same mosaic
    (bitwise) as each burst served alone, with the bursts' kernels run in
    submission order, concurrently, or pipelined."""
    from paper_1701_00581_gb300 import Engine
    ch = CS.gpu_channel("ragged")
    bursts = _bursts(4)
    eng = Engine([ch], hbm_budget_bytes=1 << 30, max_inflight=3, overlap_kernels=overlap)
    alone = [_serve_one(eng, b, 110, 150) for b in bursts]
    outs = [np.zeros((110, 150), np.float32) for _ in bursts]
    pending, k = [], 0
    while k < len(bursts) or pending:
        while k < len(bursts):
            t = eng.try_submit(0, bursts[k]["frames"], outs[k], d_over_r0=bursts[k]["d_over_r0"])
            if t is None:
                break
            pending.append((t, k))
            k += 1
        t, i = pending.pop(0)
        st, _ = eng.poll(t, -1)
        assert st == 0
    eng.close()
    for (o, _), m in zip(alone, outs):
        assert np.array_equal(o, m)


def test_two_host_threads_share_an_engine(torch):
    """Submit and poll from two host threads at once (the handle is locked
    internally): every burst's mosaic equals the same burst served alone."""
    import threading
    import time
    from paper_1701_00581_gb300 import Engine
    ch = CS.gpu_channel("ragged")
    bursts = _bursts(6)
    eng = Engine([ch], hbm_budget_bytes=1 << 30, max_inflight=2)
    alone = [_serve_one(eng, b, 110, 150)[0] for b in bursts]
    outs = [np.zeros((110, 150), np.float32) for _ in bursts]
    errors = []

    def worker(idx):
        try:
            for i in idx:
                t = None
                while t is None:
                    t = eng.try_submit(0, bursts[i]["frames"], outs[i], d_over_r0=bursts[i]["d_over_r0"])
                    if t is None:
                        time.sleep(0.001)
                st, _ = eng.poll(t, -1)
                assert st == 0
        except Exception as e:          # reported by the main thread
            errors.append(e)

    th = [threading.Thread(target=worker, args=(range(k, len(bursts), 2),)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=120)
    eng.close()
    assert not errors, errors
    for a, o in zip(alone, outs):
        assert np.array_equal(a, o)


def test_ordered_bursts_finish_in_submission_order(torch):
    """With overlap_kernels off, a burst's kernels start after the previous
    burst's have finished: once the last ticket is done, every earlier one
    is done too (a non-blocking poll finds it complete)."""
    from paper_1701_00581_gb300 import Engine
    ch = CS.gpu_channel("ragged")
    bursts = _bursts(3)
    eng = Engine([ch], hbm_budget_bytes=1 << 30, max_inflight=3)
    outs = [np.zeros((110, 150), np.float32) for _ in bursts]
    tickets = [eng.submit(0, b["frames"], o, d_over_r0=b["d_over_r0"]) for b, o in zip(bursts, outs)]
    st, res = eng.poll(tickets[-1], -1)
    assert st == 0 and res["gpu_ms"] > 0
    for t in tickets[:-1]:
        st, res = eng.poll(t, 0)
        assert st == 0 and res is not None
    eng.close()


@pytest.mark.parametrize("mode", [0, 2])
def test_stage_times(torch, mode):
    """sm_result.stage_ms: every stage of the burst graph is timed; the
    seeing stage is empty when D/r0 is given and timed when estimated; the
    stages account for the burst's device time."""
    from paper_1701_00581_gb300 import STAGE_NAMES, Engine
    ch = CS.gpu_channel("ragged")
    b = _bursts(1)[0]
    eng = Engine([ch], hbm_budget_bytes=1 << 30, max_inflight=2, overlap_kernels=mode)
    for given in (True, False):
        for _ in range(2):                    # first capture, then replay
            out = np.zeros((110, 150), np.float32)
            t = eng.submit(0, b["frames"], out, d_over_r0=b["d_over_r0"] if given else None)
            st, res = eng.poll(t, -1)
            assert st == 0
            sm = res["stage_ms"]
            assert tuple(sm) == STAGE_NAMES
            for name in STAGE_NAMES:
                if name == "seeing" and given:
                    assert sm[name] == 0.0
                else:
                    assert sm[name] > 0.0, name
            total = sum(sm.values())
            assert 0.5 * res["gpu_ms"] <= total <= 1.05 * res["gpu_ms"] + 0.05
    eng.close()


def test_torch_allocator(torch):
    """The engine's arena from torch's caching allocator gives the same
    mosaic; the tensor is held while the engine is open and released by
    close."""
    from paper_1701_00581_gb300 import Engine
    ch = CS.gpu_channel("ragged")
    b = _bursts(1)[0]
    ref_out, ref_valid = _plain(torch, ch, b)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated(0)
    budget = 1 << 30
    eng = Engine([ch], hbm_budget_bytes=budget, max_inflight=2, allocator="torch")
    assert torch.cuda.memory_allocated(0) - before >= budget
    out, valid = _serve_one(eng, b, 110, 150)
    eng.close()
    assert torch.cuda.memory_allocated(0) - before < budget
    assert np.array_equal(valid, ref_valid)
    assert np.array_equal(out, ref_out)


def test_two_channels_in_one_engine(torch):
    from paper_1701_00581_gb300 import Channel, Engine
    c0 = CS.gpu_channel("ragged")
    c1 = Channel(W=96, H=80, N=64, R=6, stride=32, taper=8, max_frames=5)
    b0 = _bursts(1)[0]
    b1 = S.make_burst(S.BurstSpec(W=96, H=80, F=5, N=64, dr0=(4.0, 6.0), counts=True), channel=12)
    eng = Engine([c0, c1], hbm_budget_bytes=1 << 30, max_inflight=2)
    o0 = np.zeros((110, 150), np.float32)
    o1 = np.zeros((80, 96), np.float32)
    t0 = eng.submit(0, b0["frames"], o0, d_over_r0=b0["d_over_r0"])
    t1 = eng.submit(1, b1["frames"], o1, d_over_r0=b1["d_over_r0"])
    assert eng.poll(t1, -1)[0] == 0 and eng.poll(t0, -1)[0] == 0
    eng.close()
    ref1, _ = _plain(torch, c1, b1)
    assert np.array_equal(o1, ref1)
    assert np.isfinite(o0).all()


def test_admission_and_error_statuses(torch):
    from paper_1701_00581_gb300 import Engine, SpeckleError, _lib
    ch = CS.gpu_channel("ragged")
    b = _bursts(1)[0]
    # a budget smaller than one burst: SM_ENOMEM, from sm_open for the shared
    # workspace, from sm_submit_burst for per-burst workspaces
    with pytest.raises(SpeckleError) as e:
        Engine([ch], hbm_budget_bytes=1 << 20, max_inflight=1)
    assert e.value.status == _lib.SM_ENOMEM
    eng = Engine([ch], hbm_budget_bytes=1 << 20, max_inflight=1, overlap_kernels=True)
    with pytest.raises(SpeckleError) as e:
        eng.submit(0, b["frames"], np.zeros((110, 150), np.float32), d_over_r0=b["d_over_r0"])
    assert e.value.status == _lib.SM_ENOMEM
    eng.close()
    eng = Engine([ch], hbm_budget_bytes=1 << 30, max_inflight=1)
    out = np.zeros((110, 150), np.float32)
    t = eng.submit(0, b["frames"], out, d_over_r0=b["d_over_r0"])
    # the only slot is taken: SM_EBUSY, nothing queued
    assert eng.try_submit(0, b["frames"], np.zeros_like(out), d_over_r0=b["d_over_r0"]) is None
    st, _ = eng.poll(t, 0)
    assert st in (_lib.SM_OK, _lib.SM_PENDING)
    if st != _lib.SM_OK:
        assert eng.poll(t, -1)[0] == _lib.SM_OK
    # a finished ticket is released
    with pytest.raises(SpeckleError) as e:
        eng.poll(t, 0)
    assert e.value.status == _lib.SM_ENOTFOUND
    # bad arguments
    with pytest.raises(SpeckleError) as e:
        eng.submit(5, b["frames"], out, d_over_r0=b["d_over_r0"])
    assert e.value.status == _lib.SM_EINVAL
    with pytest.raises(SpeckleError) as e:
        # neither stf nor d_over_r0, and one frame: the seeing cannot be estimated
        eng.submit(0, b["frames"][:1], out)
    assert e.value.status == _lib.SM_EINVAL
    eng.close()


def test_close_with_pending_tickets(torch):
    from paper_1701_00581_gb300 import Engine
    ch = CS.gpu_channel("ragged")
    bursts = _bursts(2)
    eng = Engine([ch], hbm_budget_bytes=1 << 30, max_inflight=2)
    outs = [np.zeros((110, 150), np.float32) for _ in bursts]
    for b, o in zip(bursts, outs):
        eng.submit(0, b["frames"], o, d_over_r0=b["d_over_r0"])
    eng.close()                       # waits for the device, releases everything
    eng2 = Engine([ch], hbm_budget_bytes=1 << 30, max_inflight=1)
    o, _ = _serve_one(eng2, bursts[0], 110, 150)
    eng2.close()
    assert np.isfinite(o).all()


def test_served_burst_with_estimated_seeing_matches_the_oracle(torch):
    """The path the served end-to-end number times, checked against the oracle
    directly: frames from host memory, no STF and no D/r0 (the engine
    estimates the seeing from the burst, Sect. 3.1), mosaic copied back to
    the host; image rel L2 1e-3 and the valid mask exact."""
    from oracle import speckle_oracle as O
    from paper_1701_00581_gb300 import Engine
    c = CS.RAGGED
    ch = CS.gpu_channel("ragged")
    b = _bursts(1)[0]
    eng = Engine([ch], hbm_budget_bytes=1 << 30, max_inflight=2)
    out = np.zeros((110, 150), np.float32)
    valid = np.zeros((110, 150), np.uint8)
    t = eng.submit(0, b["frames"], out, valid)
    st, res = eng.poll(t, -1)
    eng.close()
    assert st == 0 and res["d_over_r0"] > 0
    ref = O.reconstruct_burst(b["frames"], c["N"], c["stride"], CS.FC, c["R"], c["taper"], None)
    _, x_burst = O.estimate_seeing(b["frames"], c["N"], c["stride"], CS.FC, c["taper"])
    assert abs(res["d_over_r0"] - x_burst) < 2e-3 * x_burst
    v = ref["valid"]
    assert np.array_equal(valid.astype(bool), v)
    assert CS.rel_l2(out[v], ref["out"][v]) < 1e-3
    assert np.all(out[~v] == 0)


def test_poll_with_a_positive_timeout_times_out_then_completes(torch):
    """sm_poll with timeout_ms > 0 on a burst that needs longer returns
    SM_ETIMEDOUT (the ticket stays valid) and later SM_OK."""
    from paper_1701_00581_gb300 import Channel, Engine, _lib
    spec = S.BurstSpec(W=1024, H=1024, F=40, N=128, dr0=(5.0, 12.0), counts=True)
    b = S.make_burst(spec, channel=12, burst=0)
    ch = Channel(W=1024, H=1024, N=128, R=16, max_frames=40)
    eng = Engine([ch], hbm_budget_bytes=16 << 30, max_inflight=1)
    out = np.zeros((1024, 1024), np.float32)
    # the first burst captures its graph; the timed one replays it
    t = eng.submit(0, b["frames"], out)
    assert eng.poll(t, -1)[0] == _lib.SM_OK
    t = eng.submit(0, b["frames"], out)
    st, res = eng.poll(t, 1)
    assert st == _lib.SM_ETIMEDOUT and res is None
    st, res = eng.poll(t, -1)
    assert st == _lib.SM_OK and res["gpu_ms"] > 1.0
    eng.close()


def test_injected_allocation_failure_reports_on_its_ticket(torch, monkeypatch):
    """SM_FAULT=alloc:2: the second admission fails as if its arena allocation
    had; its ticket reports SM_ENOMEM once, the others are served, and the
    engine stays usable (a host-side injection: no GPU fault)."""
    from paper_1701_00581_gb300 import Engine, SpeckleError, _lib
    ch = CS.gpu_channel("ragged")
    bursts = _bursts(3)
    monkeypatch.setenv("SM_FAULT", "alloc:2")
    eng = Engine([ch], hbm_budget_bytes=1 << 30, max_inflight=2)
    monkeypatch.delenv("SM_FAULT")
    outs = [np.zeros((110, 150), np.float32) for _ in bursts]
    tickets = [eng.submit(0, b["frames"], o, d_over_r0=b["d_over_r0"]) for b, o in zip(bursts[:2], outs[:2])]
    with pytest.raises(SpeckleError) as e:
        eng.poll(tickets[1], -1)
    assert e.value.status == _lib.SM_ENOMEM
    with pytest.raises(SpeckleError) as e:           # reported once, then released
        eng.poll(tickets[1], 0)
    assert e.value.status == _lib.SM_ENOTFOUND
    assert eng.poll(tickets[0], -1)[0] == _lib.SM_OK
    # the failed burst held no slot: the engine takes two more
    t2 = eng.submit(0, bursts[2]["frames"], outs[2], d_over_r0=bursts[2]["d_over_r0"])
    t1 = eng.submit(0, bursts[1]["frames"], outs[1], d_over_r0=bursts[1]["d_over_r0"])
    assert eng.poll(t2, -1)[0] == _lib.SM_OK and eng.poll(t1, -1)[0] == _lib.SM_OK
    eng.close()
    for b, o in zip(bursts, outs):
        ref, _ = _plain(torch, ch, b)
        assert np.array_equal(o, ref)


@pytest.mark.parametrize("mode", [0, 2])
def test_results_reach_pinned_and_pageable_buffers(torch, mode):
    """The mosaic and mask are copied back on the burst's own stream: into
    page-locked caller buffers directly, into pageable ones through the
    slot's pinned staging at poll time; both give the same result, and a
    pipelined engine serves a second channel beside the first."""
    from paper_1701_00581_gb300 import Channel, Engine
    c0 = CS.gpu_channel("ragged")
    c1 = Channel(W=96, H=80, N=64, R=6, stride=32, taper=8, max_frames=5)
    b0 = _bursts(1)[0]
    b1 = S.make_burst(S.BurstSpec(W=96, H=80, F=5, N=64, dr0=(4.0, 6.0), counts=True), channel=12)
    eng = Engine([c0, c1], hbm_budget_bytes=1 << 30, max_inflight=3, overlap_kernels=mode)
    pin_out = torch.zeros((110, 150), dtype=torch.float32).pin_memory()
    pin_valid = torch.zeros((110, 150), dtype=torch.uint8).pin_memory()
    page_out = np.zeros((110, 150), np.float32)
    page_valid = np.zeros((110, 150), np.uint8)
    o1 = np.zeros((80, 96), np.float32)
    t_pin = eng.submit(0, b0["frames"], pin_out.numpy(), pin_valid.numpy(), d_over_r0=b0["d_over_r0"])
    t_1 = eng.submit(1, b1["frames"], o1, d_over_r0=b1["d_over_r0"])
    t_page = eng.submit(0, b0["frames"], page_out, page_valid, d_over_r0=b0["d_over_r0"])
    for t in (t_page, t_1, t_pin):
        assert eng.poll(t, -1)[0] == 0
    eng.close()
    ref, ref_valid = _plain(torch, c0, b0)
    assert np.array_equal(pin_out.numpy(), ref) and np.array_equal(page_out, ref)
    assert np.array_equal(pin_valid.numpy().astype(bool), ref_valid)
    assert np.array_equal(page_valid.astype(bool), ref_valid)
    plan1_out = _plain(torch, c1, b1)[0]
    assert np.array_equal(o1, plan1_out)


def test_pipelined_mode_needs_two_workspaces(torch):
    from paper_1701_00581_gb300 import Channel, Engine, SpeckleError, _lib
    ch = Channel(W=1024, H=1024, N=128, R=16, max_frames=100)
    with pytest.raises(SpeckleError) as e:
        Engine([ch], hbm_budget_bytes=4 << 30, max_inflight=2, overlap_kernels=2)
    assert e.value.status == _lib.SM_ENOMEM
    with pytest.raises(SpeckleError) as e:
        Engine([ch], hbm_budget_bytes=4 << 30, max_inflight=2, overlap_kernels=4)
    assert e.value.status == _lib.SM_EINVAL


def test_batched_engine_mode(torch):
    """overlap_kernels = 3: bursts of two channels submitted as one batch run
    through one batched launch; each burst equals itself submitted alone in
    that mode (bitwise), and the plain stage path to rounding (the batched
    launch may place the transforms differently); a single submit is a
    batch of one; a batch larger than the free slots is refused whole."""
    from paper_1701_00581_gb300 import Channel, Engine, SpeckleError, _lib
    c0 = CS.gpu_channel("ragged")
    c1 = Channel(W=96, H=80, N=64, R=6, stride=32, taper=8, max_frames=5)
    bursts = _bursts(2)
    b1 = S.make_burst(S.BurstSpec(W=96, H=80, F=5, N=64, dr0=(4.0, 6.0), counts=True), channel=12)
    eng = Engine([c0, c1], hbm_budget_bytes=2 << 30, max_inflight=4, overlap_kernels=3)
    items = [dict(channel=0, frames=bursts[0]["frames"], out=np.zeros((110, 150), np.float32),
                  valid=np.zeros((110, 150), np.uint8), d_over_r0=bursts[0]["d_over_r0"]),
             dict(channel=1, frames=b1["frames"], out=np.zeros((80, 96), np.float32), d_over_r0=b1["d_over_r0"]),
             dict(channel=0, frames=bursts[1]["frames"], out=np.zeros((110, 150), np.float32))]   # seeing estimated
    tickets = eng.submit_batch(items)
    assert len(set(tickets)) == 3
    for t in tickets:
        st, res = eng.poll(t, -1)
        assert st == 0 and res["gpu_ms"] > 0
    alone = []
    for it in items:
        o = np.zeros_like(it["out"])
        t = eng.submit_batch([dict(it, out=o, valid=None)])[0]
        assert eng.poll(t, -1)[0] == 0
        alone.append(o)
    with pytest.raises(SpeckleError) as e:
        eng.submit_batch([dict(items[0], out=np.zeros((110, 150), np.float32))] * 5)
    assert e.value.status == _lib.SM_EBUSY
    eng.close()
    for it, a in zip(items, alone):
        assert np.array_equal(it["out"], a)
    ref0, v0 = _plain(torch, c0, bursts[0])
    assert np.array_equal(items[0]["valid"].astype(bool), v0)
    assert CS.rel_l2(items[0]["out"][v0], ref0[v0]) < 1e-5
    ref1, v1 = _plain(torch, c1, b1)
    assert CS.rel_l2(items[1]["out"][v1], ref1[v1]) < 1e-5
