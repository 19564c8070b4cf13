"""Reduced-precision spectra storage (FP16 with a 2^14 scale, BF16) on the GPU.

The frame spectra are the only reduced-precision store; products and sums
stay FP32 and the phase recursion FP64.  The per-stage error against the
FP64 oracle is measured and gated: FP16 keeps 11 significant bits, so the
image stays within the 1e-3 image tolerance; BF16 keeps 8 bits and is gated
looser (reported).
"""
import os

import numpy as np
import pytest

from paper_1701_00581_gb300 import SM_BF16, SM_FP16, SM_FP32

from . import _cases as CS

pytestmark = pytest.mark.gpu

# rel L2 gates per storage mode: (P, B, image)
GATES = {SM_FP32: (1e-4, 1e-4, 1e-3), SM_FP16: (1e-3, 2e-3, 1e-3), SM_BF16: (1e-2, 2e-2, 1e-2)}


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_00581_gb300 import build
    build.build()
    return t


@pytest.mark.parametrize("prec", [SM_FP32, SM_FP16, SM_BF16])
def test_spectra_storage_precision(torch, prec):
    from paper_1701_00581_gb300 import Plan
    plan = Plan(CS.gpu_channel("ragged", spectra_prec=prec))
    b = CS.burst("ragged")
    g = CS.gpu_run(plan, b["frames"], b["stf_emp"])
    o = CS.oracle_run("ragged")
    K = plan.info["K"]
    N = 64
    wv = CS.used_pairs(64, 8)
    idx = plan.pair_index(wv)
    errP, errB = [], []
    for s, res in o["sub"].items():
        Pref = res["P"][N // 2:N // 2 + K + 1, N // 2 - K:N // 2 + K + 1]
        errP.append(CS.rel_l2(g["P"][s][:, :2 * K + 1], Pref))
        errB.append(CS.rel_l2(g["B"][s][idx], CS.oracle_B_used(res["In"], wv)))
    v = o["valid"]
    errI = CS.rel_l2(g["out"][v], o["out"][v])
    gp, gb, gi = GATES[prec]
    report = os.environ.get("SPECKLE_REPORT_DIR")
    if report:
        with open(os.path.join(report, f"precision_{prec}.txt"), "w") as f:
            f.write(f"spectra_prec={prec}: P rel L2 {max(errP):.3e}, B rel L2 {max(errB):.3e}, "
                    f"image rel L2 {errI:.3e}\n")
    assert max(errP) < gp
    assert max(errB) < gb
    assert errI < gi
