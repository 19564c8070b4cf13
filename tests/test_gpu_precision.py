"""Precision modes on the GPU: the precision sweep.

Frame spectra stored in FP32, FP16 (with a 2^14 scale) or BF16; bispectrum
sums in plain or compensated (Kahan) FP32; recursion arithmetic in FP32,
FP64 or float-float (pairs of FP32 numbers, about 48 significant bits).  The per-stage error against the FP64 oracle is measured and gated:
Every storage mode is held to the 1e-3 image tolerance of the mixed-precision
path; the per-stage spectra gates follow the mantissa (FP16 keeps 11
significant bits, BF16 8) and are reported.  Two tests
isolate the modes: Kahan sums against the exact sum of the same FP32
spectra, and the FP64 and float-float recursions against the oracle's on the
same B and M.
"""
import os

import numpy as np
import pytest

from oracle import speckle_oracle as O
from paper_1701_00581_gb300 import (SM_ACC_KAHAN, SM_ACC_PLAIN, SM_BF16, SM_FP16, SM_FP32, SM_PHASE_FF,
                                    SM_PHASE_FP32, SM_PHASE_FP64)

from . import _cases as CS

pytestmark = pytest.mark.gpu

# rel L2 gates per storage mode: (P, B, image)
GATES = {SM_FP32: (1e-4, 1e-4, 1e-3), SM_FP16: (1e-3, 2e-3, 1e-3), SM_BF16: (1e-2, 2e-2, 1e-3)}


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


# ---- accumulation and recursion precision modes (the precision sweep) ----

MODES = [  # (spectra storage, bispectrum sums, recursion arithmetic)
    (SM_FP32, SM_ACC_KAHAN, SM_PHASE_FP32),
    (SM_FP32, SM_ACC_PLAIN, SM_PHASE_FP64),
    (SM_FP32, SM_ACC_KAHAN, SM_PHASE_FP64),
    (SM_FP16, SM_ACC_KAHAN, SM_PHASE_FP64),
    (SM_BF16, SM_ACC_KAHAN, SM_PHASE_FP64),
    (SM_FP32, SM_ACC_PLAIN, SM_PHASE_FF),
    (SM_FP16, SM_ACC_KAHAN, SM_PHASE_FF),
]


@pytest.mark.parametrize("prec,acc,phase", MODES)
def test_precision_modes_match_oracle(torch, prec, acc, phase):
    from paper_1701_00581_gb300 import Plan
    plan = Plan(CS.gpu_channel("ragged", spectra_prec=prec, acc_mode=acc, phase_prec=phase))
    b = CS.burst("ragged")
    g = CS.gpu_run(plan, b["frames"], b["stf_emp"])
    o = CS.oracle_run("ragged")
    wv = CS.used_pairs(64, 8)
    idx = plan.pair_index(wv)
    errB = max(CS.rel_l2(g["B"][s][idx], CS.oracle_B_used(res["In"], wv)) for s, res in o["sub"].items())
    v = o["valid"]
    errI = CS.rel_l2(g["out"][v], o["out"][v])
    gp, gb, gi = GATES[prec]
    report = os.environ.get("SPECKLE_REPORT_DIR")
    if report:
        with open(os.path.join(report, f"precision_{prec}_{acc}_{phase}.txt"), "w") as f:
            f.write(f"spectra_prec={prec} acc_mode={acc} phase_prec={phase}: B rel L2 {errB:.3e}, "
                    f"image rel L2 {errI:.3e}\n")
    assert errB < gb
    assert errI < gi


def _centred_spectra(plan, spec):
    """GPU spectrum boxes [F][ky = -R..K][kx + K] -> FP64 centred [F][N][N]."""
    N, K, R = plan.info["N"], plan.info["K"], plan.info["R"]
    F = spec.shape[0]
    In = np.zeros((F, N, N), dtype=np.complex128)
    In[:, N // 2 - R:N // 2 + K + 1, N // 2 - K:N // 2 + K + 1] = spec[:, :, :2 * K + 1]
    return In


def test_compensated_sums_reduce_the_accumulation_error(torch):
    """100 frames: against the exact (FP64) sum of the GPU's own FP32 frame
    spectra, Kahan accumulation leaves only the rounding of the products."""
    from paper_1701_00581_gb300 import Plan
    b = CS.burst("sub64")
    wv = CS.used_pairs(64, 8)
    errs = {}
    for acc in (SM_ACC_PLAIN, SM_ACC_KAHAN):
        plan = Plan(CS.gpu_channel("sub64", acc_mode=acc))
        g = CS.gpu_run(plan, b["frames"], b["stf_emp"])
        exact = CS.oracle_B_used(_centred_spectra(plan, g["spec"][0]), wv)
        errs[acc] = CS.rel_l2(g["B"][0][plan.pair_index(wv)], exact)
    report = os.environ.get("SPECKLE_REPORT_DIR")
    if report:
        with open(os.path.join(report, "precision_accumulation.txt"), "w") as f:
            f.write(f"F=100 bispectrum sums vs exact sum of the same FP32 spectra: plain {errs[SM_ACC_PLAIN]:.3e}, "
                    f"Kahan {errs[SM_ACC_KAHAN]:.3e}\n")
    assert errs[SM_ACC_KAHAN] < 0.5 * errs[SM_ACC_PLAIN]
    assert errs[SM_ACC_KAHAN] < 1e-6


def _oracle_B_from_gpu(plan, Bg, N, R):
    """The GPU's B(w - v, v) at every used pair, in the oracle's pair layout
    (u in the upper half plane; lower-half u stored conjugated at (-u, -v))."""
    pairs = O.pair_domain(N, CS.FC, R)
    K = int(np.floor(O.cutoff_radius(N, CS.FC)))
    pidx = O._PairIndex(pairs, K, R)
    wv = CS.used_pairs(N, R)
    vals = Bg[plan.pair_index(wv)].astype(np.complex128)
    ux, uy, vx, vy = wv[:, 0] - wv[:, 2], wv[:, 1] - wv[:, 3], wv[:, 2], wv[:, 3]
    up = O.in_half_plane(ux, uy)
    B = np.zeros(len(pairs), dtype=np.complex128)
    B[pidx.find(ux[up], uy[up], vx[up], vy[up])] = vals[up]
    B[pidx.find(-ux[~up], -uy[~up], -vx[~up], -vy[~up])] = np.conj(vals[~up])
    return B, pairs


def test_fp64_recursion_matches_the_oracle_on_the_same_inputs(torch):
    """Recursion alone: the oracle's FP64 recursion on the GPU's own B and M
    against the GPU recursion in FP64, float-float and FP32 arithmetic."""
    from paper_1701_00581_gb300 import Plan
    b = CS.burst("ragged")
    N, R = 64, 8
    err = {}
    for phase in (SM_PHASE_FP32, SM_PHASE_FP64, SM_PHASE_FF):
        plan = Plan(CS.gpu_channel("ragged", phase_prec=phase))
        g = CS.gpu_run(plan, b["frames"], b["stf_emp"])
        K = plan.info["K"]
        e = 0.0
        for s in (0, plan.info["n_sub"] - 1):
            B, pairs = _oracle_B_from_gpu(plan, g["B"][s], N, R)
            M = np.zeros((N, N), dtype=np.complex128)
            M[N // 2:N // 2 + K + 1, N // 2 - K:N // 2 + K + 1] = g["M"][s][:, :2 * K + 1]
            zo = O.phase_recursion(B, pairs, M, N, CS.FC, R)
            zo = zo[N // 2:N // 2 + K + 1, N // 2 - K:N // 2 + K + 1]
            zg = g["z"][s][:, :2 * K + 1]
            m = np.abs(zo) > 0
            e = max(e, float(np.abs(zg[m] - zo[m]).max()))
        err[phase] = e
    report = os.environ.get("SPECKLE_REPORT_DIR")
    if report:
        with open(os.path.join(report, "precision_recursion.txt"), "w") as f:
            f.write(f"max |z_gpu - z_fp64 oracle| on the same B, M: FP32 arithmetic {err[SM_PHASE_FP32]:.3e}, "
                    f"FP64 arithmetic {err[SM_PHASE_FP64]:.3e}, float-float {err[SM_PHASE_FF]:.3e}\n")
    assert err[SM_PHASE_FP64] < 1e-9
    assert err[SM_PHASE_FF] < 1e-9
    assert err[SM_PHASE_FP32] < 1e-3
