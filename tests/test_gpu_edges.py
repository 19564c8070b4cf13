"""Edge cases of the channel geometry against the oracle (Sect. 2, Sect. 3.2).

* N = 128, R = 16 (the H-alpha channel's size, between the N = 64 and
  N = 256 cases elsewhere): six subfields, ragged in both directions;
* R = K, the largest offset radius a plan accepts (offsets reach the
  cutoff, so |v| < |w| and |w - v| < |w| prune most pairs);
* R = 1, the smallest: four offsets, every target reached along a
  single-step chain;
* a frame smaller than one subfield (40 x 50 px at N = 64): one ragged
  subfield, zero-padded on both axes.

Each compares the bispectrum on every used pair (1e-4 rel L2), the valid
mask (exact) and the mosaic (1e-3 rel L2) with the FP64 oracle on the
same seeded burst.
"""
import numpy as np
import pytest

from oracle import speckle_oracle as O

from . import _cases as CS

pytestmark = pytest.mark.gpu

SPEC_TOL = 1e-4
IMG_TOL = 1e-3

CASES = [
    ("n128_r16", dict(N=128, R=16, W=200, H=150, F=4)),
    ("r_equals_k", dict(N=64, R=18, W=64, H=64, F=3)),
    ("r1", dict(N=64, R=1, W=96, H=64, F=3)),
    ("frame_below_n", dict(N=64, R=8, W=40, H=50, F=3)),
]


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_00581_gb300 import build
    build.build()
    return t


@pytest.mark.parametrize("name,c", CASES, ids=[n for n, _ in CASES])
def test_geometry_edge_matches_oracle(torch, name, c):
    from paper_1701_00581_gb300 import Channel, Plan
    from synth import burst as S
    N, R = c["N"], c["R"]
    spec = S.BurstSpec(W=c["W"], H=c["H"], F=c["F"], N=N, dr0=(5.0, 9.0), counts=True)
    b = S.make_burst(spec, channel=21, burst=0)
    stride, taper = N // 2, N // 8
    plan = Plan(Channel(W=spec.W, H=spec.H, N=N, R=R, stride=stride, fc=CS.FC, taper=taper,
                        max_frames=spec.F))
    if name == "r_equals_k":
        assert plan.info["K"] == R
    g = CS.gpu_run(plan, b["frames"], b["stf_emp"])
    o = O.reconstruct_burst(b["frames"], N, stride, CS.FC, R, taper, b["stf_emp"])
    assert plan.info["n_sub"] == len(o["subs"])
    wv = CS.used_pairs(N, R)
    idx = plan.pair_index(wv)
    assert (idx >= 0).all()
    for s in range(plan.info["n_sub"]):
        assert CS.rel_l2(g["B"][s][idx], CS.oracle_B_used(o["sub"][s]["In"], wv)) < SPEC_TOL
    v = o["valid"]
    assert np.array_equal(g["valid"], v)
    assert CS.rel_l2(g["out"][v], o["out"][v]) < IMG_TOL
    assert np.all(g["out"][~v] == 0)
