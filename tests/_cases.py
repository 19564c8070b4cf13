"""Shared test cases: seeded inputs, oracle runs and GPU stage runs.

Inputs come from ``synth`` (no arithmetic of the method); expected values
come from ``oracle`` only; the GPU path is reached through the C ABI
binding.  Comparisons are element by element on the same seeded inputs.
"""
from __future__ import annotations

import functools
import math

import numpy as np

from oracle import speckle_oracle as O
from synth import burst as S

FC = 0.2885

# ragged multi-tile case: 4 x 3 subfields of 64 px (last column 54 px wide,
# last row 46 px high), 8 frames of uint16 counts, R = 8
RAGGED = dict(spec=S.BurstSpec(W=150, H=110, F=8, N=64, dr0=(5.0, 9.0), counts=True),
              N=64, stride=32, R=8, taper=8)
# one 64 x 64 subfield, 100 float32 frames (the single-subfield workload)
SUB64 = dict(spec=S.CONFIGS["subfield64"], N=64, stride=32, R=8, taper=8)


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.linalg.norm((a - b).ravel())
    n = np.linalg.norm(b.ravel())
    return float(d / n) if n > 0 else float(d)


@functools.lru_cache(maxsize=None)
def burst(name: str):
    case = RAGGED if name == "ragged" else SUB64
    return S.make_burst(case["spec"], channel=7 if name == "ragged" else 0, burst=0)


def case(name: str) -> dict:
    return RAGGED if name == "ragged" else SUB64


def used_pairs(N: int, R: int, fc: float = FC) -> np.ndarray:
    """(wx, wy, vx, vy) of every pair the phase recursion reads (test-side enumeration)."""
    U = O.domain_U(N, fc)
    Hh = U[O.in_half_plane(U[:, 0], U[:, 1])]
    Hh = Hh[(Hh ** 2).sum(1) >= 2]
    V = O.domain_V(R)
    wx = np.repeat(Hh[:, 0], len(V))
    wy = np.repeat(Hh[:, 1], len(V))
    vx = np.tile(V[:, 0], len(Hh))
    vy = np.tile(V[:, 1], len(Hh))
    w2 = wx * wx + wy * wy
    ok = (vx * vx + vy * vy < w2) & ((wx - vx) ** 2 + (wy - vy) ** 2 < w2)
    return np.stack([wx[ok], wy[ok], vx[ok], vy[ok]], axis=1)


@functools.lru_cache(maxsize=None)
def oracle_run(name: str):
    c = case(name)
    b = burst(name)
    return O.reconstruct_burst(b["frames"], c["N"], c["stride"], FC, c["R"], c["taper"], b["stf_emp"])


def oracle_B_used(In: np.ndarray, wv: np.ndarray) -> np.ndarray:
    """Oracle bispectrum at u = w - v for the listed (w, v)."""
    pairs = np.stack([wv[:, 0] - wv[:, 2], wv[:, 1] - wv[:, 3], wv[:, 2], wv[:, 3]], axis=1)
    return O.bispectrum(In, pairs)


def box_to_grid_index(N: int, K: int, R: int):
    """(row, col) of the spectrum box -> centred oracle grid indices."""
    rows = np.arange(K + R + 1)
    cols = np.arange(2 * K + 1)
    ky = rows - R
    kx = cols - K
    return ky + N // 2, kx + N // 2


def gpu_channel(name: str, **kw):
    from paper_1701_00581_gb300 import Channel
    c = case(name)
    sp = c["spec"]
    return Channel(W=sp.W, H=sp.H, N=c["N"], R=c["R"], stride=c["stride"], fc=FC, taper=c["taper"],
                   max_frames=max(sp.F, 1), **kw)


def gpu_run(plan, frames_np: np.ndarray, stf_np: np.ndarray, chunk: int = None):
    """Every stage through the C ABI; returns host copies of every buffer."""
    import torch
    F = frames_np.shape[0]
    n = plan.info["n_sub"]
    chunk = n if chunk is None else chunk
    dev = f"cuda:{plan.device}"
    frames = torch.from_numpy(frames_np).to(dev)
    stf = torch.from_numpy(np.ascontiguousarray(stf_np, dtype=np.float64)).to(dev)
    ws, lay = plan.workspace(F, chunk)
    out = torch.zeros((plan.ch.H, plan.ch.W), dtype=torch.float32, device=dev)
    valid = torch.zeros((plan.ch.H, plan.ch.W), dtype=torch.uint8, device=dev)
    res = {k: [] for k in ("spec", "flux", "mu", "P", "M", "noise", "A", "B", "z")}
    for s0 in range(0, n, chunk):
        ns = min(chunk, n - s0)
        plan.stage_spectra(frames, F, s0, ns, ws, lay)
        plan.stage_stats(F, ns, ws, lay)
        plan.stage_amplitude(ns, stf, ws, lay)
        plan.stage_bispectrum(F, ns, ws, lay)
        plan.stage_phase(ns, ws, lay)
        plan.stage_inverse(F, s0, ns, ws, lay)
        torch.cuda.synchronize()
        v = plan.views(ws, lay, F, ns)
        for k in res:
            t = v[k]
            if t.dtype in (torch.float16, torch.bfloat16):
                t = t.float()
            res[k].append(t.cpu().numpy().copy())
    plan.stage_mosaic(ws, lay, out, valid)
    torch.cuda.synchronize()
    v = plan.views(ws, lay, F, 1)
    out_np = {k: np.concatenate(vals, axis=0) for k, vals in res.items()}
    out_np["rec"] = v["rec"].cpu().numpy().copy()
    out_np["out"] = out.cpu().numpy()
    out_np["valid"] = valid.cpu().numpy().astype(bool)
    return out_np
