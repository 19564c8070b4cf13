"""Run oracle work items in parallel on the host cores (test infrastructure).

The GPU tests call the FP64 oracle on many subfields of a full-size burst;
one subfield takes tens of seconds in numpy, so the items go to a pool of
worker processes, one per host core.  The pool uses the ``spawn`` start
method: the calling process has a CUDA context, and a forked child of it
would inherit that context in an unusable state.  Frames reach the workers
as a memory-mapped ``.npy`` file and large results come back the same way.
Every number here is computed by ``oracle``; nothing is taken from the GPU.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from typing import Callable, List, Sequence

import numpy as np


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - not Linux
        return os.cpu_count() or 1


def pool_map(fn: Callable, tasks: Sequence, workers: int = None) -> List:
    """fn over tasks in spawned worker processes (BLAS threads pinned to one
    per worker, so the cores are not oversubscribed)."""
    n = max(1, min(workers or host_cores(), len(tasks)))
    keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in keep:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(n) as pool:
            return pool.map(fn, tasks, chunksize=1)
    finally:
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def cube_seeing(task) -> float:
    """Oracle D/r0 of one seeing cube (Sect. 3.1) from the frames file."""
    from oracle import speckle_oracle as O
    path, sub, N, fc, taper = task
    frames = np.load(path, mmap_mode="r")
    In, _, _ = O.frame_spectra(frames, sub, N, taper)
    P, M = O.power_mean(In)
    num, den = O.spectral_ratio(P, M, O.noise_floor(P, N, fc), frames.shape[0], N, fc)
    return O.fit_d_over_r0(num, den, N, fc)


def used_pairs(N: int, R: int, fc: float) -> np.ndarray:
    """(wx, wy, vx, vy) of every pair the phase recursion reads."""
    from oracle import speckle_oracle as O
    return O.recursion_splits(N, fc, R)


def subfield_whole(task) -> dict:
    """Oracle P, M, noise, A, B on every used pair, z and the sub-image of one
    subfield, with the given STF; B goes to ``<outdir>/B_<s>.npy``."""
    from oracle import speckle_oracle as O
    path, s, sub, N, fc, R, taper, stf, outdir = task
    frames = np.load(path, mmap_mode="r")
    In, flux, mu = O.frame_spectra(frames, sub, N, taper)
    P, M = O.power_mean(In)
    noise = O.noise_floor(P, N, fc)
    A = O.amplitude(P, noise, stf, N, fc)
    wv = used_pairs(N, R, fc)
    u = wv[:, :2] - wv[:, 2:]
    # B(w - v, v) at each used pair, then the same values in the oracle's
    # stored representation (u in the upper half plane; lower-half u as
    # conj B(-u, -v)) for the recursion
    Bw = O.bispectrum(In, np.concatenate([u, wv[:, 2:]], 1))
    up = O.in_half_plane(u[:, 0], u[:, 1])
    pairs = np.where(up[:, None], np.concatenate([u, wv[:, 2:]], 1), -np.concatenate([u, wv[:, 2:]], 1))
    Bst = np.where(up, Bw, np.conj(Bw))
    z = O.phase_recursion(Bst, pairs, M, N, fc, R)
    rec = O.inverse(A, z, float(flux.mean()), float(mu.mean()), O.window2d(sub[2], sub[3], taper))
    np.save(os.path.join(outdir, f"B_{s}.npy"), Bw)
    return {"s": s, "P": P, "M": M, "noise": noise, "A": A, "z": z, "rec": rec,
            "flux": flux, "mu": mu}


def subfield_image(task) -> tuple:
    """Oracle sub-image of one subfield with the given STF (the steps of
    ``subfield_whole`` on the used pairs, keeping only the image)."""
    from oracle import speckle_oracle as O
    path, s, sub, N, fc, R, taper, stf = task
    frames = np.load(path, mmap_mode="r")
    In, flux, mu = O.frame_spectra(frames, sub, N, taper)
    P, M = O.power_mean(In)
    A = O.amplitude(P, O.noise_floor(P, N, fc), stf, N, fc)
    wv = used_pairs(N, R, fc)
    u = wv[:, :2] - wv[:, 2:]
    Bw = O.bispectrum(In, np.concatenate([u, wv[:, 2:]], 1))
    up = O.in_half_plane(u[:, 0], u[:, 1])
    pairs = np.where(up[:, None], np.concatenate([u, wv[:, 2:]], 1), -np.concatenate([u, wv[:, 2:]], 1))
    z = O.phase_recursion(np.where(up, Bw, np.conj(Bw)), pairs, M, N, fc, R)
    rec = O.inverse(A, z, float(flux.mean()), float(mu.mean()), O.window2d(sub[2], sub[3], taper))
    return s, rec
