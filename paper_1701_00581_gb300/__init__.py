"""GB300 speckle-masking reconstruction (Li et al., arXiv:1701.00581), Python side.

A thin binding of the C ABI in ``include/speckle.h``: it marshals arguments,
and uses PyTorch only for device memory and streams.  Every step of the
reconstruction runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Dict, Optional, Sequence

import numpy as np

from . import _lib
from ._lib import (SM_ACC_KAHAN, SM_ACC_PLAIN, SM_BATCH_FUSED, SM_BATCH_GRID, SM_BATCH_TILES, SM_BF16, SM_EDGE_DROP, SM_EDGE_PAD, SM_F32,  # noqa: F401
                   SM_FP16, SM_FP32, SM_MOSAIC_BLEND, SM_MOSAIC_CENTRAL,
                   SM_PHASE_FF, SM_PHASE_FP32, SM_PHASE_FP64, SM_U16, SM_W_BISPEC, SM_W_SNR, SM_W_UNIT, SpeckleError,
                   check, load)

__all__ = ["Channel", "Plan", "Batch", "Engine", "load", "SpeckleError"]


@dataclasses.dataclass
class Channel:
    """One camera channel (sm_channel)."""
    W: int
    H: int
    N: int
    R: int
    stride: Optional[int] = None
    fc: float = 0.2885
    taper: Optional[int] = None
    spectra_prec: int = SM_FP32
    phase_weight: int = SM_W_BISPEC
    ck: float = 0.435
    max_frames: int = 100
    acc_mode: int = SM_ACC_PLAIN
    phase_prec: int = SM_PHASE_FP32
    phase_iters: int = 0
    edge_mode: int = SM_EDGE_PAD
    mosaic_mode: int = SM_MOSAIC_BLEND
    photon_gain: float = 0.0

    def to_c(self) -> _lib.sm_channel:
        return _lib.sm_channel(
            self.W, self.H, self.N, self.stride if self.stride is not None else self.N // 2, self.R,
            self.fc, self.taper if self.taper is not None else self.N // 8, self.spectra_prec,
            self.phase_weight, self.ck, self.max_frames, self.acc_mode, self.phase_prec, self.phase_iters,
            self.edge_mode, self.mosaic_mode, self.photon_gain)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Plan:
    """sm_plan: tables of one channel on one device, plus the stage calls."""

    def __init__(self, ch: Channel, device: int = 0):
        self.lib = load()
        self.ch = ch
        self.device = device
        self._c = ch.to_c()
        h = C.c_void_p()
        check(self.lib.sm_plan_create(C.byref(self._c), device, C.byref(h)), "sm_plan_create")
        self.h = h
        inf = _lib.sm_plan_info()
        check(self.lib.sm_plan_get_info(self.h, C.byref(inf)), "sm_plan_get_info")
        self.info = {n: getattr(inf, n) for n, _ in _lib.sm_plan_info._fields_}

    def close(self):
        if self.h:
            self.lib.sm_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- host queries -------------------------------------------------------
    def subfields(self) -> np.ndarray:
        out = np.zeros((self.info["n_sub"], 4), dtype=np.int32)
        check(self.lib.sm_plan_subfields(self.h, out.ctypes.data), "sm_plan_subfields")
        return out

    def cubes(self) -> np.ndarray:
        """Subfield indices of the seeing cubes (sm_plan_cubes)."""
        out = np.zeros(self.info["n_cubes"], dtype=np.int32)
        check(self.lib.sm_plan_cubes(self.h, out.ctypes.data if len(out) else None), "sm_plan_cubes")
        return out

    def pair_index(self, wv: np.ndarray) -> np.ndarray:
        wv = np.ascontiguousarray(wv, dtype=np.int32).reshape(-1, 4)
        idx = np.zeros(len(wv), dtype=np.int64)
        check(self.lib.sm_plan_pair_index(self.h, len(wv), wv.ctypes.data, idx.ctypes.data),
              "sm_plan_pair_index")
        return idx

    def model_stf(self, d_over_r0: Sequence[float]) -> np.ndarray:
        d = np.ascontiguousarray(d_over_r0, dtype=np.float64)
        out = np.zeros((self.ch.N, self.ch.N))
        check(self.lib.sm_model_stf(C.byref(self._c), len(d), d.ctypes.data, out.ctypes.data),
              "sm_model_stf")
        return out

    def layout(self, F: int, chunk: int) -> _lib.sm_workspace_layout:
        lay = _lib.sm_workspace_layout()
        check(self.lib.sm_workspace_query(self.h, F, chunk, C.byref(lay)), "sm_workspace_query")
        return lay

    # ---- device buffers -----------------------------------------------------
    def workspace(self, F: int, chunk: int):
        import torch
        lay = self.layout(F, chunk)
        ws = torch.empty(lay.bytes + 256, dtype=torch.uint8, device=f"cuda:{self.device}")
        off = (-ws.data_ptr()) % 256
        return ws[off:off + lay.bytes], lay

    def views(self, ws, lay, F: int, nsub: int) -> Dict[str, "torch.Tensor"]:
        """Typed tensor views of the workspace buffers (layouts of speckle.h)."""
        import torch
        i = self.info
        box = i["box_rows"] * i["box_pitch"]
        hb = i["hb_rows"] * i["box_pitch"]

        def v(off, n, dt, shape):
            nb = n * torch.empty((), dtype=dt).element_size()
            return ws[off:off + nb].view(dt).reshape(shape)

        prec = self.ch.spectra_prec
        if prec == SM_FP32:
            spec = v(lay.spec, nsub * F * box, torch.complex64, (nsub, F, i["box_rows"], i["box_pitch"]))
        else:
            dt = torch.float16 if prec == SM_FP16 else torch.bfloat16
            spec = v(lay.spec, nsub * F * box * 2, dt, (nsub, F, i["box_rows"], i["box_pitch"], 2))
        N = i["N"]
        return {
            "spec": spec,
            "flux": v(lay.flux, nsub * F, torch.float32, (nsub, F)),
            "mu": v(lay.mu, nsub * F, torch.float32, (nsub, F)),
            "P": v(lay.P, nsub * hb, torch.float32, (nsub, i["hb_rows"], i["box_pitch"])),
            "M": v(lay.M, nsub * hb, torch.complex64, (nsub, i["hb_rows"], i["box_pitch"])),
            "noise": v(lay.noise, nsub, torch.float32, (nsub,)),
            "A": v(lay.A, nsub * hb, torch.float32, (nsub, i["hb_rows"], i["box_pitch"])),
            "B": v(lay.B, nsub * i["n_tiles"] * i["tile_pairs"], torch.complex64,
                   (nsub, i["n_tiles"] * i["tile_pairs"])),
            "z": v(lay.z, nsub * hb, torch.complex128, (nsub, i["hb_rows"], i["box_pitch"])),
            "rec": v(lay.rec, i["n_sub"] * N * N, torch.float32, (i["n_sub"], N, N)),
            "seeing": v(lay.seeing, i["n_cubes"] + 1, torch.float64, (i["n_cubes"] + 1,)),
            "stf": v(lay.stf, N * N, torch.float64, (N, N)),
        }

    # ---- stage entry points (device tensors) -------------------------------
    def stage_gain(self, flat, dark, gain, stream=None):
        """sm_stage_gain: normalised detector gain from a flat and a dark (device float [H][W])."""
        check(self.lib.sm_stage_gain(self.h, _ptr(flat), _ptr(dark), _ptr(gain), _stream(stream)), "sm_stage_gain")

    def stage_calibrate(self, raw, F, dark, gain, out, stream=None):
        """sm_stage_calibrate: (raw - dark) / gain into float32 frames."""
        check(self.lib.sm_stage_calibrate(self.h, _ptr(raw), _frame_type(raw), F, _ptr(dark), _ptr(gain), _ptr(out),
                                          _stream(stream)), "sm_stage_calibrate")

    def stage_track(self, frames, F, ref, G, S, ref_window, cc, shifts, stream=None):
        """sm_stage_track: integer shifts (sx, sy) of every frame against frame `ref`."""
        check(self.lib.sm_stage_track(self.h, _ptr(frames), _frame_type(frames), F, ref, G, S, _ptr(ref_window),
                                      _ptr(cc), _ptr(shifts), _stream(stream)), "sm_stage_track")

    def stage_shift(self, frames, F, shifts, out, stream=None):
        """sm_stage_shift: frames shifted by their (sx, sy), edges replicated, into float32."""
        check(self.lib.sm_stage_shift(self.h, _ptr(frames), _frame_type(frames), F, _ptr(shifts), _ptr(out),
                                      _stream(stream)), "sm_stage_shift")

    def stage_spectra(self, frames, F, sub0, nsub, ws, lay, stream=None):
        ft = SM_U16 if frames.dtype.__str__().endswith("uint16") else SM_F32
        check(self.lib.sm_stage_spectra(self.h, _ptr(frames), ft, F, sub0, nsub, _ptr(ws), C.byref(lay),
                                        _stream(stream)), "sm_stage_spectra")

    def stage_stats(self, F, nsub, ws, lay, stream=None):
        check(self.lib.sm_stage_stats(self.h, F, nsub, _ptr(ws), C.byref(lay), _stream(stream)),
              "sm_stage_stats")

    def stage_amplitude(self, nsub, stf, ws, lay, stream=None):
        check(self.lib.sm_stage_amplitude(self.h, nsub, _ptr(stf), _ptr(ws), C.byref(lay), _stream(stream)),
              "sm_stage_amplitude")

    def stage_seeing(self, F, sub0, nsub, ws, lay, stream=None):
        check(self.lib.sm_stage_seeing(self.h, F, sub0, nsub, _ptr(ws), C.byref(lay), _stream(stream)),
              "sm_stage_seeing")

    def stage_seeing_stf(self, ws, lay, stream=None):
        check(self.lib.sm_stage_seeing_stf(self.h, _ptr(ws), C.byref(lay), _stream(stream)),
              "sm_stage_seeing_stf")

    def stage_bispectrum(self, F, nsub, ws, lay, stream=None):
        check(self.lib.sm_stage_bispectrum(self.h, F, nsub, _ptr(ws), C.byref(lay), _stream(stream)),
              "sm_stage_bispectrum")

    def stage_phase(self, nsub, ws, lay, stream=None):
        check(self.lib.sm_stage_phase(self.h, nsub, _ptr(ws), C.byref(lay), _stream(stream)), "sm_stage_phase")

    def stage_inverse(self, F, sub0, nsub, ws, lay, stream=None):
        check(self.lib.sm_stage_inverse(self.h, F, sub0, nsub, _ptr(ws), C.byref(lay), _stream(stream)),
              "sm_stage_inverse")

    def stage_mosaic(self, ws, lay, out, valid=None, stream=None):
        check(self.lib.sm_stage_mosaic(self.h, _ptr(ws), C.byref(lay), _ptr(out), _ptr(valid),
                                       _stream(stream)), "sm_stage_mosaic")

    def reconstruct(self, frames, F, stf, chunk, ws, lay, out, valid=None, stream=None):
        """sm_reconstruct; stf None estimates the seeing from the burst (Sect. 3.1)."""
        ft = SM_U16 if str(frames.dtype).endswith("uint16") else SM_F32
        check(self.lib.sm_reconstruct(self.h, _ptr(frames), ft, F, _ptr(stf), chunk, _ptr(ws), C.byref(lay),
                                      _ptr(out), _ptr(valid), _stream(stream)), "sm_reconstruct")

    def reconstruct_noalloc(self, frames, F, stf, out, valid=None, stream=None):
        """sm_reconstruct_noalloc: the whole path on the library's fixed scratch array,
        for callers that may not allocate device memory while running."""
        check(self.lib.sm_reconstruct_noalloc(self.h, _ptr(frames), _frame_type(frames), F, _ptr(stf),
                                              _ptr(out), _ptr(valid), _stream(stream)),
              "sm_reconstruct_noalloc")


def _frame_type(frames) -> int:
    return SM_U16 if str(frames.dtype).endswith("uint16") else SM_F32


class Batch:
    """sm_batch: several bursts' spectra and bispectra in one persistent launch.

    ``plans``: one Plan per burst (channels may differ); ``F`` and
    ``frame_types`` per burst.  The work queue is built once here."""

    def __init__(self, plans: Sequence[Plan], F: Sequence[int], frame_types: Sequence[int], lookahead: int = 0,
                 ctas_per_sm: int = 0, launch: int = 0, tile_order: int = 0):
        """0 for an option takes the tuned value (sm_batch_opts)."""
        self.lib = load()
        self.plans = list(plans)
        n = len(self.plans)
        arr = (C.c_void_p * n)(*[p.h.value for p in self.plans])
        Fs = (C.c_int * n)(*F)
        fts = (C.c_int * n)(*frame_types)
        h = C.c_void_p()
        opts = _lib.sm_batch_opts(lookahead, ctas_per_sm, launch, tile_order)
        check(self.lib.sm_batch_create(n, arr, Fs, fts, C.byref(opts), C.byref(h)), "sm_batch_create")
        self.h = h
        got = _lib.sm_batch_opts()
        check(self.lib.sm_batch_get_opts(self.h, C.byref(got)), "sm_batch_get_opts")
        self.opts = {"lookahead": got.lookahead, "ctas_per_sm": got.ctas_per_sm, "launch": got.launch,
                     "tile_order": got.tile_order}
        ni, grid, nb = C.c_int(), C.c_int(), C.c_size_t()
        check(self.lib.sm_batch_info(self.h, C.byref(ni), C.byref(grid), C.byref(nb)), "sm_batch_info")
        self.info = {"n_items": ni.value, "grid": grid.value, "device_bytes": nb.value}

    def _io(self, items):
        """items: per burst a dict with frames, ws, lay, out and optionally stf, valid."""
        io = (_lib.sm_batch_io * len(items))()
        self._keep = []
        for i, it in enumerate(items):
            lay = it["lay"]
            self._keep.append(lay)
            io[i] = _lib.sm_batch_io(_ptr(it["frames"]), _ptr(it.get("stf")), _ptr(it["ws"]), C.pointer(lay),
                                     _ptr(it.get("out")), _ptr(it.get("valid")))
        return io

    def spectra_bispectrum(self, items, stream=None):
        check(self.lib.sm_batch_spectra_bispectrum(self.h, self._io(items), _stream(stream)),
              "sm_batch_spectra_bispectrum")

    def reconstruct(self, items, stream=None):
        check(self.lib.sm_batch_reconstruct(self.h, self._io(items), _stream(stream)), "sm_batch_reconstruct")

    def status(self) -> int:
        """SM_OK, or the error the last run recorded (synchronise the stream first)."""
        return self.lib.sm_batch_status(self.h)

    def close(self):
        if self.h:
            self.lib.sm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# sm_result.stage_ms, in order
STAGE_NAMES = ("spectra", "stats", "seeing", "modulus", "bispectrum", "phase", "inverse", "mosaic")


class Engine:
    """sm_open / sm_submit_burst / sm_poll / sm_close (the serving engine)."""

    def __init__(self, channels: Sequence[Channel], hbm_budget_bytes: int, max_inflight: int = 2,
                 device: int = 0, overlap_kernels: int = 0, allocator: Optional[str] = None):
        """``overlap_kernels``: 0 the bursts' kernels in submission order, 1
        concurrently, 2 pipelined (a burst's phase, inverse and mosaic beside
        the next burst's transforms and bispectrum), 3 batched (bursts
        submitted together run through one batched launch).  ``allocator="torch"``
        takes the engine's arena from torch's caching allocator (one uint8
        tensor held until close) instead of cudaMalloc."""
        self.lib = load()
        self._ch = (_lib.sm_channel * len(channels))(*[c.to_c() for c in channels])
        self.channels = list(channels)
        self._arena: Dict[int, object] = {}
        alloc, free = _lib.DEV_ALLOC(), _lib.DEV_FREE()    # NULL: cudaMalloc / cudaFree
        if allocator == "torch":
            import torch

            def _alloc(nbytes, _ctx):
                try:
                    t = torch.empty(int(nbytes), dtype=torch.uint8, device=f"cuda:{device}")
                except RuntimeError:
                    return None
                self._arena[t.data_ptr()] = t
                return t.data_ptr()

            def _free(ptr, _ctx):
                self._arena.pop(ptr, None)

            alloc, free = _lib.DEV_ALLOC(_alloc), _lib.DEV_FREE(_free)
        elif allocator is not None:
            raise ValueError("allocator must be None or 'torch'")
        self._callbacks = (alloc, free)          # kept alive while the engine holds them
        cfg = _lib.sm_config(len(channels), self._ch, hbm_budget_bytes, max_inflight, device,
                             int(overlap_kernels), alloc, free, None)
        h = C.c_void_p()
        check(self.lib.sm_open(C.byref(cfg), C.byref(h)), "sm_open")
        self.h = h
        self._keep: Dict[int, tuple] = {}

    def submit(self, channel: int, frames, out: np.ndarray, valid: Optional[np.ndarray] = None,
               stf: Optional[np.ndarray] = None, d_over_r0: Optional[np.ndarray] = None) -> int:
        """Returns a ticket, or raises SpeckleError (status SM_EBUSY when no slot is free).

        With neither ``stf`` nor ``d_over_r0`` the seeing is estimated on the
        device from the burst itself (Sect. 3.1)."""
        on_dev = not isinstance(frames, np.ndarray)
        ft = SM_U16 if str(frames.dtype).endswith("uint16") else SM_F32
        stf = None if stf is None else np.ascontiguousarray(stf, dtype=np.float64)
        d = None if d_over_r0 is None else np.ascontiguousarray(d_over_r0, dtype=np.float64)
        b = _lib.sm_burst(channel, frames.shape[0], _ptr(frames), ft, 1 if on_dev else 0,
                          _ptr(stf), _ptr(d), _ptr(out), _ptr(valid))
        t = C.c_uint64()
        check(self.lib.sm_submit_burst(self.h, C.byref(b), C.byref(t)), "sm_submit_burst")
        self._keep[t.value] = (out, valid)
        return t.value

    def submit_batch(self, bursts) -> list:
        """sm_submit_batch (engine opened with overlap_kernels=3): ``bursts`` is
        a list of dicts with channel, frames, out and optionally valid, stf,
        d_over_r0; returns one ticket per burst, or raises SpeckleError
        (SM_EBUSY when the whole batch cannot be admitted now)."""
        n = len(bursts)
        arr = (_lib.sm_burst * n)()
        keep = []
        for i, d in enumerate(bursts):
            frames = d["frames"]
            on_dev = not isinstance(frames, np.ndarray)
            ft = SM_U16 if str(frames.dtype).endswith("uint16") else SM_F32
            stf = None if d.get("stf") is None else np.ascontiguousarray(d["stf"], dtype=np.float64)
            dr0 = None if d.get("d_over_r0") is None else np.ascontiguousarray(d["d_over_r0"], dtype=np.float64)
            keep.append((stf, dr0))
            arr[i] = _lib.sm_burst(d["channel"], frames.shape[0], _ptr(frames), ft, 1 if on_dev else 0, _ptr(stf),
                                   _ptr(dr0), _ptr(d["out"]), _ptr(d.get("valid")))
        t = (C.c_uint64 * n)()
        check(self.lib.sm_submit_batch(self.h, n, arr, t), "sm_submit_batch")
        tickets = list(t)
        for tk, d in zip(tickets, bursts):
            self._keep[tk] = (d["out"], d.get("valid"))
        return tickets

    def try_submit_batch(self, bursts) -> Optional[list]:
        try:
            return self.submit_batch(bursts)
        except SpeckleError as e:
            if e.status == _lib.SM_EBUSY:
                return None
            raise

    def try_submit(self, *args, **kw) -> Optional[int]:
        try:
            return self.submit(*args, **kw)
        except SpeckleError as e:
            if e.status == _lib.SM_EBUSY:
                return None
            raise

    def poll(self, ticket: int, timeout_ms: int = -1):
        res = _lib.sm_result()
        st = self.lib.sm_poll(self.h, ticket, timeout_ms, C.byref(res))
        if st in (_lib.SM_PENDING, _lib.SM_ETIMEDOUT):
            return st, None
        check(st, "sm_poll")
        self._keep.pop(ticket, None)
        return st, {"t_submit_ms": res.t_submit_ms, "t_done_ms": res.t_done_ms, "gpu_ms": res.gpu_ms,
                    "bytes_admitted": res.bytes_admitted, "d_over_r0": res.d_over_r0,
                    "stage_ms": dict(zip(STAGE_NAMES, list(res.stage_ms)))}

    def close(self):
        if self.h:
            self.lib.sm_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
