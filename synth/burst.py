"""Seeded synthetic bursts shaped like NVST speckle data.

The paper reconstructs bursts of 100 short exposures from three NVST channels
(Table 1: H-alpha 1024x1024, TiO and G-band 2560x2160, 10 frames/s, 16-bit
camera).  No NVST data is available here, so these generators stand in for it:

* scene: a unit background plus Gaussian blobs (granulation-like), 40 blobs
  per 64x64 px, sigma ~ U[2, 4] px, amplitude ~ U[0.05, 0.3], periodic;
* seeing: one Kolmogorov phase screen per frame (FFT method, phase PSD
  0.023 r0^(-5/3) k^(-11/3), drawn on a grid twice the pupil grid and
  cropped) over a circular pupil whose diameter is ``fc * M`` pupil pixels on
  an M x M grid, so the optics cut off at ``fc`` cycles/px (0.2885 matches the
  TiO sampling of 0.042"/px against lambda/D = 0.146", Sect. 4);
* frames: the scene circularly convolved with the frame's PSF (isoplanatic),
  Gaussian noise with sigma = mean / 50, then either kept as float32 or
  scaled to a 2000-count mean, rounded and clipped to 12 bits as uint16.

Seeds: the scene of (channel, burst) draws from ``SeedSequence((2017, channel,
burst, 0xB10B))`` and frame f from ``SeedSequence((2017, channel, burst, f))``.
Nothing here is a step of the reconstruction.
"""
from __future__ import annotations

import dataclasses
import os
from typing import Optional, Tuple

import numpy as np

try:  # scipy's pocketfft can use several threads; numpy's cannot
    import scipy.fft as _fft

    _FFT_KW = {"workers": max(1, min(16, os.cpu_count() or 1))}
except Exception:  # pragma: no cover - scipy is in both images
    _fft = np.fft
    _FFT_KW = {}

FC_DEFAULT = 0.2885


@dataclasses.dataclass(frozen=True)
class BurstSpec:
    W: int
    H: int
    F: int
    N: int                      # PSF grid = subfield size, so the STF lives on the subfield grid
    dr0: Tuple[float, float]    # D/r0 drawn uniformly per frame from [lo, hi]
    counts: bool                # True: uint16 12-bit counts; False: float32
    fc: float = FC_DEFAULT
    snr: float = 50.0
    blob_density: float = 40.0 / 64.0 ** 2


CONFIGS = {
    # one 64x64 subfield, float32 frames, D/r0 = 6
    "subfield64": BurstSpec(W=64, H=64, F=100, N=64, dr0=(6.0, 6.0), counts=False),
    # H-alpha-shaped 1024x1024 burst, 128x128 subfields
    "halpha1024": BurstSpec(W=1024, H=1024, F=100, N=128, dr0=(5.0, 12.0), counts=True),
    # TiO-shaped 2560x2160 burst, 256x256 subfields
    "tio2560": BurstSpec(W=2560, H=2160, F=100, N=256, dr0=(8.0, 15.0), counts=True),
}


def _rng(*key: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(tuple(int(k) for k in key)))


def make_object(W: int, H: int, rng: np.random.Generator,
                density: float = 40.0 / 64.0 ** 2) -> np.ndarray:
    """Unit background plus periodic Gaussian blobs, float64 [H, W]."""
    n = max(1, int(round(density * W * H)))
    xs = rng.uniform(0, W, n)
    ys = rng.uniform(0, H, n)
    sig = rng.uniform(2.0, 4.0, n)
    amp = rng.uniform(0.05, 0.3, n)
    obj = np.ones((H, W), dtype=np.float64)
    for x, y, s, a in zip(xs, ys, sig, amp):
        r = int(np.ceil(4.0 * s))
        ix = np.arange(int(np.floor(x)) - r, int(np.floor(x)) + r + 2)
        iy = np.arange(int(np.floor(y)) - r, int(np.floor(y)) + r + 2)
        gx = np.exp(-0.5 * ((ix - x) / s) ** 2)
        gy = np.exp(-0.5 * ((iy - y) / s) ** 2)
        patch = a * np.outer(gy, gx)
        np.add.at(obj, (np.mod(iy, H)[:, None], np.mod(ix, W)[None, :]), patch)
    return obj


def _pupil(M: int, fc: float) -> np.ndarray:
    dp = fc * M
    c = (M - 1) / 2.0
    y, x = np.mgrid[0:M, 0:M]
    return (((x - c) ** 2 + (y - c) ** 2) <= (dp / 2.0) ** 2).astype(np.float64)


def _psf_from_field(field: np.ndarray) -> np.ndarray:
    amp = np.fft.fft2(field)
    psf = (amp * amp.conj()).real
    return psf / psf.sum()          # origin at index [0, 0] (wrapped)


def diffraction_psf(M: int, fc: float = FC_DEFAULT) -> np.ndarray:
    """Unaberrated PSF of the circular pupil on an M x M grid, origin at [0, 0]."""
    return _psf_from_field(_pupil(M, fc).astype(np.complex128))


def kolmogorov_psf(M: int, d_over_r0: float, rng: np.random.Generator,
                   fc: float = FC_DEFAULT) -> np.ndarray:
    """Short-exposure PSF through one Kolmogorov phase screen (origin at [0, 0])."""
    dp = fc * M                      # pupil diameter in pupil pixels; D = 1 m
    dx = 1.0 / dp                    # metres per pupil pixel
    r0 = 1.0 / d_over_r0
    G = 2 * M                        # screen grid, cropped to the pupil grid
    f = np.fft.fftfreq(G, d=dx)      # cycles per metre
    fy, fx = np.meshgrid(f, f, indexing="ij")
    kap = np.hypot(fx, fy)
    kap[0, 0] = np.inf
    psd = 0.023 * r0 ** (-5.0 / 3.0) * kap ** (-11.0 / 3.0)
    dk = 1.0 / (G * dx)
    c = rng.standard_normal((G, G)) + 1j * rng.standard_normal((G, G))
    screen = (np.fft.ifft2(c * np.sqrt(psd) * dk) * (G * G)).real[:M, :M]
    return _psf_from_field(_pupil(M, fc) * np.exp(1j * screen))


def empirical_stf(psfs: np.ndarray) -> np.ndarray:
    """<|H_i|^2> of the given PSFs on their M x M grid, centred (index k + M/2)."""
    otf = np.fft.fft2(psfs, axes=(-2, -1))
    stf = np.mean((otf * otf.conj()).real, axis=0)
    return np.fft.fftshift(stf)


def _embed(psf: np.ndarray, H: int, W: int) -> np.ndarray:
    M = psf.shape[0]
    off = np.arange(M)
    off = np.where(off < M // 2, off, off - M)
    big = np.zeros((H, W), dtype=np.float64)
    np.add.at(big, (np.mod(off, H)[:, None], np.mod(off, W)[None, :]), psf)
    return big


def make_burst(spec: BurstSpec, channel: int = 0, burst: int = 0,
               device: Optional[str] = None, F: Optional[int] = None,
               psf: str = "kolmogorov", noise: bool = True) -> dict:
    """Generate one burst.

    Returns a dict with ``frames`` ([F, H, W] uint16 or float32), ``object``
    (float64 [H, W], in frame units), ``d_over_r0`` ([F] float64) and
    ``stf_emp`` (float64 [N, N], centred, from the frames' own PSFs).
    ``device`` (e.g. "cuda") runs the frame convolutions with torch.fft on
    that device; the random draws are the same numpy draws either way.
    ``psf="diffraction"`` gives seeing-free frames (all PSFs unaberrated).
    """
    F = spec.F if F is None else F
    obj = make_object(spec.W, spec.H, _rng(2017, channel, burst, 0xB10B), spec.blob_density)
    scale = 2000.0 / obj.mean() if spec.counts else 1.0
    frames = np.empty((F, spec.H, spec.W), dtype=np.uint16 if spec.counts else np.float32)
    dr0 = np.empty(F)
    psfs = np.empty((F, spec.N, spec.N))
    rngs = [_rng(2017, channel, burst, f) for f in range(F)]
    for f in range(F):
        lo, hi = spec.dr0
        dr0[f] = lo if hi == lo else rngs[f].uniform(lo, hi)
        if psf == "diffraction":
            psfs[f] = diffraction_psf(spec.N, spec.fc)
        else:
            psfs[f] = kolmogorov_psf(spec.N, dr0[f], rngs[f], spec.fc)
    if device is not None:
        import torch
        o_t = torch.fft.rfft2(torch.as_tensor(obj * scale, device=device))
    else:
        o_np = _fft.rfft2(obj * scale, **_FFT_KW)
    for f in range(F):
        big = _embed(psfs[f], spec.H, spec.W)
        if device is not None:
            import torch
            img = torch.fft.irfft2(o_t * torch.fft.rfft2(torch.as_tensor(big, device=device)),
                                   s=(spec.H, spec.W)).cpu().numpy()
        else:
            img = _fft.irfft2(o_np * _fft.rfft2(big, **_FFT_KW), s=(spec.H, spec.W), **_FFT_KW)
        if noise:
            img = img + rngs[f].standard_normal(img.shape) * (img.mean() / spec.snr)
        if spec.counts:
            frames[f] = np.clip(np.rint(img), 0, 4095).astype(np.uint16)
        else:
            frames[f] = img.astype(np.float32)
    return {
        "frames": frames,
        "object": obj * scale,
        "d_over_r0": dr0,
        "stf_emp": empirical_stf(psfs),
        "spec": spec,
    }
