"""FP64 CPU oracle of the speckle-masking reconstruction path.

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``;
the product path (the CUDA library and its Python binding) never imports,
links or runs it, and it imports nothing from the product.

It is a plain, slow, obviously correct restatement of what the paper
computes, in float64 numpy, one function per step.  The paper (Li et al.,
"High Performance Parallel Image Reconstruction for New Vacuum Solar
Telescope") names the steps but prints only Eq. 1; every other formula is
the standard one of the methods it cites (Labeyrie 1970 for the modulus;
Weigelt 1977 and Lohmann, Weigelt & Wirnitzer 1983 for the bispectrum and
the recursive phase).  Where the paper is silent the reading taken here is
stated in each docstring:

* flat/dark preprocessing (Table 2's first row): (raw - dark) / gain with
  the gain (flat - dark) normalised to mean 1;
* correlation tracking (Table 2): integer shifts maximising the cross-
  correlation with a reference frame over a central window, applied with
  the edges replicated;
* subfield grid (Sect. 2, Sect. 3.2): stride N/2, ``ceil((W-N)/s)+1`` tiles
  per axis, edge tiles keep their true extent and are zero-padded to N x N;
* apodisation (silent): separable Tukey window, taper ``t`` px per edge;
* DFT (Sect. 2): centred frequencies k in [-N/2, N/2) of the windowed,
  mean-subtracted tile, each frame divided by its windowed flux, DC := 1;
* power and mean spectrum (Sect. 3.2, Eq. 1 numerator), noise floor as the
  mean power in the half-plane corners of the (2K+1)^2 box outside the disk;
* optional photon-noise bias removal from the bispectrum (Wirnitzer 1985),
  the counts' photons per count given;
* bispectrum (Sect. 2, Sect. 3.2; Weigelt 1977) on the pair domain
  D = {u in upper half plane, |u| <= r, 0 < |v| <= R, |u+v| <= r};
* seeing (Sect. 3.1; von der Luehe 1984): D/r0 of every non-overlapping
  N x N cube by a least-squares fit of a model spectral ratio (Fried's
  long-exposure OTF squared over the model STF) to the observed one, r0
  averaged over the cubes;
* modulus (Sect. 3.2, Eq. 1) with a model STF (Sect. 3.2), filtered by the
  diffraction OTF T0;
* recursive phase (Sect. 3.2; LWW 1983), rings of equal |w|^2, anchors from
  the burst-mean spectrum, |B| weighting by default (unit and SNR weights
  as options), optionally refined by least-squares sweeps (the "or
  iteratively" of the method);
* inverse DFT, flux rescale and the mean restored under the window
  (Sect. 2, Sect. 3.2), mosaic as
  sum(rec) / sum(window) (Sect. 3.2, the merge step).

Parity of every function here is pinned by ``tests/test_oracle_pins.py``
against brute force, closed forms, invariants and library routines.
Model-STF fidelity to real seeing (the Korff constant) is parity unpinned:
the paper prints no STF model.
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

W_BISPEC = 0     # phasor terms weighted by |B| (the plain sum of B's phasors)
W_UNIT = 1       # unit-modulus phasor terms
W_SNR = 2        # terms weighted by |B| / (P(u) P(v) P(w)), i.e. |B|^2 over its speckle-noise variance


# ----------------------------------------------------------------------------
# front end (Table 2: flat/dark preprocessing)
# ----------------------------------------------------------------------------
def calib_gain(flat: np.ndarray, dark: np.ndarray) -> np.ndarray:
    """Normalised gain map of the detector: g = (flat - dark) / mean(flat - dark),
    the mean over the pixels where flat > dark; g = 0 where flat <= dark
    (dead pixels; reading: the paper names the step only)."""
    d = np.asarray(flat, dtype=np.float64) - np.asarray(dark, dtype=np.float64)
    live = d > 0
    if not live.any():
        raise ValueError("flat is nowhere above dark")
    return np.where(live, d / d[live].mean(), 0.0)


def calibrate(raw: np.ndarray, dark: np.ndarray, gain: np.ndarray) -> np.ndarray:
    """Flat/dark correction of every frame: (raw - dark) / gain, 0 where gain = 0."""
    raw = np.asarray(raw, dtype=np.float64)
    g = np.asarray(gain, dtype=np.float64)
    safe = np.where(g > 0, g, 1.0)
    return np.where(g > 0, (raw - np.asarray(dark, dtype=np.float64)) / safe, 0.0)


def track_window(W: int, H: int, G: int, S: int) -> Tuple[int, int]:
    """Origin (x0, y0) of the central G x G tracking window; the window moved
    by any shift within +-S must stay inside the frame."""
    x0, y0 = (W - G) // 2, (H - G) // 2
    if G < 1 or S < 0 or x0 < S or y0 < S or x0 + G + S > W or y0 + G + S > H:
        raise ValueError("tracking window plus search range does not fit the frame")
    return x0, y0


def track_shifts(frames: np.ndarray, ref: int, G: int, S: int) -> Tuple[np.ndarray, np.ndarray]:
    """Correlation tracking (Table 2): per frame the integer shift (sx, sy),
    |sx|, |sy| <= S, maximising C(s) = sum over the central G x G window W
    of a(x + s) (r(x) - mean_W r), r the reference frame; the first maximum
    in the order sy = -S..S, then sx = -S..S.  Returns shifts [F][2] (sx, sy)
    and C [F][2S+1][2S+1] (row sy + S, column sx + S).
    (Readings: the paper names the step only; reference = one frame of the
    burst, integer shifts.)"""
    frames = np.asarray(frames, dtype=np.float64)
    F, H, W = frames.shape
    x0, y0 = track_window(W, H, G, S)
    r = frames[ref, y0:y0 + G, x0:x0 + G]
    r = r - r.mean()
    C = np.zeros((F, 2 * S + 1, 2 * S + 1))
    for f in range(F):
        for sy in range(-S, S + 1):
            for sx in range(-S, S + 1):
                C[f, sy + S, sx + S] = np.sum(frames[f, y0 + sy:y0 + sy + G, x0 + sx:x0 + sx + G] * r)
    shifts = np.zeros((F, 2), dtype=np.int64)
    for f in range(F):
        k = int(np.argmax(C[f]))                   # first maximum in row-major order
        shifts[f] = (k % (2 * S + 1) - S, k // (2 * S + 1) - S)
    return shifts, C


def apply_shifts(frames: np.ndarray, shifts: np.ndarray) -> np.ndarray:
    """Aligned frames out_f(x, y) = a_f(x + sx, y + sy), coordinates clamped
    to the frame (edge pixels replicated; reading)."""
    frames = np.asarray(frames, dtype=np.float64)
    F, H, W = frames.shape
    out = np.empty_like(frames)
    ys, xs = np.arange(H), np.arange(W)
    for f in range(F):
        sx, sy = int(shifts[f][0]), int(shifts[f][1])
        yy = np.clip(ys + sy, 0, H - 1)
        xx = np.clip(xs + sx, 0, W - 1)
        out[f] = frames[f][np.ix_(yy, xx)]
    return out


# ----------------------------------------------------------------------------
# subfields and window (Sect. 2: partially overlapping subimage cubes)
# ----------------------------------------------------------------------------
def subfield_grid(W: int, H: int, N: int, stride: int,
                  drop_edge: bool = False) -> List[Tuple[int, int, int, int]]:
    """Overlapping subfields (x0, y0, w, h), row-major over y then x.

    The paper cuts each frame into partially overlapping cubes matching the
    isoplanatic patch (Sect. 2, Sect. 3.2).  Reading: tiles start every
    ``stride`` px; a ragged last tile keeps its true extent ``w, h < N``.
    With ``drop_edge`` only full N x N tiles are kept: at stride 64 this is
    the paper's own 37 x 30 = 1110 cubes of a 2560 x 2160 burst (Sect. 3.2).
    """
    def starts(L: int) -> List[int]:
        if drop_edge:
            return [k * stride for k in range((L - N) // stride + 1)] if L >= N else []
        n = 1 if L <= N else int(math.ceil((L - N) / stride)) + 1
        return [k * stride for k in range(n)]

    out = []
    for y0 in starts(H):
        for x0 in starts(W):
            out.append((x0, y0, min(N, W - x0), min(N, H - y0)))
    return out


def tukey(L: int, taper: int) -> np.ndarray:
    """1-D window of length L: raised-cosine ramps of ``taper`` px at both ends.

    Ramp value at pixel x is (1 - cos(pi (x + 1/2) / taper)) / 2 for
    x < taper, 1 beyond; the window is the smaller of the rising ramp read
    from each end, so it is symmetric and strictly positive.  taper = 0
    gives all ones (no apodisation).
    """
    x = np.arange(L, dtype=np.float64)
    if taper <= 0:
        return np.ones(L)

    def ramp(p: np.ndarray) -> np.ndarray:
        return np.where(p < taper, 0.5 * (1.0 - np.cos(np.pi * (p + 0.5) / taper)), 1.0)

    return np.minimum(ramp(x), ramp(L - 1 - x))


def window2d(w: int, h: int, taper: int) -> np.ndarray:
    """Separable apodisation window [h, w]."""
    return np.outer(tukey(h, taper), tukey(w, taper))


# ----------------------------------------------------------------------------
# DFT (Sect. 2: Fourier transform of every subimage)
# ----------------------------------------------------------------------------
def dft_matrix(N: int, sign: int = -1) -> np.ndarray:
    """E[k + N/2, x] = exp(sign * 2 pi i k x / N) for k in [-N/2, N/2)."""
    k = np.arange(-(N // 2), N - N // 2, dtype=np.float64)
    x = np.arange(N, dtype=np.float64)
    return np.exp(sign * 2j * np.pi * np.outer(k, x) / N)


def dft2(t: np.ndarray) -> np.ndarray:
    """I[ky + N/2, kx + N/2] = sum_{y,x} t[y, x] exp(-2 pi i (kx x + ky y) / N).

    Separable: the x sums (rows) then the y sums (columns), each as a
    product with the DFT matrix.
    """
    N = t.shape[0]
    E = dft_matrix(N, -1)
    rows = t @ E.T           # [y, kx]
    return E @ rows          # [ky, kx]


def idft2(I: np.ndarray) -> np.ndarray:
    """Inverse of dft2: (1/N^2) sum_k I(k) exp(+2 pi i k.x / N), complex [y, x]."""
    N = I.shape[0]
    E = dft_matrix(N, +1)    # [k, x]
    return (E.T @ I @ E) / (N * N)


def frame_spectra(frames: np.ndarray, sub: Tuple[int, int, int, int], N: int,
                  taper: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Normalised spectra of one subfield's frames.

    For frame i the tile of extent w x h at (x0, y0) has windowed mean
    mu_i = sum(w raw_i) / sum(w); the tile w (raw_i - mu_i) is zero-padded to
    N x N at the low corner and transformed, and the spectrum is divided by
    the frame's windowed flux f_i = mu_i sum(w).  The DC value is then set to
    1 (the normalised mean).  Subtracting the mean before the transform keeps
    the window's own spectrum, scaled by the bright background, out of the
    object's spectrum (reading; the paper names no apodisation).
    Returns (In [F, N, N] complex128 centred, flux [F], mu [F]).
    """
    x0, y0, w, h = sub
    win = window2d(w, h, taper)
    F = frames.shape[0]
    In = np.empty((F, N, N), dtype=np.complex128)
    flux = np.empty(F)
    mu = np.empty(F)
    for i in range(F):
        raw = frames[i, y0:y0 + h, x0:x0 + w].astype(np.float64)
        mu[i] = (win * raw).sum() / win.sum()
        flux[i] = mu[i] * win.sum()
        t = np.zeros((N, N))
        t[:h, :w] = win * (raw - mu[i])
        In[i] = dft2(t) / flux[i]
        In[i, N // 2, N // 2] = 1.0
    return In, flux, mu


# ----------------------------------------------------------------------------
# frequency domains
# ----------------------------------------------------------------------------
def cutoff_radius(N: int, fc: float) -> float:
    """Radius of the frequency disk U in frequency pixels (fc in cycles/px)."""
    return fc * N


def in_half_plane(kx: np.ndarray, ky: np.ndarray) -> np.ndarray:
    """Upper half plane used to store one of each Hermitian pair."""
    return (ky > 0) | ((ky == 0) & (kx > 0))


def domain_U(N: int, fc: float) -> np.ndarray:
    """All (kx, ky) with kx^2 + ky^2 <= r^2, r = fc N.  int64 [n, 2]."""
    r = cutoff_radius(N, fc)
    K = int(math.floor(r))
    ky, kx = np.mgrid[-K:K + 1, -K:K + 1]
    m = kx * kx + ky * ky <= r * r
    return np.stack([kx[m], ky[m]], axis=1).astype(np.int64)


def domain_V(R: int) -> np.ndarray:
    """Bispectrum offsets 0 < |v| <= R.  int64 [n, 2]."""
    ky, kx = np.mgrid[-R:R + 1, -R:R + 1]
    m = (kx * kx + ky * ky <= R * R) & ((kx != 0) | (ky != 0))
    return np.stack([kx[m], ky[m]], axis=1).astype(np.int64)


def pair_domain(N: int, fc: float, R: int) -> np.ndarray:
    """Pair domain D of the stored bispectrum, int64 [n, 4] = (ux, uy, vx, vy).

    u in the upper half plane with |u| <= r, v with 0 < |v| <= R and
    |u + v| <= r.  The rest of the bispectrum follows from
    B(-u, -v) = conj B(u, v) (real frames).
    """
    r2 = cutoff_radius(N, fc) ** 2
    U = domain_U(N, fc)
    U = U[in_half_plane(U[:, 0], U[:, 1])]
    V = domain_V(R)
    ux = np.repeat(U[:, 0], len(V))
    uy = np.repeat(U[:, 1], len(V))
    vx = np.tile(V[:, 0], len(U))
    vy = np.tile(V[:, 1], len(U))
    m = (ux + vx) ** 2 + (uy + vy) ** 2 <= r2
    return np.stack([ux[m], uy[m], vx[m], vy[m]], axis=1)


# ----------------------------------------------------------------------------
# power spectrum, mean spectrum, noise (Sect. 3.2, Eq. 1 numerator)
# ----------------------------------------------------------------------------
def power_mean(In: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """P = <|I_i|^2>_i and M = <I_i>_i on the full centred grid (Eq. 1 numerator)."""
    P = np.mean((In * In.conj()).real, axis=0)
    M = np.mean(In, axis=0)
    return P, M


def noise_floor(P: np.ndarray, N: int, fc: float) -> float:
    """Mean of P over {1 <= ky <= K, |kx| <= K, |k| > r}, K = floor(r).

    The optics pass nothing beyond r, so the power there is the flat
    additive-noise bias; by Hermitian symmetry the upper corners of the
    (2K+1)^2 box stand for all four.  (Reading; the paper gives no noise
    treatment.)
    """
    r = cutoff_radius(N, fc)
    K = int(math.floor(r))
    ky, kx = np.mgrid[1:K + 1, -K:K + 1]
    m = kx * kx + ky * ky > r * r
    if not m.any():
        return 0.0
    return float(P[ky[m] + N // 2, kx[m] + N // 2].mean())


# ----------------------------------------------------------------------------
# bispectrum (Sect. 2 and Sect. 3.2: speckle masking, Weigelt 1977)
# ----------------------------------------------------------------------------
def bispectrum(In: np.ndarray, pairs: np.ndarray) -> np.ndarray:
    """B(u, v) = (1/F) sum_i I_i(u) I_i(v) conj I_i(u + v) for each listed pair.

    ``In`` is [F, N, N] centred; ``pairs`` rows are (ux, uy, vx, vy).  A
    direct sum over frames, one frame at a time.
    """
    F, N, _ = In.shape
    c = N // 2
    ux, uy, vx, vy = (pairs[:, j] for j in range(4))
    B = np.zeros(len(pairs), dtype=np.complex128)
    for i in range(F):
        S = In[i]
        B += S[uy + c, ux + c] * S[vy + c, vx + c] * np.conj(S[uy + vy + c, ux + vx + c])
    return B / F


# ----------------------------------------------------------------------------
# modulus (Sect. 3.2, Eq. 1)
# ----------------------------------------------------------------------------
def otf_t0(N: int, fc: float) -> np.ndarray:
    """Diffraction OTF of a circular pupil on the centred N x N grid.

    T0(rho) = (2/pi)(acos rho - rho sqrt(1 - rho^2)) for rho = |k| / r <= 1.
    """
    r = cutoff_radius(N, fc)
    k = np.arange(-(N // 2), N - N // 2, dtype=np.float64)
    rho = np.hypot(k[None, :], k[:, None]) / r
    out = np.zeros((N, N))
    m = rho <= 1.0
    p = rho[m]
    out[m] = (2.0 / np.pi) * (np.arccos(p) - p * np.sqrt(1.0 - p * p))
    return out


def stf_model(N: int, fc: float, d_over_r0: Sequence[float], ck: float = 0.435) -> np.ndarray:
    """Model speckle transfer function on the centred grid (Sect. 3.2).

    Per frame, T0^2 exp(-6.88 (rho D/r0)^(5/3)) + ck (r0/D)^2 T0 (the
    long-exposure term squared plus the Korff speckle term); averaged over
    the frames and divided by its value at k = 0.  The paper calibrates a
    model STF with r0 but prints no model: the form and ``ck`` are readings
    (parity unpinned against real seeing).
    """
    r = cutoff_radius(N, fc)
    k = np.arange(-(N // 2), N - N // 2, dtype=np.float64)
    rho = np.hypot(k[None, :], k[:, None]) / r
    T0 = otf_t0(N, fc)
    acc = np.zeros((N, N))
    for d in d_over_r0:
        acc += T0 * T0 * np.exp(-6.88 * (rho * d) ** (5.0 / 3.0)) + ck * T0 / (d * d)
    acc /= len(d_over_r0)
    return acc / acc[N // 2, N // 2]


def amplitude(P: np.ndarray, noise: float, stf: np.ndarray, N: int, fc: float) -> np.ndarray:
    """Object modulus |O| from Eq. 1, noise-debiased and T0-filtered.

    A(u) = sqrt(max(P - noise, 0) / max(STF, 1e-4)) * T0(u) on U, 0 outside,
    A(0) = 1.  Eq. 1 gives |O|^2 = <|I|^2> / STF; the 1e-4 floor and the T0
    filter are conditioning readings (the paper is silent on both).
    """
    T0 = otf_t0(N, fc)
    A = np.sqrt(np.maximum(P - noise, 0.0) / np.maximum(stf, 1e-4)) * T0
    A[T0 <= 0] = 0.0
    A[N // 2, N // 2] = 1.0
    return A


def photon_terms(flux: np.ndarray, photon_gain: float) -> Tuple[float, float]:
    """(<1/N_f>, <1/N_f^2>) over the frames, N_f = photon_gain * flux_f the
    photon count of frame f's windowed tile."""
    n = photon_gain * np.asarray(flux, dtype=np.float64)
    return float(np.mean(1.0 / n)), float(np.mean(1.0 / (n * n)))


def bispectrum_unbiased(B: np.ndarray, pairs: np.ndarray, P: np.ndarray, a1: float, a2: float) -> np.ndarray:
    """Photon-noise bias removed from the mean bispectrum (Wirnitzer 1985).

    For Poisson photon counts the triple product of a frame's normalised
    spectrum has expectation B + (|I(u)|^2 + |I(v)|^2 + |I(u+v)|^2)/N - 2/N^2
    (N the frame's photon count, |I|^2 each including its own 1/N); so
    B_ub = B - (P(u) + P(v) + P(u+v)) <1/N> + 2 <1/N^2>, with P the measured
    mean power (P(-k) = P(k)).  Reading: the window weights each photon by
    w(x), and w^2 ~ w^3 ~ w is taken, as is the frame average of the
    products as the product of the averages.
    """
    N = P.shape[0]
    c = N // 2
    ux, uy, vx, vy = pairs.T
    wx, wy = ux + vx, uy + vy
    return B - (P[uy + c, ux + c] + P[vy + c, vx + c] + P[wy + c, wx + c]) * a1 + 2.0 * a2


# ----------------------------------------------------------------------------
# seeing (Sect. 3.1: spectral ratio technique, von der Luehe 1984)
# ----------------------------------------------------------------------------

SEEING_STOP = 0.05                 # fit annuli until the observed ratio first drops below this
SEEING_GRID = (1.0, 64.0, 256)     # D/r0 candidates: log-spaced from, to, count


def seeing_cubes(W: int, H: int, N: int, stride: int) -> List[int]:
    """Indices of the subfields that form the seeing cubes (Sect. 3.1).

    The burst is cut into non-overlapping N x N cubes from the image origin
    (80 of 256^2 for a 2560 x 2160 TiO burst).  With a stride dividing N
    these are exactly the full-size subfields whose corner lies on the N
    grid, so their spectra are the subfields' own (same window).
    """
    subs = subfield_grid(W, H, N, stride)
    return [i for i, (x0, y0, w, h) in enumerate(subs)
            if x0 % N == 0 and y0 % N == 0 and w == N and h == N]


def annulus_index(kx: np.ndarray, ky: np.ndarray) -> np.ndarray:
    """Nearest integer radius b of |k| (annuli of unit width).

    (2b - 1)^2 <= 4|k|^2 < (2b + 1)^2, evaluated in integers; |k| is never a
    half-integer on the lattice, so there are no ties.
    """
    q4 = 4 * (np.asarray(kx, dtype=np.int64) ** 2 + np.asarray(ky, dtype=np.int64) ** 2)
    s = np.array([math.isqrt(int(v)) for v in np.ravel(q4)], dtype=np.int64).reshape(np.shape(q4))
    return (s + 1) // 2


def spectral_ratio(P: np.ndarray, M: np.ndarray, noise: float, F: int, N: int,
                   fc: float) -> Tuple[np.ndarray, np.ndarray]:
    """Annulus sums of the spectral ratio |<I>|^2 / <|I|^2> (von der Luehe 1984).

    Over the half-plane domain U n H, annulus b = 0..K+1:
    num_b = sum (F |M|^2 - P) / (F - 1), the power of the mean spectrum with
    the finite-average residual removed (E|M_F|^2 = |E M|^2 + (P - |E M|^2)/F),
    and den_b = sum (P - noise), the speckle power above the noise floor.
    Both readings (debiasing and noise subtraction) are ours; the paper only
    names the technique.  P and M are on the centred N x N grid.
    """
    if F < 2:
        raise ValueError("the spectral ratio needs at least two frames")
    r = cutoff_radius(N, fc)
    K = int(math.floor(r))
    r2i = int(math.floor(r * r))
    k = np.arange(-(N // 2), N - N // 2, dtype=np.int64)
    KX, KY = np.meshgrid(k, k)
    dom = in_half_plane(KX, KY) & (KX * KX + KY * KY <= r2i)
    b = annulus_index(KX[dom], KY[dom])
    m2 = (F * np.abs(M[dom]) ** 2 - P[dom]) / (F - 1)
    num = np.zeros(K + 2)          # |k| <= r rounds to at most K + 1
    den = np.zeros(K + 2)
    for bi, a, c in zip(b, m2, P[dom] - noise):
        num[bi] += a
        den[bi] += c
    return num, den


def ratio_model(rho: np.ndarray, x: float, ck: float = 0.435) -> np.ndarray:
    """Model spectral ratio |T_LE|^2 / STF at D/r0 = x, both normalised at 0.

    Long-exposure transfer function T0 exp(-3.44 (rho x)^(5/3)) (Fried 1966)
    squared over the model STF of ``stf_model`` (normalised to 1 at 0), at
    rho = |k| / r < 1.
    """
    rho = np.asarray(rho, dtype=np.float64)
    T0 = (2.0 / np.pi) * (np.arccos(rho) - rho * np.sqrt(1.0 - rho * rho))
    e = np.exp(-6.88 * (rho * x) ** (5.0 / 3.0))
    return T0 * T0 * e * (1.0 + ck / (x * x)) / (T0 * T0 * e + ck * T0 / (x * x))


def fit_d_over_r0(num: np.ndarray, den: np.ndarray, N: int, fc: float, ck: float = 0.435) -> float:
    """D/r0 whose model ratio best matches the observed one (least squares).

    Annuli b = 1, 2, ... inside the cutoff (b < r, where the model is
    defined) are used until the first with den_b <= 0 or an observed ratio
    num_b/den_b below SEEING_STOP (the informative part of the curve, where
    it falls from 1 towards the noise).  The cost
    J(x) = sum_b (num_b/den_b - ratio_model(b/r, x))^2 is evaluated on the
    SEEING_GRID candidates; the first minimum is refined by a parabola through
    it and its neighbours in log x (not at the ends of the grid).  With no
    usable annulus the estimate is the largest candidate.
    """
    r = cutoff_radius(N, fc)
    bins = []
    for b in range(1, len(num)):
        if not b < r or not den[b] > 0.0 or num[b] / den[b] < SEEING_STOP:
            break
        bins.append(b)
    lo, hi, n = SEEING_GRID
    lx = np.log(lo) + (np.log(hi) - np.log(lo)) * (np.arange(n) / (n - 1))
    if not bins:
        return float(hi)
    bins = np.array(bins)
    eps = num[bins] / den[bins]
    rho = bins / r
    J = np.array([np.sum((eps - ratio_model(rho, math.exp(v), ck)) ** 2) for v in lx])
    i = int(np.argmin(J))
    t = lx[i]
    if 0 < i < n - 1:
        curv = J[i - 1] - 2.0 * J[i] + J[i + 1]
        if curv > 0.0:
            h = lx[1] - lx[0]
            t = lx[i] + 0.5 * h * (J[i - 1] - J[i + 1]) / curv
    return float(math.exp(t))


def estimate_seeing(frames: np.ndarray, N: int, stride: int, fc: float, taper: int,
                    ck: float = 0.435) -> Tuple[np.ndarray, float]:
    """Per-cube D/r0 and the burst's D over mean r0 (Sect. 3.1).

    Each non-overlapping cube gives an estimate from its spectral ratio; the
    estimates of r0 are averaged, so the burst value is 1 / mean(1 / x_c).
    """
    F, H, W = frames.shape
    subs = subfield_grid(W, H, N, stride)
    xs = []
    for c in seeing_cubes(W, H, N, stride):
        In, _, _ = frame_spectra(frames, subs[c], N, taper)
        P, M = power_mean(In)
        num, den = spectral_ratio(P, M, noise_floor(P, N, fc), F, N, fc)
        xs.append(fit_d_over_r0(num, den, N, fc, ck))
    if not xs:
        raise ValueError("no seeing cube: the stride must divide N and the image hold one N x N cube")
    xs = np.array(xs)
    return xs, float(1.0 / np.mean(1.0 / xs))


# ----------------------------------------------------------------------------
# recursive phase (Sect. 3.2: speckle masking phase, LWW 1983)
# ----------------------------------------------------------------------------
class _PairIndex:
    """Lookup (u, v) -> row of the stored pair list (u must be in the half plane)."""

    def __init__(self, pairs: np.ndarray, K: int, R: int):
        self.K, self.R = K, R
        self.keys = self._key(pairs[:, 0], pairs[:, 1], pairs[:, 2], pairs[:, 3])
        self.order = np.argsort(self.keys)
        self.sorted = self.keys[self.order]

    def _key(self, ux, uy, vx, vy):
        K, R = self.K, self.R
        return (((uy + K) * (2 * K + 1) + (ux + K)) * (2 * R + 1) + (vy + R)) * (2 * R + 1) + (vx + R)

    def find(self, ux, uy, vx, vy) -> np.ndarray:
        key = self._key(ux, uy, vx, vy)
        pos = np.searchsorted(self.sorted, key)
        pos = np.minimum(pos, len(self.sorted) - 1)
        if not np.all(self.sorted[pos] == key):
            raise KeyError("pair outside the stored domain")
        return self.order[pos]


def recursion_rings(N: int, fc: float) -> List[np.ndarray]:
    """Points w of the half-plane disk with |w|^2 >= 2, grouped by |w|^2 ascending."""
    U = domain_U(N, fc)
    U = U[in_half_plane(U[:, 0], U[:, 1])]
    n2 = U[:, 0] ** 2 + U[:, 1] ** 2
    U = U[n2 >= 2]
    n2 = n2[n2 >= 2]
    rings = []
    for q in np.unique(n2):
        rings.append(U[n2 == q])
    return rings


def _term_weight(b: np.ndarray, weight: int, P: Optional[np.ndarray], pu, pv, pw) -> np.ndarray:
    """Factor multiplying the |B|-weighted phasor term z(u) z(v) conj B of each split.

    W_BISPEC: 1.  W_UNIT: 1/|B| (0 where B = 0).  W_SNR: 1 / (P(u) P(v) P(w)):
    the speckle-noise variance of the mean bispectrum is about
    P(u) P(v) P(u+v) / F (Wirnitzer 1985), so the term is weighted by
    |B|^2 / variance (0 where the product is not positive).
    """
    if weight == W_BISPEC:
        return np.ones(len(b))
    if weight == W_UNIT:
        mag = np.abs(b)
        return np.where(mag > 0, 1.0 / np.where(mag > 0, mag, 1.0), 0.0)
    if weight == W_SNR:
        if P is None:
            raise ValueError("SNR weighting needs the power spectrum P")
        den = pu * pv * pw
        return np.where(den > 0, 1.0 / np.where(den > 0, den, 1.0), 0.0)
    raise ValueError("unknown weighting")


def phase_recursion(B: np.ndarray, pairs: np.ndarray, M: np.ndarray, N: int, fc: float,
                    R: int, weight: int = W_BISPEC, P: Optional[np.ndarray] = None) -> np.ndarray:
    """Unit phasors z(k) = exp(i phi(k)) of the object on the centred grid.

    Speckle masking (Sect. 2, Sect. 3.2): arg B(u, v) = phi(u) + phi(v) -
    phi(u + v), so every split w = u + v with u and v already known gives an
    estimate of phi(w).  Reading (the paper gives no details):

    * anchors phi(0) = 0, phi(e_x) = arg M(e_x), phi(e_y) = arg M(e_y), so
      the result is registered to the burst-mean image;
    * w runs over the half-plane disk in rings of equal |w|^2, ascending;
    * the phasor of w sums exp(i(phi(u) + phi(v))) conj B(u, v) over
      v with 0 < |v| <= R, u = w - v, |u|^2 < |w|^2, |v|^2 < |w|^2, reading
      B(u, v) = conj B(-u, -v) when u is in the lower half plane;
      ``W_UNIT`` divides each term by |B| (terms with B = 0 dropped),
      ``W_SNR`` divides it by P(u) P(v) P(w) (``_term_weight``);
    * z(w) = phasor / |phasor|, and z(w) = 1 when the phasor is 0;
    * z(-w) = conj z(w).
    """
    r = cutoff_radius(N, fc)
    K = int(math.floor(r))
    c = N // 2
    idx = _PairIndex(pairs, K, R)
    z = np.zeros((N, N), dtype=np.complex128)
    known = np.zeros((N, N), dtype=bool)

    def setz(kx, ky, val):
        z[ky + c, kx + c] = val
        z[-ky + c, -kx + c] = np.conj(val)
        known[ky + c, kx + c] = True
        known[-ky + c, -kx + c] = True

    setz(0, 0, 1.0 + 0j)
    for (ax, ay) in ((1, 0), (0, 1)):
        m = M[ay + c, ax + c]
        setz(ax, ay, m / abs(m) if abs(m) > 0 else 1.0 + 0j)

    V = domain_V(R)
    v2 = V[:, 0] ** 2 + V[:, 1] ** 2
    for ring in recursion_rings(N, fc):
        vals = []
        for (wx, wy) in ring:
            w2 = wx * wx + wy * wy
            ux = wx - V[:, 0]
            uy = wy - V[:, 1]
            ok = (ux * ux + uy * uy < w2) & (v2 < w2)
            ux, uy = ux[ok], uy[ok]
            vx, vy = V[ok, 0], V[ok, 1]
            upper = in_half_plane(ux, uy)
            b = np.empty(len(ux), dtype=np.complex128)
            if upper.any():
                b[upper] = B[idx.find(ux[upper], uy[upper], vx[upper], vy[upper])]
            lo = ~upper
            if lo.any():
                b[lo] = np.conj(B[idx.find(-ux[lo], -uy[lo], -vx[lo], -vy[lo])])
            if not (known[uy + c, ux + c].all() and known[vy + c, vx + c].all()):
                raise AssertionError("recursion used an unknown phase")
            terms = z[uy + c, ux + c] * z[vy + c, vx + c] * np.conj(b)
            if weight != W_BISPEC:
                pu = P[uy + c, ux + c] if P is not None else None
                pv = P[vy + c, vx + c] if P is not None else None
                pw = P[wy + c, wx + c] if P is not None else None
                terms = terms * _term_weight(b, weight, P, pu, pv, pw)
            s = terms.sum()
            vals.append(s / abs(s) if abs(s) > 0 else 1.0 + 0j)
        for (wx, wy), val in zip(ring, vals):
            setz(int(wx), int(wy), val)
    return z


def recursion_splits(N: int, fc: float, R: int) -> np.ndarray:
    """Every split (w, v) the recursion reads, as (wx, wy, vx, vy): w in H with
    2 <= |w|^2 <= r^2, v in V, |w - v| < |w| and |v| < |w|."""
    out = []
    V = domain_V(R)
    v2 = V[:, 0] ** 2 + V[:, 1] ** 2
    for ring in recursion_rings(N, fc):
        for (wx, wy) in ring:
            w2 = wx * wx + wy * wy
            ok = ((wx - V[:, 0]) ** 2 + (wy - V[:, 1]) ** 2 < w2) & (v2 < w2)
            for vx, vy in V[ok]:
                out.append((wx, wy, vx, vy))
    return np.array(out, dtype=np.int64).reshape(-1, 4)


def phase_refine(z: np.ndarray, B: np.ndarray, pairs: np.ndarray, N: int, fc: float, R: int,
                 weight: int = W_BISPEC, P: Optional[np.ndarray] = None, iters: int = 1) -> np.ndarray:
    """Iterative (least-squares) phase from the bispectrum, started from the recursion.

    The recursion uses each split w = u + v only to estimate phi(w).  Read as
    one least-squares problem, every split constrains all three phases:
    maximise  J(z) = sum over splits of  g * Re[conj B(u, v) z(u) z(v) conj z(w)]
    over unit phasors z (g the weighting factor of the recursion's terms).
    With the other phases fixed, J is largest at z(k) = S_k / |S_k| where
    S_k sums  g z(u) z(v) conj B  over the splits with w = k,
    g z(w) conj z(v) B  over those with u = k  and  g z(w) conj z(u) B  over
    those with v = k (z(-k) = conj z(k) folds lower-half occurrences onto k).
    One Jacobi sweep applies that update to every recursion point at once
    from the previous sweep's phases; the anchors (0, +-e_x, +-e_y) stay
    fixed, and a point whose S_k vanishes keeps its phase.  The paper names
    the option ("or iteratively") without details; this is our reading.
    """
    r = cutoff_radius(N, fc)
    K = int(math.floor(r))
    c = N // 2
    idx = _PairIndex(pairs, K, R)
    sp = recursion_splits(N, fc, R)
    wx, wy, vx, vy = sp.T
    ux, uy = wx - vx, wy - vy
    up = in_half_plane(ux, uy)
    b = np.empty(len(sp), dtype=np.complex128)
    b[up] = B[idx.find(ux[up], uy[up], vx[up], vy[up])]
    b[~up] = np.conj(B[idx.find(-ux[~up], -uy[~up], -vx[~up], -vy[~up])])
    g = _term_weight(b, weight, P,
                     P[uy + c, ux + c] if P is not None else None,
                     P[vy + c, vx + c] if P is not None else None,
                     P[wy + c, wx + c] if P is not None else None)
    pts = np.concatenate(recursion_rings(N, fc))
    z = z.copy()
    for _ in range(iters):
        zu, zv, zw = z[uy + c, ux + c], z[vy + c, vx + c], z[wy + c, wx + c]
        S = np.zeros((N, N), dtype=np.complex128)
        for (kx, ky, t) in ((wx, wy, g * zu * zv * np.conj(b)),
                            (ux, uy, g * zw * np.conj(zv) * b),
                            (vx, vy, g * zw * np.conj(zu) * b)):
            h = in_half_plane(kx, ky)
            np.add.at(S, (ky[h] + c, kx[h] + c), t[h])
            np.add.at(S, (-ky[~h] + c, -kx[~h] + c), np.conj(t[~h]))
        new = z.copy()
        for (px, py) in pts:
            sk = S[py + c, px + c]
            if abs(sk) > 0:
                new[py + c, px + c] = sk / abs(sk)
                new[-py + c, -px + c] = np.conj(sk / abs(sk))
        z = new
    return z


# ----------------------------------------------------------------------------
# inverse transform and mosaic (Sect. 2, Sect. 3.2)
# ----------------------------------------------------------------------------
def inverse(A: np.ndarray, z: np.ndarray, flux_mean: float, mu_mean: float,
            win: np.ndarray) -> np.ndarray:
    """Sub-image on the N x N grid (Sect. 2: inverse transform of modulus and phase).

    The non-DC part is Re IDFT(A z) times the burst-mean flux; the mean
    removed before the transform comes back as mu_mean times the window, so
    rec is the apodised sub-image.  ``win`` is the [h, w] window, placed at
    the low corner.
    """
    N = A.shape[0]
    X = A * z
    X[N // 2, N // 2] = 0.0
    rec = idft2(X).real * flux_mean
    h, w = win.shape
    rec[:h, :w] += mu_mean * win
    return rec


def mosaic(recs: Sequence[np.ndarray], subs: Sequence[Tuple[int, int, int, int]], W: int,
           H: int, taper: int, min_weight: float = 0.25) -> Tuple[np.ndarray, np.ndarray]:
    """Merge sub-images: out = sum_s rec_s / sum_s window_s (Sect. 3.2 merge step).

    Each rec_s carries its subfield's window (it is the transform of
    apodised data), so dividing by the summed windows undoes the
    apodisation.  Pixels whose summed window is below ``min_weight`` are
    marked invalid and set to 0 (reading).
    """
    num = np.zeros((H, W))
    den = np.zeros((H, W))
    for rec, (x0, y0, w, h) in zip(recs, subs):
        num[y0:y0 + h, x0:x0 + w] += rec[:h, :w]
        den[y0:y0 + h, x0:x0 + w] += window2d(w, h, taper)
    valid = den >= min_weight
    out = np.where(valid, num / np.where(valid, den, 1.0), 0.0)
    return out, valid


def mosaic_central(recs: Sequence[np.ndarray], subs: Sequence[Tuple[int, int, int, int]], W: int,
                   H: int, N: int, stride: int, taper: int) -> Tuple[np.ndarray, np.ndarray]:
    """Merge full-size sub-images by their central stride x stride blocks.

    The paper merges the aligned sub-images into a 2368 x 1920 mosaic from
    1110 cubes of 256^2 at stride 64 (Sect. 3.2): 37 x 30 blocks of 64^2,
    the central block of each sub-image, so every mosaic pixel comes from
    the one sub-image whose centre is nearest and the partial images sum
    without overlap.  Block of subfield (x0, y0): [x0 + (N - s)/2,
    x0 + (N + s)/2) on each axis; the value is rec / window there (the
    window is 1 inside the block for taper <= (N - s)/2).  Pixels outside
    every block are invalid and 0.
    """
    if (N - stride) % 2:
        raise ValueError("the central block needs N - stride even")
    h0 = (N - stride) // 2
    out = np.zeros((H, W))
    valid = np.zeros((H, W), dtype=bool)
    for rec, (x0, y0, w, h) in zip(recs, subs):
        if w != N or h != N:
            raise ValueError("the central-block mosaic takes full-size sub-images")
        win = window2d(N, N, taper)
        blk = (slice(h0, h0 + stride), slice(h0, h0 + stride))
        out[y0 + h0:y0 + h0 + stride, x0 + h0:x0 + h0 + stride] = rec[blk] / win[blk]
        valid[y0 + h0:y0 + h0 + stride, x0 + h0:x0 + h0 + stride] = True
    return out, valid


# ----------------------------------------------------------------------------
# whole path
# ----------------------------------------------------------------------------
def reconstruct_subfield(frames: np.ndarray, sub: Tuple[int, int, int, int], N: int,
                         fc: float, R: int, taper: int, stf: np.ndarray,
                         weight: int = W_BISPEC, pairs: Optional[np.ndarray] = None,
                         iters: int = 0, photon_gain: float = 0.0) -> Dict:
    """All steps for one subfield; returns every intermediate.  ``iters``
    least-squares sweeps (``phase_refine``) follow the recursion."""
    In, flux, mu = frame_spectra(frames, sub, N, taper)
    P, M = power_mean(In)
    noise = noise_floor(P, N, fc)
    if pairs is None:
        pairs = pair_domain(N, fc, R)
    B = bispectrum(In, pairs)
    if photon_gain > 0:
        B = bispectrum_unbiased(B, pairs, P, *photon_terms(flux, photon_gain))
    A = amplitude(P, noise, stf, N, fc)
    z = phase_recursion(B, pairs, M, N, fc, R, weight, P)
    if iters > 0:
        z = phase_refine(z, B, pairs, N, fc, R, weight, P, iters)
    rec = inverse(A, z, float(flux.mean()), float(mu.mean()), window2d(sub[2], sub[3], taper))
    return {"In": In, "flux": flux, "mu": mu, "P": P, "M": M, "noise": noise, "pairs": pairs,
            "B": B, "A": A, "z": z, "rec": rec}


def reconstruct_burst(frames: np.ndarray, N: int, stride: int, fc: float, R: int, taper: int,
                      stf: Optional[np.ndarray], weight: int = W_BISPEC,
                      subfields: Optional[Sequence[int]] = None, ck: float = 0.435,
                      iters: int = 0, paper_layout: bool = False, photon_gain: float = 0.0) -> Dict:
    """Whole burst: every subfield (or the listed ones), then the mosaic.

    With ``stf`` None the STF is the model at the seeing estimated from the
    burst itself (Sect. 3.1, ``estimate_seeing``), as the paper does.  With
    ``paper_layout`` only full tiles are kept and the mosaic takes their
    central blocks (``mosaic_central``).
    """
    F, H, W = frames.shape
    seeing = None
    if stf is None:
        seeing = estimate_seeing(frames, N, stride, fc, taper, ck)
        stf = stf_model(N, fc, [seeing[1]], ck)
    subs = subfield_grid(W, H, N, stride, drop_edge=paper_layout)
    pairs = pair_domain(N, fc, R)
    pick = range(len(subs)) if subfields is None else subfields
    results = {s: reconstruct_subfield(frames, subs[s], N, fc, R, taper, stf, weight, pairs, iters, photon_gain)
               for s in pick}
    out = valid = None
    if subfields is None:
        recs = [results[s]["rec"] for s in range(len(subs))]
        if paper_layout:
            out, valid = mosaic_central(recs, subs, W, H, N, stride, taper)
        else:
            out, valid = mosaic(recs, subs, W, H, taper)
    return {"subs": subs, "pairs": pairs, "sub": results, "out": out, "valid": valid,
            "seeing": seeing, "stf": stf}
