"""Oracle: the photon sketch (Sec. 2, Eq. 3) and the histogram (Sec. 2, Eq. 2).

Test infrastructure only (see ``oracle/__init__.py``).

The sketch of a pixel with photon stamps x_1..x_n is
    z_l = (1/n) sum_p exp(i w_l x_p),   w_l = 2 pi l / T,   l = 1..m
(Eq. 3 with the harmonic frequencies of Sec. 2). Because the stamps are
integers, w_l x_p = 2 pi k / T with k = (l x_p) mod T, an exact integer; the
oracle reduces the phase that way in int64 and evaluates cos/sin in float64.
The unnormalised state S_l = sum_p exp(i w_l x_p) and n are what an online
sketch keeps (Sec. 2, online update); z = S / n.
"""
from __future__ import annotations

import numpy as np

_PIXEL_BLOCK = 2048


def phase_indices(stamps, T: int, m: int) -> np.ndarray:
    """k[p, l-1] = (l * x_p) mod T for l = 1..m, exact int64: the phase index
    of exp(i w_l x_p), w_l = 2 pi l / T, in the sketch of Sec. 2, Eq. 3."""
    x = np.asarray(stamps, dtype=np.int64)
    ell = np.arange(1, m + 1, dtype=np.int64)
    return (x[:, None] * ell[None, :]) % int(T)


def _check_stream(stamps, offsets, T):
    offsets = np.asarray(offsets, dtype=np.int64)
    if offsets.ndim != 1 or offsets.size < 1 or offsets[0] != 0:
        raise ValueError("offsets must be a CSR offset array starting at 0")
    if np.any(np.diff(offsets) < 0):
        raise ValueError("offsets must be non-decreasing")
    if offsets[-1] != len(stamps):
        raise ValueError("offsets[-1] must equal the number of stamps")
    if len(stamps) and int(np.max(stamps)) >= T:
        raise ValueError("stamp >= T")
    return offsets


def sketch_stream(stamps, offsets, T: int, m: int):
    """Unnormalised sketch state of a pixel-sorted stamp stream (Sec. 2, Eq. 3
    before the division by n).

    Returns S complex128 [P, m] (S[p, l-1] = sum over the photons of pixel p
    of exp(i 2 pi k / T), k = (l x) mod T) and n int64 [P].
    """
    stamps = np.asarray(stamps)
    offsets = _check_stream(stamps, offsets, T)
    P = offsets.size - 1
    n = np.diff(offsets)
    S = np.zeros((P, m), dtype=np.complex128)
    for p0 in range(0, P, _PIXEL_BLOCK):
        p1 = min(P, p0 + _PIXEL_BLOCK)
        lo, hi = int(offsets[p0]), int(offsets[p1])
        if hi == lo:
            continue
        pix = np.repeat(np.arange(p1 - p0), n[p0:p1])
        x = stamps[lo:hi].astype(np.int64)
        for ell in range(1, m + 1):
            k = (ell * x) % T
            ang = 2.0 * np.pi * k / T
            re = np.bincount(pix, weights=np.cos(ang), minlength=p1 - p0)
            im = np.bincount(pix, weights=np.sin(ang), minlength=p1 - p0)
            S[p0:p1, ell - 1] = re + 1j * im
    return S, n


def sketch_hist(hist, m: int):
    """Unnormalised sketch of histograms with one bin per integer stamp.

    hist [P, T] (counts y_l of Eq. 2 with T' = T and unit bins). S[p, l-1] =
    sum_b y[p, b] exp(i 2 pi ((l b) mod T) / T), n[p] = sum_b y[p, b].
    """
    hist = np.asarray(hist)
    P, T = hist.shape
    b = np.arange(T, dtype=np.int64)
    ell = np.arange(1, m + 1, dtype=np.int64)
    k = (b[:, None] * ell[None, :]) % T
    F = np.exp(1j * (2.0 * np.pi * k / T))  # [T, m]
    S = np.zeros((P, m), dtype=np.complex128)
    n = np.zeros(P, dtype=np.int64)
    for p0 in range(0, P, _PIXEL_BLOCK):
        p1 = min(P, p0 + _PIXEL_BLOCK)
        y = hist[p0:p1].astype(np.float64)
        S[p0:p1] = y @ F
        n[p0:p1] = hist[p0:p1].astype(np.int64).sum(axis=1)
    return S, n


def hist_from_stream(stamps, offsets, T: int) -> np.ndarray:
    """Per-pixel histogram (Eq. 2, T' = T, unit bins) of a CSR stamp stream.

    Returns uint16 [P, T]; raises if a count exceeds 65535.
    """
    stamps = np.asarray(stamps)
    offsets = _check_stream(stamps, offsets, T)
    P = offsets.size - 1
    pix = np.repeat(np.arange(P, dtype=np.int64), np.diff(offsets))
    flat = np.bincount(pix * T + stamps.astype(np.int64), minlength=P * T)
    if flat.size and flat.max() > 65535:
        raise ValueError("histogram count exceeds uint16")
    return flat.reshape(P, T).astype(np.uint16)


def finalize(S, n) -> np.ndarray:
    """z = S / n (Eq. 3); an empty pixel (n = 0) gets z = 0."""
    S = np.asarray(S)
    n = np.asarray(n)
    z = np.zeros_like(S, dtype=np.complex128)
    nz = n > 0
    z[nz] = S[nz] / n[nz, None]
    return z


def merge_states(S_a, n_a, S_b, n_b):
    """Online update (Sec. 2): sketch states of two photon sets add."""
    return np.asarray(S_a) + np.asarray(S_b), np.asarray(n_a) + np.asarray(n_b)
