"""Seeded synthetic single-photon lidar frames.

This module is the only code shared by the FP64 oracle, the GPU tests and the
benchmark. It draws inputs; it computes nothing of the method itself (no
sketch, no characteristic function, no reconstruction step).

Observation model (Sec. 2, Eq. 1): a pixel with K surfaces at depths t_k and
reflectivities r_k records photons whose time of arrival is a mixture of the
shifted impulse response (probability alpha_k per surface) and a uniform
background over [0, T-1] (probability alpha_0).

Recipe (fixed; the same seed always gives the same frame):
  * depth map on an R x C grid: a tilted plane
    t = T (0.25 + 0.375 (r/(R-1) + c/(C-1)) / 2) with a spherical cap
    t = T (0.49 - 0.15 sqrt(1 - rho^2/rad^2)) inside the disc of radius
    rad = min(R, C)/4 centred on the grid;
  * reflectivity r ~ U(0.2, 1); a fraction of pixels gets a second surface at
    t_2 = t_1 + U(sep_lo, sep_hi) bins (kept below 0.9 T), reflectivity
    U(0.2, 1);
  * photon count n ~ Poisson(S sum_k r_k + B) with B = nbar/(1+SBR) and
    S = nbar SBR / ((1+SBR) E[sum_k r_k]); each photon independently is from
    surface k with probability S r_k/(S sum r + B), else background
    (Poisson thinning, so arrival order is already random);
  * signal stamp = round(t_k + sigma N(0,1)) mod T, background stamp
    U{0..T-1}; stamps are uint16, pixel-sorted, with uint32 CSR offsets;
  * histograms: y_l ~ Poisson(S sum_k r_k g(l - t_k) + B/T), g the Gaussian
    pulse sampled at the circular distance and normalised to unit sum.
Frames are drawn in fixed blocks of pixels so that the result does not depend
on memory limits.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BLOCK_PIXELS = 4096  # pixels drawn per block; part of the recipe


@dataclass(frozen=True)
class FrameSpec:
    rows: int
    cols: int
    T: int
    sigma: float
    mean_photons: float
    sbr: float
    two_surface_frac: float = 0.0
    sep_lo: float = 50.0
    sep_hi: float = 300.0

    @property
    def num_pixels(self) -> int:
        return self.rows * self.cols


@dataclass
class Truth:
    depth: np.ndarray  # float64 [P, 2]; second column NaN where absent
    refl: np.ndarray  # float64 [P, 2]; 0 where absent
    nsurf: np.ndarray  # int8 [P]
    alpha: np.ndarray = field(default=None)  # float64 [P, 2] photon probabilities
    alpha0: np.ndarray = field(default=None)  # float64 [P]


@dataclass
class StreamFrame:
    spec: FrameSpec
    stamps: np.ndarray  # uint16 [N], pixel-sorted
    offsets: np.ndarray  # uint32 [P+1]
    truth: Truth


def frame_seed(base_seed: int, frame: int = 0) -> np.random.SeedSequence:
    return np.random.SeedSequence([int(base_seed), int(frame)])


def impulse_response(T: int, sigma: float) -> np.ndarray:
    """Gaussian pulse indexed by circular lag tau in [0, T): peak at tau = 0."""
    tau = np.arange(T, dtype=np.float64)
    d = np.minimum(tau, T - tau)
    return np.exp(-0.5 * (d / sigma) ** 2)


def _depth_map(spec: FrameSpec) -> np.ndarray:
    R, C, T = spec.rows, spec.cols, spec.T
    r, c = np.mgrid[0:R, 0:C].astype(np.float64)
    fr = r / max(R - 1, 1)
    fc = c / max(C - 1, 1)
    t = T * (0.25 + 0.375 * (fr + fc) / 2.0)
    rad = min(R, C) / 4.0
    rho2 = (r - R / 2.0) ** 2 + (c - C / 2.0) ** 2
    inside = rho2 < rad * rad
    t[inside] = T * (0.49 - 0.15 * np.sqrt(1.0 - rho2[inside] / (rad * rad)))
    return t.reshape(-1)


def make_truth(spec: FrameSpec, rng: np.random.Generator) -> Truth:
    P = spec.num_pixels
    depth = np.full((P, 2), np.nan)
    refl = np.zeros((P, 2))
    depth[:, 0] = _depth_map(spec)
    refl[:, 0] = rng.uniform(0.2, 1.0, size=P)
    two = rng.uniform(size=P) < spec.two_surface_frac
    sep = rng.uniform(spec.sep_lo, spec.sep_hi, size=P)
    r2 = rng.uniform(0.2, 1.0, size=P)
    t2 = np.minimum(depth[:, 0] + sep, 0.9 * spec.T)
    two &= (t2 - depth[:, 0]) >= spec.sep_lo
    depth[two, 1] = t2[two]
    refl[two, 1] = r2[two]
    nsurf = (1 + two).astype(np.int8)
    ex_sum = 0.6 * (1.0 + spec.two_surface_frac)
    B = spec.mean_photons / (1.0 + spec.sbr)
    S = spec.mean_photons * spec.sbr / ((1.0 + spec.sbr) * ex_sum)
    lam = S * refl.sum(axis=1) + B
    alpha = S * refl / lam[:, None]
    alpha0 = B / lam
    return Truth(depth=depth, refl=refl, nsurf=nsurf, alpha=alpha, alpha0=alpha0)


def _rates(spec: FrameSpec, truth: Truth):
    ex_sum = 0.6 * (1.0 + spec.two_surface_frac)
    B = spec.mean_photons / (1.0 + spec.sbr)
    S = spec.mean_photons * spec.sbr / ((1.0 + spec.sbr) * ex_sum)
    return S, B


def make_stream_frame(spec: FrameSpec, seed: int, frame: int = 0) -> StreamFrame:
    """Pixel-sorted uint16 stamps with uint32 CSR offsets."""
    rng = np.random.default_rng(frame_seed(seed, frame))
    truth = make_truth(spec, rng)
    S, B = _rates(spec, truth)
    P, T = spec.num_pixels, spec.T
    lam = S * truth.refl.sum(axis=1) + B
    counts = rng.poisson(lam).astype(np.int64)
    offsets = np.zeros(P + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    if offsets[-1] >= 2**32:
        raise ValueError("frame exceeds 2^32 photons")
    stamps = np.empty(int(offsets[-1]), dtype=np.uint16)
    a1 = truth.alpha[:, 0]
    a12 = a1 + truth.alpha[:, 1]
    d1 = truth.depth[:, 0]
    d2 = np.nan_to_num(truth.depth[:, 1])
    for p0 in range(0, P, BLOCK_PIXELS):
        p1 = min(P, p0 + BLOCK_PIXELS)
        lo, hi = int(offsets[p0]), int(offsets[p1])
        if hi == lo:
            continue
        pix = np.repeat(np.arange(p0, p1), counts[p0:p1])
        u = rng.uniform(size=hi - lo)
        g = rng.standard_normal(size=hi - lo)
        bg = rng.integers(0, T, size=hi - lo)
        is1 = u < a1[pix]
        is2 = (~is1) & (u < a12[pix])
        t = np.where(is1, d1[pix], d2[pix])
        sig = np.mod(np.rint(t + spec.sigma * g).astype(np.int64), T)
        stamps[lo:hi] = np.where(is1 | is2, sig, bg).astype(np.uint16)
    return StreamFrame(spec=spec, stamps=stamps, offsets=offsets.astype(np.uint32), truth=truth)


def make_multi_surface_frame(spec: FrameSpec, n_surf: int, seed: int, frame: int = 0) -> StreamFrame:
    """Stream frame with n_surf surfaces in every pixel (the multi-surface
    scenes of Sec. 4, beyond two): the first at the depth map of make_truth,
    each next one U(sep_lo, sep_hi) bins further (mod T), reflectivities
    U(0.2, 1); Poisson counts with the same signal/background rates as
    make_stream_frame (mean over pixels of sum r = 0.6 n_surf), photons thinned
    into surfaces and background, signal stamps round(t + sigma N(0,1)) mod T.
    truth.depth / refl / alpha are [P, n_surf]."""
    rng = np.random.default_rng(frame_seed(seed, frame))
    P, T = spec.num_pixels, spec.T
    depth = np.empty((P, n_surf))
    depth[:, 0] = _depth_map(spec)
    for k in range(1, n_surf):
        depth[:, k] = np.mod(depth[:, k - 1] + rng.uniform(spec.sep_lo, spec.sep_hi, size=P), T)
    refl = rng.uniform(0.2, 1.0, size=(P, n_surf))
    B = spec.mean_photons / (1.0 + spec.sbr)
    S = spec.mean_photons * spec.sbr / ((1.0 + spec.sbr) * 0.6 * n_surf)
    lam = S * refl.sum(axis=1) + B
    alpha = S * refl / lam[:, None]
    truth = Truth(depth=depth, refl=refl, nsurf=np.full(P, n_surf, np.int8), alpha=alpha, alpha0=B / lam)
    counts = rng.poisson(lam).astype(np.int64)
    offsets = np.zeros(P + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    stamps = np.empty(int(offsets[-1]), dtype=np.uint16)
    cum = np.cumsum(alpha, axis=1)
    for p0 in range(0, P, BLOCK_PIXELS):
        p1 = min(P, p0 + BLOCK_PIXELS)
        lo, hi = int(offsets[p0]), int(offsets[p1])
        if hi == lo:
            continue
        pix = np.repeat(np.arange(p0, p1), counts[p0:p1])
        u = rng.uniform(size=hi - lo)
        g = rng.standard_normal(size=hi - lo)
        bg = rng.integers(0, T, size=hi - lo)
        k = (u[:, None] >= cum[pix]).sum(axis=1)  # surface index; n_surf = background
        sig = np.mod(np.rint(depth[pix, np.minimum(k, n_surf - 1)] + spec.sigma * g).astype(np.int64), T)
        stamps[lo:hi] = np.where(k < n_surf, sig, bg).astype(np.uint16)
    return StreamFrame(spec=spec, stamps=stamps, offsets=offsets.astype(np.uint32), truth=truth)


def make_hist_frame(spec: FrameSpec, seed: int, frame: int = 0):
    """uint16 histograms [P, T] (one bin per integer stamp) and the truth."""
    rng = np.random.default_rng(frame_seed(seed, frame))
    truth = make_truth(spec, rng)
    S, B = _rates(spec, truth)
    P, T = spec.num_pixels, spec.T
    hist = np.empty((P, T), dtype=np.uint16)
    ell = np.arange(T, dtype=np.float64)
    for p0 in range(0, P, BLOCK_PIXELS):
        p1 = min(P, p0 + BLOCK_PIXELS)
        lam = np.full((p1 - p0, T), B / T)
        for k in range(2):
            r = truth.refl[p0:p1, k]
            t = np.nan_to_num(truth.depth[p0:p1, k])
            d = np.abs(ell[None, :] - t[:, None])
            d = np.minimum(d, T - d)
            g = np.exp(-0.5 * (d / spec.sigma) ** 2)
            g /= g.sum(axis=1, keepdims=True)
            lam += (S * r)[:, None] * g
        y = rng.poisson(lam)
        if y.max(initial=0) > 65535:
            raise ValueError("histogram count exceeds uint16")
        hist[p0:p1] = y.astype(np.uint16)
    return hist, truth


def make_hist_frame_torch(spec: FrameSpec, seed: int, device="cuda"):
    """Same recipe as make_hist_frame, drawn with torch on `device` (used for
    large benchmark histograms; values differ from the numpy draw)."""
    import torch

    rng = np.random.default_rng(frame_seed(seed, 0))
    truth = make_truth(spec, rng)
    S, B = _rates(spec, truth)
    P, T = spec.num_pixels, spec.T
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    hist = torch.empty((P, T), dtype=torch.int16, device=device)
    ell = torch.arange(T, dtype=torch.float32, device=device)
    blk = 16384
    for p0 in range(0, P, blk):
        p1 = min(P, p0 + blk)
        lam = torch.full((p1 - p0, T), B / T, dtype=torch.float32, device=device)
        for k in range(2):
            r = torch.as_tensor(truth.refl[p0:p1, k], dtype=torch.float32, device=device)
            t = torch.as_tensor(np.nan_to_num(truth.depth[p0:p1, k]), dtype=torch.float32, device=device)
            d = (ell[None, :] - t[:, None]).abs()
            d = torch.minimum(d, T - d)
            g = torch.exp(-0.5 * (d / spec.sigma) ** 2)
            g = g / g.sum(dim=1, keepdim=True)
            lam += (S * r)[:, None] * g
        y = torch.poisson(lam, generator=gen).clamp_(max=65535).to(torch.int32)
        hist[p0:p1] = y.to(torch.int16)  # bit pattern of the uint16 count
        del lam, y
    return hist, truth


def make_stream_frame_torch(spec: FrameSpec, seed: int, frame: int = 0, device="cuda", block: int = 65536):
    """Same recipe as make_stream_frame, drawn with torch on `device` (used for
    the large benchmark batches; values differ from the numpy draw). Returns
    (stamps int16 tensor [N] holding the uint16 bit patterns, offsets int32
    tensor [P+1], truth)."""
    import torch

    rng = np.random.default_rng(frame_seed(seed, frame))
    truth = make_truth(spec, rng)
    S, B = _rates(spec, truth)
    P, T = spec.num_pixels, spec.T
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1000003 + int(frame))
    f64 = dict(dtype=torch.float64, device=device)
    lam = torch.as_tensor(S * truth.refl.sum(axis=1) + B, **f64)
    counts = torch.poisson(lam, generator=gen).to(torch.int64)
    offsets = torch.zeros(P + 1, dtype=torch.int64, device=device)
    offsets[1:] = torch.cumsum(counts, 0)
    N = int(offsets[-1].item())
    if N >= 2**31:
        raise ValueError("frame exceeds 2^31 photons")
    stamps = torch.empty(N, dtype=torch.int16, device=device)
    a1 = torch.as_tensor(truth.alpha[:, 0], **f64)
    a12 = a1 + torch.as_tensor(truth.alpha[:, 1], **f64)
    d1 = torch.as_tensor(truth.depth[:, 0], **f64)
    d2 = torch.as_tensor(np.nan_to_num(truth.depth[:, 1]), **f64)
    for p0 in range(0, P, block):
        p1 = min(P, p0 + block)
        lo, hi = int(offsets[p0].item()), int(offsets[p1].item())
        if hi == lo:
            continue
        pix = torch.repeat_interleave(torch.arange(p0, p1, device=device), counts[p0:p1])
        u = torch.rand(hi - lo, generator=gen, **f64)
        g = torch.randn(hi - lo, generator=gen, **f64)
        bg = torch.randint(0, T, (hi - lo,), generator=gen, device=device)
        is1 = u < a1[pix]
        is2 = (~is1) & (u < a12[pix])
        t = torch.where(is1, d1[pix], d2[pix])
        sig = torch.remainder(torch.round(t + spec.sigma * g).to(torch.int64), T)
        val = torch.where(is1 | is2, sig, bg).to(torch.int32)
        stamps[lo:hi] = torch.where(val >= 32768, val - 65536, val).to(torch.int16)
    return stamps, offsets.to(torch.int32), truth


# Workload shapes (sizes, distributions) used by tests and the benchmark.
def frame_32x32() -> FrameSpec:
    """32x32 px, T=1024, sigma=4, 100 photons/px, SBR=1, one surface."""
    return FrameSpec(rows=32, cols=32, T=1024, sigma=4.0, mean_photons=100.0, sbr=1.0)


def frame_256x256() -> FrameSpec:
    """256x256 px, T=4096, sigma=6, 1000 photons/px, SBR=0.5, 10% two surfaces."""
    return FrameSpec(rows=256, cols=256, T=4096, sigma=6.0, mean_photons=1000.0, sbr=0.5,
                     two_surface_frac=0.10)


def frame_512x512_hist() -> FrameSpec:
    """512x512 px histograms, T=4096, 10000 counts/px, SBR=0.2."""
    return FrameSpec(rows=512, cols=512, T=4096, sigma=6.0, mean_photons=10000.0, sbr=0.2)


SEED_32x32 = 20220301
SEED_256x256 = 20220302
SEED_512x512 = 20220303
SEED_BATCH = 20220304
SEED_SERVE = 20220305


def batch_specs(num_frames: int = 64, seed: int = SEED_BATCH):
    """Uneven frames: sizes {64,128,256,512}^2, T in {1024,4096}, m in {4,16},
    photons/px log-uniform [10,5000], SBR log-uniform [0.05,5]."""
    rng = np.random.default_rng(frame_seed(seed, 10**6))
    out = []
    for _ in range(num_frames):
        n = int(rng.choice([64, 128, 256, 512]))
        T = int(rng.choice([1024, 4096]))
        m = int(rng.choice([4, 16]))
        nbar = float(np.exp(rng.uniform(np.log(10.0), np.log(5000.0))))
        sbr = float(np.exp(rng.uniform(np.log(0.05), np.log(5.0))))
        sigma = 4.0 if T == 1024 else 6.0
        out.append((FrameSpec(rows=n, cols=n, T=T, sigma=sigma, mean_photons=nbar, sbr=sbr), m))
    return out
