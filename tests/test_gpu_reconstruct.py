"""GPU parity of the SRT3D reconstruction (Sec. 3, Eq. 8) against the FP64
oracle. Both sides take the same inputs (the GPU's FP32 sketch, the FP32
impulse response). Floating point decides discrete things here (argmax of the
matched filter, neighbour gating, pruning); those decisions are compared by
validity (the GPU's argmax is an argmax of the oracle's scores within FP32
rounding) or counted as flips, and depths / intensities are compared on the
points where both sides agree. Tolerances: 0.05 bin in depth, 1e-3 relative
in intensity n * alpha after a full reconstruction; tighter after one
iteration from a shared state."""
import numpy as np
import pytest
import torch

import oracle
from oracle.reconstruct import Params
from paper_2203_00952_gb300 import binding as B
from paper_2203_00952_gb300 import synth

from gpu_util import ctx, counts, dev_offsets, dev_stamps, to_complex  # noqa: F401

pytestmark = pytest.mark.gpu

DEPTH_TOL = 0.05
INTENSITY_RTOL = 1e-3
FLIP_FRAC = 1e-3


def oracle_params(**kw):
    return Params(**kw)


def gpu_params(p: Params, init_mode, iters=None):
    return B.make_params(iters=p.iters if iters is None else iters, k_max=p.k_max, radius=p.radius,
                         init_mode=init_mode, regularize=int(p.regularize), apss_h=p.apss_h, d_max=p.d_max,
                         depth_scale=p.depth_scale, prune_alpha=p.prune_alpha, smooth_lambda=p.smooth_lambda,
                         min_sep=p.min_sep, weighting=p.weighting, birth_every=p.birth_every)


def sketch_frame(ctx, fr, m):
    spec = fr.spec
    P = spec.num_pixels
    S = torch.empty(P, m, 2, device="cuda")
    n = torch.empty(P, dtype=torch.int32, device="cuda")
    z = torch.empty(P, m, 2, device="cuda")
    B.srt3d_sketch_stream(ctx, dev_stamps(fr.stamps), dev_offsets(fr.offsets), spec.T, m, 0, S, n)
    B.srt3d_finalize(ctx, S, n, m, z)
    return z, n


def gpu_reconstruct(ctx, z, n, rows, cols, T, m, h32, p: Params, init=None, iters=None):
    P = rows * cols
    K = p.k_max
    if init is None:
        depth = torch.zeros(P, K, device="cuda")
        alpha = torch.zeros(P, K, device="cuda")
        active = torch.zeros(P, K, dtype=torch.uint8, device="cuda")
        mode = B.SRT3D_INIT_MATCHED
    else:
        depth = torch.from_numpy(np.asarray(init[0], np.float32)).cuda().contiguous()
        alpha = torch.from_numpy(np.asarray(init[1], np.float32)).cuda().contiguous()
        active = torch.from_numpy(np.asarray(init[2], np.uint8)).cuda().contiguous()
        mode = B.SRT3D_INIT_GIVEN
    alpha0 = torch.zeros(P, device="cuda")
    h = torch.from_numpy(h32).cuda()
    B.srt3d_reconstruct(ctx, z, n, rows, cols, T, m, h, gpu_params(p, mode, iters), depth, alpha, active, alpha0)
    B.srt3d_sync(ctx)
    return (depth.cpu().numpy().astype(np.float64), alpha.cpu().numpy().astype(np.float64),
            active.cpu().numpy().astype(bool), alpha0.cpu().numpy().astype(np.float64))


def frame_inputs(ctx, spec, seed, m):
    fr = synth.make_stream_frame(spec, seed)
    z, n = sketch_frame(ctx, fr, m)
    h32 = synth.impulse_response(spec.T, spec.sigma).astype(np.float32)
    hh = oracle.h_hat(h32.astype(np.float64), m)
    return fr, z, n, to_complex(z), counts(n), h32, hh


def compare_state(g, r, n_np, depth_tol, rtol, flip_frac, what, T=None, outlier_frac=0.0):
    """Depths are compared on the circle of T bins when T is given (t wraps
    to [0, T) after a gradient step). `outlier_frac` allows that fraction of
    the points to exceed the tolerances: points next to a discrete decision
    that FP32 and FP64 take differently (neighbour gate, weight support,
    plane-fit acceptance)."""
    tg, ag, actg, a0g = g
    tr, ar, actr, a0r = r
    flips = int(np.count_nonzero(actg != actr))
    npts = actr.size
    assert flips <= max(1, int(flip_frac * npts)), f"{what}: {flips} activity flips of {npts}"
    both = actg & actr
    dd = np.abs(tg - tr)
    if T is not None:
        dd = np.minimum(dd, T - dd)
    dd = dd[both]
    ig = (n_np[:, None] * ag)[both]
    ir = (n_np[:, None] * ar)[both]
    rel = np.abs(ig - ir) / np.maximum(ir, 1e-12)
    allowed = int(outlier_frac * npts)
    bad_d = int(np.count_nonzero(dd > depth_tol))
    bad_i = int(np.count_nonzero(rel > rtol))
    assert bad_d <= allowed, f"{what}: {bad_d} depths beyond {depth_tol} (max {dd.max()}), {allowed} allowed"
    assert bad_i <= allowed, f"{what}: {bad_i} intensities beyond {rtol} (max {rel.max()}), {allowed} allowed"
    return flips


def check_init_validity(t_g, a_g, act_g, z, n_np, hh, T, p: Params):
    """GPU argmax must be an argmax of the oracle's scores up to FP32 rounding."""
    E2 = float(np.sum(np.abs(hh) ** 2))
    scale = np.sum(np.abs(z * np.conj(hh)[None, :]), axis=1)  # sum_l |c_l|
    tol = 1e-5 * scale + 1e-7
    s1 = oracle.matched_filter_scores(z, hh, T)
    P = z.shape[0]
    idx = np.arange(P)
    t1 = t_g[:, 0].astype(np.int64)
    assert np.all(t_g[:, 0] == t1)
    valid1 = s1[idx, t1] >= s1.max(axis=1) - tol
    assert valid1.all(), f"{np.count_nonzero(~valid1)} invalid first argmaxes"
    a1_ref = np.maximum(0.0, s1[idx, t1] / E2)
    a1_sum = a_g.sum(axis=1)
    # before the sum<=1 rescale the GPU alpha_1 equals s/E2; compare where no rescale happened
    near = np.abs(a1_ref - p.prune_alpha) <= tol / E2 + 1e-6
    act1_ref = (a1_ref >= p.prune_alpha) & (n_np > 0)
    assert np.all((act_g[:, 0] == act1_ref) | near)
    ok = act_g[:, 0] & (a1_sum < 1 - 1e-6)
    if p.k_max == 1:
        assert np.allclose(a_g[ok, 0], a1_ref[ok], atol=1e-6, rtol=1e-5)
    # later points: greedy passes on the residual of the earlier points (at
    # their pre-rescale intensities), outside every earlier exclusion zone
    w = 2 * np.pi * np.arange(1, hh.size + 1) / T
    r = z.copy()
    allowed = np.ones((P, T), bool)
    tol_acc = 1e-5 * scale
    a_prev, t_prev = a1_ref, t1
    for k in range(1, p.k_max):
        f = np.where(a_prev >= p.prune_alpha, a_prev, 0.0)
        r = r - f[:, None] * hh[None, :] * np.exp(1j * w[None, :] * t_prev[:, None])
        d = np.abs(np.arange(T)[None, :] - t_prev[:, None]) % T
        allowed &= np.minimum(d, T - d) >= p.min_sep
        sk = np.where(allowed, oracle.matched_filter_scores(r, hh, T), -np.inf)
        tk = t_g[:, k].astype(np.int64)
        scale_k = np.sum(np.abs(r * np.conj(hh)[None, :]), axis=1)
        tol_acc = tol_acc + 1e-5 * scale_k
        validk = sk[idx, tk] >= sk.max(axis=1) - (tol_acc + 1e-7)
        assert validk.all(), f"{np.count_nonzero(~validk)} invalid argmaxes of pass {k + 1}"
        a_prev, t_prev = np.maximum(0.0, sk[idx, tk] / E2), tk


def multi_surface_inputs(ctx, K, seed, m=20, rows=24, cols=28):
    # surfaces 300-700 bins apart: resolvable with m = 20 harmonics (lobe
    # width ~ T/m = 205 bins)
    spec = synth.FrameSpec(rows=rows, cols=cols, T=4096, sigma=6.0, mean_photons=1500.0, sbr=1.0, sep_lo=300.0,
                           sep_hi=700.0)
    fr = synth.make_multi_surface_frame(spec, K, seed)
    z, n = sketch_frame(ctx, fr, m)
    h32 = synth.impulse_response(spec.T, spec.sigma).astype(np.float32)
    hh = oracle.h_hat(h32.astype(np.float64), m)
    return fr, spec, z, n, to_complex(z), counts(n), h32, hh


@pytest.mark.parametrize("K", [1, 2, 3])
def test_weighted_pixelwise_iterations(ctx, K):
    # W = (Sigma_theta + ridge I)^-1 (Eq. 6) in pixelwise mode: one step from a
    # shared state, then 20 steps from the oracle's init
    spec = synth.FrameSpec(rows=20, cols=24, T=1024, sigma=4.0, mean_photons=400.0, sbr=1.0, two_surface_frac=0.3)
    m = 8
    fr, z, n, z_np, n_np, h32, hh = frame_inputs(ctx, spec, 90 + K, m)
    p = oracle_params(iters=1, k_max=K, d_max=6 * spec.sigma, min_sep=3 * spec.sigma, regularize=False,
                      weighting=1)
    s0 = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, iters=3)
    g = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, init=s0[:3], iters=1)
    eta = oracle.step_sizes(hh, n_np.max(), K, spec.T)
    r = oracle.iterate(z_np, n_np, s0[0], s0[1], s0[2], hh, spec.T, spec.rows, spec.cols, p, *eta)
    compare_state(g, r, n_np, 1e-3, 1e-4, 0.0, f"one weighted step, K = {K}", spec.T)
    p20 = oracle_params(iters=20, k_max=K, d_max=6 * spec.sigma, min_sep=3 * spec.sigma, regularize=False,
                        weighting=1)
    init = oracle.init_matched_filter(z_np, n_np, hh, spec.T, p20)[:3]
    g20 = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p20, init=init)
    r20 = oracle.reconstruct(z_np, n_np, spec.rows, spec.cols, spec.T, hh, p20, init=init)
    compare_state(g20, r20, n_np, DEPTH_TOL, INTENSITY_RTOL, 0.0, f"20 weighted steps, K = {K}", spec.T)
    # the weighted estimate differs from the unweighted one
    pu = oracle_params(iters=20, k_max=K, d_max=6 * spec.sigma, min_sep=3 * spec.sigma, regularize=False)
    gu = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, pu, init=init)
    assert np.max(np.abs(gu[0] - g20[0])) > 1e-3


def test_weighted_loss_needs_pixelwise_mode(ctx):
    T, m = 64, 4
    z = torch.zeros(4, m, 2, device="cuda")
    n = torch.zeros(4, dtype=torch.int32, device="cuda")
    h = torch.ones(T, device="cuda")
    d = torch.zeros(4, 1, device="cuda")
    a = torch.zeros(4, 1, device="cuda")
    act = torch.zeros(4, 1, dtype=torch.uint8, device="cuda")
    a0 = torch.zeros(4, device="cuda")
    for kw in (dict(weighting=1, regularize=1), dict(weighting=2, regularize=0)):
        with pytest.raises(B.SRT3DError) as ei:
            B.srt3d_reconstruct(ctx, z, n, 2, 2, T, m, h, B.make_params(**kw), d, a, act, a0)
        assert ei.value.status == B.SRT3D_EINVAL


@pytest.mark.parametrize("K", [3, 4])
def test_init_matched_filter_more_surfaces(ctx, K):
    fr, spec, z, n, z_np, n_np, h32, hh = multi_surface_inputs(ctx, K, 70 + K)
    p = oracle_params(iters=0, k_max=K, d_max=6 * spec.sigma, min_sep=3 * spec.sigma)
    g = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, 20, h32, p)
    check_init_validity(g[0], g[1], g[2], z_np, n_np, hh, spec.T, p)
    np.testing.assert_allclose(g[3], 1 - g[1].sum(axis=1), atol=1e-6)
    # the K true surfaces are found: each within 3 sigma of some active point
    d = np.abs(g[0][:, :, None] - fr.truth.depth[:, None, :])
    d = np.minimum(d, spec.T - d)
    found = (np.where(g[2][:, :, None], d, np.inf).min(axis=1) <= 3 * spec.sigma)
    assert found.mean() > 0.8


@pytest.mark.parametrize("K", [3, 4])
def test_iterations_more_surfaces(ctx, K):
    # one iteration from a shared state, then 10 from the oracle's init
    fr, spec, z, n, z_np, n_np, h32, hh = multi_surface_inputs(ctx, K, 80 + K)
    m = 20
    p = oracle_params(iters=1, k_max=K, d_max=6 * spec.sigma, min_sep=3 * spec.sigma)
    s0 = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, iters=3)
    g = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, init=s0[:3], iters=1)
    eta = oracle.step_sizes(hh, n_np.max(), K, spec.T)
    r = oracle.iterate(z_np, n_np, s0[0], s0[1], s0[2], hh, spec.T, spec.rows, spec.cols, p, *eta)
    compare_state(g, r, n_np, 1e-3, 1e-4, FLIP_FRAC, f"one iteration, K = {K}", spec.T)
    p10 = oracle_params(iters=10, k_max=K, d_max=6 * spec.sigma, min_sep=3 * spec.sigma)
    init = oracle.init_matched_filter(z_np, n_np, hh, spec.T, p10)[:3]
    g10 = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p10, init=init)
    r10 = oracle.reconstruct(z_np, n_np, spec.rows, spec.cols, spec.T, hh, p10, init=init)
    compare_state(g10, r10, n_np, DEPTH_TOL, INTENSITY_RTOL, FLIP_FRAC, f"10 iterations, K = {K}", spec.T)


@pytest.mark.parametrize("K", [1, 2])
def test_init_matched_filter(ctx, K):
    spec = synth.frame_32x32() if K == 1 else synth.FrameSpec(rows=40, cols=36, T=4096, sigma=6.0,
                                                              mean_photons=1000.0, sbr=0.5,
                                                              two_surface_frac=0.3)
    m = 4 if K == 1 else 10
    fr, z, n, z_np, n_np, h32, hh = frame_inputs(ctx, spec, 11 + K, m)
    p = oracle_params(iters=0, k_max=K, d_max=6 * spec.sigma, min_sep=3 * spec.sigma)
    g = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p)
    check_init_validity(g[0], g[1], g[2], z_np, n_np, hh, spec.T, p)
    np.testing.assert_allclose(g[3], 1 - g[1].sum(axis=1), atol=1e-6)


@pytest.mark.parametrize("K,regularize", [(1, True), (2, True), (1, False)])
def test_one_iteration_from_shared_state(ctx, K, regularize):
    spec = synth.frame_32x32() if K == 1 else synth.FrameSpec(rows=40, cols=36, T=4096, sigma=6.0,
                                                              mean_photons=1000.0, sbr=0.5,
                                                              two_surface_frac=0.3)
    m = 4 if K == 1 else 10
    fr, z, n, z_np, n_np, h32, hh = frame_inputs(ctx, spec, 21 + K, m)
    p = oracle_params(iters=1, k_max=K, d_max=6 * spec.sigma, min_sep=3 * spec.sigma, regularize=regularize)
    # shared starting state: a few GPU iterations from the GPU's init
    s0 = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, iters=3)
    g = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, init=s0[:3], iters=1)
    eta = oracle.step_sizes(hh, n_np.max(), K, spec.T)
    r = oracle.iterate(z_np, n_np, s0[0], s0[1], s0[2], hh, spec.T, spec.rows, spec.cols, p, *eta)
    compare_state(g, r, n_np, 1e-3, 1e-4, 0.0 if not regularize else FLIP_FRAC, "one iteration", spec.T)
    same = np.all(g[2] == r[2], axis=1)
    np.testing.assert_allclose(g[3][same], r[3][same], atol=1e-5)


@pytest.mark.parametrize("K,iters,regularize", [(1, 20, True), (2, 20, True), (1, 20, False)])
def test_full_reconstruction_from_oracle_init(ctx, K, iters, regularize):
    spec = synth.frame_32x32() if K == 1 else synth.FrameSpec(rows=40, cols=36, T=4096, sigma=6.0,
                                                              mean_photons=1000.0, sbr=0.5,
                                                              two_surface_frac=0.3)
    m = 4 if K == 1 else 10
    fr, z, n, z_np, n_np, h32, hh = frame_inputs(ctx, spec, 31 + K, m)
    p = oracle_params(iters=iters, k_max=K, d_max=6 * spec.sigma, min_sep=3 * spec.sigma, regularize=regularize)
    init = oracle.init_matched_filter(z_np, n_np, hh, spec.T, p)[:3]
    g = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, init=init)
    r = oracle.reconstruct(z_np, n_np, spec.rows, spec.cols, spec.T, hh, p, init=init)
    compare_state(g, r, n_np, DEPTH_TOL, INTENSITY_RTOL, FLIP_FRAC, "full reconstruction", spec.T)


def test_full_reconstruction_matched_init_quality(ctx):
    # End to end on the 32x32 frame, each side from its own matched-filter
    # init: both reach the same depth error against the synthetic truth, the
    # inits agree except at near-ties (validated in test_init_matched_filter),
    # and points whose inits agree end within the parity tolerance.
    spec = synth.frame_32x32()
    m = 4
    fr, z, n, z_np, n_np, h32, hh = frame_inputs(ctx, spec, synth.SEED_32x32, m)
    p = oracle_params(iters=20, k_max=1, d_max=6 * spec.sigma, min_sep=3 * spec.sigma)
    g0 = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, iters=0)
    r0 = oracle.init_matched_filter(z_np, n_np, hh, spec.T, p)
    init_diff = (g0[0] != r0[0]) | (g0[2] != r0[2])
    assert init_diff.mean() <= 0.01
    g = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p)
    r = oracle.reconstruct(z_np, n_np, spec.rows, spec.cols, spec.T, hh, p)
    truth = fr.truth.depth[:, 0]
    dae_g = np.abs(g[0][:, 0] - truth)[g[2][:, 0]].mean()
    dae_r = np.abs(r[0][:, 0] - truth)[r[2][:, 0]].mean()
    assert abs(dae_g - dae_r) <= 0.05 * dae_r + 0.01
    # a different (near-tie) start spreads through the 3x3 stencil; exclude a
    # 3-pixel neighbourhood of every pixel whose inits differ
    bad = init_diff[:, 0].reshape(spec.rows, spec.cols)
    zone = np.zeros_like(bad)
    for dr in range(-3, 4):
        for dc in range(-3, 4):
            zone |= np.roll(np.roll(bad, dr, 0), dc, 1)
    keep = ~zone.reshape(-1)
    assert keep.mean() > 0.9
    sub = lambda st: tuple(a[keep] for a in st)  # noqa: E731
    compare_state(sub(g), sub(r), n_np[keep], DEPTH_TOL, INTENSITY_RTOL, FLIP_FRAC, "matched-init reconstruction",
                  spec.T)


def test_full_size_256x256(ctx):
    # The benchmark's workload (256x256, T=4096, m=10, K=2, 30 iterations):
    # sampled init validity, then one iteration from the GPU's final state
    # recomputed by the oracle over all pixels.
    spec = synth.frame_256x256()
    m = 10
    fr, z, n, z_np, n_np, h32, hh = frame_inputs(ctx, spec, synth.SEED_256x256, m)
    p = oracle_params(iters=30, k_max=2, d_max=6 * spec.sigma, min_sep=3 * spec.sigma)
    g0 = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, iters=0)
    rng = np.random.default_rng(3)
    pix = rng.choice(spec.num_pixels, 200, replace=False)
    check_init_validity(g0[0][pix], g0[1][pix], g0[2][pix], z_np[pix], n_np[pix], hh, spec.T, p)
    g29 = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, iters=29)
    g30 = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, init=g29[:3], iters=1)
    eta = oracle.step_sizes(hh, n_np.max(), 2, spec.T)
    r30 = oracle.iterate(z_np, n_np, g29[0], g29[1], g29[2], hh, spec.T, spec.rows, spec.cols, p, *eta)
    compare_state(g30, r30, n_np, 1e-3, 1e-4, FLIP_FRAC, "256x256 iteration 30", spec.T, outlier_frac=1e-4)
    # quality against the synthetic truth: most first surfaces found within 3 sigma
    d = np.abs(g30[0][:, 0] - fr.truth.depth[:, 0])
    assert np.mean(g30[2][:, 0] & (d <= 3 * spec.sigma)) > 0.9


def _noise_free_inputs(spec, seed, m, n_surf=0):
    """Sketches without photon noise: z = Psi of the true surfaces (at integer
    depths, Eq. 4 with the background's exact zero), so that a birth that
    restores a dropped surface is a clear argmax (no FP32/FP64 near-tie).
    n_surf > 0: that many smooth layers in every pixel, 250 bins apart."""
    import numpy.random as npr

    if n_surf:
        truth = synth.make_multi_surface_frame(spec, n_surf, seed).truth
        for k in range(1, n_surf):
            truth.depth[:, k] = np.mod(truth.depth[:, 0] + 250.0 * k, spec.T)
    else:
        truth = synth.make_truth(spec, npr.default_rng(seed))
    t_true = np.nan_to_num(np.round(truth.depth), nan=0.0)
    act_true = np.isfinite(truth.depth)
    h32 = synth.impulse_response(spec.T, spec.sigma).astype(np.float32)
    hh = oracle.h_hat(h32.astype(np.float64), m)
    z_np = oracle.model_cf(t_true, truth.alpha, act_true, hh, spec.T)
    z32 = np.stack([z_np.real, z_np.imag], -1).astype(np.float32)
    z_np = z32[..., 0].astype(np.float64) + 1j * z32[..., 1].astype(np.float64)
    n_np = np.full(spec.num_pixels, 1000, np.int64)
    z = torch.from_numpy(z32).cuda()
    n = torch.from_numpy(n_np.astype(np.int32)).cuda()
    return truth, z, n, z_np, n_np, h32, hh


@pytest.mark.parametrize("K,regularize", [(1, True), (2, True), (3, True), (2, False)])
def test_birth_moves_against_oracle(ctx, K, regularize):
    # RT3D's birth move (every 3 iterations, not after the last) from an init
    # whose later surfaces were dropped, on noise-free sketches with as many
    # surfaces in a pixel as slots (K = 3: three smooth layers everywhere), so
    # that every birth restores a true surface: the GPU's births and iterations
    # against the oracle's point by point at the end-to-end tolerances, no
    # out-of-tolerance point allowed
    spec = synth.FrameSpec(rows=24, cols=28, T=2048, sigma=4.0, mean_photons=800.0, sbr=2.0, two_surface_frac=0.5,
                           sep_lo=150.0, sep_hi=400.0)
    m = 16
    truth, z, n, z_np, n_np, h32, hh = _noise_free_inputs(spec, 61 + K, m, n_surf=3 if K == 3 else 0)
    p = oracle_params(iters=10, k_max=K, d_max=24.0, min_sep=12.0, birth_every=3, regularize=regularize)
    t0, a0, act0, _ = oracle.init_matched_filter(z_np, n_np, hh, spec.T, p)
    act0[:, 1:] = False
    a0[:, 1:] = 0.0
    if K == 1:  # a single slot: drop every tenth pixel's point instead
        act0[::10, 0] = False
        a0[::10, 0] = 0.0
    init = (t0, a0, act0)
    g = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, init=init)
    r = oracle.reconstruct(z_np, n_np, spec.rows, spec.cols, spec.T, hh, p, init=init)
    compare_state(g, r, n_np, DEPTH_TOL, INTENSITY_RTOL, FLIP_FRAC, f"births, K = {K}", spec.T)
    born = g[2] & ~act0
    want = {1: act0[::10, 0].size, 2: (truth.nsurf == 2).sum(), 3: 2 * spec.num_pixels}[K]
    assert born.sum() >= 0.5 * want


def test_birth_moves_on_a_noisy_frame(ctx):
    # Poisson photons: a birth whose matched-filter argmax is a near-tie may
    # land a bin apart in FP32 and FP64 (a discrete decision that the two
    # precisions may take differently), so here the two sides are compared by
    # what they recover
    spec = synth.FrameSpec(rows=24, cols=28, T=2048, sigma=4.0, mean_photons=800.0, sbr=2.0, two_surface_frac=0.5,
                           sep_lo=150.0, sep_hi=400.0)
    m, K = 16, 2
    fr, z, n, z_np, n_np, h32, hh = frame_inputs(ctx, spec, 63, m)
    p = oracle_params(iters=10, k_max=K, d_max=24.0, min_sep=12.0, birth_every=3)
    t0, a0, act0, _ = oracle.init_matched_filter(z_np, n_np, hh, spec.T, p)
    act0[:, 1] = False
    a0[:, 1] = 0.0
    g = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, init=(t0, a0, act0))
    r = oracle.reconstruct(z_np, n_np, spec.rows, spec.cols, spec.T, hh, p, init=(t0, a0, act0))
    has2 = fr.truth.nsurf == 2
    truth = np.nan_to_num(fr.truth.depth, nan=-1e9)

    def found(st):
        d = np.abs(st[0][:, :, None] - truth[:, None, :])
        d = np.minimum(d, spec.T - d)
        return (np.where(st[2][:, :, None], d, np.inf)[:, :, 1].min(axis=1) <= 3 * spec.sigma)[has2].mean()

    fg, fo = found(g), found(r)
    assert fo > 0.8 and abs(fg - fo) <= 0.02
    assert abs(int(g[2].sum()) - int(r[2].sum())) <= max(2, int(0.01 * g[2].size))


def test_full_size_256x256_thirty_iterations_from_oracle_init(ctx):
    # The benchmark's workload end to end from a shared start: the oracle's
    # matched-filter init, then 30 iterations on each side (the launch shape
    # the benchmark times: one cooperative launch for all iterations),
    # compared point by point at the end-to-end tolerances (0.05 bin, 1e-3
    # relative n * alpha) with activity flips and out-of-tolerance points each
    # within the 0.1 % budget of discrete decisions taken differently in FP32
    # and FP64.
    spec = synth.frame_256x256()
    m = 10
    fr, z, n, z_np, n_np, h32, hh = frame_inputs(ctx, spec, synth.SEED_256x256, m)
    p = oracle_params(iters=30, k_max=2, d_max=6 * spec.sigma, min_sep=3 * spec.sigma)
    init = oracle.init_matched_filter(z_np, n_np, hh, spec.T, p)[:3]
    g = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, init=init)
    r = oracle.reconstruct(z_np, n_np, spec.rows, spec.cols, spec.T, hh, p, init=init)
    compare_state(g, r, n_np, DEPTH_TOL, INTENSITY_RTOL, FLIP_FRAC, "256x256, 30 iterations", spec.T,
                  outlier_frac=FLIP_FRAC)


def test_edge_cases(ctx):
    T, m = 256, 6
    h32 = synth.impulse_response(T, 3.0).astype(np.float32)
    hh = oracle.h_hat(h32.astype(np.float64), m)
    # 1x1 array; and a 3x5 array with empty pixels
    for rows, cols in ((1, 1), (3, 5)):
        P = rows * cols
        rng = np.random.default_rng(P)
        per = [np.concatenate([rng.integers(0, T, 20), np.full(30, 100 + p)]) if p % 4 != 1 else np.zeros(0, int)
               for p in range(P)]
        stamps = np.concatenate(per).astype(np.uint16)
        offsets = np.zeros(P + 1, np.uint32)
        offsets[1:] = np.cumsum([len(s) for s in per])
        S = torch.empty(P, m, 2, device="cuda")
        n = torch.empty(P, dtype=torch.int32, device="cuda")
        z = torch.empty(P, m, 2, device="cuda")
        B.srt3d_sketch_stream(ctx, dev_stamps(stamps), dev_offsets(offsets), T, m, 0, S, n)
        B.srt3d_finalize(ctx, S, n, m, z)
        for radius in (1, 2, 3):
            p = oracle_params(iters=5, k_max=2, radius=radius, d_max=12.0, min_sep=9.0)
            g = gpu_reconstruct(ctx, z, n, rows, cols, T, m, h32, p)
            r = oracle.reconstruct(to_complex(z), counts(n), rows, cols, T, hh, p,
                                   init=oracle.init_matched_filter(to_complex(z), counts(n), hh, T, p)[:3])
            empty = counts(n) == 0
            assert not g[2][empty].any() and np.all(g[3][empty] == 1.0)
            compare_state(g, r, counts(n), DEPTH_TOL, INTENSITY_RTOL, 0.0, f"edge {rows}x{cols} r={radius}", T)


def test_invalid_params_rejected(ctx):
    T, m = 64, 4
    z = torch.zeros(4, m, 2, device="cuda")
    n = torch.zeros(4, dtype=torch.int32, device="cuda")
    h = torch.ones(T, device="cuda")
    d = torch.zeros(4, 2, device="cuda")
    a = torch.zeros(4, 2, device="cuda")
    act = torch.zeros(4, 2, dtype=torch.uint8, device="cuda")
    a0 = torch.zeros(4, device="cuda")
    for kw in (dict(k_max=5), dict(k_max=0), dict(radius=0), dict(radius=4), dict(apss_h=0.0), dict(smooth_lambda=1.5),
               dict(d_max=2e6), dict(depth_scale=2e3)):
        prm = B.make_params(**kw)
        with pytest.raises(B.SRT3DError) as ei:
            B.srt3d_reconstruct(ctx, z, n, 2, 2, T, m, h, prm, d, a, act, a0)
        assert ei.value.status == B.SRT3D_EINVAL
    with pytest.raises(B.SRT3DError):
        B.srt3d_reconstruct(ctx, z, n, 2, 2, T, 64, h, B.make_params(), d, a, act, a0)


@pytest.mark.parametrize("T,m,sigma", [(8193, 12, 6.0), (65536, 32, 20.0), (64, 3, 1.5), (4613, 10, 6.0),
                                       (8192, 16, 6.0)])
def test_init_large_and_small_T(ctx, T, m, sigma):
    spec = synth.FrameSpec(rows=6, cols=5, T=T, sigma=sigma, mean_photons=400.0, sbr=1.0, two_surface_frac=0.5,
                           sep_lo=min(50.0, T / 8), sep_hi=min(300.0, T / 4))
    fr, z, n, z_np, n_np, h32, hh = frame_inputs(ctx, spec, 41, m)
    p = oracle_params(iters=0, k_max=2, d_max=6 * sigma, min_sep=3 * sigma)
    g = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, T, m, h32, p)
    check_init_validity(g[0], g[1], g[2], z_np, n_np, hh, T, p)


@pytest.mark.parametrize("iters", [1, 2])
def test_iteration_parity_on_frame_larger_than_one_wave(ctx, iters):
    # 512 x 384 pixels = 768 tiles of 16 x 16, more than the CTAs resident at
    # once: tiles of a later wave read their neighbours' halo while earlier
    # tiles have already finished, so the iteration must not update in place.
    spec = synth.FrameSpec(rows=384, cols=512, T=1024, sigma=4.0, mean_photons=120.0, sbr=1.0, two_surface_frac=0.1)
    m = 6
    fr, z, n, z_np, n_np, h32, hh = frame_inputs(ctx, spec, 61, m)
    p = oracle_params(iters=iters, k_max=2, d_max=24.0, min_sep=12.0)
    s0 = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, iters=2)
    g = gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p, init=s0[:3], iters=iters)
    eta = oracle.step_sizes(hh, n_np.max(), 2, spec.T)
    r = (s0[0], s0[1], s0[2], None)
    for _ in range(iters):
        r = oracle.iterate(z_np, n_np, r[0], r[1], r[2], hh, spec.T, spec.rows, spec.cols, p, *eta)
    # a state updated in place would put thousands of points off; decision
    # flips (e.g. a 3-neighbour plane fit at its acceptance threshold) touch
    # a handful
    compare_state(g, r, n_np, 1e-3, 1e-4, FLIP_FRAC, f"{iters} iteration(s), 768 tiles", spec.T, outlier_frac=1e-4)


def test_persistent_and_per_iteration_launches_agree_exactly(ctx, monkeypatch):
    # The same iteration arithmetic runs as one cooperative launch (all tiles
    # resident, sketches cached in shared memory, grid barrier between
    # iterations) or as one launch per iteration; results are bit-identical.
    spec = synth.FrameSpec(rows=70, cols=90, T=4096, sigma=6.0, mean_photons=400.0, sbr=0.5, two_surface_frac=0.2)
    m = 10
    fr, z, n, z_np, n_np, h32, hh = frame_inputs(ctx, spec, 71, m)
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("SRT3D_ITER_PERSISTENT", flag)
        for iters in (7, 8):
            p = oracle_params(iters=iters, k_max=2, d_max=36.0, min_sep=18.0)
            B.srt3d_profile_enable(ctx, True)
            out.append(gpu_reconstruct(ctx, z, n, spec.rows, spec.cols, spec.T, m, h32, p))
            launched = B.profile_totals(ctx)
            B.srt3d_profile_enable(ctx, False)
            if flag == "1":
                assert launched["iter_all"][1] == 1 and "iter" not in launched
            else:
                assert launched["iter"][1] == iters and "iter_all" not in launched
    for a, b in ((out[0], out[2]), (out[1], out[3])):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
