"""Pins of the FP64 oracle to things other than itself: closed forms of Eq. 3
and Eq. 4, numpy's FFT, brute force in Python integers / mpmath, finite
differences, and invariants of the reconstruction steps."""

import mpmath
import numpy as np
import pytest

import oracle
from oracle.reconstruct import Params, neighbour_weights
from paper_2203_00952_gb300 import synth

mpmath.mp.dps = 40


def _csr(per_pixel):
    stamps = np.concatenate([np.asarray(s, dtype=np.uint16) for s in per_pixel]) if per_pixel else np.zeros(0, np.uint16)
    offsets = np.zeros(len(per_pixel) + 1, dtype=np.uint32)
    offsets[1:] = np.cumsum([len(s) for s in per_pixel])
    return stamps, offsets


# ---------------------------------------------------------------- sketch (Eq. 3)

def test_phase_indices_bruteforce_python_ints():
    rng = np.random.default_rng(1)
    for T in (2, 3, 1000, 4096, 4613, 65536):
        x = rng.integers(0, T, size=50)
        x[0] = T - 1
        k = oracle.phase_indices(x, T, 64)
        for i, xv in enumerate(x):
            for ell in range(1, 65):
                assert k[i, ell - 1] == (ell * int(xv)) % T


@pytest.mark.parametrize("T", [7, 1024, 4613, 65536])
def test_single_photon_is_unit_phasor(T):
    # Eq. 3 with n = 1: z_l = exp(i 2 pi l x / T); reference via mpmath without
    # the integer phase reduction.
    for x in (0, 1, T // 3, T - 1):
        S, n = oracle.sketch_stream(*_csr([[x]]), T, 12)
        z = oracle.finalize(S, n)[0]
        for ell in range(1, 13):
            ref = mpmath.expj(2 * mpmath.pi * ell * x / T)
            assert abs(complex(ref) - z[ell - 1]) < 1e-13


def test_quarter_and_half_period_closed_forms():
    T = 4096
    S, n = oracle.sketch_stream(*_csr([[T // 4], [T // 2], [0, T // 2]]), T, 8)
    z = oracle.finalize(S, n)
    np.testing.assert_allclose(z[0, 0], 1j, atol=1e-15)  # e^{i pi/2}
    np.testing.assert_allclose(z[0, 1], -1.0, atol=1e-15)
    np.testing.assert_allclose(z[1], [(-1.0) ** ell for ell in range(1, 9)], atol=1e-15)
    # two photons half a period apart: odd harmonics cancel, even ones add
    np.testing.assert_allclose(z[2], [0 if ell % 2 else 1 for ell in range(1, 9)], atol=1e-15)


@pytest.mark.parametrize("T,m", [(8, 7), (64, 20), (1024, 32)])
def test_uniform_background_sketches_to_zero(T, m):
    # Sec. 2: at w_l = 2 pi l / T a uniform draw over all T bins has CF 0
    # (sum of the T-th roots of unity).
    S, n = oracle.sketch_stream(*_csr([np.arange(T), np.tile(np.arange(T), 3)]), T, m)
    z = oracle.finalize(S, n)
    assert np.max(np.abs(z)) < 1e-12


@pytest.mark.parametrize("T", [8, 16, 64])
def test_hist_sketch_equals_inverse_fft(T):
    # numpy's ifft uses exp(+i 2 pi l b / T) / T, the sign of Eq. 3.
    rng = np.random.default_rng(T)
    y = rng.integers(0, 50, size=(5, T)).astype(np.uint16)
    m = T - 1
    S, n = oracle.sketch_hist(y, m)
    ref = T * np.fft.ifft(y.astype(float), axis=1)[:, 1 : m + 1]
    np.testing.assert_allclose(S, ref, atol=1e-9)
    np.testing.assert_array_equal(n, y.sum(axis=1))


def test_hist_sketch_bruteforce_dft():
    T, m = 12, 5
    y = np.array([[3, 0, 1, 4, 1, 5, 9, 2, 6, 5, 3, 5]], dtype=np.uint16)
    S, n = oracle.sketch_hist(y, m)
    for ell in range(1, m + 1):
        ref = sum(int(y[0, b]) * mpmath.expj(2 * mpmath.pi * ell * b / T) for b in range(T))
        assert abs(complex(ref) - S[0, ell - 1]) < 1e-12
    assert n[0] == int(y.sum())


def test_hist_from_stream_bruteforce_and_stream_equals_hist():
    rng = np.random.default_rng(3)
    T = 97
    per = [rng.integers(0, T, size=c) for c in (0, 1, 5, 300, 0, 17)]
    stamps, offsets = _csr(per)
    H = oracle.hist_from_stream(stamps, offsets, T)
    for p, s in enumerate(per):
        ref = [0] * T
        for v in s:
            ref[int(v)] += 1
        assert H[p].tolist() == ref
    S1, n1 = oracle.sketch_stream(stamps, offsets, T, 9)
    S2, n2 = oracle.sketch_hist(H, 9)
    np.testing.assert_allclose(S1, S2, atol=1e-11)
    np.testing.assert_array_equal(n1, n2)


def test_online_chunks_merge_to_one_shot():
    # Sec. 2: the sketch can be updated photon by photon; states add.
    rng = np.random.default_rng(4)
    T, m = 1024, 6
    per = [rng.integers(0, T, size=c) for c in (40, 0, 7, 100)]
    full = oracle.sketch_stream(*_csr(per), T, m)
    cut = [rng.integers(0, len(s) + 1) for s in per]
    a = oracle.sketch_stream(*_csr([s[:c] for s, c in zip(per, cut)]), T, m)
    b = oracle.sketch_stream(*_csr([s[c:] for s, c in zip(per, cut)]), T, m)
    S, n = oracle.merge_states(a[0], a[1], b[0], b[1])
    np.testing.assert_allclose(S, full[0], atol=1e-11)
    np.testing.assert_array_equal(n, full[1])


def test_empty_pixel_finalizes_to_zero():
    S, n = oracle.sketch_stream(*_csr([[], [5]]), 16, 3)
    z = oracle.finalize(S, n)
    assert n[0] == 0 and np.all(z[0] == 0)


def test_stamp_out_of_range_rejected():
    with pytest.raises(ValueError):
        oracle.sketch_stream(*_csr([[16]]), 16, 3)


# ------------------------------------------------------------- model (Eq. 4)

def test_hhat_of_delta_is_phasor():
    T, d = 1000, 37
    h = np.zeros(T)
    h[d] = 2.5
    hh = oracle.h_hat(h, 10)
    for ell in range(1, 11):
        assert abs(complex(mpmath.expj(2 * mpmath.pi * ell * d / T)) - hh[ell - 1]) < 1e-13


def test_hhat_of_gaussian_matches_continuous_ft():
    T, sigma = 1024, 4.0
    hh = oracle.h_hat(synth.impulse_response(T, sigma), 32)
    w = 2 * np.pi * np.arange(1, 33) / T
    np.testing.assert_allclose(hh, np.exp(-0.5 * (sigma * w) ** 2), atol=1e-12)


def _sketch_real(y, m):
    # sketch of a real-valued (expected) histogram, normalised by its total
    y = np.atleast_2d(y)
    S, _ = oracle.sketch_hist(y, m)
    return S / y.sum(axis=1, keepdims=True)


def _expected_hist(T, h, t_list, a_list, a0, n):
    # Eq. 1 evaluated per bin: photons of surface k fall at (t_k + tau) mod T
    # with probability h(tau)/H; background 1/T per bin.
    H = h.sum()
    y = np.full(T, n * a0 / T)
    for t, a in zip(t_list, a_list):
        y += n * a * np.roll(h, t) / H
    return y


def test_model_cf_equals_sketch_of_expected_histogram():
    # z of the expected histogram equals Psi_theta (Eq. 4): pins the sign, the
    # circular-lag convention of h and the background reading.
    T, m = 256, 9
    h = np.exp(-0.5 * ((np.minimum(np.arange(T), T - np.arange(T)) - 1.5) / 3.0) ** 2)
    h[3] += 0.7  # asymmetric pulse so that hhat is complex
    ts, als = [40, 131], [0.3, 0.25]
    y = _expected_hist(T, h, ts, als, 0.45, 1000.0)
    S = y @ np.exp(1j * 2 * np.pi * np.outer(np.arange(T), np.arange(1, m + 1)) / T)
    z = S / y.sum()
    psi = oracle.model_cf(np.array([ts], float), np.array([als]), np.ones((1, 2), bool),
                          oracle.h_hat(h, m), T)
    np.testing.assert_allclose(z, psi[0], atol=1e-12)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(6)
    T, m, P, K = 512, 7, 4, 2
    hh = oracle.h_hat(synth.impulse_response(T, 5.0), m)
    z = rng.normal(size=(P, m)) * 0.3 + 1j * rng.normal(size=(P, m)) * 0.3
    n = rng.integers(50, 500, size=P).astype(float)
    t = rng.uniform(50, 450, size=(P, K))
    a = rng.uniform(0.1, 0.5, size=(P, K))
    act = np.ones((P, K), bool)
    act[1, 1] = False
    g_t, g_a = oracle.sketched_gradient(z, n, t, a, act, hh, T)
    eps = 1e-4
    for p in range(P):
        for k in range(K):
            for which, g in (("t", g_t), ("a", g_a)):
                tp, tm, ap, am = t.copy(), t.copy(), a.copy(), a.copy()
                if which == "t":
                    tp[p, k] += eps
                    tm[p, k] -= eps
                else:
                    ap[p, k] += eps
                    am[p, k] -= eps
                fd = (oracle.sketched_loss(z, n, tp, ap, act, hh, T)[p]
                      - oracle.sketched_loss(z, n, tm, am, act, hh, T)[p]) / (2 * eps)
                if not act[p, k]:
                    assert g[p, k] == 0
                    continue
                assert abs(fd - g[p, k]) <= 1e-6 * max(1.0, abs(fd)), (p, k, which, fd, g[p, k])


# -------------------------------------------------------------- init / steps

def _second_difference(f, x0, h):
    return (f(x0 + h) - 2.0 * f(x0) + f(x0 - h)) / (h * h)


def test_step_sizes_bound_the_curvature_of_the_loss():
    # eta_t and eta_alpha are 1 / (Lipschitz constant of the gradient) under
    # alpha <= 1 and |z_l| <= 1: the second derivative of the per-pixel loss
    # in t_k, and the largest eigenvalue of its Hessian in alpha, never exceed
    # (n / n_max) / eta, measured by finite differences of the loss itself
    rng = np.random.default_rng(12)
    T, m, K = 600, 9, 3
    hh = oracle.h_hat(synth.impulse_response(T, 3.0), m)
    n_max = 900.0
    eta_t, eta_a = oracle.step_sizes(hh, n_max, K, T)
    act = np.ones((1, K), bool)
    for _ in range(40):
        n = np.array([rng.uniform(1.0, n_max)])
        a = rng.dirichlet(np.ones(K + 1))[:K][None, :]
        t = rng.uniform(0, T, size=(1, K))
        z = rng.uniform(0, 1, size=(1, m)) * np.exp(1j * rng.uniform(0, 2 * np.pi, size=(1, m)))
        for k in range(K):
            def f(x, k=k):
                tt = t.copy()
                tt[0, k] = x
                return oracle.sketched_loss(z, n, tt, a, act, hh, T)[0]
            assert abs(_second_difference(f, t[0, k], 1e-3)) <= (n[0] / n_max) / eta_t * (1 + 1e-4)
        Hm = np.zeros((K, K))
        for i in range(K):
            for j in range(K):
                def g(di, dj):
                    aa = a.copy()
                    aa[0, i] += di
                    aa[0, j] += dj
                    return oracle.sketched_loss(z, n, t, aa, act, hh, T)[0]
                e = 1e-3
                Hm[i, j] = (g(e, e) - g(e, -e) - g(-e, e) + g(-e, -e)) / (4 * e * e)
        assert np.max(np.linalg.eigvalsh(Hm)) <= (n[0] / n_max) / eta_a * (1 + 1e-6)


def test_step_sizes_are_tight_for_a_delta_pulse():
    # the bounds are the suprema the derivation takes, over alpha <= 1 and
    # |r| <= 2: with |hhat_l| = 1, alpha = 1 and the residual r = 2 Psi (z =
    # 3 Psi) give d2L/dt2 = 2 n sum w_l^2 (1 + 2); K equal depths give the
    # alpha Hessian 2 n sum |hhat|^2 times the all-ones K x K matrix. (Under
    # |z| <= 1 the t bound is up to 3x conservative: Re(conj(r) Psi) <= 0.)
    T, m = 256, 6
    h = np.zeros(T)
    h[0] = 1.0
    hh = oracle.h_hat(h, m)
    n = np.array([300.0])
    eta_t, _ = oracle.step_sizes(hh, n[0], 1, T)
    t0 = 77.3
    w = 2 * np.pi * np.arange(1, m + 1) / T
    z = 3.0 * np.exp(1j * w * t0)[None, :]
    act1 = np.ones((1, 1), bool)
    f = lambda x: oracle.sketched_loss(z, n, np.array([[x]]), np.ones((1, 1)), act1, hh, T)[0]  # noqa: E731
    assert _second_difference(f, t0, 1e-3) == pytest.approx(1.0 / eta_t, rel=1e-5)
    K = 3
    _, eta_a = oracle.step_sizes(hh, n[0], K, T)
    actK = np.ones((1, K), bool)
    tK = np.full((1, K), t0)
    a0 = np.full((1, K), 0.2)
    z0 = np.zeros((1, m), complex)
    Hm = np.zeros((K, K))
    e = 1e-3
    for i in range(K):
        for j in range(K):
            def g(di, dj):
                aa = a0.copy()
                aa[0, i] += di
                aa[0, j] += dj
                return oracle.sketched_loss(z0, n, tK, aa, actK, hh, T)[0]
            Hm[i, j] = (g(e, e) - g(e, -e) - g(-e, e) + g(-e, -e)) / (4 * e * e)
    assert np.max(np.linalg.eigvalsh(Hm)) == pytest.approx(1.0 / eta_a, rel=1e-6)



def test_init_recovers_noise_free_single_surface():
    T, m = 1024, 4
    h = synth.impulse_response(T, 4.0)
    hh = oracle.h_hat(h, m)
    truth_t = [200, 517, 799, 333]
    truth_a = [0.5, 0.9, 0.2, 0.05]
    z = np.concatenate([_sketch_real(_expected_hist(T, h, [t], [a], 1 - a, 100.0), m)
                        for t, a in zip(truth_t, truth_a)])
    n = np.full(4, 100)
    t, alpha, active, alpha0 = oracle.init_matched_filter(z, n, hh, T, Params(k_max=1))
    np.testing.assert_array_equal(t[:, 0], truth_t)
    np.testing.assert_allclose(alpha[:, 0], truth_a, atol=1e-9)
    np.testing.assert_allclose(alpha0, 1 - np.array(truth_a), atol=1e-9)
    assert active.all()


def test_init_two_surfaces_with_delta_pulse_full_band():
    # delta pulse and m = T - 1: the matched filter is (T-1) at the surface and
    # -1 elsewhere per unit alpha, so both argmaxes are exact.
    T = 64
    h = np.zeros(T)
    h[0] = 1.0
    m = T - 1
    hh = oracle.h_hat(h, m)
    y = _expected_hist(T, h, [10, 40], [0.5, 0.3], 0.2, 1.0)
    z = _sketch_real(y, m)
    t, alpha, active, _ = oracle.init_matched_filter(z, np.array([1]), hh, T,
                                                     Params(k_max=2, min_sep=3))
    assert t[0].tolist() == [10, 40]
    np.testing.assert_allclose(alpha[0], [0.5, 0.3], atol=2.0 / T)
    assert active.all()


@pytest.mark.parametrize("truth_t,truth_a", [([10, 30, 50], [0.4, 0.3, 0.2]),
                                             ([5, 20, 37, 55], [0.3, 0.25, 0.2, 0.15])])
def test_init_k_surfaces_with_delta_pulse_full_band(truth_t, truth_a):
    # delta pulse and m = T - 1: per unit alpha the matched filter is T - 1 at
    # a surface and -1 elsewhere, so each greedy pass finds the largest
    # remaining surface exactly (the residual of the earlier passes is off by
    # O(1/T) in alpha only)
    T = 64
    h = np.zeros(T)
    h[0] = 1.0
    m = T - 1
    hh = oracle.h_hat(h, m)
    K = len(truth_t)
    y = _expected_hist(T, h, truth_t, truth_a, 1.0 - sum(truth_a), 1.0)
    z = _sketch_real(y, m)
    t, alpha, active, _ = oracle.init_matched_filter(z, np.array([1]), hh, T, Params(k_max=K, min_sep=3))
    assert t[0].tolist() == truth_t
    np.testing.assert_allclose(alpha[0], truth_a, atol=2.0 / T)
    assert active.all()


def test_init_exclusion_covers_every_earlier_point():
    # three surfaces 2 bins apart with min_sep 3: after the first pass the
    # other two lie inside its exclusion zone, so passes 2 and 3 must land
    # >= 3 bins from each earlier point
    T = 64
    h = np.zeros(T)
    h[0] = 1.0
    hh = oracle.h_hat(h, T - 1)
    y = _expected_hist(T, h, [20, 22, 24], [0.3, 0.3, 0.3], 0.1, 1.0)
    t, _, _, _ = oracle.init_matched_filter(_sketch_real(y, T - 1), np.array([1]), hh, T, Params(k_max=3, min_sep=3))
    d = np.abs(t[0][:, None] - t[0][None, :])
    d = np.minimum(d, T - d)
    assert np.all(d[~np.eye(3, dtype=bool)] >= 3)


def test_init_empty_pixel_has_no_points():
    T, m = 64, 4
    hh = oracle.h_hat(synth.impulse_response(T, 2.0), m)
    t, alpha, active, a0 = oracle.init_matched_filter(np.zeros((1, m), complex), np.array([0]),
                                                      hh, T, Params(k_max=2))
    assert not active.any() and a0[0] == 1.0 and np.all(alpha == 0)


# ---------------------------------------------------------------- APSS pins

def _grid_state(depth):
    R, C = depth.shape
    t = depth.reshape(-1, 1).astype(float)
    return t, np.ones_like(t, bool), R, C


def test_apss_plane_is_fixed_point_and_normals_exact():
    R, C = 9, 11
    rr, cc = np.mgrid[0:R, 0:C]
    gx, gy = 3.0, -1.25  # bins per pixel
    depth = 500.0 + gx * cc + gy * rr
    t, act, R, C = _grid_state(depth)
    p = Params(d_max=50.0, depth_scale=0.125, apss_h=2.5)
    nbh = neighbour_weights(t, act, R, C, p)
    nrm = oracle.plane_normals(nbh, act)
    ref = np.array([-gx * p.depth_scale, -gy * p.depth_scale, 1.0])
    ref /= np.linalg.norm(ref)
    np.testing.assert_allclose(nrm[:, 0], np.broadcast_to(ref, (R * C, 3)), atol=1e-12)
    t2 = oracle.apss_depth(t, act, nrm, nbh, p)
    np.testing.assert_allclose(t2, t, atol=1e-9)


def test_apss_sphere_with_exact_normals_is_fixed_point():
    R, C = 13, 13
    s = 0.125
    cx, cy, rad = 6.3, 5.8, 9.0
    cz = 500.0 * s + rad  # centre behind the surface, looking along +z
    rr, cc = np.mgrid[0:R, 0:C].astype(float)
    zz = cz - np.sqrt(rad ** 2 - (cc - cx) ** 2 - (rr - cy) ** 2)
    t, act, R, C = _grid_state(zz / s)
    p = Params(d_max=80.0, depth_scale=s, apss_h=2.5)
    nbh = neighbour_weights(t, act, R, C, p)
    # exact unit normals, oriented towards +z like the plane-fit normals
    nrm = np.stack([cx - cc, cy - rr, cz - zz], -1).reshape(-1, 1, 3) / rad
    t2 = oracle.apss_depth(t, act, nrm, nbh, p)
    np.testing.assert_allclose(t2, t, atol=1e-9)


def test_apss_pulls_noisy_sphere_towards_surface():
    R, C = 15, 15
    s = 0.125
    cx, cy, rad = 7.0, 7.0, 12.0
    cz = 500.0 * s + rad
    rr, cc = np.mgrid[0:R, 0:C].astype(float)
    zz = cz - np.sqrt(rad ** 2 - (cc - cx) ** 2 - (rr - cy) ** 2)
    noise = np.random.default_rng(8).normal(0, 1.0, size=zz.shape)
    t, act, R, C = _grid_state(zz / s + noise)
    p = Params(d_max=40.0, depth_scale=s, apss_h=2.5)
    nbh = neighbour_weights(t, act, R, C, p)
    t2 = oracle.apss_depth(t, act, oracle.plane_normals(nbh, act), nbh, p)
    inner = (slice(2, -2), slice(2, -2))
    err0 = np.abs(t.reshape(R, C) - zz / s)[inner].mean()
    err1 = np.abs(t2.reshape(R, C) - zz / s)[inner].mean()
    assert err1 < 0.6 * err0


def test_neighbourhood_excludes_far_depths_and_inactive_points():
    t = np.array([[100.0], [100.0 + 30.0], [101.0]])
    act = np.array([[True], [True], [False]])
    p = Params(d_max=24.0)
    nbh = neighbour_weights(t, act, 1, 3, p)
    # query 0's only neighbour with weight is itself
    assert np.count_nonzero(nbh.w[:, 0, 0]) == 1
    assert np.all(nbh.w[:, 2, 0] == 0)  # inactive query


def test_smoothing_constant_field_is_identity_and_bounded():
    R, C = 6, 7
    t = np.full((R * C, 1), 300.0) + np.random.default_rng(9).normal(0, 2, (R * C, 1))
    act = np.ones_like(t, bool)
    p = Params()
    nbh = neighbour_weights(t, act, R, C, p)
    a = np.full_like(t, 0.37)
    a2, act2, a0 = oracle.smooth_prune(a, act, nbh, p)
    np.testing.assert_allclose(a2, a, atol=1e-15)
    np.testing.assert_allclose(a0, 0.63, atol=1e-15)
    a = np.random.default_rng(10).uniform(0.1, 0.9, size=t.shape)
    a2, _, _ = oracle.smooth_prune(a, act, nbh, p)
    assert a2.min() >= a.min() - 1e-15 and a2.max() <= a.max() + 1e-15


def test_pruning_deactivates_small_intensities():
    t = np.array([[100.0], [400.0]])
    act = np.ones_like(t, bool)
    p = Params(prune_alpha=0.05, smooth_lambda=0.0)
    nbh = neighbour_weights(t, act, 1, 2, p)
    a2, act2, a0 = oracle.smooth_prune(np.array([[0.04], [0.5]]), act, nbh, p)
    assert act2[:, 0].tolist() == [False, True]
    assert a2[0, 0] == 0 and a0[0] == 1.0 and a0[1] == 0.5


# ------------------------------------------------------- whole iteration

def test_iteration_fixed_point_on_noise_free_plane():
    R, C, T, m = 8, 9, 1024, 6
    h = synth.impulse_response(T, 4.0)
    hh = oracle.h_hat(h, m)
    rr, cc = np.mgrid[0:R, 0:C]
    depth = (300 + 2 * cc + rr).reshape(-1)
    a = 0.4
    y = np.stack([_expected_hist(T, h, [d], [a], 1 - a, 200.0) for d in depth])
    z = _sketch_real(y, m)
    n = np.full(R * C, 200)
    p = Params(k_max=1, d_max=24.0)
    t0 = depth.reshape(-1, 1).astype(float)
    a0 = np.full((R * C, 1), a)
    act = np.ones((R * C, 1), bool)
    eta_t, eta_a = oracle.step_sizes(hh, 200, 1, T)
    t1, a1, act1, al0 = oracle.iterate(z, n, t0, a0, act, hh, T, R, C, p, eta_t, eta_a)
    np.testing.assert_allclose(t1, t0, atol=1e-9)
    np.testing.assert_allclose(a1, a0, atol=1e-9)
    assert act1.all()


def _dae(t, active, truth, T, tol):
    d = np.abs(t[:, 0] - truth.depth[:, 0])
    d = np.minimum(d, T - d)
    good = active[:, 0] & (d <= tol)
    return d[good].mean(), good.mean()


def test_reconstruct_small_frame_improves_on_init():
    spec = synth.frame_32x32()
    fr = synth.make_stream_frame(spec, synth.SEED_32x32)
    m = 4
    S, n = oracle.sketch_stream(fr.stamps, fr.offsets, spec.T, m)
    z = oracle.finalize(S, n)
    hh = oracle.h_hat(synth.impulse_response(spec.T, spec.sigma), m)
    p = Params(iters=20, k_max=1, d_max=24.0)
    t0, a0, act0, _ = oracle.init_matched_filter(z, n, hh, spec.T, p)
    t, a, act, al0 = oracle.reconstruct(z, n, spec.rows, spec.cols, spec.T, hh, p)
    dae0, det0 = _dae(t0, act0, fr.truth, spec.T, 3 * spec.sigma)
    dae1, det1 = _dae(t, act, fr.truth, spec.T, 3 * spec.sigma)
    assert det1 >= 0.95
    assert dae1 < dae0
    assert dae1 < 2.5
    assert np.all(al0 >= -1e-12) and np.all(al0 <= 1 + 1e-12)


# ---------------------------------------------------------------- weighted loss (Eq. 5-6, W = Sigma^-1)

def test_sigma_theta_is_the_covariance_of_sampled_photons():
    # Eq. 5: n Cov(z) -> Sigma_theta. Draw photons from the discrete model
    # (surface k with probability alpha_k at (t_k + tau) mod T, tau ~ h / H;
    # uniform background otherwise) and compare the sample covariance of
    # exp(i w_l x) with Sigma_theta.
    T, m = 256, 6
    h = synth.impulse_response(T, 3.0)
    hh = oracle.h_hat(h, m)
    t = np.array([[40.0, 171.0]])
    a = np.array([[0.35, 0.25]])
    act = np.ones((1, 2), bool)
    rng = np.random.default_rng(11)
    N = 400_000
    comp = rng.choice(3, size=N, p=[a[0, 0], a[0, 1], 1 - a[0].sum()])
    tau = rng.choice(T, size=N, p=h / h.sum())
    x = np.where(comp == 0, (40 + tau) % T, np.where(comp == 1, (171 + tau) % T, rng.integers(0, T, size=N)))
    v = np.exp(1j * 2 * np.pi * np.outer(x, np.arange(1, m + 1)) / T)
    mu = v.mean(axis=0)
    C = (v.T @ np.conj(v)) / N - np.outer(mu, np.conj(mu))
    S = oracle.sigma_theta(t, a, act, hh, T)[0]
    assert np.max(np.abs(C - S)) <= 6.0 / np.sqrt(N)


def test_sigma_theta_bounded_below_by_the_background_share():
    T, m = 512, 8
    hh = oracle.h_hat(synth.impulse_response(T, 2.0), m)
    rng = np.random.default_rng(12)
    t = rng.uniform(0, T, size=(50, 2))
    a = rng.dirichlet([1, 1, 1], size=50)[:, :2]
    act = rng.uniform(size=(50, 2)) < 0.8
    S = oracle.sigma_theta(t, a, act, hh, T)
    a0 = 1 - np.where(act, a, 0).sum(axis=1)
    lam = np.linalg.eigvalsh(S)
    assert np.all(lam[:, 0] >= a0 - 1e-12)
    np.testing.assert_allclose(S, np.conj(np.transpose(S, (0, 2, 1))), atol=1e-15)


def test_weighted_gradient_of_pure_background_is_scaled_identity_gradient():
    T, m = 128, 5
    hh = oracle.h_hat(synth.impulse_response(T, 2.0), m)
    rng = np.random.default_rng(13)
    z = rng.normal(size=(3, m)) + 1j * rng.normal(size=(3, m))
    t = rng.uniform(0, T, size=(3, 1))
    a = np.zeros((3, 1))
    act = np.zeros((3, 1), bool)
    W = oracle.weighting_matrix(t, a, act, hh, T)
    np.testing.assert_allclose(W, np.broadcast_to(np.eye(m) / (1 + oracle.SIGMA_RIDGE), W.shape), atol=1e-15)


def test_weighted_gradient_matches_finite_differences():
    T, m = 256, 6
    hh = oracle.h_hat(synth.impulse_response(T, 3.0), m)
    rng = np.random.default_rng(14)
    P, K = 4, 2
    t = rng.uniform(20, T - 20, size=(P, K))
    a = rng.uniform(0.1, 0.4, size=(P, K))
    act = np.ones((P, K), bool)
    z = oracle.model_cf(t + rng.normal(size=(P, K)), a * 1.1, act, hh, T) + 0.01 * rng.normal(size=(P, m))
    n = np.array([50, 200, 1000, 7])
    W = oracle.weighting_matrix(t, a, act, hh, T)
    g_t, g_a = oracle.weighted_gradient(z, n, t, a, act, hh, T, W)
    eps = 1e-6
    for k in range(K):
        dt = np.zeros((P, K))
        dt[:, k] = eps
        fd = (oracle.weighted_loss(z, n, t + dt, a, act, hh, T, W) -
              oracle.weighted_loss(z, n, t - dt, a, act, hh, T, W)) / (2 * eps)
        np.testing.assert_allclose(g_t[:, k], fd, rtol=1e-6, atol=1e-6)
        fd = (oracle.weighted_loss(z, n, t, a + dt, act, hh, T, W) -
              oracle.weighted_loss(z, n, t, a - dt, act, hh, T, W)) / (2 * eps)
        np.testing.assert_allclose(g_a[:, k], fd, rtol=1e-6, atol=1e-6)


def test_weighted_step_decreases_the_weighted_loss():
    # the step sizes (W = I bounds times alpha_0 + ridge) are descent steps
    # for the loss with W fixed at the start of the step
    T, m = 512, 8
    h = synth.impulse_response(T, 3.0)
    hh = oracle.h_hat(h, m)
    rng = np.random.default_rng(15)
    P, K = 64, 2
    t_true = rng.uniform(0, T, size=(P, K))
    a_true = rng.uniform(0.1, 0.4, size=(P, K))
    act = np.ones((P, K), bool)
    z = oracle.model_cf(t_true, a_true, act, hh, T)
    n = rng.integers(10, 2000, size=P)
    t = t_true + rng.normal(scale=2.0, size=(P, K))
    a = a_true * rng.uniform(0.8, 1.2, size=(P, K))
    eta_t, eta_a = oracle.step_sizes(hh, n.max(), K, T)
    W = oracle.weighting_matrix(t, a, act, hh, T)
    L0 = oracle.weighted_loss(z, n, t, a, act, hh, T, W)
    t1, a1 = oracle.gradient_step(z, n, t, a, act, hh, T, eta_t, eta_a, weighting=1)
    L1 = oracle.weighted_loss(z, n, t1, a1, act, hh, T, W)
    assert np.all(L1 <= L0 + 1e-12)
    assert np.mean(L1 < L0) > 0.9
