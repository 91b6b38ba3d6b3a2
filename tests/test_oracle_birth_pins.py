"""Pins of the oracle's birth move (the RT3D move that lets a surface appear
after init, read for the sketched loss of Sec. 3, Eq. 8, as one step of
orthogonal matching pursuit): a noise-free pixel missing a surface regains it
exactly (the residual of the least-squares fit at the existing depths is the
missing signature's component orthogonal to theirs, whose matched filter
peaks at the missing depth, and the joint least-squares coefficient there is
the missing intensity), whatever the existing points' intensities; the
exclusion zones hold against a brute-force check; and the cases where nothing
may be born leave the state unchanged."""
import numpy as np

import oracle
from oracle.reconstruct import Params
from paper_2203_00952_gb300 import synth


def _expected_hist(T, h, t_list, a_list, a0, n):
    # Eq. 1 per bin: photons of surface k at (t_k + tau) mod T w.p. h(tau)/H
    H = h.sum()
    y = np.full(T, n * a0 / T)
    for t, a in zip(t_list, a_list):
        y += n * a * np.roll(h, t) / H
    return y


def _sketch_of(y, m):
    T = y.size
    F = np.exp(1j * 2.0 * np.pi * np.outer(np.arange(T), np.arange(1, m + 1)) / T)
    return (y @ F) / y.sum()


def _pixel(T, m, sigma, ts, als, n=500.0):
    h = synth.impulse_response(T, sigma)
    z = _sketch_of(_expected_hist(T, h, ts, als, 1.0 - sum(als), n), m)[None, :]
    return z, np.array([n]), oracle.h_hat(h, m)


def test_noise_free_pixel_regains_its_missing_surface():
    T, m = 4096, 20
    z, n, hh = _pixel(T, m, 6.0, [700, 1500], [0.4, 0.25])
    t = np.array([[700.0, 0.0]])
    a = np.array([[0.4, 0.0]])
    act = np.array([[True, False]])
    t2, a2, act2, a0 = oracle.birth_step(z, n, t, a, act, hh, T, Params(k_max=2, min_sep=18.0))
    assert act2.tolist() == [[True, True]]
    assert t2[0, 1] == 1500.0 and t2[0, 0] == 700.0
    assert abs(a2[0, 1] - 0.25) < 1e-9 and abs(a2[0, 0] - 0.4) < 1e-12
    assert abs(a0[0] - 0.35) < 1e-9


def test_birth_goes_to_the_first_free_slot():
    T, m = 4096, 20
    z, n, hh = _pixel(T, m, 6.0, [700, 1500, 2600], [0.3, 0.25, 0.2])
    t = np.array([[0.0, 700.0, 0.0, 2600.0]])
    a = np.array([[0.0, 0.3, 0.0, 0.2]])
    act = np.array([[False, True, False, True]])
    t2, a2, act2, _ = oracle.birth_step(z, n, t, a, act, hh, T, Params(k_max=4, min_sep=18.0))
    assert act2.tolist() == [[True, True, False, True]]
    assert t2[0, 0] == 1500.0 and abs(a2[0, 0] - 0.25) < 1e-9


def _refit_residual(z, t_act, hh, T):
    # the residual of the real least-squares fit of z at the given depths,
    # written out with the normal equations (the oracle uses lstsq)
    w = 2 * np.pi * np.arange(1, hh.size + 1) / T
    q = hh[None, :] * np.exp(1j * w[None, :] * np.asarray(t_act, float)[:, None])
    G = np.real(np.conj(q) @ q.T)
    b = np.real(np.conj(q) @ z)
    return z - np.linalg.solve(G, b) @ q


def test_exclusion_zones_against_brute_force():
    # two surfaces 20 bins apart, a point on the first: the residual's matched
    # filter peaks beyond the second, inside an 80-bin exclusion zone around the
    # first; with min_sep = 80 the newborn keeps its distance from the nearest
    # integer of the active depth (brute force over the allowed depths),
    # without it the newborn sits on the peak
    T, m, sep = 2048, 12, 80.0
    z, n, hh = _pixel(T, m, 4.0, [900, 920], [0.3, 0.3])
    t = np.array([[900.3, 0.0]])
    a = np.array([[0.5, 0.0]])
    act = np.array([[True, False]])
    r = _refit_residual(z[0], [900.3], hh, T)
    s = oracle.matched_filter_scores(r[None, :], hh, T)[0]
    d = np.abs(np.arange(T) - 900) % T
    d = np.minimum(d, T - d)
    want = int(np.argmax(np.where(d >= sep, s, -np.inf)))  # brute force
    t_in = int(np.argmax(s))
    assert min(abs(t_in - 900), T - abs(t_in - 900)) < sep  # the unrestricted peak is excluded
    t2, a2, act2, _ = oracle.birth_step(z, n, t, a, act, hh, T, Params(k_max=2, min_sep=sep, prune_alpha=0.0))
    assert act2[0, 1] and t2[0, 1] == want
    t3, _, act3, _ = oracle.birth_step(z, n, t, a, act, hh, T, Params(k_max=2, min_sep=0.0, prune_alpha=0.0))
    assert act3[0, 1] and t3[0, 1] == t_in


def test_nothing_is_born_where_nothing_may_be():
    T, m = 1024, 8
    z, n, hh = _pixel(T, m, 4.0, [300, 600], [0.4, 0.3])
    prm = Params(k_max=2, min_sep=12.0)
    # every slot active: unchanged
    t = np.array([[300.0, 600.0]])
    a = np.array([[0.4, 0.3]])
    act = np.ones((1, 2), bool)
    t2, a2, act2, _ = oracle.birth_step(z, n, t, a, act, hh, T, prm)
    assert np.array_equal(t2, t) and np.array_equal(a2, a) and act2.all()
    # an empty pixel (n = 0, z = 0) and a pure-background pixel (z = 0 at
    # every harmonic): the residual is 0, alpha* = 0 < prune_alpha
    for nn in (0.0, 500.0):
        t2, a2, act2, a0 = oracle.birth_step(np.zeros((1, m), complex), np.array([nn]), np.zeros((1, 2)),
                                             np.zeros((1, 2)), np.zeros((1, 2), bool), hh, T, prm)
        assert not act2.any() and a0[0] == 1.0


def test_newborn_intensity_rescales_the_pixel_to_the_simplex():
    # the existing point is too bright (0.9 for 0.4): the birth still finds the
    # missing surface with its exact intensity (the fit at the existing depth
    # does not depend on the existing intensity), and the pixel's sum
    # 0.9 + 0.25 is rescaled to 1
    T, m = 4096, 20
    z, n, hh = _pixel(T, m, 6.0, [700, 1500], [0.4, 0.25])
    t = np.array([[700.0, 0.0]])
    a = np.array([[0.9, 0.0]])
    act = np.array([[True, False]])
    t2, a2, act2, a0 = oracle.birth_step(z, n, t, a, act, hh, T, Params(k_max=2, min_sep=18.0))
    assert act2.all() and t2[0, 1] == 1500.0
    assert abs(a2.sum() - 1.0) < 1e-12 and abs(a0[0]) < 1e-12
    np.testing.assert_allclose(a2[0], np.array([0.9, 0.25]) / 1.15, atol=1e-9)


def test_reconstruction_with_births_recovers_dropped_surfaces():
    # a two-surface frame whose init lost every second surface: births bring
    # them back (ground truth, not a pin of the reading)
    spec = synth.FrameSpec(rows=16, cols=16, T=2048, sigma=4.0, mean_photons=800.0, sbr=2.0,
                           two_surface_frac=0.5, sep_lo=150.0, sep_hi=400.0)
    fr = synth.make_stream_frame(spec, 44)
    m = 16
    S, n = oracle.sketch_stream(fr.stamps, fr.offsets, spec.T, m)
    z = oracle.finalize(S, n)
    hh = oracle.h_hat(synth.impulse_response(spec.T, spec.sigma), m)
    p = Params(iters=12, k_max=2, d_max=24.0, min_sep=12.0, birth_every=4)
    t0, a0, act0, _ = oracle.init_matched_filter(z, n, hh, spec.T, p)
    act0[:, 1] = False
    a0[:, 1] = 0.0
    t, a, act, _ = oracle.reconstruct(z, n, spec.rows, spec.cols, spec.T, hh, p, init=(t0, a0, act0))
    has2 = fr.truth.nsurf == 2
    d = np.abs(t[:, :, None] - np.nan_to_num(fr.truth.depth, nan=-1e9)[:, None, :])
    d = np.minimum(d, spec.T - d)
    found2 = (np.where(act[:, :, None], d, np.inf)[:, :, 1].min(axis=1) <= 3 * spec.sigma)
    assert has2.sum() > 50
    assert found2[has2].mean() > 0.9
    p0 = Params(iters=12, k_max=2, d_max=24.0, min_sep=12.0, birth_every=0)
    t_nb, _, act_nb, _ = oracle.reconstruct(z, n, spec.rows, spec.cols, spec.T, hh, p0, init=(t0, a0, act0))
    assert not act_nb[:, 1].any()
