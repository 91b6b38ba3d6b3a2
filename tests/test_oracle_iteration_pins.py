"""Pins of how one oracle iteration is composed (Sec. 3, Eq. 8: a data-term
gradient step followed by the RT3D point-cloud denoiser on depths and the
smoothing of intensities).

The individual steps are pinned in test_oracle_pins.py. These tests pin the
composition: which state each step reads. The gradient step reads the state
the iteration started from; the APSS neighbourhood, the plane normals, the
sphere fit and the intensity smoothing all read the post-gradient state
(t1, alpha1) with the pre-iteration activity.

The expected result is computed here by a route that shares no arithmetic
with the oracle's step functions:
  * the gradient by fourth-order central differences of the per-pixel loss
    n ||z - Psi||^2 (Eq. 8 with W = I), not the analytic gradient;
  * the neighbourhood by explicit loops over pixel pairs;
  * the plane normals and the algebraic sphere (Guennebaud & Gross 2007) as
    weighted least-squares problems on stacked equations solved by
    numpy.linalg.lstsq, not the closed forms;
  * the depth as the root of the sphere along the line of sight found by
    mpmath.polyroots in 50 digits.
The frames are chosen so that only one point is moved by the gradient step:
building the denoiser's neighbourhood from the pre-gradient depths, or
smoothing the pre-gradient intensities, changes the answer far beyond the
1e-9 tolerance, and each test checks that too.
"""

import mpmath
import numpy as np

import oracle
from oracle.reconstruct import Params
from paper_2203_00952_gb300 import synth


def _expected_hist(T, h, t_list, a_list, a0, n):
    # Eq. 1 per bin: photons of surface k land at (t_k + tau) mod T with
    # probability h(tau)/H; the background puts 1/T in every bin.
    H = h.sum()
    y = np.full(T, n * a0 / T)
    for t, a in zip(t_list, a_list):
        y += n * a * np.roll(h, t) / H
    return y


def _sketch_of(y, m):
    # Eq. 2-3 with one bin per stamp: z_l = sum_x y_x e^{i 2 pi l x / T} / sum y
    T = y.size
    x = np.arange(T)
    F = np.exp(1j * 2.0 * np.pi * np.outer(x, np.arange(1, m + 1)) / T)
    return (y @ F) / y.sum()


# ------------------------------------------------------ independent route

def _fd_gradient_step(z, n, t, a, act, hh, T, eta_t, eta_a):
    """Jacobi gradient step with the gradient of n ||z - Psi||^2 taken by
    fourth-order central differences around the pre-step state."""
    P, K = t.shape
    t1, a1 = t.copy(), np.where(act, a, 0.0)

    def loss(p, k, dt, da):
        tt, aa = t[p:p + 1].copy(), a[p:p + 1].copy()
        tt[0, k] += dt
        aa[0, k] += da
        return oracle.sketched_loss(z[p:p + 1], n[p:p + 1], tt, aa, act[p:p + 1], hh, T)[0]

    def d4(f, e):
        return (-f(2 * e) + 8 * f(e) - 8 * f(-e) + f(-2 * e)) / (12 * e)

    for p in range(P):
        for k in range(K):
            if not act[p, k]:
                continue
            g_t = d4(lambda e: loss(p, k, e, 0.0), 1e-3)
            g_a = d4(lambda e: loss(p, k, 0.0, e), 1e-4)
            t1[p, k] = (t[p, k] - eta_t * g_t) % T
            a1[p, k] = max(a[p, k] - eta_a * g_a, 0.0)
        s = a1[p][act[p]].sum()
        if s > 1.0:
            a1[p] /= s
    return t1, a1


def _neighbours(t, act, R, C, prm, p, k):
    """(dx, dy, dz, w, (p2, k2)) for every neighbour of point (p, k)."""
    r, c = divmod(p, C)
    out = []
    K = t.shape[1]
    for r2 in range(max(0, r - prm.radius), min(R, r + prm.radius + 1)):
        for c2 in range(max(0, c - prm.radius), min(C, c + prm.radius + 1)):
            p2 = r2 * C + c2
            for k2 in range(K):
                if not act[p2, k2]:
                    continue
                dt = t[p2, k2] - t[p, k]
                if abs(dt) > prm.d_max:
                    continue
                dx, dy, dz = float(c2 - c), float(r2 - r), dt * prm.depth_scale
                d2 = dx * dx + dy * dy + dz * dz
                if d2 >= prm.apss_h ** 2:
                    continue
                out.append((dx, dy, dz, (1.0 - d2 / prm.apss_h ** 2) ** 4, (p2, k2)))
    return out


def _normal_lstsq(nb):
    # weighted least-squares plane dz = a + b dx + c dy over the neighbours
    sw = np.sqrt([w for *_, w, _ in nb])
    A = np.array([[1.0, dx, dy] for dx, dy, *_ in nb]) * sw[:, None]
    rhs = np.array([dz for _, _, dz, *_ in nb]) * sw
    assert np.linalg.matrix_rank(A) == 3
    (_, b, c), *_ = np.linalg.lstsq(A, rhs, rcond=None)
    v = np.array([-b, -c, 1.0])
    return v / np.linalg.norm(v)


def _sphere_depth_lstsq(nb, normals):
    """Offset along the line of sight to the algebraic sphere fitted with
    normal constraints: (u, u4) minimise sum w ||u + 2 u4 p_i - n_i||^2,
    u0 makes the weighted mean of the sphere function over the points zero;
    the root of u4 z^2 + u_z z + u0 nearest the query (z = 0) is returned,
    or None without a real root."""
    rows, rhs, p_all, w_all = [], [], [], []
    for dx, dy, dz, w, q in nb:
        pv = np.array([dx, dy, dz])
        nv = normals[q]
        s = np.sqrt(w)
        for j in range(3):
            e = np.zeros(4)
            e[j] = 1.0
            e[3] = 2.0 * pv[j]
            rows.append(s * e)
            rhs.append(s * nv[j])
        p_all.append(pv)
        w_all.append(w)
    (ux, uy, uz, u4), *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
    u = np.array([ux, uy, uz])
    sw = np.sqrt(w_all)
    col = sw[:, None]
    target = -sw * np.array([u @ pv + u4 * (pv @ pv) for pv in p_all])
    (u0,), *_ = np.linalg.lstsq(col, target, rcond=None)
    with mpmath.workdps(50):
        coeffs = [mpmath.mpf(u4), mpmath.mpf(uz), mpmath.mpf(u0)]
        while coeffs and coeffs[0] == 0:
            coeffs.pop(0)  # an exact plane: the sphere degenerates to a line
        roots = mpmath.polyroots(coeffs, maxsteps=200, extraprec=200) if len(coeffs) > 1 else []
        real = [float(mpmath.re(x)) for x in roots if abs(mpmath.im(x)) < mpmath.mpf(10) ** -30]
    if not real:
        return None
    return min(real, key=abs)


def _denoise_independent(t1, a1, act, R, C, prm):
    """APSS depth projection and intensity smoothing, both on (t1, a1)."""
    P, K = t1.shape
    nbs = {(p, k): _neighbours(t1, act, R, C, prm, p, k)
           for p in range(P) for k in range(K) if act[p, k]}
    normals = {q: _normal_lstsq(nb) for q, nb in nbs.items()}
    t2, a2 = t1.copy(), np.zeros_like(a1)
    act2 = act.copy()
    lam = prm.smooth_lambda
    for (p, k), nb in nbs.items():
        assert len(nb) >= 3
        dz = _sphere_depth_lstsq(nb, normals)
        if dz is not None and abs(dz) <= prm.d_max * prm.depth_scale:
            t2[p, k] = t1[p, k] + dz / prm.depth_scale
        sw = sum(w for *_, w, _ in nb)
        swa = sum(w * a1[q] for *_, w, q in nb)
        a2[p, k] = (1.0 - lam) * a1[p, k] + lam * swa / sw
        if a2[p, k] < prm.prune_alpha:
            a2[p, k], act2[p, k] = 0.0, False
    for p in range(P):
        s = a2[p][act2[p]].sum()
        if s > 1.0:
            a2[p] /= s
    return t2, a2, act2, 1.0 - a2.sum(axis=1)


# ------------------------------------------------------------------ frames

def _plane_frame(R, C, T, m, sigma, depth_fn, alpha_fn, n_ph):
    """Noise-free sketches of a K-surface scene: z is the sketch of each
    pixel's expected histogram (Eq. 1)."""
    h = synth.impulse_response(T, sigma)
    hh = oracle.h_hat(h, m)
    P = R * C
    z = np.zeros((P, m), complex)
    for p in range(P):
        r, c = divmod(p, C)
        ds, als = depth_fn(r, c), alpha_fn(r, c)
        y = _expected_hist(T, h, ds, als, 1.0 - sum(als), n_ph)
        z[p] = _sketch_of(y, m)
    return z, np.full(P, n_ph), hh


def _run_both(z, n, t0, a0, act, hh, T, R, C, prm):
    eta_t, eta_a = oracle.step_sizes(hh, n.max(), prm.k_max, T)
    got = oracle.iterate(z, n, t0, a0, act, hh, T, R, C, prm, eta_t, eta_a)
    t1, a1 = _fd_gradient_step(z, n, t0, a0, act, hh, T, eta_t, eta_a)
    want = _denoise_independent(t1, a1, act, R, C, prm)
    wrong_t = _denoise_independent(t0, a1, act, R, C, prm)  # neighbourhood from pre-step depths
    wrong_a = _denoise_independent(t1, np.where(act, a0, 0.0), act, R, C, prm)  # smooths pre-step alpha
    return got, want, wrong_t, wrong_a, (t1, a1)


def test_iteration_composition_depth_off_plane():
    # 5x5 tilted plane, the centre pixel's depth starts 3 bins off the plane:
    # only the centre moves in the gradient step; every pixel within two
    # pixels of it is then moved by the denoiser (directly, or through the
    # normals of its neighbours).
    R, C, T, m = 5, 5, 1024, 6
    plane = lambda r, c: 400.0 + 3.0 * c - 2.0 * r  # noqa: E731
    z, n, hh = _plane_frame(R, C, T, m, 4.0, lambda r, c: [int(plane(r, c))],
                            lambda r, c: [0.4], 300.0)
    t0 = np.array([[plane(*divmod(p, C))] for p in range(R * C)])
    t0[12, 0] += 3.0
    a0 = np.full((R * C, 1), 0.4)
    act = np.ones((R * C, 1), bool)
    prm = Params(k_max=1, d_max=24.0, apss_h=2.5, depth_scale=0.125)
    (t, a, ac, al0), want, wrong_t, wrong_a, (t1, a1) = _run_both(z, n, t0, a0, act, hh, T, R, C, prm)
    # the gradient step moved exactly the centre
    moved = np.abs(t1 - t0) > 1e-12
    assert moved[12, 0] and moved.sum() == 1
    np.testing.assert_allclose(t, want[0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(a, want[1], rtol=0, atol=1e-9)
    assert np.array_equal(ac, want[2])
    np.testing.assert_allclose(al0, want[3], rtol=0, atol=1e-9)
    # the pin is sensitive to the state each step reads
    assert np.max(np.abs(wrong_t[0] - want[0])) > 1e-3
    assert np.max(np.abs(wrong_a[1] - want[1])) > 1e-5


def test_iteration_composition_alpha_off_constant_field():
    # the centre pixel's intensity starts at 0.7 in a field of 0.4 with exact
    # depths: the gradient step moves only that alpha (the depth gradient is
    # zero), and smoothing must average the post-step intensities.
    R, C, T, m = 5, 5, 1024, 6
    plane = lambda r, c: 500.0 - 1.0 * c + 2.0 * r  # noqa: E731
    z, n, hh = _plane_frame(R, C, T, m, 4.0, lambda r, c: [int(plane(r, c))],
                            lambda r, c: [0.4], 300.0)
    t0 = np.array([[plane(*divmod(p, C))] for p in range(R * C)])
    a0 = np.full((R * C, 1), 0.4)
    a0[12, 0] = 0.7
    act = np.ones((R * C, 1), bool)
    prm = Params(k_max=1, d_max=24.0, apss_h=2.5, depth_scale=0.125)
    (t, a, ac, al0), want, wrong_t, wrong_a, (t1, a1) = _run_both(z, n, t0, a0, act, hh, T, R, C, prm)
    assert abs(a1[12, 0] - a0[12, 0]) > 1e-3
    np.testing.assert_allclose(np.delete(a1, 12, 0), np.delete(a0, 12, 0), atol=1e-12)
    np.testing.assert_allclose(t, want[0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(a, want[1], rtol=0, atol=1e-9)
    assert np.array_equal(ac, want[2])
    np.testing.assert_allclose(al0, want[3], rtol=0, atol=1e-9)
    assert np.max(np.abs(wrong_a[1] - want[1])) > 1e-4


def test_iteration_composition_two_surfaces():
    # two tilted planes 120 bins apart (farther than d_max, so they never
    # mix) on a 4x5 frame; one point of the far surface starts 2 bins off and
    # one near-surface intensity is off: pins that a point's neighbours,
    # normals and smoothing come from its own surface index.
    R, C, T, m = 4, 5, 2048, 8
    near = lambda r, c: 600.0 + 2.0 * c + 1.0 * r  # noqa: E731
    far = lambda r, c: 720.0 + 1.0 * c - 2.0 * r  # noqa: E731
    z, n, hh = _plane_frame(R, C, T, m, 4.0, lambda r, c: [int(near(r, c)), int(far(r, c))],
                            lambda r, c: [0.35, 0.25], 400.0)
    P = R * C
    t0 = np.array([[near(*divmod(p, C)), far(*divmod(p, C))] for p in range(P)])
    a0 = np.tile([0.35, 0.25], (P, 1))
    t0[7, 1] += 2.0
    a0[11, 0] = 0.5
    act = np.ones((P, 2), bool)
    prm = Params(k_max=2, d_max=24.0, apss_h=2.5, depth_scale=0.125)
    (t, a, ac, al0), want, wrong_t, wrong_a, _ = _run_both(z, n, t0, a0, act, hh, T, R, C, prm)
    np.testing.assert_allclose(t, want[0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(a, want[1], rtol=0, atol=1e-9)
    assert np.array_equal(ac, want[2])
    np.testing.assert_allclose(al0, want[3], rtol=0, atol=1e-9)
    assert np.max(np.abs(wrong_t[0] - want[0])) > 1e-3
    assert np.max(np.abs(wrong_a[1] - want[1])) > 1e-5
