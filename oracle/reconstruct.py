"""Oracle: SRT3D reconstruction from sketches (Sec. 3, Eq. 8, W = I).

Test infrastructure only (see ``oracle/__init__.py``).

The paper states the objective sum_ij n_ij ||z_ij - Psi(theta_ij)||^2 + rho(theta)
and says SRT3D is RT3D (plug-and-play proximal gradient with a point-cloud
denoiser) with the histogram likelihood replaced by this sketched loss. RT3D's
own steps are not given in the paper, so this module fixes one reading of them.
Each step is a plain array computation over all pixels, in float64:

  init   per pixel, matched filter s(t) = Re sum_l conj(hhat_l e^{i w_l t}) z_l
         over integer t in [0, T); t_1 = argmax (smallest t on ties),
         alpha_1 = max(0, s(t_1) / sum_l |hhat_l|^2); point k = 2..k_max the
         same on the residual z - sum_{i<k} f_i hhat e^{i w t_i} (f_i = alpha_i
         if alpha_i >= prune_alpha, else 0), restricted to circular distance
         >= min_sep from every earlier t_i (greedy; for k_max = 2 the residual
         of the first point). A point is active iff alpha >= prune_alpha.
  grad   Jacobi gradient step on n ||z - Psi||^2 for every active point with
         global step sizes eta_t, eta_alpha (``step_sizes``); t wraps to [0,T),
         alpha >= 0, and alpha is rescaled when sum_k alpha_k > 1.
  APSS   point positions p = (col, row, t * depth_scale) relative to the query
         point; neighbours are active points of the (2r+1)^2 pixel window with
         |t_i - t_q| <= d_max and weight w = (1 - d^2/h^2)^4 (0 beyond h).
         Normals: weighted least-squares plane z = a + b x + c y over each
         point's neighbours, n = (-b, -c, 1)/|.|; (0, 0, 1) with < 3
         neighbours or a singular system (det <= 1e-6 Sw^3).
         Sphere (algebraic sphere with normal constraints, Guennebaud & Gross
         2007): u4 = 1/2 (Spn - Sp.Sn/Sw) / (Spp - Sp.Sp/Sw),
         u = (Sn - 2 u4 Sp)/Sw, u0 = -(u.Sp + u4 Spp)/Sw; the new depth is the
         root of u4 z^2 + u_z z + u0 = 0 along the line of sight nearest the
         current depth. The depth is kept when there are < 3 neighbours, no
         real root, or the move exceeds d_max bins.
  smooth alpha <- (1 - lambda) alpha + lambda sum w alpha_i / sum w with the
         same neighbours and weights; alpha < prune_alpha deactivates the
         point (alpha = 0); rescale if sum_k alpha_k > 1; alpha_0 = 1 - sum.
  birth  (RT3D's birth move, read for the sketched loss; every `birth_every`
         iterations, not after the last) per pixel with a free slot: the
         residual r = z - sum_k beta_k hhat e^{i w t_k} of the least-squares
         fit of real intensities beta to z at the active points' current
         depths (what those points cannot explain wherever their intensities
         sit, e.g. after smoothing), its matched filter over integer t at
         circular distance >= min_sep from the nearest integer of every
         active depth; t* = argmax (smallest t on ties), alpha* = the new
         point's coefficient in the least-squares fit of z by the active
         points and the new one (one step of orthogonal matching pursuit); if
         alpha* >= prune_alpha a point (t*, alpha*) is born in the first free
         slot (the other points keep their intensities); rescale if
         sum_k alpha_k > 1.
All points of an iteration read the state the iteration started from (grad
reads the previous iterate, APSS and smoothing read the post-gradient state).

Parity: the pieces are pinned separately (finite differences for the
gradient, exact planes and spheres for APSS, constant fields for smoothing,
noise-free sketches for init, the whole iteration's fixed point on a
noise-free plane, step sizes against the loss curvature), and the composition
of one iteration (which state each step reads) is pinned against an
independent computation of the same iteration: finite-difference gradient,
least-squares plane and sphere fits on stacked equations, roots in 50-digit
arithmetic (tests/test_oracle_iteration_pins.py). What stays unpinned is
only that this sequence of steps is RT3D's: the paper cites RT3D without
stating its iteration, so the reading itself has nothing in the paper to be
checked against and is checked against the synthetic ground truth instead.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .model import SIGMA_RIDGE, model_cf, sketched_gradient, weighted_gradient, weighting_matrix

_PIXEL_BLOCK = 1024


@dataclass
class Params:
    iters: int = 20
    k_max: int = 1
    radius: int = 1
    apss_h: float = 2.5
    d_max: float = 24.0
    depth_scale: float = 0.125
    prune_alpha: float = 0.02
    smooth_lambda: float = 0.5
    min_sep: float = 12.0
    regularize: bool = True
    birth_every: int = 0  # 0: no birth moves
    weighting: int = 0  # 0: W = I (SRT3D); 1: W = Sigma_theta^-1 (Eq. 6), pixelwise mode only


def step_sizes(hh, n_max: float, k_max: int, T: int):
    """Global step sizes of the sketched gradient step (a reading of the RT3D
    step that Sec. 3 adopts; Lipschitz bounds with alpha <= 1, |r| <= 2):
    eta_t = 1 / (2 n_max sum_l w_l^2 |hhat_l| (|hhat_l| + 2)),
    eta_alpha = 1 / (2 n_max k_max sum_l |hhat_l|^2)."""
    a = np.abs(np.asarray(hh))
    w = 2.0 * np.pi * np.arange(1, a.size + 1) / T
    nm = max(float(n_max), 1.0)
    eta_t = 1.0 / (2.0 * nm * np.sum(w * w * a * (a + 2.0)))
    eta_a = 1.0 / (2.0 * nm * k_max * np.sum(a * a))
    return eta_t, eta_a


def matched_filter_scores(v, hh, T: int, p0: int = 0, p1: int | None = None) -> np.ndarray:
    """s[p, t] = Re sum_l conj(hhat_l) exp(-i w_l t) v[p, l] for integer t: the
    matched filter of the sketched model (Eq. 4) against the data v, the
    reading of the init that Sec. 3 leaves to RT3D."""
    v = np.asarray(v)[p0:p1]
    m = hh.size
    t = np.arange(T, dtype=np.int64)
    ell = np.arange(1, m + 1, dtype=np.int64)
    k = (t[:, None] * ell[None, :]) % T
    E = np.exp(-1j * (2.0 * np.pi * k / T))  # [T, m]
    c = v * np.conj(hh)[None, :]
    return np.real(c @ E.T)


def _circ_dist(a, b, T):
    d = np.abs(a - b) % T
    return np.minimum(d, T - d)


def _project_simplex_cap(alpha, active):
    a = np.where(active, alpha, 0.0)
    s = a.sum(axis=1, keepdims=True)
    scale = np.where(s > 1.0, 1.0 / np.where(s > 0, s, 1.0), 1.0)
    return a * scale


def init_matched_filter(z, n, hh, T: int, params: Params):
    """Per-pixel sketched matched filter (the init reading; see the module
    docstring); returns t, alpha, active [P, K], alpha0 [P]."""
    z = np.asarray(z)
    n = np.asarray(n)
    P = z.shape[0]
    K = params.k_max
    E2 = float(np.sum(np.abs(hh) ** 2))
    w = 2.0 * np.pi * np.arange(1, hh.size + 1) / T
    t = np.zeros((P, K))
    alpha = np.zeros((P, K))
    for p0 in range(0, P, _PIXEL_BLOCK):
        p1 = min(P, p0 + _PIXEL_BLOCK)
        s = matched_filter_scores(z, hh, T, p0, p1)
        t1 = np.argmax(s, axis=1)
        a1 = np.maximum(0.0, s[np.arange(p1 - p0), t1] / E2)
        t[p0:p1, 0] = t1
        alpha[p0:p1, 0] = a1
        rows = np.arange(p1 - p0)
        grid = np.arange(T)[None, :]
        resid = z[p0:p1].copy()
        allowed = np.ones((p1 - p0, T), bool)
        for k in range(1, K):
            tk_prev, ak_prev = t[p0:p1, k - 1].astype(np.int64), alpha[p0:p1, k - 1]
            f = np.where(ak_prev >= params.prune_alpha, ak_prev, 0.0)
            resid = resid - f[:, None] * hh[None, :] * np.exp(1j * w[None, :] * tk_prev[:, None])
            allowed &= _circ_dist(grid, tk_prev[:, None], T) >= params.min_sep
            sk = np.where(allowed, matched_filter_scores(resid, hh, T), -np.inf)
            tk = np.argmax(sk, axis=1)
            t[p0:p1, k] = tk
            alpha[p0:p1, k] = np.maximum(0.0, sk[rows, tk] / E2)
    active = (alpha >= params.prune_alpha) & (n > 0)[:, None]
    alpha = _project_simplex_cap(alpha, active)
    alpha0 = 1.0 - alpha.sum(axis=1)
    return t, alpha, active, alpha0


def gradient_step(z, n, t, alpha, active, hh, T: int, eta_t: float, eta_a: float, weighting: int = 0):
    """One Jacobi gradient step on n ||z - Psi||^2_W (Eq. 8 data term).
    W = I, or (weighting = 1) W = (Sigma_theta + ridge I)^-1 evaluated at the
    current state and held fixed for the step (iteratively reweighted). Since
    Sigma_theta >= alpha_0 I (the uniform background's share of the
    covariance), ||W|| <= 1 / (alpha_0 + ridge): the W = I step sizes times
    alpha_0 + ridge of the pixel's current state stay valid bounds."""
    if weighting:
        W = weighting_matrix(t, alpha, active, hh, T)
        g_t, g_a = weighted_gradient(z, n, t, alpha, active, hh, T, W)
        a0 = np.maximum(0.0, 1.0 - np.where(active, alpha, 0.0).sum(axis=1))
        scale = (a0 + SIGMA_RIDGE)[:, None]
        eta_t, eta_a = eta_t * scale, eta_a * scale
    else:
        g_t, g_a = sketched_gradient(z, n, t, alpha, active, hh, T)
    t_new = np.where(active, np.mod(t - eta_t * g_t, T), t)
    a_new = np.where(active, np.maximum(alpha - eta_a * g_a, 0.0), 0.0)
    a_new = _project_simplex_cap(a_new, active)
    return t_new, a_new


@dataclass
class Neighbourhood:
    """Per query point (p, k) and per slot s = (dr, dc, k'):
    the neighbour's flat pixel index, offsets and weight."""

    dx: np.ndarray  # [S]
    dy: np.ndarray  # [S]
    kk: np.ndarray  # [S] neighbour's surface index
    nb: np.ndarray  # [S, P] neighbour pixel (clamped; masked by w)
    dz: np.ndarray  # [S, P, K] (t_nb - t_q) * depth_scale
    w: np.ndarray  # [S, P, K] weight; 0 for non-neighbours


def neighbour_weights(t, active, rows: int, cols: int, params: Params) -> Neighbourhood:
    """APSS neighbourhood of every point (the point-cloud denoiser of RT3D that
    Sec. 3 plugs in; Guennebaud & Gross 2007 weights; see module docstring)."""
    P, K = t.shape
    rr, cc = np.divmod(np.arange(P), cols)
    r = params.radius
    h2 = params.apss_h ** 2
    dxs, dys, kks, nbs, dzs, ws = [], [], [], [], [], []
    for dr in range(-r, r + 1):
        for dc in range(-r, r + 1):
            r2, c2 = rr + dr, cc + dc
            inb = (r2 >= 0) & (r2 < rows) & (c2 >= 0) & (c2 < cols)
            nbp = np.where(inb, r2 * cols + c2, 0)
            for k2 in range(K):
                t_nb = t[nbp, k2]
                act_nb = active[nbp, k2] & inb
                dt = t_nb[:, None] - t
                dz = dt * params.depth_scale
                d2 = dc * dc + dr * dr + dz * dz
                ok = act_nb[:, None] & active & (np.abs(dt) <= params.d_max) & (d2 < h2)
                w = np.where(ok, (1.0 - d2 / h2) ** 4, 0.0)
                dxs.append(dc)
                dys.append(dr)
                kks.append(k2)
                nbs.append(nbp)
                dzs.append(dz)
                ws.append(w)
    return Neighbourhood(np.array(dxs, float), np.array(dys, float), np.array(kks),
                         np.stack(nbs), np.stack(dzs), np.stack(ws))


def plane_normals(nbh: Neighbourhood, active) -> np.ndarray:
    """Unit normals [P, K, 3] from a weighted least-squares plane
    z = a + b x + c y over each point's neighbours (APSS reading, Sec. 3)."""
    w = nbh.w
    x = nbh.dx[:, None, None]
    y = nbh.dy[:, None, None]
    z = nbh.dz
    Sw = w.sum(0)
    Sx, Sy, Sz = (w * x).sum(0), (w * y).sum(0), (w * z).sum(0)
    Sxx, Sxy, Syy = (w * x * x).sum(0), (w * x * y).sum(0), (w * y * y).sum(0)
    Sxz, Syz = (w * x * z).sum(0), (w * y * z).sum(0)
    cnt = (w > 0).sum(0)
    M = np.stack([np.stack([Sw, Sx, Sy], -1), np.stack([Sx, Sxx, Sxy], -1),
                  np.stack([Sy, Sxy, Syy], -1)], -2)  # [P, K, 3, 3]
    rhs = np.stack([Sz, Sxz, Syz], -1)
    det = np.linalg.det(M)
    ok = active & (cnt >= 3) & (det > 1e-6 * Sw ** 3)
    Msafe = np.where(ok[..., None, None], M, np.eye(3))
    sol = np.linalg.solve(Msafe, np.where(ok[..., None], rhs, 0.0)[..., None])[..., 0]
    b, c = sol[..., 1], sol[..., 2]
    nrm = np.stack([-b, -c, np.ones_like(b)], -1)
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    nrm[~ok] = (0.0, 0.0, 1.0)
    return nrm


def apss_depth(t, active, normals, nbh: Neighbourhood, params: Params):
    """Depth projection onto the locally fitted algebraic sphere (APSS,
    Guennebaud & Gross 2007; the depth denoiser reading of Sec. 3)."""
    w = nbh.w
    x = np.broadcast_to(nbh.dx[:, None, None], w.shape)
    y = np.broadcast_to(nbh.dy[:, None, None], w.shape)
    z = nbh.dz
    nx = normals[nbh.nb, nbh.kk[:, None], 0][:, :, None]  # neighbour normals [S, P, 1]
    ny = normals[nbh.nb, nbh.kk[:, None], 1][:, :, None]
    nz = normals[nbh.nb, nbh.kk[:, None], 2][:, :, None]
    Sw = w.sum(0)
    Spx, Spy, Spz = (w * x).sum(0), (w * y).sum(0), (w * z).sum(0)
    Snx, Sny, Snz = (w * nx).sum(0), (w * ny).sum(0), (w * nz).sum(0)
    Spn = (w * (x * nx + y * ny + z * nz)).sum(0)
    Spp = (w * (x * x + y * y + z * z)).sum(0)
    cnt = (w > 0).sum(0)
    Swsafe = np.where(Sw > 0, Sw, 1.0)
    den = Spp - (Spx * Spx + Spy * Spy + Spz * Spz) / Swsafe
    densafe = np.where(den > 0, den, 1.0)
    u4 = 0.5 * (Spn - (Spx * Snx + Spy * Sny + Spz * Snz) / Swsafe) / densafe
    ux = (Snx - 2.0 * u4 * Spx) / Swsafe
    uy = (Sny - 2.0 * u4 * Spy) / Swsafe
    uz = (Snz - 2.0 * u4 * Spz) / Swsafe
    u0 = -(ux * Spx + uy * Spy + uz * Spz + u4 * Spp) / Swsafe
    disc = uz * uz - 4.0 * u4 * u0
    sq = np.sqrt(np.maximum(disc, 0.0))
    q = -0.5 * (uz + np.where(uz >= 0, sq, -sq))
    qsafe = np.where(q != 0, q, 1.0)
    z_near = u0 / qsafe
    u4safe = np.where(u4 != 0, u4, 1.0)
    z_far = np.where(u4 != 0, q / u4safe, np.inf)
    zs = np.where(np.abs(z_far) < np.abs(z_near), z_far, z_near)
    ok = (active & (cnt >= 3) & (den > 0) & (disc >= 0) & (q != 0)
          & (np.abs(zs) <= params.d_max * params.depth_scale))
    return np.where(ok, t + zs / params.depth_scale, t)


def smooth_prune(alpha, active, nbh: Neighbourhood, params: Params):
    """Intensity smoothing over the APSS neighbourhood, pruning, alpha_0 (the
    intensity step reading of Sec. 3; alpha_0 = 1 - sum alpha as in Eq. 1)."""
    w = nbh.w
    a_nb = alpha[nbh.nb, nbh.kk[:, None]][:, :, None]  # [S, P, 1]
    Sw = w.sum(0)
    Swa = (w * a_nb).sum(0)
    lam = params.smooth_lambda
    sm = np.where(Sw > 0, Swa / np.where(Sw > 0, Sw, 1.0), alpha)
    a_new = np.where(active, (1.0 - lam) * alpha + lam * sm, 0.0)
    act_new = active & (a_new >= params.prune_alpha)
    a_new = _project_simplex_cap(a_new, act_new)
    return a_new, act_new, 1.0 - a_new.sum(axis=1)


def iterate(z, n, t, alpha, active, hh, T: int, rows: int, cols: int, params: Params,
            eta_t: float, eta_a: float):
    """One SRT3D iteration: gradient step, then (if regularising) APSS depth
    projection and intensity smoothing/pruning on the post-gradient state.
    Pinned step by step and as a composition (post-gradient state feeds the
    neighbourhood, normals, sphere fit and smoothing); that RT3D's iteration
    is this sequence is a reading the paper cannot pin."""
    t1, a1 = gradient_step(z, n, t, alpha, active, hh, T, eta_t, eta_a, params.weighting)
    if not params.regularize:
        act = active.copy()
        return t1, a1, act, 1.0 - a1.sum(axis=1)
    nbh = neighbour_weights(t1, active, rows, cols, params)
    normals = plane_normals(nbh, active)
    t2 = apss_depth(t1, active, normals, nbh, params)
    a2, act2, a0 = smooth_prune(a1, active, nbh, params)
    return t2, a2, act2, a0


def birth_step(z, n, t, alpha, active, hh, T: int, params: Params):
    """RT3D birth move on the sketched loss (the reading in the module
    docstring): per pixel with a free slot, a new point at the argmax of the
    residual's matched filter outside the active points' exclusion zones, kept
    if its intensity reaches prune_alpha. Returns (t, alpha, active, alpha0)."""
    z = np.asarray(z)
    t = np.array(t, dtype=np.float64)
    act = np.array(active, dtype=bool)
    a = np.where(act, np.asarray(alpha, dtype=np.float64), 0.0)
    P, K = t.shape
    free = ~act.all(axis=1) & (np.asarray(n) > 0)
    if free.any():
        idx = np.nonzero(free)[0]
        w = 2.0 * np.pi * np.arange(1, hh.size + 1) / T
        r = z[idx].copy()

        def signatures(p, extra=None):
            # hhat e^{i w t} of the pixel's active points (and of depth `extra`)
            ts = list(t[p, act[p]]) + ([] if extra is None else [extra])
            return hh[None, :] * np.exp(1j * w[None, :] * np.array(ts, dtype=np.float64)[:, None])

        def fit(q, zp):
            # real least squares: z_p ~ sum_k beta_k q_k over the 2m real equations
            A = np.concatenate([q.real, q.imag], axis=1).T
            return np.linalg.lstsq(A, np.concatenate([zp.real, zp.imag]), rcond=None)[0]

        for j, p in enumerate(idx):
            if act[p].any():
                q = signatures(p)
                r[j] = z[p] - fit(q, z[p]) @ q
        s = matched_filter_scores(r, hh, T)
        grid = np.arange(T)[None, :]
        allowed = np.ones_like(s, bool)
        for k in range(K):
            tk = np.mod(np.floor(t[idx, k] + 0.5), T)
            near = _circ_dist(grid, tk[:, None], T) < params.min_sep
            allowed &= ~(near & act[idx, k][:, None])
        s = np.where(allowed, s, -np.inf)
        best = np.argmax(s, axis=1)
        sb = s[np.arange(idx.size), best]
        a_new = np.zeros(idx.size)
        for j, p in enumerate(idx):
            if np.isfinite(sb[j]):
                a_new[j] = max(0.0, fit(signatures(p, float(best[j])), z[p])[-1])
        born = a_new >= params.prune_alpha
        slot = np.argmin(act[idx], axis=1)  # first free slot
        for j in np.nonzero(born)[0]:
            p, k = idx[j], slot[j]
            t[p, k] = float(best[j])
            a[p, k] = a_new[j]
            act[p, k] = True
    a = _project_simplex_cap(a, act)
    return t, a, act, 1.0 - a.sum(axis=1)


def reconstruct(z, n, rows: int, cols: int, T: int, hh, params: Params, init=None):
    """Full reconstruction: init (matched filter, or `init` = (t, alpha,
    active)) then `params.iters` iterations. Returns (t, alpha, active, alpha0).
    Init and one iteration are pinned; the number of iterations and the
    reading of RT3D's loop are not fixed by the paper (parity unpinned
    beyond the ground-truth check of the small frame)."""
    z = np.asarray(z, dtype=np.complex128)
    n = np.asarray(n)
    if init is None:
        t, alpha, active, alpha0 = init_matched_filter(z, n, hh, T, params)
    else:
        t, alpha, active = (np.array(a, dtype=d) for a, d in zip(init, (float, float, bool)))
        alpha0 = 1.0 - np.where(active, alpha, 0.0).sum(axis=1)
    eta_t, eta_a = step_sizes(hh, n.max(initial=0), params.k_max, T)
    for it in range(params.iters):
        t, alpha, active, alpha0 = iterate(z, n, t, alpha, active, hh, T, rows, cols, params,
                                           eta_t, eta_a)
        if params.birth_every and (it + 1) % params.birth_every == 0 and it + 1 < params.iters:
            t, alpha, active, alpha0 = birth_step(z, n, t, alpha, active, hh, T, params)
    return t, alpha, active, alpha0
