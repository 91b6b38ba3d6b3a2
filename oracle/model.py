"""Oracle: characteristic function of the observation model and the sketched
loss (Sec. 2, Eqs. 1, 4, 5, 6; Sec. 3, Eq. 8 with W = I or W = Sigma^-1).

Test infrastructure only (see ``oracle/__init__.py``).

Readings of the paper taken here:
  * Eq. 4 writes exp(i w t) inside the sum over surfaces; it is read as
    exp(i w t_k).
  * The background term alpha_0 sinc(w T / 2) of Eq. 4 is the continuous
    approximation; for the discrete uniform law on {0..T-1} the exact
    characteristic function at w_l = 2 pi l / T (1 <= l <= T-1) is 0, so the
    background contributes nothing and alpha_0 enters only through
    sum_k alpha_k + alpha_0 = 1 (Sec. 2).
  * H = sum of h over one period; h is indexed by circular lag tau in [0, T)
    with the pulse peak at tau = 0, so a surface at depth t puts photons at
    (t + tau) mod T.
"""
from __future__ import annotations

import numpy as np


def h_hat(h, m: int) -> np.ndarray:
    """hhat_l = (1/H) sum_tau h(tau) exp(i w_l tau), l = 1..m (Eq. 4, Sec. 2)."""
    h = np.asarray(h, dtype=np.float64)
    T = h.size
    H = h.sum()
    tau = np.arange(T, dtype=np.int64)
    ell = np.arange(1, m + 1, dtype=np.int64)
    k = (ell[:, None] * tau[None, :]) % T
    return (np.exp(1j * (2.0 * np.pi * k / T)) @ h) / H


def _omega(m: int, T: int) -> np.ndarray:
    return 2.0 * np.pi * np.arange(1, m + 1, dtype=np.float64) / T


def model_cf(t, alpha, active, hh, T: int) -> np.ndarray:
    """Psi_l(theta) = sum_k alpha_k hhat_l exp(i w_l t_k) over active points:
    the characteristic function of the observation model at w_l (Sec. 2,
    Eq. 4), with the background term exactly 0 at the harmonics.

    t, alpha, active: [P, K]; hh: [m]. Returns complex128 [P, m].
    """
    t = np.asarray(t, dtype=np.float64)
    a = np.where(np.asarray(active, dtype=bool), np.asarray(alpha, dtype=np.float64), 0.0)
    w = _omega(hh.size, T)
    E = np.exp(1j * w[None, None, :] * t[:, :, None])  # [P, K, m]
    return np.einsum("pk,pkl->pl", a, E) * hh[None, :]


def sketched_loss(z, n, t, alpha, active, hh, T: int) -> np.ndarray:
    """Per-pixel n ||z - Psi_theta||^2 (Eq. 6 / Eq. 8 with W = I)."""
    r = np.asarray(z) - model_cf(t, alpha, active, hh, T)
    return np.asarray(n, dtype=np.float64) * np.sum(np.abs(r) ** 2, axis=1)


def sketched_gradient(z, n, t, alpha, active, hh, T: int):
    """Gradient of the per-pixel loss n ||z - Psi||^2 (Sec. 3, Eq. 8 with
    W = I) with respect to t_k and alpha_k.

    With r = z - Psi and E_kl = exp(i w_l t_k):
      dL/dt_k     = -2 n sum_l Re( conj(r_l) * i w_l alpha_k hhat_l E_kl )
      dL/dalpha_k = -2 n sum_l Re( conj(r_l) * hhat_l E_kl )
    Inactive points get zero gradient.
    """
    t = np.asarray(t, dtype=np.float64)
    act = np.asarray(active, dtype=bool)
    a = np.where(act, np.asarray(alpha, dtype=np.float64), 0.0)
    w = _omega(hh.size, T)
    r = np.asarray(z) - model_cf(t, alpha, active, hh, T)  # [P, m]
    E = np.exp(1j * w[None, None, :] * t[:, :, None])  # [P, K, m]
    dpsi_da = hh[None, None, :] * E  # d Psi_l / d alpha_k
    dpsi_dt = 1j * w[None, None, :] * a[:, :, None] * dpsi_da  # d Psi_l / d t_k
    nn = np.asarray(n, dtype=np.float64)[:, None]
    g_t = -2.0 * nn * np.sum(np.real(np.conj(r)[:, None, :] * dpsi_dt), axis=2)
    g_a = -2.0 * nn * np.sum(np.real(np.conj(r)[:, None, :] * dpsi_da), axis=2)
    return np.where(act, g_t, 0.0), np.where(act, g_a, 0.0)


# Ridge added to Sigma_theta before inverting it (Sigma_theta is singular for a
# noise-free point mass, alpha_0 = 0); a reading, the paper gives none.
SIGMA_RIDGE = 1e-3


def sigma_theta(t, alpha, active, hh, T: int) -> np.ndarray:
    """Sigma_theta of Eq. 5: the covariance of the vector (exp(i w_l x))_l,
    l = 1..m, for one photon x drawn from the model (Eq. 1), read as the
    Hermitian covariance
        Sigma_jk = Psi(w_j - w_k) - Psi(w_j) conj(Psi(w_k)),
    with Psi(0) = 1, Psi(w_{-d}) = conj(Psi(w_d)) and Psi(w_d) = Psi_d of
    model_cf for d >= 1 (the background vanishes at nonzero harmonics).
    Returns complex128 [P, m, m]."""
    psi = model_cf(t, alpha, active, hh, T)  # [P, m]
    P, m = psi.shape
    d = np.arange(m)[:, None] - np.arange(m)[None, :]  # j - k
    full = np.concatenate([np.conj(psi[:, ::-1]), np.ones((P, 1)), psi], axis=1)  # Psi_d, d = -m..m
    toep = full[:, d + m]  # Psi(w_j - w_k); index d + m maps d = 0 to the column of ones
    return toep - psi[:, :, None] * np.conj(psi)[:, None, :]


def weighting_matrix(t, alpha, active, hh, T: int) -> np.ndarray:
    """W = (Sigma_theta + SIGMA_RIDGE I)^-1 (the precision matrix of Eq. 6),
    [P, m, m]."""
    S = sigma_theta(t, alpha, active, hh, T)
    m = S.shape[1]
    return np.linalg.inv(S + SIGMA_RIDGE * np.eye(m)[None])


def weighted_loss(z, n, t, alpha, active, hh, T: int, W) -> np.ndarray:
    """Per-pixel n (z - Psi)^H W (z - Psi) (Eq. 6 with a given W [P, m, m])."""
    r = np.asarray(z) - model_cf(t, alpha, active, hh, T)
    return np.asarray(n, dtype=np.float64) * np.real(np.einsum("pj,pjk,pk->p", np.conj(r), W, r))


def weighted_gradient(z, n, t, alpha, active, hh, T: int, W):
    """Gradient of weighted_loss (Sec. 2, Eq. 6 with W = Sigma_theta^-1 of
    Eq. 5) with W held fixed: with r = z - Psi and
    v = W r,  dL/dtheta = -2 n Re( sum_l conj(dPsi_l/dtheta) v_l ), i.e. the
    W = I gradient of sketched_gradient with r replaced by v."""
    t = np.asarray(t, dtype=np.float64)
    act = np.asarray(active, dtype=bool)
    a = np.where(act, np.asarray(alpha, dtype=np.float64), 0.0)
    w = _omega(hh.size, T)
    r = np.asarray(z) - model_cf(t, alpha, active, hh, T)
    v = np.einsum("pjk,pk->pj", W, r)
    E = np.exp(1j * w[None, None, :] * t[:, :, None])
    dpsi_da = hh[None, None, :] * E
    dpsi_dt = 1j * w[None, None, :] * a[:, :, None] * dpsi_da
    nn = np.asarray(n, dtype=np.float64)[:, None]
    g_t = -2.0 * nn * np.sum(np.real(np.conj(v)[:, None, :] * dpsi_dt), axis=2)
    g_a = -2.0 * nn * np.sum(np.real(np.conj(v)[:, None, :] * dpsi_da), axis=2)
    return np.where(act, g_t, 0.0), np.where(act, g_a, 0.0)
