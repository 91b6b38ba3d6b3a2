"""Oracle: characteristic function of the observation model and the sketched
loss (Sec. 2, Eqs. 1, 4, 6; Sec. 3, Eq. 8 with W = I).

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
    """Psi_l(theta) = sum_k alpha_k hhat_l exp(i w_l t_k) over active points.

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
    """Gradient of the per-pixel loss with respect to t_k and alpha_k.

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
