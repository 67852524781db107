"""Closed forms and analysis used to pin the oracle (test infrastructure).

* Warm symmetric two-stream dispersion relation (Sec. 3.2, Eqs. 5-6):
      eps(w, k) = 1 + 1 / (2 (k lambda_De)^2) * sum_{s=+-1} [1 + zeta_s Z(zeta_s)] = 0,
      zeta_s = (w - s k_x u_d) / (sqrt(2) k v_te),
  with Z the plasma dispersion function, Z(z) = i sqrt(pi) w(z) for Im z > 0
  (w the Faddeeva function).  For symmetric beams the unstable root is purely
  growing, w = i gamma, and eps(i gamma) is real.
* Mode amplitude of the parallel field (Sec. 3.2, Eq. 3): E_par = k . E / |k|,
  amplitude 2 |E_hat(m)| with E_hat the 1/N-normalised forward DFT, so a
  cosine of amplitude A has 2|E_hat| = A.
* Least-squares growth-rate fit of ln(amplitude) against t (Sec. 3.2, Eq. 4).
* Boris gyration: per step the velocity turns by theta = 2 atan(w_c dt / 2).
"""

from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq
from scipy.special import wofz


def plasma_Z(zeta):
    """Plasma dispersion function via the Faddeeva function (valid for Im zeta > 0,
    and by analytic continuation of w(z) everywhere)."""
    return 1j * math.sqrt(math.pi) * wofz(zeta)


def two_stream_eps(omega, k_vec, u_d=3.0, v_te=1.0):
    k = math.sqrt(sum(kk * kk for kk in k_vec))
    kx = k_vec[0]
    total = 0.0
    for s in (+1, -1):
        zeta = (omega - s * kx * u_d) / (math.sqrt(2.0) * k * v_te)
        total += 1.0 + zeta * plasma_Z(zeta)
    klam = k * v_te  # k lambda_De with lambda_De = v_te / w_pe and w_pe = 1
    return 1.0 + total / (2.0 * klam * klam)


def two_stream_gamma(k_vec, u_d=3.0, v_te=1.0, lo=1e-4, hi=2.0):
    """Growth rate of the purely growing root, eps(i gamma) = 0."""
    f = lambda g: float(np.real(two_stream_eps(1j * g, k_vec, u_d, v_te)))  # noqa: E731
    return brentq(f, lo, hi, xtol=1e-14, rtol=1e-14, maxiter=500)


def mode_k(mode, n, dx):
    return [2.0 * math.pi * mode[a] / (n[a] * dx[a]) for a in range(len(mode))]


def mode_amplitude(E, ndim, n, dx, mode):
    """2 |E_hat_par(mode)| of a component-major node field E (ndim x cells),
    by an explicit DFT sum over the nodes."""
    n = list(n)[:ndim]
    dx = list(dx)[:ndim]
    k = mode_k(mode, n, dx)
    kn = math.sqrt(sum(kk * kk for kk in k))
    cells = int(np.prod(n))
    E = np.asarray(E, dtype=np.float64).reshape(ndim, cells)
    Epar = sum(k[a] * E[a] for a in range(ndim)) / kn
    # node coordinates, axis 0 fastest
    idx = np.arange(cells)
    phase = np.zeros(cells)
    stride = 1
    for a in range(ndim):
        ja = (idx // stride) % n[a]
        phase += k[a] * ja * dx[a]
        stride *= n[a]
    Ehat = np.sum(Epar * np.exp(-1j * phase)) / cells
    return 2.0 * abs(Ehat)


def fit_growth(t, amp, t_lo, t_hi):
    """Least-squares line through ln(amp) on t_lo <= t <= t_hi; returns
    (gamma, R^2)."""
    t = np.asarray(t, dtype=np.float64)
    y = np.log(np.asarray(amp, dtype=np.float64))
    sel = (t >= t_lo - 1e-9) & (t <= t_hi + 1e-9)
    A = np.vstack([t[sel], np.ones(sel.sum())]).T
    coef, *_ = np.linalg.lstsq(A, y[sel], rcond=None)
    pred = A @ coef
    ss_res = float(np.sum((y[sel] - pred) ** 2))
    ss_tot = float(np.sum((y[sel] - y[sel].mean()) ** 2))
    return float(coef[0]), 1.0 - ss_res / ss_tot


def fit_frequency(t, signal, omega_guess=1.0):
    """Angular frequency of a sampled oscillation by least squares on
    a cos(w t) + b sin(w t) + c, scanning w then refining by golden section."""
    t = np.asarray(t, dtype=np.float64)
    s = np.asarray(signal, dtype=np.float64)

    def resid(w):
        A = np.vstack([np.cos(w * t), np.sin(w * t), np.ones_like(t)]).T
        coef, *_ = np.linalg.lstsq(A, s, rcond=None)
        return float(np.sum((A @ coef - s) ** 2))

    ws = np.linspace(0.5 * omega_guess, 1.5 * omega_guess, 401)
    rs = [resid(w) for w in ws]
    i = int(np.argmin(rs))
    a, b = ws[max(i - 1, 0)], ws[min(i + 1, len(ws) - 1)]
    g = (math.sqrt(5.0) - 1.0) / 2.0
    c, d = b - g * (b - a), a + g * (b - a)
    for _ in range(100):
        if resid(c) < resid(d):
            b = d
        else:
            a = c
        c, d = b - g * (b - a), a + g * (b - a)
    return 0.5 * (a + b)


def boris_gyro_angle(omega_c, dt):
    return 2.0 * math.atan(0.5 * omega_c * dt)
