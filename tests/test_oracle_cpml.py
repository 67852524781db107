"""Pins of the oracle's convolutional PML (Sec. 2.2 E_Maxwell: FDTD with CPML,
Roden and Gedney 2000) on the non-periodic 2D Yee grid: with the layer switched off it
is a conducting cavity whose standing mode follows the Yee dispersion exactly; with the
layer on, a pulse leaves the box with little reflection (against the same probe in a
box too large for any reflection to return), less for thicker layers, and its energy
is absorbed."""

import math

import numpy as np
import pytest


def test_cavity_mode_without_layer(orc):
    """npml = 0: Ez = sin(pi a x / Lx) sin(pi b y / Ly), B = 0, in a conducting box is an
    eigenmode; after n steps Ez = cos(n theta) Ez0, sin(theta / 2) = (c dt / 2) K."""
    n, dx, c, dt = (21, 17), (1.0, 0.8), 1.1, 0.3
    a, b = 2, 3
    k = [math.pi * a / ((n[0] - 1) * dx[0]), math.pi * b / ((n[1] - 1) * dx[1])]
    i, j = np.meshgrid(np.arange(n[0]), np.arange(n[1]), indexing="xy")
    ez0 = (np.sin(k[0] * i * dx[0]) * np.sin(k[1] * j * dx[1])).ravel()
    f = orc.CpmlField(n, dx, dt, c, npml=0)
    f.E[2] = ez0
    K = math.sqrt(sum((2 * math.sin(k[q] * dx[q] / 2) / dx[q]) ** 2 for q in range(2)))
    theta = 2 * math.asin(0.5 * c * dt * K)
    for s in range(1, 31):
        f.step()
        np.testing.assert_allclose(f.E[2], math.cos(s * theta) * ez0, rtol=0, atol=1e-11)


def _pulse_run(orc, size, npml, steps=300, off=15):
    dt, c = 0.5, 1.0
    f = orc.CpmlField((size, size), (1.0, 1.0), dt, c, npml)
    cx = size // 2
    t0, tw = 40 * dt, 10 * dt
    J = np.zeros((3, size * size))
    rec = []
    for s in range(steps):
        t = (s + 0.5) * dt
        J[2, cx + size * cx] = -((t - t0) / tw) * math.exp(-((t - t0) / tw) ** 2)
        f.step(J)
        rec.append(f.E[2, (cx + off) + size * cx])
    return np.array(rec), f


def test_cpml_absorbs_an_outgoing_pulse(orc):
    ref, _ = _pulse_run(orc, 300, 12)
    peak = np.abs(ref).max()
    err = {}
    for npml in (8, 12, 16):
        rec, f = _pulse_run(orc, 72, npml)
        err[npml] = np.abs(rec - ref).max() / peak
    pec, _ = _pulse_run(orc, 72, 0)
    err_pec = np.abs(pec - ref).max() / peak
    assert err[12] < 6e-3 and err[16] < err[12] < err[8] < 1e-2
    assert err_pec > 0.5
    # the pulse's energy is absorbed once it has left
    _, f = _pulse_run(orc, 72, 12, steps=900)
    _, fpec = _pulse_run(orc, 72, 0, steps=900)
    assert f.energy() < 1e-6 * fpec.energy()


def test_cpml_profile_values(orc):
    """The layer's coefficients along one axis (n = 40 nodes, 10-cell layers, c = 1.5,
    dx = 0.75, step h = 0.4, cubic grading): outside the layers b = 1, c = 0, 1/kappa = 1
    (the plain FDTD update); at the outer node (depth 1) sigma is the matched value
    0.8 (m + 1) c / dx, so b = exp(-sigma_max h) and, with kappa = 1 and alpha = 0,
    c = b - 1; one cell in (depth 0.9) sigma = sigma_max 0.9^3; the profile is mirror
    symmetric and the damping grows towards the wall.  With kappa_max and alpha_max set,
    c = sigma (b - 1) / (sigma kappa + kappa^2 alpha) at a hand-evaluated point."""
    n, npml, dx, h, cl, m = 40, 10, 0.75, 0.4, 1.5, 3
    prof = orc.cpml_axis(n, npml, dx, h, cl, m=m)
    b, cc, ik = prof["int"]
    smax = 0.8 * (m + 1) * cl / dx
    inner = slice(npml, n - npml)
    np.testing.assert_array_equal(b[inner], 1.0)
    np.testing.assert_array_equal(cc[inner], 0.0)
    np.testing.assert_array_equal(ik, 1.0)
    assert b[0] == pytest.approx(math.exp(-smax * h), rel=1e-15)
    assert cc[0] == pytest.approx(b[0] - 1.0, rel=1e-14)
    assert b[1] == pytest.approx(math.exp(-smax * 0.9 ** 3 * h), rel=1e-15)
    np.testing.assert_allclose(b, b[::-1], rtol=0, atol=0)
    assert np.all(np.diff(b[: npml + 1]) > 0)
    bh, ch, _ = prof["half"]
    # half positions: node i + 1/2 mirrors node n - 2 - i + 1/2
    np.testing.assert_allclose(bh[: n - 1], bh[: n - 1][::-1], rtol=1e-15)
    assert bh[0] == pytest.approx(math.exp(-smax * 0.95 ** 3 * h), rel=1e-15)
    # kappa and alpha grading
    kmax, amax = 4.0, 0.2
    prof = orc.cpml_axis(n, npml, dx, h, cl, m=m, kappa_max=kmax, alpha_max=amax)
    b, cc, ik = prof["int"]
    d = 0.9
    sig, kap, alp = smax * d ** m, 1.0 + (kmax - 1.0) * d ** m, amax * (1.0 - d)
    bb = math.exp(-(sig / kap + alp) * h)
    assert b[1] == pytest.approx(bb, rel=1e-15)
    assert cc[1] == pytest.approx(sig * (bb - 1.0) / (sig * kap + kap * kap * alp), rel=1e-14)
    assert ik[1] == pytest.approx(1.0 / kap, rel=1e-15)
