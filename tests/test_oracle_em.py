"""Pins of the oracle's electromagnetic step (Sec. 2.2 E_Maxwell: Yee FDTD) and its
particle coupling on a periodic 2D3V grid: the exact discrete dispersion of the Yee
scheme, div B = 0, exact charge continuity of the Esirkepov current, exact
interpolation of linear fields on the staggered lattices, and Gauss's law kept by the
full cycle."""

import math

import numpy as np
import pytest

N = (24, 18)
DX = (1.0, 0.75)


def _nodes():
    i, j = np.meshgrid(np.arange(N[0]), np.arange(N[1]), indexing="xy")
    return i.ravel().astype(float), j.ravel().astype(float)


def test_yee_standing_mode_follows_the_discrete_dispersion(orc):
    """Ez = cos(k . x) with B = 0 is an eigenmode of the leapfrog Yee update: after n
    steps Ez = cos(n theta) Ez0 with sin(theta / 2) = (c dt / 2) K,
    K^2 = sum_a (2 sin(k_a dx_a / 2) / dx_a)^2 (Yee 1966)."""
    c, dt = 1.3, 0.25
    m = (3, 2)
    k = [2 * math.pi * m[a] / (N[a] * DX[a]) for a in range(2)]
    i, j = _nodes()
    ez0 = np.cos(k[0] * i * DX[0] + k[1] * j * DX[1])
    E = np.zeros((3, N[0] * N[1]))
    E[2] = ez0
    B = np.zeros_like(E)
    J = np.zeros_like(E)
    K = math.sqrt(sum((2 * math.sin(k[a] * DX[a] / 2) / DX[a]) ** 2 for a in range(2)))
    theta = 2 * math.asin(0.5 * c * dt * K)
    for step in range(1, 41):
        orc.yee_b(N, DX, E, B, 0.5 * dt)
        orc.yee_e(N, DX, B, J, c, dt, E)
        orc.yee_b(N, DX, E, B, 0.5 * dt)
        np.testing.assert_allclose(E[2], math.cos(step * theta) * ez0, rtol=0, atol=1e-11)
    assert np.abs(E[:2]).max() == 0.0 and np.abs(B[2]).max() == 0.0


def test_yee_keeps_div_b_zero(orc):
    rng = np.random.default_rng(1)
    E = rng.standard_normal((3, N[0] * N[1]))
    B = np.zeros_like(E)
    for _ in range(10):
        J = rng.standard_normal(E.shape)
        orc.yee_b(N, DX, E, B, 0.05)
        orc.yee_e(N, DX, B, J, 2.0, 0.1, E)
        orc.yee_b(N, DX, E, B, 0.05)
    assert np.abs(orc.yee_div_b(N, DX, B)).max() < 1e-12
    assert np.abs(B).max() > 0.1


def test_esirkepov_current_conserves_charge_exactly(orc):
    """rho(x1) - rho(x0) + dt div J = 0 on every node, for random moves of less than a
    cell per axis (some across the periodic boundary)."""
    rng = np.random.default_rng(2)
    npart, qw, dt = 500, -0.7, 0.3
    L = np.array([N[0] * DX[0], N[1] * DX[1]])
    x0 = rng.uniform(0, 1, (npart, 2)) * L
    d = rng.uniform(-0.99, 0.99, (npart, 2)) * np.array(DX)
    x1 = (x0 + d) % L
    vz = rng.standard_normal(npart)
    J = np.zeros((3, N[0] * N[1]))
    orc.esirkepov(N, DX, x0, x1, vz, qw, dt, J)
    rho0 = orc.deposit(2, N, DX, x0, qw)
    rho1 = orc.deposit(2, N, DX, x1, qw)
    resid = rho1 - rho0 + dt * orc.yee_div_e(N, DX, J)
    assert np.abs(resid).max() < 1e-13 * np.abs(rho0).max()
    assert np.abs(J[:2]).max() > 0.1


def test_esirkepov_without_motion_is_density_times_vz(orc):
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (200, 2)) * np.array([N[0] * DX[0], N[1] * DX[1]])
    vz = np.full(200, 1.7)
    J = np.zeros((3, N[0] * N[1]))
    orc.esirkepov(N, DX, x, x, vz, 0.4, 0.1, J)
    assert np.abs(J[:2]).max() == 0.0
    np.testing.assert_allclose(J[2], 1.7 * orc.deposit(2, N, DX, x, 0.4), rtol=0, atol=1e-13)


def test_em_gather_is_exact_for_linear_fields(orc):
    """Each component, linear in x and y on its own staggered lattice, is interpolated
    exactly (away from the periodic seam)."""
    sx = [0.5, 0.0, 0.0, 0.0, 0.5, 0.5]
    sy = [0.0, 0.5, 0.0, 0.5, 0.0, 0.5]
    i, j = _nodes()
    coef = np.array([[0.3, -0.2, 0.1], [1.0, 0.5, -0.7], [-0.4, 0.9, 0.2],
                     [0.6, 0.1, 0.3], [-0.1, -0.5, 0.8], [0.2, 0.4, -0.6]])
    F = np.zeros((6, N[0] * N[1]))
    for k in range(6):
        xs, ys = (i + sx[k]) * DX[0], (j + sy[k]) * DX[1]
        F[k] = coef[k, 0] + coef[k, 1] * xs + coef[k, 2] * ys
    rng = np.random.default_rng(4)
    x = np.column_stack([rng.uniform(2, N[0] - 3, 100) * DX[0], rng.uniform(2, N[1] - 3, 100) * DX[1]])
    out = orc.em_gather(N, DX, x, F[:3], F[3:])
    want = coef[:, 0][None, :] + np.outer(x[:, 0], coef[:, 1]) + np.outer(x[:, 1], coef[:, 2])
    np.testing.assert_allclose(out, want, rtol=0, atol=1e-12)


def test_boris_eb_gyrates_in_gathered_uniform_B(orc):
    """A uniform Bz gathered from the grid drives the exact Boris gyration."""
    E = np.zeros((3, N[0] * N[1]))
    B = np.zeros_like(E)
    B[2] = 1.5
    x = np.array([[5.3, 4.1]])
    EB = orc.em_gather(N, DX, x, E, B)
    np.testing.assert_allclose(EB[0], [0, 0, 0, 0, 0, 1.5], atol=1e-15)
    v = np.array([[1.0, 0.0, 0.2]])
    orc.boris_eb(v, EB, -1.0, 0.1)
    assert abs(math.atan2(v[0, 1], v[0, 0]) - 2 * math.atan(0.5 * 1.5 * 0.1)) < 1e-14


def test_em_cycle_keeps_gauss_law_and_div_b(orc):
    """Through full cycles with particles, div E - rho stays at its load value (zero:
    the load solves Poisson) and div B at zero."""
    from workloads import plasma
    w = plasma.maxwellian_box(2, N, ppc=6, nv=3, dt=0.1, seed=5, dx=DX)
    sim = orc.EmSimulation(N, DX, 0.1, c=3.0, weight=w.weight, B0=(0, 0, 0.5)).load(w.x, w.v)
    scale = np.abs(sim.rho).max()
    assert np.abs(sim.gauss_residual()).max() < 1e-9 * scale
    sim.step(15)
    assert np.abs(sim.gauss_residual()).max() < 1e-9 * scale
    assert np.abs(orc.yee_div_b(N, DX, sim.B)).max() < 1e-12
    assert np.abs(sim.B).max() > 0.0 and np.abs(sim.J).max() > 0.0
