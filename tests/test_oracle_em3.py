"""Pins of the oracle's 3D electromagnetic step (Sec. 2.2 E_Maxwell: FDTD on the Yee
lattice, with the Esirkepov current and staggered CIC gathers), against closed forms,
exact invariants and the pinned 2D3V step.  No GPU."""

import numpy as np
import pytest

import oracle


def _rand3(rng, n):
    return rng.normal(size=(3, n[0] * n[1] * n[2]))


def test_yee3_reduces_to_the_2d_lattice():
    """Fields that do not depend on z evolve on every z-slice exactly as the 2D3V Yee
    update (pinned by its own eigenmode test) evolves them."""
    rng = np.random.default_rng(1)
    n2, nz, dx, c, dt = (9, 7), 3, (0.7, 1.1, 0.9), 1.3, 0.2
    E2, B2, J2 = (rng.normal(size=(3, n2[0] * n2[1])) for _ in range(3))
    tile = lambda F: np.ascontiguousarray(np.tile(F, (1, nz)))  # z-independent 3D field
    n3 = (n2[0], n2[1], nz)
    E3, B3, J3 = tile(E2), tile(B2), tile(J2)
    for _ in range(3):
        oracle.yee_b(n2, dx[:2], E2, B2, 0.5 * dt)
        oracle.yee3_b(n3, dx, E3, B3, 0.5 * dt)
        oracle.yee_e(n2, dx[:2], B2, J2, c, dt, E2)
        oracle.yee3_e(n3, dx, B3, J3, c, dt, E3)
    np.testing.assert_allclose(E3, tile(E2), rtol=0, atol=1e-13)
    np.testing.assert_allclose(B3, tile(B2), rtol=0, atol=1e-13)


def _rotate(F, n):
    """Relabel the axes (x, y, z) -> (z', x', y'): the field with components (Fy, Fz, Fx)
    on the grid transposed accordingly.  Yee positions map onto Yee positions."""
    out = []
    for a in (1, 2, 0):
        G = F[a].reshape(n[2], n[1], n[0])  # [z, y, x]
        out.append(np.ascontiguousarray(G.transpose(2, 0, 1)).ravel())
    return np.ascontiguousarray(np.array(out))


def test_yee3_commutes_with_a_rotation_of_the_axes():
    """On a cubic lattice the update commutes with the cyclic relabelling of the axes:
    every curl term is checked against its rotated partner."""
    rng = np.random.default_rng(2)
    n, dx, c, dt = (5, 5, 5), (1.0, 1.0, 1.0), 1.0, 0.3
    E, B, J = _rand3(rng, n), _rand3(rng, n), _rand3(rng, n)
    Er, Br, Jr = _rotate(E, n), _rotate(B, n), _rotate(J, n)
    oracle.yee3_b(n, dx, E, B, dt)
    oracle.yee3_b(n, dx, Er, Br, dt)
    oracle.yee3_e(n, dx, B, J, c, dt, E)
    oracle.yee3_e(n, dx, Br, Jr, c, dt, Er)
    np.testing.assert_allclose(_rotate(B, n), Br, rtol=0, atol=1e-13)
    np.testing.assert_allclose(_rotate(E, n), Er, rtol=0, atol=1e-13)


def test_yee3_standing_mode_follows_the_exact_dispersion():
    """A divergence-free standing wave E = E0 cos(k.x) (E0 perpendicular to the discrete
    wave vector K_a = (2 / dx_a) sin(k_a dx_a / 2)), B = 0, oscillates as cos(n theta)
    with sin(theta / 2) = c dt |K| / 2, exactly, in the split step the cycle uses."""
    n, dx, c, dt = (8, 6, 10), (1.0, 0.8, 1.2), 1.0, 0.35
    m = (1, 2, 3)
    k = np.array([2 * np.pi * m[a] / (n[a] * dx[a]) for a in range(3)])
    K = np.array([2.0 / dx[a] * np.sin(k[a] * dx[a] / 2) for a in range(3)])
    E0 = np.cross(K, [1.0, 0.3, -0.2])  # perpendicular to K
    offs = ((0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5))
    z, y, x = np.meshgrid(*(np.arange(n[a]) for a in (2, 1, 0)), indexing="ij")
    E = np.zeros((3, n[0] * n[1] * n[2]))
    for a in range(3):
        pos = [(x + offs[a][0]) * dx[0], (y + offs[a][1]) * dx[1], (z + offs[a][2]) * dx[2]]
        E[a] = (E0[a] * np.cos(k[0] * pos[0] + k[1] * pos[1] + k[2] * pos[2])).ravel()
    E_init = E.copy()
    B = np.zeros_like(E)
    J = np.zeros_like(E)
    theta = 2.0 * np.arcsin(c * dt * np.linalg.norm(K) / 2.0)
    for s in range(1, 41):
        oracle.yee3_b(n, dx, E, B, 0.5 * dt)
        oracle.yee3_e(n, dx, B, J, c, dt, E)
        oracle.yee3_b(n, dx, E, B, 0.5 * dt)
        np.testing.assert_allclose(E, E_init * np.cos(s * theta), rtol=0, atol=1e-11)
    assert abs(theta - c * dt * np.linalg.norm(k)) > 1e-4  # the discrete, not the exact, rate


def test_yee3_keeps_div_b_zero():
    rng = np.random.default_rng(3)
    n, dx, c, dt = (6, 7, 5), (0.9, 1.0, 1.1), 1.0, 0.3
    E, J = _rand3(rng, n), _rand3(rng, n)
    B = np.zeros_like(E)
    for _ in range(20):
        oracle.yee3_b(n, dx, E, B, 0.5 * dt)
        oracle.yee3_e(n, dx, B, J, c, dt, E)
        oracle.yee3_b(n, dx, E, B, 0.5 * dt)
    assert np.abs(B).max() > 1.0
    assert np.abs(oracle.yee3_div_b(n, dx, B)).max() <= 1e-12 * np.abs(B).max()


@pytest.mark.parametrize("seed", [4, 5])
def test_esirkepov3_conserves_charge_exactly(seed):
    """rho(x1) - rho(x0) + dt div J = 0 at every node for moves under one cell per axis
    (wrapping across the periodic box included)."""
    rng = np.random.default_rng(seed)
    n, dx, dt, qw = (6, 5, 7), (1.0, 0.7, 1.3), 0.4, -0.37
    L = np.array([n[a] * dx[a] for a in range(3)])
    x0 = rng.uniform(0, 1, (300, 3)) * L
    x1 = np.mod(x0 + rng.uniform(-0.95, 0.95, (300, 3)) * np.asarray(dx), L)
    J = np.zeros((3, n[0] * n[1] * n[2]))
    oracle.esirkepov3(n, dx, x0, x1, qw, dt, J)
    rho0 = oracle.deposit(3, n, dx, x0, qw)
    rho1 = oracle.deposit(3, n, dx, x1, qw)
    res = rho1 - rho0 + dt * oracle.yee3_div_e(n, dx, J)
    assert np.abs(res).max() <= 1e-13 * np.abs(rho1).max()


def test_esirkepov3_current_of_a_straight_move():
    """A particle moving along x inside one cell row deposits only Jx, and the x-current
    summed over the grid is q w vx / V per unit volume: sum_nodes Jx dV = q w vx."""
    n, dx, dt, qw = (6, 6, 6), (1.0, 1.0, 1.0), 0.5, 0.8
    x0 = np.array([[2.3, 3.4, 1.7]])
    x1 = x0 + np.array([[0.4, 0.0, 0.0]])
    J = np.zeros((3, 216))
    oracle.esirkepov3(n, dx, x0, x1, qw, dt, J)
    assert np.abs(J[1]).max() == 0.0 and np.abs(J[2]).max() == 0.0
    assert J[0].sum() * 1.0 == pytest.approx(qw * 0.4 / dt, rel=1e-14)


def test_em3_gather_interpolates_linear_fields_exactly():
    """Each component is a linear function sampled at its own staggered positions; CIC
    on that lattice gives it back exactly at any point away from the periodic seam."""
    rng = np.random.default_rng(6)
    n, dx = (9, 8, 10), (0.8, 1.0, 1.2)
    offs = ((0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0))
    coef = rng.normal(size=(6, 4))
    z, y, x = np.meshgrid(*(np.arange(n[a]) for a in (2, 1, 0)), indexing="ij")
    F = np.zeros((6, n[0] * n[1] * n[2]))
    for q in range(6):
        pos = [(x + offs[q][0]) * dx[0], (y + offs[q][1]) * dx[1], (z + offs[q][2]) * dx[2]]
        F[q] = (coef[q, 0] + coef[q, 1] * pos[0] + coef[q, 2] * pos[1] + coef[q, 3] * pos[2]).ravel()
    lo = np.array([1.0, 1.0, 1.0]) * np.asarray(dx)
    hi = (np.array(n) - 2.0) * np.asarray(dx)
    p = lo + rng.uniform(0, 1, (50, 3)) * (hi - lo)
    got = oracle.em3_gather(n, dx, p, F[:3], F[3:])
    want = coef[:, 0][None, :] + p @ coef[:, 1:].T
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_em3_cycle_keeps_gauss_law():
    """Load (E from the Poisson potential), then full cycles with particles: div E = rho
    holds at every node to rounding, because the Esirkepov current conserves charge."""
    rng = np.random.default_rng(7)
    n, dx, dt, c = (6, 5, 4), (1.0, 1.0, 1.0), 0.1, 3.0
    npart = 4 * n[0] * n[1] * n[2]
    L = np.array([n[a] * dx[a] for a in range(3)])
    x = rng.uniform(0, 1, (npart, 3)) * L
    v = rng.normal(0, 1, (npart, 3))
    sim = oracle.EmSimulation3(n, dx, dt, c, weight=float(np.prod(L)) / npart,
                               B0=(0.0, 0.0, 0.5)).load(x, v)
    scale = np.abs(sim.rho).max()
    assert np.abs(sim.gauss_residual()).max() <= 1e-9 * scale
    sim.step(8)
    assert np.abs(sim.gauss_residual()).max() <= 1e-9 * scale
    assert np.abs(oracle.yee3_div_b(n, dx, sim.B)).max() <= 1e-12 * max(np.abs(sim.B).max(), 1e-30)


def test_em3_cold_plasma_oscillates_at_the_plasma_frequency():
    """A cold electron lattice displaced by a small sine along x (weight such that
    omega_p = 1) oscillates longitudinally in the full 3D electromagnetic cycle: the
    mode's Ex changes sign at a rate within 1 % of omega_p (the coupling's signs and
    magnitudes in 3D)."""
    n, dx, dt = (32, 4, 4), (0.5, 0.5, 0.5), 0.05
    L = np.array([n[a] * dx[a] for a in range(3)])
    gx = np.arange(2 * n[0]) / (2 * n[0]) * L[0]
    gy, gz = (np.arange(n[1]) + 0.5) * dx[1], (np.arange(n[2]) + 0.5) * dx[2]
    X, Y, Z = np.meshgrid(gx, gy, gz, indexing="ij")
    x = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    k = 2 * np.pi / L[0]
    x[:, 0] = np.mod(x[:, 0] + 0.01 * np.sin(k * x[:, 0]), L[0])
    sim = oracle.EmSimulation3(n, dx, dt, c=5.0, weight=float(np.prod(L)) / x.shape[0])
    sim.load(x, np.zeros_like(x))
    W = np.broadcast_to(np.sin(k * (np.arange(n[0]) + 0.5) * dx[0]), (n[2], n[1], n[0])).ravel()
    sig = []
    for _ in range(300):
        sim.step(1)
        sig.append(float(np.sum(sim.E[0] * W)))
    sig = np.array(sig)
    t = [(i - 1) + sig[i - 1] / (sig[i - 1] - sig[i]) for i in range(1, len(sig))
         if sig[i - 1] * sig[i] < 0]
    assert len(t) >= 4
    omega = np.pi / (np.mean(np.diff(t)) * dt)
    assert abs(omega - 1.0) < 0.01, omega
