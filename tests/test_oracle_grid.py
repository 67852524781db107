"""Pins of the oracle's particle-grid coupling and field solve against hand-worked
values, closed forms and invariants (no GPU).

Deposit / gather: Sec. 2.2 (B_Scatter, C_Gather), modules B01 / C01 in Sec. 3.1.
Poisson / E:      Sec. 2.2 (D_Poisson), modules D02 / D06 in Sec. 3.1.
"""

import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_deposit_cases():
    cases, cur = [], None
    with open(os.path.join(GOLDEN, "deposit_small.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "case":
                cur = dict(name=tok[1], ndim=int(tok[2]), n=tuple(int(t) for t in tok[3:6]),
                           dx=tuple(float(t) for t in tok[6:9]), qw=float(tok[9]), x=[], rho={})
                cases.append(cur)
            elif tok[0] == "p":
                cur["x"].append([float(t) for t in tok[1:]])
            elif tok[0] == "rho":
                for item in tok[1:]:
                    i, val = item.split(":")
                    cur["rho"][int(i)] = float(val)
    return cases


@pytest.mark.parametrize("case", _read_deposit_cases(), ids=lambda c: c["name"])
def test_deposit_hand_worked(orc, case):
    x = np.array(case["x"], dtype=np.float64)
    rho = orc.deposit(case["ndim"], case["n"], case["dx"], x, case["qw"])
    want = np.zeros_like(rho)
    for i, val in case["rho"].items():
        want[i] = val
    np.testing.assert_allclose(rho, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("ndim,n,dx", [(1, (37,), (0.7,)), (2, (13, 9), (1.0, 0.5)),
                                       (3, (5, 7, 6), (1.0, 1.3, 0.8))])
def test_deposit_total_charge(orc, ndim, n, dx):
    rng = np.random.default_rng(11)
    L = np.array([n[a] * dx[a] for a in range(ndim)])
    x = rng.random((5000, ndim)) * L
    qw = -0.37
    rho = orc.deposit(ndim, n, dx, x, qw)
    dV = float(np.prod(dx))
    assert abs(rho.sum() * dV - qw * x.shape[0]) <= 1e-12 * abs(qw) * x.shape[0]


@pytest.mark.parametrize("ndim,n,dx", [(1, (16,), (0.5,)), (2, (8, 6), (1.0, 0.75)),
                                       (3, (4, 5, 6), (1.0, 0.5, 2.0))])
def test_deposit_first_moment(orc, ndim, n, dx):
    """Linear weighting keeps each particle's position as the weighted mean of
    the nodes it touches: sum_j W_j x_j = x_p when no wrap is involved.  A
    swapped (1 - f, f) pair or a wrong corner index breaks this."""
    rng = np.random.default_rng(12)
    for _ in range(20):
        x = np.array([[rng.uniform(0, (n[a] - 1) * dx[a]) for a in range(ndim)]])
        rho = orc.deposit(ndim, n, dx, x, float(np.prod(dx)))  # qw/dV = 1 -> rho = W
        assert abs(rho.sum() - 1.0) < 1e-14
        idx = np.arange(rho.size)
        stride = 1
        for a in range(ndim):
            ja = (idx // stride) % n[a]
            stride *= n[a]
            assert abs(np.sum(rho * ja * dx[a]) - x[0, a]) < 1e-12


def test_deposit_translation(orc):
    """Shifting every particle by one cell on axis 1 rolls rho by one node."""
    rng = np.random.default_rng(13)
    n, dx = (7, 5, 4), (1.0, 0.5, 1.5)
    L = np.array([n[a] * dx[a] for a in range(3)])
    x = rng.random((300, 3)) * L
    rho = orc.deposit(3, n, dx, x, 1.0).reshape(n[2], n[1], n[0])
    x2 = x.copy()
    x2[:, 1] = np.mod(x2[:, 1] + dx[1], L[1])
    rho2 = orc.deposit(3, n, dx, x2, 1.0).reshape(n[2], n[1], n[0])
    np.testing.assert_allclose(rho2, np.roll(rho, 1, axis=1), atol=1e-13)


def test_gather_linear_field_exact(orc):
    """Linear weights interpolate a field that is linear inside the cell exactly."""
    n, dx = (10, 8), (0.5, 1.0)
    j0, j1 = np.meshgrid(np.arange(n[0]), np.arange(n[1]), indexing="xy")
    a, bx, by = 0.3, -1.7, 2.4
    Ex = (a + bx * j0 * dx[0] + by * j1 * dx[1]).ravel()
    Ey = (2 * a - by * j0 * dx[0] + 0.5 * bx * j1 * dx[1]).ravel()
    E = np.concatenate([Ex, Ey])
    rng = np.random.default_rng(14)
    x = np.stack([rng.uniform(0, (n[0] - 1) * dx[0], 200),
                  rng.uniform(0, (n[1] - 1) * dx[1], 200)], axis=1)
    Ep = orc.gather(2, n, dx, x, E)
    np.testing.assert_allclose(Ep[:, 0], a + bx * x[:, 0] + by * x[:, 1], atol=1e-12)
    np.testing.assert_allclose(Ep[:, 1], 2 * a - by * x[:, 0] + 0.5 * bx * x[:, 1], atol=1e-12)


@pytest.mark.parametrize("ndim,n,dx", [(1, (12,), (1.0,)), (2, (9, 7), (1.0, 0.6)),
                                       (3, (5, 4, 6), (0.8, 1.0, 1.1))])
def test_gather_is_adjoint_of_deposit(orc, ndim, n, dx):
    """sum_j rho_j g_j = (qw/dV) sum_p G_p with G the gathered g: gather and
    deposit use the same weights at the same nodes."""
    rng = np.random.default_rng(15)
    L = np.array([n[a] * dx[a] for a in range(ndim)])
    x = rng.random((400, ndim)) * L
    cells = int(np.prod(n))
    g = rng.standard_normal(ndim * cells)
    qw = 0.9
    rho = orc.deposit(ndim, n, dx, x, qw)
    G = orc.gather(ndim, n, dx, x, g)
    dV = float(np.prod(dx))
    for a in range(ndim):
        lhs = np.dot(rho, g[a * cells:(a + 1) * cells])
        rhs = qw / dV * G[:, a].sum()
        assert abs(lhs - rhs) < 1e-11 * (abs(lhs) + 1)


def _dft_poisson(ndim, n, dx, rho):
    """phi = IDFT(rho_hat / K^2) with K^2 = sum_a (2 sin(k_a dx_a / 2) / dx_a)^2, the
    symbol of the (2d+1)-point Laplacian; the k = 0 mode is dropped.  DFT by explicit
    complex-exponential matrices (brute force, O(N^2))."""
    cells = int(np.prod(n))
    idx = np.arange(cells)
    coords = []
    stride = 1
    for a in range(ndim):
        coords.append((idx // stride) % n[a])
        stride *= n[a]
    phase = np.zeros((cells, cells))
    K2 = np.zeros(cells)
    for a in range(ndim):
        ka = 2 * math.pi * coords[a] / (n[a] * dx[a])
        phase += np.outer(coords[a] * dx[a], ka)  # x_j . k_m
        K2 += (2 * np.sin(ka * dx[a] / 2) / dx[a]) ** 2
    F = np.exp(-1j * phase)  # rows: nodes, cols: modes
    rho_hat = F.T @ rho
    phi_hat = np.zeros_like(rho_hat)
    nz = K2 > 1e-14
    phi_hat[nz] = rho_hat[nz] / K2[nz]
    phi = (np.conj(F) @ phi_hat).real / cells
    return phi


@pytest.mark.parametrize("ndim,n,dx", [(1, (8,), (0.5,)), (2, (4, 6), (1.0, 0.7)),
                                       (3, (4, 4, 3), (1.0, 0.9, 1.2))])
def test_poisson_matches_dft_closed_form(orc, ndim, n, dx):
    rng = np.random.default_rng(16)
    rho = rng.standard_normal(int(np.prod(n)))
    phi, iters, rel = orc.poisson(ndim, n, dx, rho, rtol=1e-14)
    want = _dft_poisson(ndim, n, dx, rho)
    assert abs(phi.mean()) < 1e-13
    np.testing.assert_allclose(phi, want, atol=1e-10 * np.abs(want).max())


def test_neg_laplacian_eigenvalue(orc):
    """-lap_h applied to a Fourier mode multiplies it by K^2 = sum (2 sin(k dx/2)/dx)^2."""
    n, dx = (16, 12), (0.5, 1.0)
    j0, j1 = np.meshgrid(np.arange(n[0]), np.arange(n[1]), indexing="xy")
    k = (2 * math.pi * 3 / (n[0] * dx[0]), 2 * math.pi * 2 / (n[1] * dx[1]))
    u = np.cos(k[0] * j0 * dx[0] + k[1] * j1 * dx[1]).ravel()
    K2 = sum((2 * math.sin(k[a] * dx[a] / 2) / dx[a]) ** 2 for a in range(2))
    np.testing.assert_allclose(orc.neg_laplacian(2, n, dx, u), K2 * u, atol=1e-12)


def test_efield_of_sine_potential(orc):
    """phi = sin(k x) gives E = -(sin(k dx) / dx) cos(k x) under centred differences,
    and the periodic field sums to zero."""
    n, dx = (24,), (0.25,)
    xj = np.arange(n[0]) * dx[0]
    k = 2 * math.pi * 2 / (n[0] * dx[0])
    E = orc.efield(1, n, dx, np.sin(k * xj))
    np.testing.assert_allclose(E, -(math.sin(k * dx[0]) / dx[0]) * np.cos(k * xj), atol=1e-13)
    rng = np.random.default_rng(17)
    E3 = orc.efield(3, (4, 5, 3), (1.0, 0.5, 2.0), rng.standard_normal(60))
    for a in range(3):
        assert abs(E3[a * 60:(a + 1) * 60].sum()) < 1e-12


@pytest.mark.parametrize("ndim,n,dx", [(1, (32,), (1.0,)), (2, (16, 12), (1.0, 1.0)),
                                       (3, (6, 5, 8), (1.0, 1.0, 1.0))])
def test_no_self_force(orc, ndim, n, dx):
    """With the same weights for deposit and gather, a symmetric Green's function and
    an antisymmetric gradient, a lone particle feels no force from its own charge
    (momentum conservation); the uniform background drops out with the mean."""
    rng = np.random.default_rng(18)
    L = np.array([n[a] * dx[a] for a in range(ndim)])
    for _ in range(5):
        x = rng.random((1, ndim)) * L
        sim = orc.Simulation(ndim, n, dx, 0.1, weight=1.0, rtol=1e-14).load(x, np.zeros((1, 3)),
                                                                            half_push=False)
        Ep = orc.gather(ndim, n, dx, sim.x, sim.E)
        assert np.abs(Ep).max() < 1e-12 * (np.abs(sim.E).max() + 1e-300) + 1e-14


def test_total_force_vanishes(orc):
    """sum_p q E_p = sum_j rho_e,j E_j dV = 0 for many particles (momentum conservation
    of the momentum-conserving scheme), to the CG tolerance."""
    rng = np.random.default_rng(19)
    n, dx = (16, 16), (1.0, 1.0)
    x = rng.random((2000, 2)) * 16
    sim = orc.Simulation(2, n, dx, 0.1, weight=256 / 2000, rtol=1e-14).load(
        x, np.zeros((2000, 2)), half_push=False)
    Ep = orc.gather(2, n, dx, sim.x, sim.E)
    F = Ep.sum(axis=0)
    assert np.abs(F).max() < 1e-10 * np.abs(Ep).sum(axis=0).max()
