"""Pins of the oracle's particles in the CPML mode (Sec. 2.2 E_Maxwell with the
convolutional PML on a non-periodic grid, particle modules of Sec. 2.2, absorbing
particle walls): exact charge conservation in the interior, equality with the pinned
periodic cycle before the boundaries matter, and ballistic absorption.  No GPU."""

import numpy as np

import oracle


def _interior(n, margin):
    j, i = np.meshgrid(np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return ((i >= margin) & (i < n[0] - margin) & (j >= margin) & (j < n[1] - margin)).ravel()


def test_interior_keeps_div_e_minus_rho():
    """E starts at zero, so div E - rho starts at -rho; the Esirkepov current keeps
    that difference at every node whose update neither the layer nor the wall touches,
    while particles reach the layer and are absorbed at the walls."""
    rng = np.random.default_rng(11)
    n, dx, dt, c, npml = (40, 36), (1.0, 0.9), 0.1, 2.0, 6
    box = np.array([(n[0] - 1) * dx[0], (n[1] - 1) * dx[1]])
    x = 2.0 + rng.uniform(0, 1, (3000, 2)) * (box - 4.0)
    v = rng.normal(0, 1.5, (3000, 3))  # |v| dt well under a cell: the current's stencil
    sim = oracle.CpmlPlasma(n, dx, dt, c, npml, weight=0.05, B0=(0.0, 0.0, 0.4)).load(x, v)
    inner = _interior(n, npml + 2)
    d0 = sim.gauss_residual()[inner]
    for _ in range(40):
        sim.step(1)
        assert np.abs(sim.v[:, :2] * dt).max() < 0.9 * min(dx)
    assert sim.absorbed > 0
    d1 = sim.gauss_residual()[inner]
    assert np.abs(d1 - d0).max() <= 1e-12 * np.abs(d0).max()
    # away from the interior the layer and the walls do change it
    assert np.abs(sim.gauss_residual()[~inner] + sim.rho[~inner]).max() > 1e-6


def test_equals_the_periodic_cycle_before_the_boundaries_matter():
    """Particles in the middle of a large grid, both runs from E = B = 0 without the
    half push: for the first steps no signal reaches the layer, so fields and particles
    equal those of the periodic oracle cycle."""
    rng = np.random.default_rng(12)
    n, dx, dt, c, npml = (64, 60), (1.0, 1.0), 0.1, 2.0, 8
    x = np.array([27.0, 25.0]) + rng.uniform(0, 8.0, (500, 2))
    v = rng.normal(0, 1.0, (500, 3))
    cp = oracle.CpmlPlasma(n, dx, dt, c, npml, weight=0.3).load(x, v, half_push=False)
    pe = oracle.EmSimulation(n, dx, dt, c, weight=0.3).load(x, v, half_push=False)
    pe.E[:] = 0.0
    for _ in range(6):
        cp.step(1)
        pe.step(1)
    np.testing.assert_allclose(cp.E, pe.E, rtol=0, atol=1e-13)
    np.testing.assert_allclose(cp.B, pe.B, rtol=0, atol=1e-13)
    np.testing.assert_allclose(cp.x, pe.x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(cp.v, pe.v, rtol=0, atol=1e-12)
    assert np.abs(cp.E).max() > 1e-6 and cp.absorbed == 0


def test_ballistic_particles_are_absorbed_when_they_leave():
    """Test particles (weight 0: no current, no field) move in straight lines; each is
    absorbed at the end of the step in which it leaves the box, no earlier."""
    rng = np.random.default_rng(13)
    n, dx, dt, c, npml = (20, 16), (1.0, 1.0), 0.25, 1.0, 4
    box = np.array([19.0, 15.0])
    x = rng.uniform(0.5, 1.0, (400, 2)) * box
    v = rng.normal(0, 3.0, (400, 3))
    sim = oracle.CpmlPlasma(n, dx, dt, c, npml, weight=0.0).load(x, v, half_push=False)
    for s in range(1, 9):
        sim.step(1)
        pos = x + v[:, :2] * dt * s
        stayed = np.ones(len(x), bool)
        for k in range(1, s + 1):
            p = x + v[:, :2] * dt * k
            stayed &= np.all((p >= 0) & (p < box), axis=1)
        assert sim.x.shape[0] == int(stayed.sum())
        np.testing.assert_allclose(sim.x, pos[stayed], rtol=0, atol=1e-12)
        assert sim.absorbed == len(x) - int(stayed.sum())
    assert sim.absorbed > 0
