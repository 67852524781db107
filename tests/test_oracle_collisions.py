"""Pins of the oracle's null-collision Monte Carlo step (Sec. 2.2 G_collision, the
null-collision method of Vahedi and Surendra) with synthetic constant cross
sections, and of its counter-based generator: statistics and exact kinematics that
the method fixes whatever the implementation."""

import math

import numpy as np
import pytest

N24 = float(1 << 24)


def _params(**kw):
    p = dict(density=1.0, sigma_el=0.05, sigma_exc=0.0, eps_exc=0.0, mass_ratio=0.0,
             vmax=3.0, seed=11)
    p.update(kw)
    return p


def _beam(n, speed=1.0, seed=5, isotropic=True):
    rng = np.random.default_rng(seed)
    if isotropic:
        d = rng.standard_normal((n, 3))
        d /= np.linalg.norm(d, axis=1)[:, None]
    else:
        d = np.tile([1.0, 0.0, 0.0], (n, 1))
    return np.ascontiguousarray(d * speed)


def test_rng24_is_uniform_and_independent(orc):
    n = 1 << 20
    a = orc.rng24_fill(7, 3, 0, n, 0).astype(np.float64)
    b = orc.rng24_fill(7, 3, 0, n, 1).astype(np.float64)
    c = orc.rng24_fill(7, 4, 0, n, 0).astype(np.float64)
    assert a.max() < N24 and a.min() >= 0
    # 256-bin chi-square: mean 255, sd ~22.6; 6 sd bound
    for x in (a, b, c):
        h = np.bincount((x // (N24 / 256)).astype(np.int64), minlength=256)
        chi2 = float(np.sum((h - n / 256) ** 2 / (n / 256)))
        assert abs(chi2 - 255) < 6 * math.sqrt(2 * 255), chi2
        assert abs(x.mean() / N24 - 0.5) < 6 * math.sqrt(1 / 12 / n)
    # draws of the same particle, of neighbouring particles and of the next step
    # are uncorrelated
    for x, y in ((a, b), (a, c), (a[1:], a[:-1])):
        r = np.corrcoef(x, y)[0, 1]
        assert abs(r) < 6 / math.sqrt(n), r
    # a counter bit flips about half of the output bits (avalanche)
    flips = [bin(orc.rng24(7, 3, i, 0) ^ orc.rng24(7, 3, i ^ 1, 0)).count("1") for i in range(4096)]
    assert abs(np.mean(flips) - 12.0) < 0.5
    assert orc.rng24(7, 3, 12345, 2) == orc.rng24(7, 3, 12345, 2)


def test_mcc_real_collision_count_matches_the_null_collision_probability(orc):
    """A fraction P' = 1 - exp(-nu' dt) of the particles are candidates and a
    candidate of speed v collides with probability nu(v) / nu'; the count is binomial.
    A larger bound nu' changes the null fraction, not the real rate (to first order)."""
    n, dt = 200_000, 0.1
    for vmax in (3.0, 6.0):
        p = _params(vmax=vmax)
        v = _beam(n)
        counts = orc.mcc(v, np.arange(n), 1, p, 1.0, dt)
        nu, nu_max = p["density"] * p["sigma_el"] * 1.0, p["density"] * p["sigma_el"] * vmax
        P = orc.mcc_threshold(p["density"], p["sigma_el"], 0.0, vmax, dt) / N24
        assert abs(P - (1 - math.exp(-nu_max * dt))) < 1e-7
        mean = n * P * nu / nu_max
        assert abs(counts[0] - mean) < 5 * math.sqrt(mean), (vmax, counts, mean)
        assert abs(counts[0] - n * nu * dt) < 5 * math.sqrt(mean) + n * nu * dt * nu_max * dt
        assert counts[1] == 0 and counts[2] == 0


def test_mcc_elastic_kinematics(orc):
    """Without recoil (m/M = 0) a scattered electron keeps its speed exactly; with recoil
    its energy drops to E (1 - 2 (m/M) (1 - cos chi)), chi the deflection angle."""
    n = 50_000
    p = _params(sigma_el=10.0, vmax=1.0)  # every candidate at v = vmax collides
    v = _beam(n)
    v0 = v.copy()
    counts = orc.mcc(v, np.arange(n), 2, p, 1.0, 0.1)
    hit = np.any(v != v0, axis=1)
    assert hit.sum() == counts[0] > 0
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, rtol=0, atol=1e-14)
    mu = 0.01
    v = _beam(n)
    orc.mcc(v, np.arange(n), 2, _params(sigma_el=10.0, vmax=1.0, mass_ratio=mu), 1.0, 0.1)
    hit = np.any(v != v0, axis=1)
    cos_chi = np.sum(v[hit] * v0[hit], axis=1) / np.linalg.norm(v[hit], axis=1)
    e_ratio = np.sum(v[hit] ** 2, axis=1)
    np.testing.assert_allclose(e_ratio, 1 - 2 * mu * (1 - cos_chi), rtol=0, atol=1e-13)


def test_mcc_scattering_is_isotropic(orc):
    """A beam along +x scattered once (every particle a candidate that collides) has
    directions uniform on the sphere: zero mean, each squared component 1/3, and
    cos chi uniform on [-1, 1]."""
    n = 200_000
    p = _params(sigma_el=1e4, vmax=1.0)  # P' = 1 to FP64, nu(v) = nu'
    v = _beam(n, isotropic=False)
    counts = orc.mcc(v, np.arange(n), 3, p, 1.0, 0.1)
    assert counts[0] == n
    d = v / np.linalg.norm(v, axis=1)[:, None]
    for k in range(3):
        assert abs(d[:, k].mean()) < 6 / math.sqrt(3 * n)
        assert abs((d[:, k] ** 2).mean() - 1 / 3) < 6 * math.sqrt(4 / 45 / n)
    h, _ = np.histogram(d[:, 0], bins=20, range=(-1, 1))
    chi2 = float(np.sum((h - n / 20) ** 2 / (n / 20)))
    assert chi2 < 19 + 6 * math.sqrt(38)


def test_mcc_excitation_loses_the_threshold_energy(orc):
    """An excitation removes exactly eps_exc; electrons below the threshold never excite."""
    n, eps = 40_000, 0.3
    rng = np.random.default_rng(9)
    speed = rng.uniform(0.2, 1.5, n)  # energies 0.02 .. 1.125, about a quarter below eps
    v = _beam(n) * speed[:, None]
    v0 = v.copy()
    p = _params(sigma_el=0.0, sigma_exc=20.0, eps_exc=eps, vmax=1.5)
    counts = orc.mcc(v, np.arange(n), 4, p, 1.0, 0.1)
    e0 = 0.5 * np.sum(v0 ** 2, axis=1)
    e1 = 0.5 * np.sum(v ** 2, axis=1)
    hit = np.any(v != v0, axis=1)
    assert hit.sum() == counts[1] > 1000 and counts[0] == 0
    np.testing.assert_allclose(e0[hit] - e1[hit], eps, rtol=0, atol=1e-13)
    assert np.all(e0[hit] >= eps)


def test_mcc_momentum_relaxation(orc):
    """Isotropic elastic collisions randomise the direction, so a cold beam's mean
    velocity decays by the factor (1 - p) per step, p = P' nu / nu'."""
    n, dt, steps = 100_000, 0.1, 20
    p = _params(sigma_el=0.5, vmax=2.0)
    v = _beam(n, isotropic=False)
    ids = np.arange(n)
    for s in range(1, steps + 1):
        orc.mcc(v, ids, s, p, 1.0, dt)
    P = orc.mcc_threshold(1.0, 0.5, 0.0, 2.0, dt) / N24
    keep = (1 - P * 0.5 / 1.0) ** steps
    assert abs(v[:, 0].mean() - keep) < 6 * math.sqrt((1 - keep ** 2) / 3 / n) + 1e-3


def test_mcc_depends_on_ids_not_on_storage_order(orc):
    """The draws are keyed by particle id and step, so permuting the storage order
    (a sort) permutes the result and nothing else."""
    n = 5000
    p = _params(sigma_el=2.0, sigma_exc=1.0, eps_exc=0.2, mass_ratio=0.02, vmax=2.0)
    v = _beam(n, speed=1.2)
    w = v.copy()
    perm = np.random.default_rng(3).permutation(n)
    wp = np.ascontiguousarray(w[perm])
    c1 = orc.mcc(v, np.arange(n), 7, p, 1.0, 0.1)
    c2 = orc.mcc(wp, perm, 7, p, 1.0, 0.1)
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(wp, v[perm])


def test_simulation_with_collisions_and_sort(orc):
    """The cycle with collisions: charge stays exact, excitation energy is accounted
    for, and the ids follow the sort."""
    from workloads import plasma
    w = plasma.maxwellian_box(1, (64,), ppc=50, nv=3, dt=0.1, seed=12)
    p = _params(sigma_el=0.2, sigma_exc=0.1, eps_exc=0.5, mass_ratio=1e-3, vmax=6.0)
    sim = orc.Simulation(1, w.n, w.dx, w.dt, weight=w.weight, collisions=p).load(w.x, w.v)
    tot = np.zeros(3, np.int64)
    for s in range(5):
        sim.step(1)
        tot += sim.mcc_counts
        if s == 2:
            sim.sort((16,))
    assert tot[0] > 0 and tot[1] > 0 and tot[2] == 0
    assert sorted(sim.ids.tolist()) == list(range(w.np_))
