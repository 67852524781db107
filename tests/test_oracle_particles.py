"""Pins of the oracle's particle steps: the Boris push (Sec. 2.2 A_Pusher, module A01
in Sec. 3.1) and the Higuera-Cary push the same module lists, the position update with periodic wrap (application code in Sec. 3.1)
and the per-cell sort (a layout step the paper does not name)."""

import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_boris_pure_B_keeps_speed(orc):
    rng = np.random.default_rng(21)
    v = rng.standard_normal((8, 3))
    s0 = np.linalg.norm(v, axis=1)
    B0 = (0.3, -1.1, 2.0)
    for _ in range(10_000):
        orc.boris(3, v, None, (0, 0, 0), B0, -1.0, 0.05)
    assert np.abs(np.linalg.norm(v, axis=1) - s0).max() < 1e-12


def test_boris_gyro_angle_and_sense(orc):
    """Per step the perpendicular velocity turns by exactly 2 atan(w_c dt / 2); an
    electron (q/m = -1) in B along +z turns from +x towards +y."""
    wc, dt = 2.0, 0.05
    v = np.array([[1.0, 0.0, 0.4]])
    orc.boris(3, v, None, (0, 0, 0), (0, 0, wc), -1.0, dt)
    theta = math.atan2(v[0, 1], v[0, 0])
    assert abs(theta - 2 * math.atan(0.5 * wc * dt)) < 1e-14
    assert abs(v[0, 2] - 0.4) < 1e-15
    # after many steps the accumulated phase is k * theta (mod 2 pi)
    v = np.array([[1.0, 0.0, 0.0]])
    k = 997
    for _ in range(k):
        orc.boris(3, v, None, (0, 0, 0), (0, 0, wc), -1.0, dt)
    want = math.remainder(k * 2 * math.atan(0.5 * wc * dt), 2 * math.pi)
    assert abs(math.remainder(math.atan2(v[0, 1], v[0, 0]) - want, 2 * math.pi)) < 1e-11


def test_boris_ExB_drift(orc):
    """With uniform E perpendicular to B, u = v - E x B / |B|^2 is rotated by the
    Boris angle each step and keeps its length: the mean velocity is the E x B drift."""
    E = np.array([0.3, -0.2, 0.0])
    B = np.array([0.0, 0.0, 1.5])
    vd = np.cross(E, B) / np.dot(B, B)
    dt, qm = 0.1, -1.0
    theta = 2 * math.atan(0.5 * abs(qm) * 1.5 * dt)
    v = np.array([[0.7, 0.1, 0.2]])
    u0 = v[0] - vd
    Ep = np.zeros((1, 3))
    for k in range(1, 200):
        orc.boris(3, v, Ep, tuple(E), tuple(B), qm, dt)
        u = v[0] - vd
        ang = math.atan2(u[1], u[0]) - math.atan2(u0[1], u0[0])
        assert abs(math.remainder(ang - k * theta, 2 * math.pi)) < 1e-11
        assert abs(np.hypot(u[0], u[1]) - np.hypot(u0[0], u0[1])) < 1e-12
        assert abs(u[2] - u0[2]) < 1e-13


def test_boris_without_B_is_leapfrog(orc):
    rng = np.random.default_rng(22)
    v = rng.standard_normal((50, 2))
    Ep = rng.standard_normal((50, 2))
    want = v + (-1.0) * Ep * 0.1
    orc.boris(2, v, Ep, (0, 0, 0), (0, 0, 0), -1.0, 0.1)
    np.testing.assert_allclose(v, want, rtol=0, atol=1e-15)


def test_boris_is_time_reversible(orc):
    """A step of h followed by a step of -h with the same fields restores v (the
    backward half push relies on this)."""
    rng = np.random.default_rng(23)
    v = rng.standard_normal((20, 3))
    v0 = v.copy()
    Ep = rng.standard_normal((20, 3))
    orc.boris(3, v, Ep, (0.1, 0, 0), (0.2, 0.5, 1.0), -1.0, 0.07)
    orc.boris(3, v, Ep, (0.1, 0, 0), (0.2, 0.5, 1.0), -1.0, -0.07)
    np.testing.assert_allclose(v, v0, atol=1e-14)


# ---- Higuera-Cary (the relativistic pusher of Sec. 2.2 A_Pusher) ---------------------------

def _rand_fields(seed, n=16):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n, 3)) * 2.0
    Ep = rng.standard_normal((n, 3)) * 0.3
    return u, Ep


def test_hc_is_the_implicit_midpoint_rotation(orc):
    """The defining relation: with u-/u+ the momenta before/after the rotation,
    u+ - u- = (u- + u+) x tau / gamma(mean momentum), tau = (q/m) B h / 2."""
    u, Ep = _rand_fields(31)
    E0, B0, qm, h, c = (0.05, -0.1, 0.2), (0.3, -0.2, 1.5), -1.0, 0.08, 2.0
    u0 = u.copy()
    orc.higuera_cary(3, u, Ep, E0, B0, qm, h, c)
    eps = 0.5 * qm * h
    E = Ep + np.array(E0)
    um, up = u0 + eps * E, u - eps * E
    ub = 0.5 * (um + up)
    gb = np.sqrt(1.0 + np.sum(ub * ub, axis=1) / c ** 2)
    rhs = np.cross(um + up, eps * np.array(B0)[None, :] / gb[:, None])
    np.testing.assert_allclose(up - um, rhs, rtol=0, atol=1e-13)


def test_hc_nonrelativistic_limit_is_boris(orc):
    u, Ep = _rand_fields(32)
    v = u.copy()
    args = ((0.05, -0.1, 0.2), (0.3, -0.2, 1.5), -1.0, 0.08)
    orc.higuera_cary(3, u, Ep, *args, c=None)
    orc.boris(3, v, Ep, *args)
    np.testing.assert_allclose(u, v, rtol=0, atol=1e-14)
    # and a very large c approaches it
    u2 = _rand_fields(32)[0]
    orc.higuera_cary(3, u2, Ep, *args, c=1e7)
    np.testing.assert_allclose(u2, v, rtol=0, atol=1e-10)


def test_hc_pure_B_keeps_momentum_and_turns_at_the_midpoint_gamma(orc):
    """In pure B |u| (hence gamma) is kept; per step u turns by 2 atan(|tau| / gamma_bar)
    about B, gamma_bar the Lorentz factor of the mean momentum, in the electron's sense."""
    c, wc, h = 2.0, 1.5, 0.05
    u = np.array([[3.0, 1.0, 0.0]])
    s0 = np.linalg.norm(u)
    for _ in range(1000):
        orc.higuera_cary(3, u, None, (0, 0, 0), (0.3, -0.2, 1.1), -1.0, h, c)
    assert abs(np.linalg.norm(u) - s0) < 1e-12 * s0
    u = np.array([[3.0, 1.0, 0.0]])
    u0 = u[0].copy()
    orc.higuera_cary(3, u, None, (0, 0, 0), (0, 0, wc), -1.0, h, c)
    ub = 0.5 * (u0 + u[0])
    gb = math.sqrt(1.0 + ub.dot(ub) / c ** 2)
    ang = math.atan2(u0[0] * u[0, 1] - u0[1] * u[0, 0], u0.dot(u[0]))
    assert abs(ang - 2 * math.atan(0.5 * wc * h / gb)) < 1e-14
    # gamma_bar < gamma: the relativistic gyro-frequency is below the classical one
    assert gb < math.sqrt(1.0 + u0.dot(u0) / c ** 2)


def test_hc_relativistic_ExB_drift_is_exact(orc):
    """A particle moving with the E x B drift, u = gamma_d E x B / |B|^2, is a fixed
    point of the Higuera-Cary step at any step size (the property that sets it apart
    from Boris, which is also checked here to miss it)."""
    c, Ey, Bz, qm = 1.0, 0.5, 1.0, -1.0
    E, B = np.array([0.0, Ey, 0.0]), np.array([0.0, 0.0, Bz])
    vd = np.cross(E, B) / B.dot(B)
    ud = vd / math.sqrt(1.0 - vd.dot(vd) / c ** 2)
    for h in (0.05, 0.5, 2.0):
        u = ud[None, :].copy()
        for _ in range(10):
            orc.higuera_cary(3, u, None, tuple(E), tuple(B), qm, h, c)
        np.testing.assert_allclose(u[0], ud, rtol=0, atol=1e-14)
        v = ud[None, :].copy()
        orc.boris(3, v, None, tuple(E), tuple(B), qm, h)
        assert np.abs(v[0] - ud).max() > 1e-3


def test_hc_without_B_is_leapfrog_in_momentum(orc):
    u, Ep = _rand_fields(33)
    want = u + (-1.0) * 0.1 * Ep
    orc.higuera_cary(3, u, Ep, (0, 0, 0), (0, 0, 0), -1.0, 0.1, 0.7)
    np.testing.assert_allclose(u, want, rtol=0, atol=1e-14)


def test_lorentz_gamma_values(orc):
    """gamma = sqrt(1 + |u|^2 / c^2): |u| = c sqrt(3) gives 2 in any direction, |u| = c
    gives sqrt(2), u = 0 gives 1, and c = infinity gives 1 for any u."""
    c = 2.5
    rng = np.random.default_rng(11)
    dirs = rng.normal(size=(8, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    np.testing.assert_allclose(orc.lorentz_gamma(dirs * c * math.sqrt(3.0), c), 2.0, rtol=1e-15)
    np.testing.assert_allclose(orc.lorentz_gamma(dirs * c, c), math.sqrt(2.0), rtol=1e-15)
    assert orc.lorentz_gamma(np.zeros((1, 3)), c)[0] == 1.0
    np.testing.assert_array_equal(orc.lorentz_gamma(dirs * 1e3, None), 1.0)


def test_relativistic_kinetic_energy(orc):
    u, _ = _rand_fields(34)
    c, mw = 1.7, 2.5
    gamma = np.sqrt(1.0 + np.sum(u * u, axis=1) / c ** 2)
    assert abs(orc.kinetic_rel(u, mw, c) - mw * c ** 2 * np.sum(gamma - 1.0)) < 1e-12 * mw * c ** 2
    assert abs(orc.kinetic_rel(u, mw, None) - orc.kinetic(u, mw)) < 1e-12


def test_hc_simulation_moves_with_u_over_gamma(orc):
    """In a uniform external E (no self-field: negligible weight) the momentum grows
    by q E dt / m per step and the position advances by u / gamma dt (the
    relativistic velocity), wrapped into the box."""
    c, dt, Ex = 1.5, 0.1, 0.4
    sim = orc.Simulation(1, (64,), (1.0,), dt, weight=1e-12, E0=(Ex, 0, 0), pusher="hc", c=c)
    x0 = np.array([[10.0]])
    sim.load(x0, np.array([[0.0, 0.0, 0.0]]), half_push=False)
    x = 10.0
    u = 0.0
    for _ in range(50):
        u += -1.0 * Ex * dt
        x += u / math.sqrt(1.0 + u * u / c ** 2) * dt
        sim.step(1)
    assert abs(sim.v[0, 0] - u) < 1e-12
    assert abs(sim.x[0, 0] - (x % 64.0)) < 1e-9
    assert abs(sim.velocity()[0, 0]) < c


def test_move_wraps(orc):
    n, dx = (4, 3), (1.0, 2.0)  # L = (4, 6)
    x = np.array([[3.9, 5.5], [0.1, 0.2], [1.0, 1.0], [2.0, 3.0]])
    v = np.array([[1.0, 1.0], [-1.0, -1.0], [12.5, -13.0], [2.0, 3.0]])
    orc.move(2, n, dx, x, v, 0.1)
    want = np.array([[0.0, 5.6], [0.0, 0.1], [2.25, 5.7], [2.2, 3.3]])
    want[0, 0] = 3.9 + 0.1 - 4.0
    np.testing.assert_allclose(x, want, atol=1e-12)
    assert np.all(x >= 0) and np.all(x[:, 0] < 4) and np.all(x[:, 1] < 6)


def test_move_landing_on_L_wraps_to_zero(orc):
    x = np.array([[3.5]])
    orc.move(1, (4,), (1.0,), x, np.array([[5.0]]), 0.1)  # 3.5 + 0.5 = 4.0 = L
    assert x[0, 0] == 0.0


def test_sort_key_hand_worked(orc):
    rows, nkeys = [], None
    with open(os.path.join(GOLDEN, "sort_key_6x4_brick4x2.txt")) as f:
        for line in f:
            tok = line.split()
            if not tok or tok[0].startswith("#"):
                continue
            if tok[0] == "nkeys":
                nkeys = int(tok[1])
            elif tok[0] == "row":
                rows.append([int(t) for t in tok[1:]])
    cells = np.arange(24, dtype=np.int64)  # c = c0 + 6 c1
    key = orc.sort_key(2, (6, 4), (4, 2), cells)
    assert key.tolist() == [k for r in rows for k in r]
    assert orc.num_keys(2, (6, 4), (4, 2)) == nkeys


def test_counting_sort_is_stable_sort(orc):
    rng = np.random.default_rng(24)
    key = rng.integers(0, 37, size=5000).astype(np.int64)
    perm = orc.counting_sort(key, 37)
    want = sorted(range(key.size), key=lambda i: key[i])  # Python's sort is stable
    assert perm.tolist() == want


def test_counting_sort_rejects_out_of_range(orc):
    with pytest.raises(ValueError):
        orc.counting_sort(np.array([0, 5, 2], dtype=np.int64), 5)


def test_locate_cells_and_offsets(orc):
    x = np.array([[0.0, 0.0], [1.75, 2.5], [3.999999999999, 5.9999999999999]])
    cell, off = orc.locate(2, (4, 3), (1.0, 2.0), x)
    assert cell.tolist() == [0, 1 + 4 * 1, 3 + 4 * 2]
    np.testing.assert_allclose(off[1], [0.75, 0.25])


def test_simulation_sort_permutes_state(orc):
    rng = np.random.default_rng(25)
    n, dx = (8, 8), (1.0, 1.0)
    x = rng.random((300, 2)) * 8
    sim = orc.Simulation(2, n, dx, 0.1, weight=64 / 300).load(x, rng.standard_normal((300, 2)))
    x_before, v_before = sim.x.copy(), sim.v.copy()
    perm = sim.sort((4, 4))
    np.testing.assert_array_equal(sim.x, x_before[perm])
    np.testing.assert_array_equal(sim.v, v_before[perm])
    cell, _ = sim.cells_offsets()
    key = orc.sort_key(2, n, (4, 4), cell)
    assert np.all(np.diff(key) >= 0)
