"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.

Bars: bit-exact cell indices and sort permutations; 1e-5 relative L-infinity on
rho (electron density), E and per-particle state over <= 10 steps; exact
integer charge.  Denominators: rho by max |rho_e| of the oracle, E by
max |E| of the oracle, positions in cell units (wrapped distance), velocities
by max |v| of the oracle.
"""

import math

import numpy as np
import pytest

import oracle
import workloads
from workloads import plasma

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def pk():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2608_15249_b300 as pk
    pk.lib()
    return pk


def small_cases():
    return {
        "1d": plasma.maxwellian_box(1, (97,), ppc=50, nv=1, dt=0.1, seed=31),
        "1d3v_E0": plasma.maxwellian_box(1, (64,), ppc=64, nv=3, dt=0.1, seed=32),
        "2d": plasma.maxwellian_box(2, (40, 36), ppc=16, nv=2, dt=0.1, seed=33),
        "2d_two_stream": plasma.two_stream_2d(n=(64, 48), ppc=8, mode=(2, 1), seed=34),
        "3d_mag": plasma.magnetized_3d(n=(16, 12, 10), ppc=8, seed=35),
        # dilute: a tile of 512 sorted particles spans more nodes than the deposit's
        # shared-memory window, so the warp-scan + global-atomic path runs
        "2d_sparse": plasma.sparse_box(2, (160, 128), 1500, seed=39),
        "3d_sparse": plasma.sparse_box(3, (40, 32, 24), 1300, seed=40),
        # both axes shorter than the fixed charge window (every cell inside it, the
        # upper node of the last cell in a slot of its own)
        "2d_small": plasma.maxwellian_box(2, (24, 12), ppc=20, nv=2, dt=0.1, seed=41),
    }


def _oracle_sim(w, **kw):
    return oracle.Simulation(w.ndim, w.n, w.dx, w.dt, q=w.q, m=w.m, weight=w.weight, B0=w.B0,
                             E0=w.E0, rtol=1e-12, **kw)


def _gpu(pk, w, **over):
    over.setdefault("cg_rtol", 1e-7)
    return pk.from_workload(w, **over)


def rel_inf(a, b, denom):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / denom


def _check_load(pk, w, brick=None):
    over = {}
    if brick:
        over["brick"] = brick
    g = _gpu(pk, w, **over)
    g.load(w.x, w.v, half_push=False)
    sim = _oracle_sim(w).load(w.x, w.v, half_push=False)
    # sort permutation: bit-exact against the oracle's stable counting sort
    brick_used = [g.cfg.brick[a] for a in range(3)]
    cell_o, off_o = sim.cells_offsets()
    perm = g.get_perm()
    key = oracle.sort_key(w.ndim, w.n, brick_used, cell_o)
    want = oracle.counting_sort(key, oracle.num_keys(w.ndim, w.n, brick_used))
    # the GPU sorts with the default brick unless told otherwise: fetch its value
    np.testing.assert_array_equal(perm, want)
    cell, off, v, x = g.get_particles()
    np.testing.assert_array_equal(cell, cell_o[perm])
    assert np.max(np.abs(off - off_o[perm])) <= 2.0 ** -24
    np.testing.assert_array_equal(v, w.v[perm].astype(np.float32))
    # charge: exact integer total, rho within tolerance
    d = g.get_diag()
    assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"])
    rho = g.get_rho()
    assert rel_inf(rho, sim.rho, np.abs(sim.rho_e).max()) <= TOL
    E = g.get_E()
    assert rel_inf(E, sim.E, np.abs(sim.E).max()) <= TOL
    g.close()


@pytest.mark.parametrize("name", list(small_cases()))
def test_load_deposit_sort_field(pk, name):
    _check_load(pk, small_cases()[name])


def test_sort_with_partial_bricks(pk):
    """A grid that is not a multiple of the brick (partial bricks on both axes)."""
    w = plasma.maxwellian_box(2, (37, 29), ppc=9, nv=2, seed=36)
    _check_load(pk, w, brick=(8, 6, 1))


def test_half_push(pk):
    w = small_cases()["3d_mag"]
    g = _gpu(pk, w).load(w.x, w.v, half_push=True)
    sim = _oracle_sim(w).load(w.x, w.v, half_push=True)
    perm = g.get_perm()
    _, _, v, _ = g.get_particles(positions=False)
    assert rel_inf(v, sim.v[perm], np.abs(sim.v).max()) <= TOL
    g.close()


def _near_face(x, dx, ndim, tau):
    u = x[:, :ndim] / np.asarray(dx[:ndim])
    fr = u - np.floor(u)
    return np.any((fr < tau) | (fr > 1.0 - tau), axis=1)


@pytest.mark.parametrize("name", ["2d", "3d_mag", "2d_two_stream"])
def test_one_step_from_identical_state(pk, name):
    """From the same FP32-representable state, one step gives bit-identical cell
    indices except for particles whose oracle position lies within 1e-6 cell of a
    face (counted, at most 1e-4 of them)."""
    w = workloads.fp32_exact(small_cases()[name])
    g = _gpu(pk, w, sort_every=0).load(w.x, w.v)
    sim = _oracle_sim(w).load(w.x, w.v)
    perm = g.get_perm()
    g.step(1)
    sim.step(1)
    cell, off, v, x = g.get_particles()
    cell_o, off_o = sim.cells_offsets()
    xo = sim.x[perm]
    near = _near_face(xo, w.dx, w.ndim, 1e-6)
    assert near.sum() <= max(1, int(1e-4 * w.np_)), near.sum()
    np.testing.assert_array_equal(cell[~near], cell_o[perm][~near])
    vo = sim.v[perm]
    assert rel_inf(v, vo, np.abs(vo).max()) <= TOL
    L = np.asarray(w.L[: w.ndim])
    dxv = np.asarray(w.dx[: w.ndim])
    dist = np.abs(x - xo)
    dist = np.minimum(dist, L - dist) / dxv
    assert dist.max() <= TOL
    assert rel_inf(g.get_rho(), sim.rho, np.abs(sim.rho_e).max()) <= TOL
    assert rel_inf(g.get_E(), sim.E, np.abs(sim.E).max()) <= TOL
    g.close()


# The fused pass's fixed charge window, restated on the host: tiles of 768 (2D) or 512
# (3D) consecutive particles, in groups of 3 (2D) or 1 (3D) consecutive tiles (the
# last group shorter when the tiles run out).  The reference cell is that of the
# last particle of a group's first tile when the group has several tiles, else of
# the tile's middle particle; origin = reference minus (W / 2 - 1), wrapped, or 0 on
# an axis shorter than the window; a particle's corners go to the window when its
# cell lies within W - 2 cells above the origin (wrapped) on every axis, else to the
# global accumulator.
FW = {2: (np.array([40, 20]), 768, 3), 3: (np.array([16, 16, 8]), 512, 1)}


def fixed_window_split(cell, ndim, n):
    W, tile, group = FW[ndim]
    n = np.asarray(n[:ndim])
    c = np.stack([(cell // int(np.prod(n[:a]))) % n[a] for a in range(ndim)], 1)
    inside = np.zeros(len(c), bool)
    span = tile * group
    for first in range(0, len(c), span):
        blk = c[first:first + span]
        ref = blk[tile - 1] if len(blk) > tile else blk[(len(blk) - 1) // 2]
        org = np.where(n >= W, (ref - (W // 2 - 1)) % n, 0)
        d = (blk - org) % n
        inside[first:first + span] = (d < W - 1).all(1)
    return inside


@pytest.mark.parametrize("name,paths", [("2d_sparse", "both"), ("3d_sparse", "both"),
                                        ("2d_small", "window"), ("3d_mag", "both")])
def test_fixed_window_paths(pk, name, paths):
    """The deposit at load runs on the sorted particles: the host restatement of the
    window rule on the GPU's sorted cells shows which corners took the shared-memory
    window and which the global atomics; rho is then within 1e-5 of the oracle's."""
    w = small_cases()[name]
    g = _gpu(pk, w).load(w.x, w.v, half_push=False)
    cell, _, _, _ = g.get_particles(positions=False)
    inside = fixed_window_split(np.asarray(cell, np.int64), w.ndim, w.n)
    if paths == "both":
        assert 0 < inside.sum() < len(inside), inside.sum()
    else:
        assert inside.all()
    sim = _oracle_sim(w).load(w.x, w.v, half_push=False)
    assert rel_inf(g.get_rho(), sim.rho, np.abs(sim.rho_e).max()) <= TOL
    d = g.get_diag()
    assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"])
    g.close()


@pytest.mark.parametrize("name", ["1d", "2d_two_stream", "3d_mag", "2d_sparse", "3d_sparse",
                                  "2d_small"])
def test_ten_steps_with_sorts(pk, name):
    """Ten cycles with a sort every 3 steps: per-particle state, rho and E stay within
    1e-5 of the oracle; particle identity is tracked through the sort permutations."""
    w = small_cases()[name]
    g = _gpu(pk, w, sort_every=3).load(w.x, w.v)
    sim = _oracle_sim(w).load(w.x, w.v)
    ident = g.get_perm().copy()  # storage position -> input index
    for k in range(1, 11):
        g.step(1)
        sim.step(1)
        if k % 3 == 0:
            ident = ident[g.get_perm()]
    cell, off, v, x = g.get_particles()
    xo, vo = sim.x[ident], sim.v[ident]
    L = np.asarray(w.L[: w.ndim])
    dist = np.abs(x - xo)
    dist = np.minimum(dist, L - dist) / np.asarray(w.dx[: w.ndim])
    assert dist.max() <= TOL, dist.max()
    assert rel_inf(v, vo, np.abs(vo).max()) <= TOL
    assert rel_inf(g.get_rho(), sim.rho, np.abs(sim.rho_e).max()) <= TOL
    assert rel_inf(g.get_E(), sim.E, np.abs(sim.E).max()) <= TOL
    d = g.get_diag()
    assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"])
    assert d["step"] == 10
    # kinetic energy time-centred at the last push (t = 9 dt) against the oracle's
    assert abs(d["kinetic"] - sim.ke) <= 1e-5 * abs(sim.ke)
    assert abs(d["field_energy"] - sim.field_energy()) <= 1e-4 * sim.field_energy() + 1e-12
    g.close()


def test_fused_equals_unfused_and_is_deterministic(pk):
    w = small_cases()["2d_two_stream"]
    a = _gpu(pk, w).load(w.x, w.v)
    b = _gpu(pk, w).load(w.x, w.v)
    c = _gpu(pk, w).load(w.x, w.v)
    a.push_deposit()
    b.gather_push()
    b.deposit()
    c.push_deposit()
    fa, fb, fc = a.get_rho_fx(), b.get_rho_fx(), c.get_rho_fx()
    np.testing.assert_array_equal(fa, fb)
    np.testing.assert_array_equal(fa, fc)
    for ta, tb in zip(a.get_particles(), b.get_particles()):
        np.testing.assert_array_equal(ta, tb)
    for t in (a, b, c):
        t.close()


def test_edge_cases(pk):
    """A single particle; particles on x = 0, on a node, within an ulp of L and at L."""
    w = plasma.maxwellian_box(2, (8, 6), ppc=1, nv=2, seed=37)
    x = np.array([[0.0, 0.0], [3.0, 2.0], [np.nextafter(8.0, 0.0), np.nextafter(6.0, 0.0)],
                  [8.0, 6.0], [7.5, 0.25]])
    v = np.zeros((5, 2))
    g = pk.from_workload(w, weight=48 / 5).load(x, v, half_push=False)
    sim = oracle.Simulation(2, w.n, w.dx, w.dt, weight=48 / 5, rtol=1e-12).load(x, v,
                                                                               half_push=False)
    cell_o, _ = sim.cells_offsets()
    perm = g.get_perm()
    cell, off, _, _ = g.get_particles(positions=False)
    np.testing.assert_array_equal(cell, cell_o[perm])
    assert np.all(off >= 0) and np.all(off < 1)
    assert rel_inf(g.get_rho(), sim.rho, np.abs(sim.rho_e).max()) <= TOL
    g.close()
    one = pk.from_workload(w, weight=48.0).load(np.array([[2.3, 4.1]]), np.array([[0.1, -0.2]]))
    one.step(3)
    d = one.get_diag()
    assert d["np"] == 1 and d["charge_fx_sum"] == 1 << d["fx_bits"]
    one.close()


def test_rejects_positions_outside_the_box(pk):
    w = plasma.maxwellian_box(1, (16,), ppc=2, nv=1, seed=38)
    x = w.x.copy()
    x[3, 0] = 17.5
    g = pk.from_workload(w)
    with pytest.raises(pk.PicError) as ei:
        g.load(x, w.v)
    assert ei.value.status == -6
    g.close()


def test_boris_ExB_drift_of_test_particle(pk):
    """A particle of negligible weight in uniform E0 perpendicular to B0: the Boris
    push turns u = v - E x B / B^2 by 2 atan(w_c dt / 2) per step at constant |u|."""
    E0, B0 = (0.02, -0.01, 0.0), (0.0, 0.0, 1.5)
    dt, steps = 0.05, 40
    cfg = pk.make_config(3, (8, 8, 8), dt=dt, weight=1e-12, E0=E0, B0=B0, nv=3, sort_every=0)
    g = pk.Pic(cfg)
    v0 = np.array([[0.7, 0.1, 0.2]])
    g.load(np.array([[4.2, 3.3, 1.1]]), v0, half_push=False)
    g.step(steps)
    _, _, v, _ = g.get_particles(positions=False)
    E, B = np.array(E0), np.array(B0)
    vd = np.cross(E, B) / B.dot(B)
    theta = 2 * math.atan(0.5 * 1.5 * dt)
    u0 = v0[0] - vd
    u = v[0].astype(np.float64) - vd
    ang = math.atan2(u[1], u[0]) - math.atan2(u0[1], u0[0])
    assert abs(math.remainder(ang - steps * theta, 2 * math.pi)) < 1e-5
    assert abs(np.hypot(u[0], u[1]) - np.hypot(u0[0], u0[1])) < 1e-5
    g.close()
