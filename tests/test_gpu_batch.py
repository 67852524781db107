"""The batch form (many independent uneven instances advanced together) against the
FP64 oracle run instance by instance, with the single-instance bars (1e-5 relative
on rho, E and particle state; exact integer charge per instance)."""

import numpy as np
import pytest

import oracle
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


def instances():
    """Uneven 1D and 2D instances, nv = 2, some dilute (their tiles overflow the
    deposit window)."""
    return [
        plasma.maxwellian_box(1, (64,), ppc=40, nv=2, seed=71),
        plasma.maxwellian_box(2, (40, 36), ppc=16, nv=2, seed=72),
        plasma.sparse_box(1, (200,), 90, nv=2, seed=73),
        plasma.two_stream_2d(n=(48, 32), ppc=8, mode=(2, 1), seed=74),
        plasma.sparse_box(2, (96, 80), 700, nv=2, seed=75),
        plasma.maxwellian_box(1, (97,), ppc=33, nv=2, seed=76),
        plasma.maxwellian_box(2, (24, 20), ppc=5, nv=2, seed=77),
    ]


def _oracle(w):
    return oracle.Simulation(w.ndim, w.n, w.dx, w.dt, weight=w.weight, rtol=1e-12)


def rel(a, b, d):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / d


def test_batch_load_matches_oracle(pk):
    ws = instances()
    bt = pk.batch_from_workloads(ws, cg_rtol=1e-7, sort_every=2)
    bt.load([w.x for w in ws], [w.v for w in ws], half_push=False)
    for i, w in enumerate(ws):
        sim = _oracle(w).load(w.x, w.v, half_push=False)
        d = bt.get_diag(i)
        assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"]), i
        assert rel(bt.get_rho(i), sim.rho, np.abs(sim.rho_e).max()) <= TOL, i
        assert rel(bt.get_E(i), sim.E, np.abs(sim.E).max()) <= TOL, i
        # the load sorted each instance; its permutation is the oracle's stable sort
        cell_o, _ = sim.cells_offsets()
        brick = (64,) if w.ndim == 1 else (8, 8)
        brick = tuple(min(b, w.n[a]) for a, b in enumerate(brick))
        key = oracle.sort_key(w.ndim, w.n, brick, cell_o)
        want = oracle.counting_sort(key, oracle.num_keys(w.ndim, w.n, brick))
        np.testing.assert_array_equal(bt.get_perm(i), want)
    bt.close()


@pytest.mark.parametrize("use_graph,solver", [(1, 0), (0, 0), (1, 1), (0, 1)])
def test_batch_steps_match_oracle(pk, use_graph, solver):
    ws = instances()
    bt = pk.batch_from_workloads(ws, cg_rtol=1e-7, solver=solver)
    bt.set_tuning(use_graph=use_graph, sort_every=2)
    bt.load([w.x for w in ws], [w.v for w in ws])
    sims = [_oracle(w).load(w.x, w.v) for w in ws]
    ident = [bt.get_perm(i).copy() for i in range(len(ws))]
    for k in range(1, 7):
        bt.step(1)
        for s in sims:
            s.step(1)
        if k % 2 == 0:
            ident = [ident[i][bt.get_perm(i)] for i in range(len(ws))]
    for i, (w, sim) in enumerate(zip(ws, sims)):
        cell, off, v, x = bt.get_particles(i)
        xo, vo = sim.x[ident[i]], sim.v[ident[i]]
        L = np.asarray(w.L[: w.ndim])
        dist = np.abs(x - xo)
        dist = np.minimum(dist, L - dist)
        assert dist.max() <= TOL, (i, dist.max())
        assert rel(v, vo, np.abs(vo).max()) <= TOL, i
        assert rel(bt.get_rho(i), sim.rho, np.abs(sim.rho_e).max()) <= TOL, i
        assert rel(bt.get_E(i), sim.E, np.abs(sim.E).max()) <= TOL, i
        d = bt.get_diag(i)
        assert d["step"] == 6 and d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"])
        assert abs(d["kinetic"] - sim.ke) <= 1e-5 * sim.ke, i
    bt.close()


@pytest.mark.parametrize("solver", [0, 1])
def test_batch_graph_replay_equals_direct_launches(pk, solver):
    ws = instances()[:4]
    out = []
    for use_graph in (1, 0):
        bt = pk.batch_from_workloads(ws, solver=solver)
        bt.set_tuning(use_graph=use_graph)
        bt.load([w.x for w in ws], [w.v for w in ws])
        bt.step(5)
        out.append([(bt.get_rho(i), bt.get_particles(i)) for i in range(len(ws))])
        bt.close()
    for (ra, pa), (rb, pb) in zip(*out):
        np.testing.assert_array_equal(ra, rb)
        for a, b in zip(pa, pb):
            np.testing.assert_array_equal(a, b)


def test_batch_autotune_and_cache(pk, tmp_path):
    ws = instances()
    bt = pk.batch_from_workloads(ws)
    bt.load([w.x for w in ws], [w.v for w in ws])
    cache = str(tmp_path / "tune.txt")
    t = bt.autotune(steps_per_trial=2, cache_path=cache)
    assert t["pass_ctas_per_sm"] in (2, 3, 4, 6, 8)
    assert t["cg_iters_per_graph"] in (8, 16, 32)
    assert t["sort_every"] in (10, 20, 40)
    assert (t["pass_threads"], t["pass_per_thread"]) in PASS_SHAPES
    assert open(cache).read().strip()
    # a second tune of the same shape on this GPU comes from the cache
    t2 = bt.autotune(steps_per_trial=2, cache_path=cache)
    assert t2 == t
    bt.step(2)
    for i, w in enumerate(ws):
        d = bt.get_diag(i)
        assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"])
    bt.close()


# (threads per CTA, particles per thread) of the batch pass's kernel variants
PASS_SHAPES = [(256, 2), (128, 2), (128, 4), (256, 1), (256, 3), (512, 1)]


@pytest.mark.parametrize("shape", PASS_SHAPES)
def test_batch_pass_shapes_match_oracle(pk, shape):
    """Every shape the autotuner can pick (CTA size x particles per thread, tiles of
    their product) gives the oracle's state; the shape is switched after loading, so
    the pass tiles are rebuilt on a loaded batch."""
    ws = instances()
    bt = pk.batch_from_workloads(ws, cg_rtol=1e-7, solver=1)
    bt.set_tuning(sort_every=2)
    bt.load([w.x for w in ws], [w.v for w in ws])
    bt.set_tuning(pass_threads=shape[0], pass_per_thread=shape[1])
    sims = [_oracle(w).load(w.x, w.v) for w in ws]
    ident = [bt.get_perm(i).copy() for i in range(len(ws))]
    for k in range(1, 5):
        bt.step(1)
        for sim in sims:
            sim.step(1)
        if k % 2 == 0:
            ident = [ident[i][bt.get_perm(i)] for i in range(len(ws))]
    for i, (w, sim) in enumerate(zip(ws, sims)):
        _, _, v, x = bt.get_particles(i)
        L = np.asarray(w.L[: w.ndim])
        dist = np.abs(x - sim.x[ident[i]])
        dist = np.minimum(dist, L - dist)
        assert dist.max() <= TOL, (shape, i, dist.max())
        assert rel(v, sim.v[ident[i]], np.abs(sim.v).max()) <= TOL, (shape, i)
        assert rel(bt.get_rho(i), sim.rho, np.abs(sim.rho_e).max()) <= TOL, (shape, i)
        d = bt.get_diag(i)
        assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"]), (shape, i)
        assert abs(d["kinetic"] - sim.ke) <= 1e-5 * sim.ke, (shape, i)
    bt.close()


def test_batch_rejects_unknown_pass_shape(pk):
    ws = instances()[:2]
    bt = pk.batch_from_workloads(ws)
    with pytest.raises(pk.PicError):
        bt.set_tuning(pass_threads=384, pass_per_thread=2)
    bt.close()


@pytest.mark.parametrize("solver", [0, 1])
def test_batch_many_instances_many_items(pk, solver):
    """Many instances split into many small cell items, converging at different CG
    iterations while their blocks share launches: every instance stays finite with
    exact charge, and a sample matches the oracle after a few steps."""
    rng = np.random.default_rng(79)
    ws = []
    for i in range(40):
        if i % 3 == 0:
            ws.append(plasma.maxwellian_box(1, (int(rng.integers(32, 300)),), ppc=12, nv=2,
                                            seed=100 + i))
        else:
            n = (int(rng.integers(40, 140)), int(rng.integers(40, 140)))
            ppc = [0.05, 1, 3][i % 3]
            ws.append(plasma.sparse_box(2, n, max(64, int(ppc * n[0] * n[1])), nv=2,
                                        seed=100 + i))
    bt = pk.batch_from_workloads(ws, cg_rtol=1e-7, solver=solver)
    bt.set_tuning(item_cells=256, sort_every=2, cg_iters_per_graph=8)
    bt.load([w.x for w in ws], [w.v for w in ws])
    check = list(range(0, len(ws), 7))
    sims = {i: _oracle(ws[i]).load(ws[i].x, ws[i].v) for i in check}
    ident = {i: bt.get_perm(i).copy() for i in check}
    for k in range(1, 5):
        bt.step(1)
        for s in sims.values():
            s.step(1)
        if k % 2 == 0:
            ident = {i: ident[i][bt.get_perm(i)] for i in check}
    for i, w in enumerate(ws):
        d = bt.get_diag(i)
        assert d["error_flags"] == 0 and d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"]), i
        assert np.all(np.isfinite(bt.get_E(i))), i
    for i in check:
        w, sim = ws[i], sims[i]
        _, _, v, x = bt.get_particles(i)
        L = np.asarray(w.L[: w.ndim])
        dist = np.abs(x - sim.x[ident[i]])
        dist = np.minimum(dist, L - dist)
        assert dist.max() <= TOL, (i, dist.max())
        assert rel(v, sim.v[ident[i]], np.abs(sim.v).max()) <= TOL, i
        assert rel(bt.get_E(i), sim.E, np.abs(sim.E).max()) <= TOL, i
    bt.close()


@pytest.mark.parametrize("solver", [0, 1])
def test_batch_step_parts_equal_step(pk, solver):
    """push_deposit, a sort when due and solve_field, called apart, give bit for bit
    what the step gives."""
    ws = instances()
    a = pk.batch_from_workloads(ws, solver=solver)
    b = pk.batch_from_workloads(ws, solver=solver)
    for t in (a, b):
        t.set_tuning(sort_every=2)
        t.load([w.x for w in ws], [w.v for w in ws])
    a.step(4)
    for k in range(1, 5):
        b.push_deposit()
        if k % 2 == 0:
            b.sort()
        b.solve_field()
    for i in range(len(ws)):
        np.testing.assert_array_equal(a.get_rho(i), b.get_rho(i))
        np.testing.assert_array_equal(a.get_E(i), b.get_E(i))
        for x, y in zip(a.get_particles(i), b.get_particles(i)):
            np.testing.assert_array_equal(x, y)
    a.close()
    b.close()
