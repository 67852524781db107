"""The spectral field solve (AP_PIC_SOLVER_FFT) against the FP64 oracle, whose
Poisson solve is the Jacobi-PCG to 1e-12: the same discrete potential.

Power-of-two axes take the radix-2 path; every other length the Bluestein path,
so the cases mix both, in 1D, 2D and 3D.  Bars as for the CG path: 1e-5 relative
L-infinity on rho, phi, E and per-particle state over <= 10 steps."""

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


def cases():
    return {
        "1d_bluestein": plasma.maxwellian_box(1, (97,), ppc=50, nv=1, dt=0.1, seed=51),
        "1d_pow2": plasma.maxwellian_box(1, (64,), ppc=64, nv=3, dt=0.1, seed=52),
        "2d_bluestein": plasma.maxwellian_box(2, (40, 36), ppc=16, nv=2, dt=0.1, seed=53),
        "2d_mixed": plasma.two_stream_2d(n=(64, 48), ppc=8, mode=(2, 1), seed=54),
        "3d_bluestein": plasma.magnetized_3d(n=(16, 12, 10), ppc=8, seed=55),
        "3d_pow2": plasma.maxwellian_box(3, (16, 8, 32), ppc=4, nv=3, dt=0.1, seed=56),
        "2d_sparse": plasma.sparse_box(2, (160, 128), 1500, seed=57),
    }


def _sim(w):
    return oracle.Simulation(w.ndim, w.n, w.dx, w.dt, q=w.q, m=w.m, weight=w.weight, B0=w.B0,
                             E0=w.E0, rtol=1e-12)


def rel(a, b, d):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / d


@pytest.mark.parametrize("name", list(cases()))
def test_fft_field_at_load(pk, name):
    w = cases()[name]
    g = pk.from_workload(w, solver=pk.AP_PIC_SOLVER_FFT).load(w.x, w.v, half_push=False)
    sim = _sim(w).load(w.x, w.v, half_push=False)
    phi_o = sim.phi - sim.phi.mean()  # the spectral solve returns the zero-mean potential
    assert rel(g.get_phi(), phi_o, np.abs(phi_o).max()) <= TOL
    assert rel(g.get_E(), sim.E, np.abs(sim.E).max()) <= TOL
    d = g.get_diag()
    # the first FP32 solve's FP64 residual: floored by the rounding of an FP32 potential
    assert d["cg_iters"] == 0 and d["cg_relres"] < 1e-3
    g.close()


@pytest.mark.parametrize("name", ["1d_bluestein", "2d_mixed", "3d_bluestein", "2d_sparse"])
def test_fft_ten_steps(pk, name):
    w = cases()[name]
    g = pk.from_workload(w, solver=pk.AP_PIC_SOLVER_FFT, sort_every=3).load(w.x, w.v)
    sim = _sim(w).load(w.x, w.v)
    ident = g.get_perm().copy()
    for k in range(1, 11):
        g.step(1)
        sim.step(1)
        if k % 3 == 0:
            ident = ident[g.get_perm()]
    _, _, v, x = g.get_particles()
    L = np.asarray(w.L[: w.ndim])
    dist = np.abs(x - sim.x[ident])
    dist = np.minimum(dist, L - dist) / np.asarray(w.dx[: w.ndim])
    assert dist.max() <= TOL
    assert rel(v, sim.v[ident], np.abs(sim.v).max()) <= TOL
    assert rel(g.get_rho(), sim.rho, np.abs(sim.rho_e).max()) <= TOL
    assert rel(g.get_E(), sim.E, np.abs(sim.E).max()) <= TOL
    d = g.get_diag()
    assert d["charge_fx_sum"] == w.np_ * (1 << d["fx_bits"])
    g.close()


def test_fft_agrees_with_cg(pk):
    """Both solvers give the same E (each within its tolerance of the exact one)."""
    w = cases()["2d_mixed"]
    a = pk.from_workload(w, solver=pk.AP_PIC_SOLVER_FFT).load(w.x, w.v)
    b = pk.from_workload(w, cg_rtol=1e-7).load(w.x, w.v)
    Ea, Eb = a.get_E(), b.get_E()
    assert rel(Ea, Eb, np.abs(Eb).max()) <= TOL
    a.close()
    b.close()


@pytest.mark.parametrize("n", [(256, 128), (300, 211), (1000,), (64, 601)])
def test_fft_larger_grids(pk, n):
    """Grids of many lines and CTAs (a prime length included) against the oracle;
    (64, 601) puts two power-of-two lines in a CTA with an odd line count, so the
    last CTA holds one."""
    w = plasma.sparse_box(len(n), n, 4 * int(np.prod(n)), nv=len(n), seed=58)
    g = pk.from_workload(w, solver=pk.AP_PIC_SOLVER_FFT).load(w.x, w.v, half_push=False)
    sim = _sim(w).load(w.x, w.v, half_push=False)
    assert rel(g.get_E(), sim.E, np.abs(sim.E).max()) <= TOL
    g.close()


def test_step_graph_replay_equals_direct_launches(pk):
    """With the spectral solve ap_pic_step replays captured graphs (stage timing
    turns them off): both give the same state bit for bit, through several sorts
    (both buffer parities) and steps with and without diagnostics."""
    w = cases()["2d_mixed"]
    runs = []
    for timing in (False, True):
        g = pk.from_workload(w, solver=pk.AP_PIC_SOLVER_FFT, sort_every=2, diag_every=3)
        g.load(w.x, w.v)
        g.set_timing(timing)
        g.step(9)
        d = g.get_diag()
        runs.append((g.get_rho_fx(), g.get_E(), g.get_particles(), g.get_perm(), d))
        g.close()
    a, b = runs
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    for x, y in zip(a[2], b[2]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a[3], b[3])
    assert a[4]["step"] == b[4]["step"] == 9 and a[4]["kinetic"] == b[4]["kinetic"]


def test_step_graphs_dropped_on_reload(pk):
    """A second load on a handle drops the step graphs captured under the first (they
    hold its particle buffers and count): stepping after the reload gives, bit for
    bit, what a fresh handle with the second load gives without graphs."""
    w = cases()["2d_mixed"]
    w2 = plasma.two_stream_2d(n=(64, 48), ppc=11, mode=(1, 1), seed=60)
    # one configuration for both handles (the particle weight goes with w2's ppc)
    g = pk.from_workload(w2, solver=pk.AP_PIC_SOLVER_FFT, sort_every=2, diag_every=3)
    g.load(w.x, w.v)
    g.step(5)
    g.load(w2.x, w2.v)
    g.step(5)
    f = pk.from_workload(w2, solver=pk.AP_PIC_SOLVER_FFT, sort_every=2, diag_every=3)
    f.load(w2.x, w2.v)
    f.set_timing(True)
    f.step(5)
    np.testing.assert_array_equal(g.get_rho_fx(), f.get_rho_fx())
    np.testing.assert_array_equal(g.get_E(), f.get_E())
    for x, y in zip(g.get_particles(), f.get_particles()):
        np.testing.assert_array_equal(x, y)
    assert g.get_diag()["kinetic"] == f.get_diag()["kinetic"]
    g.close()
    f.close()


@pytest.mark.parametrize("n", [4096, 4095])
def test_fft_longest_axes(pk, n):
    """The longest axes: 4096 (the largest power-of-two line: four radix-8 passes and a
    radix-2 pass in the largest shared-memory layout) and 4095 (Bluestein on 8192
    points), on a displaced lattice, 4 per cell.  (Uniform random positions on a line
    this long give a potential thousands of times larger than E, whose FP32 storage
    alone then costs E about 1e-5; a displaced lattice keeps the potential within about
    sqrt(n) of E and the comparison at the transform's own accuracy.)"""
    rng = np.random.default_rng(59)
    ppc = 4
    npart = ppc * n
    x = (np.arange(npart) + 0.5) / ppc + rng.uniform(-0.3, 0.3, npart) / ppc
    x = np.mod(x, float(n))[:, None]
    v = rng.normal(0.0, 1.0, (npart, 1))
    cfg = pk.make_config(1, (n,), dt=0.1, nv=1, weight=1.0 / ppc, solver=pk.AP_PIC_SOLVER_FFT)
    g = pk.Pic(cfg).load(x, v, half_push=False)
    sim = oracle.Simulation(1, (n,), (1.0,), 0.1, weight=1.0 / ppc, rtol=1e-12).load(
        x, v, half_push=False)
    phi_o = sim.phi - sim.phi.mean()
    assert rel(g.get_phi(), phi_o, np.abs(phi_o).max()) <= TOL
    assert rel(g.get_E(), sim.E, np.abs(sim.E).max()) <= TOL
    g.close()
