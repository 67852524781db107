"""The absorbing layer of the electromagnetic step on the GPU (Sec. 2.2 E_Maxwell:
FDTD with CPML) against the FP64 oracle's CpmlField: a prescribed current pulse at
the centre of a non-periodic grid with a 12-cell layer; E and B within 1e-5 of the
oracle's over the whole run while the pulse crosses the layer."""

import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2608_15249_b300 as pk
    pk.lib()
    return pk


@pytest.mark.parametrize("n,dx", [((72, 72), (1.0, 1.0)), ((64, 50), (0.8, 1.0))])
def test_cpml_pulse_matches_oracle(pk, n, dx):
    c, dt, npml = 1.0, 0.5, 12
    cfg = pk.make_config(2, n, dx=dx, dt=dt, nv=3, em=1, c_light=c, em_boundary=1,
                         pml_cells=npml, sort_every=0)
    g = pk.Pic(cfg).load(np.zeros((0, 2)), np.zeros((0, 3)))
    f = oracle.CpmlField(n, dx, dt, c, npml)
    cells = n[0] * n[1]
    src = n[0] // 2 + n[0] * (n[1] // 2)
    t0, tw = 40 * dt, 10 * dt
    J = np.zeros((3, cells))
    # errors are measured against the largest field of the run: the layer absorbs the
    # pulse, so the field (and with it any relative measure) decays towards zero
    scale_e = scale_b = 0.0
    for s in range(260):
        t = (s + 0.5) * dt
        J[2, src] = -((t - t0) / tw) * math.exp(-((t - t0) / tw) ** 2)
        g.set_current(J)
        g.step(1)
        f.step(J)
        scale_e = max(scale_e, np.abs(f.E).max())
        scale_b = max(scale_b, np.abs(f.B).max())
        if s % 20 == 19:
            E, B = g.get_E().reshape(3, -1), g.get_B().reshape(3, -1)
            assert np.abs(E - f.E).max() <= 1e-5 * scale_e, s
            assert np.abs(B - f.B).max() <= 1e-5 * scale_b, s
    # the layer and the wall: tangential E on the outer nodes is zero
    E = g.get_E().reshape(3, n[1], n[0])
    assert np.all(E[2, 0, :] == 0) and np.all(E[2, :, 0] == 0) and np.all(E[0, :, -1] == 0)
    g.close()


def test_cpml_rejects_bad_thickness(pk):
    """(Particles in this mode are covered by test_gpu_cpml_particles.py.)"""
    with pytest.raises(pk.PicError):
        pk.Pic(pk.make_config(2, (20, 20), dt=0.5, nv=3, em=1, c_light=1.0, em_boundary=1,
                              pml_cells=10))
