"""The synthetic input recipes (seeded, synthetic stand-ins for the paper's workloads):
sizes, drifts, spreads, fields and ranges as the design notes state them.  No GPU."""

import math

import numpy as np

from workloads import plasma


def test_two_stream_recipe():
    w = plasma.two_stream_2d(n=(32, 32), ppc=16, seed=2)
    N = 32 * 32 * 16
    assert w.np_ == N and w.ndim == 2 and w.nv == 2
    assert np.all((w.x >= 0) & (w.x < 32.0))
    half = N // 2
    sig = 1.0 / math.sqrt(half)
    assert abs(w.v[:half, 0].mean() - 3.0) < 5 * sig
    assert abs(w.v[half:, 0].mean() + 3.0) < 5 * sig
    assert abs(w.v[:, 1].std() - 1.0) < 0.03
    assert w.weight == 32.0 * 32.0 / N and w.sort_every == 20 and w.mode == (16, 8)


def test_maxwellian_and_magnetised_recipes():
    w = plasma.maxwellian_box(3, (8, 6, 4), ppc=20, nv=3, seed=3)
    assert w.np_ == 8 * 6 * 4 * 20
    assert np.all(np.abs(w.v.mean(axis=0)) < 0.1)
    assert np.all(np.abs(w.v.std(axis=0) - 1.0) < 0.05)
    m = plasma.magnetized_3d(n=(8, 8, 8), ppc=2)
    # electron cyclotron frequency |q| B0 / m = 2 in units of the plasma frequency
    assert tuple(m.B0) == (0.0, 0.0, 2.0) and abs(m.q) * m.B0[2] / m.m == 2.0
    assert m.dt == 0.05 and m.ndim == 3 and m.nv == 3


def test_sparse_and_precision_recipes():
    s = plasma.sparse_box(2, (40, 30), 500, seed=8)
    assert s.np_ == 500 and s.nv == 2 and np.all(s.x < np.array([40.0, 30.0]))
    p = plasma.precision_3d(n=(8, 8, 8), ppc=16, noise=1.0, seed=4)
    assert p.np_ == 8 ** 3 * 16
    counts = np.bincount((p.x[:, 0].astype(int) + 8 * p.x[:, 1].astype(int) +
                          64 * p.x[:, 2].astype(int)), minlength=512)
    # the per-cell density carries the white noise on top of the Poisson spread
    assert counts.std() / counts.mean() > 1.5 * math.sqrt(1.0 / 16)


def test_batch_recipe_ranges():
    ws = plasma.batch_instances(count=24, seed=5)
    assert len(ws) == 24
    dims = {w.ndim for w in ws}
    assert dims <= {1, 2} and len(dims) == 2
    for w in ws:
        assert all(32 <= w.n[a] <= 1024 for a in range(w.ndim))
        assert 1_000 <= w.np_ <= 200_000
        assert all(1 <= k <= 4 for k in w.mode)
        L = np.array([w.n[a] * w.dx[a] for a in range(w.ndim)])
        assert np.all((w.x >= 0) & (w.x < L))
