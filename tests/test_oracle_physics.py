"""Physics pins of the oracle's assembled cycle (Listing 1, Sec. 3.1) against the
paper's printed results (Sec. 3.2) and textbook closed forms (no GPU)."""

import math
import os

import numpy as np
import pytest

import workloads
from oracle import physics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_values():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_two_stream.txt")) as f:
        for line in f:
            tok = line.split()
            if tok and not tok[0].startswith("#"):
                vals[tok[0]] = float(tok[1])
    return vals


def test_dispersion_root_matches_paper():
    """The warm symmetric two-stream relation (Eqs. 5-6) for the paper's k and
    u_d = 3 gives the printed gamma_th = 0.2616."""
    pv = _paper_values()
    k = physics.mode_k((2, 1), (64, 64), (1.0, 1.0))
    g = physics.two_stream_gamma(k)
    assert round(g, 4) == pv["gamma_th"]
    # the root is a root: |eps| vanishes there and not nearby
    assert abs(physics.two_stream_eps(1j * g, k)) < 1e-12
    assert abs(physics.two_stream_eps(1j * (g + 0.05), k)) > 1e-3


def test_dispersion_cold_limit():
    """For a large drift compared with v_te the warm relation approaches the cold
    symmetric two-stream result: with a = k_x u_d, the cold growth rate solves
    1 = 1/2 [1/(i g - a)^2 + 1/(i g + a)^2], whose positive root is
    g^2 = -(a^2 + 1/2) + sqrt(2 a^2 + 1/4)."""
    k = (0.08, 0.0)
    u_d = 8.0
    a = k[0] * u_d
    g_cold = math.sqrt(-(a * a + 0.5) + math.sqrt(2 * a * a + 0.25))
    g_warm = physics.two_stream_gamma(k, u_d=u_d, v_te=0.01)
    assert abs(g_warm - g_cold) < 2e-3 * g_cold


def test_loader_beam_centres_match_paper():
    """Wave-aligned beam velocities (Eq. 2) of the paper's load sit at +-2.683."""
    pv = _paper_values()
    w = workloads.paper_two_stream(steps=0)
    k = np.array(physics.mode_k((2, 1), (64, 64), (1.0, 1.0)))
    vpar = w.v[:, :2] @ k / np.linalg.norm(k)
    half = w.np_ // 2
    assert abs(vpar[:half].mean() - pv["v_par_beam"]) < 5e-3
    assert abs(vpar[half:].mean() + pv["v_par_beam"]) < 5e-3


def _run_energy_and_mode(orc, w, rtol=1e-10):
    sim = orc.Simulation(w.ndim, w.n, w.dx, w.dt, q=w.q, m=w.m, weight=w.weight, B0=w.B0,
                         rtol=rtol).load(w.x, w.v)
    t, amp, WE, KE = [0.0], [], [], []
    amp.append(physics.mode_amplitude(sim.E, w.ndim, w.n, w.dx, w.mode))
    WE.append(sim.field_energy())
    for s in range(1, w.steps + 1):
        sim.push()          # uses E((s-1) dt): kinetic energy centred at t = (s-1) dt
        KE.append(sim.ke)
        sim.move()
        sim.update_field()
        sim.t += sim.dt
        t.append(sim.t)
        amp.append(physics.mode_amplitude(sim.E, w.ndim, w.n, w.dx, w.mode))
        WE.append(sim.field_energy())
    return sim, np.array(t), np.array(amp), np.array(WE), np.array(KE)


def test_cold_langmuir_frequency(orc):
    """A cold 1D plasma oscillates at w_p = 1 (Debye units): the fitted frequency of
    the seeded mode lies within 1 % of w_p, and within 0.3 % of the leapfrog-plus-grid
    estimate w = (2/dt) asin(dt w_g / 2) with w_g^2 = S(k)^2 (k dx/2) cot(k dx/2),
    S(k) = sin(k dx/2)/(k dx/2) (CIC smoothing, centred differences)."""
    w = workloads.langmuir_1d()
    # the longitudinal field's real part oscillates as cos(w t): use a signed projection
    sim2 = orc.Simulation(1, w.n, w.dx, w.dt, weight=w.weight, rtol=1e-12).load(w.x, w.v)
    k = 0.5
    xj = np.arange(w.n[0]) * w.dx[0]
    sig = [np.dot(sim2.E, np.sin(k * xj))]
    ts = [0.0]
    for s in range(w.steps):
        sim2.step(1)
        sig.append(np.dot(sim2.E, np.sin(k * xj)))
        ts.append(sim2.t)
    om = physics.fit_frequency(ts, sig, 1.0)
    assert abs(om - 1.0) < 0.01
    h = k * w.dx[0] / 2
    wg = math.sqrt((math.sin(h) / h) ** 2 * h / math.tan(h))
    om_est = (2 / w.dt) * math.asin(w.dt * wg / 2)
    assert abs(om - om_est) < 3e-3


def test_cold_two_stream_growth_1d(orc):
    """Cold symmetric beams with k u = sqrt(3/8) grow at gamma = 1/(2 sqrt 2) (the
    cold limit of Eqs. 5-6); from a quiet start the fitted growth of the seeded mode
    over 10 <= t <= 22 lies within 2 % of it."""
    w = workloads.cold_two_stream_1d()
    sim, t, amp, WE, KE = _run_energy_and_mode(orc, w, rtol=1e-13)
    gamma, r2 = physics.fit_growth(t, amp, 10.0, 22.0)
    assert abs(gamma - 1.0 / (2.0 * math.sqrt(2.0))) < 0.02 / (2.0 * math.sqrt(2.0)), gamma
    assert r2 > 0.995


@pytest.mark.slow
def test_paper_two_stream_growth_and_energy(orc):
    """The paper's worked example run by the oracle from a quiet start: growth rate of
    2|E_par(2,1)| fitted on 10 <= t <= 19 within 5 % of gamma_th, the mode peaks in
    the twenties, and the total energy error stays below 0.05 % of W0 (the paper
    reports 0.0183 %).

    One realisation cannot reach the paper's 0.5 %: the displacement seed of Eq. 1
    also excites the stable roots of Eqs. 5-6, which have not died out by t = 10,
    and the random thermal velocities seed other modes.  Over velocity seeds 1-9
    the fitted rate ranged over 0.2599-0.2797 (mean 0.2695, +3.0 %); seed 7 gives
    0.2694.  The eigenmode-loaded run of the same wave vector (test of the
    diagnostics module) excites the growing root alone and pins gamma to 0.5 %."""
    pv = _paper_values()
    w = workloads.paper_two_stream()
    sim, t, amp, WE, KE = _run_energy_and_mode(orc, w)
    gamma, r2 = physics.fit_growth(t, amp, pv["fit_t_lo"], pv["fit_t_hi"])
    assert abs(gamma - pv["gamma_th"]) < 0.05 * pv["gamma_th"], gamma
    assert r2 > 0.9
    t_peak = t[np.argmax(amp)]
    assert 20.0 <= t_peak <= 30.0, t_peak
    # energy at integer times t = 0 .. (steps-1) dt
    W = KE + WE[: len(KE)]
    W0 = W[0]
    err = np.abs(W - W0).max() / W0
    assert err < 5e-4, err
