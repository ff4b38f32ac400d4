"""The library's discharge current density J(t) and its steady-state test, through the C ABI.

J(t) = eps0 dE(0,t)/dt + e0 (Gamma_i - Gamma_e)(0,t) (section "Boundary conditions") is computed on
the device every step in FP64; it is compared with the oracle's J on identical steps (the same
state and the same FP32 node field on both sides every step), checked against the plate-capacitor
closed form in an empty gap, and its first-harmonic amplitude per rf period against the discrete
closed form. The steady-state flag of pic_moments is the block-mean criterion on the per-period
mean counts, recomputed here from pic_period_counts.
"""
import math

import numpy as np
import pytest

import inputs as I
from oracle import oracle as O
from paper_1608_04601_gb300 import xsections as X

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    from paper_1608_04601_gb300 import pic
    return pic


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_current_matches_oracle_step_by_step(P, prec):
    d = I.discharge(n_cells=96, gap_m=0.025, p_Pa=60.0, V_rf_V=400.0, n_e0=6000, n_i0=6000, n_init_m3=6e14,
                    gamma_see=0.3, steps_per_period=400, T_e0_eV=4.0)
    gas = X.he_like(eps_max_eV=600.0, de_eV=1e-2)
    ref = O.Oracle(gas, d, "f32" if prec == "fp32" else "f64", sort_every=4)
    sim = P.Simulation(gas, d, seed=d.seed, precision=prec, sort_every=4, load=False)
    for sp in (0, 1):
        sim.set_state(0, sp, ref.get_state(sp))
    sim.set_field(0, ref.get_field())
    steps = 120
    Jr = []
    for n in range(steps):
        sim.step(1)
        ref.step(1)
        Jr.append(ref.last_current())
        for sp in (0, 1):
            assert np.array_equal(sim.get_state(0, sp)["c"], ref.get_state(sp)["c"]), (n, sp)
        sim.set_field(0, ref.get_field())
    Jr = np.array(Jr)
    Jg = sim.current(0)
    assert Jg.shape == (steps, 2)
    scale = np.max(np.abs(Jr[:, 0]))
    assert scale > 0 and sim.counters(0)["see_emitted"] > 0
    # step 0 follows the upload (no earlier solve on the library's side): no current there
    assert np.all(Jg[0] == 0.0)
    assert np.max(np.abs(Jg[1:] - Jr[1:])) <= 1e-9 * scale
    assert np.max(np.abs(Jg[1:, 0] - Jg[1:, 1])) <= 1e-9 * scale  # charge conservation
    m = sim.moments(0)
    assert m["J_last"] == Jg[-1, 0]
    sim.close()


def test_vacuum_gap_current_and_its_first_harmonic(P):
    """Empty gap: J_n = eps0 (V(t_{n+1}) - V(t_n)) / (d dt) = A cos(w t_{n+1/2}), A = 2 eps0 V0
    sin(w dt / 2) / (d dt); its projection on the period's first harmonic at the step midpoints is
    exactly A (discrete orthogonality over a whole period). The first step has no earlier solve (no
    load), so the check starts with the second step and the second period."""
    d = I.discharge(n_cells=64, gap_m=0.02, V_rf_V=250.0, steps_per_period=200)
    sim = P.Simulation(X.he_like(eps_max_eV=20.0, de_eV=1e-2), d, precision="fp32", load=False)
    assert sim.count(0, 0) == 0 and sim.count(0, 1) == 0
    sim.step(3 * 200)
    J = sim.current(0, 1, 3 * 200 - 1)
    w, dt = 2 * math.pi * d.f_rf_Hz, d.dt_s
    n = np.arange(1, 3 * 200)
    ref = I.EPS0 * d.V_rf_V * (np.sin(w * (n + 1) * dt) - np.sin(w * n * dt)) / (d.gap_m * dt)
    A = 2 * I.EPS0 * d.V_rf_V * math.sin(w * dt / 2) / (d.gap_m * dt)
    assert np.max(np.abs(J[:, 0] - ref)) <= 1e-9 * A
    assert np.max(np.abs(J[:, 1] - ref)) <= 1e-9 * A
    amp = sim.current_amplitude(0)
    assert amp.size == 3
    assert np.allclose(amp[1:], A, rtol=1e-9, atol=0)
    m = sim.moments(0)
    assert m["periods_done"] == 3 and m["J_amp"] == amp[-1]
    assert m["steady"] is False and m["steady_period"] is None and m["steady_metric"] == -1.0
    sim.close()


def test_steady_state_flag_is_the_block_mean_criterion(P):
    """A small He-like discharge over 160 rf periods: the library's steady-state period and metric
    equal the block-mean criterion evaluated on its own per-period mean counts."""
    from paper_1608_04601_gb300.steady import steady_period
    d = I.discharge(n_cells=64, gap_m=0.025, p_Pa=30.0, V_rf_V=200.0, n_e0=3000, n_i0=3000, n_init_m3=4e14,
                    steps_per_period=200)
    sim = P.Simulation(X.he_like(eps_max_eV=300.0, de_eV=1e-2), d, precision="fp32", sort_every=8, use_graph=True)
    sim.step(160 * 200)
    pc = sim.period_counts(0)
    m = sim.moments(0)
    assert m["periods_done"] == 160 == pc.shape[0]
    ks = steady_period(pc)
    assert m["steady_period"] == ks and m["steady"] == (ks is not None)
    a = pc[-50:].mean(0)
    b = pc[-100:-50].mean(0)
    assert m["steady_metric"] == pytest.approx(np.max(np.abs(a - b) / a), rel=1e-12)
    sim.close()
