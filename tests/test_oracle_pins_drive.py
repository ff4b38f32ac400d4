"""Pins of the oracle's per-period current amplitude and current-driven mode (section "Boundary
conditions", Eq. adaptivevoltage: V0_new = V0_old J0 / J_calc after every rf period).

An empty gap is a linear load with a closed form: with phi(0,t) = V0 sin(w t) the current density
of step n is J_n = eps0 V0 (sin w t_{n+1} - sin w t_n) / (d dt) = A cos(w t_{n+1/2}) with
A = 2 eps0 V0 sin(w dt / 2) / (d dt), and its first-harmonic projection over a whole period at the
step midpoints is exactly A. The first step after an upload has no earlier solve (J = 0), so period
0 is short of one term; from period 1 on the amplitude is A(V0) to rounding, and in the
current-driven mode the voltage after period 1 is exactly the one that gives J0.
"""
import math

import numpy as np
import pytest

import inputs as I
from oracle import oracle as O
from paper_1608_04601_gb300 import xsections as X

P = 200


def _vacuum(V0=250.0):
    d = I.discharge(n_cells=64, gap_m=0.02, V_rf_V=V0, steps_per_period=P, n_e0=1, n_i0=1)
    gas = X.he_like(eps_max_eV=20.0, de_eV=1e-2)
    o = O.Oracle(gas, d, "f64", load=False)
    return o, d


def _A_per_volt(d):
    w, dt = 2 * math.pi * d.f_rf_Hz, d.dt_s
    return 2 * I.EPS0 * math.sin(w * dt / 2) / (d.gap_m * dt)


def test_fixed_voltage_amplitude_is_the_closed_form():
    o, d = _vacuum()
    o.set_current_drive(P, 0.0)
    o.step(4 * P)
    amp, V0, Vn = o.period_history()
    assert amp.size == 4 and np.all(V0 == d.V_rf_V) and Vn == d.V_rf_V
    assert np.allclose(amp[1:], d.V_rf_V * _A_per_volt(d), rtol=1e-11, atol=0)
    assert amp[0] < amp[1]  # period 0 lacks the first step's current


def test_current_drive_reaches_the_target_after_one_full_period():
    J0 = 7.0
    o, d = _vacuum()
    o.set_current_drive(P, J0)
    o.step(4 * P)
    amp, V0, Vn = o.period_history()
    # the rule, period by period
    assert V0[0] == d.V_rf_V
    for k in range(3):
        assert V0[k + 1] == V0[k] * (J0 / amp[k])
    # linear load: after the first full period the voltage is the closed-form one and J_calc = J0
    V_star = J0 / _A_per_volt(d)
    assert V0[2] == pytest.approx(V_star, rel=1e-11)
    assert np.allclose(amp[2:], J0, rtol=1e-11, atol=0)
    assert Vn == pytest.approx(V_star, rel=1e-11)
    # the first correction already moves towards the target (period 0 is short by one step)
    assert abs(amp[1] - J0) < abs(amp[0] - J0)
