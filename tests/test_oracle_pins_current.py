"""Pins of the oracle's discharge current density (CPU, FP64 build).

J(t) = eps0 dE(0,t)/dt + e0 (Gamma_i - Gamma_e)(0,t) (arXiv:1608.04601, section "Boundary
conditions", the equation for the current density that the fluid models take as input). The
oracle evaluates it over every step from the change of the electrode field between two solves and
the charge of the superparticles absorbed or emitted at the electrode during the sweep.
"""
import math

import numpy as np

import inputs as I
from oracle import oracle as O
from paper_1608_04601_gb300 import xsections as X


def _empty(n):
    return {"c": np.zeros(n, np.int32), "f": np.zeros(n), "vx": np.zeros(n), "vy": np.zeros(n), "vz": np.zeros(n)}


def test_vacuum_gap_displacement_current_closed_form():
    """No charge in the gap: the potential is linear, E(0,t) = V0 sin(w t) / d, and the current is
    the displacement current of a plate capacitor, J_n = eps0 (V(t_{n+1}) - V(t_n)) / (d dt) exactly
    (up to rounding); at z = d it is the same. The first step after creation has no earlier field."""
    d = I.discharge(n_cells=64, gap_m=0.02, V_rf_V=250.0, steps_per_period=200)
    o = O.Oracle(X.he_like(eps_max_eV=20.0, de_eV=1e-2), d, "f64", load=False)
    o.set_state(0, _empty(0))
    o.set_state(1, _empty(0))
    w, dt, eps0 = 2 * math.pi * d.f_rf_Hz, d.dt_s, I.EPS0
    for n in range(260):
        o.step(1)
        J = o.last_current()
        if n == 0:
            assert J[0] == 0.0 and J[1] == 0.0
            continue
        ref = eps0 * d.V_rf_V * (math.sin(w * (n + 1) * dt) - math.sin(w * n * dt)) / (d.gap_m * dt)
        scale = eps0 * d.V_rf_V * w / d.gap_m
        assert abs(J[0] - ref) <= 1e-9 * scale, (n, J, ref)
        assert abs(J[1] - ref) <= 1e-9 * scale


def test_current_is_the_same_at_both_electrodes():
    """Conservation of charge: with equal electron and ion weights, an ionization is neutral and the
    gap's net charge changes only by what the electrodes absorb or emit; by Gauss's law over the
    gap (the discrete form holds exactly: the node volumes dx/2 at the walls and dx inside add up
    to the charge of all superparticles) J at z = 0 and J at z = d must then agree to rounding.
    The discharge is driven at 400 V with secondary emission, so the step's absorbed electrons and
    ions at both walls, the ionization births and the emitted electrons all enter."""
    d = I.discharge(n_cells=96, gap_m=0.025, p_Pa=60.0, V_rf_V=400.0, n_e0=6000, n_i0=6000, n_init_m3=6e14,
                    gamma_see=0.3, steps_per_period=400, T_e0_eV=4.0)
    assert d.w_e == d.w_i
    o = O.Oracle(X.he_like(eps_max_eV=600.0, de_eV=1e-2), d, "f64", sort_every=4)
    J = []
    for _ in range(300):
        o.step(1)
        J.append(o.last_current())
    J = np.array(J)
    c = o.counters()
    assert c["see_emitted"] > 0 and c["collisions_e"][3] > 0
    assert min(c["absorbed"][0]) > 0 and min(c["absorbed"][1]) > 0
    scale = np.max(np.abs(J[:, 0]))
    assert scale > 0
    assert np.max(np.abs(J[:, 0] - J[:, 1])) <= 1e-9 * scale
    # the conduction part is present: the displacement current alone would break the equality
    assert np.max(np.abs(np.diff(J[:, 0]))) > 1e-6 * scale


def test_current_of_a_charge_sheet_absorbed_in_one_step():
    """Grounded plates, no collisions, n electrons at z_s = (c + f) dx with no velocity: their field
    is that of a charge sheet. Then every one of them reaches z = 0 within one step and is absorbed.
    The step's current is the same at both electrodes and equals e w n z_s / (d dt): at z = 0 the
    conduction part e w n / dt (negative charge leaving towards -z) less the displacement part of
    the sheet's field at z = 0 vanishing, eps0 E(0) = e w n (d - z_s) / d; at z = d only the
    displacement part of E(d) = -e w n z_s / (eps0 d) vanishing."""
    N, gap, c0, f0 = 32, 0.02, 10, 0.5
    d = I.discharge(n_cells=N, gap_m=gap, V_rf_V=0.0, n_e0=1000, n_i0=1000, n_init_m3=1e14)
    gas = X.GasTables("none", 4.002602 * I.AMU, (1e9,), 2e9, 1.0, np.zeros((11, 3)), np.zeros((11, 2)))
    o = O.Oracle(gas, d, "f64", load=False)
    n = 400
    st = _empty(n)
    st["c"][:] = c0
    st["f"][:] = f0
    o.set_state(0, st)
    o.set_state(1, _empty(0))
    o.set_field(np.zeros(N + 1))
    o.sweep()                      # the electrons stay and are deposited
    o.solve()                      # the first solve of the run: no current yet
    assert np.all(o.last_current() == 0.0)
    E = o.get_field64()
    sig = I.E_CH * d.w_e * n
    zs = (c0 + f0) * gap / N
    assert abs(I.EPS0 * E[0] - sig * (gap - zs) / gap) <= 1e-12 * sig
    assert abs(I.EPS0 * E[N] + sig * zs / gap) <= 1e-12 * sig
    st["vz"][:] = -(c0 + f0 + 1.0) * (gap / N) / d.dt_s
    o.set_state(0, st)
    o.sweep()                      # every electron is absorbed at z = 0
    assert o.counters()["absorbed"][0][0] == n and o.count(0) == 0
    o.solve()
    J = o.last_current()
    ref = sig * zs / (gap * d.dt_s)
    assert abs(J[0] - ref) <= 1e-12 * ref and abs(J[1] - ref) <= 1e-12 * ref
