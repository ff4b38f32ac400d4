"""Pins of the two push schemes of the oracle against the exact expectation of their discrete
dynamics (section "PIC/MCC simulation procedure": velocity Verlet, chosen over leapfrog for its
faster convergence in dt).

Electrons in a uniform field (acceleration a along z), one elastic process of constant rate nu
(sigma proportional to 1/v) on an infinitely heavy target: every collision turns the velocity to an
isotropic direction at the same speed, so its mean after a collision is zero whatever it was
before. A particle collides in a step with probability p = 1 - exp(-nu dt) (null-collision
method with nu_max = nu). The mean of the stored velocity (the one each step's drift uses) then
obeys, per step,
  velocity Verlet (collision between the two half kicks):  m' = (1 - p)(m + a dt/2) + a dt/2
  leapfrog (collision after the full kick v + a dt):       m' = (1 - p)(m + a dt)
with fixed points m_V = a dt (1 - p/2) / p and m_L = a dt (1 - p) / p, against the continuum
drift a / nu. With x = nu dt: m_V nu / a = x (1 - p/2) / p = 1 + x^2/12 + O(x^4), second order in
dt, and m_L nu / a = x (1 - p) / p = 1 - x/2 + O(x^2), first order.
"""
import math

import numpy as np
import pytest

import inputs as I
from oracle import oracle as O
from paper_1608_04601_gb300 import xsections as X

NU = 1.0e9          # collision frequency, 1/s
E0 = -1.0e3         # V/m: electrons accelerate towards +z
N_CELLS, GAP = 4096, 10.0


def _mean_drift(leapfrog: bool, x: float, n=200_000, seed=5):
    dt = x / NU
    # the mean relaxes by (1 - p) per step: average after 8 / p steps, over 100 steps
    first = int(8.0 / -math.expm1(-x)) + 1
    steps = first + 100
    d = I.discharge(n_cells=N_CELLS, gap_m=GAP, V_rf_V=0.0, n_e0=n, n_i0=1, n_init_m3=1e8,
                    steps_per_period=max(1, round(1.0 / (13.56e6 * dt))), p_Pa=30.0)
    d = d.scaled(f_rf_Hz=1.0 / (d.steps_per_period * dt))  # so that d.dt_s == dt
    n_gas = d.p_Pa / (I.K_B * d.T_gas_K)
    gas = X.constant_nu(NU / n_gas, 1.0e6 * I.AMU, eps_max_eV=2000.0, de_eV=1e-3)
    o = O.Oracle(gas, d, "f64", load=False)
    o.set_scheme(leapfrog)
    rng = np.random.default_rng(seed)
    st = I.maxwell_state(rng, n, N_CELLS, math.sqrt(I.E_CH * 0.5 / I.M_E), np.float64,
                         cells=rng.integers(N_CELLS // 2 - 8, N_CELLS // 2 + 8, n))
    o.set_state(0, st)
    o.set_state(1, {k: v[:1] for k, v in I.maxwell_state(rng, 1, N_CELLS, 0.0).items()})
    o.set_field(np.full(N_CELLS + 1, E0))
    means = []
    for k in range(steps):
        o.step_index = k
        o.sweep()  # no field solve: the field stays uniform
        if k >= first:
            means.append(float(np.mean(o.get_state(0)["vz"])))
    assert o.count(0) == n  # nobody reached a wall
    a = -I.E_CH / I.M_E * E0
    p = 1.0 - math.exp(-x)
    return np.mean(means) * NU / a, x, p


@pytest.mark.parametrize("x", [0.4, 0.1])
def test_velocity_verlet_drift_is_its_discrete_fixed_point(x):
    got, x, p = _mean_drift(False, x)
    assert got == pytest.approx(x * (1 - p / 2) / p, abs=0.01)


@pytest.mark.parametrize("x", [0.4, 0.1])
def test_leapfrog_drift_is_its_discrete_fixed_point(x):
    got, x, p = _mean_drift(True, x)
    assert got == pytest.approx(x * (1 - p) / p, abs=0.01)


def test_orders_of_convergence():
    """The closed forms themselves: Verlet's error is second order in dt, leapfrog's first order."""
    for x in (0.4, 0.2, 0.1, 0.05):
        p = -math.expm1(-x)
        eV, eL = x * (1 - p / 2) / p - 1, x * (1 - p) / p - 1
        assert eV == pytest.approx(x * x / 12, rel=0.05)
        assert eL == pytest.approx(-x / 2, rel=0.25)


@pytest.mark.parametrize("leapfrog", [False, True])
def test_a_collision_keeps_the_speed_of_the_velocity_it_acts_on(leapfrog):
    """One step on the infinitely heavy target: a colliding electron keeps its speed, that of v_n
    (velocity Verlet) or of v_{n+1/2} (leapfrog); particles that did not collide have the two half
    kicks. The stored velocity after the step is v_n' + K E (Verlet) or v_{n+1/2}' (leapfrog),
    K = (q/m) dt / 2."""
    x, n = 0.4, 20_000
    dt = x / NU
    d = I.discharge(n_cells=N_CELLS, gap_m=GAP, V_rf_V=0.0, n_e0=n, n_i0=1, n_init_m3=1e8, p_Pa=30.0,
                    steps_per_period=100)
    d = d.scaled(f_rf_Hz=1.0 / (100 * dt))
    n_gas = d.p_Pa / (I.K_B * d.T_gas_K)
    gas = X.constant_nu(NU / n_gas, 1.0e6 * I.AMU, eps_max_eV=2000.0, de_eV=1e-3)
    o = O.Oracle(gas, d, "f64", load=False)
    o.set_scheme(leapfrog)
    rng = np.random.default_rng(2)
    st = I.maxwell_state(rng, n, N_CELLS, 1.0e6, np.float64, cells=np.full(n, N_CELLS // 2))
    o.set_state(0, st)
    o.set_state(1, {k: v[:1] for k, v in I.maxwell_state(rng, 1, N_CELLS, 0.0).items()})
    o.set_field(np.full(N_CELLS + 1, E0))
    K = -I.E_CH / I.M_E * dt / 2
    o.sweep()
    out = o.get_state(0)
    assert out["c"].size == n  # survivors keep their order; nobody leaves in one step
    vn = np.stack([st["vx"], st["vy"], st["vz"] + K * E0])           # v_n
    vh = np.stack([st["vx"], st["vy"], st["vz"] + K * E0 + K * E0])  # v_{n+1/2}
    w = np.stack([out["vx"], out["vy"], out["vz"]])
    if not leapfrog:
        w = w - np.array([0.0, 0.0, K * E0])[:, None]                 # v_n after the collision
    ref = vh if leapfrog else vn
    moved = np.max(np.abs(w - ref), axis=0) > 1e-6 * np.linalg.norm(ref, axis=0)
    assert 0.25 < moved.mean() < 0.42  # about p = 1 - exp(-0.4) of them collided
    speed = np.linalg.norm(w[:, moved], axis=0)
    # the target's recoil changes the speed by at most 2 beta, beta = m_e / (m_e + M) = 5.5e-10
    assert np.allclose(speed, np.linalg.norm(ref[:, moved], axis=0), rtol=3e-9, atol=0)
