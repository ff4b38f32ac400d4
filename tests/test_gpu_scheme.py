"""The leapfrog variant of the push on the device (pic_options.leapfrog), against the oracle and as
a dt-convergence study.

  * bit-exact lockstep with the oracle in the leapfrog scheme (FP32 and FP64 stores, with
    ionization and ion collisions): event counters, cells, order and every stored value after
    each step;
  * the study (section "PIC/MCC simulation procedure": velocity Verlet was chosen for its faster
    convergence in dt): electrons with a constant collision rate on an infinitely heavy target in
    a uniform field drift at a / nu in the continuum; the mean stored velocity of 1e6 electrons
    for nu dt = 0.4 ... 0.05 matches each scheme's discrete fixed point, whose error is second
    order in dt for velocity Verlet and first order for leapfrog (fitted orders asserted).
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
def test_leapfrog_steps_bit_exact(P, prec):
    d = I.discharge(n_cells=96, gap_m=0.025, p_Pa=80.0, V_rf_V=500.0, n_e0=8000, n_i0=8000, n_init_m3=6e14,
                    gamma_see=0.3, steps_per_period=400, T_e0_eV=8.0)
    gas = X.he_like(eps_max_eV=800.0, de_eV=1e-2)
    ref = O.Oracle(gas, d, "f32" if prec == "fp32" else "f64", sort_every=4)
    ref.set_scheme(True)
    sim = P.Simulation(gas, d, seed=d.seed, precision=prec, sort_every=4, load=False, leapfrog=True)
    for sp in (0, 1):
        sim.set_state(0, sp, ref.get_state(sp))
    sim.set_field(0, ref.get_field())
    for n in range(30):
        sim.step(1)
        ref.step(1)
        assert sim.counters(0) == ref.counters(), n
        for sp in (0, 1):
            a, b = sim.get_state(0, sp), ref.get_state(sp)
            for k in ("c", "f", "vx", "vy", "vz"):
                assert np.array_equal(a[k], b[k]), (n, sp, k)
        sim.set_field(0, ref.get_field())
    c = sim.counters(0)
    assert c["collisions_e"][3] > 0 and sum(c["collisions_i"]) > 0  # ionization and ion collisions happened
    sim.close()


NU, E0, N_CELLS, GAP = 1.0e9, -1.0e3, 4096, 10.0


def _drift(P, leapfrog, x, n=1_000_000):
    dt = x / NU
    d = I.discharge(n_cells=N_CELLS, gap_m=GAP, V_rf_V=0.0, n_e0=n, n_i0=1, n_init_m3=1e8, p_Pa=30.0,
                    steps_per_period=100)
    d = d.scaled(f_rf_Hz=1.0 / (100 * dt))
    n_gas = d.p_Pa / (I.K_B * d.T_gas_K)
    gas = X.constant_nu(NU / n_gas, 1.0e6 * I.AMU, eps_max_eV=2000.0, de_eV=1e-3)
    sim = P.Simulation(gas, d, seed=9, precision="fp64", load=False, leapfrog=leapfrog)
    rng = np.random.default_rng(4)
    st = I.maxwell_state(rng, n, N_CELLS, math.sqrt(I.E_CH * 0.5 / I.M_E), np.float64,
                         cells=rng.integers(N_CELLS // 2 - 8, N_CELLS // 2 + 8, n))
    sim.set_state(0, 0, st)
    sim.set_state(0, 1, {k: v[:1] for k, v in I.maxwell_state(rng, 1, N_CELLS, 0.0).items()})
    sim.set_field(0, np.full(N_CELLS + 1, E0))
    p = -math.expm1(-x)
    first = int(8.0 / p) + 1
    means = []
    for k in range(first + 100):
        sim.step_index = k
        sim.sweep()  # no solve: the field stays uniform
        if k >= first:
            means.append(float(np.mean(sim.get_state(0, 0)["vz"])))
    assert sim.count(0, 0) == n
    sim.close()
    a = -I.E_CH / I.M_E * E0
    return np.mean(means) * NU / a, p


def test_dt_convergence_of_the_two_schemes(P):
    xs = [0.4, 0.2, 0.1, 0.05]
    err = {False: [], True: []}
    for lf in (False, True):
        for x in xs:
            got, p = _drift(P, lf, x)
            fixed = x * (1 - p) / p if lf else x * (1 - p / 2) / p
            print(f"leapfrog={lf} nu dt={x}: drift / (a/nu) = {got:.5f}, discrete fixed point {fixed:.5f}")
            assert got == pytest.approx(fixed, abs=0.004)
            err[lf].append(abs(fixed - 1.0))
    # orders of convergence of the fixed points (the measured drifts match them, above)
    sV = np.polyfit(np.log(xs), np.log(err[False]), 1)[0]
    sL = np.polyfit(np.log(xs), np.log(err[True]), 1)[0]
    assert 1.9 < sV < 2.1 and 0.9 < sL < 1.1, (sV, sL)
    # and the measured leapfrog error is well resolved at every dt, Verlet's at the largest
    assert err[True][-1] > 0.02 and err[False][0] > 0.01
