"""Pins of the oracle's kinetic diagnostics (CPU, FP64 build) against closed forms.

The quantities are the ones the paper compares (section "Results"): the time- and space-averaged
isotropic distribution f0(U)/n_e (normalised so that the integral of sqrt(U) f0/n_e dU is 1), the
density of fast electrons (energy above a threshold, e0 V0 / 4 in the paper), and the profiles of
the electric field, density, mean energy U_e, particle flux Gamma_e, energy flux Q_e, ionization
rate S and heating -e0 E Gamma_e at a fixed rf phase. Every check uses a state whose moments are
known in closed form: a uniform Maxwellian at rest or drifting along z, a constant ionization rate
coefficient, a uniform field.
"""
import math

import numpy as np
import pytest
from scipy import special

import inputs as I
from oracle import oracle as O
from paper_1608_04601_gb300 import xsections as X

N, GAP = 64, 0.02


def _no_coll_gas(n_pts=20001, de=5e-3):
    z = np.zeros(n_pts)
    return X.GasTables("none", 4.002602 * I.AMU, (1e9,), 2e9, de, np.stack([z, z, z], 1), np.stack([z, z], 1))


def _oracle(gas, n, T_eV, drift=0.0, E0=0.0, seed=0, st=None):
    d = I.discharge(n_cells=N, gap_m=GAP, V_rf_V=0.0, n_e0=n, n_i0=n, n_init_m3=1e15, steps_per_period=400)
    o = O.Oracle(gas, d, "f64", load=False)
    rng = np.random.default_rng(seed)
    if st is None:
        st = I.maxwell_state(rng, n, N, math.sqrt(I.E_CH * T_eV / I.M_E), np.float64, drift=(0.0, 0.0, drift))
    # the diagnostics see v_n = v* + (q/m) E dt/2: store v* so that v_n is the Maxwellian sample
    st["vz"] = st["vz"] - (-I.E_CH / I.M_E) * E0 * d.dt_s / 2
    o.set_state(0, st)
    o.set_state(1, {k: v[:1] for k, v in I.maxwell_state(rng, 1, N, 0.0).items()})
    o.set_field(np.full(N + 1, E0))
    return o, d, st


def test_maxwellian_eedf_density_energy_and_fast_fraction():
    n, T = 400_000, 3.0
    o, d, st = _oracle(_no_coll_gas(), n, T)
    bins, de = 160, 0.25
    o.set_diagnostics(period_steps=1, phase_step=0, sample_every=1, eedf_bins=bins, eedf_de_eV=de, fast_eV=10.0)
    o.step(1)
    g = o.diagnostics()
    assert g["snapshots"] == 1 and g["samples"] == 1
    # f0(U)/n_e of a Maxwellian: 2 / sqrt(pi) T^{-3/2} exp(-U/T); compare bin averages where counts are large
    U = (np.arange(bins) + 0.5) * de
    lo, hi = np.arange(bins) * de, (np.arange(bins) + 1) * de
    p_bin = special.gammainc(1.5, hi / T) - special.gammainc(1.5, lo / T)   # probability of each bin
    expect = p_bin / (de * np.sqrt(U))
    counts = g["eedf"] * (n * de * np.sqrt(U))
    good = p_bin * n > 400
    assert good.sum() > 40
    assert np.all(np.abs(g["eedf"][good] - expect[good]) <= 5 * expect[good] / np.sqrt(p_bin[good] * n))
    assert abs(counts.sum() - n) < 1e-6 * n
    # density: the loaded one; mean energy 3/2 T; no net flux
    inner = slice(1, N)
    assert np.mean(g["n_e"][inner]) == pytest.approx(d.w_e * n / GAP, rel=5e-3)
    # the wall nodes own half a cell: the same density there (about 3000 particles each, 10 %)
    assert g["n_e"][0] == pytest.approx(d.w_e * n / GAP, rel=0.1)
    assert g["n_e"][N] == pytest.approx(d.w_e * n / GAP, rel=0.1)
    assert np.mean(g["mean_eps"][inner]) == pytest.approx(1.5 * T, rel=5e-3)
    vth = math.sqrt(I.E_CH * T / I.M_E)
    assert abs(np.mean(g["gamma_e"][inner])) <= 5 * (d.w_e * n / GAP) * vth / math.sqrt(n)
    # fast electrons: the Maxwellian's fraction above 10 eV, regularised upper incomplete gamma
    frac = special.gammaincc(1.5, 10.0 / T)
    got = np.mean(g["n_fast"][inner]) / np.mean(g["n_e"][inner])
    assert abs(got - frac) <= 5 * math.sqrt(frac / n) + 1e-3 * frac
    assert np.allclose(g["n_fast_avg"], g["n_fast"], rtol=0, atol=0)  # one sample, one snapshot: the same


def test_drifting_maxwellian_fluxes_and_heating():
    """Drift v_d along z, temperature T, uniform field E0: Gamma_e = n v_d,
    Q_e = n v_d (m v_d^2 / 2 + 5/2 e T), U_e = 3/2 T + m v_d^2 / (2 e), heating -e0 E0 Gamma_e."""
    n, T, vd, E0 = 400_000, 2.0, 4.0e5, -2.0e6
    o, d, st = _oracle(_no_coll_gas(), n, T, drift=vd, E0=E0)
    o.set_diagnostics(period_steps=1, phase_step=0, sample_every=0, eedf_bins=8, eedf_de_eV=1.0, fast_eV=1e9)
    o.step(1)
    g = o.diagnostics()
    inner = slice(1, N)
    ne = d.w_e * n / GAP
    vth = math.sqrt(I.E_CH * T / I.M_E)
    Gam = np.mean(g["gamma_e"][inner])
    assert abs(Gam - ne * vd) <= 5 * ne * vth / math.sqrt(n) + 1e-3 * ne * vd
    Qe = ne * vd * (0.5 * I.M_E * vd ** 2 + 2.5 * I.E_CH * T)
    assert np.mean(g["q_e"][inner]) == pytest.approx(Qe, rel=0.03)
    assert np.mean(g["mean_eps"][inner]) == pytest.approx(1.5 * T + 0.5 * I.M_E * vd ** 2 / I.E_CH, rel=5e-3)
    assert np.allclose(g["E"], E0)
    assert np.allclose(g["heating"], -I.E_CH * E0 * g["gamma_e"], rtol=1e-14, atol=0)
    assert g["samples"] == 0 and np.all(g["n_fast"] == 0)


def test_ionization_rate_of_a_constant_rate_coefficient():
    """sigma_iz proportional to 1/v with a zero threshold: every electron has the rate coefficient
    k_iz, so S = n_gas n_e k_iz at every node. A nonzero elastic rate checks that only the
    ionization channel is counted. Energies are drawn in [1, 20] eV, away from the table's first
    interval (where the 1/v form is cut off); each electron's k_iz is rounded to a multiple of
    2^-72 m^3/s (relative 5e-9 at this k_iz), hence the tolerance."""
    k_iz = 2e-14
    gas = X.constant_nu(5e-14, 4.002602 * I.AMU, eps_max_eV=60.0, de_eV=5e-3, k_iz=k_iz)
    n = 100_000
    st = I.energy_state(np.random.default_rng(3), n, N, 1.0, 20.0, I.M_E)
    o, d, st = _oracle(gas, n, 0.0, st=st)
    o.set_diagnostics(period_steps=4, phase_step=0, sample_every=0, eedf_bins=8, eedf_de_eV=1.0, fast_eV=1e9)
    o.step(1)
    g = o.diagnostics()
    n_gas = d.p_Pa / (I.K_B * d.T_gas_K)
    assert g["snapshots"] == 1
    assert np.allclose(g["ion_rate"], n_gas * g["n_e"] * k_iz, rtol=2e-8, atol=0)


def test_averages_over_snapshots_and_samples():
    """Three snapshots (every step) and two samples (every second step) of a slowly evolving gas in
    a held field: the field average is the held field, and the fast-electron density averaged
    over the samples carries the same number of fast electrons as the one over the snapshots."""
    n, T, E0 = 100_000, 3.0, 150.0
    o, d, st = _oracle(_no_coll_gas(), n, T, E0=E0)
    o.set_diagnostics(period_steps=1, phase_step=0, sample_every=2, eedf_bins=8, eedf_de_eV=1.0, fast_eV=8.0)
    for _ in range(3):
        o.set_field(np.full(N + 1, E0))
        o.step(1)
    g = o.diagnostics()
    assert g["snapshots"] == 3 and g["samples"] == 2
    assert np.allclose(g["E"], E0, rtol=1e-15, atol=0)
    V = np.full(N + 1, GAP / N)
    V[0] = V[N] = GAP / N / 2
    a, b = np.sum(g["n_fast"] * V), np.sum(g["n_fast_avg"] * V)
    assert a > 0 and b == pytest.approx(a, rel=2e-3)


def test_phase_schedule_and_reset():
    """Snapshots at the steps n with n % period == phase only; samples every sample_every steps;
    the reset clears everything."""
    o, d, st = _oracle(_no_coll_gas(), 2000, 2.0)
    o.set_diagnostics(period_steps=5, phase_step=2, sample_every=3, eedf_bins=8, eedf_de_eV=1.0, fast_eV=1.0)
    o.step(11)                 # steps 0..10: phases at 2, 7; samples at 0, 3, 6, 9
    g = o.diagnostics()
    assert g["snapshots"] == 2 and g["samples"] == 4
    o.reset_diagnostics()
    g = o.diagnostics()
    assert g["snapshots"] == 0 and g["samples"] == 0 and np.all(g["n_e"] == 0) and np.all(g["eedf"] == 0)
