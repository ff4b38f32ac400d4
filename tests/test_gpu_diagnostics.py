"""The library's kinetic diagnostics (pic_set_diagnostics / pic_diagnostics) against the oracle.

Each step both sides start from the same particles and the same node field, so the snapshots and
samples see identical electrons; the accumulators are exact integer sums, so the read-outs must be
identical to the last bit: node field, density, mean energy, particle and energy flux, ionization
rate, heating, fast-electron densities, the EEDF and the counts. Cases: FP32 and FP64 stores at a
few thousand particles with the sort every 4 steps (dense and region layouts), a 2e6-electron
store between repacks (several slices of chunks), and the graph path (rf periods as CUDA graphs
with the diagnostic launches inside) against step-by-step launching.
"""
import numpy as np
import pytest

import inputs as I
from oracle import oracle as O
from paper_1608_04601_gb300 import xsections as X
from paper_1608_04601_gb300.workloads import c3

pytestmark = pytest.mark.gpu

KEYS = ("E", "n_e", "mean_eps", "gamma_e", "q_e", "heating", "ion_rate", "n_fast", "n_fast_avg", "eedf",
        "snapshots", "samples")


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    from paper_1608_04601_gb300 import pic
    return pic


def _same(a, b, where=""):
    for k in KEYS:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), f"{where}: {k}"


def _lockstep(P, ref, sim, steps):
    for n in range(steps):
        sim.step(1)
        ref.step(1)
        for sp in (0, 1):
            assert np.array_equal(sim.get_state(0, sp)["c"], ref.get_state(sp)["c"]), (n, sp)
        sim.set_field(0, ref.get_field())


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_diagnostics_match_oracle_bit_for_bit(P, prec):
    d = I.discharge(n_cells=96, gap_m=0.025, p_Pa=60.0, V_rf_V=400.0, n_e0=6000, n_i0=6000, n_init_m3=6e14,
                    gamma_see=0.3, steps_per_period=400, T_e0_eV=4.0)
    gas = X.he_like(eps_max_eV=600.0, de_eV=1e-2)
    ref = O.Oracle(gas, d, "f32" if prec == "fp32" else "f64", sort_every=4)
    sim = P.Simulation(gas, d, seed=d.seed, precision=prec, sort_every=4, load=False)
    for sp in (0, 1):
        sim.set_state(0, sp, ref.get_state(sp))
    sim.set_field(0, ref.get_field())
    cfg = dict(period_steps=5, phase_step=2, sample_every=3, eedf_bins=96, eedf_de_eV=0.25, fast_eV=12.0)
    ref.set_diagnostics(**cfg)
    sim.set_diagnostics(**cfg)
    _lockstep(P, ref, sim, 23)
    a, b = sim.diagnostics(0), ref.diagnostics()
    assert a["snapshots"] == 5 and a["samples"] == 8   # phases 2, 7, .., 22; samples 0, 3, .., 21
    assert np.all(a["n_e"] > 0) and np.any(a["n_fast"] > 0) and np.any(a["ion_rate"] > 0)
    _same(a, b, prec)
    # the reset clears both; the next snapshot and sample are again identical
    sim.reset_diagnostics()
    ref.reset_diagnostics()
    _lockstep(P, ref, sim, 6)
    a, b = sim.diagnostics(0), ref.diagnostics()
    assert a["snapshots"] == 1 and a["samples"] == 2
    _same(a, b, prec + " after reset")
    sim.close()


def test_diagnostics_of_a_large_store_between_repacks(P):
    """2e6 + 2e6 particles (the 500 V He-like discharge at a tenth of its size) on 4000 cells, no
    sort: the diagnostics walk region layouts of several slices of chunks, and at 4000 cells the
    seven node arrays of a step with both a snapshot and a sample (7 x 8 x 4001 bytes) exceed one
    launch's shared memory, so that step takes two launches."""
    d = c3().scaled(n_e0=2_000_000, n_i0=2_000_000, n_cells=4000)
    gas = X.by_name(d.gas, eps_max_eV=d.eps_max_eV, de_eV=d.de_eV)
    ref = O.Oracle(gas, d, "f32", sort_every=0)
    sim = P.Simulation(gas, d, seed=d.seed, precision="fp32", sort_every=0, block=256, ppt=2, load=False)
    for sp in (0, 1):
        sim.set_state(0, sp, ref.get_state(sp))
    sim.set_field(0, ref.get_field())
    cfg = dict(period_steps=3, phase_step=0, sample_every=3, eedf_bins=400, eedf_de_eV=0.5,
               fast_eV=d.V_rf_V / 4)
    ref.set_diagnostics(**cfg)
    sim.set_diagnostics(**cfg)
    _lockstep(P, ref, sim, 7)
    a, b = sim.diagnostics(0), ref.diagnostics()
    assert a["snapshots"] == 3 and a["samples"] == 3
    _same(a, b, "2e6")
    sim.close()


def test_graph_periods_take_the_same_diagnostics_as_single_steps(P):
    """Same seed, same discharge: rf periods as CUDA graphs (schedules that repeat every period) and
    step-by-step launches give identical diagnostics; a schedule that does not repeat every period
    runs step by step under use_graph and still gives the single-step result."""
    d = I.discharge(n_cells=64, gap_m=0.025, p_Pa=30.0, V_rf_V=200.0, n_e0=3000, n_i0=3000, n_init_m3=4e14,
                    steps_per_period=200)
    gas = X.he_like(eps_max_eV=300.0, de_eV=1e-2)
    for cfg in (dict(period_steps=200, phase_step=50, sample_every=10, eedf_bins=120, eedf_de_eV=0.25,
                     fast_eV=50.0),
                dict(period_steps=200, phase_step=50, sample_every=7, eedf_bins=120, eedf_de_eV=0.25,
                     fast_eV=50.0)):
        out = []
        for graph in (False, True):
            sim = P.Simulation(gas, d, seed=5, precision="fp32", sort_every=8, use_graph=graph)
            sim.step(200)            # one period without diagnostics (graph captured without them)
            sim.set_diagnostics(**cfg)
            sim.step(3 * 200)
            out.append(sim.diagnostics(0))
            sim.close()
        assert out[0]["snapshots"] == 3
        assert out[0]["samples"] == len([n for n in range(200, 800) if n % cfg["sample_every"] == 0])
        _same(out[0], out[1], f"graph vs steps, sample_every {cfg['sample_every']}")
