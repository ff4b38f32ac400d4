"""One-period CUDA graphs and batched discharges: same results as plain launches, bit for bit."""
import numpy as np
import pytest

import inputs as I
from paper_1608_04601_gb300 import xsections as X

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    from paper_1608_04601_gb300 import pic
    return pic


def _states(sim, nd):
    return [[sim.get_state(d, sp) for sp in (0, 1)] for d in range(nd)]


def test_graph_replay_matches_plain_launches(P):
    d = I.discharge(n_cells=128, n_e0=20000, n_i0=20000, V_rf_V=150.0, n_init_m3=4e14, steps_per_period=40,
                    gamma_see=0.1, seed=5)
    gas = X.he_like(eps_max_eV=300.0, de_eV=1e-2)
    out = []
    for graph in (False, True):
        sim = P.Simulation(gas, d, precision="fp32", sort_every=8, use_graph=graph)
        sim.step(40 * 3 + 7)      # three periods (graph replays) and a remainder
        sim.sync()
        out.append((_states(sim, 1), sim.get_field(0)[1], sim.moments(0)))
        sim.close()
    (s0, E0, m0), (s1, E1, m1) = out
    for sp in (0, 1):
        for k in ("c", "f", "vx", "vy", "vz"):
            assert np.array_equal(s0[0][sp][k], s1[0][sp][k])
    assert np.array_equal(E0, E1)
    assert np.array_equal(m0["n_e"], m1["n_e"]) and m0["steps"] == m1["steps"] == 127


def test_batch_equals_discharges_run_alone(P):
    """A batch of discharges advances each exactly as it would alone (same seed, own discharge id)."""
    gases = [X.he_like(eps_max_eV=300.0, de_eV=1e-2), X.ar_like(eps_max_eV=300.0, de_eV=1e-2)]
    specs = [("he", 0, 64, 20.0, 3000, 150.0), ("ar", 1, 96, 40.0, 7000, 250.0), ("he", 0, 128, 80.0, 500, 350.0)]
    dis = []
    for k, (g, gi, N, p, n, V) in enumerate(specs):
        dis.append((I.discharge(gas=g, n_cells=N, p_Pa=p, n_e0=n, n_i0=n, V_rf_V=V, n_init_m3=4e14,
                                steps_per_period=100, discharge_id=k, seed=9), gi))
    batch = P.Simulation(gases, dis, seed=9, precision="fp32", sort_every=5)
    batch.step(60)
    batch.sync()
    for k, (d, gi) in enumerate(dis):
        alone = P.Simulation(gases, [(d, gi)], seed=9, precision="fp32", sort_every=5)
        alone.step(60)
        alone.sync()
        for sp in (0, 1):
            a, b = batch.get_state(k, sp), alone.get_state(0, sp)
            for key in ("c", "f", "vx", "vy", "vz"):
                assert np.array_equal(a[key], b[key]), (k, sp, key)
        assert np.array_equal(batch.get_field(k)[1], alone.get_field(0)[1])
        alone.close()
    batch.close()
