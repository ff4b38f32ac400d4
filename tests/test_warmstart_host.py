"""Host logic of the warm-start pipeline (no GPU): the discharge family, the network's input
features and the profile <-> target transforms."""
import numpy as np

from paper_1608_04601_gb300 import warmstart as W


def test_family_is_seeded_and_inside_its_box():
    a, b = W.family(20, 3), W.family(20, 3)
    assert [(d.p_Pa, d.V_rf_V, d.gap_m, d.f_rf_Hz) for d in a] == [(d.p_Pa, d.V_rf_V, d.gap_m, d.f_rf_Hz) for d in b]
    for d in a:
        assert W.P_RANGE[0] <= d.p_Pa <= W.P_RANGE[1] and W.V_RANGE[0] <= d.V_rf_V <= W.V_RANGE[1]
        assert W.GAP_RANGE[0] <= d.gap_m <= W.GAP_RANGE[1] and W.F_RANGE[0] <= d.f_rf_Hz <= W.F_RANGE[1]
        assert d.steps_per_period == 400
        assert abs(d.dt_s * d.f_rf_Hz * d.steps_per_period - 1.0) < 1e-12
    assert len({d.discharge_id for d in W.family(5, 1, first_id=100)}) == 5


def test_features_are_order_one():
    f = np.stack([W.features(d) for d in W.family(200, 4)])
    assert f.shape == (200, 5) and np.all(np.abs(f) <= 1.0)


def test_target_round_trip():
    d = W.family(1, 5)[0]
    z = np.linspace(0, d.gap_m, d.n_cells + 1)
    m = {"n_e": 3e15 * np.sin(np.pi * z / d.gap_m) ** 2 + 1e13, "n_i": 3.2e15 * np.sin(np.pi * z / d.gap_m) + 2e13,
         "mean_eps": 2.0 + 3.0 * (2 * z / d.gap_m - 1) ** 2}
    y = W.to_target(m, d)
    assert y.shape == (3 * W.NPTS,)
    back = W.from_target(y)
    s = np.linspace(0, d.gap_m, W.NPTS)
    assert np.allclose(back[0], np.interp(s, z, m["n_e"]), rtol=1e-5)
    assert np.allclose(back[1], np.interp(s, z, m["n_i"]), rtol=1e-5)
    assert np.allclose(back[2], np.interp(s, z, m["mean_eps"]), rtol=1e-5)


def test_density_floor_and_energy_floor():
    d = W.family(1, 6)[0]
    m = {k: np.zeros(d.n_cells + 1) for k in ("n_e", "n_i", "mean_eps")}
    back = W.from_target(W.to_target(m, d))
    assert np.allclose(back[0], 1e12) and np.allclose(back[1], 1e12) and np.allclose(back[2], 0.1)


def test_sign_test_probabilities():
    """One-sided sign test: P(at least k of n fair coin flips) -- closed forms for small n."""
    assert W.sign_test_p(8, 8) == 1 / 256
    assert W.sign_test_p(7, 8) == 9 / 256
    assert W.sign_test_p(0, 5) == 1.0
    assert abs(W.sign_test_p(10, 12) - (66 + 12 + 1) / 4096) < 1e-15
