"""Pins of the oracle's collision decisions and scattering laws (CPU, FP64 build).

Null-collision method and scattering of arXiv:1608.04601, section "PIC/MCC simulation procedure"
and Table "reactions": a particle is a candidate with P_null = 1 - exp(-nu_max dt); a candidate
undergoes process j when u nu_max falls into the j-th interval of the cumulative rates at its
energy, and otherwise a null collision; rates are linear interpolations of the tabulated sigma v;
scattering is isotropic (in the centre-of-mass frame for ion-atom pairs) except the backward ion
process. Each pin below is chosen so that a plausible slip in the oracle fails it: comparing
against the rate of one process instead of the cumulative sum, an off-by-one process column or
table row, swapped interpolation weights, a direction drawn in the wrong frame, or a wrong
emission law for secondary electrons.
"""
import math

import numpy as np
import pytest
from scipy import stats

import inputs as I
from oracle import oracle as O
from paper_1608_04601_gb300 import xsections as X

HEAVY = 1e7 * I.AMU  # target mass: elastic scattering leaves the speed unchanged


def _rates_gas(mass, de, n_pts, k_e_cols, k_i_cols, eps_exc, eps_iz):
    """Gas whose tabulated sigma v (electrons, lab energy) and sigma g (ions, centre-of-mass energy)
    are the given rate-coefficient columns (m^3/s) on the grid eps_k = k de."""
    eps = np.arange(n_pts) * de
    v = np.sqrt(2 * I.E_CH * np.maximum(eps, 1e-6 * de) / I.M_E)
    g = np.sqrt(4 * I.E_CH * np.maximum(eps, 1e-6 * de) / mass)
    se = np.stack([k / v for k in k_e_cols], 1)
    si = np.stack([k / g for k in k_i_cols], 1)
    return X.GasTables("rates", mass, tuple(eps_exc), eps_iz, de, np.ascontiguousarray(se),
                       np.ascontiguousarray(si))


def _discharge(p=30.0, n_cells=64):
    return I.discharge(n_cells=n_cells, p_Pa=p, gap_m=1.0, steps_per_period=400)


def _run_once(gas, d, e_state=None, i_state=None, seed_rng=0):
    o = O.Oracle(gas, d, "f64", load=False)
    o.set_field(np.zeros(d.n_cells + 1))
    rng = np.random.default_rng(seed_rng)
    o.set_state(0, e_state if e_state is not None else I.speed_state(rng, 1, d.n_cells, 0.0))
    o.set_state(1, i_state if i_state is not None else I.speed_state(rng, 1, d.n_cells, 0.0))
    o.sweep()
    return o


def _within(k, n, p, z=5.0):
    return abs(k - n * p) <= z * math.sqrt(n * p * (1 - p))


def test_electron_process_selection_multinomial():
    """Four electron processes with constant rates in the ratio 1:2:3:4 at the particles' energy and
    a larger total elsewhere in the table (nu_max = 20 k, so half of the candidates are null):
    the counts of elastic, excitation 1, excitation 2 and ionization are multinomial with
    probabilities P_null j k / nu_max, the null collisions take the rest, nothing else happens."""
    d = _discharge()
    n_gas = d.p_Pa / (I.K_B * d.T_gas_K)
    k = 0.5 / (20 * n_gas * d.dt_s)  # nu_max dt = 0.5
    de, n_pts = 1e-2, 10001
    eps = np.arange(n_pts) * de
    hi = eps >= 50.0
    cols = [np.where(hi, 11 * k, k), np.full(n_pts, 2 * k), np.full(n_pts, 3 * k), np.full(n_pts, 4 * k)]
    # thresholds far below the particles' 10 eV: every selected inelastic process is real
    gas = _rates_gas(HEAVY, de, n_pts, cols, [np.zeros(n_pts)] * 2, (0.05, 0.1), 0.15)
    n = 1_000_000
    rng = np.random.default_rng(21)
    e = I.speed_state(rng, n, d.n_cells, math.sqrt(2 * I.E_CH * 10.0 / I.M_E))
    o = _run_once(gas, d, e_state=e)
    c = o.counters()
    P = -math.expm1(-20 * k * n_gas * d.dt_s)
    assert _within(c["candidates"][0], n, P)
    for j in range(4):
        assert _within(c["collisions_e"][j], n, P * (j + 1) / 20), (j, c["collisions_e"])
    real = sum(c["collisions_e"])
    assert _within(c["candidates"][0] - real, n, P * 10 / 20)
    assert c["null_inelastic"] == 0 and c["collisions_i"] == [0, 0] and c["table_clamped"] == [0, 0]
    # the ionizations added one electron and one ion each
    assert o.count(0) == n + c["collisions_e"][3] and o.count(1) == 1 + c["collisions_e"][3]


def test_ion_process_selection_multinomial():
    """Isotropic and backward ion processes with constant rates 1:2 below 50 eV (centre of mass) and
    nu_max = 7 k from a larger isotropic rate above: counts are multinomial with P_null k_j / nu_max."""
    d = _discharge()
    n_gas = d.p_Pa / (I.K_B * d.T_gas_K)
    k = 0.3 / (7 * n_gas * d.dt_s)
    de, n_pts = 1e-2, 10001
    eps = np.arange(n_pts) * de
    cols_i = [np.where(eps >= 50.0, 5 * k, k), np.full(n_pts, 2 * k)]
    z = np.zeros(n_pts)
    gas = _rates_gas(39.948 * I.AMU, de, n_pts, [z, z, z], cols_i, (1e9,), 2e9)
    n = 600_000
    rng = np.random.default_rng(22)
    ions = I.speed_state(rng, n, d.n_cells, math.sqrt(2 * I.E_CH * 10.0 / (39.948 * I.AMU)))  # 5 eV c.m.
    o = _run_once(gas, d, i_state=ions)
    c = o.counters()
    P = -math.expm1(-7 * k * n_gas * d.dt_s)
    assert _within(c["candidates"][1], n, P)
    assert _within(c["collisions_i"][0], n, P / 7), c["collisions_i"]
    assert _within(c["collisions_i"][1], n, 2 * P / 7), c["collisions_i"]
    assert c["collisions_e"] == [0, 0, 0, 0]


@pytest.mark.parametrize("eps_eV", [10.25, 10.5, 10.75, 17.2, 23.9])
def test_rate_interpolation_on_a_coarse_grid(eps_eV):
    """sigma v tabulated every 1 eV with strongly different neighbouring rows: a particle at
    eps = (i + f) eV collides with probability P_null ((1 - f) r_i + f r_{i+1}) / nu_max, the linear
    interpolation of rows i and i + 1 (brute force over 2e5 particles; a neighbouring row pair or
    swapped weights moves the rate by 25 % or more)."""
    d = _discharge()
    n_gas = d.p_Pa / (I.K_B * d.T_gas_K)
    de, n_pts = 1.0, 41
    a = 1.0 + 3.0 * ((np.arange(n_pts) * 7) % 5) / 4.0  # row pattern 1, 3.25, 2.5, 1.75, 4, ...
    k0 = 0.6 / (a.max() * n_gas * d.dt_s)
    r = k0 * a
    z = np.zeros(n_pts)
    gas = _rates_gas(HEAVY, de, n_pts, [r, z, z], [z, z], (1e9,), 2e9)
    i, f = int(eps_eV // de), eps_eV / de - int(eps_eV // de)
    expect = (1 - f) * r[i] + f * r[i + 1]
    for other in ((1 - f) * r[i + 1] + f * r[i + 2], (1 - f) * r[i - 1] + f * r[i], f * r[i] + (1 - f) * r[i + 1]):
        assert abs(other / expect - 1) > 0.05 or abs(f - 0.5) < 1e-9  # the pin can tell them apart
    n = 200_000
    rng = np.random.default_rng(int(eps_eV * 100))
    e = I.speed_state(rng, n, d.n_cells, math.sqrt(2 * I.E_CH * eps_eV / I.M_E))
    o = _run_once(gas, d, e_state=e)
    P = -math.expm1(-k0 * a.max() * n_gas * d.dt_s)
    p = P * expect / r.max()
    got = o.counters()["collisions_e"][0]
    assert _within(got, n, p), (got, n * p)
    for wrong in ((1 - f) * r[i + 1] + f * r[i + 2], (1 - f) * r[i - 1] + f * r[i]):
        assert not _within(got, n, P * wrong / r.max())


def _ks_uniform_sphere(u, label):
    u = u / np.linalg.norm(u, axis=1)[:, None]
    assert stats.kstest(u[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-4, label
    az = np.arctan2(u[:, 1], u[:, 0])
    assert stats.kstest(az, "uniform", args=(-math.pi, 2 * math.pi)).pvalue > 1e-4, label


def test_ion_isotropic_scattering_is_isotropic_in_the_centre_of_mass_frame():
    """Equal-mass isotropic scattering: the post-collision relative velocity g' is uniform on the
    sphere, and so is its angle to the incoming relative velocity (cos chi uniform on [-1, 1]).
    A direction drawn in the lab frame instead leaves cos chi biased towards forward scattering."""
    M = 39.948 * I.AMU
    n_pts, de = 4001, 1e-2
    z = np.zeros(n_pts)
    g = np.sqrt(4 * I.E_CH * np.maximum(np.arange(n_pts) * de, 1e-9) / M)
    gas = X.GasTables("iso", M, (1e9,), 2e9, de, np.stack([z, z, z], 1), np.ascontiguousarray(np.stack([1e-8 / g, z], 1)))
    d = I.discharge(n_cells=64, p_Pa=1000.0, seed=99)
    n = 20000
    rng = np.random.default_rng(31)
    st = I.energy_state(rng, n, 64, 0.5, 20.0, M)
    st["c"][:] = 32
    o = _run_once(gas, d, i_state=st)
    assert o.counters()["collisions_i"][0] == n
    out = o.get_state(1)
    sig_n = math.sqrt(I.K_B * 300.0 / M)
    vn = np.zeros((n, 3))
    for k in range(n):  # the atom's velocity from its stream (call 1 of the ion)
        q = O.philox([k, 0, (1 << 8) | 1, 0], [99, 0])
        a0, a1 = O.box_muller(O.uniform(q[0]), O.uniform(q[1]))
        a2, _ = O.box_muller(O.uniform(q[2]), O.uniform(q[3]))
        vn[k] = sig_n * np.array([a0, a1, a2])
    v = np.stack([st["vx"], st["vy"], st["vz"]], 1)
    vp = np.stack([out["vx"], out["vy"], out["vz"]], 1)
    gin = v - vn
    gout = vp - (v + vn - vp)  # ion minus atom after the collision
    assert np.allclose(np.linalg.norm(gout, axis=1), np.linalg.norm(gin, axis=1), rtol=1e-12)
    _ks_uniform_sphere(gout, "g'")
    cchi = np.sum(gin * gout, 1) / (np.linalg.norm(gin, axis=1) * np.linalg.norm(gout, axis=1))
    assert stats.kstest(cchi, "uniform", args=(-1, 2)).pvalue > 1e-4


def _forced(col, eps_th, n_exc=1):
    n_pts, de = 40001, 5e-3
    eps = np.arange(n_pts) * de
    v = np.sqrt(2 * I.E_CH * np.maximum(eps, 1e-9) / I.M_E)
    cols = [np.zeros(n_pts) for _ in range(2 + n_exc)]
    cols[col] = np.where(eps > eps_th, 1e-10 / v, 0.0)
    z = np.zeros(n_pts)
    exc = (eps_th,) if col == 1 else (1e9,)
    iz = eps_th if col == 2 + n_exc - 1 else 2e9
    return X.GasTables("forced", 4.002602 * I.AMU, exc, iz, de, np.ascontiguousarray(np.stack(cols, 1)),
                       np.ascontiguousarray(np.stack([z, z], 1)))


def test_excitation_and_ionization_directions_are_isotropic():
    """After an excitation the electron's direction is uniform on the sphere and independent of the
    incoming one; after an ionization both electrons' directions are, independently of each other."""
    rng = np.random.default_rng(32)
    n = 20000
    st = I.energy_state(rng, n, 64, 30.0, 150.0, I.M_E)
    st["c"][:] = 32
    v = np.stack([st["vx"], st["vy"], st["vz"]], 1)
    o = _run_once(_forced(1, 19.8), I.discharge(n_cells=64), e_state=st)
    assert o.counters()["collisions_e"][1] == n
    out = o.get_state(0)
    vp = np.stack([out["vx"], out["vy"], out["vz"]], 1)
    _ks_uniform_sphere(vp, "excitation")
    c = np.sum(v * vp, 1) / (np.linalg.norm(v, axis=1) * np.linalg.norm(vp, axis=1))
    assert stats.kstest(c, "uniform", args=(-1, 2)).pvalue > 1e-4
    o = _run_once(_forced(2, 24.6), I.discharge(n_cells=64), e_state=st)
    assert o.counters()["collisions_e"][3] == n
    out = o.get_state(0)
    w = np.stack([out["vx"], out["vy"], out["vz"]], 1)
    a, b = w[:n], w[n:]  # the scattered electrons, then the ejected ones in parent order
    _ks_uniform_sphere(a, "ionization, scattered")
    _ks_uniform_sphere(b, "ionization, ejected")
    c = np.sum(a * b, 1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1))
    assert stats.kstest(c, "uniform", args=(-1, 2)).pvalue > 1e-4


def test_secondary_electron_velocity_law():
    """Added option (not in the paper): an emitted electron leaves the wall with the flux-weighted
    half-Maxwellian of kT = 2 eV in its normal component, P(v_n <= v) = 1 - exp(-v^2 / (2 s^2)),
    s^2 = kT / m_e (a Rayleigh law), Maxwellian tangential components of the same s, the three
    independent, mean energy 2 kT."""
    M = 4.002602 * I.AMU
    d = I.discharge(n_cells=32, gamma_see=0.5, steps_per_period=400)
    n_pts, de = 101, 1.0
    z = np.zeros(n_pts)
    gas = X.GasTables("none", M, (1e9,), 2e9, de, np.stack([z, z, z], 1), np.stack([z, z], 1))
    n = 60000
    rng = np.random.default_rng(33)
    dx = d.gap_m / 32
    st = {"c": np.where(np.arange(n) % 2 == 0, 0, 31).astype(np.int32), "f": rng.uniform(0, 1, n),
          "vx": np.zeros(n), "vy": np.zeros(n), "vz": np.zeros(n)}
    st["vz"] = np.where(st["c"] == 0, -1.0, 1.0) * 3 * dx / d.dt_s
    o = _run_once(gas, d, i_state=st)
    k = o.counters()["see_emitted"]
    assert _within(k, n, 0.5)
    born = {kk: vv[1:] for kk, vv in o.get_state(0).items()}
    s = math.sqrt(I.E_CH * 2.0 / I.M_E)
    vnorm = np.abs(born["vz"])
    assert stats.kstest(vnorm, lambda x: 1 - np.exp(-x ** 2 / (2 * s * s))).pvalue > 1e-4
    # the normal speed is not a half-normal of the same s (what a plain Maxwellian would give)
    assert stats.kstest(vnorm, "halfnorm", args=(0, s)).pvalue < 1e-6
    for key in ("vx", "vy"):
        assert stats.kstest(born[key] / s, "norm").pvalue > 1e-4
    # the three components are independent (|r| ~ 1 / sqrt(k) between any two) and a flux member's
    # energy is Gamma(3, kT) distributed: mean 2 kT, variance 3 (kT)^2
    for a, b in (("vx", "vy"), ("vx", "vz"), ("vy", "vz")):
        x, y = born[a], (np.abs(born[b]) if b == "vz" else born[b])
        assert abs(np.corrcoef(x, y)[0, 1]) < 5 / math.sqrt(k)
    eps = 0.5 * I.M_E * (born["vx"] ** 2 + born["vy"] ** 2 + born["vz"] ** 2) / I.E_CH
    assert abs(eps.mean() - 4.0) <= 5 * math.sqrt(3 * 4.0 / k)
