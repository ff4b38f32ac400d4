"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test states the passage of arXiv:1608.04601 it checks, and the fact
(closed form, invariant, brute force, published vector) that pins it. All run
on the CPU with the FP64 build unless stated.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import inputs as I
from oracle import oracle as O
from paper_1608_04601_gb300 import xsections as X

HERE = os.path.dirname(os.path.abspath(__file__))


def _gas_custom(mass, n_pts, de, sig_e_cols, sig_i_cols, eps_exc=(1e9,), eps_iz=2e9):
    return X.GasTables("custom", mass, tuple(eps_exc), eps_iz, de, np.ascontiguousarray(np.stack(sig_e_cols, 1)),
                       np.ascontiguousarray(np.stack(sig_i_cols, 1)))


# --------------------------------------------------------------------------- RNG and own functions

def test_philox_known_answers():
    """Philox4x32-10 (Salmon et al. SC'11) against the published known-answer vectors."""
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_uniform_exact_and_open():
    assert O.uniform(0) == 2.0 ** -24
    assert O.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    rng = np.random.default_rng(0)
    for x in rng.integers(0, 2 ** 32, 2000):
        assert O.uniform(int(x)) == ((int(x) >> 9) + 0.5) * 2.0 ** -23


def _ulp32(x):
    x = np.abs(np.float32(x))
    return float(np.spacing(x)) if x > 0 else 2.0 ** -149


def test_own_log_against_libm():
    """Own log agrees with the correctly rounded log to 3 ulp over the whole Box-Muller range."""
    rng = np.random.default_rng(11)
    xs = np.concatenate([(np.arange(1 << 12) + 0.5) * 2.0 ** -12, rng.uniform(2 ** -25, 1, 4000),
                         2.0 ** rng.uniform(-25, 30, 2000), [2 ** -25, 1 - 2 ** -24, 0.70710677, 1.4142135]])
    worst = 0.0
    for x in xs.astype(np.float32):
        got = O.logf(float(x))
        ref = math.log(float(x))
        worst = max(worst, abs(got - ref) / _ulp32(ref))
    assert worst <= 3.0, worst


def test_own_sincospi_against_libm():
    """Own sin(pi y), cos(pi y) agree with libm to 2^-22 absolute on [0, 2]."""
    ys = np.concatenate([np.linspace(0, 2, 4001), np.random.default_rng(3).uniform(0, 2, 3000)]).astype(np.float32)
    for y in ys:
        s, c = O.sincospif(float(y))
        assert abs(s - math.sin(math.pi * float(y))) <= 2 ** -22
        assert abs(c - math.cos(math.pi * float(y))) <= 2 ** -22
        assert s * s + c * c == pytest.approx(1.0, abs=4e-7)


def test_box_muller_and_isotropy_statistics():
    n = 40000
    words = np.array([O.philox([k, 7, 0, 0], [1, 2]) for k in range(n)], dtype=np.uint64)
    u = ((words >> 9).astype(np.float64) + 0.5) * 2.0 ** -23
    n0 = np.empty(n)
    n1 = np.empty(n)
    d = np.empty((n, 3))
    for k in range(n):
        n0[k], n1[k] = O.box_muller(u[k, 0], u[k, 1])
        d[k] = O.isotropic(u[k, 2], u[k, 3])
    assert stats.kstest(n0, "norm").pvalue > 1e-4
    assert stats.kstest(n1, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(n0, n1)[0, 1]) < 5 / math.sqrt(n)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
    assert stats.kstest(d[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-4
    az = np.arctan2(d[:, 1], d[:, 0])
    assert stats.kstest(az, "uniform", args=(-math.pi, 2 * math.pi)).pvalue > 1e-4
    assert np.all(np.abs(d.mean(0)) < 5 / math.sqrt(3 * n))


# --------------------------------------------------------------------------- field solve

def test_poisson_uniform_charge_closed_form():
    """Eq. (poisson) with uniform rho0 and phi(0) = V0, phi(d) = VN:
    phi = V0 + (VN - V0) z/d + rho0 z(d-z)/(2 eps0). The 3-point stencil is exact for quadratics, so
    the nodes agree to round-off; E = -phi' is linear and the central / half-cell wall formulas
    reproduce it exactly. (The discharge grounds z = d; the solver also takes a nonzero VN.)"""
    for N, d, V0, VN, rho0 in [(128, 0.025, 200.0, 0.0, 3e-5), (2048, 0.05, -500.0, 0.0, -1e-4),
                               (7, 0.01, 13.0, 0.0, 2e-6), (64, 0.02, 100.0, -40.0, 5e-6), (9, 0.01, 0.0, 25.0, 0.0)]:
        dx = d / N
        z = np.arange(N + 1) * dx
        phi, E = O.poisson(np.full(N + 1, rho0), dx, V0, VN)
        phi_ref = V0 + (VN - V0) * z / d + rho0 * z * (d - z) / (2 * I.EPS0)
        E_ref = (V0 - VN) / d - rho0 * (d - 2 * z) / (2 * I.EPS0)
        scale = abs(V0) + abs(VN) + abs(rho0) * d * d / I.EPS0
        assert np.max(np.abs(phi - phi_ref)) <= 1e-12 * scale * N
        assert np.max(np.abs(E - E_ref)) <= 1e-11 * ((abs(V0) + abs(VN)) / d + abs(rho0) * d / I.EPS0) * N


def test_poisson_random_charge_dense_solve():
    rng = np.random.default_rng(5)
    N, dx, V = 300, 1e-4, 77.0
    rho = rng.normal(0, 1e-5, N + 1)
    phi, E = O.poisson(rho, dx, V, 0.0)
    A = np.zeros((N - 1, N - 1))
    b = -rho[1:N] * dx * dx / I.EPS0
    for k in range(N - 1):
        A[k, k] = -2
        if k > 0:
            A[k, k - 1] = 1
        if k < N - 2:
            A[k, k + 1] = 1
    b[0] -= V
    ref = np.linalg.solve(A, b)
    assert np.max(np.abs(phi[1:N] - ref)) <= 1e-12 * np.max(np.abs(ref))
    # Gauss's law over the half cells and the interior central difference
    assert E[0] == pytest.approx((phi[0] - phi[1]) / dx - rho[0] * dx / (2 * I.EPS0), rel=1e-14)
    assert E[N] == pytest.approx((phi[N - 1] - phi[N]) / dx + rho[N] * dx / (2 * I.EPS0), rel=1e-14)
    assert np.allclose(E[1:N], (phi[:N - 1] - phi[2:]) / (2 * dx), rtol=1e-14, atol=0)


# --------------------------------------------------------------------------- CIC, gather, push

def _no_collision_gas(mass=4.002602 * I.AMU):
    n_pts, de = 101, 1.0
    z = np.zeros(n_pts)
    return _gas_custom(mass, n_pts, de, [z, z, z], [z, z])


def test_deposit_conserves_charge_and_node_cases():
    """Cloud-in-cell (section 'PIC/MCC simulation procedure'): weight 1-f to node c, f to node c+1;
    the fixed-point total is exactly 2^32 per particle, and a particle on a node puts all of it there."""
    N = 32
    o = O.Oracle(_no_collision_gas(), I.discharge(n_cells=N, dt_s=None) if False else I.discharge(n_cells=N),
                 "f64", load=False)
    rng = np.random.default_rng(1)
    st = I.maxwell_state(rng, 5000, N, 0.0)
    st["f"][:10] = 0.0
    st["c"][:10] = 5
    st["f"][10] = 0.25
    st["c"][10] = 9
    o.set_state(0, st)
    o.set_state(1, I.maxwell_state(rng, 10, N, 0.0))
    o.set_field(np.zeros(N + 1))
    o.sweep()
    De = o.get_deposit(0)
    assert De.sum() == 5000 * 2 ** 32
    ref = np.zeros(N + 1, np.int64)
    for c, f in zip(st["c"], st["f"]):
        F = int(np.rint(f * 2.0 ** 32))
        ref[c] += 2 ** 32 - F
        ref[c + 1] += F
    assert np.array_equal(De, ref)
    one = O.Oracle(_no_collision_gas(), I.discharge(n_cells=N), "f64", load=False)
    one.set_state(0, {"c": [9], "f": [0.25], "vx": [0.0], "vy": [0.0], "vz": [0.0]})
    one.set_state(1, {"c": [5], "f": [0.0], "vx": [0.0], "vy": [0.0], "vz": [0.0]})
    one.set_field(np.zeros(N + 1))
    one.sweep()
    d0, d1 = one.get_deposit(0), one.get_deposit(1)
    assert d0[9] == 3 * 2 ** 30 and d0[10] == 2 ** 30 and d0.sum() == 2 ** 32
    assert d1[5] == 2 ** 32 and d1.sum() == 2 ** 32


def test_gather_linear_field_and_kick_sign():
    """Linear interpolation of a linear node field is exact; one sweep from rest kicks v_z by
    (q/m) E(x) dt for each species (electrons against the field, ions along it)."""
    N, gap, dt = 16, 0.016, 1e-11
    d = I.discharge(n_cells=N, gap_m=gap, steps_per_period=int(round(1 / (13.56e6 * dt))))
    dt = d.dt_s
    o = O.Oracle(_no_collision_gas(), d, "f64", load=False)
    z = np.arange(N + 1) * (gap / N)
    E = 1000.0 + 2.5e5 * z
    o.set_field(E)
    rng = np.random.default_rng(2)
    n = 200
    st = {"c": rng.integers(2, N - 2, n).astype(np.int32), "f": rng.uniform(0, 1, n),
          "vx": np.zeros(n), "vy": np.zeros(n), "vz": np.zeros(n)}
    o.set_state(0, st)
    o.set_state(1, st)
    o.sweep()
    zp = (st["c"] + st["f"]) * (gap / N)
    Ep = 1000.0 + 2.5e5 * zp
    for sp, qm in ((0, -I.E_CH / I.M_E), (1, I.E_CH / (4.002602 * I.AMU))):
        out = o.get_state(sp)
        assert out["c"].size == n
        assert np.allclose(out["vz"], qm * Ep * dt, rtol=1e-12, atol=0)


def test_field_free_push_is_exact_and_conserves_energy():
    """No field, no collisions: x_n = x_0 + v t exactly to round-off, speeds unchanged (velocity Verlet)."""
    N, gap = 64, 0.05
    d = I.discharge(n_cells=N, gap_m=gap)
    o = O.Oracle(_no_collision_gas(), d, "f64", load=False)
    o.set_field(np.zeros(N + 1))
    rng = np.random.default_rng(3)
    n = 300
    st = {"c": np.full(n, N // 2, np.int32), "f": rng.uniform(0, 1, n), "vx": rng.normal(0, 1e5, n),
          "vy": rng.normal(0, 1e5, n), "vz": rng.uniform(-1, 1, n) * 0.3 * (gap / 2) / (20 * d.dt_s)}
    o.set_state(0, st)
    o.set_state(1, {k: v[:1] for k, v in st.items()})
    for k in range(20):
        o.step_index = k
        o.sweep()
    out = o.get_state(0)
    dx = gap / N
    z = (out["c"] + out["f"]) * dx
    z_ref = (st["c"] + st["f"]) * dx + st["vz"] * 20 * d.dt_s
    assert np.max(np.abs(z - z_ref)) <= 1e-12 * gap
    assert np.array_equal(out["vx"], st["vx"]) and np.array_equal(out["vz"], st["vz"])


def test_constant_field_parabola():
    """Velocity Verlet integrates constant acceleration exactly: z = z0 + v0 t + a t^2 / 2.
    The stored velocity is v0 - a dt / 2 (the half back-kick of the load)."""
    N, gap = 64, 0.05
    d = I.discharge(n_cells=N, gap_m=gap)
    dt = d.dt_s
    o = O.Oracle(_no_collision_gas(), d, "f64", load=False)
    E0 = -350.0
    o.set_field(np.full(N + 1, E0))
    a = (-I.E_CH / I.M_E) * E0
    rng = np.random.default_rng(4)
    n, steps = 100, 30
    v0 = rng.uniform(-1, 1, n) * 2e5
    st = {"c": np.full(n, 20, np.int32), "f": rng.uniform(0, 1, n), "vx": np.zeros(n), "vy": np.zeros(n),
          "vz": v0 - 0.5 * a * dt}
    o.set_state(0, st)
    o.set_state(1, {k: v[:1] for k, v in st.items()})
    for k in range(steps):
        o.step_index = k
        o.sweep()
    out = o.get_state(0)
    assert out["c"].size == n
    t = steps * dt
    dx = gap / N
    z = (out["c"] + out["f"]) * dx
    z_ref = (st["c"] + st["f"]) * dx + v0 * t + 0.5 * a * t * t
    assert np.max(np.abs(z - z_ref)) <= 1e-11 * gap


def test_harmonic_oscillation_in_uniform_background_charge():
    """Uniform fixed positive charge n0 e between grounded plates (V = 0): the node field is exactly
    E = e n0 (z - d/2) / eps0 (the 3-point stencil is exact for the quadratic potential) and the
    CIC gather of a linear field is exact, so a test electron released at rest at d/2 + A is a
    harmonic oscillator of omega^2 = e^2 n0 / (m_e eps0). Velocity Verlet then gives exactly
    z_n - d/2 = A cos(w n dt) with cos(w dt) = 1 - (omega dt)^2 / 2 (the numerical frequency
    (2/dt) arcsin(omega dt / 2)). Pins gather, both half kicks, drift and the Poisson solve
    together: a wrong kick factor, sign or kick placement fails it."""
    N, gap, n0 = 64, 0.025, 8e14
    m_per_cell = 16
    d = I.discharge(n_cells=N, gap_m=gap, n_e0=10 ** 15, n_i0=N * m_per_cell, n_init_m3=n0, V_rf_V=0.0)
    dt, dx = d.dt_s, gap / N
    o = O.Oracle(_no_collision_gas(mass=1.0), d, "f64", load=False)   # ions of 1 kg: they stay put
    k = np.arange(N * m_per_cell)
    ions = {"c": (k // m_per_cell).astype(np.int32), "f": ((k % m_per_cell) + 0.5) / m_per_cell,
            "vx": np.zeros(k.size), "vy": np.zeros(k.size), "vz": np.zeros(k.size)}
    A = 0.2 * gap
    z0 = gap / 2 + A
    c0 = int(z0 // dx)
    e = {"c": np.array([c0], np.int32), "f": np.array([z0 / dx - c0]), "vx": np.zeros(1), "vy": np.zeros(1),
         "vz": np.zeros(1)}
    # the oracle deposits the ions (field-free sweep) and solves for their field
    o.set_field(np.zeros(N + 1))
    o.set_state(1, ions)
    o.set_state(0, e)
    o.sweep()
    o.solve()
    eps0 = 8.8541878128e-12
    E_z0 = I.E_CH * n0 * (z0 - gap / 2) / eps0
    assert np.allclose(o.get_field64(), I.E_CH * n0 * (np.arange(N + 1) * dx - gap / 2) / eps0, rtol=1e-9,
                       atol=1e-9 * abs(E_z0))
    # released at rest: the stored velocity is v_0 - (q/m) E(z0) dt / 2
    e["vz"] = np.array([-(-I.E_CH / I.M_E) * E_z0 * dt / 2])
    o.set_state(0, e)
    omega = math.sqrt(I.E_CH ** 2 * n0 / (I.M_E * eps0))
    assert 0.1 < omega * dt < 1.0
    w = math.acos(1 - 0.5 * (omega * dt) ** 2) / dt
    for n in range(1, 201):
        o.step(1)
        st = o.get_state(0)
        z = (st["c"][0] + st["f"][0]) * dx
        assert abs((z - gap / 2) - A * math.cos(w * n * dt)) <= 1e-9 * A, n


# --------------------------------------------------------------------------- MCC

def test_brute_force_collision_probability_electrons():
    """Null-collision method (section 'PIC/MCC simulation procedure'): a particle is a candidate with
    P_null = 1 - exp(-nu_max dt) and collides for real with nu(eps)/nu_max, so
    P = P_null nu/nu_max, within nu dt * nu_max dt / 2 of the exact 1 - exp(-n sigma v dt)."""
    sig = 1e-19
    g = X.constant_sigma(sigma_el=sig, eps_max_eV=100.0, de_eV=1e-2)
    d = I.discharge(n_cells=64, p_Pa=30.0, steps_per_period=int(1 / (13.56e6 * 7.4e-11)))
    o = O.Oracle(g, d, "f64", load=False)
    o.set_field(np.zeros(65))
    n = 1_000_000
    eps = 10.0
    v = math.sqrt(2 * I.E_CH * eps / I.M_E)
    rng = np.random.default_rng(6)
    o.set_state(0, I.speed_state(rng, n, 64, v))
    o.set_state(1, I.speed_state(rng, 1, 64, 0.0))
    o.sweep()
    k = o.counters()["collisions_e"][0]
    n_gas = d.p_Pa / (I.K_B * d.T_gas_K)
    nu = n_gas * sig * v
    vmax = math.sqrt(2 * I.E_CH * 100.0 / I.M_E)
    numax = n_gas * sig * vmax
    dt = d.dt_s
    p_alg = -math.expm1(-numax * dt) * nu / numax
    p_exact = -math.expm1(-nu * dt)
    assert abs(p_alg - p_exact) <= nu * dt * numax * dt / 2
    se = math.sqrt(p_alg * (1 - p_alg) / n)
    assert abs(k / n - p_alg) <= 5 * se
    assert abs(k / n - p_exact) <= 5 * se + nu * dt * numax * dt / 2


def test_collision_rate_above_the_table_is_the_last_row():
    """Above the table's last energy the last row is used: with sigma_el = 1e-20 m^2 everywhere but
    1e-19 at the last point (100 eV), an electron at 150 eV has the last row's rate sigma v(100 eV),
    which is the table's maximum, so it collides with the candidate probability itself,
    P = 1 - exp(-nu_max dt) (the row before would give a tenth of that)."""
    n_pts, de = 101, 1.0
    sig = np.full(n_pts, 1e-20)
    sig[-1] = 1e-19
    z = np.zeros(n_pts)
    g = _gas_custom(4.002602 * I.AMU, n_pts, de, [sig, z, z], [z, z])
    d = I.discharge(n_cells=64, p_Pa=30.0, steps_per_period=int(1 / (13.56e6 * 7.4e-11)))
    o = O.Oracle(g, d, "f64", load=False)
    o.set_field(np.zeros(65))
    n = 200_000
    v = math.sqrt(2 * I.E_CH * 150.0 / I.M_E)
    rng = np.random.default_rng(8)
    o.set_state(0, I.speed_state(rng, n, 64, v))
    o.set_state(1, I.speed_state(rng, 1, 64, 0.0))
    o.sweep()
    k = o.counters()["collisions_e"][0]
    n_gas = d.p_Pa / (I.K_B * d.T_gas_K)
    numax = n_gas * 1e-19 * math.sqrt(2 * I.E_CH * 100.0 / I.M_E)
    p = -math.expm1(-numax * d.dt_s)
    assert 0.05 < p < 0.6
    assert abs(k / n - p) <= 5 * math.sqrt(p * (1 - p) / n)


def test_brute_force_collision_probability_ions_centre_of_mass():
    """Ion tables are indexed by the centre-of-mass energy eps_cm = M g^2 / 4 (equal masses; helium
    caption of Fig. 'Cross_He'): with constant sigma the collision probability is 1 - exp(-n sigma g dt)."""
    M = 4.002602 * I.AMU
    sig = 3e-19
    n_pts, de = 20001, 1e-2
    z = np.zeros(n_pts)
    g = _gas_custom(M, n_pts, de, [z, z, z], [np.full(n_pts, sig), z])
    d = I.discharge(n_cells=64, p_Pa=30.0, steps_per_period=int(1 / (13.56e6 * 1e-9)))
    o = O.Oracle(g, d, "f64", load=False)
    o.set_field(np.zeros(65))
    n = 400_000
    v = 1.0e5
    rng = np.random.default_rng(7)
    o.set_state(1, I.speed_state(rng, n, 64, v))
    o.set_state(0, I.speed_state(rng, 1, 64, 0.0))
    o.sweep()
    k = o.counters()["collisions_i"][0]
    n_gas = d.p_Pa / (I.K_B * d.T_gas_K)
    dt = d.dt_s
    gmax = math.sqrt(4 * I.E_CH * (n_pts - 1) * de / M)
    numax = n_gas * sig * gmax
    p_alg = -math.expm1(-numax * dt) * (v / gmax)   # thermal target motion: (790/1e5)^2 correction
    se = math.sqrt(p_alg * (1 - p_alg) / n)
    assert abs(k / n - p_alg) <= 5 * se + 1e-4 * p_alg
    # a lab-frame lookup would be off by sqrt(2)
    assert abs(k / n - p_alg * math.sqrt(2)) > 50 * se


def test_exponential_free_flight():
    """Constant nu (sigma proportional to 1/v): the first real collision after t is exp(-nu t)
    distributed at the step times (the null-collision candidates are Bernoulli(P_null) per step)."""
    M = 1e6 * I.AMU
    k_el = 2e-14
    g = X.constant_nu(k_el, M, eps_max_eV=10.0, de_eV=1e-3)
    d = I.discharge(n_cells=64, p_Pa=30.0, gap_m=1.0, steps_per_period=int(1 / (13.56e6 * 2e-10)))
    dt = d.dt_s
    o = O.Oracle(g, d, "f64", load=False)
    o.set_field(np.zeros(65))
    n, steps = 50_000, 60
    rng = np.random.default_rng(8)
    st = I.speed_state(rng, n, 64, 1e5)   # 28 meV: well inside the tabulated range
    o.set_state(0, st)
    o.set_state(1, I.speed_state(rng, 1, 64, 0.0))
    first = np.full(n, -1)
    prev = st["vx"].copy()
    for k in range(steps):
        o.step_index = k
        o.sweep()
        cur = o.get_state(0)["vx"]
        hit = (cur != prev) & (first < 0)
        first[hit] = k + 1
        prev = cur.copy()
    assert o.count(0) == n
    n_gas = d.p_Pa / (I.K_B * d.T_gas_K)
    nu = n_gas * k_el
    t_grid = np.arange(1, steps + 1) * dt
    cdf_ref = 1 - np.exp(-nu * t_grid)
    emp = np.array([(first[first > 0] <= j).sum() for j in range(1, steps + 1)]) / n
    eps = math.sqrt(math.log(2 / 1e-6) / (2 * n))  # DKW bound
    assert np.max(np.abs(emp - cdf_ref)) <= eps


def _forced_gas(mass, col, k, eps_th=0.0, n_exc=1):
    """Every candidate takes process `col` (sigma*v = k for eps > eps_th); nu_max dt >> 1 makes every
    particle a candidate."""
    n_pts, de = 40001, 5e-3
    eps = np.arange(n_pts) * de
    v = np.sqrt(2 * I.E_CH * np.maximum(eps, 1e-9) / I.M_E)
    cols = [np.zeros(n_pts) for _ in range(2 + n_exc)]
    cols[col] = np.where(eps > eps_th, k / v, 0.0)
    z = np.zeros(n_pts)
    exc = (eps_th,) if col == 1 else (1e9,)
    iz = eps_th if col == 2 + n_exc - 1 else 2e9
    return _gas_custom(mass, n_pts, de, cols, [z, z], eps_exc=exc, eps_iz=iz)


def test_elastic_collision_conserves_energy_and_momentum():
    """Elastic electron-atom collision as two-body kinematics, target at rest: with the recoil
    V' = (m/M)(v - v'), kinetic energy and momentum are conserved to round-off, and the speed in the
    centre-of-mass frame is unchanged."""
    M = 4.002602 * I.AMU
    g = _forced_gas(M, 0, 1e-10)
    d = I.discharge(n_cells=64, p_Pa=30.0, steps_per_period=400)
    o = O.Oracle(g, d, "f64", load=False)
    o.set_field(np.zeros(65))
    rng = np.random.default_rng(9)
    n = 20000
    st = I.energy_state(rng, n, 64, 1.0, 150.0, I.M_E)
    st["c"][:] = 32
    o.set_state(0, st)
    o.set_state(1, I.speed_state(rng, 1, 64, 0.0))
    o.sweep()
    assert o.counters()["collisions_e"][0] == n
    out = o.get_state(0)
    v = np.stack([st["vx"], st["vy"], st["vz"]], 1)
    vp = np.stack([out["vx"], out["vy"], out["vz"]], 1)
    Vp = (I.M_E / M) * (v - vp)
    ke0 = 0.5 * I.M_E * (v ** 2).sum(1)
    ke1 = 0.5 * I.M_E * (vp ** 2).sum(1) + 0.5 * M * (Vp ** 2).sum(1)
    assert np.max(np.abs(ke1 - ke0) / ke0) < 1e-12
    beta = I.M_E / (I.M_E + M)
    vcm = beta * v
    assert np.allclose(np.linalg.norm(vp - vcm, axis=1), (1 - beta) * np.linalg.norm(v, axis=1), rtol=1e-13)
    # isotropic scattering (section 'PIC/MCC simulation procedure'): directions uniform on the sphere
    u = (vp - vcm) / np.linalg.norm(vp - vcm, axis=1)[:, None]
    assert stats.kstest(u[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-4
    assert np.all(np.abs(u.mean(0)) < 5 / math.sqrt(3 * n))


def test_excitation_loses_exactly_the_threshold():
    M = 4.002602 * I.AMU
    eth = 19.8
    g = _forced_gas(M, 1, 1e-10, eps_th=eth)
    o = O.Oracle(g, I.discharge(n_cells=64), "f64", load=False)
    o.set_field(np.zeros(65))
    rng = np.random.default_rng(10)
    n = 10000
    st = I.energy_state(rng, n, 64, eth + 0.5, 150.0, I.M_E)
    st["c"][:] = 32
    o.set_state(0, st)
    o.set_state(1, I.speed_state(rng, 1, 64, 0.0))
    o.sweep()
    assert o.counters()["collisions_e"][1] == n
    out = o.get_state(0)
    e0 = 0.5 * I.M_E * (st["vx"] ** 2 + st["vy"] ** 2 + st["vz"] ** 2) / I.E_CH
    e1 = 0.5 * I.M_E * (out["vx"] ** 2 + out["vy"] ** 2 + out["vz"] ** 2) / I.E_CH
    assert np.max(np.abs((e0 - e1) - eth)) < 1e-11 * np.max(e0)


def test_ionization_shares_remaining_energy_equally():
    """Ionization (section 'PIC/MCC simulation procedure'): the energy left after the threshold is
    split equally between the two electrons; one ion is born per event, at the parent's position."""
    M = 4.002602 * I.AMU
    eiz = 24.6
    g = _forced_gas(M, 2, 1e-10, eps_th=eiz)
    o = O.Oracle(g, I.discharge(n_cells=64), "f64", load=False)
    o.set_field(np.zeros(65))
    rng = np.random.default_rng(12)
    n = 8000
    st = I.energy_state(rng, n, 64, eiz + 1.0, 200.0, I.M_E)
    st["c"][:] = 32
    o.set_state(0, st)
    o.set_state(1, I.speed_state(rng, 1, 64, 0.0))
    o.sweep()
    assert o.counters()["collisions_e"][3] == n
    out = o.get_state(0)
    assert out["c"].size == 2 * n
    e0 = 0.5 * I.M_E * (st["vx"] ** 2 + st["vy"] ** 2 + st["vz"] ** 2) / I.E_CH
    e = 0.5 * I.M_E * (out["vx"] ** 2 + out["vy"] ** 2 + out["vz"] ** 2) / I.E_CH
    e1, e2 = e[:n], e[n:]         # survivors in input order, then the secondaries in parent order
    assert np.max(np.abs(e1 + e2 - (e0 - eiz))) < 1e-11 * np.max(e0)
    assert np.max(np.abs(e1 - e2)) < 1e-11 * np.max(e0)
    ions = o.get_state(1)
    assert ions["c"].size == 1 + n
    born = {k: v[1:] for k, v in ions.items()}
    # the newborn ion starts at the parent's position and drifts with its thermal velocity
    d = I.discharge(n_cells=64)
    shift = (born["c"] + born["f"]) - (st["c"] + st["f"])
    assert np.allclose(shift, born["vz"] * d.dt_s / (d.gap_m / 64), rtol=1e-6, atol=1e-12)
    sig_n = math.sqrt(I.K_B * 300.0 / M)
    assert abs(np.std(born["vx"]) / sig_n - 1) < 5 / math.sqrt(2 * n)


def test_ion_isotropic_and_backward_elastic_conserve():
    """Ion-atom elastic processes (Table 'reactions'), equal masses, target from the Maxwellian of the
    gas: isotropic scattering conserves momentum and energy of the pair; backward scattering swaps
    the two velocities. The target velocity is recomputed here from its random stream."""
    M = 39.948 * I.AMU
    n_pts, de = 4001, 1e-2
    z = np.zeros(n_pts)
    gr = np.sqrt(4 * I.E_CH * np.maximum(np.arange(n_pts) * de, 1e-9) / M)
    for col in (0, 1):
        si = [z, z]
        si[col] = 1e-8 / gr
        g = _gas_custom(M, n_pts, de, [z, z, z], si)
        d = I.discharge(n_cells=64, p_Pa=1000.0, seed=99)
        o = O.Oracle(g, d, "f64", load=False)
        o.set_field(np.zeros(65))
        rng = np.random.default_rng(13 + col)
        n = 5000
        st = I.energy_state(rng, n, 64, 0.5, 20.0, M)
        st["c"][:] = 32
        o.set_state(1, st)
        o.set_state(0, I.speed_state(rng, 1, 64, 0.0))
        o.sweep()
        assert o.counters()["collisions_i"][col] == n
        out = o.get_state(1)
        sig_n = math.sqrt(I.K_B * 300.0 / M)
        vn = np.zeros((n, 3))
        for k in range(n):
            q = O.philox([k, 0, (1 << 8) | 1, 0], [99, 0])
            a0, a1 = O.box_muller(O.uniform(q[0]), O.uniform(q[1]))
            a2, _ = O.box_muller(O.uniform(q[2]), O.uniform(q[3]))
            vn[k] = sig_n * np.array([a0, a1, a2], dtype=np.float64)
        v = np.stack([st["vx"], st["vy"], st["vz"]], 1)
        vp = np.stack([out["vx"], out["vy"], out["vz"]], 1)
        if col == 1:
            assert np.allclose(vp, vn, rtol=0, atol=1e-9)
        else:
            Vp = v + vn - vp
            e0 = (v ** 2).sum(1) + (vn ** 2).sum(1)
            e1 = (vp ** 2).sum(1) + (Vp ** 2).sum(1)
            assert np.max(np.abs(e1 - e0) / e0) < 1e-12


def test_drift_velocity_maxwell_molecules():
    """Constant nu, isotropic elastic scattering off infinitely heavy atoms, uniform field: the
    scheme's mean stored velocity obeys E[v*] = a dt (2 - p) / (2 p), p = 1 - exp(-nu dt) (one step
    of the recursion), which tends to the Maxwell-molecule drift a / nu = qE/(m nu) as nu dt -> 0."""
    M = 1e7 * I.AMU
    k_el = 1.4e-13
    g = X.constant_nu(k_el, M, eps_max_eV=400.0, de_eV=1e-2)
    d = I.discharge(n_cells=64, gap_m=1.0, p_Pa=30.0, steps_per_period=int(1 / (13.56e6 * 2e-10)))
    dt = d.dt_s
    o = O.Oracle(g, d, "f64", load=False)
    E0 = -1000.0
    o.set_field(np.full(65, E0))
    a = (-I.E_CH / I.M_E) * E0
    rng = np.random.default_rng(14)
    n = 100_000
    o.set_state(0, I.speed_state(rng, n, 64, 3e5))
    o.set_state(1, I.speed_state(rng, 1, 64, 0.0))
    means = []
    for k in range(150):
        o.step_index = k
        o.sweep()
        if k >= 50:
            means.append(o.get_state(0)["vz"].mean())
    assert o.count(0) == n
    n_gas = d.p_Pa / (I.K_B * d.T_gas_K)
    nu = n_gas * k_el
    p = -math.expm1(-nu * dt)
    vd_scheme = a * dt * (2 - p) / (2 * p)
    got = float(np.mean(means))
    assert abs(got / vd_scheme - 1) < 0.01
    assert abs(vd_scheme / (a / nu) - 1) < nu * dt


def test_growth_with_zero_threshold_ionization():
    """Zero-threshold ionization at constant nu, no field: E[N_n] = N_0 (1 + P)^n, P = 1 - exp(-nu dt);
    every ionization adds one ion."""
    M = 4.002602 * I.AMU
    k_iz = 1e-13
    g = X.constant_nu(0.0, M, eps_max_eV=50.0, de_eV=1e-2, k_iz=k_iz)
    d = I.discharge(n_cells=64, gap_m=1.0, p_Pa=30.0, steps_per_period=int(1 / (13.56e6 * 2e-10)))
    o = O.Oracle(g, d, "f64", load=False)
    o.set_field(np.zeros(65))
    rng = np.random.default_rng(15)
    n0, steps = 20000, 8
    o.set_state(0, I.speed_state(rng, n0, 64, 1e6))
    o.set_state(1, I.speed_state(rng, 1, 64, 0.0))
    for k in range(steps):
        o.step_index = k
        o.sweep()
    n_gas = d.p_Pa / (I.K_B * d.T_gas_K)
    P = -math.expm1(-n_gas * k_iz * d.dt_s)
    m = 1 + P
    mean = n0 * m ** steps
    var = n0 * P * (1 - P) * m ** (steps - 1) * (m ** steps - 1) / (m - 1)
    ne = o.count(0)
    assert abs(ne - mean) <= 5 * math.sqrt(var)
    assert o.count(1) - 1 == ne - n0
    assert o.counters()["collisions_e"][3] == ne - n0


# --------------------------------------------------------------------------- walls, load, moments, sort

def test_wall_flux_one_sided_maxwellian():
    """Full absorption at the electrodes: the particle flux onto a wall from a uniform field-free
    Maxwellian is n v_th / 4, v_th = sqrt(8 kT / (pi m)) (the 1/4 v_th term of Eq. 'BCparticles')."""
    N, gap = 64, 0.025
    d = I.discharge(n_cells=N, gap_m=gap)
    o = O.Oracle(_no_collision_gas(), d, "f64", load=False)
    o.set_field(np.zeros(N + 1))
    T = 2.0
    sig = math.sqrt(I.E_CH * T / I.M_E)
    dt = 1e-3 * gap / sig
    d2 = I.discharge(n_cells=N, gap_m=gap, steps_per_period=int(round(1 / (13.56e6 * dt))))
    dt = d2.dt_s
    o = O.Oracle(_no_collision_gas(), d2, "f64", load=False)
    o.set_field(np.zeros(N + 1))
    rng = np.random.default_rng(16)
    n = 2_000_000
    o.set_state(0, I.maxwell_state(rng, n, N, sig))
    o.set_state(1, I.maxwell_state(rng, 1, N, 0.0))
    o.sweep()
    ab = o.counters()["absorbed"][0]
    vth = math.sqrt(8 * I.E_CH * T / (math.pi * I.M_E))
    expect = (n / gap) * vth / 4 * dt
    for side in (0, 1):
        assert abs(ab[side] - expect) <= 5 * math.sqrt(expect) + 1e-3 * expect


def _half_kick(o, d, sp, st):
    """(q/m) E(x, 0) dt / 2 at each particle of species sp (He-like mass for ions), with E the
    oracle's t = 0 node field interpolated linearly: what the load subtracted from v_z."""
    E = o.get_field()
    qm = -I.E_CH / I.M_E if sp == 0 else I.E_CH / (4.002602 * I.AMU)
    Ez = E[st["c"]] + st["f"] * (E[st["c"] + 1] - E[st["c"]])
    return qm * Ez * d.dt_s / 2


def test_load_positions_and_velocities():
    """Homogeneous quasi-neutral start (section 'Boundary conditions and initial values'): uniform
    positions, Maxwellian velocities at T_e0 and T_i0."""
    d = I.discharge(n_cells=128, n_e0=30000, n_i0=30000, V_rf_V=0.0, T_e0_eV=2.0, T_i0_K=300.0)
    o = O.Oracle(X.he_like(eps_max_eV=50, de_eV=1e-2), d, "f64", load=True)
    for sp, sig in ((0, math.sqrt(I.E_CH * 2.0 / I.M_E)), (1, math.sqrt(I.K_B * 300 / (4.002602 * I.AMU)))):
        st = o.get_state(sp)
        z = (st["c"] + st["f"]) / 128
        assert stats.kstest(z, "uniform").pvalue > 1e-4
        # every cell, the last one included, holds its binomial share n / N
        cnt = np.bincount(st["c"], minlength=128)
        assert cnt.size == 128 and np.all(np.abs(cnt - 30000 / 128) <= 5 * math.sqrt(30000 / 128))
        assert stats.kstest(st["vx"] / sig, "norm").pvalue > 1e-4
        assert stats.kstest(st["vy"] / sig, "norm").pvalue > 1e-4
        # v_z: the stored value plus the half kick of the t = 0 field is the Maxwellian sample,
        # independent of the other two components
        vz0 = st["vz"] + _half_kick(o, d, sp, st)
        assert stats.kstest(vz0 / sig, "norm").pvalue > 1e-4
        for a, b in ((st["vx"], st["vy"]), (st["vx"], vz0), (st["vy"], vz0)):
            assert abs(np.corrcoef(a, b)[0, 1]) < 5 / math.sqrt(a.size)


def test_moments_of_uniform_load():
    """Density moments integrate to w N exactly (charge conservation with half-cell wall volumes) and
    the mean energy of a 2 eV Maxwellian is 3 eV."""
    n = 200_000
    d = I.discharge(n_cells=128, n_e0=n, n_i0=n, V_rf_V=0.0, T_e0_eV=2.0, n_init_m3=1e14,
                    steps_per_period=100000)
    o = O.Oracle(X.he_like(eps_max_eV=50, de_eV=1e-2), d, "f64", load=True)
    o.step(1)
    m = o.moments()
    dx = d.gap_m / d.n_cells
    V = np.full(d.n_cells + 1, dx)
    V[0] = V[-1] = dx / 2
    w = d.w_e
    absorbed = sum(m["absorbed"][0])
    assert np.sum(m["n_e"] * V) == pytest.approx(w * (n - absorbed + (o.count(0) - n + absorbed)), rel=1e-12)
    Q = m["mean_eps"]
    # energy moment at (x_n, v_n) of the first step = the loaded velocities
    st_ne = m["n_e"]
    mean_eps = np.sum(Q * st_ne * V) / np.sum(st_ne * V)
    assert abs(mean_eps - 3.0) < 5 * math.sqrt(1.5) * 2.0 / math.sqrt(n) + 0.01


def test_stable_sort_by_cell():
    d = I.discharge(n_cells=64, n_e0=5000, n_i0=5000, V_rf_V=100.0)
    o = O.Oracle(X.he_like(eps_max_eV=100, de_eV=1e-2), d, "f64", load=True)
    o.sweep()
    before = [o.get_state(s) for s in (0, 1)]
    o.sort()
    for s in (0, 1):
        after = o.get_state(s)
        perm = np.argsort(before[s]["c"], kind="stable")
        for k in ("c", "f", "vx", "vy", "vz"):
            assert np.array_equal(after[k], before[s][k][perm])


def test_secondary_emission_count_is_binomial():
    """Added option (not in the paper): each absorbed ion emits an electron with probability gamma."""
    M = 4.002602 * I.AMU
    d = I.discharge(n_cells=32, gamma_see=0.3, steps_per_period=400)
    o = O.Oracle(_no_collision_gas(M), d, "f64", load=False)
    o.set_field(np.zeros(33))
    rng = np.random.default_rng(17)
    n = 20000
    dx = d.gap_m / 32
    st = {"c": np.where(np.arange(n) % 2 == 0, 0, 31).astype(np.int32), "f": rng.uniform(0, 1, n),
          "vx": np.zeros(n), "vy": np.zeros(n), "vz": np.zeros(n)}
    st["vz"] = np.where(st["c"] == 0, -1.0, 1.0) * 3 * dx / d.dt_s
    o.set_state(1, st)
    o.set_state(0, I.speed_state(rng, 1, 32, 0.0))
    o.sweep()
    c = o.counters()
    ab = c["absorbed"][1][0] + c["absorbed"][1][1]
    assert ab == n
    k = c["see_emitted"]
    assert abs(k - 0.3 * n) <= 5 * math.sqrt(0.3 * 0.7 * n)
    e = o.get_state(0)
    born = {kk: v[1:] for kk, v in e.items()}
    assert born["c"].size == k
    left = born["c"] == 0
    assert np.all(born["vz"][left] > 0) and np.all(born["vz"][~left] < 0)
    assert np.all(born["f"][left] == 0.0)


def test_f32_build_runs_and_matches_physics_build_statistically():
    """The decision-precision build takes the same steps; after a short run its moments agree with the
    FP64 build within the seed spread."""
    d = I.discharge(n_cells=64, n_e0=20000, n_i0=20000, V_rf_V=150.0, n_init_m3=4e14, steps_per_period=400)
    g = X.he_like(eps_max_eV=200, de_eV=1e-2)
    o64 = O.Oracle(g, d, "f64", sort_every=1)
    o32 = O.Oracle(g, d, "f32", sort_every=1)
    o64.step(100)
    o32.step(100)
    n64, n32 = o64.count(0), o32.count(0)
    assert abs(n64 - n32) < 0.05 * n64
    m64, m32 = o64.moments(), o32.moments()
    rel = np.linalg.norm(m64["n_i"] - m32["n_i"]) / np.linalg.norm(m64["n_i"])
    assert rel < 0.05


def test_steady_state_criterion():
    """Block-mean steady-state criterion: a count that relaxes exponentially to a plateau is steady
    once 50-period means 50 periods apart differ by < 1e-3; pure noise of 1e-2 per period is
    averaged down by the blocks."""
    from paper_1608_04601_gb300.steady import steady_period
    k = np.arange(2000)
    m = 1e5 * (1 + 0.5 * np.exp(-k / 100.0))
    ks = steady_period(np.stack([m, m], 1))
    # |mean_a - mean_b| / mean_a ~ 0.5 e^{-k/100} (e^{0.5} - 1) * (100/50) (1 - e^{-0.5}) < 1e-3
    exact = next(kk for kk in range(100, 2000)
                 if abs(np.mean(m[kk - 50:kk]) - np.mean(m[kk - 100:kk - 50])) / np.mean(m[kk - 50:kk]) < 1e-3)
    assert ks == exact
    rng = np.random.default_rng(0)
    flat = 1e5 * (1 + 1e-3 * rng.standard_normal((400, 2)))
    assert steady_period(flat) == 100
    assert steady_period(np.stack([m, m * 0 + 1e5], 1)[:150]) is None


def _tent_profiles(P, gap, n0e, n0i):
    """Tent electron density, flat ion density and a linear mean energy on P points over [0, gap]:
    piecewise linear, so the trapezoid integrals of the loader are exact."""
    z = np.linspace(0.0, gap, P)
    ne = n0e * np.minimum(z, gap - z) / (gap / 2)
    ni = np.full(P, n0i)
    eps = 2.0 + 4.0 * z / gap
    return z, np.stack([ne, ni, eps])


def test_warm_load_follows_profiles():
    """Warm start from density and mean-energy profiles (the paper's proposal of initial values
    closer to the periodic state, section 'Numerical parameters and initial values'): the count is
    the profile integral over the weight, positions follow the density, electron velocities are
    Maxwellian with kT = 2/3 of the local mean energy, ion velocities Maxwellian at T_gas."""
    P, gap, N = 33, 0.025, 64
    # weights of 1e14 m^-3 x gap / 1000: about 20000 electrons and 15000 ions from these profiles
    d = I.discharge(n_cells=N, n_e0=1000, n_i0=1000, V_rf_V=0.0, n_init_m3=1e14, gap_m=gap)
    o = O.Oracle(X.he_like(eps_max_eV=50, de_eV=1e-2), d, "f64", load=False)
    z, prof = _tent_profiles(P, gap, 4e15, 1.5e15)
    o.load_profiles(*prof)
    assert o.count(0) > 15000 and o.count(1) > 10000
    ne_int, ni_int = 4e15 * gap / 2, 1.5e15 * gap  # exact integrals of the tent and the flat profile
    assert o.count(0) == math.floor(ne_int / d.w_e + 0.5)
    assert o.count(1) == math.floor(ni_int / d.w_i + 0.5)
    for sp in (0, 1):
        st = o.get_state(sp)
        x = (st["c"] + st["f"]) / N * gap
        n = x.size
        # fraction below each profile point = the exact cumulative integral there
        frac = np.array([np.mean(x < zj) for zj in z[1:-1]])
        u = z[1:-1] / gap
        cdf = np.where(u <= 0.5, 2 * u ** 2, 1 - 2 * (1 - u) ** 2) if sp == 0 else u
        assert np.all(np.abs(frac - cdf) <= 5 * np.sqrt(cdf * (1 - cdf) / n) + 1e-12)
        if sp == 0:
            sig = np.sqrt(I.E_CH * (2.0 + 4.0 * x / gap) * 2.0 / (3.0 * I.M_E))
        else:
            sig = np.full(n, math.sqrt(I.K_B * d.T_gas_K / (4.002602 * I.AMU)))
        for k in ("vx", "vy"):
            assert stats.kstest(st[k] / sig, "norm").pvalue > 1e-4
        vz0 = st["vz"] + _half_kick(o, d, sp, st)
        assert stats.kstest(vz0 / sig, "norm").pvalue > 1e-4
        for a, b in ((st["vx"], st["vy"]), (st["vx"], vz0), (st["vy"], vz0)):
            assert abs(np.corrcoef(a, b)[0, 1]) < 5 / math.sqrt(n)
    # the field is solved at t = 0 from the loaded charge: non-zero, since n_e != n_i
    assert np.max(np.abs(o.get_field())) > 0


def test_warm_load_clips_negative_density_and_loads_empty_species():
    """A zero ion profile loads no ions; negative profile values count as zero."""
    P, gap = 9, 0.025
    d = I.discharge(n_cells=32, n_e0=1, n_i0=1, V_rf_V=0.0, n_init_m3=1e14, gap_m=gap)
    o = O.Oracle(X.he_like(eps_max_eV=50, de_eV=1e-2), d, "f64", load=False)
    z = np.linspace(0, gap, P)
    ne = np.where(z < gap / 2, 2e15, -1e15)  # negative half clipped to zero
    o.load_profiles(ne, np.zeros(P), np.full(P, 3.0))
    assert o.count(1) == 0
    A = sum(0.5 * (max(ne[j], 0) + max(ne[j + 1], 0)) * (gap / (P - 1)) for j in range(P - 1))
    assert o.count(0) == math.floor(A / d.w_e + 0.5)
    st = o.get_state(0)
    assert np.all((st["c"] + st["f"]) / 32 * gap <= z[P // 2 + 1])


def test_cold_load_stores_the_half_back_kicked_velocity():
    """The load stores v* = v_0 - (q/m) E(x_0, 0) dt / 2, so that the first half kick of the first
    step gives v_0 (the Verlet start). With T_e0 = T_i0 = 0 the loaded velocities are zero, and
    with twice as many ions as electrons the space charge makes a field at t = 0 (V_rf sin 0 = 0):
    the stored v_z is exactly minus the half kick of the field at the particle."""
    d = I.discharge(n_cells=64, n_e0=20000, n_i0=40000, V_rf_V=300.0, T_e0_eV=0.0, T_i0_K=0.0, n_init_m3=1e15)
    o = O.Oracle(X.he_like(eps_max_eV=50, de_eV=1e-2), d, "f64", load=True)
    E = o.get_field()
    assert np.max(np.abs(E)) > 1e3
    M = X.he_like(eps_max_eV=50, de_eV=1e-2).mass_kg
    for sp, qm in ((0, -I.E_CH / I.M_E), (1, I.E_CH / M)):
        st = o.get_state(sp)
        assert np.all(st["vx"] == 0) and np.all(st["vy"] == 0)
        Ez = E[st["c"]] + st["f"] * (E[st["c"] + 1] - E[st["c"]])
        kick = qm * Ez * d.dt_s / 2
        assert np.allclose(st["vz"], -kick, rtol=1e-12, atol=1e-12 * np.max(np.abs(kick)))
        assert np.max(np.abs(st["vz"])) > 0


def test_energy_moment_is_split_by_cic_and_clamped():
    """The electron energy moment at (x_n, v_n) is deposited like charge: (1 - f) of it at node c, f
    at node c + 1, in 2^-12 eV units, each electron's energy clamped at 16384 eV (2^26 units)."""
    o = O.Oracle(_no_collision_gas(4.002602 * I.AMU), I.discharge(n_cells=32), "f64", load=False)
    o.set_field(np.zeros(33))
    e1, e2 = 10.0, 20000.0
    v1, v2 = math.sqrt(2 * I.E_CH * e1 / I.M_E), math.sqrt(2 * I.E_CH * e2 / I.M_E)
    st = {"c": np.array([3, 20], np.int32), "f": np.array([0.25, 0.5]), "vx": np.array([v1, v2]),
          "vy": np.zeros(2), "vz": np.zeros(2)}
    o.set_state(0, st)
    o.set_state(1, {k: v[:1] for k, v in st.items()})
    o.sweep()
    Q = o.get_energy_deposit()
    u1 = e1 * 4096
    assert abs(Q[3] - 0.75 * u1) <= 1 and abs(Q[4] - 0.25 * u1) <= 1
    assert Q[20] == 2 ** 25 and Q[21] == 2 ** 25
    assert np.sum(Q) == Q[3] + Q[4] + 2 ** 26


def test_excitation_levels_lose_their_own_thresholds():
    """Two excitation levels (Table 'reactions' lists two for each gas) at 10 and 15 eV: an electron
    of 20 eV that excites level j leaves with exactly 20 eV - eps_j, isotropically."""
    M = 4.002602 * I.AMU
    n_pts, de = 40001, 5e-3
    eps = np.arange(n_pts) * de
    v = np.sqrt(2 * I.E_CH * np.maximum(eps, 1e-9) / I.M_E)
    z = np.zeros(n_pts)
    c1 = np.where(eps > 10.0, 1e-10 / v, 0.0)
    c2 = np.where(eps > 15.0, 1e-10 / v, 0.0)
    g = _gas_custom(M, n_pts, de, [z, c1, c2, z], [z, z], eps_exc=(10.0, 15.0))
    o = O.Oracle(g, I.discharge(n_cells=64), "f64", load=False)
    o.set_field(np.zeros(65))
    rng = np.random.default_rng(41)
    n = 6000
    st = I.energy_state(rng, n, 64, 20.0, 20.0, I.M_E)
    st["c"][:] = 32
    o.set_state(0, st)
    o.set_state(1, I.speed_state(rng, 1, 64, 0.0))
    o.sweep()
    c = o.counters()["collisions_e"]
    assert c[1] + c[2] == n and c[1] > n // 3 and c[2] > n // 3
    out = o.get_state(0)
    e = 0.5 * I.M_E * (out["vx"] ** 2 + out["vy"] ** 2 + out["vz"] ** 2) / I.E_CH
    at10, at5 = np.abs(e - 10.0) < 1e-9, np.abs(e - 5.0) < 1e-9
    assert at10.sum() == c[1] and at5.sum() == c[2]


def test_newborns_get_the_half_kick_of_their_birth():
    """Velocity Verlet with collisions at v_n: the ionizing electron gets its second half kick after
    the collision, and both newborns (born at t_n) get one half kick from the field at the parent.
    In a uniform field E0 the scattered and the ejected electron therefore both have
    |v - (q/m) E0 dt/2 z| = sqrt((eps_n - eps_iz) / 2) in speed units, and the newborn ions' mean v_z
    is (e / M) E0 dt/2 (their thermal v_z averages out)."""
    M = 4.002602 * I.AMU
    eiz = 24.6
    g = _forced_gas(M, 2, 1e-10, eps_th=eiz)
    d = I.discharge(n_cells=64)
    o = O.Oracle(g, d, "f64", load=False)
    E0 = 1e5
    o.set_field(np.full(65, E0))
    rng = np.random.default_rng(43)
    n = 8000
    # 80-200 eV: after the first half kick (up to 1.6e6 m/s here) every electron is still above
    # the threshold, so every one ionizes
    st = I.energy_state(rng, n, 64, 80.0, 200.0, I.M_E)
    st["c"][:] = 32
    o.set_state(0, st)
    o.set_state(1, I.speed_state(rng, 1, 64, 0.0))
    o.sweep()
    assert o.counters()["collisions_e"][3] == n
    Ke = -I.E_CH / I.M_E * E0 * d.dt_s / 2
    vzn = st["vz"] + Ke
    eps_n = 0.5 * I.M_E * (st["vx"] ** 2 + st["vy"] ** 2 + vzn ** 2) / I.E_CH
    out = o.get_state(0)
    s2 = (out["vx"] ** 2 + out["vy"] ** 2 + (out["vz"] - Ke) ** 2) * 0.5 * I.M_E / I.E_CH
    ref = (eps_n - eiz) / 2
    assert np.max(np.abs(s2[:n] - ref)) < 1e-9 * np.max(ref)
    assert np.max(np.abs(s2[n:] - ref)) < 1e-9 * np.max(ref)
    ions = o.get_state(1)
    vz_i = ions["vz"][1:]
    Ki = I.E_CH / M * E0 * d.dt_s / 2
    sig_n = math.sqrt(I.K_B * 300.0 / M)
    assert abs(np.mean(vz_i) - Ki) <= 5 * sig_n / math.sqrt(n)
    assert Ki > 10 * sig_n / math.sqrt(n)


def test_sort_schedule():
    """Periodic sorting: with sort_every = k the store is sorted by cell (stably) after the sweep of
    step n when (n + 1) % k == 0, and only then; the first load is in random cell order."""
    d = I.discharge(n_cells=64, n_e0=4000, n_i0=4000, V_rf_V=100.0, steps_per_period=400)
    o = O.Oracle(X.he_like(eps_max_eV=100, de_eV=1e-2), d, "f64", sort_every=4, load=True)
    sorted_ = lambda: all(np.all(np.diff(o.get_state(sp)["c"]) >= 0) for sp in (0, 1))
    assert not sorted_()
    for n in range(8):
        o.step(1)
        assert sorted_() == ((n + 1) % 4 == 0), n


def test_mean_energy_divides_by_the_density_at_x_n():
    """The mean electron energy is the energy moment at (x_n, v_n) over the density moment at x_n
    (the same particles at the same time), not the density after the push: electrons that sit on
    node 10 and cross two cells in the step report their energy at node 10 and none at node 12."""
    N = 32
    d = I.discharge(n_cells=N, steps_per_period=400)
    o = O.Oracle(_no_collision_gas(), d, "f64", load=False)
    o.set_field(np.zeros(N + 1))
    dx = d.gap_m / N
    vz = 2.0 * dx / d.dt_s
    eps = 0.5 * I.M_E * vz * vz / I.E_CH
    n = 100
    st = {"c": np.full(n, 10, np.int32), "f": np.zeros(n), "vx": np.zeros(n), "vy": np.zeros(n), "vz": np.full(n, vz)}
    o.set_state(0, st)
    o.set_state(1, {k: v[:1] for k, v in st.items()})
    # the density moment at x_n is the previous sweep's deposit: n electrons on node 10
    D = np.zeros(N + 1, np.int64)
    D[10] = n * 2 ** 32
    o.set_deposit(0, D)
    o.reset_moments()
    o.step(1)
    m = o.moments()
    assert abs(m["mean_eps"][10] - eps) <= 2.0 ** -12 + 1e-12 * eps
    assert m["mean_eps"][12] == 0.0


def test_warm_load_temperature_is_interpolated_between_profile_points():
    """Electron temperature of the warm load: kT = 2/3 of the mean energy interpolated linearly at the
    sampled position. Two profile points, 1 eV at z = 0 and 9 eV at z = d, uniform density."""
    gap, N = 0.025, 64
    d = I.discharge(n_cells=N, n_e0=1000, n_i0=1000, V_rf_V=0.0, n_init_m3=1e14, gap_m=gap)
    o = O.Oracle(X.he_like(eps_max_eV=50, de_eV=1e-2), d, "f64", load=False)
    o.load_profiles(np.array([1e15, 1e15]), np.array([1e15, 1e15]), np.array([1.0, 9.0]))
    st = o.get_state(0)
    assert st["c"].size == 10000  # 1e15 m^-3 x 2.5 cm over the weight 2.5e9
    x = (st["c"] + st["f"]) / N
    sig = np.sqrt(I.E_CH * (2.0 / 3.0) * (1.0 + 8.0 * x) / I.M_E)
    for k in ("vx", "vy"):
        assert stats.kstest(st[k] / sig, "norm").pvalue > 1e-4


def test_moment_reset_counts_absorptions_since_the_reset():
    """After reset_moments the moments average over the steps since the reset, and the absorbed
    counts they report are those since the reset."""
    d = I.discharge(n_cells=64, n_e0=5000, n_i0=5000, V_rf_V=200.0, steps_per_period=200)
    o = O.Oracle(X.he_like(eps_max_eV=100, de_eV=1e-2), d, "f64", load=True)
    o.step(40)
    a0 = np.array(o.counters()["absorbed"], dtype=np.int64)
    o.reset_moments()
    o.step(30)
    a1 = np.array(o.counters()["absorbed"], dtype=np.int64)
    m = o.moments()
    assert m["steps"] == 30
    assert np.all(a0 > 0) or a0.sum() > 0
    assert np.array_equal(np.array(m["absorbed"], dtype=np.int64), a1 - a0)
