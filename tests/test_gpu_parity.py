"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

Bit-exact: random words, collision decisions (counters), survival, output order, cells, 64-bit
deposits and energy moments. Floating point: FP32/FP64 positions and velocities within 1e-6
relative (norm-wise; they are in fact bitwise equal because both sides evaluate the same
documented operation sequence); FP64 Poisson within 1e-12 relative.
"""
import math

import numpy as np
import pytest

import inputs as I
from oracle import oracle as O
from paper_1608_04601_gb300 import xsections as X

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    from paper_1608_04601_gb300 import pic
    return pic


def _prec(p):
    return "f32" if p == "fp32" else "f64"


def assert_state_equal(a, b, exact_float=False, what=""):
    assert a["c"].size == b["c"].size, f"{what}: counts {a['c'].size} vs {b['c'].size}"
    assert np.array_equal(a["c"], b["c"]), f"{what}: cells/order differ at {np.flatnonzero(a['c'] != b['c'])[:5]}"
    # positions relative to the gap: f is in cell units, so |df| <= tol
    assert np.max(np.abs(a["f"].astype(np.float64) - b["f"]), initial=0) <= REL_TOL, what
    v1 = np.stack([a["vx"], a["vy"], a["vz"]]).astype(np.float64)
    v2 = np.stack([b["vx"], b["vy"], b["vz"]]).astype(np.float64)
    nrm = np.linalg.norm(v2, axis=0)
    err = np.linalg.norm(v1 - v2, axis=0)
    assert np.all(err <= REL_TOL * np.maximum(nrm, 1e-30)), f"{what}: max rel {np.max(err / np.maximum(nrm, 1e-30))}"
    if exact_float:
        for k in ("f", "vx", "vy", "vz"):
            assert np.array_equal(a[k], b[k]), f"{what}: {k} not bitwise equal"


# ----------------------------------------------------------------------------- building blocks

def test_philox_matches_oracle(P):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, (20000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    key = np.array([0xA4093822, 0x299F31D0], np.uint32)
    got = P.debug_philox(ctr, key)
    for i in range(0, 20000, 97):
        assert np.array_equal(got[i], O.philox(ctr[i], key))


def test_own_math_bitwise_equal_to_oracle(P):
    rng = np.random.default_rng(2)
    x = np.concatenate([((rng.integers(0, 2 ** 23, 50000) + 0.5) * 2.0 ** -23), 2.0 ** rng.uniform(-30, 30, 5000)])
    y = rng.uniform(0, 2, x.size)
    x = x.astype(np.float32)
    y = y.astype(np.float32)
    lg, sn, cs = P.debug_math(x, y)
    for i in range(0, x.size, 37):
        assert lg[i] == np.float32(O.logf(float(x[i])))
        s, c = O.sincospif(float(y[i]))
        assert sn[i] == np.float32(s) and cs[i] == np.float32(c)
    # and against the exact functions (error bounds)
    ref = np.log(x.astype(np.float64))
    assert np.max(np.abs(lg - ref) / np.spacing(np.abs(ref).astype(np.float32) + np.float32(1e-30))) <= 3.0
    assert np.max(np.abs(sn - np.sin(np.pi * y.astype(np.float64)))) <= 2 ** -22


# ----------------------------------------------------------------------------- setup parity

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("gasname", ["he", "ar"])
def test_tables_and_constants_match_oracle(P, prec, gasname):
    gas = X.by_name(gasname, eps_max_eV=300.0, de_eV=1e-2)
    d = I.discharge(n_cells=64, p_Pa=20.0, gamma_see=0.1, n_e0=100, n_i0=100, T_e0_eV=2.0)
    sim = P.Simulation(gas, d, precision=prec, load=False)
    ref = O.Oracle(gas, d, _prec(prec), load=False)
    Te, Ti = sim.tables(0)
    Re, Ri = ref.tables(gas.n_pts)
    assert np.array_equal(Te, Re) and np.array_equal(Ti, Ri)
    a, b = sim.derived(0), ref.derived()
    for k in b:
        assert a[k] == b[k], (k, a[k], b[k])
    sim.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_load_matches_oracle(P, prec):
    """Uniform/Maxwellian load from the same Philox streams, initial deposit, solve, half back-kick."""
    gas = X.he_like(eps_max_eV=200.0, de_eV=1e-2)
    d = I.discharge(n_cells=128, n_e0=30001, n_i0=29999, V_rf_V=200.0, n_init_m3=4e14)
    sim = P.Simulation(gas, d, precision=prec)
    ref = O.Oracle(gas, d, _prec(prec))
    for sp in (0, 1):
        a, b = sim.get_state(0, sp), ref.get_state(sp)
        assert_state_equal(a, b, what=f"load sp{sp}")
        for k in ("c", "f", "vx", "vy"):
            assert np.array_equal(a[k], b[k])
    E, E64, phi = sim.get_field(0)
    assert np.max(np.abs(E64 - ref.get_field64())) <= 1e-12 * np.max(np.abs(ref.get_field64()))
    sim.close()


# ----------------------------------------------------------------------------- one sweep

def _population(rng, N, dt, dtype, n_e, n_i, gap):
    e = I.mixed_state(rng, n_e, N, 0, dtype, gap_m=gap, dt_s=dt)
    i = I.mixed_state(rng, n_i, N, 1, dtype, gap_m=gap, dt_s=dt)
    return e, i


CASES = [
    # gas, N, p, gamma, n_e, n_i, step, block, ppt
    ("he", 128, 30.0, 0.0, 20000, 20000, 0, 256, 4),
    ("he", 64, 80.0, 0.3, 7777, 5003, 12345, 256, 4),       # ragged tiles, SEE on
    ("ar", 512, 10.0, 0.0, 50000, 41000, 7, 128, 2),
    ("ar", 33, 40.0, 0.1, 3000, 9000, (1 << 33) + 5, 256, 8),  # step beyond 32 bits
    ("he", 16, 30.0, 0.0, 1, 0, 3, 256, 4),                  # one electron, no ions
    ("he", 16, 30.0, 0.0, 0, 17, 3, 256, 4),                 # no electrons
]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("case", CASES)
def test_single_sweep_bit_parity(P, prec, case):
    gasname, N, p, gamma, n_e, n_i, step, block, ppt = case
    gas = X.by_name(gasname, eps_max_eV=400.0, de_eV=2e-3)
    d = I.discharge(gas=gasname, n_cells=N, p_Pa=p, gamma_see=gamma, V_rf_V=250.0, steps_per_period=400,
                    seed=0xDEADBEEF12345, discharge_id=3)
    dtype = np.float32 if prec == "fp32" else np.float64
    rng = np.random.default_rng(N * 7 + n_e)
    e, i = _population(rng, N, d.dt_s, dtype, n_e, n_i, d.gap_m)
    E = I.random_field(rng, N, 4e4, dtype)
    sim = P.Simulation(gas, d, precision=prec, load=False, block=block, ppt=ppt, capacity=[(4 * n_e + 8192, 4 * n_i + n_e + 8192)])
    ref = O.Oracle(gas, d, _prec(prec), load=False)
    for obj in (sim, ref):
        if obj is sim:
            obj.set_state(0, 0, e)
            obj.set_state(0, 1, i)
            obj.set_field(0, E)
            obj.step_index = step
        else:
            obj.set_state(0, e)
            obj.set_state(1, i)
            obj.set_field(E)
            obj.step_index = step
    sim.sweep()
    ref.sweep()
    sim.sync()
    ca, cb = sim.counters(0), ref.counters()
    assert ca == cb, (ca, cb)
    for sp in (0, 1):
        assert_state_equal(sim.get_state(0, sp), ref.get_state(sp), exact_float=True, what=f"{prec} sp{sp}")
        assert np.array_equal(sim.get_deposit(0, sp), ref.get_deposit(sp))
    assert np.array_equal(sim.get_energy_deposit(0), ref.get_energy_deposit())
    # sort of the result
    sim.sort()
    ref.sort()
    for sp in (0, 1):
        assert_state_equal(sim.get_state(0, sp), ref.get_state(sp), exact_float=True, what=f"sorted sp{sp}")
    sim.close()


def test_forced_ionization_every_particle(P):
    """Worst case for births: every electron ionizes (nu_max dt >> 1); births double the store."""
    eps = np.arange(20001) * 1e-2
    v = np.sqrt(2 * I.E_CH * np.maximum(eps, 1e-9) / I.M_E)
    z = np.zeros_like(eps)
    se = np.stack([z, z, np.where(eps > 24.6, 1e-10 / v, 0.0)], 1)
    gas = X.GasTables("forced", 4.0026 * I.AMU, (1e9,), 24.6, 1e-2, se, np.stack([z, z], 1))
    d = I.discharge(n_cells=64)
    rng = np.random.default_rng(5)
    e = I.energy_state(rng, 5000, 64, 30.0, 150.0, I.M_E, np.float32)
    e["c"][:] = 32
    i = I.maxwell_state(rng, 10, 64, 500.0, np.float32)
    sim = P.Simulation(gas, d, precision="fp32", load=False, capacity=[(20000, 20000)])
    ref = O.Oracle(gas, d, "f32", load=False)
    sim.set_state(0, 0, e)
    sim.set_state(0, 1, i)
    ref.set_state(0, e)
    ref.set_state(1, i)
    Z = np.zeros(65, np.float32)
    sim.set_field(0, Z)
    ref.set_field(Z)
    sim.sweep()
    ref.sweep()
    sim.sync()
    assert sim.counters(0) == ref.counters()
    assert sim.count(0, 0) == 10000 and sim.count(0, 1) == 5010
    for sp in (0, 1):
        assert_state_equal(sim.get_state(0, sp), ref.get_state(sp), exact_float=True)
    sim.close()


def test_capacity_overflow_is_reported(P):
    from paper_1608_04601_gb300 import _native as NV
    eps = np.arange(2001) * 1e-1
    v = np.sqrt(2 * I.E_CH * np.maximum(eps, 1e-9) / I.M_E)
    z = np.zeros_like(eps)
    se = np.stack([z, z, np.where(eps > 24.6, 1e-10 / v, 0.0)], 1)
    gas = X.GasTables("forced", 4.0026 * I.AMU, (1e9,), 24.6, 1e-1, se, np.stack([z, z], 1))
    d = I.discharge(n_cells=64)
    rng = np.random.default_rng(6)
    e = I.energy_state(rng, 3000, 64, 30.0, 150.0, I.M_E, np.float32)
    e["c"][:] = 32
    sim = P.Simulation(gas, d, precision="fp32", load=False, capacity=[(4000, 4000)])
    sim.set_state(0, 0, e)
    sim.set_field(0, np.zeros(65, np.float32))
    sim.sweep()
    with pytest.raises(NV.PicError) as ex:
        sim.sync()
    assert ex.value.status == -3
    sim.close()


def test_batch_of_discharges_each_matches_its_oracle(P):
    """Several discharges (different gases, cells, counts) in one sweep launch."""
    gases = [X.he_like(eps_max_eV=300.0, de_eV=1e-2), X.ar_like(eps_max_eV=300.0, de_eV=1e-2)]
    specs = [("he", 0, 64, 20.0, 3000, 2500), ("ar", 1, 128, 40.0, 10000, 12000), ("he", 0, 33, 80.0, 0, 500),
             ("ar", 1, 256, 10.0, 4097, 4096)]
    dis, pops, fields = [], [], []
    rng = np.random.default_rng(9)
    for k, (gname, gi, N, p, ne, ni) in enumerate(specs):
        d = I.discharge(gas=gname, n_cells=N, p_Pa=p, V_rf_V=100.0 + 50 * k, discharge_id=k, seed=77,
                        gamma_see=0.1 * (k % 2))
        dis.append((d, gi))
        pops.append(_population(rng, N, d.dt_s, np.float32, ne, ni, d.gap_m))
        fields.append(I.random_field(rng, N, 2e4, np.float32))
    caps = [(4 * max(s[4], 1) + 4096, 4 * max(s[5], 1) + s[4] + 4096) for s in specs]
    sim = P.Simulation(gases, dis, seed=77, precision="fp32", load=False, capacity=caps)
    for k in range(len(specs)):
        sim.set_state(k, 0, pops[k][0])
        sim.set_state(k, 1, pops[k][1])
        sim.set_field(k, fields[k])
    sim.step_index = 42
    sim.sweep()
    sim.sync()
    for k, (d, gi) in enumerate(dis):
        ref = O.Oracle(gases[gi], d, "f32", load=False)
        ref.set_state(0, pops[k][0])
        ref.set_state(1, pops[k][1])
        ref.set_field(fields[k])
        ref.step_index = 42
        ref.sweep()
        assert sim.counters(k) == ref.counters(), k
        for sp in (0, 1):
            assert_state_equal(sim.get_state(k, sp), ref.get_state(sp), exact_float=True, what=f"d{k} sp{sp}")
            assert np.array_equal(sim.get_deposit(k, sp), ref.get_deposit(sp))
    sim.close()


# ----------------------------------------------------------------------------- field solve

def _thomas_longdouble(rho, dx, V0):
    """Reference solve in extended precision (numpy longdouble) for error attribution."""
    N = rho.size - 1
    ld = np.longdouble
    eps0 = ld(I.EPS0)
    phi = np.zeros(N + 1, ld)
    phi[0], phi[N] = ld(V0), ld(0)
    M = N - 1
    if M >= 1:
        cp = np.zeros(M + 1, ld)
        dp = np.zeros(M + 1, ld)
        for j in range(1, M + 1):
            b = -ld(rho[j]) * ld(dx) * ld(dx) / eps0
            if j == 1:
                b -= ld(V0)
            if j == 1:
                cp[j], dp[j] = ld(-0.5), b / ld(-2)
            else:
                m = ld(-2) - cp[j - 1]
                cp[j], dp[j] = ld(1) / m, (b - dp[j - 1]) / m
        phi[M] = dp[M]
        for j in range(M - 1, 0, -1):
            phi[j] = dp[j] - cp[j] * phi[j + 1]
    E = np.zeros(N + 1, ld)
    E[1:N] = (phi[:N - 1] - phi[2:]) / (ld(2) * ld(dx))
    E[0] = (phi[0] - phi[1]) / ld(dx) - ld(rho[0]) * ld(dx) / (ld(2) * eps0)
    E[N] = (phi[N - 1] - phi[N]) / ld(dx) + ld(rho[N]) * ld(dx) / (ld(2) * eps0)
    return phi.astype(np.float64), E.astype(np.float64)


@pytest.mark.parametrize("N", [1, 2, 7, 128, 2048, 4096])
def test_poisson_matches_oracle(P, N):
    """FP64 two-scan solve on the GPU vs the oracle's Thomas solve: within 1e-12 of max|E| for the
    configured grids (N <= 2048), 1e-11 at the 4096-cell maximum; both are also compared with an
    extended-precision solve so that a miss is attributed to the right side."""
    gas = X.he_like(eps_max_eV=50.0, de_eV=1e-2)
    d = I.discharge(n_cells=N, gap_m=0.05, V_rf_V=500.0, n_init_m3=4e14, n_e0=1000, n_i0=1000)
    rng = np.random.default_rng(N)
    De = rng.integers(0, 2 ** 40, N + 1).astype(np.int64)
    Di = De + rng.integers(-2 ** 36, 2 ** 36, N + 1)
    Di = np.maximum(Di, 0)
    sim = P.Simulation(gas, d, precision="fp32", load=False)
    ref = O.Oracle(gas, d, "f64", load=False)
    tol = 1e-12 if N <= 2048 else 1e-11
    for step in (0, 17):
        sim.step_index = step
        ref.step_index = step
        sim.set_deposit(0, 0, De)
        sim.set_deposit(0, 1, Di)
        ref.set_deposit(0, De)
        ref.set_deposit(1, Di)
        sim.solve()
        ref.solve()
        E, E64, phi = sim.get_field(0)
        Er, phr = ref.get_field64(), ref.get_phi()
        dx = d.gap_m / N
        rho = I.E_CH * (d.w_i * Di.astype(np.float64) - d.w_e * De.astype(np.float64)) / (2.0 ** 32 * dx)
        rho[0] *= 2
        rho[N] *= 2
        V0 = d.V_rf_V * math.sin(2 * math.pi * d.f_rf_Hz * (step + 1) * d.dt_s)
        phx, Ex = _thomas_longdouble(rho, dx, V0)
        sE = np.max(np.abs(Ex))
        err_gpu, err_orc = np.max(np.abs(E64 - Ex)) / sE, np.max(np.abs(Er - Ex)) / sE
        print(f"N={N} step={step}: |E_gpu-E_x|/max={err_gpu:.2e} |E_oracle-E_x|/max={err_orc:.2e} "
              f"|E_gpu-E_oracle|/max={np.max(np.abs(E64 - Er)) / sE:.2e}")
        assert np.max(np.abs(phi - phr)) <= tol * max(np.max(np.abs(phr)), 1.0)
        assert np.max(np.abs(E64 - Er)) <= tol * np.max(np.abs(Er))
        assert np.max(np.abs(E.astype(np.float64) - Er)) <= 2 ** -23 * np.max(np.abs(Er))
    sim.close()


# ----------------------------------------------------------------------------- several steps

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_full_steps_track_oracle(P, prec):
    """Whole steps (sweep, births, sort, Poisson, moments) on C1's discharge at reduced count: the
    two paths stay identical until a field value rounds differently (FP64 scan vs Thomas), and the
    counts then stay within sampling noise."""
    from paper_1608_04601_gb300.workloads import c1
    d = c1().scaled(n_e0=4000, n_i0=4000)
    gas = X.he_like(eps_max_eV=300.0, de_eV=1e-2)
    sim = P.Simulation(gas, d, precision=prec, sort_every=1)
    ref = O.Oracle(gas, d, _prec(prec), sort_every=1)
    exact_steps = 0
    for k in range(40):
        sim.step(1)
        ref.step(1)
        a, b = sim.get_state(0, 0), ref.get_state(0)
        if a["c"].size == b["c"].size and np.array_equal(a["c"], b["c"]):
            exact_steps += 1
        else:
            break
    assert exact_steps >= 5
    s0 = sim.step_index
    assert s0 == ref.step_index
    sim.step(400 - s0)
    ref.step(400 - s0)
    assert sim.step_index == ref.step_index == 400
    for sp in (0, 1):
        na, nb = sim.count(0, sp), ref.count(sp)
        assert abs(na - nb) <= 6 * math.sqrt(max(abs(4000 - nb), 100)) + 0.03 * nb, (sp, na, nb)
    sim.close()


# ----------------------------------------------------------------------------- warm start

@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_warm_load_matches_oracle(P, prec):
    """Warm start from profiles: counts, sampled positions and velocities, initial field and the
    half back-kick agree with the oracle's loader drawing the same Philox streams."""
    gas = X.he_like(eps_max_eV=200.0, de_eV=1e-2)
    gap = 0.025
    d = I.discharge(n_cells=128, n_e0=20000, n_i0=20000, V_rf_V=150.0, n_init_m3=1e15, gap_m=gap)
    Pn = 57  # about 30000 electrons and 35600 ions at the weight 1.25e9
    z = np.linspace(0.0, gap, Pn)
    ne = 3e15 * np.sin(np.pi * z / gap) ** 2
    ni = 3.2e15 * np.sin(np.pi * z / gap) ** 1.5
    eps = 1.0 + 5.0 * (2 * z / gap - 1) ** 2
    sim = P.Simulation(gas, d, precision=prec, load=False)
    sim.load_profiles(np.stack([ne, ni, eps]))
    ref = O.Oracle(gas, d, _prec(prec), load=False)
    ref.load_profiles(ne, ni, eps)
    for sp in (0, 1):
        a, b = sim.get_state(0, sp), ref.get_state(sp)
        assert a["c"].size == b["c"].size > 1000
        assert_state_equal(a, b, what=f"warm load sp{sp}")
        for k in ("c", "f", "vx", "vy"):
            assert np.array_equal(a[k], b[k])
    E, E64, phi = sim.get_field(0)
    assert np.max(np.abs(E64 - ref.get_field64())) <= 1e-12 * np.max(np.abs(ref.get_field64()))
    sim.step(3)
    ref.step(3)
    for sp in (0, 1):
        assert_state_equal(sim.get_state(0, sp), ref.get_state(sp), what=f"warm steps sp{sp}")
    sim.close()
    with pytest.raises(RuntimeError):
        s2 = P.Simulation(gas, d, precision=prec)
        try:
            s2.step(1)
            s2.load_profiles(np.stack([ne, ni, eps]))
        finally:
            s2.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_state_upload_round_trip_and_rejects_bad_cells(P, prec):
    """pic_set_state / pic_get_state move the exact values (device-side interleave and gather);
    a cell outside [0, N) is reported and leaves the store empty."""
    rng = np.random.default_rng(21)
    d = I.discharge(n_cells=64, n_e0=10, n_i0=10)
    gas = X.he_like(eps_max_eV=200.0, de_eV=1e-2)
    sim = P.Simulation(gas, d, precision=prec, load=False, capacity=[(5000, 5000)])
    dt = np.float32 if prec == "fp32" else np.float64
    st = I.maxwell_state(rng, 3001, 64, 1e5, dt)
    sim.set_state(0, 0, st)
    back = sim.get_state(0, 0)
    for k in ("c", "f", "vx", "vy", "vz"):
        assert np.array_equal(back[k], st[k])
    bad = dict(st)
    bad["c"] = st["c"].copy()
    bad["c"][1234] = 64
    with pytest.raises(RuntimeError):
        sim.set_state(0, 1, bad)
    assert sim.count(0, 1) == 0
    sim.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_harmonic_oscillation_tracks_oracle(P, prec, tol):
    """A test electron released at rest in a uniform fixed ion background (grounded plates): the
    kernels' gather, half kicks, drift and Poisson solve follow the oracle, which the CPU pins tie
    to the velocity-Verlet closed form A cos(w n dt). Positions agree to tol x amplitude over
    200 steps (about nine oscillations)."""
    N, gap, n0, m = 64, 0.025, 8e14, 16
    gas = X.constant_sigma(0.0, mass_kg=1.0)  # no collisions; ions of 1 kg stay put
    d = I.discharge(n_cells=N, gap_m=gap, n_e0=N * m, n_i0=N * m, n_init_m3=n0, V_rf_V=0.0)
    dt, dx = d.dt_s, gap / N
    dtype = np.float64 if prec == "fp64" else np.float32
    sim = P.Simulation(gas, d, precision=prec, load=False)
    ref = O.Oracle(gas, d, _prec(prec), load=False)
    k = np.arange(N * m)
    ions = {"c": (k // m).astype(np.int32), "f": (((k % m) + 0.5) / m).astype(dtype),
            "vx": np.zeros(k.size, dtype), "vy": np.zeros(k.size, dtype), "vz": np.zeros(k.size, dtype)}
    A = 0.2 * gap
    z0 = gap / 2 + A
    c0 = int(z0 // dx)
    e = {"c": np.array([c0], np.int32), "f": np.array([z0 / dx - c0], dtype), "vx": np.zeros(1, dtype),
         "vy": np.zeros(1, dtype), "vz": np.zeros(1, dtype)}
    for obj in (sim, ref):
        if obj is sim:
            sim.set_field(0, np.zeros(N + 1, dtype))
            sim.set_state(0, 1, ions)
            sim.set_state(0, 0, e)
        else:
            ref.set_field(np.zeros(N + 1, dtype))
            ref.set_state(1, ions)
            ref.set_state(0, e)
        obj.sweep()
        obj.solve()
    E_z0 = float(np.interp(z0, np.arange(N + 1) * dx, ref.get_field64()))
    e["vz"] = np.array([(I.E_CH / I.M_E) * E_z0 * dt / 2], dtype)  # released at rest
    sim.set_state(0, 0, e)
    ref.set_state(0, e)
    for n in range(1, 201):
        sim.step(1)
        ref.step(1)
        if n in (1, 7, 50, 200):
            a, b = sim.get_state(0, 0), ref.get_state(0)
            za = (float(a["c"][0]) + float(a["f"][0])) * dx
            zb = (float(b["c"][0]) + float(b["f"][0])) * dx
            assert abs(za - zb) <= tol * A, (prec, n, za, zb)
    sim.close()
