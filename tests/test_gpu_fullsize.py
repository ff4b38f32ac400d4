"""Bit-exact GPU-vs-oracle parity at the sizes and launch settings the benchmark runs.

The 1e6 + 1e6 particle Ar-like discharge (512 cells, 2000 steps per rf period) and the He-like
500 V discharge with secondary emission at 2e6 + 2e6 (2048 cells), advanced by whole library
steps (pic_step: sweep, post-sweep grid, the sort every 16 steps) at the benchmark's launch
shapes. These stores span several slices of sweep chunks, so the output offsets that the
post-sweep grid derives from the slice sums of earlier slices are exercised; between sorts the
sweep reads aged stores chunk by chunk through their region layouts. Each step both sides start from the same
state and the same FP32 node field (the oracle's, fed to the library after its own solve, so that
a last-bit difference of the two FP64 Poisson solvers cannot make the paths diverge), and the
result must be identical: event counters, particle order, cells and every FP32 value bit for bit,
and at the end the cycle-averaged moments built from the exact integer deposits.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1608_04601_gb300 import xsections as X
from paper_1608_04601_gb300.workloads import c2, c3

pytestmark = pytest.mark.gpu

SLICE_CHUNKS = 4096  # sweep chunks per slice of the post-sweep grid


@pytest.fixture(scope="module")
def P():
    import __graft_entry__ as g
    g.build()
    from paper_1608_04601_gb300 import pic
    return pic


def _workload(name):
    if name == "c2":
        return c2()
    # the 500 V He-like discharge with secondary emission at a tenth of its particles
    return c3().scaled(n_e0=2_000_000, n_i0=2_000_000)


# workload, block, particles per thread, sort period, steps. Without a sort the library repacks the
# stores (order-preserving) every 50 steps at 2000 steps per period; 56 steps cover one repack.
CASES = [("c2", 256, 2, 16, 32), ("c2", 256, 4, 16, 32), ("c2", 128, 4, 16, 32), ("c3-tenth", 256, 2, 16, 32),
         ("c2", 256, 2, 0, 56)]


@pytest.mark.parametrize("case", CASES, ids=[f"{a}-{b}x{c}-sort{k}" for a, b, c, k, _ in CASES])
def test_fullsize_steps_bit_exact(P, case):
    name, block, ppt, K, steps = case
    d = _workload(name)
    gas = X.by_name(d.gas, eps_max_eV=d.eps_max_eV, de_eV=d.de_eV)
    ref = O.Oracle(gas, d, "f32", sort_every=K)
    sim = P.Simulation(gas, d, seed=d.seed, precision="fp32", sort_every=K, block=block, ppt=ppt, load=False)
    for sp in (0, 1):
        sim.set_state(0, sp, ref.get_state(sp))
    sim.set_field(0, ref.get_field())
    chunk = 32 * ppt
    assert min(ref.count(0), ref.count(1)) > SLICE_CHUNKS * chunk  # at least two slices per store
    for n in range(steps):
        sim.step(1)
        ref.step(1)
        if n == 0:  # moments from step 1 on (the library's x_n deposit of step 0 is the upload's)
            sim.reset_moments()
            ref.reset_moments()
        assert sim.step_index == ref.step_index == n + 1
        assert sim.counters(0) == ref.counters(), f"step {n}: counters"
        for sp in (0, 1):
            a, b = sim.get_state(0, sp), ref.get_state(sp)
            assert a["c"].size == b["c"].size, f"step {n} sp{sp}: counts {a['c'].size} vs {b['c'].size}"
            assert np.array_equal(a["c"], b["c"]), f"step {n} sp{sp}: order/cells"
            for k in ("f", "vx", "vy", "vz"):
                assert np.array_equal(a[k], b[k]), f"step {n} sp{sp}: {k}"
        # the two FP64 solves agree to their rounding (the oracle's tridiagonal elimination loses up
        # to a few units of 2^-52 per node, so the bound grows with N); the next step starts from
        # the oracle's field on both
        E, E64, _ = sim.get_field(0)
        R64 = ref.get_field64()
        assert np.max(np.abs(E64 - R64)) <= 4e-15 * d.n_cells * np.max(np.abs(R64))
        sim.set_field(0, ref.get_field())
    ma, mb = sim.moments(0), ref.moments()
    assert ma["steps"] == mb["steps"] == steps - 1
    for k in ("n_e", "n_i", "mean_eps"):
        assert np.array_equal(ma[k], mb[k]), k
    sim.close()
