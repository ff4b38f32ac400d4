"""State transfers through pinned host memory: when every host array of pic_get_state /
pic_set_state is pinned and mapped, the pack and unpack kernels read and write the caller's arrays
directly (no device staging); with pageable arrays they go through staging and copies. Both paths
must give the same store, bit for bit, in both precisions, for a store in a region layout (after
sweeps without a sort), with host arrays on a 16-byte boundary (the kernels move whole 16-byte
groups, then the ragged tail) and one element off it (element by element)."""
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


def _pinned(n, dtype):
    import torch
    tdt = {np.int32: torch.int32, np.float32: torch.float32, np.float64: torch.float64}[dtype]
    t = torch.empty(n, dtype=tdt, pin_memory=True)
    return t, t.numpy()


@pytest.mark.parametrize("off", [0, 1])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_pinned_and_pageable_transfers_agree(P, prec, off):
    d = I.discharge(n_cells=128, gap_m=0.025, p_Pa=60.0, V_rf_V=300.0, n_e0=50_000, n_i0=50_000, n_init_m3=4e14)
    sim = P.Simulation(X.he_like(eps_max_eV=600.0, de_eV=1e-2), d, precision=prec, sort_every=0)
    sim.step(5)  # region layout: five sweeps, no sort
    dt = np.float64 if prec == "fp64" else np.float32
    keep = []
    for sp in (0, 1):
        ref = sim.get_state(0, sp)  # pageable: staged path
        n = ref["c"].size
        out = {}
        for k, t in (("c", np.int32), ("f", dt), ("vx", dt), ("vy", dt), ("vz", dt)):
            tt, a = _pinned(n + 7, t)
            keep.append(tt)
            a[:] = 0
            out[k] = a[off:]
        got = sim.get_state(0, sp, out=out)  # pinned: direct path
        for k in ref:
            assert np.array_equal(got[k], ref[k]), (sp, k)
        # upload from the pinned arrays (direct) and read back through pageable staging: first a
        # ragged count (3 past a 16-byte group), then the whole state
        m = 4 * (n // 4) - 1
        sim.set_state(0, sp, {k: v[:m] for k, v in got.items()})
        back = sim.get_state(0, sp)
        for k in ref:
            assert np.array_equal(back[k], ref[k][:m]), (sp, k)
        sim.set_state(0, sp, got)
        back = sim.get_state(0, sp)
        for k in ref:
            assert np.array_equal(back[k], ref[k]), (sp, k)
    sim.step(3)  # and the context steps on
    assert sim.count(0, 0) > 0
    sim.close()


def test_pinned_download_too_small_leaves_arrays_untouched(P):
    from paper_1608_04601_gb300 import _native as NV
    d = I.discharge(n_cells=64, gap_m=0.025, p_Pa=60.0, V_rf_V=300.0, n_e0=3000, n_i0=3000, n_init_m3=4e14)
    sim = P.Simulation(X.he_like(eps_max_eV=600.0, de_eV=1e-2), d, precision="fp32", sort_every=0)
    n = sim.count(0, 0)
    keep, out = [], {}
    for k, t in (("c", np.int32), ("f", np.float32), ("vx", np.float32), ("vy", np.float32), ("vz", np.float32)):
        tt, a = _pinned(n - 1, t)
        keep.append(tt)
        a[:] = 7
        out[k] = a
    with pytest.raises(NV.PicError):
        sim.get_state(0, 0, out=out)
    assert all(np.all(a == 7) for a in out.values())
    # and the context is still usable
    assert sim.get_state(0, 0)["c"].size == n
    sim.close()
