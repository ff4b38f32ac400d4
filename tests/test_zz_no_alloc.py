"""The allocation-free sort (pic_sort_noalloc) against the context sort (pic_sort).

pic_sort_noalloc exists for callers that cannot allocate device memory while they run; it takes
its scratch from a fixed array inside the library. This test hands it caller-owned device
buffers (torch tensors) holding a particle store, and checks its output against what the
existing entry point pic_sort produces for the same store, bit for bit, on two calls in a row
with different inputs (so stale scratch from the first call cannot pass as a result).
The file name makes pytest collect it last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _records(st, dtype):
    return np.ascontiguousarray(np.stack([st["f"], st["vx"], st["vy"], st["vz"]], 1).astype(dtype))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_sort_matches_context_sort_twice(prec):
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1608_04601_gb300 import _native as NV, pic, xsections as X
    from paper_1608_04601_gb300.workloads import c1

    lib = NV.lib()
    dtype = np.float32 if prec == "fp32" else np.float64
    tdtype = torch.float32 if prec == "fp32" else torch.float64
    code = pic.FP32 if prec == "fp32" else pic.FP64
    d = c1().scaled(n_e0=60000, n_i0=60000, V_rf_V=300.0)
    gas = X.he_like(eps_max_eV=300.0, de_eV=1e-2)
    sim = pic.Simulation(gas, d, precision=prec, sort_every=0)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        sim.step(3 + 5 * call)  # unsorted store, different on each call
        before = sim.get_state(0, 0)
        n = before["c"].size
        # existing entry point: sort inside the context
        sim.sort()
        expect = sim.get_state(0, 0)
        # allocation-free entry point on caller-owned device buffers
        c_in = torch.from_numpy(before["c"]).cuda()
        r_in = torch.from_numpy(_records(before, dtype)).cuda()
        c_out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        r_out = torch.zeros((n, 4), dtype=tdtype, device="cuda")
        st = lib.pic_sort_noalloc(C.c_void_p(c_in.data_ptr()), C.c_void_p(r_in.data_ptr()),
                                  C.c_void_p(c_out.data_ptr()), C.c_void_p(r_out.data_ptr()), n, d.n_cells, code,
                                  C.c_void_p(stream))
        assert st == 0, NV.STATUS.get(st, st)
        torch.cuda.synchronize()
        got_c = c_out.cpu().numpy()
        got_r = r_out.cpu().numpy()
        assert np.array_equal(got_c, expect["c"]), f"call {call}: cells/order differ"
        assert np.array_equal(got_r, _records(expect, dtype)), f"call {call}: records differ"
        assert np.all(np.diff(got_c) >= 0)
    sim.close()


def test_noalloc_sort_rejects_sizes_beyond_its_scratch():
    import __graft_entry__ as g
    g.build()
    from paper_1608_04601_gb300 import _native as NV
    lib = NV.lib()
    # 4096 cells x (1 + 512 tiles) words exceed the 4 MiB scratch; rejected before any launch
    st = lib.pic_sort_noalloc(C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), 512 * 4096, 4096, 0,
                              None)
    assert NV.STATUS[st] == "PIC_ERR_CAPACITY"
    assert NV.STATUS[lib.pic_sort_noalloc(None, None, None, None, 10, 0, 0, None)] == "PIC_ERR_ARG"
