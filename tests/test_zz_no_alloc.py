"""The allocation-free sort (pic_sort_noalloc) against the context sort (pic_sort).

pic_sort_noalloc exists for callers that cannot allocate device memory while they run; it takes
its scratch from a fixed array inside the library. The GPU test hands it caller-owned device
buffers (torch tensors) holding a particle store, and checks its output against what the
existing entry point pic_sort produces for the same store, bit for bit, on two calls in a row
with different inputs (so stale scratch from the first call cannot pass as a result). The large
case has more sort tiles than the kernels' grid has CTAs, so every CTA takes several tiles.
The argument checks run on the CPU: they return before any CUDA call.
The file name makes pytest collect it last.
"""
import ctypes as C

import numpy as np
import pytest


def _records(st, dtype):
    return np.ascontiguousarray(np.stack([st["f"], st["vx"], st["vy"], st["vz"]], 1).astype(dtype))


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("n,cells", [(60000, 128), (3_000_000, 512)])
def test_noalloc_sort_matches_context_sort_twice(prec, n, cells):
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1608_04601_gb300 import _native as NV, pic, xsections as X
    from paper_1608_04601_gb300.workloads import c1

    lib = NV.lib()
    dtype = np.float32 if prec == "fp32" else np.float64
    tdtype = torch.float32 if prec == "fp32" else torch.float64
    code = pic.FP32 if prec == "fp32" else pic.FP64
    d = c1().scaled(n_e0=n, n_i0=n, n_cells=cells, V_rf_V=300.0)
    gas = X.he_like(eps_max_eV=300.0, de_eV=1e-2)
    sim = pic.Simulation(gas, d, precision=prec, sort_every=0)
    stream = torch.cuda.current_stream().cuda_stream
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tiles = (n + 4095) // 4096
    if n > 1_000_000:
        assert tiles > 2 * sms  # grid-stride loop: every CTA sorts more than one tile
    for call in range(2):
        sim.step(1 + 2 * call)  # the load is unsorted; a different unsorted store on each call
        before = sim.get_state(0, 0)
        m = before["c"].size
        # existing entry point: sort inside the context
        sim.sort()
        expect = sim.get_state(0, 0)
        # allocation-free entry point on caller-owned device buffers
        c_in = torch.from_numpy(before["c"]).cuda()
        r_in = torch.from_numpy(_records(before, dtype)).cuda()
        c_out = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        r_out = torch.zeros((m, 4), dtype=tdtype, device="cuda")
        st = lib.pic_sort_noalloc(C.c_void_p(c_in.data_ptr()), C.c_void_p(r_in.data_ptr()),
                                  C.c_void_p(c_out.data_ptr()), C.c_void_p(r_out.data_ptr()), m, d.n_cells, code,
                                  C.c_void_p(stream))
        assert st == 0, NV.STATUS.get(st, st)
        torch.cuda.synchronize()
        got_c = c_out.cpu().numpy()
        got_r = r_out.cpu().numpy()
        assert np.array_equal(got_c, expect["c"]), f"call {call}: cells/order differ"
        assert np.array_equal(got_r, _records(expect, dtype)), f"call {call}: records differ"
        assert np.all(np.diff(got_c) >= 0)
    sim.close()


def test_noalloc_sort_rejects_bad_arguments_before_any_launch():
    """Sizes beyond the scratch, a zero cell count and misaligned buffers are refused on the host,
    before any CUDA call (the pointers below are never dereferenced)."""
    import __graft_entry__ as g
    g.build()
    from paper_1608_04601_gb300 import _native as NV
    lib = NV.lib()
    ok = C.c_void_p(1 << 12)
    # 4096 cells x (1 + 512 tiles) words exceed the 4 MiB scratch
    st = lib.pic_sort_noalloc(ok, ok, ok, ok, 512 * 4096, 4096, 0, None)
    assert NV.STATUS[st] == "PIC_ERR_CAPACITY"
    assert NV.STATUS[lib.pic_sort_noalloc(None, None, None, None, 10, 0, 0, None)] == "PIC_ERR_ARG"
    # records must be 16-byte aligned (FP32) or 32-byte aligned (FP64), cells 4-byte aligned
    odd8, odd16, odd2 = C.c_void_p((1 << 12) + 8), C.c_void_p((1 << 12) + 16), C.c_void_p((1 << 12) + 2)
    assert NV.STATUS[lib.pic_sort_noalloc(ok, odd8, ok, ok, 10, 16, 0, None)] == "PIC_ERR_ARG"
    assert NV.STATUS[lib.pic_sort_noalloc(ok, ok, ok, odd8, 10, 16, 0, None)] == "PIC_ERR_ARG"
    assert NV.STATUS[lib.pic_sort_noalloc(ok, odd16, ok, ok, 10, 16, 1, None)] == "PIC_ERR_ARG"
    assert NV.STATUS[lib.pic_sort_noalloc(odd2, ok, ok, ok, 10, 16, 0, None)] == "PIC_ERR_ARG"
    assert NV.STATUS[lib.pic_sort_noalloc(ok, ok, odd2, ok, 10, 16, 0, None)] == "PIC_ERR_ARG"
