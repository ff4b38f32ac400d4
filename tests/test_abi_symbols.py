"""The C-ABI library loads and exports every entry point include/pic.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b((?:pic|mlp)_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("pic_create", "pic_batch_create", "pic_step", "pic_moments", "pic_destroy", "pic_sweep",
                 "pic_solve", "pic_sort", "pic_sync", "mlp_create", "mlp_forward", "mlp_loss_grad", "mlp_adam"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1608_04601_gb300 import build as B
    lib_path = B.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_prototypes_cover_the_header():
    from paper_1608_04601_gb300 import _native as NV
    assert set(_declared()) <= set(NV.PROTOTYPES), set(_declared()) - set(NV.PROTOTYPES)


def test_struct_layouts_match_header_sizes():
    """The binding's structures have the sizes of the C structures (checked by a tiny host-only C program)."""
    import subprocess
    import tempfile
    from paper_1608_04601_gb300 import _native as NV
    src = r'''
#include <stdio.h>
#include "pic.h"
int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(pic_gas), sizeof(pic_weights), sizeof(pic_discharge),
 sizeof(pic_options), sizeof(pic_moments_t), sizeof(pic_counters), sizeof(pic_derived));return 0;}
'''
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "s.c")
        exe = os.path.join(td, "s")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    py = [ctypes.sizeof(t) for t in (NV.PicGas, NV.PicWeights, NV.PicDischarge, NV.PicOptions, NV.PicMoments,
                                     NV.PicCounters, NV.PicDerived)]
    assert sizes == py


def test_oracle_and_library_share_no_code():
    """The oracle sources include nothing of the library and vice versa."""
    lib_dir = os.path.join(ROOT, "paper_1608_04601_gb300")
    for dp, _, fs in os.walk(lib_dir):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                t = open(os.path.join(dp, f)).read()
                assert "oracle" not in re.findall(r"^\s*(?:from|import|#include)\s+\S*", t, flags=re.M).__str__()
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".h", ".py")):
            t = open(os.path.join(ROOT, "oracle", f)).read()
            assert "pic_internal" not in t and "paper_1608_04601_gb300.pic" not in t and "pic.h\"" not in t
