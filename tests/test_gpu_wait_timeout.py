"""The bounded device-side wait (the mbarrier wait of the sweep's bulk-copy staging) runs out
cleanly: a barrier that nothing completes makes the wait give up after its poll limit, the call
reports PIC_ERR_TIMEOUT, and the device context stays usable (a simulation steps afterwards).
No fault, trap or hang is involved: the kernel returns on its own with nothing in flight."""
import pytest

import inputs as I
from paper_1608_04601_gb300 import xsections as X

pytestmark = pytest.mark.gpu


def test_wait_gives_up_and_reports_timeout():
    import __graft_entry__ as g
    g.build()
    from paper_1608_04601_gb300 import pic, _native as NV
    assert pic.debug_wait(False, 4096) == -4          # PIC_ERR_TIMEOUT
    assert pic.debug_wait(True, 4096) == NV.PIC_OK    # the same wait, completed by an arrival
    assert pic.debug_wait(False, 0) == -1             # poll limit out of range: rejected on the host
    d = I.discharge(n_cells=64, gap_m=0.025, V_rf_V=100.0, n_e0=2000, n_i0=2000, n_init_m3=2e14)
    sim = pic.Simulation(X.he_like(eps_max_eV=200.0, de_eV=1e-2), d, precision="fp32", sort_every=4)
    sim.step(20)
    assert sim.step_index == 20 and sim.count(0, 0) > 0
    sim.close()
