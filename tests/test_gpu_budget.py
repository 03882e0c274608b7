"""Allocation failure, injected on the host: a device-memory budget makes the
library's next allocation fail the way a failed cudaMalloc does (MSM_ENOMEM),
with no GPU fault.  The call that needed the memory fails cleanly, the handle
stays usable, and once there is room again the results are the bits a fresh
handle gives."""
import numpy as np
import pytest

from paper_1309_1889_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def api(torch):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1309_1889_gb300 import api as a
    return a


def test_budget_turns_the_next_allocation_into_enomem(api, torch):
    small = inputs.water_box(300, 1.5, margin=0.5, with_velocities=False)
    big = inputs.water_box(3000, 3.1, margin=0.5, with_velocities=False)
    try:
        m = api.MSM(a=1.2, h=0.25, levels=3, precision="fp32")
        e0, f0, p0 = m.energy_forces(small.pos, small.q, small.box)
        held = api.set_device_budget(0)
        assert held > 0
        api.set_device_budget(held + 1024)                 # no room for the larger system's buffers
        with pytest.raises(api.MSMError) as ei:
            m.energy_forces(big.pos, big.q, big.box)
        assert ei.value.code == -3 and "budget" in str(ei.value)
        # the handle stays usable within its buffers, and after the budget is lifted
        e1, f1, p1 = m.energy_forces(small.pos, small.q, small.box)
        api.set_device_budget(0)
        e2, f2, p2 = m.energy_forces(big.pos, big.q, big.box)
        ref = api.MSM(a=1.2, h=0.25, levels=3, precision="fp32").energy_forces(big.pos, big.q, big.box)
        assert float(e2) == float(ref[0]) and np.array_equal(f2, ref[1]) and np.array_equal(p2, ref[2])
        assert float(e1) == float(e0) and np.array_equal(f1, f0)
    finally:
        api.set_device_budget(0)
