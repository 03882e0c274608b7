"""msm_cell_list_noalloc: the cell binning for callers that must not allocate
device memory (their device memory belongs to another allocator with a fixed
budget, or they cannot afford cudaMalloc's device-wide synchronisation).  Its
scratch is a static array inside the library, so two calls in a row must
still each produce exactly the cell list of the regular path: the second call
must not see the first call's leftovers.

Collected last on purpose (file name), so a run stopping at its first failure
has already run every other test.  Runs alone in a fresh process too.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1309_1889_gb300 import inputs

pytestmark = pytest.mark.gpu

H = 0.25


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


def _regular(api, torch, s):
    """Cell list of the regular (allocating) path: one evaluation, then msm_cell_list."""
    m = api.MSM(a=1.2, h=H, levels=3, precision="fp32")
    d = lambda x: torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")
    m.energy_forces(d(s.pos), d(s.q), s.box)
    perm, start = m.cell_list(s.n)
    m.close()
    return perm, start


def _noalloc(api, torch, s):
    nc = [int(np.floor(s.box[3 + k] / H)) + 1 for k in range(3)]
    ncells = nc[0] * nc[1] * nc[2]
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    perm = torch.full((s.n,), -7, dtype=torch.int32, device="cuda")
    start = torch.full((ncells + 1,), -7, dtype=torch.int32, device="cuda")
    box = (C.c_double * 6)(*[float(v) for v in s.box])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = api.lib().msm_cell_list_noalloc(s.n, C.c_void_p(pos.data_ptr()), box, H, C.c_void_p(perm.data_ptr()),
                                         C.c_void_p(start.data_ptr()), ncells + 1, stream)
    assert rc == 0, api.lib().msm_last_error().decode()
    return perm.cpu().numpy().astype(np.int64), start.cpu().numpy().astype(np.int64)


def test_noalloc_cell_list_equals_regular_path_on_two_calls_in_a_row(api, torch):
    first = inputs.water_box(3000, 3.1, margin=0.5, with_velocities=False)
    second = inputs.random_cloud(5003, (2.7, 3.3, 1.9), seed=8, margin=0.0)   # other box, other cell count
    ref1 = _regular(api, torch, first)
    ref2 = _regular(api, torch, second)
    got1 = _noalloc(api, torch, first)
    got2 = _noalloc(api, torch, second)
    assert np.array_equal(got1[0], ref1[0]) and np.array_equal(got1[1], ref1[1])
    assert np.array_equal(got2[0], ref2[0]) and np.array_equal(got2[1], ref2[1])
    # and once more on the first system after the second one filled the scratch
    got3 = _noalloc(api, torch, first)
    assert np.array_equal(got3[0], ref1[0]) and np.array_equal(got3[1], ref1[1])


def test_noalloc_rejects_oversized_requests(api, torch):
    s = inputs.random_cloud(10, 1.0, seed=1)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    perm = torch.empty(10, dtype=torch.int32, device="cuda")
    start = torch.empty(8, dtype=torch.int32, device="cuda")
    big = (C.c_double * 6)(0, 0, 0, 100.0, 100.0, 100.0)     # 401^3 cells: far beyond the fixed scratch
    rc = api.lib().msm_cell_list_noalloc(10, C.c_void_p(pos.data_ptr()), big, H, C.c_void_p(perm.data_ptr()),
                                         C.c_void_p(start.data_ptr()), 401 ** 3 + 1, None)
    assert rc == -1 and b"scratch" in api.lib().msm_last_error()


def _noalloc_rc(api, torch, pos_np, box, ncells):
    pos = torch.tensor(pos_np, dtype=torch.float64, device="cuda")
    n = pos_np.shape[0]
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    start = torch.empty(ncells + 1, dtype=torch.int32, device="cuda")
    cbox = (C.c_double * 6)(*[float(v) for v in box])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return api.lib().msm_cell_list_noalloc(n, C.c_void_p(pos.data_ptr()), cbox, H, C.c_void_p(perm.data_ptr()),
                                           C.c_void_p(start.data_ptr()), ncells + 1, stream)


def test_noalloc_recovers_after_failed_calls(api, torch):
    """A call that fails on the device (an atom outside the box, a NaN coordinate)
    leaves its status word and histogram in the shared array; the next valid call
    must clear them and still give the regular path's cell list bit for bit."""
    s = inputs.water_box(3000, 3.1, margin=0.5, with_velocities=False)
    ref = _regular(api, torch, s)
    nc = [int(np.floor(s.box[3 + k] / H)) + 1 for k in range(3)]
    ncells = nc[0] * nc[1] * nc[2]
    bad = s.pos.copy(); bad[123, 1] = s.box[1] - 0.01                  # below the box
    assert _noalloc_rc(api, torch, bad, s.box, ncells) == -2           # MSM_ERANGE
    got = _noalloc(api, torch, s)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    bad = s.pos.copy(); bad[7, 0] = np.nan
    assert _noalloc_rc(api, torch, bad, s.box, ncells) == -1           # MSM_EINVAL
    got = _noalloc(api, torch, s)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_noalloc_rejects_arrays_of_another_gpu(api, torch):
    """Arrays allocated on a GPU other than the current one are refused before any launch."""
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    s = inputs.random_cloud(10, 1.0, seed=1)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda:1")
    perm = torch.empty(10, dtype=torch.int32, device="cuda:0")
    start = torch.empty(6 ** 3 + 1, dtype=torch.int32, device="cuda:0")
    with torch.cuda.device(0):
        box = (C.c_double * 6)(*[float(v) for v in s.box])
        rc = api.lib().msm_cell_list_noalloc(10, C.c_void_p(pos.data_ptr()), box, H, C.c_void_p(perm.data_ptr()),
                                             C.c_void_p(start.data_ptr()), 6 ** 3 + 1, None)
    assert rc == -1 and b"current device" in api.lib().msm_last_error()
