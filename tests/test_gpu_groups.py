"""The pair passes' two ways of giving a warp its i atoms -- 32-atom groups cut
from columns of cells (the default) and bricks of cells (MSM_FLAG_BRICKS) -- give
the same bits: each i atom adds its in-range j atoms in ascending slot order
whatever set of rows its warp walks, and the j atoms a warp's box test drops or
keeps beyond a add exact zeros (Sec. 3, step 1).  Through the C ABI, both
precisions, point charges and the water model (Coulomb and LJ passes), ragged
boxes, a batch, dynamics and the 1M-atom box.
"""
import numpy as np
import pytest

from paper_1309_1889_gb300 import inputs

pytestmark = pytest.mark.gpu

A, H = 1.2, 0.25


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


def _dev(torch, x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def _sys(torch, s, vel=False):
    return inputs.System(pos=_dev(torch, s.pos), q=_dev(torch, s.q), mass=_dev(torch, s.mass), box=s.box,
                         vel=_dev(torch, s.vel) if vel else None, n_mol=s.n_mol,
                         lj=torch.tensor(s.lj, device="cuda"))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("case", ["water3k", "cloud_ragged", "cloud_flat", "cloud_one_column", "dense_small",
                                  "dense_layers", "sparse"])
def test_groups_and_bricks_give_the_same_short_range_bits(api, torch, prec, case):
    """Besides water and ragged clouds: a cloud dense enough that some cell layers of a
    column hold more atoms than a lane sorts by z (they keep the cell order), and a
    sparse box whose column width reaches its upper bound of 8 cells."""
    s = {"water3k": lambda: inputs.water_box(3000, 3.1, margin=0.5, with_velocities=False),
         "cloud_ragged": lambda: inputs.random_cloud(5003, (2.7, 3.3, 1.9), seed=8, margin=0.0),
         "cloud_flat": lambda: inputs.random_cloud(900, (5.0, 4.0, 0.2), seed=10, margin=0.0),
         "cloud_one_column": lambda: inputs.random_cloud(700, (0.4, 0.45, 6.0), seed=9, margin=0.0),
         "dense_small": lambda: inputs.random_cloud(400, (0.9, 0.8, 0.7), seed=11, margin=0.0),
         "dense_layers": lambda: inputs.random_cloud(6000, (1.5, 1.5, 1.5), seed=12, margin=0.0),
         "sparse": lambda: inputs.random_cloud(150, (6.0, 6.0, 6.0), seed=13, margin=0.0)}[case]()
    out = []
    for bricks in (False, True):
        m = api.MSM(a=A, h=H, levels=3, precision=prec, bricks=bricks)
        e, f, p = m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
        out.append((float(e), f, p) + tuple(m.stage_atoms(s.n)))
    assert out[0][0] == out[1][0]
    assert torch.equal(out[0][1], out[1][1]) and torch.equal(out[0][2], out[1][2])
    assert np.array_equal(out[0][3], out[1][3]) and np.array_equal(out[0][4], out[1][4])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_groups_and_bricks_give_the_same_water_model_bits(api, torch, prec):
    """Coulomb pass and the LJ pass over the LJ-site cell list."""
    s = inputs.water_box(3000, 3.1, margin=0.5, seed=12, with_velocities=False)
    out = []
    for bricks in (False, True):
        m = api.MSM(a=A, h=H, levels=3, precision=prec, model="water", wall_k=5000.0, wall_width=0.6, bricks=bricks)
        out.append(m.system_forces(_sys(torch, s)))
    assert float(out[0][0]) == float(out[1][0])
    assert torch.equal(out[0][1], out[1][1]) and torch.equal(out[0][2], out[1][2])


def test_groups_and_bricks_give_the_same_trajectories_and_batches(api, torch):
    waters = [inputs.water_box(n, (n / 100.0) ** (1 / 3), margin=0.8, seed=60 + n, vel_seed=61 + n)
              for n in (600, 1500, 2400)]
    kw = dict(a=A, h=H, levels=3, precision="fp32", model="water", wall_k=1e4, wall_width=0.6)
    res = []
    for bricks in (False, True):
        devs = [_sys(torch, s, vel=True) for s in waters]
        uk = api.MSM(bricks=bricks, **kw).md_run_batched(devs, dt=0.002, n_steps=6)
        res.append((devs, uk))
    for d0, d1 in zip(res[0][0], res[1][0]):
        assert torch.equal(d0.pos, d1.pos) and torch.equal(d0.vel, d1.vel)
    for u0, u1 in zip(res[0][1], res[1][1]):
        assert torch.equal(u0, u1)


def test_groups_and_bricks_give_the_same_bits_at_full_size(api, torch):
    """1,000,000 atoms in a 21.5 nm water box, 5 levels, FP32, water model."""
    cfg = inputs.WORKLOADS["water1M"]
    s = inputs.water_box(cfg["n_atoms"], cfg["region"], margin=0.5, with_velocities=False)
    out = []
    for bricks in (False, True):
        m = api.MSM(a=A, h=H, levels=cfg["levels"], precision="fp32", model="water", bricks=bricks)
        e, f, p = m.system_forces(_sys(torch, s))
        out.append((float(e), f, p))
        del m
    assert out[0][0] == out[1][0]
    assert torch.equal(out[0][1], out[1][1]) and torch.equal(out[0][2], out[1][2])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_autotuned_group_widths_change_no_result(api, torch, prec):
    """The autotuner times the group column widths around the density heuristic on the
    first evaluation of a geometry (Coulomb and LJ passes); whichever it keeps, the
    results are the untuned ones, on that evaluation and on the next."""
    s = inputs.water_box(3000, 3.1, margin=0.6, seed=74, vel_seed=75)
    res = {}
    for tune in (False, True):
        m = api.MSM(a=A, h=H, levels=3, precision=prec, model="water", autotune=tune)
        res[tune] = [m.system_forces(_sys(torch, s)) for _ in range(2)]
    for k in range(2):
        assert float(res[True][k][0]) == float(res[False][k][0])
        assert torch.equal(res[True][k][1], res[False][k][1]) and torch.equal(res[True][k][2], res[False][k][2])
