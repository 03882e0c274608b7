"""The FP32 short-range passes on packed FP32x2 pairs against the scalar loop.

The packed step does, for each of its two queued neighbours, the IEEE
operations of the scalar loop in the same order, and every accumulator still
takes one neighbour at a time in queue order; so the two give the same bits,
for the short-range sums themselves and for everything computed from them
(the water model's totals include the O-O Lennard-Jones pass).
MSM_FLAG_SCALAR_PAIRS selects the scalar loop.  The cases cover odd queue
tails (the packed step then reads one pad entry of charge zero), systems with
no pair at all, both models, a batch of uneven systems and the 1,000,000-atom
water box in the launch configuration of the timed run.
"""
import numpy as np
import pytest

from paper_1309_1889_gb300 import inputs

pytestmark = pytest.mark.gpu

A, H = 1.2, 0.25
WALL = dict(wall_k=1.0e4, wall_width=0.8)


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


def _bits(x):
    x = x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)
    return np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)


def _same(a, b):
    return np.array_equal(_bits(a), _bits(b))


def _water_dev(torch, s):
    t = lambda x: torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")
    return inputs.System(pos=t(s.pos), q=t(s.q), mass=t(s.mass), box=s.box, vel=t(s.vel), n_mol=s.n_mol,
                         lj=torch.tensor(s.lj, device="cuda"))


def _eval(api, torch, s, model, scalar, levels=3):
    m = api.MSM(a=A, h=H, levels=levels, precision="fp32", model=model, scalar_pairs=scalar, **WALL)
    if model == "water":
        e, f, p = m.system_forces(_water_dev(torch, s))
    else:
        e, f, p = m.energy_forces(s.pos, s.q, s.box)
    torch.cuda.synchronize()
    phi_s, f_s = m.stage_atoms(len(s.q))
    m.close()
    return dict(e=np.array([float(e)]), f=_bits(f), p=_bits(p), phi_short=phi_s, f_short=f_s)


@pytest.mark.parametrize("n,L,seed", [(1, 2.0, 1), (2, 0.5, 2), (7, 1.0, 3), (333, 2.2, 4), (2401, 3.4, 5),
                                      (5000, 3.9, 6)])
def test_charges_packed_equal_scalar(api, torch, n, L, seed):
    s = inputs.random_cloud(n, L, seed=seed, neutral=n > 1, margin=0.3)
    pk, sc = _eval(api, torch, s, "charges", False), _eval(api, torch, s, "charges", True)
    for k in pk:
        assert _same(pk[k], sc[k]), k
    if n > 1:
        assert np.any(pk["phi_short"] != 0)


@pytest.mark.parametrize("n,L", [(3000, 3.1), (20_000, 5.9)])
def test_water_packed_equal_scalar(api, torch, n, L):
    s = inputs.water_box(n, L, margin=1.0, seed=11, vel_seed=12)
    pk, sc = _eval(api, torch, s, "water", False), _eval(api, torch, s, "water", True)
    for k in pk:
        assert _same(pk[k], sc[k]), k


def test_batch_packed_equal_scalar(api, torch):
    systems = [inputs.random_cloud(n, L, seed=40 + k, neutral=True, margin=0.3)
               for k, (n, L) in enumerate(((701, 2.6), (0, 1.5), (2399, 3.4), (1303, 3.0)))]
    offsets = np.cumsum([0] + [len(s.q) for s in systems])
    pos = np.concatenate([s.pos for s in systems]); q = np.concatenate([s.q for s in systems])
    boxes = [s.box for s in systems]
    out = []
    for scalar in (False, True):
        m = api.MSM(a=A, h=H, levels=3, precision="fp32", scalar_pairs=scalar)
        out.append(m.energy_forces_batched(offsets, pos, q, boxes))
        m.close()
    for x, y in zip(out[0], out[1]):
        assert _same(x, y)


def test_water1M_packed_equal_scalar(api, torch):
    """The 1,000,000-atom box of the timed run (5 levels), autotuned bricks."""
    s = inputs.water_box(1_000_000, 21.5, margin=1.0, seed=0, vel_seed=1)
    pk, sc = _eval(api, torch, s, "water", False, levels=5), _eval(api, torch, s, "water", True, levels=5)
    for k in pk:
        assert _same(pk[k], sc[k]), k
