"""Batches of independent systems, CUDA-graph replay and the brick autotuner
through the C ABI.

The paper runs its fine propagators for independent time slices in parallel
(Sec. 4); the library's form of that is a batch: B systems of any sizes and
boxes evaluated by the same launches, one per stage.  Nothing in one system's
arithmetic depends on another system, on the brick shape the autotuner picks
or on whether a step was replayed from a CUDA graph, so every check here is
bitwise: a system inside a batch gives exactly the bits it gives alone.
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


def _dev(torch, s, with_force=False):
    t = lambda x: torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")
    d = inputs.System(pos=t(s.pos), q=t(s.q), mass=t(s.mass), box=s.box, vel=t(s.vel), n_mol=s.n_mol,
                      lj=torch.tensor(s.lj, device="cuda"))
    if with_force:
        d.force = torch.zeros_like(d.pos)
    return d


def _clouds():
    """Uneven point-charge systems: sizes and boxes differ, one is empty."""
    out = []
    for k, (n, L) in enumerate(((700, 2.6), (0, 1.5), (2400, 3.4), (1300, 3.0))):
        s = inputs.random_cloud(n, L, seed=20 + k, neutral=True, margin=0.3)
        out.append(s)
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_charges_equal_single_calls(api, torch, prec):
    systems = _clouds()
    m = api.MSM(a=A, h=H, levels=3, precision=prec)
    singles = [m.energy_forces(s.pos, s.q, s.box) for s in systems]
    offsets = np.cumsum([0] + [len(s.q) for s in systems])
    pos = np.concatenate([s.pos for s in systems]); q = np.concatenate([s.q for s in systems])
    boxes = np.stack([np.asarray(s.box, dtype=np.float64) for s in systems])
    mb = api.MSM(a=A, h=H, levels=3, precision=prec)
    e, f, p = mb.energy_forces_batched(offsets, pos, q, boxes)
    for b, (es, fs, ps) in enumerate(singles):
        o0, o1 = offsets[b], offsets[b + 1]
        assert e[b] == es
        assert np.array_equal(f[o0:o1], fs) and np.array_equal(p[o0:o1], ps)


def test_batch_uses_the_launches_of_one_system(api, torch):
    """One launch per stage for the whole batch: B systems cost the launches of one."""
    systems = [s for s in _clouds() if len(s.q)]
    m = api.MSM(a=A, h=H, levels=3, precision="fp32", autotune=False)
    s0 = systems[0]
    m.energy_forces(s0.pos, s0.q, s0.box)
    k0 = api.kernel_launches()
    m.energy_forces(s0.pos, s0.q, s0.box)
    single = api.kernel_launches() - k0
    offsets = np.cumsum([0] + [len(s.q) for s in systems])
    pos = np.concatenate([s.pos for s in systems]); q = np.concatenate([s.q for s in systems])
    boxes = np.stack([np.asarray(s.box, dtype=np.float64) for s in systems])
    mb = api.MSM(a=A, h=H, levels=3, precision="fp32", autotune=False)
    mb.energy_forces_batched(offsets, pos, q, boxes)
    k1 = api.kernel_launches()
    mb.energy_forces_batched(offsets, pos, q, boxes)
    batched = api.kernel_launches() - k1
    assert batched == single


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_water_forces_equal_single_calls(api, torch, prec):
    waters = [inputs.water_box(n, L, margin=0.6, seed=30 + k, vel_seed=40 + k)
              for k, (n, L) in enumerate(((600, 1.9), (1500, 2.5), (300, 1.5)))]
    kw = dict(a=A, h=H, levels=3, precision=prec, model="water", wall_k=1e4, wall_width=0.5)
    m = api.MSM(**kw)
    singles = [m.system_forces(_dev(torch, s)) for s in waters]
    devs = [_dev(torch, s, with_force=True) for s in waters]
    mb = api.MSM(**kw)
    e = mb.system_forces_batched(devs)
    for b, (es, fs, ps) in enumerate(singles):
        assert e[b] == float(es)
        assert torch.equal(devs[b].force, fs)
        assert devs[b].force_valid == 1 and devs[b].energy == float(es)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_md_run_batched_equals_single_runs(api, torch, prec):
    waters = [inputs.water_box(n, L, margin=0.8, seed=50 + k, vel_seed=60 + k)
              for k, (n, L) in enumerate(((450, 1.8), (1200, 2.4)))]
    kw = dict(a=A, h=H, levels=3, precision=prec, model="water", wall_k=1e4, wall_width=0.6)
    ref = []
    for s in waters:
        d = _dev(torch, s)
        uk = api.MSM(**kw).md_run(d, dt=0.002, n_steps=8)
        ref.append((d.pos.clone(), d.vel.clone(), uk.clone()))
    devs = [_dev(torch, s) for s in waters]
    uk = api.MSM(**kw).md_run_batched(devs, dt=0.002, n_steps=8)
    for b, (x, v, u) in enumerate(ref):
        assert torch.equal(devs[b].pos, x) and torch.equal(devs[b].vel, v)
        assert torch.equal(uk[b], u)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_replay_equals_eager_steps(api, torch, prec):
    s = inputs.water_box(900, 2.2, margin=0.8, seed=70, vel_seed=71)
    out = {}
    for graphs in (False, True):
        m = api.MSM(a=A, h=H, levels=3, precision=prec, model="water", wall_k=1e4, wall_width=0.6, graphs=graphs)
        d = _dev(torch, s)
        k0 = api.kernel_launches()
        uk = m.md_run(d, dt=0.002, n_steps=12)
        out[graphs] = (d.pos, d.vel, uk, api.kernel_launches() - k0)
    assert torch.equal(out[True][0], out[False][0]) and torch.equal(out[True][1], out[False][1])
    assert torch.equal(out[True][2], out[False][2])
    assert out[True][3] == out[False][3]            # replayed kernels are counted as launched


def test_graph_reused_across_calls_and_refreshed_when_inputs_move(api, torch):
    """A second md_run on the same arrays replays the cached graph; one on new
    arrays recaptures; both equal a graph-free run."""
    s = inputs.water_box(600, 1.9, margin=0.8, seed=72, vel_seed=73)
    kw = dict(a=A, h=H, levels=3, precision="fp32", model="water", wall_k=1e4, wall_width=0.6)
    m = api.MSM(**kw)
    ref = api.MSM(graphs=False, **kw)
    d1, r1 = _dev(torch, s), _dev(torch, s)
    for _ in range(2):
        m.md_run(d1, dt=0.002, n_steps=5, record=False)
        ref.md_run(r1, dt=0.002, n_steps=5, record=False)
    d2, r2 = _dev(torch, s), _dev(torch, s)
    m.md_run(d2, dt=0.002, n_steps=5, record=False)
    ref.md_run(r2, dt=0.002, n_steps=5, record=False)
    assert torch.equal(d1.pos, r1.pos) and torch.equal(d2.pos, r2.pos)


def test_autotuned_bricks_change_no_result(api, torch):
    """The brick shapes are timed only on the brick path (MSM_FLAG_BRICKS)."""
    s = inputs.water_box(3000, 3.1, margin=0.6, seed=74, vel_seed=75)
    res = {}
    for tune in (False, True):
        m = api.MSM(a=A, h=H, levels=3, precision="fp32", model="water", autotune=tune, bricks=True)
        e, f, p = m.system_forces(_dev(torch, s))
        res[tune] = (float(e), f, p)
    assert res[True][0] == res[False][0]
    assert torch.equal(res[True][1], res[False][1]) and torch.equal(res[True][2], res[False][2])


def test_uneven_water_batch_like_the_seven_cubes(api, torch):
    """The uneven-batch workload scaled down 40x: seven water cubes whose atom
    counts follow 20k : 50k : 100k : 150k : 200k : 230k : 250k, stepped as one
    batch; each equals its own run and keeps its rigid geometry."""
    sizes = (500, 1250, 2500, 3750, 5000, 5750, 6250)
    waters = [inputs.water_box(n, (n / 100.0) ** (1 / 3), margin=0.8, seed=80 + k, vel_seed=90 + k)
              for k, n in enumerate(sizes)]
    kw = dict(a=A, h=H, levels=3, precision="fp32", model="water", wall_k=1e4, wall_width=0.6)
    devs = [_dev(torch, s) for s in waters]
    api.MSM(**kw).md_run_batched(devs, dt=0.002, n_steps=4, record=False)
    for k in (0, 3, 6):
        d = _dev(torch, waters[k])
        api.MSM(**kw).md_run(d, dt=0.002, n_steps=4, record=False)
        assert torch.equal(devs[k].pos, d.pos)
    for s, d in zip(waters, devs):
        x = d.pos.cpu().numpy()[: 3 * s.n_mol].reshape(-1, 3, 3)
        oh = np.linalg.norm(x[:, 0] - x[:, 1], axis=1)
        assert np.abs(oh / inputs.D_OH - 1).max() < 2e-6


def test_batch_with_more_cells_than_one_scan_pass_holds(api, torch):
    """Two sparse 65 nm boxes (~18 M finest cells each, 36 M in the batch: the cell
    scan runs its block sums in several passes) give the bits they give alone."""
    systems = [inputs.random_cloud(3000, 65.0, seed=110 + k, neutral=True, margin=0.3) for k in range(2)]
    m = api.MSM(a=A, h=H, levels=6, precision="fp32", autotune=False)
    singles = [m.energy_forces(s.pos, s.q, s.box) for s in systems]
    offsets = np.cumsum([0] + [len(s.q) for s in systems])
    pos = np.concatenate([s.pos for s in systems]); q = np.concatenate([s.q for s in systems])
    boxes = np.stack([np.asarray(s.box, dtype=np.float64) for s in systems])
    mb = api.MSM(a=A, h=H, levels=6, precision="fp32", autotune=False)
    e, f, p = mb.energy_forces_batched(offsets, pos, q, boxes)
    for b, (es, fs, ps) in enumerate(singles):
        o0, o1 = offsets[b], offsets[b + 1]
        assert e[b] == es
        assert np.array_equal(f[o0:o1], fs) and np.array_equal(p[o0:o1], ps)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_beyond_one_group_of_plane_descriptors(api, torch, prec):
    """13 systems of 3 levels have 26 (system, level) lattice cutoffs, more than the
    24 TMA descriptors one launch carries: the lattice cutoff runs as two launches,
    and every system still gets exactly the bits it gets alone."""
    systems = [inputs.random_cloud(300 + 37 * k, 1.6 + 0.05 * k, seed=60 + k, neutral=True, margin=0.3)
               for k in range(13)]
    m = api.MSM(a=A, h=H, levels=3, precision=prec)
    singles = [m.energy_forces(s.pos, s.q, s.box) for s in systems]
    offsets = np.cumsum([0] + [len(s.q) for s in systems])
    pos = np.concatenate([s.pos for s in systems]); q = np.concatenate([s.q for s in systems])
    boxes = np.stack([np.asarray(s.box, dtype=np.float64) for s in systems])
    mb = api.MSM(a=A, h=H, levels=3, precision=prec)
    e, f, p = mb.energy_forces_batched(offsets, pos, q, boxes)
    for b, (es, fs, ps) in enumerate(singles):
        o0, o1 = offsets[b], offsets[b + 1]
        assert e[b] == es
        assert np.array_equal(f[o0:o1], fs) and np.array_equal(p[o0:o1], ps)
