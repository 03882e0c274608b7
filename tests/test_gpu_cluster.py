"""GPU parity of the cluster-pair short-range pass (MSM_FLAG_CLUSTER_PAIRS, FP32)
against the FP64 oracle (Sec. 3, step 1: the g* sum over pairs within a), and its
own invariants, through the C ABI.

Bars as for the default pass in test_gpu_msm.py: relative RMS <= 1e-4 for the
short-range potentials and forces, each atom within 2e-3 of the RMS magnitude,
whole-MSM energy within 1e-6 |U|.  Batching, repetition and graph replay are
bitwise.
"""
import numpy as np
import pytest

import oracle
from paper_1309_1889_gb300 import inputs

pytestmark = pytest.mark.gpu

A, H = 1.2, 0.25
TOL = dict(f=1e-4, p=1e-4, e=1e-6, fmax=2e-3)


def rel_rms(x, ref):
    x = np.asarray(x, dtype=np.float64); ref = np.asarray(ref, dtype=np.float64)
    den = np.sqrt((ref ** 2).sum())
    return float(np.sqrt(((x - ref) ** 2).sum()) / (den if den > 0 else 1.0))


def max_rel(x, ref):
    x = np.asarray(x, dtype=np.float64); ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim == 1:
        x, ref = x[:, None], ref[:, None]
    rms = np.sqrt((ref ** 2).sum(1).mean())
    return float(np.linalg.norm(x - ref, axis=1).max() / (rms if rms > 0 else 1.0))


def check_short(phi, f, ophi, of):
    assert rel_rms(phi, ophi) <= TOL["p"] and max_rel(phi, ophi) <= TOL["fmax"]
    assert rel_rms(f, of) <= TOL["f"] and max_rel(f, of) <= TOL["fmax"]


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


def _cp(api, **kw):
    kw.setdefault("a", A); kw.setdefault("h", H); kw.setdefault("levels", 3)
    return api.MSM(precision="fp32", cluster_pairs=True, **kw)


@pytest.mark.parametrize("case", ["water3k", "cloud_ragged", "cloud_one_column", "cloud_flat", "dense_small"])
def test_cluster_short_range_matches_oracle(api, torch, case):
    """Boxes whose cell counts are odd (a last column of one cell), a box one column
    wide, a flat box one cell layer thick in z, and a box smaller than the cutoff."""
    s = {"water3k": lambda: inputs.water_box(3000, 3.1, margin=0.5, with_velocities=False),
         "cloud_ragged": lambda: inputs.random_cloud(5003, (2.7, 3.3, 1.9), seed=8, margin=0.0),
         "cloud_one_column": lambda: inputs.random_cloud(700, (0.4, 0.45, 6.0), seed=9, margin=0.0),
         "cloud_flat": lambda: inputs.random_cloud(900, (5.0, 4.0, 0.2), seed=10, margin=0.0),
         "dense_small": lambda: inputs.random_cloud(400, (0.9, 0.8, 0.7), seed=11, margin=0.0)}[case]()
    m = _cp(api)
    m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
    phi, f = m.stage_atoms(s.n)
    ophi, of = oracle.short_range(s.pos, s.q, A, s.box)
    check_short(phi, f, ophi, of)


def test_cluster_long_cutoff_takes_the_runs_in_segments(api, torch):
    """a = 2.4 nm on h = 0.2 nm cells: ~14 x 14 candidate columns per cluster, more than
    the run list holds, so the runs are taken in segments."""
    a, h = 2.4, 0.2
    s = inputs.random_cloud(3000, (4.0, 4.0, 4.0), seed=41, neutral=True, margin=0.2)
    m = _cp(api, a=a, h=h, levels=1)
    e, f, p = m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
    phi, fs = m.stage_atoms(s.n)
    ophi, of = oracle.short_range(s.pos, s.q, a, s.box)
    check_short(phi, fs, ophi, of)
    ref = oracle.msm(s.pos, s.q, s.box, a, h, 1)
    assert abs(float(e) - ref["energy"]) <= TOL["e"] * abs(ref["energy"])


@pytest.mark.parametrize("n", [1, 2, 9])
def test_cluster_tiny_systems(api, torch, n):
    s = inputs.random_cloud(n, (1.0, 1.0, 1.0), seed=100 + n, margin=0.1)
    m = _cp(api)
    m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
    phi, f = m.stage_atoms(s.n)
    ophi, of = oracle.short_range(s.pos, s.q, A, s.box)
    if n == 1:
        assert np.all(phi == 0) and np.all(f == 0)
    else:
        check_short(phi, f, ophi, of)


def test_cluster_empty_system(api, torch):
    m = _cp(api)
    e, f, p = m.energy_forces(np.zeros((0, 3)), np.zeros(0), [0, 0, 0, 2.0, 2.0, 2.0])
    assert e == 0.0 and f.shape == (0, 3)


def test_cluster_water_model_matches_oracle(api, torch):
    s = inputs.water_box(900, 2.1, margin=0.5, with_velocities=False)
    ref = oracle.model_forces(s, A, H, 3, wall_k=5000.0, wall_width=0.6)
    m = _cp(api, model="water", wall_k=5000.0, wall_width=0.6)
    sd = inputs.System(pos=_dev(torch, s.pos), q=_dev(torch, s.q), mass=_dev(torch, s.mass), box=s.box,
                       n_mol=s.n_mol, lj=torch.tensor(s.lj, device="cuda"))
    e, f, p = m.system_forces(sd)
    assert abs(float(e) - ref["energy"]) <= TOL["e"] * abs(ref["energy"])
    f, p = f.cpu().numpy(), p.cpu().numpy()
    assert rel_rms(f, ref["forces"]) <= TOL["f"] and max_rel(f, ref["forces"]) <= TOL["fmax"]
    assert rel_rms(p, ref["pot"]) <= TOL["p"] and max_rel(p, ref["pot"]) <= TOL["fmax"]


def test_cluster_simple_cutoff_matches_oracle(api, torch):
    s = inputs.water_box(3000, 3.1, margin=0.5, with_velocities=False)
    ref = oracle.cutoff(s.pos, s.q, 0.9, "cutoff")
    m = _cp(api, a=0.9, method="cutoff")
    e, f, p = m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
    assert abs(float(e) - ref["energy"]) <= TOL["e"] * abs(ref["energy"])
    f = f.cpu().numpy()
    assert rel_rms(f, ref["forces"]) <= TOL["f"] and max_rel(f, ref["forces"]) <= TOL["fmax"]


def test_cluster_and_default_passes_agree_to_rounding(api, torch):
    """The cluster pairs and the default 32-atom groups sum the same terms in different orders."""
    s = inputs.water_box(3000, 3.1, margin=0.5, with_velocities=False)
    out = []
    for cp in (False, True):
        m = api.MSM(a=A, h=H, levels=3, precision="fp32", cluster_pairs=cp)
        m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
        out.append(m.stage_atoms(s.n))
    assert rel_rms(out[1][0], out[0][0]) <= 1e-5 and rel_rms(out[1][1], out[0][1]) <= 1e-5
    assert not (np.array_equal(out[1][0], out[0][0]) and np.array_equal(out[1][1], out[0][1]))


def test_cluster_batch_and_repeats_are_bitwise(api, torch):
    systems = [inputs.random_cloud(n, L, seed=n, margin=0.2) for n, L in ((100, 1.5), (731, 2.4), (2050, 2.9))]
    offs = np.cumsum([0] + [s.n for s in systems])
    pos = np.concatenate([s.pos for s in systems]); q = np.concatenate([s.q for s in systems])
    boxes = np.stack([s.box for s in systems])
    m = _cp(api)
    e, f, p = m.energy_forces_batched(offs, _dev(torch, pos), _dev(torch, q), boxes)
    for k, s in enumerate(systems):
        e1, f1, p1 = m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
        e2, f2, p2 = m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
        assert float(e[k]) == float(e1) == float(e2)
        assert torch.equal(f[offs[k]:offs[k + 1]], f1) and torch.equal(f1, f2)
        assert torch.equal(p[offs[k]:offs[k + 1]], p1) and torch.equal(p1, p2)


def test_cluster_md_follows_oracle_and_replays_bitwise(api, torch):
    s = inputs.water_box(600, 1.8, margin=0.5, seed=3, vel_seed=4)
    ox, ov, ouk = oracle.md_run(s, a=A, h=H, levels=3, dt=0.002, n_steps=8, wall_k=1e4, wall_width=0.4)
    res = []
    for graphs in (True, False):
        m = _cp(api, model="water", graphs=graphs, wall_k=1e4, wall_width=0.4)
        d = inputs.System(pos=_dev(torch, s.pos), q=_dev(torch, s.q), mass=_dev(torch, s.mass), box=s.box,
                          vel=_dev(torch, s.vel), n_mol=s.n_mol, lj=torch.tensor(s.lj, device="cuda"))
        uk = m.md_run(d, dt=0.002, n_steps=8)
        res.append((d.pos.clone(), d.vel.clone(), uk.clone()))
    for u, v in zip(*res):
        assert torch.equal(u, v)
    assert np.abs(res[0][0].cpu().numpy() - ox).max() <= 1e-5
    assert np.abs(res[0][2].cpu().numpy() - ouk).max() <= 1e-5 * np.abs(ouk).max()


def test_cluster_full_size_rows_match_oracle(api, torch):
    """1,000,000 atoms in a 21.5 nm water box, 5 levels: sampled short-range rows
    against the oracle; the whole FP32 result against the FP64 path."""
    cfg = inputs.WORKLOADS["water1M"]
    s = inputs.water_box(cfg["n_atoms"], cfg["region"], margin=0.5, with_velocities=False)
    pos, q = _dev(torch, s.pos), _dev(torch, s.q)
    m32 = _cp(api, levels=cfg["levels"])
    e32, f32, p32 = m32.energy_forces(pos, q, s.box)
    phi32, fs32 = m32.stage_atoms(s.n)
    rng = np.random.default_rng(2)
    tg = rng.choice(s.n, 512, replace=False)
    ophi, of = oracle.short_range(s.pos, s.q, A, s.box, targets=tg)
    assert rel_rms(phi32[tg], ophi) <= 1e-4 and rel_rms(fs32[tg], of) <= 1e-4
    assert max_rel(phi32[tg], ophi) <= TOL["fmax"] and max_rel(fs32[tg], of) <= TOL["fmax"]
    del m32
    m64 = api.MSM(a=A, h=H, levels=cfg["levels"], precision="fp64")
    e64, f64, p64 = m64.energy_forces(pos, q, s.box)
    assert abs(float(e32) - float(e64)) <= 1e-6 * abs(float(e64))
    f32, f64 = f32.cpu().numpy(), f64.cpu().numpy()
    assert rel_rms(f32, f64) <= 1e-4 and max_rel(f32, f64) <= TOL["fmax"]


@pytest.mark.parametrize("kw", [dict(precision="fp64"), dict(precision="fp32", method="wolf", wolf_alpha=2.0),
                                dict(precision="fp32", scalar_pairs=True)])
def test_cluster_flag_is_ignored_where_documented(api, torch, kw):
    """FP64, Wolf summation and the scalar pair loop keep the default pass: the flag
    changes no bit there."""
    s = inputs.water_box(1500, 2.5, margin=0.5, with_velocities=False)
    out = []
    for cp in (False, True):
        m = api.MSM(a=A, h=H, levels=3, cluster_pairs=cp, **kw)
        out.append(m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box))
    assert float(out[0][0]) == float(out[1][0])
    assert torch.equal(out[0][1], out[1][1]) and torch.equal(out[0][2], out[1][2])
