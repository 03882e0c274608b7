"""GPU parity of the coarse propagators' electrostatics (Sec. 5): the simple cutoff
and Wolf summation, against the FP64 oracle, through the C ABI.

Bars as for the MSM: FP64 relative RMS <= 1e-12, FP32 relative RMS <= 1e-4 (per
atom <= 2e-3 of the RMS magnitude), energy <= 1e-12 (FP64) and 1e-6 (FP32) of
|U|; trajectories of the FP64 path within 1e-9 nm of the oracle's after 10 steps;
parareal with a cutoff coarse propagator keeps its invariants bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1309_1889_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(f=1e-12, e=1e-12, fmax=1e-10), "fp32": dict(f=1e-4, e=1e-6, fmax=2e-3)}
METHODS = [("cutoff", 0.0), ("wolf", 2.5)]


def rel_rms(x, ref):
    return float(np.sqrt(((x - ref) ** 2).sum() / (ref ** 2).sum()))


def max_rel(x, ref):
    if ref.ndim == 1:
        x, ref = x[:, None], ref[:, None]
    return float(np.linalg.norm(x - ref, axis=1).max() / np.sqrt((ref ** 2).sum(1).mean()))


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


def _check(e, f, p, ref, t):
    assert abs(float(e) - ref["energy"]) <= t["e"] * abs(ref["energy"])
    for got, want in ((f, ref["forces"]), (p, ref["pot"])):
        got = got.cpu().numpy() if hasattr(got, "cpu") else got
        assert rel_rms(got, want) <= t["f"] and max_rel(got, want) <= t["fmax"]


@pytest.mark.parametrize("method,alpha", METHODS)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["water3k", "ragged"])
def test_cutoff_charges_match_oracle(api, torch, method, alpha, prec, case):
    # point charges of water-like boxes (no near-coincident charges, as in the workloads);
    # "ragged": 684 molecules + 1 filler in a non-cubic box, shorter cutoff
    if case == "water3k":
        s, a = inputs.water_box(3000, 3.1, margin=0.5, with_velocities=False), 1.2
    else:
        s, a = inputs.water_box(2053, (2.9, 2.1, 3.3), margin=0.2, seed=21, with_velocities=False), 0.8
    ref = oracle.cutoff(s.pos, s.q, a, method, alpha)
    m = api.MSM(a=a, h=0.25, precision=prec, method=method, wolf_alpha=alpha)
    e, f, p = m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
    _check(e, f, p, ref, TOL[prec])
    # the pair set is the MSM's short-range one: the same count of ordered pairs within a
    mm = api.MSM(a=a, h=0.25, levels=2, precision=prec)
    mm.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
    assert m.count_pairs() == mm.count_pairs()


@pytest.mark.parametrize("method,alpha", METHODS)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cutoff_water_model_matches_oracle(api, torch, method, alpha, prec):
    s = inputs.water_box(900, 2.1, margin=0.5, with_velocities=False)
    kw = dict(wall_k=5000.0, wall_width=0.6)
    ref = oracle.model_forces(s, 0.8, 0.25, 1, method=method, wolf_alpha=alpha, **kw)
    m = api.MSM(a=0.8, h=0.25, precision=prec, model="water", method=method, wolf_alpha=alpha, **kw)
    sd = inputs.System(pos=_dev(torch, s.pos), q=_dev(torch, s.q), mass=_dev(torch, s.mass), box=s.box,
                       n_mol=s.n_mol, lj=torch.tensor(s.lj, device="cuda"))
    e, f, p = m.system_forces(sd)
    _check(e, f, p, ref, TOL[prec])
    with pytest.raises(api.MSMError):
        m.grid_shape(0)                        # no grids for the cutoff methods


@pytest.mark.parametrize("method,alpha", METHODS)
def test_cutoff_md_matches_oracle(api, torch, method, alpha):
    s = inputs.water_box(90, 1.0, margin=0.5, seed=3, vel_seed=4)
    ox, ov, ouk = oracle.md_run(s, a=0.8, h=0.25, levels=1, dt=0.002, n_steps=10, method=method, wolf_alpha=alpha)
    m = api.MSM(a=0.8, h=0.25, precision="fp64", model="water", method=method, wolf_alpha=alpha)
    t = lambda x: _dev(torch, x)
    d = inputs.System(pos=t(s.pos), q=t(s.q), mass=t(s.mass), box=s.box, vel=t(s.vel), n_mol=s.n_mol,
                      lj=torch.tensor(s.lj, device="cuda"))
    uk = m.md_run(d, dt=0.002, n_steps=10).cpu().numpy()
    assert np.abs(d.pos.cpu().numpy() - ox).max() <= 1e-9
    assert np.abs(uk - ouk).max() <= 1e-9 * np.abs(ouk).max()


FINE = dict(a=1.2, h=0.25, levels=2, dt=0.002, steps=4)


@pytest.mark.parametrize("method,alpha", METHODS)
def test_parareal_with_cutoff_coarse_propagator(api, torch, method, alpha):
    """Parareal whose G is a cutoff method: the invariants hold bit for bit (k = 0 is
    the G sweep; after k iterations the first k+1 slice ends are serial F; k =
    n_slices is serial F), and the FP64 run matches the oracle's."""
    s = inputs.water_box(45, 0.8, margin=0.5, seed=5, vel_seed=6)
    G = dict(a=0.8, h=0.5, levels=1, dt=0.004, steps=2, method=method, wolf_alpha=alpha)
    n_slices = 4

    def serial(p):
        m = api.MSM(a=p["a"], h=p["h"], levels=p["levels"], precision="fp64", model="water",
                    method=p.get("method", "msm"), wolf_alpha=p.get("wolf_alpha", 0.0))
        t = lambda x: _dev(torch, x)
        d = inputs.System(pos=t(s.pos), q=t(s.q), mass=t(s.mass), box=s.box, vel=t(s.vel), n_mol=s.n_mol,
                          lj=torch.tensor(s.lj, device="cuda"))
        xs = [s.pos.copy()]
        for _ in range(n_slices):
            m.md_run(d, dt=p["dt"], n_steps=p["steps"], record=False)
            xs.append(d.pos.cpu().numpy().copy())
        return np.array(xs)

    gx, fx = serial(G), serial(FINE)
    xs, vs, it, dx, conv = api.parareal_run(G, FINE, s, n_slices, 0, 0.0, precision="fp64")
    assert it == 0 and np.array_equal(xs, gx)
    xs, vs, it, dx, conv = api.parareal_run(G, FINE, s, n_slices, 2, 0.0, precision="fp64")
    assert np.array_equal(xs[:3], fx[:3])
    oxs, ovs, oit, odx, orc = oracle.parareal(s, G, FINE, n_slices=n_slices, max_iter=2, tol=0.0)
    assert oit == 2 and np.abs(xs - oxs).max() < 1e-9
    xs, vs, it, dx, conv = api.parareal_run(G, FINE, s, n_slices, n_slices, 0.0, precision="fp64")
    assert np.array_equal(xs, fx)
