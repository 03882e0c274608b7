"""GPU multiple time stepping (Sec. 3: the MSM suits a multiple-time-step
integrator; the impulse method with SHAKE/RATTLE, grid part as the slow force)
against the FP64 oracle and its own invariants, through the C ABI.

Bars as for plain velocity Verlet: the FP64 path follows the oracle's
trajectory to 1e-9 nm, the FP32 path to 1e-5 nm; graph replay, batching and a
factor of 1 are bitwise.
"""
import numpy as np
import pytest

import oracle
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


def _dev_sys(torch, s):
    t = lambda x: torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")
    return inputs.System(pos=t(s.pos), q=t(s.q), mass=t(s.mass), box=s.box, vel=t(s.vel), n_mol=s.n_mol,
                         lj=torch.tensor(s.lj, device="cuda"))


@pytest.fixture(scope="module")
def small_water():
    return inputs.water_box(90, 1.0, margin=0.5, seed=3, vel_seed=4)


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("prec,tol_x,tol_e", [("fp64", 1e-9, 1e-9), ("fp32", 1e-5, 1e-5)])
def test_mts_matches_oracle(api, torch, small_water, k, prec, tol_x, tol_e):
    s = small_water
    n = 4 * k
    ox, ov, ouk = oracle.md_run(s, a=A, h=H, levels=3, dt=0.002, n_steps=n, mts=k, wall_k=1e4, wall_width=0.4)
    m = api.MSM(a=A, h=H, levels=3, precision=prec, model="water", mts=k, wall_k=1e4, wall_width=0.4)
    d = _dev_sys(torch, s)
    uk = m.md_run(d, dt=0.002, n_steps=n).cpu().numpy()
    assert np.abs(d.pos.cpu().numpy() - ox).max() <= tol_x
    assert np.abs(d.vel.cpu().numpy() - ov).max() <= 1e3 * tol_x
    assert np.abs(uk - ouk).max() <= tol_e * np.abs(ouk).max()
    # the bar separates the two integrators: plain velocity Verlet ends farther away
    px, _, _ = oracle.md_run(s, a=A, h=H, levels=3, dt=0.002, n_steps=n, wall_k=1e4, wall_width=0.4)
    assert np.abs(ox - px).max() > 4 * tol_x


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_factor_one_is_plain_velocity_verlet(api, torch, small_water, prec):
    s = small_water
    out = []
    for kw in ({}, {"mts": 1}):
        m = api.MSM(a=A, h=H, levels=3, precision=prec, model="water", **kw)
        d = _dev_sys(torch, s)
        uk = m.md_run(d, dt=0.002, n_steps=6)
        out.append((d.pos, d.vel, uk))
    for u, w in zip(*out):
        assert torch.equal(u, w)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_replay_and_batching_are_bitwise(api, torch, small_water, prec):
    """Outer steps replayed from one captured graph, run launch by launch, and
    stepped inside a batch of two systems all give the same bits."""
    s = small_water
    w = inputs.water_box(150, 1.2, margin=0.5, seed=7, vel_seed=8)
    res = {}
    for graphs in (True, False):
        m = api.MSM(a=A, h=H, levels=3, precision=prec, model="water", mts=2, graphs=graphs)
        d = _dev_sys(torch, s)
        uk = m.md_run(d, dt=0.002, n_steps=8)
        res[graphs] = (d.pos.clone(), d.vel.clone(), uk.clone())
    for u, v in zip(res[True], res[False]):
        assert torch.equal(u, v)
    m = api.MSM(a=A, h=H, levels=3, precision=prec, model="water", mts=2)
    d1, d2 = _dev_sys(torch, s), _dev_sys(torch, w)
    ukb = m.md_run_batched([d1, d2], dt=0.002, n_steps=8)
    assert torch.equal(d1.pos, res[True][0]) and torch.equal(d1.vel, res[True][1])
    assert torch.equal(ukb[0], res[True][2])
    m2 = api.MSM(a=A, h=H, levels=3, precision=prec, model="water", mts=2)
    d3 = _dev_sys(torch, w)
    m2.md_run(d3, dt=0.002, n_steps=8, record=False)
    assert torch.equal(d2.pos, d3.pos) and torch.equal(d2.vel, d3.vel)


def test_end_forces_are_the_whole_forces(api, torch, small_water):
    """With forces carried in the system, md_run returns the whole force at the
    end positions (fast + slow parts of the final split evaluation)."""
    s = small_water
    m = api.MSM(a=A, h=H, levels=3, precision="fp64", model="water", mts=3)
    d = _dev_sys(torch, s)
    d.force = torch.zeros_like(d.pos)
    m.md_run(d, dt=0.002, n_steps=6, record=False)
    ref = oracle.model_forces(s, a=A, h=H, levels=3, pos=d.pos.cpu().numpy())
    f = d.force.cpu().numpy()
    assert np.sqrt(((f - ref["forces"]) ** 2).sum() / (ref["forces"] ** 2).sum()) <= 1e-12
    assert abs(d.energy - ref["energy"]) <= 1e-12 * 0.5 * np.abs(s.q * ref["pot"]).sum()


def test_mts_needs_whole_outer_steps_and_the_msm(api, torch, small_water):
    s = small_water
    m = api.MSM(a=A, h=H, levels=3, precision="fp32", model="water", mts=2)
    d = _dev_sys(torch, s)
    with pytest.raises(api.MSMError):
        m.md_run(d, dt=0.002, n_steps=5)
    with pytest.raises(api.MSMError):
        api.MSM(a=A, h=H, levels=1, precision="fp32", model="water", mts=2, method="cutoff")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_mts_with_verlet_lists_equals_cell_search(api, torch, prec, tol):
    """The fast steps' short-range sum from Verlet lists (skin 0.1 nm) follows the
    every-step cell search to rounding under multiple time stepping too."""
    s = inputs.water_box(3000, 3.1, margin=1.0, seed=7, vel_seed=8)
    out = {}
    for skin in (0.0, 0.1):
        m = api.MSM(a=A, h=H, levels=3, precision=prec, model="water", mts=3, list_skin=skin,
                    wall_k=1e4, wall_width=0.8)
        d = _dev_sys(torch, s)
        uk = m.md_run(d, dt=0.002, n_steps=30).cpu().numpy()
        out[skin] = (d.pos.cpu().numpy(), uk)
    assert np.abs(out[0.0][0] - out[0.1][0]).max() <= tol
    assert np.abs(out[0.0][1] - out[0.1][1]).max() <= 10 * tol * np.abs(out[0.0][1]).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_parareal_with_a_multiple_time_step_fine_propagator(api, torch, prec):
    """Parareal (Sec. 4) around a fine propagator that itself steps the grid part every
    second step: after as many iterations as slices the result is the serial
    multiple-time-step run, bit for bit."""
    s = inputs.water_box(45, 0.8, margin=0.5, seed=5, vel_seed=6)
    fine = dict(a=1.2, h=0.25, levels=2, dt=0.002, steps=4, mts=2)
    coarse = dict(a=0.8, h=0.5, levels=2, dt=0.004, steps=2)
    n_slices = 3
    m = api.MSM(a=1.2, h=0.25, levels=2, precision=prec, model="water", mts=2)
    d = _dev_sys(torch, s)
    xs_ref = [d.pos.cpu().numpy().copy()]
    for _ in range(n_slices):
        m.md_run(d, dt=0.002, n_steps=4, record=False)
        xs_ref.append(d.pos.cpu().numpy().copy())
    xs, vs, it, dx, conv = api.parareal_run(coarse, fine, s, n_slices, n_slices, 0.0, precision=prec)
    assert np.array_equal(xs, np.array(xs_ref))
