"""GPU velocity Verlet (+ SHAKE/RATTLE water completion) and parareal against the
FP64 oracle and against their own invariants (Secs. 2 and 4), through the C ABI.

Bars: the FP64 path follows the oracle's trajectory to 1e-9 nm over 10 steps
(both solve the same constraint equations to 1e-12 relative, so they differ
only by rounding amplified over a few steps); the FP32 path to 1e-5 nm (FP32
forces carry ~1e-6 relative error; 10 steps of 2 fs move an atom ~1e-2 nm).
Parareal invariants are bitwise: the library's F and G are deterministic.
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


@pytest.mark.parametrize("prec,tol_x,tol_e", [("fp64", 1e-9, 1e-9), ("fp32", 1e-5, 1e-5)])
def test_md_matches_oracle(api, torch, small_water, prec, tol_x, tol_e):
    s = small_water
    ox, ov, ouk = oracle.md_run(s, a=A, h=H, levels=3, dt=0.002, n_steps=10)
    m = api.MSM(a=A, h=H, levels=3, precision=prec, model="water")
    d = _dev_sys(torch, s)
    uk = m.md_run(d, dt=0.002, n_steps=10).cpu().numpy()
    assert np.abs(d.pos.cpu().numpy() - ox).max() <= tol_x
    assert np.abs(d.vel.cpu().numpy() - ov).max() <= 1e3 * tol_x
    scale = np.abs(ouk).max()
    assert np.abs(uk - ouk).max() <= tol_e * scale


def test_md_keeps_rigid_geometry(api, torch, small_water):
    s = small_water
    for prec, tol in (("fp64", 1e-11), ("fp32", 2e-6)):
        m = api.MSM(a=A, h=H, levels=3, precision=prec, model="water")
        d = _dev_sys(torch, s)
        m.md_run(d, dt=0.002, n_steps=20, record=False)
        x = d.pos.cpu().numpy()[: 3 * s.n_mol].reshape(-1, 3, 3)
        oh = np.linalg.norm(x[:, 0] - x[:, 1], axis=1)
        hh = np.linalg.norm(x[:, 1] - x[:, 2], axis=1)
        assert np.abs(oh / inputs.D_OH - 1).max() <= tol
        assert np.abs(hh / inputs.d_hh() - 1).max() <= tol


def test_md_is_time_reversible_on_gpu(api, torch, small_water):
    s = small_water
    m = api.MSM(a=A, h=H, levels=3, precision="fp64", model="water")
    d = _dev_sys(torch, s)
    m.md_run(d, dt=0.002, n_steps=15, record=False)
    d.vel.neg_()
    m.md_run(d, dt=0.002, n_steps=15, record=False)
    assert np.abs(d.pos.cpu().numpy() - s.pos).max() < 1e-9


def test_md_split_runs_with_carried_forces_equal_one_run(api, torch, small_water):
    s = small_water
    m = api.MSM(a=A, h=H, levels=3, precision="fp32", model="water")
    d1 = _dev_sys(torch, s)
    m.md_run(d1, dt=0.002, n_steps=6, record=False)
    d2 = _dev_sys(torch, s)
    d2.force = torch.zeros_like(d2.pos)
    for _ in range(6):
        m.md_run(d2, dt=0.002, n_steps=1, record=False)
    assert torch.equal(d1.pos, d2.pos) and torch.equal(d1.vel, d2.vel)


def test_md_host_buffers_equal_device_buffers(api, torch, small_water):
    s = small_water
    m = api.MSM(a=A, h=H, levels=3, precision="fp32", model="water")
    d = _dev_sys(torch, s)
    m.md_run(d, dt=0.002, n_steps=5, record=False)
    hs = inputs.System(pos=s.pos.copy(), q=s.q, mass=s.mass, box=s.box, vel=s.vel.copy(), n_mol=s.n_mol, lj=s.lj)
    m.md_run(hs, dt=0.002, n_steps=5, record=False)
    assert np.array_equal(hs.pos, d.pos.cpu().numpy()) and np.array_equal(hs.vel, d.vel.cpu().numpy())


def test_nve_energy_error_is_second_order(api, torch):
    """Velocity Verlet's energy error is second order in dt (Sec. 2's integrator):
    over the same 50 fs from the same state, halving dt cuts the largest total-energy
    deviation about four-fold, in FP64 and in FP32; and the FP32 path's deviation at
    the smaller step stays that of the FP64 path (its arithmetic adds no visible
    error of its own)."""
    s = inputs.water_box(3000, 3.1, margin=1.0)
    out = {}
    for prec in ("fp64", "fp32"):
        fl = []
        for dt, n in ((0.002, 25), (0.001, 50)):
            m = api.MSM(a=A, h=H, levels=3, precision=prec, model="water", wall_k=1e4, wall_width=0.8)
            d = _dev_sys(torch, s)
            uk = m.md_run(d, dt=dt, n_steps=n).cpu().numpy()
            assert np.all(np.isfinite(uk))
            e = uk.sum(1)
            fl.append(np.abs(e - e[0]).max())
        out[prec] = fl
        assert fl[1] < fl[0] / 2.5, (prec, fl)
    assert abs(out["fp32"][1] - out["fp64"][1]) < 0.1 * out["fp64"][1], out


# ------------------------------------------------------------------ parareal

FINE = dict(a=1.2, h=0.25, levels=2, dt=0.002, steps=4)
COARSE = dict(a=0.8, h=0.5, levels=2, dt=0.004, steps=2)


@pytest.fixture(scope="module")
def pr_sys():
    return inputs.water_box(45, 0.8, margin=0.5, seed=5, vel_seed=6)


def _serial(api, torch, s, p, prec, n_slices):
    m = api.MSM(a=p["a"], h=p["h"], levels=p["levels"], precision=prec, model="water")
    d = _dev_sys(torch, s)
    xs = [d.pos.cpu().numpy().copy()]; vs = [d.vel.cpu().numpy().copy()]
    for _ in range(n_slices):
        m.md_run(d, dt=p["dt"], n_steps=p["steps"], record=False)
        xs.append(d.pos.cpu().numpy().copy()); vs.append(d.vel.cpu().numpy().copy())
    return np.array(xs), np.array(vs)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_parareal_invariants_are_bitwise(api, torch, pr_sys, prec):
    s = pr_sys
    n_slices = 4
    gx, gv = _serial(api, torch, s, COARSE, prec, n_slices)
    fx, fv = _serial(api, torch, s, FINE, prec, n_slices)
    xs, vs, it, dx, conv = api.parareal_run(COARSE, FINE, s, n_slices, 0, 0.0, precision=prec)
    assert it == 0 and np.array_equal(xs, gx) and np.array_equal(vs, gv)
    for k in (1, 2):
        xs, vs, it, dx, conv = api.parareal_run(COARSE, FINE, s, n_slices, k, 0.0, precision=prec)
        assert it == k
        assert np.array_equal(xs[: k + 1], fx[: k + 1]) and np.array_equal(vs[: k + 1], fv[: k + 1])
    xs, vs, it, dx, conv = api.parareal_run(COARSE, FINE, s, n_slices, n_slices, 0.0, precision=prec)
    assert np.array_equal(xs, fx) and np.array_equal(vs, fv)


def test_parareal_matches_oracle(api, torch, pr_sys):
    s = pr_sys
    oxs, ovs, oit, odx, orc = oracle.parareal(s, COARSE, FINE, n_slices=3, max_iter=2, tol=0.0)
    xs, vs, it, dx, conv = api.parareal_run(COARSE, FINE, s, 3, 2, 0.0, precision="fp64")
    assert it == oit == 2
    assert np.abs(xs - oxs).max() < 1e-9
    assert np.abs(vs - ovs).max() < 1e-6


def test_parareal_converges_to_tolerance(api, torch, pr_sys):
    s = pr_sys
    xs, vs, it, dx, conv = api.parareal_run(COARSE, FINE, s, 6, 6, 1e-6, precision="fp32")
    assert conv and dx <= 1e-6 and it <= 6
    fx, _ = _serial(api, torch, s, FINE, "fp32", 6)
    assert np.abs(xs - fx).max() <= 1e-5


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_verlet_lists_equal_cell_search(api, torch, prec, tol):
    """md_run with Verlet lists (skin 0.1 nm, rebuilt when an atom moved more than
    skin/2) follows the every-step cell search to rounding: both sum exactly the
    pairs within a."""
    s = inputs.water_box(3000, 3.1, margin=1.0, seed=7, vel_seed=8)
    out = {}
    for skin in (0.0, 0.1):
        m = api.MSM(a=A, h=H, levels=3, precision=prec, model="water", list_skin=skin, wall_k=1e4, wall_width=0.8)
        d = _dev_sys(torch, s)
        uk = m.md_run(d, dt=0.002, n_steps=30).cpu().numpy()
        out[skin] = (d.pos.cpu().numpy(), uk)
    assert np.abs(out[0.0][0] - out[0.1][0]).max() <= tol
    assert np.abs(out[0.0][1] - out[0.1][1]).max() <= 10 * tol * np.abs(out[0.0][1]).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_windowed_parareal_invariants(api, torch, pr_sys, prec):
    """The sliding window (Sec. 4's computational window): a full window with
    tol = 0 gives parareal_run's iterates bit for bit; a one-slice window is the
    serial fine run (one iteration per slice); a two-slice window iterated to the
    end gives every slice exactly."""
    s = pr_sys
    n_slices = 5
    fx, fv = _serial(api, torch, s, FINE, prec, n_slices)
    for k in (1, 2):
        a = api.parareal_run(COARSE, FINE, s, n_slices, k, 0.0, precision=prec)
        b = api.parareal_run(COARSE, FINE, s, n_slices, k, 0.0, precision=prec, window=n_slices)
        assert a[2] == b[2] == k
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    xs, vs, it, dx, conv = api.parareal_run(COARSE, FINE, s, n_slices, 50, 0.0, precision=prec, window=1)
    assert conv and it == n_slices
    assert np.array_equal(xs, fx) and np.array_equal(vs, fv)
    xs, vs, it, dx, conv = api.parareal_run(COARSE, FINE, s, n_slices, 50, 0.0, precision=prec, window=2)
    assert conv and np.array_equal(xs, fx) and np.array_equal(vs, fv)


def test_windowed_parareal_matches_oracle(api, torch, pr_sys):
    s = pr_sys
    for window, iters in ((2, 3), (3, 2)):
        oxs, ovs, oit, odx, orc = oracle.parareal_window(s, COARSE, FINE, n_slices=5, window=window,
                                                         max_iter=iters, tol=0.0)
        xs, vs, it, dx, conv = api.parareal_run(COARSE, FINE, s, 5, iters, 0.0, precision="fp64", window=window)
        assert it == oit == iters and not conv
        reached = np.any(oxs != 0, axis=(1, 2))
        assert np.array_equal(np.any(xs != 0, axis=(1, 2)), reached)
        assert np.abs(xs[reached] - oxs[reached]).max() < 1e-9
        assert np.abs(vs[reached] - ovs[reached]).max() < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_parareal_resumes_from_a_checkpoint_bit_for_bit(api, torch, pr_sys, prec):
    """Checkpoint and resume: the iterate after k iterations (what parareal_run
    returns when max_iter stops it), fed back with k, continues to exactly the
    iterates of one uninterrupted run; so does a second resume, and a resume of a
    finished run changes nothing."""
    s = pr_sys
    n_slices = 5
    whole = api.parareal_run(COARSE, FINE, s, n_slices, 4, 0.0, precision=prec)
    part = api.parareal_run(COARSE, FINE, s, n_slices, 2, 0.0, precision=prec)
    assert part[2] == 2
    xs, vs = part[0].copy(), part[1].copy()                   # the checkpoint, as a caller would keep it
    r1 = api.parareal_run(COARSE, FINE, s, n_slices, 1, 0.0, precision=prec, resume=(xs, vs, 2))
    assert r1[2] == 3
    r2 = api.parareal_run(COARSE, FINE, s, n_slices, 1, 0.0, precision=prec, resume=(r1[0], r1[1], 3))
    assert r2[2] == 4
    assert np.array_equal(r2[0], whole[0]) and np.array_equal(r2[1], whole[1])
    assert r2[3] == whole[3]
    done = api.parareal_run(COARSE, FINE, s, n_slices, n_slices, 0.0, precision=prec)
    again = api.parareal_run(COARSE, FINE, s, n_slices, 3, 0.0, precision=prec,
                             resume=(done[0], done[1], n_slices))
    assert again[2] == n_slices + 1 and again[4]
    assert np.array_equal(again[0], done[0]) and np.array_equal(again[1], done[1])
