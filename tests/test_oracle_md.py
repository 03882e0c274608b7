"""Pins for the oracle's velocity Verlet + SHAKE/RATTLE dynamics and parareal (Secs. 2 and 4).

  * velocity Verlet is time reversible: N steps forward, velocities negated,
    N steps back returns to the start;
  * its energy error is second order: halving dt cuts the total-energy
    fluctuation about four-fold;
  * rigid bonds stay at their lengths and bond-relative velocities vanish;
  * parareal: zero iterations is the sequential G sweep; after k iterations the
    first k+1 slice ends equal the serial fine trajectory bitwise; with G = F
    one iteration reproduces the serial trajectory to rounding.
"""
import numpy as np
import pytest

import oracle
from paper_1309_1889_gb300 import inputs

FINE = dict(a=1.2, h=0.25, levels=2)


@pytest.fixture(scope="module")
def small_water():
    return inputs.water_box(24, 0.9, margin=0.5, seed=3, vel_seed=4)


def _bonds(x, n_mol):
    m = x[: 3 * n_mol].reshape(n_mol, 3, 3)
    return (np.linalg.norm(m[:, 0] - m[:, 1], axis=1), np.linalg.norm(m[:, 0] - m[:, 2], axis=1),
            np.linalg.norm(m[:, 1] - m[:, 2], axis=1))


def test_rigid_geometry_is_kept(small_water):
    s = small_water
    x, v, uk = oracle.md_run(s, dt=0.002, n_steps=10, **FINE)
    oh1, oh2, hh = _bonds(x, s.n_mol)
    assert np.allclose(oh1, inputs.D_OH, rtol=1e-11) and np.allclose(oh2, inputs.D_OH, rtol=1e-11)
    assert np.allclose(hh, inputs.d_hh(), rtol=1e-11)
    m = x[: 3 * s.n_mol].reshape(s.n_mol, 3, 3); w = v[: 3 * s.n_mol].reshape(s.n_mol, 3, 3)
    for i, j in ((0, 1), (0, 2), (1, 2)):
        assert np.abs(((m[:, i] - m[:, j]) * (w[:, i] - w[:, j])).sum(-1)).max() < 1e-12
    assert np.all(np.isfinite(uk))


def test_velocity_verlet_is_time_reversible(small_water):
    s = small_water
    x1, v1, _ = oracle.md_run(s, dt=0.002, n_steps=15, **FINE)
    x2, v2, _ = oracle.md_run(s, dt=0.002, n_steps=15, x=x1, v=-v1, **FINE)
    assert np.abs(x2 - s.pos).max() < 1e-9
    assert np.abs(-v2 - s.vel).max() < 1e-6


def test_energy_error_is_second_order(small_water):
    s = small_water
    flucts = []
    for dt, n in ((0.002, 10), (0.001, 20)):
        _, _, uk = oracle.md_run(s, dt=dt, n_steps=n, **FINE)
        e = uk.sum(1)
        flucts.append(np.abs(e - e[0]).max())
    assert flucts[1] < flucts[0] / 2.5


def _run_serial(s, p, n_slices):
    xs = [s.pos.copy()]; vs = [s.vel.copy()]
    for _ in range(n_slices):
        x, v, _ = oracle.md_run(s, a=p["a"], h=p["h"], levels=p["levels"], dt=p["dt"], n_steps=p["steps"],
                                x=xs[-1], v=vs[-1], method=p.get("method", "msm"),
                                wolf_alpha=p.get("wolf_alpha", 0.0))
        xs.append(x); vs.append(v)
    return np.array(xs), np.array(vs)


# coarse propagators: MSM with a shorter cutoff and coarser grid, the simple cutoff
# (Sec. 5, the paper's choice) and Wolf summation (Sec. 5, its proposed later G)
COARSE = {"msm": dict(a=0.8, h=0.5, levels=2, dt=0.004, steps=2),
          "cutoff": dict(a=0.8, h=0.5, levels=1, dt=0.004, steps=2, method="cutoff"),
          "wolf": dict(a=0.8, h=0.5, levels=1, dt=0.004, steps=2, method="wolf", wolf_alpha=2.5)}


@pytest.fixture(scope="module", params=sorted(COARSE))
def pr_setup(request):
    s = inputs.water_box(15, 0.8, margin=0.5, seed=5, vel_seed=6)
    F = dict(a=1.2, h=0.25, levels=2, dt=0.002, steps=4)
    return s, F, COARSE[request.param]


def test_parareal_zero_iterations_is_the_coarse_sweep(pr_setup):
    s, F, G = pr_setup
    xs, vs, it, dx, rc = oracle.parareal(s, G, F, n_slices=3, max_iter=0, tol=0.0)
    gx, gv = _run_serial(s, G, 3)
    assert it == 0
    assert np.array_equal(xs, gx) and np.array_equal(vs, gv)


def test_parareal_exact_slices_after_k_iterations(pr_setup):
    s, F, G = pr_setup
    n_slices = 4
    fx, fv = _run_serial(s, F, n_slices)
    for k in (1, 2):
        xs, vs, it, dx, rc = oracle.parareal(s, G, F, n_slices=n_slices, max_iter=k, tol=0.0)
        assert it == k
        assert np.array_equal(xs[: k + 1], fx[: k + 1]) and np.array_equal(vs[: k + 1], fv[: k + 1])
        if k < n_slices:
            assert not np.array_equal(xs[-1], fx[-1])
    xs, vs, it, dx, rc = oracle.parareal(s, G, F, n_slices=n_slices, max_iter=n_slices, tol=0.0)
    assert np.array_equal(xs, fx) and np.array_equal(vs, fv)


def test_parareal_with_fine_as_coarse_converges_in_one_iteration(pr_setup):
    s, F, _ = pr_setup
    fx, fv = _run_serial(s, F, 3)
    xs, vs, it, dx, rc = oracle.parareal(s, F, F, n_slices=3, max_iter=2, tol=1e-12)
    assert np.abs(xs - fx).max() < 1e-12
    assert it <= 2 and rc == 0


def test_wall_bounce_is_elastic():
    """A lone rigid molecule thrown at a face of the flat-bottom wall comes back
    (part of its translation turns into rotation: the wall pushes atoms, not the
    centre of mass) with its kinetic energy kept -- the wall is conservative --
    and the wall force is minus the gradient of its energy."""
    s = inputs.water_box(3, 0.6, margin=0.6, seed=1, vel_seed=2)
    s.vel[:] = 0.0
    s.vel[:, 0] = -1.5                                      # nm/ps towards the x0 face
    kw = dict(a=1.2, h=0.25, levels=2, wall_k=5000.0, wall_width=0.5)
    m = s.mass[:3]
    v0 = (m[:, None] * s.vel[:3]).sum(0) / m.sum()
    x, v, uk = oracle.md_run(s, dt=0.001, n_steps=800, **kw)
    v1 = (m[:, None] * v[:3]).sum(0) / m.sum()
    assert x[:3, 0].min() > s.box[0]                        # never reached the face
    assert v1[0] > 0.9 * abs(v0[0])                           # reflected
    assert uk[-1, 1] == pytest.approx(uk[0, 1], rel=2e-3)      # no energy left in the wall
    e = uk.sum(1)
    assert np.abs(e - e[0]).max() < 1e-3 * uk[:, 1].max()
    # F = -dU/dx inside the wall zone
    pos = s.pos.copy(); pos[:, 0] -= pos[:, 0].min() - (s.box[0] + 0.2)
    sw = inputs.System(pos=pos, q=s.q, mass=s.mass, box=s.box, n_mol=1, lj=s.lj)
    f = oracle.model_forces(sw, 1.2, 0.25, 2, wall_k=5000.0, wall_width=0.5)["forces"]
    d = 1e-6
    pp = pos.copy(); pp[0, 0] += d
    pm = pos.copy(); pm[0, 0] -= d
    ep = oracle.model_forces(sw, 1.2, 0.25, 2, pos=pp, wall_k=5000.0, wall_width=0.5)["energy"]
    em = oracle.model_forces(sw, 1.2, 0.25, 2, pos=pm, wall_k=5000.0, wall_width=0.5)["energy"]
    assert f[0, 0] == pytest.approx(-(ep - em) / (2 * d), rel=1e-6)


def test_projection_restores_rigid_geometry_and_conserves_momenta():
    """The projection of a corrected parareal state (water completion): every
    distorted molecule gets its rigid bond lengths and zero bond-parallel relative
    velocities back; each correction moves two atoms by opposite mass-weighted
    amounts along their bond, so the centre of mass and the linear momentum are
    conserved exactly, and the velocity stage conserves the angular momentum
    taken at the projected positions."""
    s = inputs.water_box(60, 1.0, margin=0.5, seed=11, vel_seed=12)
    rng = np.random.default_rng(3)
    x = s.pos.copy(); v = s.vel.copy()
    k = 3 * s.n_mol
    x[:k] += rng.normal(0.0, 0.004, (k, 3))           # distort every molecule
    v[:k] += rng.normal(0.0, 0.5, (k, 3))
    xp, vp = oracle.project_rigid(x, v, s.mass, s.n_mol)
    oh1, oh2, hh = _bonds(xp, s.n_mol)
    assert np.allclose(oh1, inputs.D_OH, rtol=1e-12, atol=0) and np.allclose(oh2, inputs.D_OH, rtol=1e-12, atol=0)
    assert np.allclose(hh, inputs.d_hh(), rtol=1e-12, atol=0)
    m3 = xp[:k].reshape(-1, 3, 3); w3 = vp[:k].reshape(-1, 3, 3)
    for i, j in ((0, 1), (0, 2), (1, 2)):
        assert np.abs(((m3[:, i] - m3[:, j]) * (w3[:, i] - w3[:, j])).sum(-1)).max() <= 1e-14
    mm = s.mass[:k].reshape(-1, 3, 1)
    com0 = (mm * x[:k].reshape(-1, 3, 3)).sum(1); com1 = (mm * m3).sum(1)
    p0 = (mm * v[:k].reshape(-1, 3, 3)).sum(1); p1 = (mm * w3).sum(1)
    assert np.abs(com1 - com0).max() < 1e-13 and np.abs(p1 - p0).max() < 1e-12
    L_mid = np.cross(m3, mm * v[:k].reshape(-1, 3, 3)).sum(1)     # new positions, old velocities
    L1 = np.cross(m3, mm * w3).sum(1)
    assert np.abs(L1 - L_mid).max() < 1e-12
    assert np.array_equal(xp[k:], x[k:]) and np.array_equal(vp[k:], v[k:])   # single sites untouched


def test_projection_leaves_rigid_molecules_bitwise_unchanged():
    s = inputs.water_box(60, 1.0, margin=0.5, seed=11, vel_seed=12)
    x, v, _ = oracle.md_run(s, dt=0.002, n_steps=3, **FINE)       # SHAKE/RATTLE output
    xp, vp = oracle.project_rigid(x, v, s.mass, s.n_mol)
    assert np.array_equal(xp, x) and np.array_equal(vp, v)


def test_windowed_parareal_with_full_window_is_plain_parareal(pr_setup):
    """A window as long as the run, tol = 0: the same iterates bit for bit."""
    s, F, G = pr_setup
    for k in (1, 2, 6):
        a = oracle.parareal(s, G, F, n_slices=4, max_iter=k, tol=0.0)
        b = oracle.parareal_window(s, G, F, n_slices=4, window=4, max_iter=k, tol=0.0)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        if k < 4:
            assert a[2] == b[2] == k and a[3] == b[3]
        else:
            # the window knows slice 3 is exact after iteration 4; plain parareal needs a
            # fifth iteration to see no change
            assert b[2] == 4 and b[4] == 0 and a[2] == 5 and a[3] == 0.0


def test_windowed_parareal_small_windows_reach_serial_fine(pr_setup):
    """W = 1 is the serial fine run (one iteration per slice); W = 2 with tol = 0
    iterated to the end also gives every slice exactly."""
    s, F, G = pr_setup
    fx, fv = _run_serial(s, F, 5)
    xs, vs, it, dx, rc = oracle.parareal_window(s, G, F, n_slices=5, window=1, max_iter=50, tol=0.0)
    assert rc == 0 and it == 5
    assert np.array_equal(xs, fx) and np.array_equal(vs, fv)
    xs, vs, it, dx, rc = oracle.parareal_window(s, G, F, n_slices=5, window=2, max_iter=50, tol=0.0)
    assert rc == 0 and np.array_equal(xs, fx) and np.array_equal(vs, fv)
    # one iteration of a 2-slice window: slice 0's end is exact, slice 1's is G-corrected,
    # the slices beyond the window are not reached
    xs, vs, it, dx, rc = oracle.parareal_window(s, G, F, n_slices=5, window=2, max_iter=1, tol=0.0)
    assert rc == -6 and it == 1
    assert np.array_equal(xs[1], fx[1]) and not np.array_equal(xs[2], fx[2])
    assert not np.any(xs[3:])
