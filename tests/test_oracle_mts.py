"""Pins for the oracle's multiple time stepping (Sec. 3: the MSM suits a
multiple-time-step integrator; the impulse method with SHAKE/RATTLE).

  * the split adds up: fast + slow forces are the model's forces, bit-close;
  * each part is a gradient: F_slow = -dU_slow/dr and F_fast = -d(U - U_slow)/dr
    by central differences (a dropped term, a wrong sign or a part filed under
    the wrong clock fails one of them);
  * for bare charges the fast part is k_e times the short-range sum, checked
    against the O(N^2) brute-force short-range routine;
  * one fast step per slow step is plain velocity Verlet, bit for bit;
  * the impulse integrator is time reversible and its energy error at the ends
    of outer steps is second order in dt;
  * n_steps that is not a multiple of the factor is rejected.
"""
import numpy as np
import pytest

import oracle
from paper_1309_1889_gb300 import inputs

FINE = dict(a=1.2, h=0.25, levels=2)
KE = oracle.KE


@pytest.fixture(scope="module")
def small_water():
    return inputs.water_box(24, 0.9, margin=0.5, seed=3, vel_seed=4)


def test_split_adds_up_to_the_model_forces(small_water):
    s = small_water
    tot = oracle.model_forces(s, **FINE)
    sp = oracle.model_forces_split(s, **FINE)
    f = sp["f_fast"] + sp["f_slow"]
    assert np.abs(f - tot["forces"]).max() <= 1e-11 * np.abs(tot["forces"]).max()
    # U is a small difference of large terms here: held to the scale of its terms
    scale = 0.5 * np.abs(s.q * tot["pot"]).sum()
    assert abs(sp["energy"] - tot["energy"]) <= 1e-13 * scale
    # both parts are of the size of the forces (neither is empty)
    assert np.abs(sp["f_slow"]).max() > 1e-3 * np.abs(tot["forces"]).max()
    assert np.abs(sp["f_fast"]).max() > 1e-3 * np.abs(tot["forces"]).max()


def _num_grad(energy_of, x, idx, h=1e-6):
    g = np.zeros((len(idx), 3))
    for r, i in enumerate(idx):
        for d in range(3):
            xp = x.copy(); xm = x.copy()
            xp[i, d] += h; xm[i, d] -= h
            g[r, d] = (energy_of(xp) - energy_of(xm)) / (2 * h)
    return g


def test_each_part_is_a_gradient(small_water):
    s = small_water
    sp = oracle.model_forces_split(s, **FINE)
    idx = [0, 1, 5, 13, 22]

    def slow(x):
        return oracle.model_forces_split(s, pos=x, **FINE)["energy_slow"]

    def fast(x):
        r = oracle.model_forces_split(s, pos=x, **FINE)
        return r["energy"] - r["energy_slow"]

    gs = _num_grad(slow, s.pos, idx)
    gf = _num_grad(fast, s.pos, idx)
    scale = np.abs(sp["f_slow"][idx]).max()
    assert np.abs(-gs - sp["f_slow"][idx]).max() <= 1e-5 * max(scale, 1.0)
    scale = np.abs(sp["f_fast"][idx]).max()
    assert np.abs(-gf - sp["f_fast"][idx]).max() <= 1e-5 * max(scale, 1.0)


def test_fast_part_of_bare_charges_is_the_short_range_sum():
    s = inputs.random_cloud(60, (1.6, 1.6, 1.6), seed=5, neutral=True, margin=0.3)
    sys = inputs.System(pos=s.pos, q=s.q, mass=np.ones(s.n), box=s.box, n_mol=0, lj=np.zeros(s.n, np.uint8))
    sp = oracle.model_forces_split(sys, eps=0.0, **FINE)
    phi, fsr = oracle.short_range(s.pos, s.q, FINE["a"], s.box, brute=True)
    assert np.abs(sp["f_fast"] - KE * fsr).max() <= 1e-12 * np.abs(KE * fsr).max()


def test_one_fast_step_per_slow_step_is_plain_velocity_verlet(small_water):
    s = small_water
    a = oracle.md_run(s, dt=0.002, n_steps=6, **FINE)
    for k in (0, 1):
        b = oracle.md_run(s, dt=0.002, n_steps=6, mts=k, **FINE)
        for u, w in zip(a, b):
            assert np.array_equal(u, w)


@pytest.mark.parametrize("k", [2, 3])
def test_impulse_integrator_is_time_reversible(small_water, k):
    s = small_water
    x1, v1, _ = oracle.md_run(s, dt=0.002, n_steps=6 * k, mts=k, **FINE)
    x2, v2, _ = oracle.md_run(s, dt=0.002, n_steps=6 * k, x=x1, v=-v1, mts=k, **FINE)
    assert np.abs(x2 - s.pos).max() < 1e-9
    assert np.abs(-v2 - s.vel).max() < 1e-6
    # and it is not plain velocity Verlet
    x0, _, _ = oracle.md_run(s, dt=0.002, n_steps=6 * k, **FINE)
    assert np.abs(x0 - x1).max() > 1e-9


def test_impulse_energy_error_is_second_order(small_water):
    s = small_water
    k = 2
    flucts = []
    for dt, n in ((0.002, 12), (0.001, 24)):
        _, _, uk = oracle.md_run(s, dt=dt, n_steps=n, mts=k, **FINE)
        e = uk.sum(1)[::k]                       # ends of outer steps: the whole energy
        flucts.append(np.abs(e - e[0]).max())
    assert flucts[1] < flucts[0] / 2.5


def test_steps_must_fill_outer_steps(small_water):
    with pytest.raises(oracle.OracleError):
        oracle.md_run(small_water, dt=0.002, n_steps=5, mts=2, **FINE)


def test_lone_molecule_has_no_fast_electrostatics():
    """One rigid molecule: its three pairs are excluded, so with no Lennard-Jones
    partner and no wall the fast part vanishes (the short-range g* of the excluded
    pairs is removed with them) and the slow part is only the grid's error."""
    w = inputs.water_box(3, 0.3, margin=0.6, seed=1, vel_seed=2)
    sp = oracle.model_forces_split(w, **FINE)
    ex = KE * abs(w.q[0] * w.q[1]) / inputs.D_OH          # size of one excluded term
    assert np.abs(sp["f_fast"]).max() <= 1e-12 * ex / inputs.D_OH
    assert abs(sp["energy"] - sp["energy_slow"]) <= 1e-12 * ex
    assert abs(sp["energy_slow"]) < 1e-2 * ex


def test_uncharged_sites_have_no_slow_part(small_water):
    """With every charge zero only the Lennard-Jones term and the wall act: all of
    it is fast, the slow part is exactly zero."""
    s = small_water
    z = inputs.System(pos=s.pos, q=np.zeros(s.n), mass=s.mass, box=s.box, vel=s.vel, n_mol=s.n_mol, lj=s.lj)
    sp = oracle.model_forces_split(z, wall_k=1e4, wall_width=0.8, **FINE)
    assert np.all(sp["f_slow"] == 0.0) and sp["energy_slow"] == 0.0
    tot = oracle.model_forces(z, wall_k=1e4, wall_width=0.8, **FINE)
    assert np.abs(sp["f_fast"] - tot["forces"]).max() <= 1e-12 * np.abs(tot["forces"]).max()
    assert np.abs(tot["forces"]).max() > 0
