"""Pins for the oracle's rigid-water completion (outside the paper; Sec. 2 lists
U_all = bonded + van der Waals + Coulomb, of which the paper treats Coulomb).

The completion adds to the MSM Coulomb energy (i) the removal of the three
intramolecular pairs of every (O, H, H) triple and (ii) an O-O Lennard-Jones
12-6 term cut and shifted at a.  Nothing here retypes the oracle's formulas:

  * Lennard-Jones: properties that fix its two parameters and the shift --
    the energy crosses -U_shift at r = sigma, its minimum sits at
    r = 2^(1/6) sigma with depth -epsilon - U_shift, the tail at r >> sigma
    is the dispersion -C6/r^6 with C6 = 4 eps sigma^6, the energy vanishes at
    and beyond a, scales linearly in epsilon and is invariant under a joint
    scaling of (r, sigma, a); the force is -dU/dr (central differences).
  * Exclusions: an isolated molecule's model energy is only the grid's
    interpolation error of its smooth part (tiny against the excluded pairs'
    Coulomb energy, and falling as h falls); two molecules give the direct
    Coulomb sum between their charges within the paper's MSM error bound; the
    whole model force is -dU/dr by central differences, on atoms of the same
    and of different molecules.
  * The paper's printed gamma coefficients and MSM error bound
    (tests/golden/paper_constants.json) pin gamma and the whole evaluation.
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_1309_1889_gb300 import inputs

A, H = 1.2, 0.25
SIGMA, EPS = 0.315061, 0.6364          # nm, kJ/mol: the O-O parameters of the completion
CONST = json.loads((Path(__file__).resolve().parent / "golden" / "paper_constants.json").read_text())


def _pair(r, sigma=SIGMA, eps=EPS, a=A, axis=0):
    """Two uncharged LJ sites r apart inside a 3.4 nm box; returns (U, F)."""
    pos = np.full((2, 3), 1.7)
    pos[0, axis] -= r / 2
    pos[1, axis] += r / 2
    s = inputs.System(pos=pos, q=np.zeros(2), mass=np.ones(2), box=np.array([0, 0, 0, 3.4, 3.4, 3.4]),
                      n_mol=0, lj=np.ones(2, dtype=np.uint8))
    out = oracle.model_forces(s, a, H, 3, sigma=sigma, eps=eps)
    return out["energy"], out["forces"]


def _shift(sigma=SIGMA, eps=EPS, a=A):
    """U_LJ(a) of the unshifted potential, obtained from the oracle itself as
    U(sigma) = 0 - U_shift (the zero crossing of 12-6 is at sigma)."""
    return -_pair(sigma, sigma, eps, a)[0]


def test_lj_zero_crossing_and_minimum():
    sh = _shift()
    # the shift is the unshifted potential at a: tiny and negative (attractive tail)
    assert -1e-2 < sh < 0
    rmin = 2.0 ** (1.0 / 6.0) * SIGMA
    u_min, f_min = _pair(rmin)
    assert u_min + sh == pytest.approx(-EPS, rel=1e-12)
    assert np.abs(f_min).max() < 1e-10
    # a minimum: higher on both sides
    assert _pair(0.98 * rmin)[0] > u_min and _pair(1.02 * rmin)[0] > u_min


def test_lj_dispersion_tail():
    sh = _shift()
    for r in (0.8, 0.95, 1.1):
        u = _pair(r)[0] + sh
        c6 = 4.0 * EPS * SIGMA ** 6
        # the repulsive r^-12 part is (sigma/r)^6 ~ 1e-3 of the tail here
        assert u == pytest.approx(-c6 / r ** 6, rel=5e-3)
        assert u > -c6 / r ** 6          # the r^-12 part is repulsive


def test_lj_vanishes_at_and_beyond_cutoff_and_is_continuous():
    for r in (A + 1e-9, 1.5):
        u, f = _pair(r)
        assert u == 0.0 and np.abs(f).max() == 0.0
    # the potential is shifted, not force-shifted: just inside a the energy is ~0 but
    # the force is the dispersion tail's 6 C6 / a^7 (the repulsion is ~1e-3 of it)
    u, f = _pair(A - 1e-12)
    assert abs(u) < 1e-13
    assert f[1, 0] == pytest.approx(-6.0 * 4.0 * EPS * SIGMA ** 6 / A ** 7, rel=2e-3)
    u, _ = _pair(A - 1e-7)
    assert abs(u) < 1e-8


def test_lj_scales_with_epsilon_and_jointly_with_length():
    r = 0.37
    u1, f1 = _pair(r)
    u2, f2 = _pair(r, eps=2.0 * EPS)
    assert u2 == pytest.approx(2.0 * u1, rel=1e-13)
    assert np.allclose(f2, 2.0 * f1, rtol=1e-13, atol=0)
    # U(lambda r; lambda sigma, lambda a) = U(r; sigma, a); F scales as 1/lambda
    lam = 0.8
    u3, f3 = _pair(lam * r, sigma=lam * SIGMA, a=lam * A)
    assert u3 == pytest.approx(u1, rel=1e-12)
    assert np.allclose(f3 * lam, f1, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("r", [0.28, 0.31, 0.36, 0.5, 0.9])
def test_lj_force_is_minus_energy_gradient(r):
    d = 1e-6
    up, _ = _pair(r + d)
    um, _ = _pair(r - d)
    _, f = _pair(r)
    dudr = (up - um) / (2 * d)
    # the second site moves +r/2 along x: F_1x = -dU/dr, F_0 = -F_1
    assert f[1, 0] == pytest.approx(-dudr, rel=1e-6, abs=1e-8)
    assert f[0, 0] == -f[1, 0]


def _molecules(centers, rots, sigma=SIGMA, eps=EPS):
    """Rigid TIP3P-geometry molecules at the given O positions and rotations."""
    half = math.radians(inputs.ANGLE_HOH_DEG) / 2.0
    body = np.array([[0.0, 0.0, 0.0],
                     [inputs.D_OH * math.sin(half), inputs.D_OH * math.cos(half), 0.0],
                     [-inputs.D_OH * math.sin(half), inputs.D_OH * math.cos(half), 0.0]])
    pos = np.concatenate([c + body @ R.T for c, R in zip(centers, rots)])
    k = len(centers)
    q = np.tile([inputs.Q_O, inputs.Q_H, inputs.Q_H], k)
    m = np.tile([inputs.M_O, inputs.M_H, inputs.M_H], k)
    lj = np.tile(np.array([1, 0, 0], dtype=np.uint8), k)
    box = np.array([0.0, 0.0, 0.0, 3.0, 3.0, 3.0])
    return inputs.System(pos=pos, q=q, mass=m, box=box, n_mol=k, lj=lj)


def _rot(ax, ang):
    c, s = math.cos(ang), math.sin(ang)
    R = np.eye(3)
    i, j = [(1, 2), (0, 2), (0, 1)][ax]
    R[i, i] = c; R[j, j] = c; R[i, j] = -s; R[j, i] = s
    return R


def _excluded_coulomb(s):
    tot = 0.0
    for mo in range(s.n_mol):
        for i, j in ((0, 1), (0, 2), (1, 2)):
            a, b = 3 * mo + i, 3 * mo + j
            tot += oracle.KE * s.q[a] * s.q[b] / np.linalg.norm(s.pos[a] - s.pos[b])
    return tot


def test_isolated_molecule_energy_is_only_grid_error():
    """One molecule: MSM minus the three excluded pairs' full Coulomb energy leaves
    only the grids' interpolation error of their smooth part and of the self term.
    Subtracting the wrong kernel (g* alone, the smooth part alone, no 1/2, a wrong
    sign) leaves a term of the size of the excluded energy (~850 kJ/mol)."""
    s = _molecules([np.array([1.43, 1.52, 1.61])], [_rot(0, 0.3) @ _rot(2, 1.1)])
    excl = abs(_excluded_coulomb(s))
    assert excl > 800.0
    errs = []
    for h in (0.25, 0.125):
        u = oracle.model_forces(s, A, h, 3, eps=0.0)["energy"]
        errs.append(abs(u))
    assert errs[0] < 1e-2 * excl
    assert errs[1] < errs[0]
    # the forces left on a lone molecule are grid errors only: far below the excluded
    # pairs' own Coulomb forces (k_e q_i q_j / r^2, ~5e3 kJ/mol/nm for O-H)
    f = oracle.model_forces(s, A, H, 3, eps=0.0)["forces"]
    f_excl = oracle.KE * abs(inputs.Q_O * inputs.Q_H) / inputs.D_OH ** 2
    assert np.abs(f).max() < 1e-3 * f_excl


@pytest.mark.parametrize("sep", [0.29, 0.6, 1.9])
def test_two_molecules_give_the_intermolecular_direct_sum(sep):
    """Two molecules (LJ off): the model energy approximates the direct Coulomb sum
    over the nine intermolecular pairs only, within the paper's MSM error bound
    (Sec. 3: < 1 % for a > 0.8 nm, C^2 gamma, cubic Phi), at a separation inside
    the cutoff, near it and beyond it."""
    bound = CONST["msm_potential_relative_error_bound"]["value"]
    c0 = np.array([0.9, 1.4, 1.3])
    s = _molecules([c0, c0 + np.array([sep, 0.05, -0.03])], [_rot(1, 0.4), _rot(0, 2.2) @ _rot(1, -0.7)])
    u_direct = 0.0
    for i in range(3):
        for j in range(3, 6):
            u_direct += oracle.KE * s.q[i] * s.q[j] / np.linalg.norm(s.pos[i] - s.pos[j])
    u = oracle.model_forces(s, A, H, 3, eps=0.0)["energy"]
    # the error is relative to the interaction's own scale: the largest intermolecular term
    scale = max(abs(u_direct), max(abs(oracle.KE * s.q[i] * s.q[j] / np.linalg.norm(s.pos[i] - s.pos[j]))
                                   for i in range(3) for j in range(3, 6)) * 1e-2)
    assert abs(u - u_direct) < bound * scale


def test_model_force_is_minus_energy_gradient():
    """Central differences of the full model energy (MSM + exclusions + LJ + wall)
    against the model forces, on an O and an H of one molecule and an O of another
    that is within the LJ cutoff."""
    s = inputs.water_box(60, 0.85, margin=0.5, seed=5, with_velocities=False)
    kw = dict(wall_k=5000.0, wall_width=0.6)
    ref = oracle.model_forces(s, A, H, 3, **kw)
    d = 1e-6
    checked = 0
    for atom in (0, 1, 3 * 7, 3 * 11 + 2):
        for ax in range(3):
            xp = s.pos.copy(); xp[atom, ax] += d
            xm = s.pos.copy(); xm[atom, ax] -= d
            up = oracle.model_forces(s, A, H, 3, pos=xp, **kw)["energy"]
            um = oracle.model_forces(s, A, H, 3, pos=xm, **kw)["energy"]
            g = -(up - um) / (2 * d)
            assert ref["forces"][atom, ax] == pytest.approx(g, rel=2e-5, abs=2e-3)
            checked += 1
    assert checked == 12


def test_gamma_equals_the_printed_taylor_polynomial():
    c0, c1, c2 = CONST["gamma_taylor_c2"]["coefficients_rho0_rho2_rho4"]
    for rho in np.linspace(0.0, 0.999, 37):
        assert oracle.gamma(rho) == pytest.approx(c0 + c1 * rho ** 2 + c2 * rho ** 4, rel=1e-15, abs=1e-15)
    # the self term gamma(0)/a of the potential
    assert oracle.gamma(0.0) == c0


def test_msm_within_printed_bound_on_a_water_box():
    bound = CONST["msm_potential_relative_error_bound"]["value"]
    s = inputs.water_box(240, 1.4, margin=0.5, seed=9, with_velocities=False)
    m = oracle.msm(s.pos, s.q, s.box, A, H, 3)
    d = oracle.direct(s.pos, s.q)
    rel = np.sqrt(((m["pot"] - d["pot"]) ** 2).sum() / (d["pot"] ** 2).sum())
    assert rel < bound


def test_model_potentials_are_charge_derivatives():
    """phi_i = dU/dq_i for the whole model (exclusions included; LJ does not depend
    on q), by central differences in the charges, on atoms of several molecules."""
    import dataclasses
    s = inputs.water_box(60, 0.85, margin=0.5, seed=5, with_velocities=False)
    ref = oracle.model_forces(s, A, H, 3)
    d = 1e-5
    for atom in (0, 1, 2, 3 * 9 + 1, 3 * 13):
        qp = s.q.copy(); qp[atom] += d
        qm = s.q.copy(); qm[atom] -= d
        up = oracle.model_forces(dataclasses.replace(s, q=qp), A, H, 3)["energy"]
        um = oracle.model_forces(dataclasses.replace(s, q=qm), A, H, 3)["energy"]
        assert ref["pot"][atom] == pytest.approx((up - um) / (2 * d), rel=1e-7, abs=1e-7)


def test_oracle_results_do_not_depend_on_the_thread_count():
    s = inputs.water_box(300, 1.5, margin=0.5, seed=4, with_velocities=False)
    k = oracle.num_threads()
    try:
        oracle.set_num_threads(1)
        one = oracle.model_forces(s, A, H, 3)
    finally:
        oracle.set_num_threads(k)
    many = oracle.model_forces(s, A, H, 3)
    assert one["energy"] == many["energy"]
    assert np.array_equal(one["forces"], many["forces"]) and np.array_equal(one["pot"], many["pot"])
