"""Pins for the oracle's whole MSM evaluation (Sec. 3) against independent facts.

  * short range: cell-list sum == brute-force all-pairs sum; Newton's third law;
  * whole MSM vs the direct Coulomb sum (Sec. 2, eq. coulomb): the paper quotes
    < 1 % relative potential error for cutoffs above 0.8 nm with C^2 gamma and
    cubic Phi (Sec. 3); the error falls as h falls at fixed a;
  * forces are -dU/dr (central differences), potentials dU/dq, U = 1/2 q.phi,
    U quadratic in q;
  * invariance under shifting atoms and box origin together, under whole-grid
    shifts, and under the grid's own symmetries (axis swaps);
  * MSM does not conserve momentum (Sec. 3), but the net force is small and
    shrinks with h.
"""
import json
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_1309_1889_gb300 import inputs

A, H = 1.2, 0.25
GOLDEN = Path(__file__).resolve().parent / "golden"


def rel_rms(x, ref):
    return float(np.sqrt(((x - ref) ** 2).sum() / (ref ** 2).sum()))


@pytest.fixture(scope="module")
def water300():
    return inputs.water_box(300, 1.5, margin=0.5, with_velocities=False)


def test_short_range_cell_list_equals_brute_force(water300):
    s = water300
    p1, f1 = oracle.short_range(s.pos, s.q, A, s.box)
    p2, f2 = oracle.short_range(s.pos, s.q, A, s.box, brute=True)
    assert np.allclose(p1, p2, rtol=1e-13, atol=1e-12)
    assert np.allclose(f1, f2, rtol=1e-13, atol=1e-11)
    # Newton's third law for the pair part
    assert np.abs(f1.sum(0)).max() < 1e-10 * np.abs(f1).max() * s.n
    # evaluating a subset returns the same rows
    tg = np.array([5, 17, 250, 0])
    p3, f3 = oracle.short_range(s.pos, s.q, A, s.box, targets=tg)
    assert np.array_equal(p3, p1[tg]) and np.array_equal(f3, f1[tg])


def test_short_range_of_an_isolated_pair():
    # two charges r apart: phi = q_other g*(r); force along the pair with magnitude -q1 q2 g*'(r)
    box = np.array([0, 0, 0, 3.0, 3.0, 3.0])
    r = 0.7
    pos = np.array([[1.0, 1.2, 1.1], [1.0 + r, 1.2, 1.1]])
    q = np.array([0.6, -0.9])
    p, f = oracle.short_range(pos, q, A, box)
    gs = 1 / r - (15 / 8 - 5 / 4 * (r / A) ** 2 + 3 / 8 * (r / A) ** 4) / A
    assert p[0] == pytest.approx(-0.9 * gs, rel=1e-14) and p[1] == pytest.approx(0.6 * gs, rel=1e-14)
    assert f[0, 0] == pytest.approx(-f[1, 0], rel=1e-15)
    assert f[0, 1] == 0 and f[0, 2] == 0


def test_msm_matches_direct_sum_within_paper_bound(water300):
    s = water300
    m = oracle.msm(s.pos, s.q, s.box, A, H, 3)
    d = oracle.direct(s.pos, s.q)
    assert abs(m["energy"] - d["energy"]) / abs(d["energy"]) < 1e-2
    assert rel_rms(m["pot"], d["pot"]) < 1e-2
    assert rel_rms(m["forces"], d["forces"]) < 1e-2


def test_msm_error_falls_with_h():
    s = inputs.random_cloud(250, 2.0, seed=9, margin=0.3)
    d = oracle.direct(s.pos, s.q)
    errs = []
    for h in (0.5, 0.25, 0.125):
        m = oracle.msm(s.pos, s.q, s.box, A, h, 2)
        errs.append(rel_rms(m["forces"], d["forces"]))
    assert errs[0] > 2 * errs[1] > 4 * errs[2]
    slope = np.log(errs[0] / errs[2]) / np.log(4.0)
    assert slope > 1.5


def test_msm_single_level_is_grid_smoothing_of_gamma():
    # l = 1: the top level is the finest grid; result still approximates Coulomb
    s = inputs.random_cloud(120, 1.6, seed=2, margin=0.3)
    d = oracle.direct(s.pos, s.q)
    m1 = oracle.msm(s.pos, s.q, s.box, A, H, 1)
    m3 = oracle.msm(s.pos, s.q, s.box, A, H, 3)
    assert rel_rms(m1["forces"], d["forces"]) < 2e-2
    assert rel_rms(m3["forces"], d["forces"]) < 2e-2


def test_forces_are_minus_energy_gradient(water300):
    s = water300
    m = oracle.msm(s.pos, s.q, s.box, A, H, 3)
    rng = np.random.default_rng(0)
    delta = 1e-5
    for i in rng.choice(s.n, 6, replace=False):
        for d in range(3):
            pp = s.pos.copy(); pp[i, d] += delta
            pm = s.pos.copy(); pm[i, d] -= delta
            fd = -(oracle.msm(pp, s.q, s.box, A, H, 3)["energy"] - oracle.msm(pm, s.q, s.box, A, H, 3)["energy"]) / (2 * delta)
            assert m["forces"][i, d] == pytest.approx(fd, rel=2e-5, abs=2e-3)


def test_potentials_are_charge_derivatives_and_energy_is_quadratic(water300):
    s = water300
    m = oracle.msm(s.pos, s.q, s.box, A, H, 3)
    assert m["energy"] == pytest.approx(0.5 * (s.q * m["pot"]).sum(), rel=1e-13)
    m2 = oracle.msm(s.pos, 2.0 * s.q, s.box, A, H, 3)
    assert m2["energy"] == pytest.approx(4.0 * m["energy"], rel=1e-13)
    for i in (0, 1, 150, 299):
        dq = 1e-3
        qp = s.q.copy(); qp[i] += dq
        qm = s.q.copy(); qm[i] -= dq
        fd = (oracle.msm(s.pos, qp, s.box, A, H, 3)["energy"] - oracle.msm(s.pos, qm, s.box, A, H, 3)["energy"]) / (2 * dq)
        assert m["pot"][i] == pytest.approx(fd, rel=1e-9)


def test_invariant_under_joint_shift_and_grid_shift(water300):
    s = water300
    m = oracle.msm(s.pos, s.q, s.box, A, H, 3)
    shift = np.array([0.37, -1.1, 2.3])
    box = s.box.copy(); box[:3] += shift
    m2 = oracle.msm(s.pos + shift, s.q, box, A, H, 3)
    assert m2["energy"] == pytest.approx(m["energy"], rel=1e-12)
    assert np.allclose(m2["forces"], m["forces"], rtol=1e-9, atol=1e-8)
    # moving the atoms by whole finest-grid steps inside a larger box moves the grids with them
    big = s.box.copy(); big[:3] -= 4 * H; big[3:] += 8 * H
    e_a = oracle.msm(s.pos, s.q, big, A, H, 3)["energy"]
    e_b = oracle.msm(s.pos + 2 * H, s.q, big, A, H, 3)["energy"]
    # a whole-level-(l-1) shift (2^{l-1} h = 4h) maps every grid to itself
    e_c = oracle.msm(s.pos + 4 * H, s.q, big, A, H, 3)["energy"]
    assert e_c == pytest.approx(e_a, rel=1e-12)
    assert e_b == pytest.approx(e_a, rel=1e-4)


def test_invariant_under_axis_swap(water300):
    s = water300
    m = oracle.msm(s.pos, s.q, s.box, A, H, 3)
    perm = [2, 0, 1]
    box = np.concatenate([s.box[:3][perm], s.box[3:][perm]])
    m2 = oracle.msm(s.pos[:, perm], s.q, box, A, H, 3)
    assert m2["energy"] == pytest.approx(m["energy"], rel=1e-12)
    assert np.allclose(m2["forces"], m["forces"][:, perm], rtol=1e-10, atol=1e-8)


def test_net_force_small_and_shrinking_with_h():
    s = inputs.random_cloud(200, 2.0, seed=4, margin=0.3)
    ratios = []
    for h in (0.5, 0.25):
        f = oracle.msm(s.pos, s.q, s.box, A, h, 2)["forces"]
        ratios.append(np.linalg.norm(f.sum(0)) / (np.sqrt(s.n) * np.sqrt((f ** 2).sum(1).mean())))
    assert ratios[0] < 0.05 and ratios[1] < ratios[0]
    assert ratios[1] > 0.0  # MSM does not conserve momentum exactly


def test_stage_outputs_compose(water300):
    s = water300
    lv = 3
    m = oracle.msm(s.pos, s.q, s.box, A, H, lv, stages=True)
    q0 = oracle.anterpolate(s.pos, s.q, s.box, H, lv)
    assert np.array_equal(q0, m["qgrids"][0])
    q1 = oracle.restrict(q0, s.box, H, lv, 0)
    assert np.array_equal(q1, m["qgrids"][1])
    top = oracle.top_level(m["qgrids"][2], s.box, A, H, lv)
    assert np.array_equal(top, m["ugrids"][2])
    u1 = oracle.prolongate(m["ucuts"][1], top, s.box, H, lv, 1)
    assert np.array_equal(u1, m["ugrids"][1])
    phi_l, g_l = oracle.interpolate(s.pos, m["ugrids"][0], s.box, H, lv)
    assert np.array_equal(phi_l, m["phi_long"])
    ke = oracle.KE
    pot = ke * (m["phi_short"] + m["phi_long"] - s.q * 15 / (8 * A))
    assert np.allclose(pot, m["pot"], rtol=1e-15, atol=0)


def test_golden_regression():
    """Stored values written by tests/golden/make_golden.py (which calls only the oracle)."""
    g = json.loads((GOLDEN / "oracle_water300.json").read_text())
    s = inputs.water_box(g["n_atoms"], g["region"], margin=g["margin"], with_velocities=False)
    m = oracle.msm(s.pos, s.q, s.box, g["a"], g["h"], g["levels"])
    assert m["energy"] == pytest.approx(g["energy"], rel=1e-12)
    idx = np.array(g["force_rows"])
    assert np.allclose(m["forces"][idx], np.array(g["forces"]), rtol=1e-10, atol=1e-9)
