"""Pins for the oracle's cutoff electrostatics, the coarse propagators of Sec. 5:
the simple cutoff (Coulomb's law for pairs within a; the paper's chosen G) and
Wolf summation (Wolf et al. 1999; the paper's proposed later G).

  * simple cutoff with a beyond the system's diameter is the direct Coulomb sum
    (Sec. 2, eq. coulomb; oracle.direct is pinned on its own); an isolated pair
    gives Coulomb's law inside a and nothing beyond; a rigid molecule alone
    gives exactly zero (its pairs are skipped);
  * Wolf summation with alpha = 0 on a neutral system whose pairs all lie
    inside a is the direct sum exactly (the shift and self terms cancel);
    with damping it reproduces the Madelung constant of rock salt,
    1.747565, at the central ion of an NaCl cluster (the test system of Wolf
    et al.), where the plain cutoff fails badly;
  * both: forces are -dU/dr and potentials dU/dq (central differences);
  * in the water model the cutoff methods skip the intramolecular pairs:
    two molecules closer than a give the intermolecular direct sum exactly.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1309_1889_gb300 import inputs

MADELUNG_NACL = 1.747565


def test_simple_cutoff_beyond_the_system_is_the_direct_sum():
    s = inputs.random_cloud(300, 1.3, seed=4)
    c = oracle.cutoff(s.pos, s.q, 3.0, "cutoff")
    d = oracle.direct(s.pos, s.q)
    assert c["energy"] == pytest.approx(d["energy"], rel=1e-12)
    assert np.allclose(c["forces"], d["forces"], rtol=1e-11, atol=1e-9)
    assert np.allclose(c["pot"], d["pot"], rtol=1e-11, atol=1e-9)


@pytest.mark.parametrize("r,inside", [(0.31, True), (1.19, True), (1.21, False), (2.5, False)])
def test_simple_cutoff_isolated_pair(r, inside):
    pos = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
    q = np.array([0.7, -0.4])
    c = oracle.cutoff(pos, q, 1.2, "cutoff")
    coul = oracle.KE * q[0] * q[1] / r
    if inside:
        assert c["energy"] == pytest.approx(coul, rel=1e-14)
        # Coulomb's law along the axis: F_1 = k_e q0 q1 / r^2 (repulsive if same sign)
        assert c["forces"][1, 0] == pytest.approx(oracle.KE * q[0] * q[1] / r ** 2, rel=1e-14)
        assert c["pot"][0] == pytest.approx(oracle.KE * q[1] / r, rel=1e-14)
    else:
        assert c["energy"] == 0.0 and np.all(c["forces"] == 0.0) and np.all(c["pot"] == 0.0)


def test_cutoff_methods_skip_the_pairs_of_a_rigid_molecule():
    s = inputs.water_box(3, 0.5, margin=0.5, with_velocities=False)
    for method, alpha in (("cutoff", 0.0), ("wolf", 2.0)):
        c = oracle.cutoff(s.pos, s.q, 1.2, method, alpha, n_mol=1)
        assert np.all(c["forces"] == 0.0)
        if method == "cutoff":
            assert c["energy"] == 0.0
        else:
            # only the neutralisation self term remains: -k_e [erfc(alpha a)/(2a) + alpha/sqrt(pi)] sum q^2
            selfc = math.erfc(2.0 * 1.2) / (2 * 1.2) + 2.0 / math.sqrt(math.pi)
            assert c["energy"] == pytest.approx(-oracle.KE * selfc * (s.q ** 2).sum(), rel=1e-13)


def test_wolf_undamped_neutral_system_inside_the_cutoff_is_the_direct_sum():
    s = inputs.random_cloud(200, 1.0, seed=6)            # neutral, diameter < sqrt(3) < a
    c = oracle.cutoff(s.pos, s.q, 2.0, "wolf", 0.0)
    d = oracle.direct(s.pos, s.q)
    assert c["energy"] == pytest.approx(d["energy"], rel=1e-10)
    assert np.allclose(c["forces"], d["forces"], rtol=1e-10, atol=1e-8)


def _nacl(K=9, r0=0.2):
    g = np.arange(-K, K + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X, Y, Z], -1).reshape(-1, 3) * r0 + 5.0
    q = ((-1.0) ** (X + Y + Z)).reshape(-1).astype(np.float64)
    centre = int(np.flatnonzero(((X == 0) & (Y == 0) & (Z == 0)).reshape(-1))[0])
    return pos, q, centre


def test_wolf_reproduces_the_madelung_constant_of_rock_salt():
    r0 = 0.2
    pos, q, c = _nacl(r0=r0)
    w = oracle.cutoff(pos, q, 6.5 * r0, "wolf", 0.5 / r0, ke=1.0)
    assert w["pot"][c] * r0 == pytest.approx(-MADELUNG_NACL, abs=2e-5)
    # the plain cutoff at the same radius misses it by far (the artefact Wolf removes)
    p = oracle.cutoff(pos, q, 6.5 * r0, "cutoff", ke=1.0)
    assert abs(p["pot"][c] * r0 + MADELUNG_NACL) > 0.5


@pytest.mark.parametrize("method,alpha", [("cutoff", 0.0), ("wolf", 2.5)])
def test_cutoff_forces_and_potentials_are_derivatives(method, alpha):
    s = inputs.random_cloud(80, 1.6, seed=12)
    a = 0.9
    # no pair of the moved atoms within 1e-3 of the cutoff: the simple cutoff's energy jumps there
    r = np.linalg.norm(s.pos[:, None] - s.pos[None], axis=-1)
    assert np.abs(r[[0, 17, 55]] - a).min() > 1e-3
    ref = oracle.cutoff(s.pos, s.q, a, method, alpha)
    d = 1e-6
    for atom in (0, 17, 55):
        for ax in range(3):
            xp = s.pos.copy(); xp[atom, ax] += d
            xm = s.pos.copy(); xm[atom, ax] -= d
            g = -(oracle.cutoff(xp, s.q, a, method, alpha)["energy"]
                  - oracle.cutoff(xm, s.q, a, method, alpha)["energy"]) / (2 * d)
            assert ref["forces"][atom, ax] == pytest.approx(g, rel=1e-6, abs=1e-5)
        qp = s.q.copy(); qp[atom] += d
        qm = s.q.copy(); qm[atom] -= d
        g = (oracle.cutoff(s.pos, qp, a, method, alpha)["energy"]
             - oracle.cutoff(s.pos, qm, a, method, alpha)["energy"]) / (2 * d)
        assert ref["pot"][atom] == pytest.approx(g, rel=1e-7, abs=1e-6)
    assert ref["energy"] == pytest.approx(0.5 * (s.q * ref["pot"]).sum(), rel=1e-13)


def test_water_model_with_cutoff_is_the_intermolecular_direct_sum():
    """Two molecules closer than a, LJ off: the model with the simple cutoff is the
    direct Coulomb sum over the nine intermolecular pairs, to rounding."""
    s = inputs.water_box(6, 0.45, margin=0.5, seed=2, with_velocities=False)
    assert s.n_mol == 2
    u_direct = 0.0
    for i in range(3):
        for j in range(3, 6):
            u_direct += oracle.KE * s.q[i] * s.q[j] / np.linalg.norm(s.pos[i] - s.pos[j])
    m = oracle.model_forces(s, 1.2, 0.25, 1, eps=0.0, method="cutoff")
    assert m["energy"] == pytest.approx(u_direct, rel=1e-13)
    # and the model's atoms outside the box are rejected, as for the MSM
    bad = s.pos.copy(); bad[0, 0] = s.box[0] - 0.1
    with pytest.raises(oracle.OracleError):
        oracle.model_forces(dataclasses.replace(s, pos=bad), 1.2, 0.25, 1, method="cutoff")
