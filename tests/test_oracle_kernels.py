"""Pins for the oracle's smoothing function, level kernels and nodal basis.

Every check here comes from a property the paper fixes (Sec. 3), not from the
oracle's own formulas: C^2 matching of gamma to 1/rho at rho = 1 (three
conditions that fix the three Taylor coefficients), the telescoping identity
g* + g^0 + ... + g^{l-1} = 1/r, the cutoffs of g* and g^k, the scaling between
levels, and the interpolating / polynomial-reproducing properties of the
cubic C1 basis Phi.
"""
import math

import numpy as np
import pytest

import oracle


def test_gamma_matches_inverse_from_one_on():
    for rho in [1.0, 1.0000001, 1.5, 2.0, 7.3, 1e3]:
        assert oracle.gamma(rho) == pytest.approx(1.0 / rho, rel=1e-15)


def test_gamma_is_c2_at_one():
    # value, slope and curvature of the polynomial branch must equal those of
    # 1/rho at rho = 1: (1, -1, 2).  These three conditions fix gamma.
    e = 1e-4
    g = oracle.gamma
    left = [g(1 - 2 * e), g(1 - e), g(1 - 1e-12)]
    assert left[2] == pytest.approx(1.0, abs=1e-11)
    d1 = (g(1 - 1e-7) - g(1 - 2e-7)) / 1e-7
    assert d1 == pytest.approx(-1.0, abs=1e-6)
    def d2(c):   # second difference of the polynomial branch centred at c < 1
        return (g(c + e) - 2 * g(c) + g(c - e)) / e**2
    # linear extrapolation of the curvature to rho = 1 from the left; 1/rho has 2 there
    assert 2 * d2(1 - 3 * e) - d2(1 - 6 * e) == pytest.approx(2.0, abs=1e-4)
    # even, smooth below 1: gamma is a polynomial in rho^2 with gamma'(0) = 0
    assert (g(1e-4) - g(0.0)) / 1e-4 == pytest.approx(0.0, abs=1e-3)


def test_dgamma_is_derivative():
    for rho in [0.05, 0.3, 0.7, 0.99, 1.01, 1.7, 4.0]:
        e = 1e-6
        fd = (oracle.gamma(rho + e) - oracle.gamma(rho - e)) / (2 * e)
        assert oracle.dgamma(rho) == pytest.approx(fd, rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("levels", [1, 2, 3, 5, 6])
def test_kernel_telescoping_sums_to_inverse_distance(levels):
    a = 1.2
    for r in [0.05, 0.3, 0.9, 1.19, 1.2, 1.7, 2.5, 4.9, 9.7, 20.0, 60.0]:
        total = oracle.gstar(r, a) + sum(oracle.gk(r, a, k, levels) for k in range(levels))
        assert total == pytest.approx(1.0 / r, rel=2e-14)


def test_gstar_vanishes_beyond_cutoff_and_is_continuous():
    a = 1.2
    assert oracle.gstar(a, a) == 0.0
    assert oracle.gstar(1.5 * a, a) == 0.0
    assert abs(oracle.gstar(a * (1 - 1e-9), a)) < 1e-9
    # force of g* also vanishes at the cutoff (C^1 smoothing)
    assert abs(oracle.dgstar(a * (1 - 1e-9), a)) < 1e-8
    for r in [0.1, 0.5, 1.1]:
        e = 1e-7
        fd = (oracle.gstar(r + e, a) - oracle.gstar(r - e, a)) / (2 * e)
        assert oracle.dgstar(r, a) == pytest.approx(fd, rel=1e-6)


def test_level_kernels_vanish_beyond_twice_their_cutoff():
    a, l = 1.2, 5
    for k in range(l - 1):
        c = 2 ** (k + 1) * a
        assert oracle.gk(c, a, k, l) == 0.0
        assert oracle.gk(1.3 * c, a, k, l) == 0.0
        assert abs(oracle.gk(c * (1 - 1e-9), a, k, l)) < 1e-9
    # the top level kernel does not vanish: it is gamma(r/2^{l-1}a)/(2^{l-1}a)
    assert oracle.gk(100.0, a, l - 1, l) == pytest.approx(1 / 100.0, rel=1e-15)


def test_level_kernel_scaling_between_levels():
    a, l = 1.2, 6
    for k in range(l - 1):
        for r in [0.0, 0.25, 0.8, 1.3, 2.0]:
            assert oracle.gk(2**k * r, a, k, l) == pytest.approx(2.0**-k * oracle.gk(r, a, 0, l), rel=1e-14, abs=1e-300)


def test_self_term_limit():
    # g*(r) + gamma(0)/a -> 1/r as r -> 0: the smooth self potential is gamma(0)/a = 15/(8a)
    a = 1.2
    r = 1e-6
    assert 1.0 / r - oracle.gstar(r, a) == pytest.approx(15.0 / (8.0 * a), rel=1e-6)


def test_phi_interpolates_and_has_support_two():
    assert oracle.Phi(0.0) == 1.0
    for t in [1.0, -1.0, 2.0, -2.0, 2.5, -3.0, 10.0]:
        assert oracle.Phi(t) == 0.0


def test_phi_is_c1():
    for t0 in [1.0, 2.0]:
        e = 1e-8
        assert oracle.Phi(t0 - e) == pytest.approx(oracle.Phi(t0 + e), abs=1e-7)
        assert oracle.dPhi(t0 - e) == pytest.approx(oracle.dPhi(t0 + e), abs=1e-6)
    assert oracle.dPhi(0.0) == 0.0


@pytest.mark.parametrize("t", [0.0, 0.13, 0.5, 0.77, 0.999999])
def test_phi_reproduces_quadratics_but_not_cubics(t):
    mus = np.arange(-1, 3)
    w = np.array([oracle.Phi(t - m) for m in mus])
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert (w * mus).sum() == pytest.approx(t, abs=1e-15)
    assert (w * mus**2).sum() == pytest.approx(t * t, abs=1e-14)
    if 0.05 < t < 0.95 and abs(t - 0.5) > 0.05:   # t = 1/2 is exact by symmetry
        assert abs((w * mus**3).sum() - t**3) > 1e-4


def test_dphi_is_derivative():
    for t in [-1.7, -1.2, -0.6, -0.1, 0.1, 0.4, 0.9, 1.1, 1.5, 1.95]:
        e = 1e-7
        fd = (oracle.Phi(t + e) - oracle.Phi(t - e)) / (2 * e)
        assert oracle.dPhi(t) == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_restriction_taps_are_phi_at_half_integers():
    # Phi(n/2) for n = -3..3 gives the 1-D restriction stencil [-1, 0, 9, 16, 9, 0, -1]/16
    taps = [oracle.Phi(n / 2.0) for n in range(-3, 4)]
    assert taps == [-1 / 16, 0.0, 9 / 16, 1.0, 9 / 16, 0.0, -1 / 16]
