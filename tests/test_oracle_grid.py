"""Pins for the oracle's binning and grid operators (Sec. 3 long-range steps).

Checks come from the mathematics, not from the oracle's formulas:
  * binning == numpy's stable argsort of floor((x - x0)/h) keys;
  * anterpolation and restriction preserve charge, dipole and quadratic
    moments (Phi reproduces polynomials of degree <= 2);
  * interpolation and prolongation reproduce quadratic fields exactly;
  * anterpolation is the transpose of interpolation, restriction of
    prolongation (the operators are built from the same phi^k_mu);
  * lattice cutoff / top level equal all-pairs grid sums (brute force).
"""
import numpy as np
import pytest

import oracle
from paper_1309_1889_gb300 import inputs

A, H = 1.2, 0.25


def _cloud(n=400, L=2.3, seed=3):
    return inputs.random_cloud(n, L, seed=seed, margin=0.0)


def test_binning_matches_stable_argsort():
    s = _cloud(2000, 2.7, seed=5)
    cell, key, perm, start = oracle.bin_atoms(s.pos, s.box, H)
    t = (s.pos - s.box[:3]) * (1.0 / H)
    c = np.floor(t).astype(np.int64)
    assert np.array_equal(cell, c)
    nc = np.floor(s.box[3:] / H).astype(np.int64) + 1
    k = (c[:, 2] * nc[1] + c[:, 1]) * nc[0] + c[:, 0]
    assert np.array_equal(key, k)
    assert np.array_equal(perm, np.argsort(k, kind="stable"))
    counts = np.bincount(k, minlength=int(np.prod(nc)))
    assert np.array_equal(start, np.concatenate([[0], np.cumsum(counts)]))


def test_binning_rejects_bad_atoms():
    s = _cloud(50, 2.0)
    pos = s.pos.copy(); pos[7, 1] = np.nan
    with pytest.raises(oracle.OracleError):
        oracle.bin_atoms(pos, s.box, H)
    pos = s.pos.copy(); pos[3, 0] = s.box[0] - 1e-9
    with pytest.raises(oracle.OracleError):
        oracle.bin_atoms(pos, s.box, H)
    pos = s.pos.copy(); pos[3, 2] = s.box[2] + s.box[5] + 0.3
    with pytest.raises(oracle.OracleError):
        oracle.bin_atoms(pos, s.box, H)


def _coords(box, h, levels, k):
    lo, hi = oracle.grid_dims(box, h, levels)
    ax = [np.arange(lo[k, d], hi[k, d] + 1) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


def test_grid_extents():
    box = np.array([0, 0, 0, 21.5, 21.5, 21.5])
    shapes = oracle.grid_shapes(box, 0.25, 5)
    assert shapes == [(90, 90, 90), (48, 48, 48), (27, 27, 27), (16, 16, 16), (11, 11, 11)]
    lo, hi = oracle.grid_dims(np.array([0, 0, 0, 30.0, 65.0, 65.0]), 0.25, 6)
    assert tuple(hi[0] - lo[0] + 1) == (124, 264, 264)


def test_anterpolation_preserves_moments():
    s = _cloud()
    levels = 2
    q0 = oracle.anterpolate(s.pos, s.q, s.box, H, levels)
    X, Y, Z = _coords(s.box, H, levels, 0)
    t = (s.pos - s.box[:3]) / H
    assert q0.sum() == pytest.approx(s.q.sum(), abs=1e-12)
    for G, d in ((X, 0), (Y, 1), (Z, 2)):
        assert (q0 * G).sum() == pytest.approx((s.q * t[:, d]).sum(), abs=1e-10)
        assert (q0 * G * G).sum() == pytest.approx((s.q * t[:, d] ** 2).sum(), abs=1e-9)
    assert (q0 * X * Y).sum() == pytest.approx((s.q * t[:, 0] * t[:, 1]).sum(), abs=1e-9)


def _quad(X, Y, Z):
    return 0.7 + 0.3 * X - 0.2 * Y + 0.05 * Z + 0.02 * X * X - 0.03 * Y * Z + 0.01 * Z * Z + 0.015 * X * Y


def test_interpolation_reproduces_quadratics_and_gradients():
    s = _cloud()
    levels = 2
    X, Y, Z = _coords(s.box, H, levels, 0)
    u0 = _quad(X, Y, Z)
    phi, grad = oracle.interpolate(s.pos, u0, s.box, H, levels)
    t = (s.pos - s.box[:3]) / H
    exact = _quad(t[:, 0], t[:, 1], t[:, 2])
    assert np.allclose(phi, exact, rtol=0, atol=1e-12)
    gx = (0.3 + 0.04 * t[:, 0] + 0.015 * t[:, 1]) / H
    gy = (-0.2 - 0.03 * t[:, 2] + 0.015 * t[:, 0]) / H
    gz = (0.05 - 0.03 * t[:, 1] + 0.02 * t[:, 2]) / H
    assert np.allclose(grad, np.stack([gx, gy, gz], 1), rtol=0, atol=1e-11)


def test_anterpolation_is_transpose_of_interpolation():
    s = _cloud(300)
    levels = 2
    rng = np.random.default_rng(11)
    shp = oracle.grid_shapes(s.box, H, levels)[0][::-1]
    u = rng.standard_normal(shp)
    q0 = oracle.anterpolate(s.pos, s.q, s.box, H, levels)
    phi, _ = oracle.interpolate(s.pos, u, s.box, H, levels)
    assert (q0 * u).sum() == pytest.approx((s.q * phi).sum(), rel=1e-12)


@pytest.mark.parametrize("k", [0, 1])
def test_restriction_preserves_moments(k):
    box = np.array([0, 0, 0, 3.1, 2.6, 2.9])
    levels = 3
    rng = np.random.default_rng(k)
    shp = oracle.grid_shapes(box, H, levels)
    qk = rng.standard_normal(shp[k][::-1])
    qk1 = oracle.restrict(qk, box, H, levels, k)
    Xf, Yf, Zf = _coords(box, H, levels, k)
    Xc, Yc, Zc = _coords(box, H, levels, k + 1)
    assert qk1.sum() == pytest.approx(qk.sum(), abs=1e-10)
    for F, Cc in ((Xf, Xc), (Yf, Yc), (Zf, Zc)):
        assert (qk1 * 2 * Cc).sum() == pytest.approx((qk * F).sum(), abs=1e-9)
        assert (qk1 * (2 * Cc) ** 2).sum() == pytest.approx((qk * F * F).sum(), abs=1e-7)


def test_restriction_of_an_impulse_is_the_tap_product():
    box = np.array([0, 0, 0, 2.0, 2.0, 2.0])
    levels = 2
    shp = oracle.grid_shapes(box, H, levels)
    lo, hi = oracle.grid_dims(box, H, levels)
    qk = np.zeros(shp[0][::-1])
    nu = np.array([4, 3, 5])
    qk[tuple((nu - lo[0])[::-1])] = 1.0
    qc = oracle.restrict(qk, box, H, levels, 0)
    taps = {-3: -1 / 16, -2: 0.0, -1: 9 / 16, 0: 1.0, 1: 9 / 16, 2: 0.0, 3: -1 / 16}
    Xc, Yc, Zc = _coords(box, H, levels, 1)
    exp = np.zeros_like(qc)
    for idx in np.ndindex(qc.shape):
        m = np.array([Xc[idx], Yc[idx], Zc[idx]])
        off = nu - 2 * m
        if np.all(np.abs(off) <= 3):
            exp[idx] = taps[off[0]] * taps[off[1]] * taps[off[2]]
    assert np.array_equal(qc, exp)


def test_prolongation_reproduces_quadratics_and_is_restriction_transpose():
    box = np.array([0, 0, 0, 2.6, 3.0, 2.2])
    levels = 3
    k = 1
    shp = oracle.grid_shapes(box, H, levels)
    Xc, Yc, Zc = _coords(box, H, levels, k + 1)
    Xf, Yf, Zf = _coords(box, H, levels, k)
    uc = _quad(2 * Xc, 2 * Yc, 2 * Zc)                # a quadratic in level-k units
    zero = np.zeros(shp[k][::-1])
    uf = oracle.prolongate(zero, uc, box, H, levels, k)
    # exact where the fine point's full coarse support lies inside the coarse grid
    lo, hi = oracle.grid_dims(box, H, levels)
    inner = np.ones(uf.shape, bool)
    for F, d in ((Xf, 0), (Yf, 1), (Zf, 2)):
        inner &= (F - 3 >= 2 * lo[k + 1, d]) & (F + 3 <= 2 * hi[k + 1, d])
    assert inner.sum() > 50
    assert np.allclose(uf[inner], _quad(Xf, Yf, Zf)[inner], atol=1e-12)
    # adjointness
    rng = np.random.default_rng(4)
    q = rng.standard_normal(shp[k][::-1]); u = rng.standard_normal(shp[k + 1][::-1])
    Rq = oracle.restrict(q, box, H, levels, k)
    Pu = oracle.prolongate(zero, u, box, H, levels, k)
    assert (Rq * u).sum() == pytest.approx((q * Pu).sum(), rel=1e-12)
    # the cut-off part is added unchanged
    ucut = rng.standard_normal(shp[k][::-1])
    assert np.allclose(oracle.prolongate(ucut, u, box, H, levels, k), ucut + Pu, atol=1e-13)


def _gk_table(a, h, k, levels, dmax):
    # g^k at every integer offset (in level-k grid units): values from the pinned kernel
    tab = {}
    for d2 in range(3 * dmax * dmax + 1):
        tab[d2] = oracle.gk(np.sqrt(d2) * h * 2**k, a, k, levels)
    return tab


@pytest.mark.parametrize("k", [0, 1])
def test_lattice_cutoff_equals_all_pairs_sum(k):
    box = np.array([0, 0, 0, 1.9, 2.2, 1.7])
    levels = 3
    shp = oracle.grid_shapes(box, H, levels)[k]
    rng = np.random.default_rng(7 + k)
    qk = rng.standard_normal(shp[::-1])
    u = oracle.lattice_cutoff(qk, box, A, H, levels, k)
    X, Y, Z = _coords(box, H, levels, k)
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    D2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    tab = _gk_table(A, H, k, levels, int(np.abs(P).max() * 2 + 2))
    G = np.vectorize(tab.__getitem__)(D2)
    ref = (G @ qk.ravel()).reshape(qk.shape)
    assert np.allclose(u, ref, rtol=1e-13, atol=1e-13)


def test_lattice_cutoff_of_an_impulse_is_the_kernel():
    box = np.array([0, 0, 0, 5.0, 5.0, 5.0])
    levels = 2
    shp = oracle.grid_shapes(box, H, levels)[0]
    lo, _ = oracle.grid_dims(box, H, levels)
    q = np.zeros(shp[::-1])
    nu = np.array([10, 9, 11])
    q[tuple((nu - lo[0])[::-1])] = 1.0
    u = oracle.lattice_cutoff(q, box, A, H, levels, 0)
    X, Y, Z = _coords(box, H, levels, 0)
    r = np.sqrt((X - nu[0]) ** 2 + (Y - nu[1]) ** 2 + (Z - nu[2]) ** 2) * H
    ref = np.vectorize(lambda x: oracle.gk(x, A, 0, levels))(r)
    assert np.allclose(u, ref, rtol=1e-14, atol=1e-15)
    assert np.all(u[r >= 2 * A] == 0.0)
    assert np.count_nonzero(u) > 3000


def test_top_level_equals_all_pairs_sum():
    box = np.array([0, 0, 0, 2.1, 2.0, 2.3])
    levels = 2
    k = levels - 1
    shp = oracle.grid_shapes(box, H, levels)[k]
    qt = np.random.default_rng(2).standard_normal(shp[::-1])
    u = oracle.top_level(qt, box, A, H, levels)
    X, Y, Z = _coords(box, H, levels, k)
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    D2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    tab = _gk_table(A, H, k, levels, int(np.abs(P).max() * 2 + 2))
    G = np.vectorize(tab.__getitem__)(D2)
    assert np.allclose(u.ravel(), G @ qt.ravel(), rtol=1e-13, atol=1e-13)
