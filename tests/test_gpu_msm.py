"""GPU parity of the MSM evaluation against the FP64 CPU oracle (Sec. 3).

Every call goes through the C ABI (libmsm_gb300.so via the ctypes binding).
Bars:
  * cell lists (binning, sort order, cell starts): bit-exact;
  * FP64 path: relative RMS <= 1e-12 for forces, potentials and every stage,
    relative energy <= 1e-12;
  * FP32 path: relative force RMS <= 1e-4 and relative potential RMS <= 1e-4,
    relative energy <= 1e-6.
Per atom, besides the RMS bars: max_i |F_i - F_i^ref| <= MAX_F * F_rms and
max_i |phi_i - phi_i^ref| <= MAX_F * phi_rms (FP32: 2e-3, FP64: 1e-10), so a few
atoms wrong by a fraction of a percent cannot hide inside an RMS over thousands.
The FP32 energy bar follows from the arithmetic: U = 1/2 sum q_i phi_i is
accumulated in FP64 from per-atom potentials whose FP32 parts (short-range sum,
grid potential) have independent relative errors of ~1e-6, while the large terms
that cancel inside U -- every atom's self term and, in the water model, the
excluded pairs' smooth terms -- are formed in FP64.  The one exception is a
single atom, whose U is nothing but the cancelled self energy: there the bar is
relative to that self energy.
"""
import numpy as np
import pytest

import oracle
from paper_1309_1889_gb300 import inputs

pytestmark = pytest.mark.gpu

A, H = 1.2, 0.25
TOL = {"fp64": dict(f=1e-12, p=1e-12, e=1e-12, fmax=1e-10, vir=1e-12),
       "fp32": dict(f=1e-4, p=1e-4, e=1e-6, fmax=2e-3, vir=1e-6)}


def rel_rms(x, ref):
    x = np.asarray(x, dtype=np.float64); ref = np.asarray(ref, dtype=np.float64)
    den = np.sqrt((ref ** 2).sum())
    return float(np.sqrt(((x - ref) ** 2).sum()) / (den if den > 0 else 1.0))


def max_rel(x, ref):
    """Largest per-atom error over the RMS magnitude of the reference (vectors by norm)."""
    x = np.asarray(x, dtype=np.float64); ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim == 1:
        x, ref = x[:, None], ref[:, None]
    rms = np.sqrt((ref ** 2).sum(1).mean())
    return float(np.linalg.norm(x - ref, axis=1).max() / (rms if rms > 0 else 1.0))


def check_atoms(f, p, ref_f, ref_p, t):
    assert rel_rms(f, ref_f) <= t["f"] and max_rel(f, ref_f) <= t["fmax"]
    assert rel_rms(p, ref_p) <= t["p"] and max_rel(p, ref_p) <= t["fmax"]


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


@pytest.fixture(scope="module")
def water3k():
    return inputs.water_box(3000, 3.1, margin=0.5, with_velocities=False)


@pytest.fixture(scope="module")
def water3k_ref(water3k):
    s = water3k
    return oracle.msm(s.pos, s.q, s.box, A, H, 3, stages=True)


def _dev(torch, x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def test_cell_list_is_bit_exact(api, torch, water3k):
    for s in (water3k, inputs.random_cloud(5003, (2.7, 3.3, 1.9), seed=8, margin=0.0)):
        m = api.MSM(a=A, h=H, levels=3, precision="fp32")
        m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
        perm, start = m.cell_list(s.n)
        _, _, operm, ostart = oracle.bin_atoms(s.pos, s.box, H)
        assert np.array_equal(perm, operm)
        assert np.array_equal(start, ostart)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_short_range_matches_oracle(api, torch, water3k, water3k_ref, prec):
    s = water3k
    m = api.MSM(a=A, h=H, levels=3, precision=prec)
    m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
    phi, f = m.stage_atoms(s.n)
    t = TOL[prec]
    assert rel_rms(phi, water3k_ref["phi_short"]) <= t["p"]
    assert rel_rms(f, water3k_ref["f_short"]) <= t["f"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_every_grid_stage_matches_oracle(api, torch, water3k, water3k_ref, prec):
    s = water3k
    m = api.MSM(a=A, h=H, levels=3, precision=prec)
    m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
    ref = water3k_ref
    tol = TOL[prec]["p"]
    for k in range(3):
        assert m.grid_shape(k)[0] == ref["grid_shapes"][k]
        assert rel_rms(m.stage_grid(k, "q"), ref["qgrids"][k]) <= tol, ("q", k)
        assert rel_rms(m.stage_grid(k, "u"), ref["ugrids"][k]) <= tol, ("u", k)
    for k in range(2):
        assert rel_rms(m.stage_grid(k, "ucut"), ref["ucuts"][k]) <= tol, ("ucut", k)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_msm_matches_oracle_on_water(api, torch, water3k, water3k_ref, prec):
    s = water3k
    m = api.MSM(a=A, h=H, levels=3, precision=prec)
    e, f, p, vir = m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box, virial=True)
    ref = water3k_ref
    t = TOL[prec]
    assert abs(float(e) - ref["energy"]) <= t["e"] * abs(ref["energy"])
    check_atoms(f.cpu().numpy(), p.cpu().numpy(), ref["forces"], ref["pot"], t)
    # virial sum_i r_i . F_i, against the oracle's forces, relative to sum_i |r_i . F_i|
    vir_ref = (s.pos * ref["forces"]).sum()
    assert abs(float(vir) - vir_ref) <= t["vir"] * np.abs((s.pos * ref["forces"]).sum(1)).sum()


# ragged sizes, non-cubic boxes, every level count, empty-ish systems
CASES = [
    (1, (1.0, 1.0, 1.0), 1), (2, (1.3, 0.9, 1.1), 2), (33, (1.7, 1.7, 1.7), 2), (257, (2.3, 1.1, 3.4), 3),
    (1000, (2.0, 2.0, 2.0), 1), (1531, (3.3, 2.2, 2.7), 4), (4099, (3.1, 3.1, 3.1), 5),
]


@pytest.mark.parametrize("n,L,levels", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_msm_matches_oracle_on_clouds(api, torch, n, L, levels, prec):
    s = inputs.random_cloud(n, L, seed=n, margin=0.2)
    ref = oracle.msm(s.pos, s.q, s.box, A, H, levels)
    m = api.MSM(a=A, h=H, levels=levels, precision=prec)
    e, f, p = m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
    t = TOL[prec]
    # a single atom's U is its grid self energy minus the exact self term, nothing else:
    # the bar is relative to that self energy 1/2 k_e q^2 gamma(0)/a there
    scale = abs(ref["energy"]) if n > 1 else 0.5 * oracle.KE * (s.q ** 2).sum() * 15.0 / (8.0 * A)
    assert abs(float(e) - ref["energy"]) <= t["e"] * scale
    if n > 1:
        check_atoms(f.cpu().numpy(), p.cpu().numpy(), ref["forces"], ref["pot"], t)
    else:
        assert rel_rms(p.cpu().numpy(), ref["pot"]) <= t["p"]


def test_host_and_device_inputs_give_identical_bits(api, torch, water3k):
    s = water3k
    m = api.MSM(a=A, h=H, levels=3, precision="fp32")
    e1, f1, p1 = m.energy_forces(s.pos, s.q, s.box)                       # numpy -> host pointers
    e2, f2, p2 = m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
    assert e1 == float(e2)
    assert np.array_equal(f1, f2.cpu().numpy()) and np.array_equal(p1, p2.cpu().numpy())


def test_repeated_runs_are_bitwise_identical(api, torch, water3k):
    s = water3k
    for prec in ("fp32", "fp64"):
        m = api.MSM(a=A, h=H, levels=3, precision=prec)
        r1 = m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
        r2 = m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
        assert float(r1[0]) == float(r2[0])
        assert torch.equal(r1[1], r2[1]) and torch.equal(r1[2], r2[2])


def test_empty_system(api, torch):
    m = api.MSM(a=A, h=H, levels=3, precision="fp32")
    e, f, p = m.energy_forces(np.zeros((0, 3)), np.zeros(0), [0, 0, 0, 2.0, 2.0, 2.0])
    assert e == 0.0 and f.shape == (0, 3)


def test_out_of_box_and_non_finite_atoms_are_rejected(api, torch, water3k):
    s = water3k
    m = api.MSM(a=A, h=H, levels=3, precision="fp32")
    # valid atoms have 0 <= (x - x0)/h < floor(L/h) + 1: the box rounded up to whole cells of h
    pos = s.pos.copy(); pos[17, 2] = s.box[2] + (np.floor(s.box[5] / H) + 1) * H + 1e-9
    with pytest.raises(api.MSMError) as ei:
        m.energy_forces(pos, s.q, s.box)
    assert ei.value.name == "ERANGE"
    pos = s.pos.copy(); pos[3, 1] = s.box[1] - 1e-12
    with pytest.raises(api.MSMError) as ei:
        m.energy_forces(pos, s.q, s.box)
    assert ei.value.name == "ERANGE"
    pos = s.pos.copy(); pos[5, 0] = np.nan
    with pytest.raises(api.MSMError) as ei:
        m.energy_forces(pos, s.q, s.box)
    assert ei.value.name == "EINVAL"
    # the handle stays usable after an error
    e, f, p = m.energy_forces(s.pos, s.q, s.box)
    assert np.isfinite(e)


def test_batched_uneven_systems_equal_single_evaluations(api, torch):
    systems = [inputs.random_cloud(n, L, seed=n, margin=0.2) for n, L in ((100, 1.5), (731, 2.4), (2050, 2.9))]
    offs = np.cumsum([0] + [s.n for s in systems])
    pos = np.concatenate([s.pos for s in systems]); q = np.concatenate([s.q for s in systems])
    boxes = np.stack([s.box for s in systems])
    m = api.MSM(a=A, h=H, levels=3, precision="fp32")
    e, f, p = m.energy_forces_batched(offs, _dev(torch, pos), _dev(torch, q), boxes)
    for k, s in enumerate(systems):
        e1, f1, p1 = m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
        assert float(e[k]) == float(e1)
        assert torch.equal(f[offs[k]:offs[k + 1]], f1) and torch.equal(p[offs[k]:offs[k + 1]], p1)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_water_model_matches_oracle(api, torch, prec):
    # atoms within 0.6 nm of a face feel the flat-bottom wall (margin 0.5 nm)
    s = inputs.water_box(900, 2.1, margin=0.5, with_velocities=False)
    ref = oracle.model_forces(s, A, H, 3, wall_k=5000.0, wall_width=0.6)
    m = api.MSM(a=A, h=H, levels=3, precision=prec, model="water", wall_k=5000.0, wall_width=0.6)
    sd = inputs.System(pos=_dev(torch, s.pos), q=_dev(torch, s.q), mass=_dev(torch, s.mass), box=s.box,
                       n_mol=s.n_mol, lj=torch.tensor(s.lj, device="cuda"))
    e, f, p = m.system_forces(sd)
    t = TOL[prec]
    # FP64: the oracle forms U by subtracting the excluded pairs' full Coulomb energy (~1.4e2 x |U|
    # here) from its all-pairs MSM energy, the GPU path by skipping those pairs' g* and subtracting
    # their smooth part; the two FP64 roundings differ by ~1e-16 of that energy, which exceeds
    # 1e-12 |U|.  The FP32 bar is 1e-6 |U| itself (the FP32 rounding is far above the oracle's).
    scale = abs(ref["energy"]) + (_excluded_pair_energy(s) if prec == "fp64" else 0.0)
    assert abs(float(e) - ref["energy"]) <= t["e"] * scale
    check_atoms(f.cpu().numpy(), p.cpu().numpy(), ref["forces"], ref["pot"], t)


def _excluded_pair_energy(s):
    x = s.pos[: 3 * s.n_mol].reshape(-1, 3, 3); q = s.q[: 3 * s.n_mol].reshape(-1, 3)
    tot = 0.0
    for a, b in ((0, 1), (0, 2), (1, 2)):
        tot += np.abs(oracle.KE * q[:, a] * q[:, b] / np.linalg.norm(x[:, a] - x[:, b], axis=1)).sum()
    return tot


def test_fp32_and_fp64_paths_agree_at_full_size(api, torch):
    """1,000,000 atoms in a 21.5 nm water box, 5 levels (the throughput workload):
    sampled short-range rows against the oracle, the FP32 path against the FP64 path."""
    cfg = inputs.WORKLOADS["water1M"]
    s = inputs.water_box(cfg["n_atoms"], cfg["region"], margin=0.5, with_velocities=False)
    pos, q = _dev(torch, s.pos), _dev(torch, s.q)
    m32 = api.MSM(a=A, h=H, levels=cfg["levels"], precision="fp32")
    m64 = api.MSM(a=A, h=H, levels=cfg["levels"], precision="fp64")
    e32, f32, p32 = m32.energy_forces(pos, q, s.box)
    e64, f64, p64 = m64.energy_forces(pos, q, s.box)
    assert abs(float(e32) - float(e64)) <= 1e-6 * abs(float(e64))
    check_atoms(f32.cpu().numpy(), p32.cpu().numpy(), f64.cpu().numpy(), p64.cpu().numpy(), TOL["fp32"])
    rng = np.random.default_rng(0)
    tg = rng.choice(s.n, 512, replace=False)
    ophi, of = oracle.short_range(s.pos, s.q, A, s.box, targets=tg)
    phi64, fs64 = m64.stage_atoms(s.n)
    assert rel_rms(phi64[tg], ophi) <= 1e-12 and rel_rms(fs64[tg], of) <= 1e-12
    phi32, fs32 = m32.stage_atoms(s.n)
    assert rel_rms(phi32[tg], ophi) <= 1e-4 and rel_rms(fs32[tg], of) <= 1e-4


def test_paper_scale_box_fp32_matches_fp64_and_oracle_rows(api, torch):
    """12,700,000 atoms of the water-like model in a 30 x 65 x 65 nm box, 6 levels (the
    paper-scale workload): one FP32 evaluation against the FP64 path (forces and energy),
    sampled short-range rows against the oracle."""
    cfg = inputs.WORKLOADS["water12.7M"]
    s = inputs.water_box(cfg["n_atoms"], cfg["region"], margin=0.5, with_velocities=False)
    pos, q = _dev(torch, s.pos), _dev(torch, s.q)
    m32 = api.MSM(a=A, h=H, levels=cfg["levels"], precision="fp32")
    e32, f32, p32 = m32.energy_forces(pos, q, s.box)
    rng = np.random.default_rng(1)
    tg = rng.choice(s.n, 256, replace=False)
    phi32, fs32 = m32.stage_atoms(s.n)
    f32h = f32.cpu().numpy()
    del m32, f32, p32
    m64 = api.MSM(a=A, h=H, levels=cfg["levels"], precision="fp64")
    e64, f64, p64 = m64.energy_forces(pos, q, s.box)
    assert abs(float(e32) - float(e64)) <= 1e-6 * abs(float(e64))
    assert rel_rms(f32h, f64.cpu().numpy()) <= 1e-4
    ophi, of = oracle.short_range(s.pos, s.q, A, s.box, targets=tg)
    phi64, fs64 = m64.stage_atoms(s.n)
    assert rel_rms(phi64[tg], ophi) <= 1e-12 and rel_rms(fs64[tg], of) <= 1e-12
    assert rel_rms(phi32[tg], ophi) <= 1e-4 and rel_rms(fs32[tg], of) <= 1e-4


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_long_cutoff_takes_the_row_list_in_segments(api, torch, prec):
    """a = 2.4 nm on h = 0.2 nm cells (one level, dense top level): a warp's candidate
    rows outnumber its row list, so the short-range kernel walks them in segments; the
    short-range sums and the whole result still match the oracle."""
    a, h = 2.4, 0.2
    s = inputs.random_cloud(3000, (4.0, 4.0, 4.0), seed=41, neutral=True, margin=0.2)
    m = api.MSM(a=a, h=h, levels=1, precision=prec)
    e, f, p = m.energy_forces(_dev(torch, s.pos), _dev(torch, s.q), s.box)
    phi, fs = m.stage_atoms(s.n)
    t = TOL[prec]
    ophi, of = oracle.short_range(s.pos, s.q, a, s.box)
    assert rel_rms(phi, ophi) <= t["f"] and rel_rms(fs, of) <= t["f"]
    ref = oracle.msm(s.pos, s.q, s.box, a, h, 1)
    assert abs(float(e) - ref["energy"]) <= t["e"] * abs(ref["energy"])
    check_atoms(f.cpu().numpy(), p.cpu().numpy(), ref["forces"], ref["pot"], t)


def _water1m_device(torch, s, with_vel=False):
    t = lambda x: _dev(torch, x)
    return inputs.System(pos=t(s.pos), q=t(s.q), mass=t(s.mass), box=s.box, vel=t(s.vel) if with_vel else None,
                         n_mol=s.n_mol, lj=torch.tensor(s.lj, device="cuda"))


def _fp32_fp64_pair(api, sd, levels):
    out = {}
    for prec in ("fp64", "fp32"):
        m = api.MSM(a=A, h=H, levels=levels, precision=prec, model="water", wall_k=1e4, wall_width=0.8)
        e, f, p = m.system_forces(sd)
        out[prec] = (float(e), f.cpu().numpy(), p.cpu().numpy())
        m.close()
    return out["fp64"], out["fp32"]


def test_water_model_fp32_energy_at_full_size(api, torch):
    """The 1,000,000-atom water model (exclusions, LJ, wall) on the jittered-lattice
    start: FP32 forces within the FP32 bars, per atom too, and the FP32 energy within
    1e-6 of the energy's own scale, sum_i |q_i phi_i| / 2.  On this start the random
    orientations leave |U| at ~0.3 % of that scale (0.6 kJ/mol per molecule), and the
    FP32 pair sum carries a bias proportional to N (~3e-6 kJ/mol per atom: the rsqrt
    approximation's ulp errors, weighted by the charge products of the pairs, and the
    FP32 rounding of the gamma coefficients, both amplified by the intermolecular 1/r
    energy inside the cutoff spheres, ~+6e7 kJ/mol here), which is 1.4e-5 of |U|
    there.  The relaxed state below holds 1e-6 of |U| itself."""
    cfg = inputs.WORKLOADS["water1M"]
    s = inputs.water_box(cfg["n_atoms"], cfg["region"], margin=1.0, with_velocities=False)
    (e64, f64, p64), (e32, f32, p32) = _fp32_fp64_pair(api, _water1m_device(torch, s), cfg["levels"])
    scale = 0.5 * float(np.abs(s.q * p64).sum())
    print(f"lattice start: U64 {e64:.6f}, |dU| {abs(e32 - e64):.4f} kJ/mol = {abs(e32 - e64) / abs(e64):.2e} of |U|, "
          f"{abs(e32 - e64) / scale:.2e} of sum|q phi|/2 = {scale:.4e}")
    assert abs(e32 - e64) <= 1e-6 * scale
    check_atoms(f32, p32, f64, p64, TOL["fp32"])


def test_water_model_fp32_energy_relaxed_full_size(api, torch):
    """The same 1,000,000-atom box after 2 ps of its own FP32 dynamics with the
    velocities rescaled to 300 K every 0.1 ps (a liquid-like state: hydrogen-bonded
    orientations, |U| tens of kJ/mol per molecule): the FP32 energy within 1e-6 of
    |U| of the FP64 path's, forces within the FP32 bars.  The comparison is of the
    two GPU paths on one input; the FP64 path matches the oracle to 1e-12 elsewhere."""
    cfg = inputs.WORKLOADS["water1M"]
    s = inputs.water_box(cfg["n_atoms"], cfg["region"], margin=1.0, seed=0, vel_seed=1)
    d = _water1m_device(torch, s, with_vel=True)
    dof = 6 * s.n_mol + 3 * (s.n - 3 * s.n_mol)
    kb = 0.0083144626
    m = api.MSM(a=A, h=H, levels=cfg["levels"], precision="fp32", model="water", wall_k=1e4, wall_width=0.8)
    for _ in range(20):
        uk = m.md_run(d, 0.002, 50)
        d.vel.mul_(float(np.sqrt(0.5 * dof * kb * 300.0 / float(uk[-1, 1]))))
    m.close()
    torch.cuda.synchronize()
    (e64, f64, p64), (e32, f32, p32) = _fp32_fp64_pair(api, d, cfg["levels"])
    print(f"relaxed: U64 {e64:.6f}, |dU| {abs(e32 - e64):.4f} kJ/mol = {abs(e32 - e64) / abs(e64):.2e} of |U|")
    assert abs(e32 - e64) <= 1e-6 * abs(e64)
    check_atoms(f32, p32, f64, p64, TOL["fp32"])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_full_size_repeats_are_bitwise_identical(api, torch, prec):
    """1,000,000 atoms, 5 levels: two evaluations give the same bits, the lattice-cutoff
    grids of levels 0..3 included.  The lattice cutoff splits each tile's input planes
    between two blocks that add their partial sums into the zeroed output with atomic
    adds (hundreds of tiles in flight); two addends onto zero commute, so the order in
    which they land cannot show."""
    cfg = inputs.WORKLOADS["water1M"]
    s = inputs.water_box(cfg["n_atoms"], cfg["region"], margin=0.5, with_velocities=False)
    pos, q = _dev(torch, s.pos), _dev(torch, s.q)
    m = api.MSM(a=A, h=H, levels=cfg["levels"], precision=prec)
    runs = []
    for _ in range(2):
        e, f, p = m.energy_forces(pos, q, s.box)
        runs.append((float(e), f.clone(), p.clone(), [m.stage_grid(k, "ucut") for k in range(cfg["levels"] - 1)]))
    assert runs[0][0] == runs[1][0]
    assert torch.equal(runs[0][1], runs[1][1]) and torch.equal(runs[0][2], runs[1][2])
    for g0, g1 in zip(runs[0][3], runs[1][3]):
        assert np.array_equal(g0, g1)
