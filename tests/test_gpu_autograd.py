"""msm_energy as a torch.autograd.Function: its backward returns dU/dr = -F and
dU/dq = phi (Sec. 2: F = -dU/dr), checked against central finite differences
of the library's FP64 energy and against the oracle's analytic forces.

Workload: 100,000 atoms of water-like charges in a 10 nm cube, 4 levels;
finite differences with a 1e-5 nm step on 64 random atoms (seed 2).
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


def test_backward_returns_forces_and_potentials(api, torch):
    s = inputs.water_box(3000, 3.1, margin=0.5, with_velocities=False)
    m = api.MSM(a=A, h=H, levels=3, precision="fp32")
    pos = torch.tensor(s.pos, device="cuda", requires_grad=True)
    q = torch.tensor(s.q, device="cuda", requires_grad=True)
    U = api.msm_energy(pos, q, s.box, m)
    (2.5 * U).backward()
    e, f, p = m.energy_forces(pos.detach(), q.detach(), s.box)
    assert float(U.detach()) == float(e)
    assert torch.equal(pos.grad, -2.5 * f) and torch.equal(q.grad, 2.5 * p)


@pytest.fixture(scope="module")
def water100k():
    cfg = inputs.WORKLOADS["water100k"]
    return inputs.water_box(cfg["n_atoms"], cfg["region"], margin=0.5, with_velocities=False)


def test_gradients_match_finite_differences_and_oracle(api, torch, water100k):
    s = water100k
    levels = inputs.WORKLOADS["water100k"]["levels"]
    rng = np.random.default_rng(2)
    atoms = rng.choice(s.n, 64, replace=False)
    m32 = api.MSM(a=A, h=H, levels=levels, precision="fp32")
    m64 = api.MSM(a=A, h=H, levels=levels, precision="fp64")
    pos = torch.tensor(s.pos, device="cuda", requires_grad=True)
    q = torch.tensor(s.q, device="cuda", requires_grad=True)
    U = api.msm_energy(pos, q, s.box, m32)
    U.backward()
    g32 = pos.grad.cpu().numpy()[atoms]
    e64, f64, p64 = m64.energy_forces(pos.detach(), q.detach(), s.box)
    g64 = -f64.cpu().numpy()[atoms]
    # central differences of the FP64 energy, step 1e-5 nm
    delta = 1e-5
    fd = np.zeros((64, 3))
    x = pos.detach().clone()
    for k, i in enumerate(atoms):
        for d in range(3):
            x[i, d] += delta
            ep = float(m64.energy_forces(x, q.detach(), s.box, forces=False, potentials=False)[0])
            x[i, d] -= 2 * delta
            em = float(m64.energy_forces(x, q.detach(), s.box, forces=False, potentials=False)[0])
            x[i, d] += delta
            fd[k, d] = (ep - em) / (2 * delta)
    scale = np.sqrt((g64 ** 2).sum())
    assert np.sqrt(((fd - g64) ** 2).sum()) / scale < 1e-6      # FD truncation + FP64 rounding of U
    assert np.sqrt(((g32 - g64) ** 2).sum()) / scale < 1e-4
    # the oracle's analytic forces on the same 64 atoms
    ref = oracle.msm(s.pos, s.q, s.box, A, H, levels)
    go = -ref["forces"][atoms]
    assert np.sqrt(((g64 - go) ** 2).sum()) / scale < 1e-12
    assert np.sqrt(((g32 - go) ** 2).sum()) / scale < 1e-4
    # dU/dq against the oracle's potentials
    dq = q.grad.cpu().numpy()
    assert np.sqrt(((dq - ref["pot"]) ** 2).sum() / (ref["pot"] ** 2).sum()) < 1e-4


def test_forward_computes_only_what_backward_needs(api, torch):
    """Only positions need a gradient: the energy is the same bits, pos.grad is -F and
    q gets no gradient; only charges: q.grad is phi."""
    s = inputs.water_box(900, 2.0, margin=0.5, with_velocities=False)
    m = api.MSM(a=A, h=H, levels=3, precision="fp32")
    e, f, p = m.energy_forces(torch.tensor(s.pos, device="cuda"), torch.tensor(s.q, device="cuda"), s.box)
    pos = torch.tensor(s.pos, device="cuda", requires_grad=True)
    q = torch.tensor(s.q, device="cuda")
    U = api.msm_energy(pos, q, s.box, m)
    U.backward()
    assert float(U.detach()) == float(e) and torch.equal(pos.grad, -f) and q.grad is None
    pos = torch.tensor(s.pos, device="cuda")
    q = torch.tensor(s.q, device="cuda", requires_grad=True)
    U = api.msm_energy(pos, q, s.box, m)
    U.backward()
    assert float(U.detach()) == float(e) and torch.equal(q.grad, p)


def test_batched_energies_differentiate_per_system(api, torch):
    """Three uneven systems in one batched evaluation: energies (B,) equal single
    evaluations bit for bit, and a weighted sum sum_b w_b U_b gives each system's
    atoms -w_b F and w_b phi."""
    systems = [inputs.random_cloud(n, L, seed=70 + k, neutral=True, margin=0.3)
               for k, (n, L) in enumerate(((500, 2.2), (1300, 3.0), (800, 2.6)))]
    m = api.MSM(a=A, h=H, levels=3, precision="fp32")
    offsets = np.cumsum([0] + [s.n for s in systems])
    pos = torch.tensor(np.concatenate([s.pos for s in systems]), device="cuda", requires_grad=True)
    q = torch.tensor(np.concatenate([s.q for s in systems]), device="cuda", requires_grad=True)
    boxes = np.stack([np.asarray(s.box, dtype=np.float64) for s in systems])
    U = api.msm_energy_batched(offsets, pos, q, boxes, m)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda")
    (w * U).sum().backward()
    for b, s in enumerate(systems):
        e, f, p = api.MSM(a=A, h=H, levels=3, precision="fp32").energy_forces(
            torch.tensor(s.pos, device="cuda"), torch.tensor(s.q, device="cuda"), s.box)
        o0, o1 = offsets[b], offsets[b + 1]
        assert float(U[b].detach()) == float(e)
        assert torch.equal(pos.grad[o0:o1], -w[b] * f) and torch.equal(q.grad[o0:o1], w[b] * p)
