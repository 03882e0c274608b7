"""FP64 CPU oracle for the multilevel summation method (MSM), velocity Verlet and parareal.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product package never imports
it, and it imports nothing from the product package.

The arithmetic lives in ``msm_oracle.c`` (plain C, FP64, ``-ffp-contract=off``);
this module compiles it with gcc on first use and marshals numpy arrays.
Every function cites the part of the paper it follows in the C source.
Parity is pinned by ``tests/test_oracle_*.py`` (closed forms, brute force,
polynomial exactness, direct Coulomb sums, finite differences, parareal
invariants) -- no function here is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sysconfig
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "msm_oracle.c"
BUILD = HERE / "_build"
LIB = BUILD / "liboracle.so"

KE = 138.935458  # 1/(4 pi eps0) in kJ mol^-1 nm e^-2

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (OpenMP if available).  Idempotent."""
    BUILD.mkdir(exist_ok=True)
    if LIB.exists() and not force and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp.so")
    try:
        subprocess.run(base + ["-fopenmp", str(SRC), "-o", str(tmp), "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [str(SRC), "-o", str(tmp), "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(LIB))
        d, i, i64, p = C.c_double, C.c_int, C.c_int64, C.c_void_p
        for name in ("orc_gamma", "orc_dgamma", "orc_Phi", "orc_dPhi"):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [d]
        L.orc_gstar.restype = d; L.orc_gstar.argtypes = [d, d]
        L.orc_dgstar.restype = d; L.orc_dgstar.argtypes = [d, d]
        L.orc_gk.restype = d; L.orc_gk.argtypes = [d, d, i, i]
        L.orc_grid_dims.restype = i; L.orc_grid_dims.argtypes = [p, d, i, p, p]
        L.orc_bin.restype = i; L.orc_bin.argtypes = [i64, p, p, d, p, p, p, p]
        L.orc_short_range_brute.restype = None; L.orc_short_range_brute.argtypes = [i64, p, p, d, p, p]
        L.orc_short_range.restype = i; L.orc_short_range.argtypes = [i64, p, p, d, p, i64, p, p, p]
        L.orc_anterpolate.restype = i; L.orc_anterpolate.argtypes = [p, p, d, p, i64, p, p, p]
        L.orc_restrict.restype = None; L.orc_restrict.argtypes = [p, p, i, p, p]
        L.orc_lattice_cutoff.restype = None; L.orc_lattice_cutoff.argtypes = [p, p, i, i, d, d, p, p]
        L.orc_top_level.restype = None; L.orc_top_level.argtypes = [p, p, i, d, d, p, p]
        L.orc_prolongate.restype = None; L.orc_prolongate.argtypes = [p, p, i, p, p, p]
        L.orc_interpolate.restype = None; L.orc_interpolate.argtypes = [p, p, d, p, i64, p, p, p, p]
        L.orc_msm.restype = i; L.orc_msm.argtypes = [p, i, i64, p, p, p, p, p, p, p]
        L.orc_direct.restype = None; L.orc_direct.argtypes = [i64, p, p, d, p, p, p]
        L.orc_cutoff.restype = i; L.orc_cutoff.argtypes = [i, d, d, d, i64, i64, p, p, p, p, p]
        L.orc_model_forces.restype = i
        L.orc_model_forces.argtypes = [p, i, i64, i64, p, p, p, p, p, p, p]
        L.orc_model_forces_split.restype = i
        L.orc_model_forces_split.argtypes = [p, i, i64, i64, p, p, p, p, p, p, p, p]
        L.orc_md_run.restype = i
        L.orc_md_run.argtypes = [p, i, i64, i64, p, p, p, p, p, p, d, i, p]
        L.orc_parareal.restype = i
        L.orc_parareal.argtypes = [p, p, i64, i64, p, p, p, p, i, i, d, p, p, p, p]
        L.orc_parareal_window.restype = i
        L.orc_parareal_window.argtypes = [p, p, i64, i64, p, p, p, p, i, i, i, d, p, p, p, p]
        L.orc_num_threads.restype = i; L.orc_num_threads.argtypes = []
        L.orc_set_num_threads.restype = None; L.orc_set_num_threads.argtypes = [i]
        L.orc_project_rigid.restype = i
        L.orc_project_rigid.argtypes = [i64, i64, p, d, d, p, p]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc != 0:
        raise OracleError(f"oracle returned status {rc}")


# --- scalar functions -------------------------------------------------------

def gamma(rho):
    return lib().orc_gamma(float(rho))


def dgamma(rho):
    return lib().orc_dgamma(float(rho))


def gstar(r, a):
    return lib().orc_gstar(float(r), float(a))


def dgstar(r, a):
    return lib().orc_dgstar(float(r), float(a))


def gk(r, a, k, levels):
    return lib().orc_gk(float(r), float(a), int(k), int(levels))


def Phi(t):
    return lib().orc_Phi(float(t))


def dPhi(t):
    return lib().orc_dPhi(float(t))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(k: int) -> None:
    """Threads of the oracle's OpenMP loops (its results are the same for any count)."""
    lib().orc_set_num_threads(int(k))


# --- grids -----------------------------------------------------------------

def grid_dims(box, h, levels):
    """(lo, hi) arrays of shape (levels, 3): inclusive index range per level and axis."""
    lo = np.zeros((levels, 3), dtype=np.int64)
    hi = np.zeros((levels, 3), dtype=np.int64)
    _check(lib().orc_grid_dims(_ptr(_f64(box)), float(h), int(levels), _ptr(lo), _ptr(hi)))
    return lo, hi


def grid_shapes(box, h, levels):
    lo, hi = grid_dims(box, h, levels)
    return [tuple(int(v) for v in (hi[k] - lo[k] + 1)) for k in range(levels)]


def bin_atoms(pos, box, h):
    """Bit-exact binning: (cell (n,3), key (n,), perm (n,), cell_start (ncells+1,))."""
    pos = _f64(pos); box = _f64(box)
    n = pos.shape[0]
    nc = [int(np.floor(box[3 + d] / h)) + 1 for d in range(3)]
    cell = np.zeros((n, 3), dtype=np.int64)
    key = np.zeros(n, dtype=np.int64)
    perm = np.zeros(n, dtype=np.int64)
    start = np.zeros(nc[0] * nc[1] * nc[2] + 1, dtype=np.int64)
    _check(lib().orc_bin(n, _ptr(pos), _ptr(box), float(h), _ptr(cell), _ptr(key), _ptr(perm), _ptr(start)))
    return cell, key, perm, start


def short_range(pos, q, a, box, targets=None, brute=False):
    pos = _f64(pos); q = _f64(q)
    n = pos.shape[0]
    if brute:
        phi = np.zeros(n); f = np.zeros((n, 3))
        lib().orc_short_range_brute(n, _ptr(pos), _ptr(q), float(a), _ptr(phi), _ptr(f))
        return phi, f
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    m = n if t is None else t.shape[0]
    phi = np.zeros(m); f = np.zeros((m, 3))
    _check(lib().orc_short_range(n, _ptr(pos), _ptr(q), float(a), _ptr(_f64(box)),
                                 0 if t is None else m, _ptr(t), _ptr(phi), _ptr(f)))
    return phi, f


def anterpolate(pos, q, box, h, levels):
    lo, hi = grid_dims(box, h, levels)
    shp = tuple(int(v) for v in (hi[0] - lo[0] + 1))
    out = np.zeros(shp[::-1])  # (nz, ny, nx), x fastest
    pos = _f64(pos); q = _f64(q)
    _check(lib().orc_anterpolate(_ptr(lo), _ptr(hi), float(h), _ptr(_f64(box)), pos.shape[0],
                                 _ptr(pos), _ptr(q), _ptr(out)))
    return out


def restrict(qk, box, h, levels, k):
    lo, hi = grid_dims(box, h, levels)
    shp = tuple(int(v) for v in (hi[k + 1] - lo[k + 1] + 1))
    out = np.zeros(shp[::-1])
    lib().orc_restrict(_ptr(lo), _ptr(hi), int(k), _ptr(_f64(qk)), _ptr(out))
    return out


def lattice_cutoff(qk, box, a, h, levels, k):
    lo, hi = grid_dims(box, h, levels)
    out = np.zeros_like(_f64(qk))
    lib().orc_lattice_cutoff(_ptr(lo), _ptr(hi), int(k), int(levels), float(a), float(h), _ptr(_f64(qk)), _ptr(out))
    return out


def top_level(qt, box, a, h, levels):
    lo, hi = grid_dims(box, h, levels)
    out = np.zeros_like(_f64(qt))
    lib().orc_top_level(_ptr(lo), _ptr(hi), int(levels), float(a), float(h), _ptr(_f64(qt)), _ptr(out))
    return out


def prolongate(ucut, uk1, box, h, levels, k):
    lo, hi = grid_dims(box, h, levels)
    out = np.zeros_like(_f64(ucut))
    lib().orc_prolongate(_ptr(lo), _ptr(hi), int(k), _ptr(_f64(ucut)), _ptr(_f64(uk1)), _ptr(out))
    return out


def interpolate(pos, u0, box, h, levels):
    lo, hi = grid_dims(box, h, levels)
    pos = _f64(pos)
    n = pos.shape[0]
    phi = np.zeros(n); grad = np.zeros((n, 3))
    lib().orc_interpolate(_ptr(lo), _ptr(hi), float(h), _ptr(_f64(box)), n, _ptr(pos), _ptr(_f64(u0)),
                          _ptr(phi), _ptr(grad))
    return phi, grad


class _Stage(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in
                ("phi_short", "f_short", "phi_long", "grad_long", "qgrid", "ucut", "ugrid")]


def msm(pos, q, box, a, h, levels, ke=KE, stages=False):
    """One MSM evaluation: dict(energy, forces (n,3), pot (n,), [stage arrays])."""
    pos = _f64(pos); q = _f64(q); box = _f64(box)
    n = pos.shape[0]
    forces = np.zeros((n, 3)); pot = np.zeros(n); e = np.zeros(1)
    prm = _f64([a, h, ke])
    st = None
    out = {}
    if stages:
        shapes = grid_shapes(box, h, levels)
        sizes = [int(np.prod(s)) for s in shapes]
        tot = sum(sizes)
        arrs = dict(phi_short=np.zeros(n), f_short=np.zeros((n, 3)), phi_long=np.zeros(n),
                    grad_long=np.zeros((n, 3)), qgrid=np.zeros(tot), ucut=np.zeros(tot), ugrid=np.zeros(tot))
        st = _Stage(**{k: v.ctypes.data for k, v in arrs.items()})
        out.update(arrs)
        out["grid_shapes"] = shapes
    _check(lib().orc_msm(_ptr(prm), int(levels), n, _ptr(pos), _ptr(q), _ptr(box), _ptr(e), _ptr(forces),
                         _ptr(pot), None if st is None else C.byref(st)))
    if stages:
        off = np.cumsum([0] + sizes)
        out["qgrids"] = [out["qgrid"][off[k]:off[k + 1]].reshape(shapes[k][::-1]) for k in range(levels)]
        out["ugrids"] = [out["ugrid"][off[k]:off[k + 1]].reshape(shapes[k][::-1]) for k in range(levels)]
        out["ucuts"] = [out["ucut"][off[k]:off[k + 1]].reshape(shapes[k][::-1]) for k in range(levels - 1)]
    out.update(energy=float(e[0]), forces=forces, pot=pot)
    return out


def direct(pos, q, ke=KE):
    pos = _f64(pos); q = _f64(q)
    n = pos.shape[0]
    e = np.zeros(1); f = np.zeros((n, 3)); p = np.zeros(n)
    lib().orc_direct(n, _ptr(pos), _ptr(q), float(ke), _ptr(e), _ptr(f), _ptr(p))
    return dict(energy=float(e[0]), forces=f, pot=p)


METHODS = {"msm": 0, "cutoff": 1, "wolf": 2}


def cutoff(pos, q, a, method="cutoff", alpha=0.0, ke=KE, n_mol=0):
    """Coarse-propagator electrostatics (Sec. 5): simple cutoff or Wolf summation,
    brute force over all pairs.  dict(energy, forces, pot)."""
    pos = _f64(pos); q = _f64(q)
    n = pos.shape[0]
    e = np.zeros(1); f = np.zeros((n, 3)); p = np.zeros(n)
    _check(lib().orc_cutoff(METHODS[method], float(a), float(alpha), float(ke), n, int(n_mol), _ptr(pos), _ptr(q),
                            _ptr(e), _ptr(f), _ptr(p)))
    return dict(energy=float(e[0]), forces=f, pot=p)


# --- water model, dynamics, parareal ----------------------------------------

LJ_SIGMA = 0.315061    # nm, O-O
LJ_EPSILON = 0.6364    # kJ/mol


def model_params(a, h, ke=KE, sigma=LJ_SIGMA, eps=LJ_EPSILON, d_oh=0.09572, d_hh=None, wall_k=0.0, wall_width=0.0,
                 method="msm", wolf_alpha=0.0, mts=0):
    """mts: fast steps per slow step of md_run's multiple time stepping (<= 1: plain velocity Verlet)."""
    if d_hh is None:
        import math
        d_hh = 2.0 * d_oh * math.sin(math.radians(104.52) / 2.0)
    return _f64([a, h, ke, sigma, eps, d_oh, d_hh, wall_k, wall_width, METHODS[method], wolf_alpha, mts])


def model_forces(sys, a, h, levels, ke=KE, pos=None, **kw):
    x = _f64(sys.pos if pos is None else pos)
    mdp = model_params(a, h, ke, **kw)
    n = x.shape[0]
    e = np.zeros(1); f = np.zeros((n, 3)); p = np.zeros(n)
    lj = np.ascontiguousarray(sys.lj, dtype=np.uint8)
    _check(lib().orc_model_forces(_ptr(mdp), int(levels), n, int(sys.n_mol), _ptr(x), _ptr(_f64(sys.q)),
                                  _ptr(lj), _ptr(_f64(sys.box)), _ptr(e), _ptr(f), _ptr(p)))
    return dict(energy=float(e[0]), forces=f, pot=p)


def model_forces_split(sys, a, h, levels, ke=KE, pos=None, **kw):
    """The model's forces split for multiple time stepping: fast (short-range g*
    over non-excluded pairs, Lennard-Jones, wall) and slow (grid part minus the
    excluded pairs' smooth part); energy and its slow part."""
    x = _f64(sys.pos if pos is None else pos)
    mdp = model_params(a, h, ke, **kw)
    n = x.shape[0]
    e = np.zeros(1); es = np.zeros(1); ff = np.zeros((n, 3)); fs = np.zeros((n, 3))
    lj = np.ascontiguousarray(sys.lj, dtype=np.uint8)
    _check(lib().orc_model_forces_split(_ptr(mdp), int(levels), n, int(sys.n_mol), _ptr(x), _ptr(_f64(sys.q)),
                                        _ptr(lj), _ptr(_f64(sys.box)), _ptr(e), _ptr(es), _ptr(ff), _ptr(fs)))
    return dict(energy=float(e[0]), energy_slow=float(es[0]), f_fast=ff, f_slow=fs)


def md_run(sys, a, h, levels, dt, n_steps, ke=KE, x=None, v=None, **kw):
    """Velocity Verlet + SHAKE/RATTLE (with mts=k > 1: the multiple-time-step
    impulse method, the grid part every k steps).  Returns (x, v, uk (n_steps+1, 2))."""
    x = _f64(sys.pos if x is None else x).copy()
    v = _f64(sys.vel if v is None else v).copy()
    mdp = model_params(a, h, ke, **kw)
    n = x.shape[0]
    uk = np.zeros((n_steps + 1, 2))
    lj = np.ascontiguousarray(sys.lj, dtype=np.uint8)
    _check(lib().orc_md_run(_ptr(mdp), int(levels), n, int(sys.n_mol), _ptr(x), _ptr(v), _ptr(_f64(sys.q)),
                            _ptr(_f64(sys.mass)), _ptr(lj), _ptr(_f64(sys.box)), float(dt), int(n_steps), _ptr(uk)))
    return x, v, uk


def project_rigid(x, v, mass, n_mol, d_oh=0.09572, d_hh=None):
    """Project distorted rigid triples of (x, v) back onto the constraints (copies;
    molecules within the threshold are returned unchanged).  Returns (x, v)."""
    import math
    if d_hh is None:
        d_hh = 2.0 * d_oh * math.sin(math.radians(104.52) / 2.0)
    x = _f64(x).copy(); v = _f64(v).copy()
    _check(lib().orc_project_rigid(len(mass), int(n_mol), _ptr(_f64(mass)), float(d_oh), float(d_hh), _ptr(x), _ptr(v)))
    return x, v


def _pack(p, ke):
    mdp = model_params(p["a"], p["h"], ke, wall_k=p.get("wall_k", 0.0), wall_width=p.get("wall_width", 0.0),
                       method=p.get("method", "msm"), wolf_alpha=p.get("wolf_alpha", 0.0), mts=p.get("mts", 0))
    return _f64(list(mdp) + [p["dt"], p["steps"], p["levels"]])


def parareal_window(sys, G: dict, F: dict, n_slices, window, max_iter, tol, ke=KE):
    """Parareal over a sliding window of at most `window` slices (Sec. 4).
    Returns (xs, vs, iters, last_dx, status)."""
    n = sys.n
    xs = np.zeros((n_slices + 1, n, 3)); vs = np.zeros((n_slices + 1, n, 3))
    xs[0] = sys.pos; vs[0] = sys.vel
    it = C.c_int(0); dx = C.c_double(0)
    lj = np.ascontiguousarray(sys.lj, dtype=np.uint8)
    rc = lib().orc_parareal_window(_ptr(_pack(G, ke)), _ptr(_pack(F, ke)), n, int(sys.n_mol), _ptr(_f64(sys.q)),
                                   _ptr(_f64(sys.mass)), _ptr(lj), _ptr(_f64(sys.box)), int(n_slices), int(window),
                                   int(max_iter), float(tol), _ptr(xs), _ptr(vs), C.byref(it), C.byref(dx))
    if rc not in (0, -6):
        _check(rc)
    return xs, vs, it.value, dx.value, rc


def parareal(sys, G: dict, F: dict, n_slices, max_iter, tol, ke=KE):
    """G, F: dict(a, h, levels, dt, steps[, method, wolf_alpha, wall_k, wall_width]).
    Returns (xs, vs, iters, last_dx, status)."""
    n = sys.n

    def pack(p):
        return _pack(p, ke)

    xs = np.zeros((n_slices + 1, n, 3)); vs = np.zeros((n_slices + 1, n, 3))
    xs[0] = sys.pos; vs[0] = sys.vel
    it = C.c_int(0); dx = C.c_double(0)
    lj = np.ascontiguousarray(sys.lj, dtype=np.uint8)
    rc = lib().orc_parareal(_ptr(pack(G)), _ptr(pack(F)), n, int(sys.n_mol), _ptr(_f64(sys.q)),
                            _ptr(_f64(sys.mass)), _ptr(lj), _ptr(_f64(sys.box)), int(n_slices), int(max_iter),
                            float(tol), _ptr(xs), _ptr(vs), C.byref(it), C.byref(dx))
    if rc not in (0, -6):
        _check(rc)
    return xs, vs, it.value, dx.value, rc
