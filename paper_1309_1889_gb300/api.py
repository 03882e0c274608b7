"""Thin ctypes binding of libmsm_gb300.so (C ABI in include/msm.h).

Argument marshalling only: every step of the multilevel summation method,
of velocity Verlet and of parareal runs in the library's CUDA kernels.  Torch
tensors (CUDA, float64, contiguous) are passed as device pointers with the
current torch stream; numpy arrays are passed as host pointers and the
library stages them itself.  There is no CPU fallback: if the library is
missing, every call raises.
"""
from __future__ import annotations

import ctypes as C
import math
from pathlib import Path

import numpy as np

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "libmsm_gb300.so"

KE = 138.935458
FP64, FP32 = 0, 1
MODEL_CHARGES, MODEL_WATER = 0, 1
FLAG_GRAPHS, FLAG_AUTOTUNE, FLAG_SCALAR_PAIRS, FLAG_CLUSTER_PAIRS, FLAG_BRICKS = 1, 2, 4, 8, 16
METHODS = {"msm": 0, "cutoff": 1, "wolf": 2}
CODES = {-1: "EINVAL", -2: "ERANGE", -3: "ENOMEM", -4: "ECUDA", -5: "ETIMEOUT", -6: "ENOCONV"}


class MSMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{CODES.get(code, code)}: {msg}")
        self.code = code
        self.name = CODES.get(code, str(code))


class Params(C.Structure):
    _fields_ = [("a", C.c_double), ("h", C.c_double), ("n_levels", C.c_int32), ("precision", C.c_int32),
                ("coulomb_k", C.c_double), ("gamma_kind", C.c_int32), ("basis_kind", C.c_int32),
                ("model", C.c_int32), ("flags", C.c_int32), ("lj_sigma", C.c_double),
                ("lj_epsilon", C.c_double), ("d_oh", C.c_double), ("d_hh", C.c_double),
                ("wall_k", C.c_double), ("wall_width", C.c_double), ("list_skin", C.c_double),
                ("method", C.c_int32), ("mts_steps", C.c_int32), ("wolf_alpha", C.c_double)]


class SystemC(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_mol", C.c_int64), ("x", C.c_void_p), ("v", C.c_void_p),
                ("q", C.c_void_p), ("m", C.c_void_p), ("lj", C.c_void_p), ("box", C.c_double * 6),
                ("f", C.c_void_p), ("f_valid", C.c_int32), ("reserved0", C.c_int32), ("energy", C.c_double)]


_lib = None
EXPORTS = ("msm_default_params", "msm_create", "msm_destroy", "msm_energy_forces", "msm_energy_forces_batched",
           "msm_system_forces", "md_run", "parareal_run", "msm_grid_shape", "msm_stage_grid", "msm_cell_list",
           "msm_stage_atoms", "msm_kernel_launches", "msm_last_error", "msm_profile_enable", "msm_profile_read",
           "msm_stage_name", "msm_count_pairs", "msm_cell_list_noalloc", "msm_list_stats",
           "msm_system_forces_batched", "md_run_batched", "msm_diag_convert", "parareal_run_window",
           "parareal_resume", "msm_set_device_budget")


def lib():
    """Load libmsm_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH.name} is not built: run __graft_entry__.build() "
                               "(or python -m paper_1309_1889_gb300.build)")
        L = C.CDLL(str(LIB_PATH))
        P, p, i32, i64, d = C.POINTER, C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.msm_default_params.argtypes = [P(Params)]; L.msm_default_params.restype = None
        L.msm_create.argtypes = [P(Params), P(p)]; L.msm_create.restype = C.c_int
        L.msm_destroy.argtypes = [p]; L.msm_destroy.restype = None
        L.msm_energy_forces.argtypes = [p, i64, p, p, P(d), p, p, p, p, p]; L.msm_energy_forces.restype = C.c_int
        L.msm_energy_forces_batched.argtypes = [p, i32, p, p, p, p, p, p, p, p]
        L.msm_energy_forces_batched.restype = C.c_int
        L.msm_system_forces.argtypes = [p, P(SystemC), p, p, p, p]; L.msm_system_forces.restype = C.c_int
        L.md_run.argtypes = [p, P(SystemC), d, i32, p, p]; L.md_run.restype = C.c_int
        L.msm_system_forces_batched.argtypes = [p, i32, P(SystemC), p, p]
        L.msm_system_forces_batched.restype = C.c_int
        L.md_run_batched.argtypes = [p, i32, P(SystemC), d, i32, p, p]; L.md_run_batched.restype = C.c_int
        L.parareal_run.argtypes = [P(Params), d, i32, P(Params), d, i32, P(SystemC), i32, i32, d, p, p,
                                   P(i32), P(d), p]
        L.parareal_run.restype = C.c_int
        L.parareal_run_window.argtypes = [P(Params), d, i32, P(Params), d, i32, P(SystemC), i32, i32, i32, d, p, p,
                                          P(i32), P(d), p]
        L.parareal_run_window.restype = C.c_int
        L.parareal_resume.argtypes = [P(Params), d, i32, P(Params), d, i32, P(SystemC), i32, i32, i32, d, p, p,
                                      P(i32), P(d), p]
        L.parareal_resume.restype = C.c_int
        L.msm_set_device_budget.argtypes = [i64]; L.msm_set_device_budget.restype = i64
        L.msm_grid_shape.argtypes = [p, i32, p, p]; L.msm_grid_shape.restype = C.c_int
        L.msm_stage_grid.argtypes = [p, i32, i32, p, i64]; L.msm_stage_grid.restype = C.c_int
        L.msm_cell_list.argtypes = [p, p, p, p]; L.msm_cell_list.restype = C.c_int
        L.msm_stage_atoms.argtypes = [p, i32, p, i64]; L.msm_stage_atoms.restype = C.c_int
        L.msm_kernel_launches.argtypes = []; L.msm_kernel_launches.restype = C.c_int64
        L.msm_profile_enable.argtypes = [p, i32]; L.msm_profile_enable.restype = C.c_int
        L.msm_profile_read.argtypes = [p, p, p, i32, i32]; L.msm_profile_read.restype = C.c_int
        L.msm_stage_name.argtypes = [i32]; L.msm_stage_name.restype = C.c_char_p
        L.msm_count_pairs.argtypes = [p, P(i64)]; L.msm_count_pairs.restype = C.c_int
        L.msm_list_stats.argtypes = [p, p, i32]; L.msm_list_stats.restype = C.c_int
        L.msm_cell_list_noalloc.argtypes = [i64, p, P(d), d, p, p, i64, p]
        L.msm_cell_list_noalloc.restype = C.c_int
        L.msm_diag_convert.argtypes = [i64, p, p, p, p, p]; L.msm_diag_convert.restype = C.c_int
        L.msm_last_error.argtypes = []; L.msm_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise MSMError(rc, lib().msm_last_error().decode())


def kernel_launches() -> int:
    return int(lib().msm_kernel_launches())


def diag_convert(x, y):
    """The library's integer-pipe conversions on CUDA tensors: (binary32 of the
    float64 tensor x, binary64 of the float32 tensor y)."""
    t = _torch()
    if x.dtype != t.float64 or y.dtype != t.float32 or not x.is_cuda or not y.is_cuda or x.numel() != y.numel():
        raise ValueError("x: float64 CUDA tensor, y: float32 CUDA tensor of the same size")
    x = x.contiguous(); y = y.contiguous()
    x32 = t.empty_like(x, dtype=t.float32); y64 = t.empty_like(y, dtype=t.float64)
    _check(lib().msm_diag_convert(x.numel(), x.data_ptr(), x32.data_ptr(), y.data_ptr(), y64.data_ptr(),
                                  t.cuda.current_stream().cuda_stream))
    return x32, y64


# --------------------------------------------------------------- marshalling

def _torch():
    import torch
    return torch


def _is_tensor(x) -> bool:
    try:
        import torch
        return isinstance(x, torch.Tensor)
    except ImportError:  # pragma: no cover
        return False


def _ptr(x):
    """Device pointer of a CUDA tensor or host pointer of a numpy array."""
    if x is None:
        return None
    if _is_tensor(x):
        if x.is_cuda:
            if not x.is_contiguous():
                raise ValueError("tensors must be contiguous")
            return C.c_void_p(x.data_ptr())
        x = x.numpy()
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("arrays must be C-contiguous")
    return x.ctypes.data_as(C.c_void_p)


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover
        pass
    return None


def _box(box):
    b = np.asarray(box, dtype=np.float64).reshape(6)
    return (C.c_double * 6)(*b.tolist())


def make_params(a=1.2, h=0.25, levels=3, precision="fp32", model="charges", ke=KE, lj_sigma=0.315061,
                lj_epsilon=0.6364, d_oh=0.09572, d_hh=None, wall_k=0.0, wall_width=0.0,
                list_skin=0.0, graphs=True, autotune=True, scalar_pairs=False, method="msm",
                wolf_alpha=0.0, mts=0, cluster_pairs=False, bricks=False) -> Params:
    """mts: multiple time stepping of md_run (the grid part every `mts` steps; 0 or 1: off).
    cluster_pairs: the FP32 short-range Coulomb pass on cluster pairs.
    bricks: the pair passes on bricks of cells instead of 32-atom groups (diagnostic: same bits)."""
    p = Params()
    p.a, p.h, p.n_levels = float(a), float(h), int(levels)
    p.precision = {"fp64": FP64, "fp32": FP32, FP64: FP64, FP32: FP32}[precision]
    p.coulomb_k = float(ke)
    p.gamma_kind = p.basis_kind = 0
    p.model = {"charges": MODEL_CHARGES, "water": MODEL_WATER, 0: 0, 1: 1}[model]
    p.lj_sigma, p.lj_epsilon = float(lj_sigma), float(lj_epsilon)
    p.d_oh = float(d_oh)
    p.d_hh = float(d_hh) if d_hh is not None else 2.0 * d_oh * math.sin(math.radians(104.52) / 2.0)
    p.wall_k, p.wall_width = float(wall_k), float(wall_width)
    p.list_skin = float(list_skin)
    p.flags = ((FLAG_GRAPHS if graphs else 0) | (FLAG_AUTOTUNE if autotune else 0)
               | (FLAG_SCALAR_PAIRS if scalar_pairs else 0) | (FLAG_CLUSTER_PAIRS if cluster_pairs else 0)
               | (FLAG_BRICKS if bricks else 0))
    p.method = METHODS[method] if isinstance(method, str) else int(method)
    p.wolf_alpha = float(wolf_alpha)
    p.mts_steps = int(mts)
    return p


class MSM:
    """A handle: method parameters plus the device scratch of one evaluation stream."""

    def __init__(self, a=1.2, h=0.25, levels=3, precision="fp32", model="charges", **kw):
        self.params = make_params(a, h, levels, precision, model, **kw)
        self._h = C.c_void_p()
        _check(lib().msm_create(C.byref(self.params), C.byref(self._h)))

    def close(self):
        if self._h:
            lib().msm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- evaluation -----------------------------------------------------------
    def energy_forces(self, pos, q, box, *, forces=True, potentials=True, virial=False, stream=None):
        """U, F (n, 3), phi (n,), [virial] for point charges.

        CUDA tensors in -> CUDA tensors out (no host synchronisation beyond the
        library's status check); numpy in -> numpy out.
        """
        n = int(pos.shape[0])
        dev = _is_tensor(pos) and pos.is_cuda
        if dev:
            torch = _torch()
            out_f = torch.empty((n, 3), dtype=torch.float64, device=pos.device) if forces else None
            out_p = torch.empty((n,), dtype=torch.float64, device=pos.device) if potentials else None
            e = torch.empty(2, dtype=torch.float64, device=pos.device)
            _check(lib().msm_energy_forces(self._h, n, _ptr(pos), _ptr(q), _box(box), _ptr(e), _ptr(out_f),
                                           _ptr(out_p), C.c_void_p(e.data_ptr() + 8) if virial else None,
                                           _stream(stream)))
            res = (e[0], out_f, out_p)
            return res + (e[1],) if virial else res
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.float64)
        out_f = np.empty((n, 3)) if forces else None
        out_p = np.empty(n) if potentials else None
        e = np.zeros(2)
        _check(lib().msm_energy_forces(self._h, n, _ptr(pos), _ptr(q), _box(box), _ptr(e[0:1]), _ptr(out_f),
                                       _ptr(out_p), e[1:2].ctypes.data_as(C.c_void_p) if virial else None,
                                       _stream(stream)))
        res = (float(e[0]), out_f, out_p)
        return res + (float(e[1]),) if virial else res

    def energy_forces_batched(self, offsets, pos, q, boxes, stream=None):
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        boxes = np.ascontiguousarray(boxes, dtype=np.float64)
        n_sys = len(offsets) - 1
        n = int(offsets[-1])
        dev = _is_tensor(pos) and pos.is_cuda
        if dev:
            torch = _torch()
            e = torch.empty(n_sys, dtype=torch.float64, device=pos.device)
            f = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
            p = torch.empty(n, dtype=torch.float64, device=pos.device)
        else:
            pos = np.ascontiguousarray(pos, dtype=np.float64); q = np.ascontiguousarray(q, dtype=np.float64)
            e = np.empty(n_sys); f = np.empty((n, 3)); p = np.empty(n)
        _check(lib().msm_energy_forces_batched(self._h, n_sys, _ptr(offsets), _ptr(pos), _ptr(q), _ptr(boxes),
                                               _ptr(e), _ptr(f), _ptr(p), _stream(stream)))
        return e, f, p

    def system_forces(self, sys, stream=None):
        """U, F, phi of a System-like object (water model if the handle has it)."""
        s, keep = _system_struct(sys)
        n = int(s.n)
        dev = _is_tensor(sys.pos) and sys.pos.is_cuda
        if dev:
            torch = _torch()
            e = torch.empty(1, dtype=torch.float64, device=sys.pos.device)
            f = torch.empty((n, 3), dtype=torch.float64, device=sys.pos.device)
            p = torch.empty(n, dtype=torch.float64, device=sys.pos.device)
            _check(lib().msm_system_forces(self._h, C.byref(s), _ptr(e), _ptr(f), _ptr(p), _stream(stream)))
            return e[0], f, p
        e = np.zeros(1); f = np.empty((n, 3)); p = np.empty(n)
        _check(lib().msm_system_forces(self._h, C.byref(s), _ptr(e), _ptr(f), _ptr(p), _stream(stream)))
        return float(e[0]), f, p

    def md_run(self, sys, dt, n_steps, record=True, stream=None):
        """Advance sys.pos / sys.vel in place; returns (U, K) per step (n_steps+1, 2) or None."""
        s, keep = _system_struct(sys, need_v=True)
        dev = _is_tensor(sys.pos) and sys.pos.is_cuda
        uk = None
        if record:
            if dev:
                uk = _torch().empty((n_steps + 1, 2), dtype=_torch().float64, device=sys.pos.device)
            else:
                uk = np.zeros((n_steps + 1, 2))
        _check(lib().md_run(self._h, C.byref(s), float(dt), int(n_steps), _ptr(uk), _stream(stream)))
        if s.f:
            sys.force_valid = int(s.f_valid)
            sys.energy = float(s.energy)
        return uk

    def system_forces_batched(self, systems, stream=None):
        """Energies (list) and forces of independent System-like objects in one batched
        evaluation; each system needs a `force` array/tensor (n, 3) to receive F."""
        arr = (SystemC * len(systems))()
        keep = []
        for b, sy in enumerate(systems):
            s, k = _system_struct(sy)
            arr[b] = s
            keep.append((s, k))
        e = np.zeros(len(systems))
        _check(lib().msm_system_forces_batched(self._h, len(systems), arr, _ptr(e), _stream(stream)))
        for b, sy in enumerate(systems):
            if arr[b].f:
                sy.force_valid = int(arr[b].f_valid)
                sy.energy = float(arr[b].energy)
        return e

    def md_run_batched(self, systems, dt, n_steps, record=True, stream=None):
        """md_run for independent systems stepped together (one launch per stage for all).

        Advances every system's pos / vel in place; returns (U, K) per system and
        step, shape (n_sys, n_steps+1, 2), or None."""
        arr = (SystemC * len(systems))()
        keep = []
        for b, sy in enumerate(systems):
            s, k = _system_struct(sy, need_v=True)
            arr[b] = s
            keep.append((s, k))
        dev = _is_tensor(systems[0].pos) and systems[0].pos.is_cuda
        uk = None
        if record:
            if dev:
                uk = _torch().empty((len(systems), n_steps + 1, 2), dtype=_torch().float64,
                                    device=systems[0].pos.device)
            else:
                uk = np.zeros((len(systems), n_steps + 1, 2))
        _check(lib().md_run_batched(self._h, len(systems), arr, float(dt), int(n_steps), _ptr(uk), _stream(stream)))
        for b, sy in enumerate(systems):
            if arr[b].f:
                sy.force_valid = int(arr[b].f_valid)
                sy.energy = float(arr[b].energy)
        return uk

    # -- profiling ------------------------------------------------------------
    def profile(self, on=True):
        _check(lib().msm_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, reset=True):
        """{stage name: (total ms, launches)} accumulated while profiling was on."""
        ms = np.zeros(32); cnt = np.zeros(32, dtype=np.int64)
        k = lib().msm_profile_read(self._h, _ptr(ms), _ptr(cnt), 32, 1 if reset else 0)
        return {lib().msm_stage_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(k)}

    def list_stats(self) -> dict:
        v = np.zeros(8, dtype=np.int64)
        _check(lib().msm_list_stats(self._h, _ptr(v), 8))
        keys = ("builds", "overflows", "cap_entries", "cap_lj_entries", "row_slots", "max_entries_seen",
                "max_lj_entries_seen", "max_rows_seen")
        return {k: int(x) for k, x in zip(keys, v)}

    def count_pairs(self) -> int:
        """Ordered pairs (i, j != i) with r_ij < a in the last evaluation."""
        out = C.c_int64(0)
        _check(lib().msm_count_pairs(self._h, C.byref(out)))
        return int(out.value)

    # -- inspection -----------------------------------------------------------
    def grid_shape(self, level):
        shp = np.zeros(3, dtype=np.int64); lo = np.zeros(3, dtype=np.int64)
        _check(lib().msm_grid_shape(self._h, int(level), _ptr(shp), _ptr(lo)))
        return tuple(int(v) for v in shp), tuple(int(v) for v in lo)

    def stage_grid(self, level, which):
        """which: 'q' (charges), 'ucut' (lattice-cutoff potential), 'u' (potential); array (nz, ny, nx)."""
        w = {"q": 0, "ucut": 1, "u": 2}[which]
        shp, _ = self.grid_shape(level)
        out = np.empty(shp[::-1])
        _check(lib().msm_stage_grid(self._h, int(level), w, _ptr(out), out.size))
        return out

    def cell_list(self, n):
        nc = C.c_int64(0)
        _check(lib().msm_cell_list(self._h, None, None, C.byref(nc)))
        perm = np.empty(n, dtype=np.int64); start = np.empty(nc.value + 1, dtype=np.int64)
        _check(lib().msm_cell_list(self._h, _ptr(perm), _ptr(start), C.byref(nc)))
        return perm, start

    def stage_atoms(self, n):
        """Short-range potential sum_j q_j g*(r_ij) and force sum (before k_e), caller's atom order."""
        phi = np.empty(n); f = np.empty((n, 3))
        _check(lib().msm_stage_atoms(self._h, 0, _ptr(phi), n))
        _check(lib().msm_stage_atoms(self._h, 1, _ptr(f), 3 * n))
        return phi, f


def _system_struct(sys, need_v=False):
    """Build an msm_system from an object with pos, vel, q, mass, lj, n_mol, box."""
    s = SystemC()
    s.n = int(sys.pos.shape[0])
    s.n_mol = int(getattr(sys, "n_mol", 0))
    keep = []

    def arr(x, dtype):
        if x is None:
            return None
        if _is_tensor(x):
            return x
        a = np.ascontiguousarray(x, dtype=dtype)
        keep.append(a)
        return a

    pos = sys.pos
    if not (_is_tensor(pos) or (isinstance(pos, np.ndarray) and pos.dtype == np.float64 and pos.flags["C_CONTIGUOUS"])):
        raise ValueError("sys.pos must be a float64 C-contiguous array or a CUDA tensor (updated in place)")
    s.x = _ptr(pos)
    vel = getattr(sys, "vel", None)
    if need_v and vel is None:
        raise ValueError("velocities required")
    s.v = _ptr(vel) if vel is not None else None
    s.q = _ptr(arr(sys.q, np.float64))
    m = getattr(sys, "mass", None)
    s.m = _ptr(arr(m, np.float64)) if m is not None else None
    lj = getattr(sys, "lj", None)
    s.lj = _ptr(arr(lj, np.uint8)) if lj is not None else None
    b = np.asarray(sys.box, dtype=np.float64).reshape(6)
    for d in range(6):
        s.box[d] = float(b[d])
    f = getattr(sys, "force", None)          # optional (n, 3) float64: forces carried between md_run calls
    if f is not None:
        if not (_is_tensor(f) or (isinstance(f, np.ndarray) and f.dtype == np.float64 and f.flags["C_CONTIGUOUS"])):
            raise ValueError("sys.force must be a float64 C-contiguous array or a CUDA tensor")
        s.f = _ptr(f)
        s.f_valid = int(getattr(sys, "force_valid", 0))
        s.energy = float(getattr(sys, "energy", 0.0))
    s._keep = keep
    return s, keep


def parareal_run(G: dict, F: dict, sys, n_slices: int, max_iter: int, tol: float, model="water",
                 precision="fp32", stream=None, window=None, resume=None):
    """Parareal over md_run: G and F are dict(a, h, levels, dt, steps[, method, wolf_alpha,
    wall_k, wall_width, ...]); method "cutoff" or "wolf" makes a cutoff coarse propagator.

    window: None runs parareal_run (every slice iterated); an integer runs
    parareal_run_window with at most that many slices per iteration.
    resume: (xs, vs, k) -- continue, through parareal_resume, from the iterate that
    an earlier call returned after k iterations (at most max_iter more).

    Returns (xs (n_slices+1, n, 3), vs, iterations, last max |dx|, converged)."""
    def params(P):
        return make_params(P["a"], P["h"], P.get("levels", 1), P.get("precision", precision), model,
                           wall_k=P.get("wall_k", 0.0), wall_width=P.get("wall_width", 0.0),
                           list_skin=P.get("list_skin", 0.0), graphs=P.get("graphs", True),
                           autotune=P.get("autotune", True), method=P.get("method", "msm"),
                           wolf_alpha=P.get("wolf_alpha", 0.0), mts=P.get("mts", 0))
    pg, pf = params(G), params(F)
    s, keep = _system_struct(sys, need_v=True)
    n = int(s.n)
    xs = np.zeros((n_slices + 1, n, 3)); vs = np.zeros((n_slices + 1, n, 3))
    it = C.c_int32(0); dx = C.c_double(0)
    xs[0] = np.asarray(sys.pos.cpu() if _is_tensor(sys.pos) else sys.pos)
    vs[0] = np.asarray(sys.vel.cpu() if _is_tensor(sys.vel) else sys.vel)
    if resume is not None:
        rx, rv, rk = resume
        xs[:] = np.asarray(rx); vs[:] = np.asarray(rv)
        rc = lib().parareal_resume(C.byref(pg), float(G["dt"]), int(G["steps"]), C.byref(pf), float(F["dt"]),
                                   int(F["steps"]), C.byref(s), int(n_slices), int(rk), int(max_iter), float(tol),
                                   _ptr(xs), _ptr(vs), C.byref(it), C.byref(dx), _stream(stream))
    elif window is None:
        rc = lib().parareal_run(C.byref(pg), float(G["dt"]), int(G["steps"]), C.byref(pf), float(F["dt"]),
                                int(F["steps"]), C.byref(s), int(n_slices), int(max_iter), float(tol), _ptr(xs),
                                _ptr(vs), C.byref(it), C.byref(dx), _stream(stream))
    else:
        rc = lib().parareal_run_window(C.byref(pg), float(G["dt"]), int(G["steps"]), C.byref(pf), float(F["dt"]),
                                       int(F["steps"]), C.byref(s), int(n_slices), int(window), int(max_iter),
                                       float(tol), _ptr(xs), _ptr(vs), C.byref(it), C.byref(dx), _stream(stream))
    if rc != 0 and not (rc == -6 and lib().msm_last_error().decode().startswith("parareal:")):
        _check(rc)                     # a propagator failed (not merely a slow convergence)
    return xs, vs, it.value, dx.value, rc == 0


def set_device_budget(nbytes: int) -> int:
    """Cap the device memory the library allocates (0: no cap); returns the bytes it holds."""
    return int(lib().msm_set_device_budget(int(nbytes)))


# ----------------------------------------------------------------- autograd

def msm_energy(pos, q, box, msm: MSM):
    """U(pos, q) as a differentiable torch scalar; backward gives dU/dpos = -F and dU/dq = phi.
    The forward asks the library only for what the backward will need: forces if pos
    requires a gradient, potentials if q does."""
    return _MSMEnergy.apply(pos, q, box, msm)


def msm_energy_batched(offsets, pos, q, boxes, msm: MSM):
    """Energies of independent systems of uneven sizes from one batched evaluation
    (systems b = offsets[b] .. offsets[b+1] of pos (N, 3) and q (N,), box b = boxes[b]),
    as a differentiable torch tensor (B,); backward gives each system's dU_b/dpos = -F
    and dU_b/dq = phi, scaled by that system's incoming gradient."""
    return _MSMEnergyBatched.apply(pos, q, offsets, boxes, msm)


def _make_function():
    torch = _torch()

    class MSMEnergyFn(torch.autograd.Function):
        """Forward: one MSM evaluation (energy, with forces and potentials from the same pass).

        Backward: the analytic gradient of the quadratic form U = 1/2 q^T K(r) q.
        dU/dq_i = phi_i (K symmetric: every interpolation operator I^k is
        symmetric in its two arguments, Sec. 3), dU/dr_i = -F_i, where F_i
        was formed by the transposed chain interpolation^T (= anterpolation
        weights' gradients) applied to the prolonged grid potential.
        """

        @staticmethod
        def forward(ctx, pos, q, box, msm):
            need_f, need_p = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
            e, f, p = msm.energy_forces(pos.detach().contiguous(), q.detach().contiguous(), box,
                                        forces=need_f, potentials=need_p)
            ctx.save_for_backward(f if need_f else None, p if need_p else None)
            return e.reshape(())

        @staticmethod
        def backward(ctx, g):
            f, p = ctx.saved_tensors
            return (-g * f if f is not None else None), (g * p if p is not None else None), None, None

    return MSMEnergyFn


def _make_batched_function():
    torch = _torch()

    class MSMEnergyBatchedFn(torch.autograd.Function):
        """Forward: one batched evaluation of B independent systems (energies (B,)).
        Backward: system b's atoms get -g_b F_i (pos) and g_b phi_i (q)."""

        @staticmethod
        def forward(ctx, pos, q, offsets, boxes, msm):
            off = np.ascontiguousarray(offsets, dtype=np.int64)
            e, f, p = msm.energy_forces_batched(off, pos.detach().contiguous(), q.detach().contiguous(), boxes)
            counts = torch.as_tensor(np.diff(off), device=pos.device)
            ctx.save_for_backward(f, p, counts)
            return e

        @staticmethod
        def backward(ctx, g):
            f, p, counts = ctx.saved_tensors
            ga = torch.repeat_interleave(g, counts)               # each atom: its system's gradient
            return -ga[:, None] * f, ga * p, None, None, None

    return MSMEnergyBatchedFn


class _Lazy:
    _fn = None

    def apply(self, *args):
        if _Lazy._fn is None:
            _Lazy._fn = _make_function()
        return _Lazy._fn.apply(*args)


_MSMEnergy = _Lazy()


class _LazyBatched:
    _fn = None

    def apply(self, *args):
        if _LazyBatched._fn is None:
            _LazyBatched._fn = _make_batched_function()
        return _LazyBatched._fn.apply(*args)


_MSMEnergyBatched = _LazyBatched()
