"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/msm.h declares; argument validation that
happens before any CUDA call works without a GPU.  No kernel is launched."""
import ctypes as C
import re
import shutil
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not Path("/usr/local/cuda/bin/nvcc").exists(),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def L():
    from paper_1309_1889_gb300 import api, build
    build.build()
    return api.lib()


def declared():
    text = (ROOT / "include" / "msm.h").read_text()
    return [n for n in re.findall(r"^MSM_API\s+[\w\s\*]*?\**\s*(\w+)\s*\(", text, re.M)]


def test_header_declares_the_boundary():
    names = set(declared())
    for want in ("msm_create", "msm_destroy", "msm_energy_forces", "md_run", "parareal_run",
                 "msm_energy_forces_batched", "msm_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(L):
    from paper_1309_1889_gb300 import api
    names = declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(api.EXPORTS)


def test_default_params_and_validation_without_gpu(L):
    from paper_1309_1889_gb300 import api
    p = api.Params()
    L.msm_default_params(C.byref(p))
    assert p.a == 1.2 and p.h == 0.25 and p.n_levels == 3 and p.precision == api.FP32
    assert abs(p.coulomb_k - 138.935458) < 1e-12
    h = C.c_void_p()
    bad = api.make_params(a=-1.0)
    assert L.msm_create(C.byref(bad), C.byref(h)) == -1
    assert b"positive" in L.msm_last_error()
    bad = api.make_params(levels=0)
    assert L.msm_create(C.byref(bad), C.byref(h)) == -1
    bad = api.make_params(a=5.0, h=0.25)          # 2a/h = 40: lattice-cutoff radius too large
    assert L.msm_create(C.byref(bad), C.byref(h)) == -1
    bad = api.make_params()
    bad.flags = 32                                # no such flag
    assert L.msm_create(C.byref(bad), C.byref(h)) == -1
    assert b"unknown flags" in L.msm_last_error()


def test_flag_values_match_the_header():
    from paper_1309_1889_gb300 import api
    hdr = (ROOT / "include" / "msm.h").read_text()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define MSM_FLAG_(\w+)\s+(\d+)", hdr)}
    assert defs == {"GRAPHS": api.FLAG_GRAPHS, "AUTOTUNE": api.FLAG_AUTOTUNE, "SCALAR_PAIRS": api.FLAG_SCALAR_PAIRS,
                    "CLUSTER_PAIRS": api.FLAG_CLUSTER_PAIRS, "BRICKS": api.FLAG_BRICKS}
    assert api.make_params().flags == api.FLAG_GRAPHS | api.FLAG_AUTOTUNE
    assert api.make_params(scalar_pairs=True, graphs=False, autotune=False).flags == api.FLAG_SCALAR_PAIRS


def test_library_is_built_for_sm_103a():
    from paper_1309_1889_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_method_values_and_validation(L):
    from paper_1309_1889_gb300 import api
    hdr = (ROOT / "include" / "msm.h").read_text()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define MSM_METHOD_(\w+)\s+(\d+)", hdr)}
    assert defs == {"MSM": 0, "CUTOFF": 1, "WOLF": 2}
    assert {k.upper(): v for k, v in api.METHODS.items()} == defs
    p = api.Params()
    L.msm_default_params(C.byref(p))
    assert p.method == 0 and p.wolf_alpha == 0.0
    h = C.c_void_p()
    bad = api.make_params(method=3)
    assert L.msm_create(C.byref(bad), C.byref(h)) == -1 and b"unknown method" in L.msm_last_error()
    bad = api.make_params(method="wolf", wolf_alpha=-1.0)
    assert L.msm_create(C.byref(bad), C.byref(h)) == -1 and b"wolf_alpha" in L.msm_last_error()
    bad = api.make_params(method="wolf", wolf_alpha=2.0, list_skin=0.1)
    assert L.msm_create(C.byref(bad), C.byref(h)) == -1 and b"Verlet lists" in L.msm_last_error()


def test_multiple_time_stepping_validation(L):
    """mts_steps defaults to 0 (plain velocity Verlet), must be >= 0, and above 1
    needs the MSM: the cutoff methods have no grid part to put on the slow clock."""
    from paper_1309_1889_gb300 import api
    p = api.Params()
    L.msm_default_params(C.byref(p))
    assert p.mts_steps == 0
    h = C.c_void_p()
    bad = api.make_params(mts=-1)
    assert L.msm_create(C.byref(bad), C.byref(h)) == -1 and b"mts_steps" in L.msm_last_error()
    bad = api.make_params(mts=2, method="cutoff")
    assert L.msm_create(C.byref(bad), C.byref(h)) == -1 and b"multiple time stepping" in L.msm_last_error()


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof and field offsets of msm_params and msm_system as a C compiler lays them
    out from include/msm.h, against the ctypes structures of the binding."""
    from paper_1309_1889_gb300 import api
    src = tmp_path / "layout.c"
    fields_p = [f[0] for f in api.Params._fields_]
    fields_s = [f[0] for f in api.SystemC._fields_]
    body = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{ROOT / "include" / "msm.h"}"', 'int main(void){',
            'printf("%zu\\n", sizeof(msm_params));']
    body += [f'printf("%zu\\n", offsetof(msm_params, {f}));' for f in fields_p]
    body += ['printf("%zu\\n", sizeof(msm_system));']
    body += [f'printf("%zu\\n", offsetof(msm_system, {f}));' for f in fields_s]
    body += ['return 0;}']
    src.write_text("\n".join(body))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = [C.sizeof(api.Params)] + [getattr(api.Params, f).offset for f in fields_p]
    want += [C.sizeof(api.SystemC)] + [getattr(api.SystemC, f).offset for f in fields_s]
    assert got == want


def test_device_budget_round_trip(L):
    """The budget call needs no GPU: it sets or clears the cap and reports the bytes held."""
    assert L.msm_set_device_budget(1 << 20) == 0
    assert L.msm_set_device_budget(0) == 0
