"""C-ABI checks that need no GPU: the library builds and loads, exports every
entry point declared in include/chad.h, agrees with the input generator on
the parameter layout, and rejects invalid arguments before touching CUDA."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2311_08927_gb300 import build as B
from paper_2311_08927_gb300 import chad as CH
from paper_2311_08927_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return CH.lib()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(chad_[a-z0-9_]+)\s*\(",
                            src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    decl = declared_functions()
    assert len(decl) >= 11
    for name in decl:
        assert hasattr(L, name), name
    assert set(CH.exported_symbols()) <= set(decl)


def test_param_layout(L):
    assert L.chad_abi_version() == 3
    assert CH.param_names() == I.PARAM_NAMES
    assert L.chad_param_name(-1) is None and L.chad_param_name(len(I.PARAM_NAMES)) is None


def _cfg(**over):
    keep = []

    def arr(x, dt=np.float64):
        a = np.ascontiguousarray(x, dtype=dt)
        keep.append(a)
        return a
    counts = arr([10], np.int64)
    cfg = CH.chad_config()
    cfg.n_digesters = 1
    cfg.n_particles = counts.ctypes.data_as(CH._i64p)
    cfg.V_liq = arr([3400.0]).ctypes.data_as(CH._dp)
    cfg.V_gas = arr([300.0]).ctypes.data_as(CH._dp)
    cfg.params = arr(I.default_params()).ctypes.data_as(CH._dp)
    cfg.atol = arr(np.full(29, 1e-9)).ctypes.data_as(CH._dp)
    cfg.rtol = 1e-6
    cfg.max_steps_per_interval = 100
    cfg.max_newton_iters = 50
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg, keep


@pytest.mark.parametrize("over,msg", [
    (dict(n_digesters=0), "n_digesters"),
    (dict(precision=7), "precision"),
    (dict(headspace=3), "headspace"),
    (dict(rtol=0.0), "rtol"),
    (dict(rtol=float("nan")), "rtol"),
    (dict(max_steps_per_interval=0), "max_steps"),
    (dict(max_newton_iters=0), "max_newton"),
    (dict(fixed_substeps=-1), "fixed_substeps"),
    (dict(learned=2), "learned"),
])
def test_create_rejects_invalid_config_without_gpu(L, over, msg):
    cfg, keep = _cfg(**over)
    ctx = C.c_void_p()
    code = L.chad_create(C.byref(cfg), C.byref(ctx))
    assert code == 1 and not ctx.value
    assert msg.split("_")[0] in L.chad_last_error(None).decode()


def test_create_rejects_null_and_bad_atol(L):
    ctx = C.c_void_p()
    assert L.chad_create(None, C.byref(ctx)) == 1
    cfg, keep = _cfg()
    assert L.chad_create(C.byref(cfg), None) == 1
    bad = np.full(29, 1e-9)
    bad[3] = -1.0
    cfg.atol = bad.ctypes.data_as(CH._dp)
    assert L.chad_create(C.byref(cfg), C.byref(ctx)) == 1
    assert "atol" in L.chad_last_error(None).decode()


def test_create_rejects_bad_parameters(L):
    p = I.default_params()
    p[I.PIDX["K_S_su"]] = 0.0
    cfg, keep = _cfg()
    cfg.params = p.ctypes.data_as(CH._dp)
    ctx = C.c_void_p()
    assert L.chad_create(C.byref(cfg), C.byref(ctx)) == 1
    assert "half-saturation" in L.chad_last_error(None).decode()
    p = I.default_params()
    p[I.PIDX["pH_UL_ac"]] = p[I.PIDX["pH_LL_ac"]]
    cfg.params = p.ctypes.data_as(CH._dp)
    assert L.chad_create(C.byref(cfg), C.byref(ctx)) == 1


def test_null_context_calls_are_invalid(L):
    assert L.chad_step(None, 60.0, 1) == 1
    assert L.chad_synchronize(None) == 1
    assert L.chad_load_particles(None, 0, 0, None, None, None, None, None, 0) == 1
    assert L.chad_read_states(None, 0, None, None, None, None, None, None, 0) == 1
    assert L.chad_set_diffusion(None, 0, 1e-6, 0.01) == 1
    assert L.chad_diffusion_info(None, None, None, None, None) == 1
    assert L.chad_diffusion_kernel_times(None, 1, None, None) == 1
    assert L.chad_set_positions(None, 0, 0, None, 0) == 1
    assert L.chad_set_positions_by_id(None, 0, 0, None, None, 0) == 1
    assert L.chad_get_interval(None, None) == 1
    assert L.chad_set_interval(None, 0) == 1
    assert L.chad_load_frame(None, 0, b"x", None, None) == 1
    assert L.chad_read_frame(None, 0, None, None, None, None, None, None) == 1
    L.chad_destroy(None)


def test_normal_build_has_no_bounds_checks(L):
    assert CH.chad_debug_bounds() == (0, 0)


def _cc():
    import shutil
    return shutil.which("gcc") or shutil.which("cc")


def build_c_caller(out_path):
    """Compile and link tests/c/run_digester.c (plain C99) against the library."""
    import subprocess
    pkg = os.path.dirname(B.LIB)
    cuda_lib = "/usr/local/cuda/lib64"
    cmd = [_cc(), "-std=c99", "-Wall", "-Wextra", "-Werror", "-O2",
           os.path.join(ROOT, "tests", "c", "run_digester.c"), "-I", os.path.join(ROOT, "include"),
           "-L", pkg, "-lchad", f"-Wl,-rpath,{pkg}", "-L", cuda_lib, f"-Wl,-rpath-link,{cuda_lib}",
           "-o", str(out_path)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return str(out_path)


def test_header_compiles_as_c_and_a_c_program_links(L, tmp_path):
    """include/chad.h is plain C: a C99 program using it compiles with every
    warning as an error and links against libchad.so (every call it uses
    resolves); running it needs a GPU (tests/test_gpu_parity.py)."""
    if _cc() is None:
        pytest.skip("no C compiler")
    assert os.path.exists(build_c_caller(tmp_path / "run_digester"))

