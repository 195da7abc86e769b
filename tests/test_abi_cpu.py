"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every function include/rve.h declares, its structs have the
layout the header gives them, and calls without a device fail with a status
code instead of crashing."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rve.h")


@pytest.fixture(scope="module")
def pkg():
    from paper_2103_04770_gb300 import _build
    _build.build()
    import paper_2103_04770_gb300 as p
    p.lib()
    return p


def _declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rve_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(pkg):
    names = _declared_functions()
    assert len(names) >= 19
    lib = ctypes.CDLL(pkg._binding.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps every declared entry point under the same name
    assert set(names) <= set(pkg._binding._SIGNATURES)
    for n in names:
        assert callable(getattr(pkg, n))


def test_struct_layout_matches_header(pkg, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rve.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu\\n", sizeof(rve_phase_params), sizeof(rve_solver_options),'
                   ' sizeof(rve_step_info), offsetof(rve_step_info, sigma), offsetof(rve_phase_params, eps_C));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    b = pkg._binding
    assert int(out[0]) == ctypes.sizeof(b.PhaseParams)
    assert int(out[1]) == ctypes.sizeof(b.SolverOptions)
    assert int(out[2]) == ctypes.sizeof(b.StepInfo)
    assert int(out[3]) == b.StepInfo.sigma.offset
    assert int(out[4]) == b.PhaseParams.eps_C.offset


def test_host_only_calls(pkg):
    assert pkg.rve_status_string(pkg.RVE_ERR_NOT_CONVERGED) == "iteration budget exhausted"
    o = pkg.rve_default_options(pkg.RVE_MIXED)
    assert o.cg_rtol == 1e-3 and o.min_stag == 2
    o64 = pkg.rve_default_options(pkg.RVE_FP64)
    assert o64.cg_rtol == 1e-8


def test_argument_errors_without_device(pkg):
    lib = pkg.lib()
    # invalid arguments are rejected before any device work
    n = (ctypes.c_int * 3)(15, 16, 1)
    L = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    h = ctypes.c_void_p()
    assert lib.rve_create(ctypes.byref(h), 2, n, L, 0, 1, None) == pkg.RVE_ERR_ARG   # odd N1
    n = (ctypes.c_int * 3)(16, 14, 1)                                                # 14 = 2 * 7
    assert lib.rve_create(ctypes.byref(h), 2, n, L, 0, 1, None) == pkg.RVE_ERR_ARG
    assert lib.rve_create(ctypes.byref(h), 4, n, L, 0, 1, None) == pkg.RVE_ERR_ARG
    assert lib.rve_step_increment(None, None) == pkg.RVE_ERR_ARG
    assert lib.rve_step_increment_adaptive(None, 7, None) == pkg.RVE_ERR_ARG
    assert pkg.rve_status_string(pkg.RVE_ERR_TIMEOUT) == "device wait for a tile copy timed out"
    assert pkg.rve_status_string(pkg.RVE_ERR_LOAD_PATH_END) == "load path finished"
    # the binding's constants are the header's
    h_text = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                               "rve.h")).read()
    for name, val in re.findall(r"\b(RVE_(?:OK|ERR_\w+))\s*=\s*(-?\d+)", h_text):
        assert getattr(pkg, name) == int(val), name
    lib.rve_free(None)


@pytest.mark.skipif(os.environ.get("CUDA_VISIBLE_DEVICES", None) is None and
                    os.path.exists("/dev/nvidia0"), reason="a GPU is present")
def test_create_without_device_reports_status(pkg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pkg.RVEError) as ei:
        pkg.rve_create(2, (16, 16), (16.0, 16.0), pkg.RVE_FP64, 1)
    assert ei.value.status in (pkg.RVE_ERR_CUDA, pkg.RVE_ERR_OOM)


def test_batch_adjoint_and_field_calls_reject_bad_arguments(pkg):
    """The batch, autotuning, graph, stiffness-field and adjoint entry
    points validate their arguments before any device work."""
    lib = pkg.lib()
    b = ctypes.c_void_p()
    assert lib.rve_batch_create(ctypes.byref(b), 0, None, 0) == pkg.RVE_ERR_ARG
    assert lib.rve_batch_create(None, 1, None, 0) == pkg.RVE_ERR_ARG
    assert lib.rve_batch_step(None, None) == pkg.RVE_ERR_ARG
    assert lib.rve_batch_size(None) == 0
    lib.rve_batch_free(None)
    assert lib.rve_set_graphs(None, 1) == pkg.RVE_ERR_ARG
    assert lib.rve_set_gamma_tile(None, 1) == pkg.RVE_ERR_ARG
    assert lib.rve_get_gamma_tile(None, None) == pkg.RVE_ERR_ARG
    assert lib.rve_autotune(None, 1, None, None, None) == pkg.RVE_ERR_ARG
    assert lib.rve_set_stiffness_field(None, None) == pkg.RVE_ERR_ARG
    J = ctypes.c_double()
    assert lib.rve_adjoint_forward(None, 5, ctypes.byref(J)) == pkg.RVE_ERR_ARG
    assert lib.rve_adjoint_backward(None, 1.0, None, None, None, None) == pkg.RVE_ERR_ARG
