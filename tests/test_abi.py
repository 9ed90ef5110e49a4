"""The C-ABI library builds, loads and exports every entry point that
include/pevc.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pevc_[a-z_]+)\s*\(", text)))


def _builder():
    import importlib.util
    spec = importlib.util.spec_from_file_location("pevc_build", os.path.join(ROOT, "paper_2003_04776_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_library_builds_and_exports_declared_symbols():
    b = _builder()
    lib_path = b.build()
    names = _declared("pevc.h")
    assert {"pevc_plan", "pevc_solve", "pevc_solve_batched", "pevc_destroy", "pevc_strerror"} <= set(names)
    lib = ctypes.CDLL(lib_path)
    for nm in names:
        assert hasattr(lib, nm), nm
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pevc_\w+)", out))
    assert set(names) <= exported


def test_python_binding_mirrors_abi_names():
    import paper_2003_04776_gb300 as pevc
    for nm in _declared("pevc.h"):
        assert hasattr(pevc, nm), nm
    assert pevc.pevc_strerror(0) == "success"
    assert "invalid" in pevc.pevc_strerror(-3)


def test_library_targets_sm103a_only():
    b = _builder()
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_null_plan_and_bad_arguments_are_rejected_without_gpu():
    import paper_2003_04776_gb300 as pevc
    # argument checks run before any CUDA call
    st, m = pevc.pevc_solve(None, 0, 1, 0, 1, 0, 0, 0, 1, 0)
    assert st == -1
    assert pevc.pevc_destroy(None) == 0
    st, info = pevc.pevc_plan_info(None)
    assert st == -1


def test_backtransform_argument_checks_without_gpu():
    import paper_2003_04776_gb300 as pevc
    # a missing plan is rejected before any CUDA call
    assert pevc.pevc_backtransform(None, 0, 1, 1, 0, 1, 1, None, 0, 1) == -1
    assert pevc.BT_EMULATED == 4 and pevc.NO_NORMALISE == 1



def test_complex_solve_argument_checks_without_gpu():
    import paper_2003_04776_gb300 as pevc
    # a missing plan is rejected before any CUDA call
    assert pevc.pevc_solve_cplx(None, 0, 1, 0, 1, 0, 0, 0, 1, 0) == (-1, 0)
    assert pevc.pevc_solve_left(None, 0, 1, 0, 1, 0, 0, 0, 1, 0)[0] == -1


def test_watchdog_selftest_argument_checks_without_gpu():
    import paper_2003_04776_gb300 as pevc
    assert pevc.pevc_watchdog_selftest(None, 1, 1000) == -1
    assert pevc.ERR_TIMEOUT == 4
