"""GPU test files that pytest does not collect yet (kernels written but not
yet run on a GPU) must still import and call only what exists, so that
renaming them into the suite is the only step left."""
import importlib.util
import inspect
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def test_pending_gpu_tests_import_and_use_existing_api():
    import paper_2003_04776_gb300 as pevc
    spec = importlib.util.spec_from_file_location("gpu_pending", os.path.join(HERE, "gpu_pending.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)                      # imports only; no GPU work at import time
    tests = [n for n, f in inspect.getmembers(mod, inspect.isfunction) if n.startswith("test_")]
    assert len(tests) >= 9
    src = inspect.getsource(mod)
    for name in ("solve_cplx", "solve_cplx_left", "backtransform_cplx"):
        assert hasattr(pevc.Plan, name) and f".{name}(" in src
    for name in ("pevc_solve_cplx", "pevc_watchdog_selftest", "ERR_NONFINITE", "ERR_INDEFINITE", "ERR_TIMEOUT"):
        assert hasattr(pevc, name)
    assert mod.pytestmark.name == "gpu"             # joins the GPU suite once renamed
