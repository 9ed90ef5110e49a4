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


def test_scheduler_autotune_and_flag_checks_without_gpu():
    import paper_2003_04776_gb300 as pevc
    assert pevc.pevc_scheduler_selftest(None, 1, 1000) == -1
    assert pevc.pevc_autotune_log(None)[0] == -1
    # flags are checked before any CUDA call: both walks at once, an unknown bit
    assert pevc.pevc_plan(100, 1, pevc.FP64, 0, pevc.STAGE_WALK | pevc.DEVICE_WALK)[0] == -6
    assert pevc.pevc_plan(100, 1, pevc.FP64, 0, 1 << 10)[0] == -6
    assert pevc.pevc_plan(100, 1, pevc.FP64, 48, 0)[0] == -5
    assert (pevc.STAGE_WALK, pevc.AUTOTUNE, pevc.DEVICE_WALK, pevc.BT_CUBLAS) == (8, 16, 32, 64)


def test_dag_host_task_lists_are_topological():
    """The scheduler's task list (built on the host by dag_stage_tasks, run
    here through a tiny host harness compiled from the library's source) is a
    topological order of Algorithm 1's task graph: every task's dependences
    come before it, and the counts match the targets the device waits for."""
    import subprocess
    import tempfile
    src = os.path.join(ROOT, "paper_2003_04776_gb300", "csrc")
    harness = r'''
#include <cstdio>
#include <vector>
#include <map>
#include <tuple>
#include "dag.cuh"
using namespace pevc;
int main() {
  // M tiles; chunks per tile and sub-chunks per tile vary (zero for tile 2)
  const int M = 6;
  int dchunk_first[M + 1], sub_first[M + 1];
  const int nch[M] = {3, 1, 0, 2, 4, 1}, nsub[M] = {2, 1, 0, 1, 3, 1};
  dchunk_first[0] = sub_first[0] = 0;
  for (int j = 0; j < M; ++j) { dchunk_first[j + 1] = dchunk_first[j] + nch[j]; sub_first[j + 1] = sub_first[j] + nsub[j]; }
  std::vector<int4> t(100000);
  int c = dag_stage_tasks(0, M, M, dchunk_first, sub_first, t.data(), 0, (int)t.size());
  for (int i = M - 1; i >= 1; --i) c = dag_stage_tasks(0, M, i, dchunk_first, sub_first, t.data(), c, (int)t.size());
  if (c < 0 || c > dag_task_bound(M, 128)) { printf("bad count %d\n", c); return 1; }
  std::map<std::pair<int,int>, int> dcnt, utile;
  std::map<std::tuple<int,int,int>, int> usub;
  for (int q = 0; q < c; ++q) {
    const int type = t[q].x >> 24, y = t[q].y, j = t[q].z;
    if (type == kTaskDiag) {
      if (utile[{y, j}] != (j - y) * nsub[j]) { printf("diag %d %d early\n", y, j); return 2; }
      dcnt[{y, j}]++;
    } else if (type == kTaskTip) {
      dcnt[{j, j}]++;
    } else {
      const int i = t[q].w >> 8, s = t[q].w & 255;
      if (dcnt[{i, j}] != nch[j] || usub[{y, j, s}] != j - i || !(y < i && i <= j)) { printf("upd early\n"); return 3; }
      usub[{y, j, s}]++;
      utile[{y, j}]++;
    }
  }
  for (int i = 0; i < M; ++i)
    for (int j = i; j < M; ++j)
      if (dcnt[{i, j}] != nch[j] || (i < j && utile[{i, j}] != (j - i) * nsub[j])) { printf("incomplete %d %d\n", i, j); return 4; }
  printf("ok %d\n", c);
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        cpp = os.path.join(d, "h.cu")
        with open(cpp, "w") as f:
            f.write(harness)
        exe = os.path.join(d, "h")
        nvcc = "/usr/local/cuda/bin/nvcc"
        r = subprocess.run([nvcc, "-std=c++17", "-I", src, "-I", os.path.join(ROOT, "include"), cpp,
                            os.path.join(src, "dag.cu"), "-o", exe, "-gencode", "arch=compute_103a,code=sm_103a"],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        out = subprocess.run([exe], capture_output=True, text=True)
        assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout
