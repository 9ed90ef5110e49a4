"""Builds the kernel emulation library for the tests -- TEST INFRASTRUCTURE.

The real-pencil path (host driver, pre-pass, diagonal solves, FP64 updates,
the task-graph scheduler (its CTAs run one after another, so the first takes
every task, in an order where each one's dependences are already met),
the split-precision path with its mma.sync update, post-pass, left flips) and
the complex-pencil path are preprocessed from the library's CUDA sources into
host C++ (launch syntax into emu::launch calls, dynamic shared memory onto the
emulated block's buffer, the L2 prefetch hint dropped, the PTX of the FP64 and
BF16 and E4M3 mma.sync, ldmatrix and cp.async onto their models) and compiled with g++
against the cuda_runtime.h stand-in beside this file.  The tcgen05 update and
the cuBLAS pieces are stubbed out (without tensor maps the split path takes
its mma.sync update); the back-transform normalisation kernels, the
bounded-wait self-test and the epilogue's flushing helpers are compiled on their own.  The result goes to tests/emu/_build/libpevc_emu.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import re
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_2003_04776_gb300", "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpevc_emu.so")
FILES = ["api.cu", "prepass.cu", "diag.cu", "dag.cu", "update_f64.cu", "post.cu", "left.cu", "cplx.cu", "split.cu"]
# headers that hold kernel code with PTX: converted like the sources, and
# included from the build directory
HEADERS = ["diag_tile.cuh"]

# split.cu's PTX helpers, replaced by their models in cuda_runtime.h
SPLIT_HELPERS = {
    "void cp_async16(": "__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) "
                        "{ emu::cp_async16(smem, gmem, valid); }",
    "void cp_async_commit(": "__device__ __forceinline__ void cp_async_commit() {}",
    "void cp_async_wait(": "template <int N>\n__device__ __forceinline__ void cp_async_wait() {}",
    "void ldmatrix_x4(": "__device__ __forceinline__ void ldmatrix_x4(unsigned (&r)[4], const void* smem) "
                         "{ emu::ldmatrix_x4(r, smem); }",
    "void mma_bf16(": "__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, "
                      "unsigned b1) { emu::mma_bf16(c, a, b0, b1); }",
    "void mma_fp8(": "__device__ __forceinline__ void mma_fp8(float (&c)[4], const unsigned (&a)[4], unsigned b0, "
                     "unsigned b1) { emu::mma_e4m3(c, a, b0, b1); }",
}


def _replace_function(src: str, marker: str, new_def: str) -> str:
    """Replaces the definition containing `marker` (from the start of its
    declaration, a template line included, to its closing brace)."""
    i = src.index(marker)
    start = src.rfind("\n", 0, i) + 1
    prev = src.rfind("\n", 0, start - 1) + 1
    if src[prev:start].startswith("template"):
        start = prev
    j = src.index("{", i)
    depth = 0
    for k in range(j, len(src)):
        depth += src[k] == "{"
        depth -= src[k] == "}"
        if depth == 0:
            return src[:start] + new_def + src[k + 1:]
    raise RuntimeError(marker)


def _convert(src: str, name: str) -> str:
    if name == "split.cu":
        for marker, new_def in SPLIT_HELPERS.items():
            src = _replace_function(src, marker, new_def)
    src = re.sub(r'#include "([\w.]+)"',
                 lambda m: f'#include "{BUILD if m.group(1) in HEADERS else CSRC}/{m.group(1)}"', src)
    src = re.sub(r"extern __shared__ (?:__align__\(\d+\) )?([\w ]+?) (\w+)\[\];",
                 r"\1* \2 = reinterpret_cast<\1*>(emu::dyn_smem);", src)
    src = re.sub(r"\b(k_\w+(?:<[^<>()]*>)?)<<<", r"emu::launch(\1, ", src)
    src = src.replace(">>>(", ", ")
    src = re.sub(r'\s*asm volatile\("prefetch\.global\.L2[^"]*"[^;]*;', "", src)
    src = re.sub(r'asm volatile\("mma\.sync.*?"d"\(b\)\);', "emu::dmma_m8n8k4(c0, c1, a, b);", src, flags=re.S)
    if "asm" in src:
        raise RuntimeError(f"{name}: inline PTX the emulation does not model")
    return src


STUBS = '''
#include <array>
#include <vector>
#include "{csrc}/common.cuh"
#include "{csrc}/split.cuh"
namespace pevc {{
// the tcgen05 update is outside the emulation: no tensor maps, so the split
// path takes its mma.sync update at every tile order
int update_tc_setup() {{ return 0; }}
int make_tensor_maps(SplitWorkspace& w) {{ w.tc_ok = false; return 0; }}
cudaError_t launch_update_tc(const Problem&, const SplitWorkspace&, int, int, int, const int*, const double*, int, int, bool,
                             cudaStream_t, bool) {{ return 1; }}
int bt_handle(void**, cudaStream_t) {{ return PEVC_ERR_UNSUPPORTED; }}
void bt_handle_destroy(void*) {{}}
int bt_gemm(void*, bool, int, int, const double*, int, const double*, int, double*, int) {{ return PEVC_ERR_UNSUPPORTED; }}
int autotune_pick(int, int, int, unsigned, void*, int*, int*, unsigned*, std::vector<std::array<double, 4>>*) {{
  return PEVC_ERR_UNSUPPORTED;
}}
int bt_zgemm(void*, int, int, const double*, int, const double*, int, double*, int) {{ return PEVC_ERR_UNSUPPORTED; }}
}}
'''


# The scalar helpers of common.cuh that the tcgen05 epilogue and the
# protection are built from, exported one by one for unit tests.
HELPERS = '''
#include "{csrc}/common.cuh"
extern "C" {{
double emu_i64_scaled_fast(long long t, int e, int* slow) {{
  bool s = false;
  const double r = pevc::i64_scaled_fast(t, e, s);
  *slow = s;
  return r;
}}
double emu_i64_scaled(long long t, int e) {{ return pevc::i64_scaled(t, e); }}
double emu_pow2_scale_fast(double y, int sh, int* slow) {{
  bool s = false;
  const double r = pevc::pow2_scale_fast(y, sh, s);
  *slow = s;
  return r;
}}
double emu_pow2_scale(double x, int e) {{ return pevc::pow2_scale(x, e); }}
int emu_exp_ub(double x) {{ return pevc::exp_ub(x); }}
int emu_protect_update(double y, double t, double x) {{ return pevc::protect_update(y, t, x); }}
int emu_protect_update_ub(double y, double t, double x) {{ return pevc::protect_update_ub(y, t, x); }}
int emu_protect_division(double b, int sh, double t) {{ return pevc::protect_division(b, sh, t); }}
double emu_max_nonneg(double x, double y) {{ return pevc::max_nonneg(x, y); }}
long long emu_alloc_count() {{ return g_emu_allocs.load(); }}
}}
'''


def _bt_source() -> str:
    src = open(os.path.join(CSRC, "backtransform.cu")).read()
    body = src[src.index("struct BtBest {"):src.index("// X = Z V for complex128 column-major arrays")]
    return (f'#include "{CSRC}/common.cuh"\nnamespace pevc {{\n{_convert(body, "backtransform.cu")}\n'
            "cudaError_t launch_bt_normalise(double* X, int ldx, int n, int m, const signed char* kind, cudaStream_t s) {\n"
            "  if (m > 0 && n > 0) emu::launch(k_bt_normalise, m, 256, 0, s, X, ldx, n, kind);\n  return 0;\n}\n"
            "cudaError_t launch_bt_normalise_c(double* X, int ldx, int n, int m, cudaStream_t s) {\n"
            "  if (m > 0 && n > 0) emu::launch(k_bt_normalise_c, m, 256, 0, s, X, ldx, n);\n  return 0;\n}\n}\n"
            'extern "C" void emu_bt_normalise(double* X, int ldx, int n, int m, const signed char* k) '
            "{ pevc::launch_bt_normalise(X, ldx, n, m, k, nullptr); }\n"
            'extern "C" void emu_bt_normalise_c(double* X, int ldx, int n, int m) '
            "{ pevc::launch_bt_normalise_c(X, ldx, n, m, nullptr); }\n")


def _ftz_source() -> str:
    """The flushing product helpers of update_tc.cu's epilogue (the correction
    sweeps'), compiled as host code and exported for unit tests."""
    src = open(os.path.join(CSRC, "update_tc.cu")).read()
    body = src[src.index("__device__ __forceinline__ double i64_scaled_ftz"):src.index("// Upper 32 bits of |x|'s bit pattern")]
    return (f'#include "{CSRC}/common.cuh"\nnamespace pevc {{\n{body}\n}}\n'
            'extern "C" double emu_i64_scaled_ftz(long long t, int e, int* slow) {\n'
            "  bool s = false;\n  const double r = pevc::i64_scaled_ftz(t, e, s);\n  *slow = s;\n  return r;\n}\n"
            'extern "C" double emu_pow2_scale_ftz(double y, int sh, int* slow) {\n'
            "  bool s = false;\n  const double r = pevc::pow2_scale_ftz(y, sh, s);\n  *slow = s;\n  return r;\n}\n")


def _watchdog_source() -> str:
    """watchdog.cu with its mbarrier PTX replaced by the model in cuda_runtime.h
    (the wait helper of tc.cuh restated on the modelled try_wait)."""
    src = open(os.path.join(CSRC, "watchdog.cu")).read()
    src = src.replace('#include "tc.cuh"\n', "")
    src = src.replace('#include "common.cuh"', f'#include "{CSRC}/common.cuh"')
    src = re.sub(r'asm volatile\("mbarrier\.arrive.*?\(&bar\)\)\);', "emu::mbar_arrive(&bar);", src, flags=re.S)
    src = re.sub(r"\b(k_\w+)<<<", r"emu::launch(\1, ", src).replace(">>>(", ", ")
    helpers = ("namespace pevc {\n"
               "inline void mbar_init(uint64_t* m, uint32_t c) { emu::mbar_init(m, c); }\n"
               "inline bool mbar_wait_cycles(uint64_t* m, uint32_t parity, long long limit) {\n"
               "  if (emu::mbar_try_wait(m, parity)) return true;\n"
               "  const long long t0 = clock64();\n"
               "  while (!emu::mbar_try_wait(m, parity))\n"
               "    if (clock64() - t0 > limit) return false;\n"
               "  return true;\n}\n}\n")
    src = src.replace("namespace pevc {", helpers + "namespace pevc {", 1)
    if "asm" in src:
        raise RuntimeError("watchdog.cu: inline PTX the emulation does not model")
    return src


def build() -> str:
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(HERE, f) for f in ("build.py", "cuda_runtime.h", "cuda_bf16.h")]
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    srcs = []
    for f in HEADERS:
        with open(os.path.join(BUILD, f), "w") as fh:
            fh.write(_convert(open(os.path.join(CSRC, f)).read(), f))
    for f in FILES:
        out = os.path.join(BUILD, f.replace(".cu", ".cpp"))
        with open(out, "w") as fh:
            fh.write(_convert(open(os.path.join(CSRC, f)).read(), f))
        srcs.append(out)
    for name, text in (("stubs.cpp", STUBS.format(csrc=CSRC)), ("bt.cpp", _bt_source()),
                       ("watchdog.cpp", _watchdog_source()), ("helpers.cpp", HELPERS.format(csrc=CSRC)),
                       ("ftz.cpp", _ftz_source())):
        out = os.path.join(BUILD, name)
        with open(out, "w") as fh:
            fh.write(text)
        srcs.append(out)

    def cc(src):
        obj = src[:-4] + ".o"
        cmd = ["g++", "-std=c++20", "-O1", "-fPIC", "-pthread", "-w", "-I", HERE, "-I", os.path.join(ROOT, "include"),
               "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError(f"g++ failed for {src}:\n{r.stderr[-4000:]}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(cc, srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run(["g++", "-shared", "-pthread", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError(r.stderr[-4000:])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build())
