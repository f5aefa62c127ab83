"""Build the CUDA library libgspoisson.so in-tree for sm_103a.

Each translation unit is compiled by nvcc in its own process (in parallel), then linked
into paper_1612_01799_gb300/libgspoisson.so.  Objects go to _build/ at the repo root.
build(debug=True) builds the debug variant libgspoisson_debug.so (GSP_DEBUG: bounds-checked
shared-memory and index accesses, relocatable device code so that one device-wide
flag word serves every unit) from the same sources, objects in _build_debug/.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "libgspoisson.so")
BUILD = os.path.join(ROOT, "_build")
OUT_DEBUG = os.path.join(PKG, "libgspoisson_debug.so")
BUILD_DEBUG = os.path.join(ROOT, "_build_debug")
SOURCES = ["capi.cpp", "setup.cpp", "passes_f32.cu", "passes_f64.cu", "passes_df.cu",
           "passes_f32_a.cu", "passes_f32_b.cu", "passes_f32_c.cu",
           "passes_f64_a.cu", "passes_f64_b.cu", "passes_f64_c.cu",
           "passes_df_1.cu", "passes_df_2.cu", "passes_df_3.cu", "passes_df_4.cu", "passes_df_5.cu",
           "passes_df_6.cu", "passes_df_7.cu", "passes_df_8.cu", "passes_df_9.cu",
           "noalloc.cu", "reduce.cu", "sample.cu", "selector.cu", "selftest.cu", "setup_device.cu", "debug.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgspoisson")
    return cand


def _deps(src):
    """Sources and headers whose change forces a rebuild of src."""
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return [os.path.join(CSRC, src), os.path.join(ROOT, "include", "poisson.h")] + hdrs


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra_flags=(), debug=False):
    nvcc = _nvcc()
    bdir, out = (BUILD_DEBUG, OUT_DEBUG) if debug else (BUILD, OUT)
    os.makedirs(bdir, exist_ok=True)
    flags = ["-std=c++20", "-O3", "-lineinfo", "-Xcompiler", "-fPIC"] + ARCH + list(extra_flags)
    link_flags = []
    if debug:
        flags += ["-DGSP_DEBUG", "-rdc=true"]
        link_flags = ["-rdc=true"]
    jobs = []
    for src in SOURCES:
        obj = os.path.join(bdir, src + ".o")
        if force or _stale(obj, _deps(src)):
            cmd = [nvcc] + flags + ["-I", os.path.join(ROOT, "include"), "-c",
                                    os.path.join(CSRC, src), "-o", obj]
            jobs.append(cmd)
    objs = [os.path.join(bdir, s + ".o") for s in SOURCES]

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            sys.stderr.write(r.stderr)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _stale(out, objs):
        tmp = out + ".%d.tmp" % os.getpid()
        run([nvcc, "-shared"] + link_flags + ARCH + ["-o", tmp] + objs)
        os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
