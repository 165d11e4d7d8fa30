"""Build libzef.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel into _build/ and linked into
_build/libzef.so.  `python -m paper_2203_10000_gb300.build` or
`__graft_entry__.build()` runs it.  `build(debug=True)` (or `--debug`) builds
the debug variant into _build_debug/libzef.so: the same sources with
ZEF_DEBUG_BOUNDS defined, whose kernels check the indices they compute and
report a failed check as ZEF_ERR_BOUNDS instead of touching memory.  The
binding loads it when the environment variable ZEF_LIBRARY names it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libzef.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libzef.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          "-I", os.path.join(ROOT, "include"), "-I", CSRC]
PER_FILE = {
    # FP32 hot loop: flush denormals so rsqrtf/__fdividef map to single MUFU ops
    "zef_label.cu": ["-ftz=true", "-Xptxas", "-v"],
}
SOURCES = ["zef_host.cpp", "zef_tree.cpp", "zef_label.cu", "zef_refine.cu", "zef_relabel.cu", "zef_post.cu", "zef_noalloc.cu"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _newer(src_paths, out) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(p) > t for p in src_paths)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    out_dir = BUILD_DEBUG if debug else BUILD
    lib = LIB_DEBUG if debug else LIB
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    extra = ["-DZEF_DEBUG_BOUNDS"] if debug else []
    headers = [os.path.join(ROOT, "include", "zef.h"), os.path.join(CSRC, "zef_internal.h")]
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(out_dir, s + ".o")
        objs.append(obj)
        if force or _newer([src] + headers, obj):
            cmd = [nvcc, *ARCH, *COMMON, *extra, *PER_FILE.get(s, []), "-c", src, "-o", obj]
            if s.endswith(".cpp"):
                cmd = [nvcc, *COMMON, *extra, "-x", "c++", "-c", src, "-o", obj]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    if force or jobs or not os.path.exists(lib):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-lpthread", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
