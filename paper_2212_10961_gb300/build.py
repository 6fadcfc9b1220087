"""Build the CUDA library in-tree for sm_103a (GB300), in two flavours:
``libgrf.so`` (release) and ``libgrf_checked.so`` (the same sources with
-DGRF_CHECKED=1: device-side index checks that count and skip out-of-range
accesses, selected at run time with GRF_LIBRARY=checked).

Every translation unit of both flavours is compiled by nvcc in parallel and
linked into one shared library per flavour next to this file.  Host code uses
portable flags only, so the same command builds on x86-64 and on Arm hosts.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgrf.so")
FLAVOURS = {"release": (LIB, os.path.join(BUILD, "release"), []),
            "checked": (os.path.join(PKG, "libgrf_checked.so"), os.path.join(BUILD, "checked"),
                        ["-DGRF_CHECKED=1"])}
SOURCES = ["synth_fwd.cu", "synth_bwd.cu", "synth_grid.cu", "synth_grid_bwd.cu", "plan.cu", "maps.cu", "grf_host.cpp"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _compile(src, out_dir, defines, verbose_ptxas=False):
    out = os.path.join(out_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-I", INCLUDE, "-I", CSRC] + defines + ["-c", os.path.join(CSRC, src), "-o", out]
    if src.endswith(".cu"):
        cmd += ["-Xptxas", "-warn-spills"]
        if verbose_ptxas:
            cmd += ["-Xptxas", "-v"]
    else:
        cmd = [nvcc(), "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + defines + \
              ["-x", "c++", "-c", os.path.join(CSRC, src), "-o", out]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, res.stdout, res.stderr))
    return out, res.stderr


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "grf.h"), __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force=False, verbose_ptxas=False, flavours=("release", "checked")):
    """Compile and link each flavour whose library is older than a source;
    returns the release library's path."""
    todo = [f for f in flavours if force or _stale(FLAVOURS[f][0])]
    if not todo:
        return LIB
    jobs = []
    for f in todo:
        _, out_dir, defines = FLAVOURS[f]
        os.makedirs(out_dir, exist_ok=True)
        jobs += [(f, src, out_dir, defines) for src in SOURCES]
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(lambda j: (j[0],) + _compile(j[1], j[2], j[3], verbose_ptxas), jobs))
    if verbose_ptxas:
        for _, _, log in results:
            if log:
                sys.stderr.write(log)
    for f in todo:
        lib = FLAVOURS[f][0]
        objs = [o for g, o, _ in results if g == f]
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [nvcc(), ARCH, "-shared", "-cudart", "shared", "-o", tmp] + objs
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (res.stdout, res.stderr))
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
    print(LIB)
