"""Build liblms.so in-tree: nvcc for the sm_103a kernels, g++ for the host code.

Three translation units compiled in parallel, linked by nvcc with the static
CUDA runtime.  Output: paper_1606_00803_gb300/_build/liblms.so.
"""
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "liblms.so")
# debug build with device-side bounds checks (-DLMS_CHECKS), objects kept apart from the release build
CHECKED_DIR = os.path.join(OUT_DIR, "checked")
LIB_CHECKED = os.path.join(OUT_DIR, "liblms_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home():
    for cand in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [os.path.join(INCLUDE, "lms.h")]


def is_stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force=False, verbose=False, checked=False):
    """Compile liblms.so (checked: liblms_checked.so, with device bounds checks) if a source is newer
    than it (or force); returns its path."""
    lib = LIB_CHECKED if checked else LIB
    obj_dir = CHECKED_DIR if checked else OUT_DIR
    if not force and not is_stale(lib):
        return lib
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(obj_dir, exist_ok=True)
    inc = ["-I" + INCLUDE, "-I" + CSRC, "-I" + os.path.join(cuda, "include")]
    host_flags = ["-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wno-unused-function"]
    jobs = []
    objs = []
    for src in sorted(os.listdir(CSRC)):
        path = os.path.join(CSRC, src)
        obj = os.path.join(obj_dir, src + ".o")
        if src.endswith(".cu"):
            cmd = [nvcc] + ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
                                   "-c", path, "-o", obj] + inc + (["-DLMS_CHECKS"] if checked else [])
            cmd += os.environ.get("LMS_NVCC_FLAGS", "").split()
        elif src.endswith(".cpp"):
            cmd = ["g++"] + host_flags + ["-c", path, "-o", obj] + inc
        else:
            continue
        objs.append(obj)
        jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in jobs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("liblms build failed:\n" + "\n".join(failed))
    tmp = lib + ".tmp%d" % os.getpid()
    link = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("liblms link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
