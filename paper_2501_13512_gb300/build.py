"""Builds libvie.so in the package directory with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel into ``_build/``; the shared
library links the CUDA runtime statically, so it needs only the driver.
Rebuilds only when a source or header is newer than the library.
"""
import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
SOURCES = ["fft.cu", "krylov.cu", "fields.cu", "api.cu", "profile.cu", "inner.cu", "noalloc.cu", "batch.cu",
           "farfield.cu", "rooftop.cu"]
HEADERS = [os.path.join(CSRC, "vie_internal.cuh"), os.path.join(CSRC, "fft_core.cuh"), os.path.join(CSRC, "fft_reg.cuh"),
           os.path.join(ROOT, "include", "vie.h")]
LIB = os.path.join(HERE, "libvie.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
                "-I" + os.path.join(ROOT, "include")] + os.environ.get("VIE_NVCC_FLAGS", "").split()


def nvcc_path():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvie")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile and link libvie.so; returns its path."""
    nvcc = nvcc_path()
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + HEADERS):
            jobs.append([nvcc] + FLAGS + ["-c", s, "-o", o])

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, p

    log = []
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for cmd, p in ex.map(run, jobs):
            log.append(p.stderr)
            if p.returncode != 0:
                raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + p.stdout + p.stderr)
    if force or jobs or _stale(LIB, objs):
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB] + objs
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + p.stdout + p.stderr)
    if verbose:
        print("\n".join(log))
    with open(os.path.join(bdir, "ptxas.log"), "a") as f:
        f.write("\n".join(log))
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
