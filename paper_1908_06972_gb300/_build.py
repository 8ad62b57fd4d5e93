"""Build the CUDA library libprivft.so in-tree (sm_103a only).

Sources are compiled in parallel with nvcc (-gencode arch=compute_103a,code=sm_103a)
and linked into ``paper_1908_06972_gb300/_build/libprivft.so`` with the CUDA
runtime linked statically.  Nothing here needs a GPU.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
SO = os.path.join(OUT, "libprivft.so")
SOURCES = ["ntt.cu", "poly.cu", "ckks.cu", "serve.cu", "train.cu", "queue.cu", "hostmath.cpp"]
HEADERS = ["pft_internal.h", "evaluator.h", "modarith.cuh", os.path.join("..", "..", "include", "privft.h")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale():
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, ptxas_info=False):
    """Compile and link; returns the path of the shared library."""
    if not force and not _stale():
        return SO
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    common = ["-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off"]
    if ptxas_info:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + common
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose or ptxas_info:
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = SO + ".tmp.%d" % os.getpid()
    cmd = [cc, "-shared", ARCH, "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
