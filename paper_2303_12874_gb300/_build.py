"""Build libqpic.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel; the objects link into
paper_2303_12874_gb300/_build/libqpic.so.  No cmake, no torch extension
machinery: the library is plain C ABI.

build(check=True) makes the checked variant in _build_check/: the same
sources with QPIC_CHECK defined, whose kernels test their index and
displacement invariants and report a violation as QPIC_ECHECK (no trap).
The binding loads it when QPIC_CHECKED=1 is in the environment.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libqpic.so")
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(BUILD_CHECK, "libqpic.so")
SOURCES = ["api.cu", "k_fields.cu", "k_particles.cu", "host_numerics.cpp", "noalloc.cu", "k_fp64.cu",
           "k_reduced.cu"]
# the particle kernel, one object per (mode parts, deposit variant or batched
# phase, group of tile shapes) so that the instantiations compile in parallel:
# (object name, defines).  The kernels for 5 and 7 parts take about a minute
# per tile shape, so they get one object per shape.
_SHAPES = {1: (31,), 3: (31,), 5: (1, 2, 4, 8, 16), 7: (1, 2, 4, 8, 16)}
GPD_OBJECTS = [("gpd_np%d_%s_s%d" % (np_, kind, m),
                ["-DGPD_NP=%d" % np_, "-DGPD_FA=%d" % fa, "-DGPD_BATCH=%d" % bt, "-DGPD_SHAPES=%d" % m])
               for np_ in (1, 3, 5, 7) for kind, fa, bt in (("fa0", 0, 0), ("fa1", 1, 0), ("batch", 0, 1))
               for m in _SHAPES[np_]]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "qpic.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, verbose=False, extra=(), check=False):
    bdir, lib = (BUILD_CHECK, LIB_CHECK) if check else (BUILD, LIB)
    if check:
        extra = tuple(extra) + ("-DQPIC_CHECK",)
    if not force and not _stale(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    objs = []

    def compile_one(job):
        src, name, defs = job if isinstance(job, tuple) else (job, os.path.splitext(job)[0], [])
        obj = os.path.join(bdir, name + ".o")
        cmd = [nvcc()] + ARCH + FLAGS + list(extra) + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    # the longest translation units first
    jobs = [("gpd_inst.cu", name, defs) for name, defs in GPD_OBJECTS[::-1]] + list(SOURCES)
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(compile_one, jobs))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv,
                extra=("-Xptxas", "-v") if "--ptxas" in sys.argv else ()))
