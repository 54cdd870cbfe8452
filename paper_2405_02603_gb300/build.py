"""Build libfsp.so, the CUDA library behind include/fsp.h, for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel, then linked
into one shared library under paper_2405_02603_gb300/_build/.  No cmake, one
-gencode (compute_103a -> sm_103a), host code portable between x86_64 and
aarch64 (no CPU-specific flags).
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libfsp.so")
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "fsp.h")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
           "-Xptxas", "-warn-spills"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfsp.so")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    deps = [HEADER] + [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    return max(os.path.getmtime(d) for d in deps)


def library_path():
    return LIB


def needs_build():
    return (not os.path.exists(LIB)) or os.path.getmtime(LIB) < _deps()


def _compile(src, extra):
    obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc()] + ARCH + NVFLAGS + extra + ["-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, r.returncode, r.stdout + r.stderr


def build(force=False, verbose=False, extra=None):
    """Compile every csrc/*.cu and link libfsp.so (skipped when up to date)."""
    if not force and not needs_build():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    extra = list(extra or [])
    if verbose:
        extra += ["-Xptxas", "-v"]
    srcs = sources()
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(max(8, os.cpu_count() or 8), len(srcs))) as ex:
        results = list(ex.map(lambda s: _compile(s, extra), srcs))
    failed = [r for r in results if r[2] != 0]
    for src, _, rc, log in results:
        if log.strip() and (verbose or rc != 0):
            sys.stderr.write("== %s\n%s\n" % (os.path.basename(src), log))
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(os.path.basename(f[0]) for f in failed))
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + [r[1] for r in results]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
