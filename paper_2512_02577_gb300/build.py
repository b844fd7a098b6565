"""Build the in-tree shared library ``libpmg.so`` for sm_103a.

Every CUDA translation unit is compiled by nvcc in parallel: the runtime and
vector kernels, and ``csrc/inst.cu`` once per kernel part -- each polynomial
degree 1..8 x dimension 2, 3 x precision double, float, selected by -D flags
-- so that no single unit dominates the build; the host set-up code by nvcc as
C++.  First ``csrc/gen_coef.cpp`` (host code, with the library's own
set-up) writes ``_build/coef_tables.h``: the per-degree 1D coefficient blocks
as compile-time initialisers for the kernels.  Objects go to ``_build/``; the library is linked next to this file.  An
object is rebuilt when its source or a header it includes (transitively) is
newer than it.
"""
import concurrent.futures
import glob
import os
import re
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpmg.so")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "--expt-relaxed-constexpr", "-lineinfo", "-Xcompiler", "-fPIC",
         "-I" + CSRC, "-I" + INCLUDE, "-I" + BUILD]


PART_SRC = os.path.join(CSRC, "inst.cu")
DEGREES, DIMS, PRECS = range(1, 9), (2, 3), (0, 1)


GEN_SRC = [os.path.join(CSRC, "gen_coef.cpp"), os.path.join(CSRC, "setup.cpp")]
GEN_HEADER = os.path.join(BUILD, "coef_tables.h")


def _generate_tables(verbose):
    """Compile and run gen_coef (host code) and write coef_tables.h into the
    build directory, rewriting it only when its contents change."""
    exe = os.path.join(BUILD, "gen_coef")
    if any(_stale(exe, s) for s in GEN_SRC):
        cmd = [NVCC, "-std=c++17", "-O2", "-I" + CSRC, "-I" + INCLUDE] + GEN_SRC + ["-o", exe]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("gen_coef build failed:\n%s%s" % (r.stdout, r.stderr))
    r = subprocess.run([exe], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("gen_coef failed:\n" + r.stderr)
    old = open(GEN_HEADER).read() if os.path.exists(GEN_HEADER) else None
    if old != r.stdout:
        with open(GEN_HEADER, "w") as f:
            f.write(r.stdout)


def _units():
    """(source, object name, extra flags), heaviest kernel parts first."""
    units = [(PART_SRC, "inst_k%d_d%d_p%d.o" % (k, d, p), ["-DPMG_K=%d" % k, "-DPMG_DIM=%d" % d, "-DPMG_PREC=%d" % p])
             for k in reversed(DEGREES) for d in reversed(DIMS) for p in PRECS]
    others = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    units += [(s, os.path.basename(s) + ".o", []) for s in others if s not in (PART_SRC, GEN_SRC[0])]
    return units


_INCLUDE_RE = re.compile(r'^\s*#\s*include\s*"([^"]+)"', re.M)


def _includes(path, seen=None):
    """Every project header that ``path`` includes, transitively (quoted
    includes resolved next to the including file, then in include/)."""
    seen = set() if seen is None else seen
    with open(path) as f:
        text = f.read()
    for name in _INCLUDE_RE.findall(text):
        for base in (os.path.dirname(path), INCLUDE, BUILD):
            h = os.path.normpath(os.path.join(base, name))
            if os.path.exists(h):
                if h not in seen:
                    seen.add(h)
                    _includes(h, seen)
                break
    return seen


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(f) > t for f in [src] + sorted(_includes(src)))


def _compile(src, obj, extra, verbose):
    cmd = [NVCC] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    return obj


def build(verbose=False, jobs=None):
    """Compile (incrementally) and link libpmg.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    _generate_tables(verbose)
    objs, todo = [], []
    for s, name, extra in _units():
        o = os.path.join(BUILD, name)
        objs.append(o)
        if _stale(o, s):
            todo.append((s, o, extra))
    jobs = jobs or min(len(todo) or 1, os.cpu_count() or 4)
    if todo:
        with concurrent.futures.ThreadPoolExecutor(max_workers=jobs) as ex:
            futs = [ex.submit(_compile, s, o, extra, verbose) for s, o, extra in todo]
            for f in futs:
                f.result()
    if todo or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [NVCC] + ARCH + ["-shared", "-o", LIB] + objs
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
