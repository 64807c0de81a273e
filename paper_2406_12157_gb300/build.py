"""Build ``libshe.so`` (the C-ABI library) for sm_103a with nvcc, in-tree.

Each ``csrc/*.cu`` translation unit is compiled in parallel to an object
file, then linked into ``paper_2406_12157_gb300/_build/libshe.so``.  The
fused 1D kernel's instantiation unit (``step1d_inst.cu``) is compiled once per
(precision, wall, equation, scheme, material table) variant, and once per
(precision, wall, equation) for the implicit schemes, 32 objects, so that its
template instances compile in parallel too.  One ``-gencode``
(compute_103a -> sm_103a); no CMake.  An object is recompiled only when its
source or any header is newer than it; the library is relinked when an
object changed.
"""
import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libshe.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", INCLUDE]


def nvcc():
    exe = shutil.which("nvcc")
    if exe is None:
        cand = "/usr/local/cuda/bin/nvcc"
        if os.path.exists(cand):
            exe = cand
    if exe is None:
        raise RuntimeError("nvcc not found: libshe needs the CUDA toolkit to build")
    return exe


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


# Units compiled once per variant: file name -> list of (object tag, defines).
VARIANTS = {
    "step1d_inst.cu": [
        ("%s_%s_%s_%s%s" % (real[0], "dir" if d else "per", "sp" if s else "heat", "pc" if pc else "fe",
                            "_var" if v else ""),
         ["-DSHE_V_REAL=%s" % real, "-DSHE_V_DIR=%d" % d, "-DSHE_V_SP=%d" % s, "-DSHE_V_PC=%d" % pc,
          "-DSHE_V_VAR=%d" % v])
        for real in ("float", "double") for d in (0, 1) for s in (0, 1) for pc in (0, 1) for v in (0, 1)
        if not (v and s)] + [    # the material table is for heat rods
        ("%s_%s_%s_theta" % (real[0], "dir" if d else "per", "sp" if s else "heat"),
         ["-DSHE_V_REAL=%s" % real, "-DSHE_V_DIR=%d" % d, "-DSHE_V_SP=%d" % s, "-DSHE_V_IMP=1"])
        for real in ("float", "double") for d in (0, 1) for s in (0, 1)],
    # the fused covariance kernels: explicit or implicit step, without and with the time correlation
    "step1d_cov.cu": [("fe", ["-DSHE_COV_TC=0", "-DSHE_COV_IMP=0"]), ("tc", ["-DSHE_COV_TC=1", "-DSHE_COV_IMP=0"]),
                      ("imp", ["-DSHE_COV_TC=0", "-DSHE_COV_IMP=1"]),
                      ("imp_tc", ["-DSHE_COV_TC=1", "-DSHE_COV_IMP=1"])],
}


def jobs():
    """(source, object path, extra defines) of every object of the library."""
    out = []
    for src in sources():
        base = os.path.basename(src)
        for tag, defs in VARIANTS.get(base, [("", [])]):
            obj = os.path.join(OUT_DIR, base + ("." + tag if tag else "") + ".o")
            out.append((src, obj, defs))
    return out


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _obj_stale(src, obj, newest_header):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return os.path.getmtime(src) > t or newest_header > t


def _compile(src, obj, extra):
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, res.stdout, res.stderr))
    return obj, res.stderr


def build(force=False, verbose=False, extra_flags=()):
    """Compile every CUDA source (stale objects only, unless `force`) and
    link libshe.so; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    extra = list(extra_flags)
    newest_header = max([os.path.getmtime(f) for f in _headers()] + [0.0])
    all_jobs = jobs()
    todo = [j for j in all_jobs if force or extra or _obj_stale(j[0], j[1], newest_header)]
    objs = [o for _, o, _ in all_jobs]
    if not todo and os.path.exists(LIB) and all(os.path.getmtime(o) <= os.path.getmtime(LIB) for o in objs):
        return LIB
    # longest units first (the variant objects and the larger kernels)
    todo.sort(key=lambda j: -os.path.getsize(j[0]) - (10 ** 6 if j[2] else 0))
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda j: _compile(j[0], j[1], j[2] + extra), todo))
    if verbose:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-ldl"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (res.stdout, res.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    flags = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v or bool(flags), extra_flags=flags))
