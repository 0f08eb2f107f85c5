"""Build the accr C-ABI library (``libaccr.so``) in-tree with nvcc for sm_103a.

Every ``csrc/*.cu`` file is compiled to an object in parallel, then linked
into ``paper_1412_1127_gb300/libaccr.so`` with the static CUDA runtime, so the
library loads without a GPU (for symbol checks) and needs only the driver at
run time.  Only the ``accr_*`` entry points are exported.
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libaccr.so")
DEBUG_BUILD = os.path.join(PKG, "_build_debug")
DEBUG_LIB = os.path.join(PKG, "libaccr_debug.so")  # bounds-checked build (-DACCR_DEBUG)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr",
                     "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                     "-I", INCLUDE, "-I", CSRC]


def nvcc():
    for c in [os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"]:
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


# Autotuned compile-time constants: (key in the table's "vectors", macro, source)
TUNED = [("tile_vectors", "ACCR_BATCH_BU", "batch.cu"), ("warp_vectors", "ACCR_BATCH_SU", "batch.cu"),
         ("min_ctas_per_sm", "ACCR_BATCH_MINB", "batch.cu"), ("reduce_vectors", "ACCR_REDUCE_RU", "reduce.cu"),
         ("row_vectors", "ACCR_ROW_RU", "rowreduce.cu")]
TUNED_SOURCES = sorted({src for _, _, src in TUNED})


def tuned_defines(table=None, source="batch.cu"):
    """Compile-time definitions of one source from the autotuner's table
    ("vectors" in tuning.json): the vectors in flight of the batched-region,
    single-region and row kernels."""
    import json
    path = table or os.path.join(PKG, "tuning.json")
    try:
        with open(path) as f:
            v = json.load(f).get("vectors") or {}
    except (OSError, ValueError):
        v = {}
    return ["-D%s=%d" % (macro, int(v[key])) for key, macro, src in TUNED if src == source and key in v]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, jobs=None, defines=None, build_dir=None, lib=None, debug=False):
    """Compile and link libaccr.so if any source, header or the tuning table
    changed.  `defines` ({source name: [flags]}), `build_dir` and `lib`
    override the tuned definitions and the output paths; debug=True builds
    the bounds-checked library libaccr_debug.so (-DACCR_DEBUG) instead."""
    if debug:
        build_dir, lib = build_dir or DEBUG_BUILD, lib or DEBUG_LIB
    build_dir, lib = build_dir or BUILD, lib or LIB
    extra = ["-DACCR_DEBUG"] if debug else []
    os.makedirs(build_dir, exist_ok=True)
    srcs, hdrs = _sources(), _headers()
    table = os.path.join(PKG, "tuning.json")
    objs = [os.path.join(build_dir, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def defs_for(s):
        name = os.path.basename(s)
        if defines is not None:
            return list(defines.get(name, [])) if isinstance(defines, dict) else []
        return tuned_defines(source=name)

    def deps(s):  # the tuned widths reach their own sources only
        tuned = os.path.basename(s) in TUNED_SOURCES and os.path.exists(table)
        return [s] + hdrs + ([table] if tuned else [])
    todo = [(s, o) for s, o in zip(srcs, objs) if force or _stale(o, deps(s))]

    def compile_one(so):
        s, o = so
        cmd = [nvcc()] + NVCC_FLAGS + extra + defs_for(s) + ["-c", s, "-o", o + ".tmp"]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (s, r.stdout, r.stderr))
        os.replace(o + ".tmp", o)
        return r.stderr

    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            for msg in ex.map(compile_one, todo):
                if msg and verbose:
                    print(msg)
    if force or todo or _stale(lib, objs):
        tmp = lib + ".%d.tmp" % os.getpid()
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread", "-ldl", "-lrt"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)
    return lib


def build_variant(source, defines, out_dir):
    """A library whose `source` (a csrc file name, e.g. "batch.cu") is built
    with `defines` instead of the tuned ones; the other objects are the main
    build's.  The autotuner times such variants.  Returns the library's path."""
    build()
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(CSRC, source)
    obj = os.path.join(out_dir, source[:-3] + ".o")
    lib = os.path.join(out_dir, "libaccr.so")
    r = subprocess.run([nvcc()] + NVCC_FLAGS + list(defines) + ["-c", src, "-o", obj], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for a variant of %s:\n%s%s" % (source, r.stdout, r.stderr))
    objs = [o for o in (os.path.join(BUILD, os.path.basename(x)[:-3] + ".o") for x in _sources())
            if os.path.basename(o) != source[:-3] + ".o"]
    r = subprocess.run([nvcc()] + ARCH + ["-shared", "-o", lib, obj] + objs + ["-lpthread", "-ldl", "-lrt"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed for a variant of %s:\n%s%s" % (source, r.stdout, r.stderr))
    return lib


def build_batch_variant(defines, out_dir):
    return build_variant("batch.cu", defines, out_dir)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
