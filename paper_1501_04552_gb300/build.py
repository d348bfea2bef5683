"""Build libkg.so (the CUDA library behind include/kg.h) in-tree for sm_103a.

Each translation unit is compiled by its own nvcc process in parallel, then linked
into paper_1501_04552_gb300/libkg.so.  Object files go to paper_1501_04552_gb300/_build/.
kg_inst.cu is compiled fifteen times, once per (precision, share) of the pass
launchers (csrc/kg_inst.h), so that the heavy kernel templates build in parallel.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libkg.so")
# (source, extra defines, object name); the double-float shares first: they take longest
UNITS = ([("kg_inst.cu", ["-DKG_PREC_ID=%d" % p, "-DKG_PART=%d" % s], "kg_inst_p%d_s%d.o" % (p, s))
          for p in (1, 2, 0) for s in range(5)] +
         [(f, [], f.replace(".cu", ".o")) for f in
          ["kg_inst_tables.cu", "kg_common.cu", "kg_api.cu", "kg_host.cu", "kg_ensemble.cu", "kg_mlp.cu",
           "kg_noalloc.cu"]])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-warn-spills"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _sources_mtime():
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "kg.h")]
    return max(os.path.getmtime(p) for p in paths)


def build(force=False, verbose=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(unit):
        src, defs, name = unit
        obj = os.path.join(BUILD, name)
        cmd = [nvcc] + ARCH + FLAGS + defs + ["-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, src),
                                              "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(UNITS), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
