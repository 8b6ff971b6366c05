"""Build the CUDA library (sm_103a) in-tree: paper_2102_02655_gb300/_build/libcglbm.so.

Translation units are compiled in parallel with nvcc and linked into one
shared library exporting the C ABI of include/lbm.h.
"""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libcglbm.so")
SOURCES = ["lbm_api.cu", "lbm_plain.cu", "lbm_fused_f32.cu", "lbm_fused_f64.cu", "lbm_fused_f16.cu",
           "lbm_fused_bf16.cu", "lbm_serve.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]
# The FP32 and FP64 fused bulk kernels' global loads bypass L1 (cached in L2
# only): each population is read once per step and L1 serves under 3% of
# them, so L1 allocation only competes with the spill and shared-memory
# traffic (FP32: 0.676 -> 0.665 ms per step on the 512x128x128 print run).
# The 16-bit kernels keep L1 (two warps' 64-byte loads share a line; with the
# flag they measured 2% slower).
FILE_FLAGS = {f: ["-Xptxas", "-dlcm=cg"] for f in ("lbm_fused_f32.cu", "lbm_fused_f64.cu")}


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(ROOT, "include", "lbm.h"), os.path.abspath(__file__)]
    return max(os.path.getmtime(f) for f in files)


def flag_set(extra=()):
    """Every flag the library is compiled with, per translation unit."""
    return "\n".join("%s: %s" % (src, " ".join(ARCH + FLAGS + FILE_FLAGS.get(src, []) + list(extra)))
                     for src in SOURCES)


def _stamp():
    return os.path.join(OUT_DIR, "flags.txt")


def build(force=False, verbose=False, extra=()):
    """Compile (if sources, this script or the flags changed) and return the
    library path. The flags the library was built with are written beside it."""
    os.makedirs(OUT_DIR, exist_ok=True)
    flags = flag_set(extra)
    fresh = os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps()
    if fresh and os.path.exists(_stamp()):
        with open(_stamp()) as f:
            fresh = f.read() == flags
    else:
        fresh = False
    if not force and fresh:
        return LIB
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *FILE_FLAGS.get(src, []), *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", *objs, "-o", tmp, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(_stamp(), "w") as f:
        f.write(flags)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv, extra=["-Xptxas", "-v"] if "-v" in sys.argv else []))
