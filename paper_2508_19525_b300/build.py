"""Build the CUDA library libblb.so in-tree for sm_103a (B300).

nvcc cross-compiles without a GPU.  The library is a plain C-ABI shared object
(include/blb.h); the Python binding loads it with ctypes.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libblb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-fast-math",
         "--expt-relaxed-constexpr"]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale():
    if not os.path.exists(LIB):
        return True
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps += [os.path.join(ROOT, "include", "blb.h"), __file__, CSRC]  # the directory: a source removed
    return max(os.path.getmtime(f) for f in deps) > os.path.getmtime(LIB)


def build(force=False, verbose=False, extra=(), asan=False):
    """Compile every csrc/*.cu for sm_103a and link libblb.so.  asan=True adds
    AddressSanitizer to the host code (debug builds; run python with the
    sanitizer runtime preloaded and ASAN_OPTIONS=protect_shadow_gap=0)."""
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    san = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fno-omit-frame-pointer", "-g"] if asan else []
    extra = list(extra) + san
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    objs = []
    procs = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), src))
        objs.append(obj)
    failed = []
    for p, src in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append(src + "\n" + out.decode(errors="replace"))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    cmd = [nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *objs, "-lcudart"] + (["-Xcompiler", "-fsanitize=address"] if asan else [])
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


PEAKS_SRC = os.path.join(HERE, "peaks", "peaks.cu")
PEAKS_LIB = os.path.join(HERE, "libblb_peaks.so")


def build_peaks(force=False):
    """The benchmark's integer-rate microbenchmark (include/blb_peaks.h) as a
    library of its own, libblb_peaks.so: it is not part of libblb.so."""
    if not force and os.path.exists(PEAKS_LIB) and os.path.getmtime(PEAKS_LIB) >= max(
            os.path.getmtime(PEAKS_SRC), os.path.getmtime(os.path.join(ROOT, "include", "blb_peaks.h")), os.path.getmtime(__file__)):
        return PEAKS_LIB
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    cmd = [nvcc, *ARCH, *FLAGS, "-I", os.path.join(ROOT, "include"), "-shared", "-o", PEAKS_LIB + ".tmp", PEAKS_SRC,
           "-lcudart"]
    subprocess.run(cmd, check=True)
    os.replace(PEAKS_LIB + ".tmp", PEAKS_LIB)
    return PEAKS_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [], asan="--asan" in sys.argv))
    print(build_peaks(force="--force" in sys.argv))
