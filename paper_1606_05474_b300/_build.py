"""Build the CUDA library libhelios.so in-tree for sm_103a (nvcc, no JIT)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SO = os.path.join(HERE, "libhelios.so")
SOURCES = [os.path.join(HERE, "csrc", "helios_api.cu"), os.path.join(HERE, "csrc", "helios_noalloc.cu"),
           os.path.join(HERE, "csrc", "helios_mlp.cu"), os.path.join(HERE, "csrc", "helios_peaks.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", "helios_kernels.cuh"), os.path.join(HERE, "csrc", "helios_setup.h"),
                  os.path.join(ROOT, "include", "helios.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
         "-Xcompiler", "-fPIC,-ffp-contract=off", "--expt-relaxed-constexpr"]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source to an object in parallel (under a build folder next to this file),
    then link the shared library."""
    newest = max(os.path.getmtime(f) for f in DEPS)
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= newest:
        return SO
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    tag = f"{os.getpid()}"
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(bdir, os.path.basename(src) + f".{tag}.o")
        cmd = [NVCC, *FLAGS, "-I", os.path.join(ROOT, "include"), "-c", "-o", obj, src]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        objs.append(obj)
        procs.append(subprocess.Popen(cmd))
    rcs = [p.wait() for p in procs]
    try:
        if any(rcs):
            raise subprocess.CalledProcessError(max(rcs), "nvcc -c (see the compiler output above)")
        tmp = SO + f".tmp{tag}"
        subprocess.check_call([NVCC, "-shared", "-cudart", "shared", "-gencode", "arch=compute_103a,code=sm_103a",
                               "-o", tmp, *objs])
        os.replace(tmp, SO)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return SO


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
