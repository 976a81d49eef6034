"""Build the CUDA library libhelios.so in-tree for sm_103a (nvcc, no JIT)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SO = os.path.join(HERE, "libhelios.so")
SOURCES = [os.path.join(HERE, "csrc", "helios_api.cu"), os.path.join(HERE, "csrc", "helios_noalloc.cu"),
           os.path.join(HERE, "csrc", "helios_mlp.cu"), os.path.join(HERE, "csrc", "helios_peaks.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", "helios_mlp.cu"), os.path.join(HERE, "csrc", "helios_kernels.cuh"), os.path.join(ROOT, "include", "helios.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
         "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared", "-cudart", "shared", "--expt-relaxed-constexpr"]


def build(force: bool = False, verbose: bool = False) -> str:
    newest = max(os.path.getmtime(f) for f in DEPS)
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= newest:
        return SO
    tmp = SO + f".tmp{os.getpid()}"
    cmd = [NVCC, *FLAGS, "-I", os.path.join(ROOT, "include"), "-o", tmp, *SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
