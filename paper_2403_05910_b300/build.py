"""Build the sm_103a C-ABI library paper_2403_05910_b300/libxf.so with nvcc."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libxf.so")
# (source, extra flags): the adjoint launchers compile once per reconstruction
UNITS = [("xf_api.cu", []), ("xf_batch.cu", []),
         ("xf_adjoint_launch.cu", ["-DXF_ADJ_REC=5"]),
         ("xf_adjoint_launch.cu", ["-DXF_ADJ_REC=6"]),
         ("xf_adjoint_launch.cu", ["-DXF_ADJ_REC=7"])]
SOURCES = sorted({os.path.join(CSRC, u) for u, _ in UNITS})
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-shared", "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    return files + [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source to an object in parallel (one nvcc per source),
    then link the shared library; rebuilt only when a source is newer."""
    newest = max(os.path.getmtime(f) for f in _deps())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tag = f".tmp{os.getpid()}"
    objs = [os.path.join(CSRC, f"{u}.{k}{tag}.o") for k, (u, _) in enumerate(UNITS)]
    compile_flags = [f for f in FLAGS if f != "-shared"]
    procs = [subprocess.Popen([NVCC, *compile_flags, *extra,
                               *(["-Xptxas", "-v"] if verbose else []),
                               "-c", "-o", obj, os.path.join(CSRC, u)])
             for (u, extra), obj in zip(UNITS, objs)]
    codes = [p.wait() for p in procs]
    try:
        if any(codes):
            raise subprocess.CalledProcessError(max(codes), "nvcc -c")
        tmp = LIB + tag
        subprocess.check_call([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                               "-o", tmp, *objs])
        os.replace(tmp, LIB)
    finally:
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
