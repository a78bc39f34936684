"""Build librimg.so (the CUDA library behind include/rimg.h) in-tree for sm_103a.

    python -m paper_2112_02779_b300.build [--verbose]

nvcc cross-compiles without a GPU.  The shared library lands in
paper_2112_02779_b300/_lib/librimg.so and statically links the CUDA runtime.
"""
import argparse
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "librimg.so")
SOURCES = ["rimg_api.cu", "kernels_prep.cu", "kernel_icp.cu", "rimg_noalloc.cu", "kernel_gemm.cu", "rimg_cnn.cu", "kernel_sdf.cu", "kernel_points.cu", "kernel_center.cu"]
# Per-file nvcc options of the default build.  The FP32 registration, sensor
# and fusion kernels flush denormals (FP32 values below 2^-126 are zero in
# their inputs and results): ranges, coordinates and normals are never that
# small, and it removes the denormal handling around reciprocal and
# reciprocal-square-root approximations in the per-pixel code.
_FTZ = ["-ftz=true"]
SOURCE_FLAGS = {"kernel_icp.cu": _FTZ, "kernels_prep.cu": _FTZ, "kernel_sdf.cu": _FTZ, "kernel_points.cu": _FTZ,
                "kernel_center.cu": _FTZ}
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(ROOT, "include", "rimg.h"))
    return files


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(verbose=False, force=False, out=None, defines=(), flags=None):
    """Compile every CUDA source into one shared library (default: the
    in-tree librimg.so).  `defines` are extra -D tunables (e.g. RIMG_RING=2);
    `flags` maps a source file to extra nvcc options for it alone.  Sources
    compile to objects in parallel, then one link step."""
    lib = out or LIB
    flags = dict(SOURCE_FLAGS if flags is None else flags)
    if not force and out is None and not defines and up_to_date():
        return LIB
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    objdir = lib + ".objs"
    os.makedirs(objdir, exist_ok=True)
    common = [NVCC, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2",
              "-I", os.path.join(ROOT, "include")] + [f"-D{d}" for d in defines]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
        res = subprocess.run(common + list(flags.get(src, ())) + ["-c", "-o", obj, os.path.join(CSRC, src)],
                             capture_output=True, text=True)
        return src, obj, res

    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    failed = [r for r in results if r[2].returncode != 0]
    for src, _, res in results:
        if res.returncode != 0 or verbose:
            sys.stderr.write(f"== {src}\n" + res.stdout + res.stderr)
    if failed:
        raise RuntimeError("nvcc failed building librimg.so: " + ", ".join(r[0] for r in failed))
    tmp = lib + ".tmp"
    res = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp] + [r[1] for r in results], capture_output=True,
                         text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed linking librimg.so")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--out", default=None, help="output path (default: in-tree _lib/librimg.so)")
    ap.add_argument("-D", dest="defines", action="append", default=[], help="extra tunable, e.g. -D RIMG_RING=2")
    a = ap.parse_args()
    print(build(verbose=a.verbose, force=a.force, out=a.out, defines=a.defines))
