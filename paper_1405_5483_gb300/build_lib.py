"""Compiles the CUDA library libmpm.so in-tree (sm_103a only).

Every translation unit is compiled in parallel with nvcc, then linked into
paper_1405_5483_gb300/_build/libmpm.so with the CUDA runtime linked
statically, so the library loads on a machine without a GPU (for symbol
checks) and needs only the NVIDIA kernel driver when it runs.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmpm.so")

SOURCES = ["host_build.cpp", "capi.cu", "scan.cu", "encode.cu", "verify.cu", "sort.cu", "jit.cpp",
           "tune.cpp", "batch.cu", "mlp.cu"]
# sources of the kernels compiled at run time, embedded as C++ raw strings:
# each generated file is the concatenation of its parts (file names, or
# literal text)
_NS_OPEN, _NS_CLOSE = "namespace mpm {\n", "}  // namespace mpm\n"
JIT_SOURCES = {
    # the single-text specialised scan
    "scan_jit_src.inc": ["keyhash.h", "multiword.h", "scan_jit_args.h", "ptx_common.cuh",
                         "window_check.cuh", "jit_types.h", _NS_OPEN, "scan_stage.cuh",
                         _NS_CLOSE, "scan_jit.cuh"],
    # the batched kernel: prelude, the stage primitives and the lane scan
    # (once per parameter set of a batch), the kernel
    "batch_prelude_src.inc": ["keyhash.h", "multiword.h", "ptx_common.cuh", "window_check.cuh",
                              "jit_types.h", "batch_args.h"],
    "batch_stage_src.inc": ["scan_stage.cuh", "batch_lane.cuh"],
    "batch_kernel_src.inc": ["batch_jit.cuh"],
}
JIT_PARTS = sorted({p for parts in JIT_SOURCES.values() for p in parts if p.endswith((".h", ".cuh"))})
GEN = os.path.join(OUT, "gen")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I" + INCLUDE, "-I" + CSRC, "-I" + GEN]


def _write_jit_source():
    """Embeds the run-time compiled kernels' sources as C++ raw strings."""
    os.makedirs(GEN, exist_ok=True)
    for name, parts in JIT_SOURCES.items():
        text = ""
        for part in parts:
            if part.endswith((".h", ".cuh")):
                with open(os.path.join(CSRC, part)) as f:
                    text += "// ---- %s\n" % part + f.read().replace("#pragma once", "") + "\n"
            else:
                text += part
        assert ")MPMJIT\"" not in text
        out = os.path.join(GEN, name)
        body = 'R"MPMJIT(' + text + ')MPMJIT"\n'
        if not os.path.exists(out) or open(out).read() != body:
            with open(out, "w") as f:
                f.write(body)


def _deps_mtime():
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return max(os.path.getmtime(p) for p in paths)


def build(force=False, verbose=False):
    """Builds libmpm.so if any source is newer; returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    nvcc = _nvcc()
    _write_jit_source()
    objdir = os.path.join(OUT, "obj")
    os.makedirs(objdir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(objdir, src + ".o")
        cmd = [nvcc] + _flags() + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd[1:1] = ["-x", "cu"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), p.stderr))
        if verbose and p.stderr.strip():
            sys.stderr.write(p.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs + ["-ldl"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), p.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
