"""Build libphipm.so (the C ABI of include/phipm.h) in-tree with nvcc for sm_103a.

The nine solver-kernel instances (basis element type x team form) are compiled from
phipm_kernels.cu as separate objects, in parallel with the C ABI's object, and
linked into one shared library (no relocatable device code: every kernel is
launched from the object that defines it)."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libphipm.so")
SOURCES = ["phipm_capi.cu", "phipm_kernels.cu"]
HEADERS = ["phipm_common.cuh", "phipm_elem.cuh", "phipm_engine.cuh", "phipm_mlp.cuh", "phipm_mlp_train.cuh",
           "phipm_launch.h"]
# (object name, source, macros): the C ABI plus one object per (element type, team form)
UNITS = [("capi", "phipm_capi.cu", [])] + [
    (f"kern_e{e}_f{f}", "phipm_kernels.cu", [f"-DPM_ELEM={e}", f"-DPM_FORM={f}"]) for e in range(3) for f in range(3)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in [os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"]:
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "phipm.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def _code_only(text: str) -> str:
    """C/C++ source without comments and blank-line runs, so that the hash of a kernel
    build does not change with its comments (string literals keep their contents)."""
    import re
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"' or c == "'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    code = "".join(out)
    return "\n".join(l.rstrip() for l in code.splitlines() if l.strip())


def source_hash() -> str:
    """sha256 of the CUDA sources and the ABI header with comments stripped (identifies
    the code of a kernel build)."""
    import hashlib
    h = hashlib.sha256()
    for f in sorted(SOURCES + HEADERS):
        h.update(_code_only(open(os.path.join(CSRC, f)).read()).encode())
    h.update(_code_only(open(os.path.join(ROOT, "include", "phipm.h")).read()).encode())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False, lib: str = LIB, defines: tuple = ()) -> str:
    """Compile the library if it is missing or older than its sources; return its path.
    lib and defines build a variant elsewhere (e.g. a phase-timer probe build with
    defines=("-DPM_PHASE_PROBE",) into another file); the default is the product library."""
    if lib == LIB and not defines and not force and not _stale():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    objdir = os.path.join(os.path.dirname(lib), f"obj{os.getpid()}")
    os.makedirs(objdir, exist_ok=True)
    common = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
              *defines]
    if verbose:
        common.append("-Xptxas=-v")

    def compile_unit(unit):
        name, src, macros = unit
        obj = os.path.join(objdir, name + ".o")
        cmd = common + macros + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        return obj, r

    workers = max(1, min(len(UNITS), os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(compile_unit, UNITS))
    for obj, r in results:
        if r.stdout or r.stderr:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise subprocess.CalledProcessError(r.returncode, r.args)
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run([_nvcc(), *ARCH, "-shared", "-o", tmp] + [o for o, _ in results], check=True)
    os.replace(tmp, lib)
    for o, _ in results:
        os.unlink(o)
    os.rmdir(objdir)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
