"""Builds libsnp.so in-tree for sm_103a with nvcc (no cmake, no torch build).

Every translation unit is compiled in parallel; the result goes to
``paper_2408_04343_gb300/_build/libsnp.so``.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsnp.so")
# The bounds-checked debug build (-DSNP_CHECK_BOUNDS): every kernel checks
# its data-dependent indices and reports an out-of-range one as an error
# instead of reading outside a buffer.  Built by build(check_bounds=True);
# the binding loads it when SNP_CHECK_BOUNDS=1 is set in the environment.
CHECK_DIR = os.path.join(HERE, "_build_check")
CHECK_LIB = os.path.join(CHECK_DIR, "libsnp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), check_bounds: bool = False) -> str:
    out_dir, lib = (CHECK_DIR, CHECK_LIB) if check_bounds else (OUT_DIR, LIB)
    if check_bounds:
        extra = tuple(extra) + ("-DSNP_CHECK_BOUNDS",)
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(HERE, "..", "include", "*.h"))
    objs, procs = [], []
    for src in sources():
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        objs.append(obj)
        if not force and not _stale(obj, [src] + headers):
            continue
        cmd = [cc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
               "-I", os.path.join(HERE, "..", "include"), "-c", src, "-o", obj, *extra]
        if src.endswith(".cu"):
            cmd[1:1] = ["-x", "cu"]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    if force or procs or not os.path.exists(lib):
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "shared",
                               "-Xlinker", "-rpath,$ORIGIN"])
        os.replace(tmp, lib)
    return lib



# The files one engine's step kernel is built and launched from: its
# translation unit, the device headers, the packer that lays out its inputs
# and the host code that launches it.  A DRAM-traffic record taken with ncu
# stays valid while these files are unchanged.
ENGINE_SOURCES = {
    "tiled": ["kernels_tiled.cu", "device_common.cuh", "kernels.h", "snp_internal.h", "system.h", "pack.cpp",
              "api.cu"],
    "launch": ["kernels_step.cu", "device_common.cuh", "kernels.h", "snp_internal.h", "system.h", "pack.cpp",
               "api.cu"],
}


def _digest(paths) -> str:
    import hashlib
    h = hashlib.sha256()
    for p in sorted(paths):
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def sources_hash() -> str:
    """Digest of every kernel and host source of libsnp."""
    return _digest(sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")))


def engine_sources_hash(engine: str) -> str:
    """Digest of the files one engine's step kernel depends on (ties an ncu
    traffic record to the code it was taken on)."""
    return _digest([os.path.join(CSRC, n) for n in ENGINE_SOURCES[engine]])


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
