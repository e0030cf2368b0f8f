"""Builds libperm.so in-tree: every CUDA/C++ source of csrc/ compiled for
sm_103a by nvcc (in parallel), linked with NVRTC and the static CUDA runtime.

    python -m paper_2501_15126_gb300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libperm.so")

SOURCES = ["host.cpp", "api.cpp", "codegen.cpp", "batch.cpp", "tune.cpp", "server.cpp", "generic.cu",
           "generic_f64.cu", "generic_dd.cu", "generic_r64.cu", "generic_r96.cu", "generic_r128.cu", "generic_r160.cu",
           "generic_r192.cu", "microbench.cu", "noalloc.cu", "checkpoint.cpp", "xshared.cu"]
EMBED = ["core.cuh", "devmat.h"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _embedded_source() -> str:
    parts = ["// generated by build.py: device headers handed to NVRTC\n"]
    for name in EMBED:
        text = open(os.path.join(CSRC, name)).read()
        sym = "perm_embedded_" + name.replace(".", "_")
        parts.append('extern const char *%s;\nconst char *%s = R"PERMSRC(%s)PERMSRC";\n' % (sym, sym, text))
    return "".join(parts)


def _digest() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        h.update(name.encode())
        h.update(open(os.path.join(CSRC, name), "rb").read())
    h.update(open(os.path.join(INCLUDE, "perm.h"), "rb").read())
    h.update(open(os.path.abspath(__file__), "rb").read())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    digest = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == digest:
        return LIB
    emb = os.path.join(BUILD, "embedded.cpp")
    with open(emb, "w") as f:
        f.write(_embedded_source())
    common = [nvcc(), ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
              "-I", INCLUDE, "-I", CSRC, "-c"]
    jobs = []
    for src in SOURCES + [emb]:
        path = src if os.path.isabs(src) else os.path.join(CSRC, src)
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        jobs.append((common + [path, "-o", obj], obj))
    objs = []
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        futs = {ex.submit(subprocess.run, cmd, capture_output=True, text=True): (cmd, obj) for cmd, obj in jobs}
        for fut in cf.as_completed(futs):
            cmd, obj = futs[fut]
            r = fut.result()
            if verbose and (r.stdout or r.stderr):
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
            objs.append(obj)
    tmp = LIB + ".tmp.%d" % os.getpid()
    link = [nvcc(), ARCH, "-shared", "-o", tmp] + sorted(objs) + [
        "-cudart", "static", "-lnvrtc", "-ldl", "-lpthread", "-lrt",
        "-Xlinker", "-rpath", "-Xlinker", "/usr/local/cuda/lib64"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s%s" % (" ".join(link), r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
