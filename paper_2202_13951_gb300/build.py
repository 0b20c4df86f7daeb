"""Compile the CUDA library in-tree: paper_2202_13951_gb300/liborbg.so.

sm_103a only (``-gencode arch=compute_103a,code=sm_103a``), cudart linked
statically, translation units compiled in parallel.  ``python -m
paper_2202_13951_gb300.build`` or ``build()``.
"""
import hashlib
import os
import re
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJDIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liborbg.so")
SOURCES = ["orbg_plain.cu", "orbg_batched.cu", "orbg_noalloc.cu",
           "orbg_probe.cu", "orbg_fit.cu", "orbg_api.cpp", "orbg_serve.cpp",
           "orbg_tables.cpp"]
# the batched kernels: one object per (keys per lane, syndrome words) pair
INST = "orbg_batched_inst.cu"
INST_KW = [(k, w) for k in (1, 2, 4, 8) for w in (1, 2, 4)]
# the per-block fitted decoder: one object per keys per lane
FS_INST = "orbg_fitted_search_inst.cu"
FS_K = (1, 2, 4, 8)
HEADERS = ["orbg_internal.h", "orbg_decode_block.cuh", "orbg_batched.cuh", "orbg_heavy.cuh",
           "orbg_fit.cuh", "orbg_fitted_search.cuh", "orbg_regions.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return exe


STAMP = LIB + ".sha256"


def _digest(extra=()):
    """SHA-256 of every source, header and flag the library is built from,
    and of the compiler's path: the library is rebuilt whenever this
    changes (file times are not trusted: a copied tree keeps them)."""
    h = hashlib.sha256()
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS + [INST, FS_INST]]
    deps.append(os.path.join(ROOT, "include", "orbg.h"))
    deps.append(os.path.abspath(__file__))
    for d in deps:
        h.update(os.path.basename(d).encode())
        with open(d, "rb") as f:
            h.update(hashlib.sha256(f.read()).digest())
    h.update(repr(list(extra)).encode())
    h.update(nvcc().encode())
    return h.hexdigest()


_COMMENT = re.compile(rb"/\*.*?\*/|//[^\n]*", re.S)


def kernel_digest(names=None):
    """SHA-256 of device code (the CUDA sources and the headers they
    include, with their comments removed): all of it, or the files `names`
    of the source directory.  Profiler figures taken on one build stay
    valid while the kernels they cover are unchanged, whatever happens to
    the host-only C++ around them or to the comments."""
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        if names is not None and name not in names:
            continue
        if name.endswith((".cu", ".cuh")) or name == "orbg_internal.h":
            h.update(name.encode())
            with open(os.path.join(CSRC, name), "rb") as f:
                h.update(hashlib.sha256(_COMMENT.sub(b"", f.read())).digest())
    return h.hexdigest()


def _stale(digest):
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return True
    with open(STAMP) as f:
        return f.read().strip() != digest


def build(force=False, verbose=False, extra=()):
    digest = _digest(extra)
    if not force and not _stale(digest):
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I",
              os.path.join(ROOT, "include"), "-I", CSRC]
    procs = []
    objs = []
    # the largest instantiations first, so the slowest compiles start at once
    units = [(INST, "orbg_batched_k%dw%d.o" % (k, w),
              ["-DORBG_INST_K=%d" % k, "-DORBG_INST_W=%d" % w])
             for k, w in sorted(INST_KW, key=lambda kw: -kw[0] * kw[1])]
    units += [(FS_INST, "orbg_fitted_search_k%d.o" % k, ["-DORBG_FS_K=%d" % k])
              for k in sorted(FS_K, reverse=True)]
    units += [(s, s + ".o", []) for s in SOURCES]
    for s, o, defs in units:
        obj = os.path.join(OBJDIR, o)
        cmd = [cc, "-c", os.path.join(CSRC, s), "-o", obj] + common + defs
        if s.endswith(".cu"):
            cmd += ARCH + ["-lineinfo"] + list(extra)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = LIB + ".%d.tmp" % os.getpid()
    link = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-lpthread"]
    subprocess.check_call(link)
    os.replace(tmp, LIB)
    with open(STAMP + ".tmp", "w") as f:
        f.write(digest + "\n")
    os.replace(STAMP + ".tmp", STAMP)
    print("liborbg.so: compiled %d units for sm_103a" % len(units), file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else [])
    print(LIB)
