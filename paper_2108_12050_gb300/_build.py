"""Builds libmhfd.so in-tree (nvcc, sm_103a) and warms the fused-kernel cache.

    python -m paper_2108_12050_gb300._build            # library only
    python -m paper_2108_12050_gb300._build --warm     # + precompile standard ladders

The fused detection kernel is compiled at run time by NVRTC for each ladder;
``warm()`` compiles the ladders used by the tests and the benchmark ahead of
time, in parallel processes, into the on-disk cache next to the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import multiprocessing as mp
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(os.path.dirname(PKG), "_build")
LIB = os.path.join(PKG, "libmhfd.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cpp", "jit.cpp", "stretch.cu", "post.cu", "plain.cu", "probe.cu", "noalloc.cu",
           "soft.cu"]
EMBED = ["mhfd_types.h", "detect_kernel.cuh"]


def _raw_literal(name, text):
    # split into chunks below the compilers' string-literal limits
    parts = []
    step = 12000
    for i in range(0, len(text), step):
        parts.append('R"MHFDSRC(' + text[i:i + step] + ')MHFDSRC"')
    return "static const char *%s =\n%s;\n" % (name, "\n".join(parts))


def write_embed():
    types = open(os.path.join(CSRC, "mhfd_types.h")).read()
    kern = open(os.path.join(CSRC, "detect_kernel.cuh")).read()
    body = ("// generated by _build.py from mhfd_types.h and detect_kernel.cuh\n" +
            _raw_literal("kTypesSrc", types) + _raw_literal("kKernelSrc", kern))
    path = os.path.join(CSRC, "kernel_src.inc")
    if not os.path.exists(path) or open(path).read() != body:
        with open(path, "w") as f:
            f.write(body)


def _inputs_digest():
    h = hashlib.sha1()
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cpp", ".h", ".cuh", ".inc")):
            h.update(f.encode())
            h.update(open(os.path.join(CSRC, f), "rb").read())
    h.update(open(os.path.join(os.path.dirname(PKG), "include", "mhfd.h"), "rb").read())
    h.update(" ".join(ARCH).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def _compile(src):
    obj = os.path.join(BUILD, src + ".o")
    cmd = [NVCC, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
           "-I" + os.path.join(os.path.dirname(PKG), "include"), "-c",
           os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    return obj


def build_lib(force=False):
    """Compile and link libmhfd.so; a no-op when sources are unchanged."""
    write_embed()
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "libmhfd.stamp")
    digest = _inputs_digest()
    if (not force and os.path.exists(LIB) and os.path.exists(stamp)
            and open(stamp).read() == digest):
        return LIB
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs,
           "-L" + os.path.join(CUDA, "lib64"), "-L" + os.path.join(CUDA, "lib64", "stubs"),
           "-lnvrtc", "-Xlinker", "-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


# ladders compiled ahead of time: (n, t_min, t_max, nms, store); store 1 is
# the stack-storing variant, 2 the soft-score forward, 3 the soft-score
# adjoint's single-level blurs
STANDARD_VARIANTS = [
    (10, 1.0, 10.0, 0, 0), (10, 1.0, 10.0, 0, 1),     # 512^2 uint8 workload
    (10, 1.0, 10.0, 1, 0), (10, 1.0, 10.0, 1, 1),
    (16, 1.0, 12.0, 0, 0), (16, 1.0, 12.0, 0, 1),     # 4096^2 uint16 workload
    (16, 1.0, 12.0, 1, 0), (16, 1.0, 12.0, 0, 2), (16, 1.0, 12.0, 0, 3),
    (4, 1.0, 4.0, 0, 0), (4, 1.0, 4.0, 0, 1),         # small ladders of the tests
    (4, 1.0, 4.0, 1, 0), (4, 1.0, 4.0, 1, 1), (4, 1.0, 4.0, 0, 2), (4, 1.0, 4.0, 0, 3),
]


def _precompile_one(args):
    n, tmin, tmax, nms, store = args[:5]
    shape = args[5] if len(args) > 5 else None
    response = args[6] if len(args) > 6 else "dog"
    tc = args[7] if len(args) > 7 else True
    sys.path.insert(0, os.path.dirname(PKG))
    from paper_2108_12050_gb300 import _native
    return _native.precompile(n=n, t_min=tmin, t_max=tmax, nms=nms, store=store,
                              tile_shape=shape, response=response, tensor_cores=tc)


def _tuned_variants():
    """Variants the autotuner recorded (tuned_tiles.json), all GPU models."""
    import json
    import re
    path = os.path.join(PKG, "tuned_tiles.json")
    out = []
    try:
        tab = json.load(open(path))
    except Exception:
        return out
    for key, ent in tab.items():
        m = re.match(r"n(\d+)_t([0-9.e+-]+)-([0-9.e+-]+)_(paper|local26)_tr4(_log)?(_tc)?$", key)
        if not m:
            continue
        for best in ent.values():
            shape = best.get("shape")
            if shape and len(shape) in (5, 6):
                nms = 0 if m.group(4) == "paper" else 1
                log = m.group(5) is not None
                # (tensor-core shapes are the vertical-pass kernel's: 2)
                tc = 2 if m.group(6) is not None else False
                # an FFMA shape of the paper rule serves detectors built with
                # tensor_cores=False; a vertical-pass tensor-core shape, with
                # its companion, detectors built with tensor_cores=2 (and the
                # default ones of the LoG response and of 26-neighbour ladders
                # beyond 16 layers)
                stores = (0, 1) if (nms == 1 or log) else (0, 1, 2)
                for store in stores:
                    out.append((int(m.group(1)), float(m.group(2)), float(m.group(3)), nms,
                                store, tuple(int(v) for v in shape), "log" if log else "dog",
                                tc))
    return out


def warm(variants=None, workers=None):
    """Precompile fused-kernel variants into the cache (CPU only)."""
    build_lib()
    variants = list(variants or (STANDARD_VARIANTS + _tuned_variants()))
    workers = workers or min(len(variants), os.cpu_count() or 4)
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        return list(ex.map(_precompile_one, variants))


if __name__ == "__main__":
    build_lib(force="--force" in sys.argv)
    if "--warm" in sys.argv:
        print(warm())
    print(LIB)
