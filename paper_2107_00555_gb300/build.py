"""Builds the dcp shared library in-tree (``paper_2107_00555_gb300/_lib/libdcp.so``).

Host sources (graph IR, fusion passes, code generator, NVRTC driver, runtime,
C ABI) are compiled with g++; CUDA sources with nvcc for sm_103a only.  The
kernel skeletons under ``csrc/kernels`` are embedded into the library as
strings and specialised / compiled for sm_103a by NVRTC when a graph is
fused.  The build needs no GPU and takes a few seconds.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
KDIR = os.path.join(CSRC, "kernels")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libdcp.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

EMBED = [("dcp_device.cuh", "device_header_source"),
         ("k_map.cuh", "kernel_map_source"),
         ("k_stencil2d.cuh", "kernel_stencil2d_source"),
         ("k_stencil3d.cuh", "kernel_stencil3d_source"),
         ("k_stencil2d_stream.cuh", "kernel_stream_source"),
         ("k_axis.cuh", "kernel_axis_source"),
         ("k_math64.cuh", "kernel_math64_source"),
         ("k_stencil_adj.cuh", "kernel_adj_source"),
         ("k_stencil2d_coop.cuh", "kernel_coop_source")]


def _embed_source() -> str:
    out = ["// generated by build.py: kernel skeletons embedded for NVRTC",
           '#include "dcp_internal.h"', "namespace dcp {"]
    for fname, fn in EMBED:
        path = os.path.join(KDIR, fname)
        if not os.path.exists(path):
            out.append('const char* %s() { return ""; }' % fn)
            continue
        text = open(path).read()
        # split into chunks below the compilers' string-literal limits
        chunks = [text[i:i + 12000] for i in range(0, len(text), 12000)]
        out.append("const char* %s() {" % fn)
        out.append("  static const char* s =")
        for c in chunks:
            out.append('    R"DCPSRC(%s)DCPSRC"' % c)
        out.append("  ;\n  return s;\n}")
    out.append("}  // namespace dcp")
    return "\n".join(out) + "\n"


def _sources():
    cpp = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    return cpp, cu


def _stamp(paths):
    h = hashlib.sha1()
    for p in sorted(paths):
        h.update(p.encode())
        h.update(open(p, "rb").read())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libdcp.so if any source changed; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cpp, cu = _sources()
    kernels = sorted(glob.glob(os.path.join(KDIR, "*.cuh")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.h"))) + [os.path.join(ROOT, "include", "dcp.h")]
    stamp = _stamp(cpp + cu + kernels + headers + [__file__])
    stamp_file = os.path.join(BUILD, "stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file) and \
            open(stamp_file).read() == stamp:
        return LIB
    embed = os.path.join(BUILD, "kernels_embed.cpp")
    with open(embed, "w") as f:
        f.write(_embed_source())
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", os.path.join(CUDA, "include")]
    jobs = []
    objs = []
    for src in cpp + [embed]:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-Wall", "-Wno-unused-function",
                     "-c", src, "-o", obj] + inc)
    for src in cu:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        jobs.append([NVCC] + ARCH + ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
                                    "-c", src, "-o", obj] + inc)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        return r

    with cf.ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        list(ex.map(run, jobs))
    tmp = LIB + ".tmp%d" % os.getpid()
    run(["g++", "-shared", "-o", tmp] + objs +
        ["-L", os.path.join(CUDA, "lib64"),
         "-Wl,-rpath," + os.path.join(CUDA, "lib64"),
         "-lnvrtc", "-lcudart", "-lpthread"])
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
