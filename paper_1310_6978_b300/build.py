"""Build libfbg.so in-tree: nvcc for sm_103a (device code) and the host C++.

Usage: python -m paper_1310_6978_b300.build [--force]
The device header fbg_device.cuh is also embedded as text (for NVRTC).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(ROOT, "_build")
SO = os.path.join(HERE, "libfbg.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-Wall", f"-I{os.path.join(ROOT, 'include')}", f"-I{CSRC}"]

SOURCES = ["parse.cpp", "ground.cpp", "lower.cpp", "emit.cpp", "jit.cpp", "api.cpp", "batch.cpp", "serve.cpp", "autotune.cpp",
           "cache.cpp",
           "interp.cu", "noalloc.cu", "peaks.cu"]


def _embed_header() -> str:
    """The device header as text, for NVRTC: fbg_device_header (fbg_device.cuh)."""
    parts = [("fbg_device_header", "fbg_device.cuh")]
    body = "// generated by build.py from the device headers\nnamespace fbg {\n"
    for sym, fn in parts:
        src = open(os.path.join(CSRC, fn)).read()
        body += f'extern const char {sym}[] = R"FBGSRC({src})FBGSRC";\n'
    body += "}\n"
    path = os.path.join(OUT, "fbg_device_header.cpp")
    if not os.path.exists(path) or open(path).read() != body:
        with open(path, "w") as f:
            f.write(body)
    return path


def _headers_mtime() -> float:
    m = 0.0
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            if f.endswith((".h", ".hpp", ".cuh")):
                m = max(m, os.path.getmtime(os.path.join(d, f)))
    return m


def _compile(src: str, force: bool, hdr_m: float) -> str:
    obj = os.path.join(OUT, os.path.basename(src) + ".o")
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_m):
        return obj
    cmd = [NVCC, *ARCH, *COMMON, "-c", src, "-o", obj]
    if src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if src.endswith(".cu"):
        with open(obj + ".ptxas.txt", "w") as f:
            f.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    hdr_m = _headers_mtime()
    srcs = [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    srcs.append(_embed_header())
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, force, hdr_m), srcs))
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(SO) or os.path.getmtime(SO) < newest:
        tmp = SO + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lnvrtc", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, SO)
    if verbose:
        print(SO)
    return SO


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
