"""Build libmdist.so (the CUDA enumerator + C-ABI) and libmdist_probe.so (measurement
probes that only the tests and the benchmark load) in-tree with nvcc for sm_103a.

Each translation unit is compiled in its own nvcc process (in parallel), then linked
into its shared library with the CUDA runtime linked statically.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
PROBE_SRC = os.path.join(HERE, "probe")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmdist.so")
PROBE_LIB = os.path.join(HERE, "libmdist_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def sources(d: str = CSRC) -> list[str]:
    return sorted(os.path.join(d, f) for f in os.listdir(d) if f.endswith((".cu", ".cpp")))


def _deps() -> list[str]:
    inc = os.path.join(os.path.dirname(HERE), "include")
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(PROBE_SRC, f) for f in os.listdir(PROBE_SRC)]
    files += [os.path.join(inc, f) for f in os.listdir(inc)]
    return files


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of libmdist.so."""
    newest = max(os.path.getmtime(f) for f in _deps() + [__file__])
    if (not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest and os.path.exists(PROBE_LIB) and
            os.path.getmtime(PROBE_LIB) >= newest):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    srcs = sources() + sources(PROBE_SRC)

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, os.path.basename(os.path.dirname(src)) + "_" + os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *os.environ.get("MDIST_NVCC_EXTRA", "").split(), "-c", src, "-o", obj]
        if verbose:
            cmd.append("-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, srcs))
    n_main = len(sources())
    for lib, part in ((LIB, objs[:n_main]), (PROBE_LIB, objs[n_main:])):
        tmp = lib + ".tmp"
        r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *part], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
