"""Build libht (the CUDA library behind include/ht.h) in-tree for sm_103a.

Each .cu file under csrc/ is compiled in parallel with nvcc, then linked into
paper_1309_6275_gb300/_build/libht.so.  The benchmark's roofline probe
(probe/, include/ht_probe.h) is a separate library, _build/libht_probe.so.
Rebuilds only when a source is newer than the library (or when forced).
"""
import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libht.so")
PROBE_SRC = os.path.join(HERE, "probe", "probe.cu")
PROBE_LIB = os.path.join(BUILD, "libht_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(os.path.dirname(HERE), "include", "*.h")) + [__file__]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force=False, verbose=False, ptxas_info=False):
    """Compile libht.so if needed; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose or ptxas_info:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max(1, len(sources()))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def build_probe(force=False):
    """Compile the roofline probe library (benchmark only); returns its path."""
    deps = [PROBE_SRC, os.path.join(os.path.dirname(HERE), "include", "ht_probe.h"),
            os.path.join(os.path.dirname(HERE), "include", "ht.h"), __file__]
    if (not force and os.path.exists(PROBE_LIB) and
            all(os.path.getmtime(p) <= os.path.getmtime(PROBE_LIB) for p in deps)):
        return PROBE_LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = PROBE_LIB + f".tmp{os.getpid()}"
    cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, "-shared", "-o", tmp, PROBE_SRC, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {PROBE_SRC}:\n{r.stderr}")
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
