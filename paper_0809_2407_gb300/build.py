"""Builds libtsqr.so in-tree for sm_103a (GB300) with nvcc.

The translation units compile in parallel, then link into ``paper_0809_2407_gb300/_build``.
Re-running is cheap: nothing is rebuilt unless a source or header is newer than the library.
"""
import concurrent.futures
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libtsqr.so")
# measurement tooling for the benchmark (FMA-pipe peaks), kept out of the TSQR library
PROBE_SRC = os.path.join(CSRC, "probe", "fma_probe.cu")
PROBE_LIB = os.path.join(OUT_DIR, "libtsqr_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(ROOT, "include", "tsqr.h"), os.path.abspath(__file__)]


def _stale():
    if not os.path.exists(LIB) or not os.path.exists(PROBE_LIB):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(PROBE_LIB))
    return any(os.path.getmtime(p) > t for p in _deps() + [PROBE_SRC])


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles and links libtsqr.so if needed; returns its path.  Raises on compiler errors."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
        cmd = [NVCC] + FLAGS + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    def compile_probe():
        tmp = PROBE_LIB + ".tmp.%d" % os.getpid()
        r = subprocess.run([NVCC] + FLAGS + ["-shared", "-o", tmp, PROBE_SRC], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (PROBE_SRC, r.stdout, r.stderr))
        os.replace(tmp, PROBE_LIB)

    with concurrent.futures.ThreadPoolExecutor(max_workers=8) as ex:
        probe = ex.submit(compile_probe)
        objs = list(ex.map(compile_one, _sources()))
        probe.result()
    tmp = LIB + ".tmp.%d" % os.getpid()
    r = subprocess.run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
