"""Build the device library liblst.so for sm_103a (in-tree, under _build/)."""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liblst.so")
SOURCES = ["k_chain.cu", "k_pixel_clean.cu", "k_mlp.cu", "lst_api.cu", "lst_mlp_api.cu", "lst_static.cu", "lst_peaks.cu"]
HEADERS = ["lst_device.cuh", "lst_kernels.cuh", "lst_warp.cuh", "lst_mlp.cuh", "lst_pdl.cuh", "lst_ff.cuh"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def _newest_input():
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(os.path.dirname(HERE), "include", "lst.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _compile(src):
    obj = os.path.join(OUT, src.replace(".cu", ".o"))
    log = obj + ".log"
    cmd = [NVCC] + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    with open(log, "w") as f:
        f.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr[-4000:]}")
    return obj


def build(force=False, verbose=False):
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([NVCC, "-shared", "-o", tmp] + objs + ["-lcudart"])
    os.replace(tmp, LIB)
    if verbose:
        for s in SOURCES:
            with open(os.path.join(OUT, s.replace(".cu", ".o.log"))) as f:
                sys.stdout.write(f.read())
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
