"""Build the CUDA library libsllbm.so in-tree for sm_103a (nvcc, no cmake).

Each translation unit is compiled in parallel; the shared object lands next
to this file.  checked=True builds the bounds-checked debug variant
libsllbm_checked.so (-DSLLBM_CHECKED: every index a step kernel takes from a
record table is range-checked into the device status word) from the same
sources into its own object folder.
Usage: python -m paper_2412_09051_gb300.build [--jobs N] [--checked]
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libsllbm.so")
BUILD = os.path.join(HERE, "_build")
OUT_CHECKED = os.path.join(HERE, "libsllbm_checked.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-I", os.path.join(HERE, "..", "include")]
SOURCES = ["capi.cu", "setup.cu", "util.cu", "step_f32.cu", "step_f32_3d.cu", "step_f64.cu", "step_p4.cu",
           "step_p4_f64.cu", "host_geometry.cpp", "mlp_train.cu", "stats.cu", "step_rowcopy.cu", "step_tmem.cu",
           "step_tmem2.cu", "generic.cu"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _compile(src, verbose_ptxas=False, checked=False):
    obj = os.path.join(BUILD_CHECKED if checked else BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + ARCH + FLAGS + (["-DSLLBM_CHECKED"] if checked else [])
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj, r.stderr


def _stale(out):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "sllbm.h")]
    return any(os.path.getmtime(f) > t for f in files if os.path.isfile(f))


def build(force=False, jobs=None, verbose_ptxas=False, checked=False):
    out = OUT_CHECKED if checked else OUT
    if not force and not _stale(out):
        return out
    os.makedirs(BUILD_CHECKED if checked else BUILD, exist_ok=True)
    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    logs = []
    with cf.ThreadPoolExecutor(jobs) as ex:
        futs = [ex.submit(_compile, s, verbose_ptxas, checked) for s in SOURCES]
        objs = []
        for f in futs:
            o, log = f.result()
            objs.append(o)
            logs.append(log)
    tmp = out + ".tmp"
    cmd = [_nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr)
    os.replace(tmp, out)
    if verbose_ptxas:
        sys.stderr.write("".join(logs))
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--ptxas" in sys.argv, checked="--checked" in sys.argv))
