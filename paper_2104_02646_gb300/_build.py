"""Build the CUDA library libgradsim.so in-tree for sm_103a (plain nvcc).

Translation units compile in parallel; the result lands in
paper_2104_02646_gb300/_lib/libgradsim.so.  The checked variant
libgradsim_check.so (the step kernels compiled with -DGS_CHECK: every table
index is range-checked on the device, see gs_kernels.cu) is built beside it
from the same objects plus a checked copy of the kernels.  Rebuilds only
when a source or header is newer than the library.
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libgradsim.so")
LIB_CHECKED = os.path.join(OUT, "libgradsim_check.so")
CHECKED_TU = "gs_kernels.cu"  # the translation unit whose code GS_CHECK changes
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-I", CSRC, "-I", INCLUDE]


def nvcc():
    for c in (os.environ.get("CUDA_HOME", "") + "/bin/nvcc", "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(f) > t for f in deps)


def _link(objs, lib):
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    """Build libgradsim.so and (with ``checked``) libgradsim_check.so; returns
    the path of libgradsim.so."""
    need_main = force or _stale(LIB)
    need_checked = checked and (force or _stale(LIB_CHECKED))
    if not need_main and not need_checked:
        return LIB
    os.makedirs(OUT, exist_ok=True)

    def compile_one(job):
        src, defs, suffix = job
        obj = os.path.join(OUT, os.path.basename(src) + suffix + ".o")
        cmd = [nvcc()] + ARCH + FLAGS + defs + ["-c", src, "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    jobs = [(src, [], "") for src in sources()]
    if need_checked:
        jobs.append((os.path.join(CSRC, CHECKED_TU), ["-DGS_CHECK"], ".check"))
    objs = {}
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 2)) as ex:
        for job, (obj, err) in zip(jobs, ex.map(compile_one, jobs)):
            objs[(os.path.basename(job[0]), job[2])] = obj
            if verbose and err:
                sys.stderr.write(err)
    plain = [objs[(os.path.basename(s), "")] for s in sources()]
    _link(plain, LIB)
    if need_checked:
        _link([objs[(CHECKED_TU, ".check")] if os.path.basename(o) == CHECKED_TU + ".o" else o for o in plain],
              LIB_CHECKED)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
