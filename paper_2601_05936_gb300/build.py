"""Build the lsb CUDA library (liblsb.so) in-tree for sm_103a with nvcc.

Five translation units are compiled in parallel and linked into
paper_2601_05936_gb300/_lib/liblsb.so.  Nothing here runs on the GPU.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liblsb.so")
SOURCES = ["lsb_lb.cu", "lsb_ls.cu", "lsb_adj.cu", "lsb_adj_ls.cu", "lsb_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-static-global-template-stub=false",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "lsb.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra=(), out=None):
    """Compile liblsb.so if any source is newer than it; returns the path.

    ``extra`` adds nvcc flags and ``out`` writes the library elsewhere (for
    comparing compile-time variants)."""
    if out is None and not force and not _stale():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    exe = nvcc()
    odir = LIBDIR if out is None else os.path.dirname(os.path.abspath(out))
    os.makedirs(odir, exist_ok=True)
    tag = "" if out is None else "_" + os.path.basename(out).replace(".so", "")
    objs = [os.path.join(odir, s.replace(".cu", tag + ".o")) for s in SOURCES]

    def comp(src_obj):
        src, obj = src_obj
        cmd = [exe, *flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        list(ex.map(comp, zip(SOURCES, objs)))
    target = LIB if out is None else out
    tmp = target + ".tmp"
    # every symbol resolved at link time: a missing definition fails the build, not the load
    r = subprocess.run([exe, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-Xlinker", "--no-undefined"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, target)
    return target


if __name__ == "__main__":
    print(build(force=True, verbose=True))
