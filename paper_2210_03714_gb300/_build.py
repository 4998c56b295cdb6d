"""In-tree build of libfm.so (CUDA for sm_103a) with nvcc, one process per
translation unit so the build stays short on a many-core host."""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "lib", "libfm.so")

CU = ["fm_api.cu", "fm_launch.cu", "fm_inst_real.cu", "fm_inst_cplx.cu", "fm_grid.cu", "fm_bgrid.cu",
      "fm_trid.cu", "fm_band.cu", "fm_team.cu"]
CPP = ["fm_coeffs.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INC]


def _nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _sources():
    srcs = [os.path.join(CSRC, f) for f in CU + CPP if os.path.exists(os.path.join(CSRC, f))]
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(INC, "fm.h"))
    return srcs, hdrs


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    srcs, hdrs = _sources()
    return all(os.path.getmtime(f) <= t for f in srcs + hdrs + [__file__])


def build(force=False, verbose=False):
    """Compile every translation unit in parallel and link lib/libfm.so."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    srcs, _ = _sources()
    procs = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        objs.append(o)
        if s.endswith(".cu"):
            cmd = [_nvcc()] + ARCH + NVFLAGS + ["-c", s, "-o", o]
        else:
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-I", INC, "-c", s, "-o", o]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for s, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((s, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        msg = "\n".join("%s:\n%s" % (s, o[-4000:]) for s, o in failed)
        raise RuntimeError("libfm build failed:\n" + msg)
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call([_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
