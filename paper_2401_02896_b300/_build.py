"""Build libsphdvr.so in-tree with nvcc for sm_103a (B300).

The shared library lands in ``paper_2401_02896_b300/lib/`` so that it travels
with the source tree; no JIT cache is involved.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libsphdvr.so")
INCLUDE = os.path.join(ROOT, "include")

CU = ["api.cu", "sort.cu", "dataset.cu", "frame.cu", "server.cu", "static_scratch.cu", "plan.cu", "scatter.cu",
      "quanta.cu", "peak.cu", "autotune.cu"]
# the render kernels: one source compiled once per polynomial degree
DEGREES = range(1, 7)
RENDER_INST = "render_inst.cu"
CPP = ["lutgen.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _sources():
    return [os.path.join(CSRC, f) for f in CU + CPP + [RENDER_INST]] + [
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))
    ] + [os.path.join(INCLUDE, "sphdvr.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force=False, verbose=False, jobs=None):
    if not force and up_to_date():
        return LIB
    os.makedirs(os.path.join(LIBDIR, "obj"), exist_ok=True)
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-I", CSRC, "-Xcompiler", "-fPIC", "-Xcompiler", "-fopenmp"]
    cmds, objs = [], []
    for f in CU:
        o = os.path.join(LIBDIR, "obj", f + ".o")
        cmds.append([NVCC] + ARCH + common + ["-lineinfo", "-Xptxas", "-v" if verbose else "-O3", "-c",
                                               os.path.join(CSRC, f), "-o", o])
        objs.append(o)
    for d in DEGREES:
        o = os.path.join(LIBDIR, "obj", "render_d%d.o" % d)
        cmds.append([NVCC] + ARCH + common + ["-DSPHDVR_D=%d" % d, "-lineinfo", "-Xptxas", "-v" if verbose else "-O3",
                                               "-c", os.path.join(CSRC, RENDER_INST), "-o", o])
        objs.append(o)
    for f in CPP:
        o = os.path.join(LIBDIR, "obj", f + ".o")
        cmds.append(["g++", "-O2", "-std=c++17", "-fPIC", "-fopenmp", "-I", INCLUDE, "-I", CSRC,
                     "-I", "/usr/local/cuda/include", "-c", os.path.join(CSRC, f), "-o", o])
        objs.append(o)
    procs = []
    for c in cmds:
        procs.append((c, subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = False
    for c, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed = True
            sys.stderr.write("FAILED: %s\n" % " ".join(c))
    if failed:
        raise RuntimeError("libsphdvr build failed")
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-Xcompiler", "-fopenmp", "-lgomp"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
