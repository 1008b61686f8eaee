"""In-tree build of libjet.so for sm_103a (nvcc only, no cmake).

Generates the closure header, compiles every translation unit in parallel
(one SIMT unit per compiled channel set) and links the shared library into
``paper_2606_29702_gb300/lib/libjet.so``.
"""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libjet.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def n_classes():
    sys.path.insert(0, CSRC)
    try:
        import gen_closures
        return len(gen_closures.CLASSES)
    finally:
        sys.path.pop(0)


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    return cmd, r.returncode, r.stdout


def build(verbose=False, jobs=None):
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    subprocess.check_call([sys.executable, os.path.join(CSRC, "gen_closures.py"),
                           os.path.join(CSRC, "jet_closures_gen.h")])
    cc = nvcc()
    units = []
    for name in ("jet_api.cu", "jet_reduce.cu", "jet_tc.cu", "jet_noalloc.cu"):
        units.append((os.path.join(CSRC, name), os.path.join(BUILD, name.replace(".cu", ".o")), []))
    for k in range(n_classes()):
        units.append((os.path.join(CSRC, "jet_simt_inst.cu"), os.path.join(BUILD, "jet_simt_%d.o" % k),
                      ["-DJET_CLASS_ID=%d" % k]))
        units.append((os.path.join(CSRC, "jet_tc_inst.cu"), os.path.join(BUILD, "jet_tc_%d.o" % k),
                      ["-DJET_CLASS_ID=%d" % k]))
    cmds = [[cc] + ARCH + FLAGS + extra + ["-c", src, "-o", obj] for src, obj, extra in units]
    jobs = jobs or max(1, min(len(cmds), os.cpu_count() or 1))
    failed = []
    with cf.ThreadPoolExecutor(jobs) as ex:
        for cmd, rc, out in ex.map(_run, cmds):
            if verbose or rc != 0:
                sys.stdout.write(" ".join(cmd) + "\n" + out)
            if rc != 0:
                failed.append(cmd[-1])
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(failed))
    link = [cc] + ARCH + ["-shared", "-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64", "-o", LIB] + [o for _, o, _ in units]
    cmd, rc, out = _run(link)
    if rc != 0:
        raise RuntimeError("link failed:\n" + out)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
