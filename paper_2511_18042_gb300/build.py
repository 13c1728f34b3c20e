"""Build the CUDA library in-tree (nvcc, sm_103a only)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libcgflow.so")
# FMA-throughput probe of the benchmark's arithmetic roofline (own library)
PROBE = os.path.join(OUT_DIR, "libcgprobe.so")

COMMON = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
          "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]
# FP64 parity units: no contraction of a*b+c on device or host.  The sweep is
# compiled once per (form, dimension), in parallel: FP64 without contraction,
# FP64 with fused multiply-add, FP32 (mixed form) with contraction.
FP64 = ["-fmad=false", "-Xcompiler", "-ffp-contract=off"]
UNITS = [("cg_api.cu", "cg_api.o", FP64)]
for _nd in (1, 2, 3):
    UNITS.append(("cg_sweep_inst.cu", "cg_sweep_f64_%d.o" % _nd,
                  FP64 + ["-DCGK_SWEEP_ND=%d" % _nd, "-DCGK_SWEEP_UNIT=0"]))
    UNITS.append(("cg_sweep_inst.cu", "cg_sweep_f64c_%d.o" % _nd,
                  ["-fmad=true", "-DCGK_SWEEP_ND=%d" % _nd, "-DCGK_SWEEP_UNIT=1"]))
    UNITS.append(("cg_sweep_inst.cu", "cg_sweep_f32_%d.o" % _nd,
                  ["-fmad=true", "-prec-div=false", "-prec-sqrt=false", "-DCGK_SWEEP_ND=%d" % _nd,
                   "-DCGK_SWEEP_UNIT=2"]))
NVCC_FLAGS = COMMON + FP64


def _sources_mtime():
    t = 0.0
    for d in (SRC, os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            t = max(t, os.path.getmtime(os.path.join(d, f)))
    return t


def build(force=False, verbose=False):
    if not force and os.path.exists(LIB) and os.path.exists(PROBE) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    objs, procs = [], []
    for src, oname, flags in UNITS:
        obj = os.path.join(OUT_DIR, oname)
        cmd = ["nvcc"] + COMMON + flags + ["-c", "-o", obj, os.path.join(SRC, src)]
        if verbose:
            print(" ".join(cmd))
        procs.append(subprocess.Popen(cmd))
        objs.append(obj)
    pcmd = ["nvcc"] + COMMON + ["-shared", "-o", PROBE + ".tmp%d" % os.getpid(), os.path.join(SRC, "cg_probe.cu")]
    if verbose:
        print(" ".join(pcmd))
    procs.append(subprocess.Popen(pcmd))
    for p in procs:
        if p.wait() != 0:
            raise subprocess.CalledProcessError(p.returncode, "nvcc")
    os.replace(PROBE + ".tmp%d" % os.getpid(), PROBE)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp] + objs
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
