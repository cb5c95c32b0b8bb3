"""Build libpotts_lr.so for sm_103a in-tree (paper_1308_5426_gb300/_build/).

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library with a plain C ABI (include/potts_lr.h).
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libpotts_lr.so")
SOURCES = ["api.cu", "sweep.cu", "sweep_rf_a.cu", "sweep_rf_b.cu", "sweep_rf_c.cu", "sweep_rf_d.cu", "sweep_rf_e.cu",
           "sweep_rf_f.cu", "sweep_rf_g.cu", "sweep_rf_h.cu", "aux_kernels.cu", "rebuild_tc.cu", "probe.cu",
           "measure_static.cu", "sweep_sched.cu", "sweep_direct.cu", "sweep_rf_dispatch.cu", "sweep_cluster.cu",
           "sweep_rfx_a.cu", "sweep_rfx_b.cu", "sweep_rfx_c.cu", "sweep_rfx_d.cu", "sweep_rfx_e.cu", "sweep_rfx_f.cu",
           "sweep_rfc_f.cu", "sweep_rfc_fq.cu", "sweep_rfc_x.cu", "jstar.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"] + ARCH


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "potts_lr.h"))
    return files


def _compile(src, extra):
    obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
    cmd = [_nvcc()] + NVCC_FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile (if any source is newer than the library) and return its path."""
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(f) <= t for f in _deps()):
            return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra)), SOURCES))
    if verbose:
        for _, err in results:
            if err.strip():
                print(err, file=sys.stderr)
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(force=True, verbose=v, extra=["-Xptxas", "-v"] if v else []))
