"""Build ``libmact.so`` in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into one shared
library next to this file.  No fast-math: the kernels rely on IEEE division
and square root where they use them.  Rebuilds only when a source or header
is newer than the library (or when forced).
"""
import concurrent.futures as cf
import glob
import os
import re
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libmact.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmact.so")
    return cand


BATCH_INST = "k_batch_inst.cu"
LUT_INST = "k_lut_inst.cu"       # compiled once per interpolation method (0..3)
# cube-root forms of the batched kernels: (exact, Horner degree; 0 = FP64 polynomial)
BATCH_FORMS = [(1, 4), (0, 4), (0, 6), (0, 0)]


def batch_shapes():
    """The (threads, sub-blocks) launch shapes listed by MACT_BATCH_SHAPES."""
    src = open(os.path.join(CSRC, "convert_common.cuh")).read()
    m = re.search(r"#define MACT_BATCH_SHAPES\(X\)(.*)", src)
    if not m:
        raise RuntimeError("MACT_BATCH_SHAPES not found in convert_common.cuh")
    return [(int(t), int(b)) for t, b in re.findall(r"X\((\d+),\s*(\d+)\)", m.group(1))]


def sources():
    return sorted(p for p in glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp"))
                  if os.path.basename(p) not in (BATCH_INST, LUT_INST))


def units():
    """(source, object name, extra defines) of every object of the library:
    one per source file, k_lut_inst.cu once per interpolation method and
    k_batch_inst.cu once per (form, shape) pair."""
    out = [(src, os.path.basename(src) + ".o", []) for src in sources()]
    for m in range(4):
        out.append((os.path.join(CSRC, LUT_INST), "k_lut_m%d.o" % m, ["-DMACT_LUT_METHOD_ID=%d" % m]))
    inst = os.path.join(CSRC, BATCH_INST)
    for exact, rdeg in BATCH_FORMS:
        for t, sb in batch_shapes():
            out.append((inst, "k_batch_e%d_r%d_t%d_s%d.o" % (exact, rdeg, t, sb),
                        ["-DMACT_FORM_EXACT=%d" % exact, "-DMACT_FORM_RDEG=%d" % rdeg,
                         "-DMACT_SHAPE_T=%d" % t, "-DMACT_SHAPE_S=%d" % sb]))
    return out


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + [os.path.join(CSRC, BATCH_INST), os.path.join(CSRC, LUT_INST)] + \
        glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force=False, verbose=False, ptxas_v=False):
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                    "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]
    if ptxas_v:
        flags += ["-Xptxas", "-v"]

    def compile_one(unit):
        src, name, defs = unit
        obj = os.path.join(BUILD, name)
        cmd = [cc, "-c", src, "-o", obj] + flags + defs
        if src.endswith(".cpp"):
            cmd = [cc, "-x", "cu", "-c", src, "-o", obj] + flags + defs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s %s:\n%s\n%s" % (src, " ".join(defs), r.stdout, r.stderr))
        return obj, r.stderr

    # longest units first (the LUT and batched kernels), so the pool ends together
    todo = sorted(units(), key=lambda u: (0 if ("k_lut" in u[1] or "k_batch" in u[1]) else 1, u[1]))
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 2)) as ex:
        results = list(ex.map(compile_one, todo))
    if verbose or ptxas_v:
        for obj, err in results:
            if err.strip():
                print(err, file=sys.stderr)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc, "-shared", "-o", tmp] + [o for o, _ in results] + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv))
