"""Builds libapm.so (the C-ABI library) in-tree for sm_103a with nvcc.

The translation units are compiled in parallel; the result lands in
paper_1410_0010_gb300/_build/libapm.so.  No CMake, no torch extension
machinery: plain nvcc, one -gencode.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libapm.so")
# the bounds-checked debug library (-DAPM_BOUNDS_CHECK), loaded with APM_LIB
BOUNDS_DIR = os.path.join(HERE, "_build_bounds")

# (source, object, extra flags): k_fft_col.cu is compiled once per precision
# and column pass, k_fft_fast.cu once per pass
SOURCES = [("apm_api.cu", "apm_api.o", []), ("k_green.cu", "k_green.o", []),
           ("k_deposit.cu", "k_deposit.o", []), ("k_fft_x.cu", "k_fft_x.o", []),
           ("k_field.cu", "k_field.o", []), ("k_evolve.cu", "k_evolve.o", []),
           ("apm_noalloc.cu", "apm_noalloc.o", []), ("k_order.cu", "k_order.o", [])] + [
    ("k_fft_col.cu", f"k_fft_col_{p}_{m}.o", [f"-DAPM_COL_FP64={1 if p == 'f64' else 0}", f"-DAPM_COL_MODE={m}"])
    for p in ("f32", "f64") for m in (0, 1, 2, 3)] + [
    ("k_fft_fast.cu", f"k_fft_fast_{m}.o", [f"-DAPM_FAST_MODE={m}"]) for m in (0, 1, 2, 3, 4, 5)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
          "--expt-relaxed-constexpr"]
# the deposit must round exactly like a plain IEEE evaluation: no contraction
PER_FILE = {"k_deposit.cu": ["-fmad=false"]}


def nvcc():
    return os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra=(), out_dir=OUT_DIR):
    """Compile the stale translation units and link libapm.so in `out_dir`.
    Extra nvcc flags come from `extra` and the APM_NVCC_FLAGS environment
    variable."""
    lib_path = os.path.join(out_dir, "libapm.so")
    os.makedirs(out_dir, exist_ok=True)
    extra = list(extra) + os.environ.get("APM_NVCC_FLAGS", "").split()
    headers = [os.path.join(CSRC, h) for h in sorted(os.listdir(CSRC)) if h.endswith(".cuh")]
    headers.append(os.path.join(INCLUDE, "apm.h"))
    objs, jobs = [], []
    for src, oname, flags in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(out_dir, oname)
        objs.append(obj)
        if force or _stale(obj, [path] + headers):
            cmd = [nvcc(), *ARCH, *COMMON, *PER_FILE.get(src, []), *flags, *extra, "-c", path, "-o", obj]
            jobs.append(cmd)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4) or 1) as ex:
        for out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out)
    if force or jobs or _stale(lib_path, objs):
        tmp = lib_path + ".tmp"
        run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, lib_path)
    return lib_path


def build_probe(force=False):
    """The compute-peak probe (csrc/peak_probe.cu), a standalone program that
    prints the measured FP32/FP64/INT32 and reduction rates as JSON; bench.py
    --probe-peaks runs it."""
    src = os.path.join(CSRC, "peak_probe.cu")
    exe = os.path.join(OUT_DIR, "peak_probe")
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or _stale(exe, [src]):
        r = subprocess.run([nvcc(), *ARCH, "-O3", "-std=c++17", src, "-o", exe + ".tmp"],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
        os.replace(exe + ".tmp", exe)
    return exe


def build_bounds_checked(force=False, verbose=False):
    """The debug library: every data- or hierarchy-dependent global index is
    tested before use (APM_BOUNDS_CHECK; apm_sync_status reports APM_E_BOUNDS)."""
    return build(force=force, verbose=verbose, extra=["-DAPM_BOUNDS_CHECK"], out_dir=BOUNDS_DIR)


if __name__ == "__main__":
    import sys
    if "--bounds-check" in sys.argv:
        print(build_bounds_checked(force="--force" in sys.argv, verbose=True))
    else:
        print(build(force="--force" in sys.argv, verbose=True,
                    extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
