"""Compile the oracle's C core into oracle/_build/liboracle.so.

Test infrastructure only: the product library never links or loads it.
Flags keep every floating-point operation rounded as written
(-ffp-contract=off, no fast-math).
"""
import os
import shutil
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "apm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "liboracle.so")


def _openmp_ok(cc):
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        with open(src, "w") as f:
            f.write("#include <omp.h>\nint main(void){return omp_get_max_threads() > 0 ? 0 : 1;}\n")
        r = subprocess.run([cc, "-fopenmp", src, "-o", os.path.join(d, "t")],
                           capture_output=True)
        return r.returncode == 0


def build(force=False):
    """Build liboracle.so if missing or older than its source; return its path."""
    if (not force and os.path.exists(OUT)
            and os.path.getmtime(OUT) >= os.path.getmtime(SRC)):
        return OUT
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = os.environ.get("CC") or shutil.which("gcc") or "cc"
    flags = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]
    if _openmp_ok(cc):
        flags.append("-fopenmp")
    tmp = OUT + ".tmp"
    subprocess.run([cc, *flags, SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True))
