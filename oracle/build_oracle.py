"""Compile the oracle's C part (csr_omp.c, the OpenMP CSR product) with gcc.

TEST INFRASTRUCTURE ONLY: the library never uses it.  The shared object goes
to oracle/_lib/ (git-ignored); nothing is compiled when it is newer than its
source.  Portable flags only (the same source builds on x86_64 and aarch64).
"""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csr_omp.c")
OUT = os.path.join(HERE, "_lib", "liboracle_csr.so")


def build():
    """Build the oracle's shared object if needed; returns its path, or None without gcc."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        return None
    if os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    tmp = OUT + f".{os.getpid()}.tmp"
    p = subprocess.run([cc, "-O2", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp], capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"gcc failed on csr_omp.c:\n{p.stdout}\n{p.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build())
