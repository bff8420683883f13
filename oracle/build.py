"""Compile the CPU oracle (test infrastructure) into oracle/_build/libmporacle.so.

The oracle is plain C compiled with -ffp-contract=off so that no a*b+c is
fused behind the algorithms' back; OpenMP only splits rows of C between
threads.  Run as ``python -m oracle.build`` or call ``build()``.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mp_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmporacle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
          "-fPIC", "-shared", "-fopenmp", "-Wall"]


def build(force=False, src=SRC, out=LIB, extra=()):
    """Compile ``src`` to ``out`` unless it is up to date; return the path."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    hdr = os.path.join(HERE, "mp_oracle.h")
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", *CFLAGS, "-I", HERE, *extra, "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
