"""Build the FP64 CPU oracle library (test infrastructure only).

Compiles ``mdpd_oracle.c`` with the host C compiler into ``libmdpd_oracle.so``
beside it.  ``-ffp-contract=off`` keeps every ``a*b + c`` rounded twice, as
written; OpenMP is used when the compiler supports it (the oracle gathers per
particle, so its results do not depend on the thread count).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mdpd_oracle.c")
LIB = os.path.join(HERE, "libmdpd_oracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cc = os.environ.get("CC", "gcc")
    base = [cc, "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-Wall", "-Wno-unknown-pragmas", SRC, "-o", LIB + ".tmp", "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        if r.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            return LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


if __name__ == "__main__":
    print(build(force=True, verbose=True))
