"""Build the oracle's shared library with gcc (test infrastructure only).

Plain portable C (no x86 intrinsics, no -march=native) so it builds the same
on x86_64 and aarch64.  OpenMP is used when the compiler supports it.
"""
from __future__ import annotations

import subprocess
from pathlib import Path

HERE = Path(__file__).resolve().parent


def build(verbose: bool = False) -> Path:
    out = HERE / "_build" / "liboracle.so"
    out.parent.mkdir(parents=True, exist_ok=True)
    src = HERE / "modal_oracle.c"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", str(src), "-o", str(out)]
    for extra in (["-fopenmp"], []):
        cmd = base[:5] + extra + base[5:] + ["-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            if verbose:
                print(" ".join(cmd))
            return out
    raise RuntimeError("oracle build failed:\n" + r.stderr)


if __name__ == "__main__":
    print(build(verbose=True))
