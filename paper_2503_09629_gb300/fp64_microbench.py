"""Build and run the FP64 issue-rate microbenchmark (csrc/fp64_microbench.cu,
a standalone program outside libsubcyc.so) on GPU 0:

    python -m paper_2503_09629_gb300.fp64_microbench

It prints the DADD, DMUL and DFMA issue rates, the rate of fma(x, 1, a) with
a literal and with a run-time 1, and DFMA throughput against warps per SM and
independent chains per thread.
"""
import os
import subprocess
import sys

from paper_2503_09629_gb300 import buildlib


def build() -> str:
    """Compile the microbenchmark for sm_103a into the package's build folder."""
    src = os.path.join(buildlib.SRC, "fp64_microbench.cu")
    os.makedirs(buildlib.OUT_DIR, exist_ok=True)
    exe = os.path.join(buildlib.OUT_DIR, "fp64_microbench")
    if buildlib._stale(exe, [src]):
        subprocess.check_call([buildlib.nvcc()] + buildlib.ARCH + ["-O3", "-std=c++17", "-o", exe, src])
    return exe


def main() -> int:
    return subprocess.call([build()])


if __name__ == "__main__":
    sys.exit(main())
