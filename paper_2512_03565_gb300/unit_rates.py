"""Compiles and runs unit_rates.cu (sm_103a) and prints its per-SM throughputs.

The numbers justify the arithmetic design of the force path: FP64 and
float->double conversion rates on GB300 are far below FP32, so pair math is
FP32 and the per-particle FP64 fold converts with integer operations.
Usage: python -m paper_2512_03565_gb300.unit_rates [out.txt]
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    exe = os.path.join(HERE, "_build", "unit_rates")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "unit_rates.cu")], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    print(out, end="")
    if argv:
        open(argv[0], "w").write(out)


if __name__ == "__main__":
    main()
