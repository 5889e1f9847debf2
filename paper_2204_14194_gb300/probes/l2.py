"""Build and run the L2 row-streaming bandwidth probe: ``python -m paper_2204_14194_gb300.probes.l2``."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    out = os.path.join(HERE, "_build", "l2_rows")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", out,
                    os.path.join(HERE, "l2_rows.cu")], check=True)
    return subprocess.run([out]).returncode


if __name__ == "__main__":
    sys.exit(main())
