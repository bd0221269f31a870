import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "_build")


def main():
    os.makedirs(OUT, exist_ok=True)
    rc = 0
    for name in ("rates", "tcgen05_rate"):
        exe = os.path.join(OUT, "fq_" + name)
        subprocess.run(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                        os.path.join(HERE, name + ".cu")], check=True)
        rc = rc or subprocess.run([exe]).returncode
    sys.exit(rc)


if __name__ == "__main__":
    main()
