"""Writes the golden files of this folder.  Calls only the CPU oracle.

mc_table.txt -- the marching-cubes case table generated from first principles by oracle/mc.py
                (Lorensen-Cline marching cubes, used in Sec. IV-D and Sec. V-A.4 of the paper; the
                paper prints no table).  One row per case: case, triangle count, then the padded
                local-edge triples (-1 = unused).  The CUDA library generates its own table with
                independent code; a test requires the two to be identical.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import mc  # noqa: E402


def main():
    ntri, tab = mc.build_table()
    with open(os.path.join(HERE, "mc_table.txt"), "w") as f:
        f.write("# marching-cubes case table (oracle/mc.py); case ntri then 5 x 3 local edges\n")
        f.write("# corner c = (c&1, c>>1&1, c>>2&1); edge 4a+t along axis a; inside = value < iso\n")
        for c in range(256):
            f.write(" ".join(str(int(x)) for x in [c, ntri[c]] + tab[c].ravel().tolist()) + "\n")


if __name__ == "__main__":
    main()
