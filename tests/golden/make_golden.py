"""Writes the regression fixtures in this folder from the CPU oracle alone.

Run from the repository root: ``python tests/golden/make_golden.py``. It calls only
``oracle/`` (and the seeded generators in ``synth/``); no value here comes from the CUDA
library. The paper prints no numeric worked example (its Fig. 3 example is a picture), so
these fixtures freeze the oracle's output on two small inputs whose meaning is checked
independently: the Laplacian one against the closed form of the 5-point stencil squared,
the uniform one against a dense product (tests/test_golden.py).
"""

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth   # noqa: E402

CASES = {
    "uniform_40x40_d0.1_seed21": lambda: (synth.uniform_random(40, 40, 0.1, 21),) * 2,
    "laplacian2d_g5_squared": lambda: (synth.laplacian2d(5),) * 2,
}


def write(name, A, B):
    out = oracle.spgemm(A, B)
    path = os.path.join(HERE, name + ".txt")
    with open(path, "w") as f:
        f.write(f"# C = A*B, {name}; written by tests/golden/make_golden.py from oracle/ only\n")
        f.write(f"# rows cols nnz\n{A.rows} {B.cols} {out.nnz}\n")
        f.write("# row_ptr\n" + " ".join(str(int(x)) for x in out.row_ptr) + "\n")
        f.write("# col\n" + " ".join(str(int(x)) for x in out.col) + "\n")
        f.write("# val (float64, hex)\n" + " ".join(float(x).hex() for x in out.val) + "\n")


if __name__ == "__main__":
    for name, make in CASES.items():
        A, B = make()
        write(name, A, B)
        print("wrote", name)
