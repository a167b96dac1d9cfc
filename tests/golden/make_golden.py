"""Writes the stored expected values under tests/golden/ from the CPU oracle only.

Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle  # noqa: E402


def main():
    # Sketching matrices of Sec. 2.3 (SRHT with zero padding, Rademacher) and the
    # Gaussian N(0, 1/k) sketch, under the Philox4x32-10 entry convention.
    # The sparse-sign sketch is the block construction of the sparse JL transform.
    for kind, k, n, seed in [("srht", 5, 12, 3), ("rademacher", 6, 9, 4), ("gauss", 4, 7, 5),
                             ("sparse", 19, 6, 6)]:
        T = oracle.theta_dense(kind, k, n, seed)
        path = os.path.join(HERE, f"theta_{kind}_k{k}_n{n}_seed{seed}.txt")
        with open(path, "w") as f:
            f.write(f"# Theta ({k} x {n}) for the {kind} sketch, seed {seed}; Sec. 2.3 definitions,\n")
            f.write("# entries by the project's Philox4x32-10 convention; written by make_golden.py\n")
            np.savetxt(f, T, fmt="%.17e")


if __name__ == "__main__":
    main()
