"""Writes the golden fixtures of this folder; calls only the oracle.

dft_2x4x4.txt: the forward 3-D DFT X[k] = sum_j x[j] exp(-2 pi i (j0 k0 / 2 + j1 k1 / 4 + j2 k2 / 4))
(the plain definition of the transform, AccFFT Section 2) of a fixed 2x4x4 array of Gaussian
integers, x[j0, j1, j2] = ((j0 + 2 j1 + 3 j2) mod 5 - 2) + i ((j0 j1 + j2) mod 3 - 1).  For
lengths 2 and 4 every root of unity is one of 1, -i, -1, i, so every bin is a Gaussian integer:
the oracle's FP64 result is rounded to it (the rounding is checked to be below 1e-9).  The paper
prints no numeric transform values (its result figures are timing plots), so no fixture here is
the paper's own.

Run from the repository root: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle  # noqa: E402

SHAPE = (2, 4, 4)


def golden_input():
    x = np.zeros(SHAPE, dtype=np.complex128)
    for j0 in range(SHAPE[0]):
        for j1 in range(SHAPE[1]):
            for j2 in range(SHAPE[2]):
                x[j0, j1, j2] = complex((j0 + 2 * j1 + 3 * j2) % 5 - 2, (j0 * j1 + j2) % 3 - 1)
    return x


def main():
    oracle.build()
    X = oracle.c2c(golden_input(), -1, "naive")
    R = np.round(X.real), np.round(X.imag)
    assert np.max(np.abs(X.real - R[0])) < 1e-9 and np.max(np.abs(X.imag - R[1])) < 1e-9
    with open(os.path.join(HERE, "dft_2x4x4.txt"), "w") as fh:
        fh.write("# forward 3-D DFT of the 2x4x4 Gaussian-integer array of make_golden.py\n")
        fh.write("# (AccFFT Section 2: the transform is the plain 3-D DFT); k0 k1 k2 re im\n")
        for k0 in range(SHAPE[0]):
            for k1 in range(SHAPE[1]):
                for k2 in range(SHAPE[2]):
                    fh.write("%d %d %d %d %d\n" % (k0, k1, k2, int(R[0][k0, k1, k2]), int(R[1][k0, k1, k2])))


if __name__ == "__main__":
    main()
