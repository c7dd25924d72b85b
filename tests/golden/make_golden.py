"""Writes tests/golden/dense_lu_8x6x10.json using only oracle/ and numpy.

The paper prints no worked numerical example of the projection (Sec. 5.4 gives
the equations only), so this fixture holds values fixed by a second, slower
method: the dense LU solve of the bordered 7-point system (L p = f, sum p = 0)
and of the unsplit variable-coefficient Eq. (30) on an 8x6x10 grid, with inputs
drawn inline from numpy.random.default_rng(2024).

Run:  python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle import ppe_oracle as O  # noqa: E402

SHAPE = (10, 6, 8)          # (Nz, Ny, Nx)
LENGTHS = (2 * math.pi, 3.0, 5.0)
SEED = 2024


def inputs():
    rng = np.random.default_rng(SEED)
    f = rng.standard_normal(SHAPE)
    rho = 120.0 + 520.0 * rng.random(SHAPE)
    src = rng.standard_normal(SHAPE)
    return f, rho, src


def main():
    f, rho, src = inputs()
    h = O.spacings(SHAPE, LENGTHS)
    p = O.dense_zero_mean_solve(O.dense_operator(lambda q: O.laplacian(q, h), SHAPE), f)
    q = O.var_coeff_solve_dense(src, rho, LENGTHS)
    doc = {
        "what": "dense LU solutions on an 8x6x10 grid (x fastest), zero mean",
        "citation": "Eq. (34) left side L p = f and Eq. (30) D[(1/rho_f) G q] = src, Sec. 5.4; "
                    "7-point finite-volume operators on the staggered mesh, Sec. 5",
        "shape_zyx": SHAPE, "lengths_xyz": LENGTHS, "seed": SEED,
        "p_dense_lu": [float(x) for x in p.ravel()],
        "q_var_coeff_dense_lu": [float(x) for x in q.ravel()],
    }
    with open(os.path.join(HERE, "dense_lu_8x6x10.json"), "w") as fh:
        json.dump(doc, fh, indent=0)


if __name__ == "__main__":
    main()
