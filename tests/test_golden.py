"""The spectral oracle against stored dense-LU solutions (tests/golden)."""
import json
import os
import sys

import numpy as np

from oracle import ppe_oracle as O

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)
import make_golden as G  # noqa: E402


def test_dense_lu_fixture():
    with open(os.path.join(HERE, "dense_lu_8x6x10.json")) as fh:
        doc = json.load(fh)
    f, rho, src = G.inputs()
    shape = tuple(doc["shape_zyx"])
    p_ref = np.asarray(doc["p_dense_lu"]).reshape(shape)
    assert O.rel_linf(O.ppe_solve(f, tuple(doc["lengths_xyz"])), p_ref) < 1e-12
    q_ref = np.asarray(doc["q_var_coeff_dense_lu"]).reshape(shape)
    # q solves Eq. (30): its variable-coefficient residual is at rounding level
    res = O.var_coeff_apply(q_ref, rho, tuple(doc["lengths_xyz"])) - (src - src.mean())
    assert np.max(np.abs(res)) < 1e-10 * np.max(np.abs(src))
