"""The multi-step split study on the GPU (libppe backend) against the same
driver run with the oracle backend."""
import math

import numpy as np
import pytest

from paper_2103_01874_gb300 import split_study

pytestmark = pytest.mark.gpu


def test_gpu_sequence_matches_oracle_sequence():
    from test_split_study import OracleBackend
    L = (2 * math.pi,) * 3
    kw = dict(n=32, rho_l=1000.0, rho_g=10.0, phi=0.1, steps=12)
    g = split_study.run(**kw)
    o = split_study.run(backend=OracleBackend(L), **kw)
    e_g, e_o = np.array(g["errors"]), np.array(o["errors"])
    assert np.all(np.abs(e_g - e_o) <= 1e-6 * np.maximum(e_o, 1e-3))
    assert np.allclose(g["errors_exact_history"], o["errors_exact_history"], rtol=1e-6, atol=1e-9)


def test_gpu_constant_density_and_constant_pressure_are_exact():
    assert split_study.run(n=32, rho_l=100.0, rho_g=100.0, phi=0.2, steps=6)["max_error"] < 1e-11
    assert split_study.run(n=32, rho_l=640.0, rho_g=60.0, phi=0.0, steps=6)["max_error"] < 1e-10
