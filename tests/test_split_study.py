"""The multi-step split study (split_study.py) run with the oracle as its
backend on the CPU: the driver's construction makes the unsplit pressure
exact, so the split error vanishes at constant density and for a pressure
constant in time, and is second order in the phase advance per step."""
import math

import numpy as np
import pytest

from oracle import ppe_oracle as O
from paper_2103_01874_gb300 import split_study


class OracleBackend:
    def __init__(self, lengths):
        self.L = lengths

    def dev(self, a):
        return np.array(a, dtype=np.float64)

    def project(self, u, v, w, S, rho, p_n, p_nm1, dt):
        out = O.ppe_project(u, v, w, S, rho, p_n, p_nm1, dt, self.L)
        return [out["p"], out["u"], out["v"], out["w"]]

    def correct(self, u, v, w, rho, p, p_n, p_nm1, dt, rho0):
        return list(O.ppe_correct(u, v, w, rho, p, p_n, p_nm1, rho0, dt, self.L))

    @staticmethod
    def lin(a, x, b, y):
        return a * x + b * y

    @staticmethod
    def maxabs(x):
        return float(np.abs(x).max())


B = OracleBackend((2 * math.pi,) * 3)


def test_constant_density_is_exact():
    r = split_study.run(n=16, rho_l=100.0, rho_g=100.0, phi=0.2, steps=6, backend=B)
    assert r["max_error"] < 1e-11


def test_pressure_constant_in_time_is_exact():
    r = split_study.run(n=16, rho_l=640.0, rho_g=60.0, phi=0.0, steps=6, backend=B)
    assert r["max_error"] < 1e-10


def test_second_order_in_the_phase_advance():
    e1 = split_study.run(n=16, rho_l=640.0, rho_g=120.0, phi=0.1, steps=8, backend=B)
    e2 = split_study.run(n=16, rho_l=640.0, rho_g=120.0, phi=0.05, steps=8, backend=B)
    ratio = e1["max_error_exact_history"] / e2["max_error_exact_history"]
    assert 3.0 < ratio < 5.0, ratio
    assert e1["max_error"] > 1e-8  # the case is not trivially exact
