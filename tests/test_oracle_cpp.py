"""Pins of the C++ FP64 oracle (oracle/ppe_oracle.cpp), against the mathematics
and against the numpy oracle (a second oracle, itself pinned in
test_oracle_pins.py).

Brute force (the O4 checks): its FFT against the O(N^2) DFT sum for lengths of
radix 2 and 3, its DCT-II against the cosine sum written out here, DCT-III as
its inverse, its Thomas solve against a dense solve of the same tridiagonal
matrix.  Then the whole projection: discrete eigenfunctions (O1), the 7-point
residual (O2), the stored dense-LU fixture (O3), the divergence identity (O6),
zero mean (O8), the two y methods against each other, and agreement with the
numpy oracle on walls, outflow, both face rules and radix-3 grids.  Planted
mistakes inside the oracle (a flipped y diagonal, a dropped split term, a
flipped S) each trip a pin.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import cpp
from oracle import ppe_oracle as O
from paper_2103_01874_gb300 import fields

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("n", [8, 12, 16, 24, 32, 48, 96, 256, 384])
@pytest.mark.parametrize("inverse", [False, True])
def test_fft_matches_direct_dft(n, inverse):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    a = cpp.fft(x, inverse)
    # the O(N^2) sum of the definition, written out here in long double with the
    # exponent k m reduced modulo n in integers first
    k = np.arange(n)
    sgn = 1 if inverse else -1
    two_pi = 8 * np.arctan(np.longdouble(1))
    ang = two_pi * (np.outer(k, k) % n).astype(np.longdouble) / n
    ref = (np.cos(ang) + 1j * sgn * np.sin(ang)) @ x.astype(np.clongdouble)
    err = np.abs(a - ref).max() / np.abs(ref).max()
    assert err <= 1e-14 * max(1.0, math.log2(n)), err
    # and against the oracle's own direct sum
    assert np.abs(cpp.dft_direct(x, inverse) - ref).max() / np.abs(ref).max() <= 1e-13


def test_fft_of_a_pure_tone():
    n = 48
    x = np.exp(2j * np.pi * 5 * np.arange(n) / n)
    X = cpp.fft(x)
    expect = np.zeros(n, complex)
    expect[5] = n
    assert np.abs(X - expect).max() <= 1e-12


@pytest.mark.parametrize("n", [8, 16, 27, 64, 96])
def test_dct2_matches_cosine_sum_and_dct3_inverts(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal(n)
    X = cpp.dct2(x)
    j = np.arange(n)
    ref = np.array([np.sum(x * np.cos(np.pi * k * (j + 0.5) / n)) for k in range(n)])
    assert np.abs(X - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(cpp.dct3(X) - x).max() <= 1e-13 * np.abs(x).max()


def _tridiag(sub, diag, sup):
    n = len(diag)
    m = np.diag(diag)
    m[np.arange(1, n), np.arange(n - 1)] = sub[1:]
    m[np.arange(n - 1), np.arange(1, n)] = sup[:-1]
    return m


@pytest.mark.parametrize("n", [2, 8, 17, 64])
def test_thomas_matches_dense_solve(n):
    rng = np.random.default_rng(n)
    sub, sup = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    diag = 2.5 + rng.uniform(0, 1, n)  # diagonally dominant
    d = rng.standard_normal(n)
    x = cpp.thomas(sub, diag, sup, d)
    ref = np.linalg.solve(_tridiag(sub, diag, sup), d)
    assert np.abs(x - ref).max() <= 1e-14 * np.abs(ref).max()
    # the Neumann line of the 7-point operator with a shift lam < 0
    a, lam = 3.0, -0.7
    diag = np.full(n, -2 * a + lam)
    diag[0] = diag[-1] = -a + lam
    x = cpp.thomas(np.full(n, a), diag, np.full(n, a), d)
    ref = np.linalg.solve(_tridiag(np.full(n, a), diag, np.full(n, a)), d)
    assert np.abs(x - ref).max() <= 1e-13 * np.abs(ref).max()


CASES = [
    ((32, 24, 16), "multimode", 4.0, (2 * math.pi, 5.0, 3.0), 0, 0),
    ((18, 27, 12), "single", 2.0, (1.0, 4.0, 3.0), 0, 0),      # radix 3, odd ny
    ((16, 16, 16), "multimode", 3.0, (2 * math.pi,) * 3, 1, 0),  # harmonic face rule
    ((24, 16, 12), "single", 2.0, (2 * math.pi, 5.0, 2.0), 0, 1),  # outflow top
]


@pytest.mark.parametrize("shape,recipe,width,lengths,rule,bc", CASES)
def test_matches_numpy_oracle(shape, recipe, width, lengths, rule, bc):
    fl = fields.make_fields(*shape, seed=sum(shape), recipe=recipe, width=width, lx=lengths[0], ly=lengths[1],
                            lz=lengths[2])
    a = cpp.project_fields(fl, rule=rule, bc_top=bc)
    b = O.project_fields(fl, rule=rule, bc_top=bc)
    assert a["rho0"] == b["rho0"]
    for k in ("f", "p", "u", "v", "w"):
        assert O.rel_linf(a[k], b[k]) <= 1e-13, k


def test_y_methods_agree():
    fl = fields.make_fields(24, 32, 16, seed=9, recipe="multimode", width=4.0)
    a = cpp.project_fields(fl, y_method=0)
    b = cpp.project_fields(fl, y_method=1)
    for k in ("p", "u", "v", "w"):
        assert O.rel_linf(a[k], b[k]) <= 1e-13, k


@pytest.mark.parametrize("bc", [0, 1])
def test_discrete_eigenfunction(bc):
    """O1: p* = cos(2 pi a x/Lx + phi) Y_b(j) cos(2 pi c z/Lz + psi) with Y_b the
    cosine (walls) or quarter-wave (outflow) eigenvector of the y operator;
    f = lam p* exactly, so the solve returns p*."""
    nx, ny, nz = 24, 18, 12
    L = (2 * math.pi, 3.0, 5.0)
    dx, dy, dz = L[0] / nx, L[1] / ny, L[2] / nz
    a, b, c = 3, 5, 2
    x = (np.arange(nx) + 0.5) * dx
    z = (np.arange(nz) + 0.5) * dz
    j = np.arange(ny)
    kb = b + (0.5 if bc else 0.0)
    Y = np.cos(np.pi * kb * (j + 0.5) / ny)
    p = (np.cos(2 * np.pi * a * x / L[0] + 0.3)[None, None, :] * Y[None, :, None]
         * np.cos(2 * np.pi * c * z / L[2] - 1.1)[:, None, None])
    lam = (-(4 / dx**2) * math.sin(math.pi * a / nx) ** 2 - (4 / dy**2) * math.sin(math.pi * kb / (2 * ny)) ** 2
           - (4 / dz**2) * math.sin(math.pi * c / nz) ** 2)
    got = cpp.solve(lam * p, L, bc_top=bc)
    assert O.rel_linf(got, p) <= 1e-13
    # and the oracle's 7-point operator maps p* to lam p*
    assert O.rel_linf(cpp.laplacian(p, L, bc_top=bc), lam * p) <= 1e-13


def test_residual_and_zero_mean():
    """O2, O8: L p = f - mean(f) to rounding, and mean(p) = 0."""
    fl = fields.make_fields(32, 16, 24, seed=4, recipe="multimode", width=4.0)
    r = cpp.project_fields(fl)
    L = (fl.lx, fl.ly, fl.lz)
    res = r["f"] - r["f"].mean() - cpp.laplacian(r["p"], L)
    assert np.abs(res).max() <= 1e-13 * np.abs(r["f"]).max()
    assert abs(r["p"].mean()) <= 1e-15 * np.abs(r["p"]).max()


def test_dense_lu_fixture():
    """O3: the stored dense-LU solution of the bordered 8x6x10 system
    (written by tests/golden/make_golden.py from the numpy oracle's dense LU)."""
    with open(os.path.join(GOLDEN, "dense_lu_8x6x10.json")) as fh:
        g = json.load(fh)
    shape = tuple(g["shape_zyx"])
    f = np.random.default_rng(g["seed"]).standard_normal(shape)  # the fixture's right side, as its script draws it
    p_ref = np.array(g["p_dense_lu"]).reshape(shape)
    got = cpp.solve(f, tuple(g["lengths_xyz"]))
    assert O.rel_linf(got, p_ref) <= 1e-12


def test_divergence_identity():
    """O6: the corrected velocity has D u^{n+1} = S (S zero-mean on the cells)."""
    fl = fields.make_fields(24, 16, 16, seed=6, recipe="multimode", width=3.0)
    r = cpp.project_fields(fl)
    h = O.spacings(fl.shape, (fl.lx, fl.ly, fl.lz))
    div_new = O.div(r["u"], r["v"], r["w"], h)
    assert np.abs(div_new - fl.S).max() <= 1e-11 * np.abs(O.div(fl.u, fl.v, fl.w, h)).max()


@pytest.mark.parametrize("mutation", [1, 2, 3])
def test_planted_mistakes_trip_a_pin(mutation):
    fl = fields.make_fields(16, 16, 16, seed=8, recipe="multimode", width=3.0)
    good = cpp.project_fields(fl)
    bad = cpp.project_fields(fl, mutation=mutation)
    h = O.spacings(fl.shape, (fl.lx, fl.ly, fl.lz))
    caught = []
    # O2 residual against the true operator
    res = bad["f"] - bad["f"].mean() - cpp.laplacian(bad["p"], (fl.lx, fl.ly, fl.lz))
    caught.append(np.abs(res).max() > 1e-10 * np.abs(bad["f"]).max())
    # O6 divergence identity
    caught.append(np.abs(O.div(bad["u"], bad["v"], bad["w"], h) - fl.S).max()
                  > 1e-9 * np.abs(O.div(fl.u, fl.v, fl.w, h)).max())
    # cross-check against the numpy oracle
    caught.append(O.rel_linf(bad["p"], O.project_fields(fl)["p"]) > 1e-10)
    assert any(caught), mutation
    assert O.rel_linf(good["p"], O.project_fields(fl)["p"]) <= 1e-13
