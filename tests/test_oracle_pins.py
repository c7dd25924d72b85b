"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

The paper prints no worked example of the projection, so every pin here is a
closed form, an identity, brute force or a dense direct solve:
  O1 discrete eigenfunctions of L and the eigenvalue formula
  O2 7-point residual of the solve
  O3 dense LU of L (bordered with the zero-mean constraint)
  O4 brute-force loops for G, D, L and the face densities
  O5 constant-density limit: the classic projection, p independent of p_hat
  O6 divergence identity D u^{n+1} = S (Eq. (31) constraint)
  O7 split exactness: p^n = p^{n-1} = q solving Eq. (30) returns q (Eq. (32) text)
  O8 zero mean
  O9 shift and reflection symmetry
Anisotropic grids and box lengths are used so that a swapped axis or spacing fails.
"""
import math

import numpy as np
import pytest

from oracle import ppe_oracle as O
from paper_2103_01874_gb300.fields import make_fields

LENGTHS = (2 * math.pi, 3.0, 5.0)


def _bf_lap(q, h):
    """Brute-force 7-point finite-volume Laplacian with pure Python loops."""
    dx, dy, dz = h
    nz, ny, nx = q.shape
    out = np.zeros_like(q)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = q[k, j, i]
                fx = (q[k, j, (i + 1) % nx] - c) / dx - (c - q[k, j, (i - 1) % nx]) / dx
                fz = (q[(k + 1) % nz, j, i] - c) / dz - (c - q[(k - 1) % nz, j, i]) / dz
                top = (q[k, j + 1, i] - c) / dy if j + 1 < ny else 0.0
                bot = (c - q[k, j - 1, i]) / dy if j > 0 else 0.0
                out[k, j, i] = fx / dx + (top - bot) / dy + fz / dz
    return out


def test_laplacian_brute_force():
    rng = np.random.default_rng(11)
    shape = (5, 4, 6)
    q = rng.standard_normal(shape)
    h = O.spacings(shape, LENGTHS)
    np.testing.assert_allclose(O.laplacian(q, h), _bf_lap(q, h), rtol=0, atol=1e-12)


def test_grad_div_brute_force():
    rng = np.random.default_rng(12)
    nz, ny, nx = 4, 5, 3
    h = O.spacings((nz, ny, nx), LENGTHS)
    dx, dy, dz = h
    q = rng.standard_normal((nz, ny, nx))
    gx, gy, gz = O.grad(q, h)
    a = rng.standard_normal((nz, ny, nx))
    b = rng.standard_normal((nz, ny + 1, nx))
    c = rng.standard_normal((nz, ny, nx))
    d = O.div(a, b, c, h)
    for k in range(nz):
        for j in range(ny + 1):
            for i in range(nx):
                want = 0.0 if j in (0, ny) else (q[k, j, i] - q[k, j - 1, i]) / dy
                assert gy[k, j, i] == pytest.approx(want, abs=1e-13)
                if j == ny:
                    continue
                assert gx[k, j, i] == pytest.approx((q[k, j, i] - q[k, j, i - 1]) / dx, abs=1e-13)
                assert gz[k, j, i] == pytest.approx((q[k, j, i] - q[k - 1, j, i]) / dz, abs=1e-13)
                want = ((a[k, j, (i + 1) % nx] - a[k, j, i]) / dx + (b[k, j + 1, i] - b[k, j, i]) / dy
                        + (c[(k + 1) % nz, j, i] - c[k, j, i]) / dz)
                assert d[k, j, i] == pytest.approx(want, abs=1e-12)


@pytest.mark.parametrize("rule", [O.FACE_ARITHMETIC, O.FACE_HARMONIC])
def test_face_density_brute_force(rule):
    rng = np.random.default_rng(13)
    nz, ny, nx = 3, 4, 5
    rho = 100 + 500 * rng.random((nz, ny, nx))
    rx, ry, rz = O.face_density(rho, rule)

    def mean(a, b):
        return 0.5 * (a + b) if rule == O.FACE_ARITHMETIC else 2 * a * b / (a + b)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                assert rx[k, j, i] == pytest.approx(mean(rho[k, j, i - 1], rho[k, j, i]), rel=1e-15)
                assert rz[k, j, i] == pytest.approx(mean(rho[k - 1, j, i], rho[k, j, i]), rel=1e-15)
                if j > 0:
                    assert ry[k, j, i] == pytest.approx(mean(rho[k, j - 1, i], rho[k, j, i]), rel=1e-15)


def _eigenfunction(shape, a, b, c, phi, psi):
    nz, ny, nx = shape
    lx, _, lz = LENGTHS
    x = (np.arange(nx) + 0.5) * lx / nx
    z = (np.arange(nz) + 0.5) * lz / nz
    j = np.arange(ny)
    return (np.cos(2 * math.pi * a * x / lx + phi)[None, None, :]
            * np.cos(math.pi * b * (j + 0.5) / ny)[None, :, None]
            * np.cos(2 * math.pi * c * z / lz + psi)[:, None, None])


@pytest.mark.parametrize("shape", [(24, 8, 12), (16, 12, 32), (9, 6, 8)])
@pytest.mark.parametrize("abc", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (3, 2, 5), (2, 5, 1)])
def test_eigenfunction_manufactured(shape, abc):
    """O1: L p* = lam p* exactly for the discrete eigenfunctions, and the solve
    of lam p* returns p*."""
    nz, ny, nx = shape
    a, b, c = abc
    a, b, c = a % (nx // 2), b % ny, c % (nz // 2)
    if (a, b, c) == (0, 0, 0):
        b = 1
    h = O.spacings(shape, LENGTHS)
    dx, dy, dz = h
    p = _eigenfunction(shape, a, b, c, 0.3, -1.1)
    lam = (-(4 / dx**2) * math.sin(math.pi * a / nx) ** 2
           - (4 / dy**2) * math.sin(math.pi * b / (2 * ny)) ** 2
           - (4 / dz**2) * math.sin(math.pi * c / nz) ** 2)
    np.testing.assert_allclose(O.laplacian(p, h), lam * p, rtol=0, atol=1e-12 * abs(lam))
    sol = O.ppe_solve(lam * p, LENGTHS)
    assert O.rel_linf(sol, p - p.mean()) < 1e-13


def test_eigenvalue_table_matches_formula():
    shape = (6, 5, 8)
    lam = O.eigenvalues(shape, LENGTHS)
    dx, dy, dz = O.spacings(shape, LENGTHS)
    for kz in range(6):
        for ky in range(5):
            for kx in range(5):
                want = (-(4 / dx**2) * math.sin(math.pi * kx / 8) ** 2
                        - (4 / dy**2) * math.sin(math.pi * ky / 10) ** 2
                        - (4 / dz**2) * math.sin(math.pi * kz / 6) ** 2)
                assert lam[kz, ky, kx] == pytest.approx(want, rel=1e-14, abs=1e-14)


@pytest.mark.parametrize("shape", [(8, 8, 8), (10, 4, 6), (6, 9, 4)])
def test_dense_lu(shape):
    """O3: the spectral solve equals the dense LU solve of the bordered 7-point system."""
    rng = np.random.default_rng(21)
    f = rng.standard_normal(shape)
    h = O.spacings(shape, LENGTHS)
    mat = O.dense_operator(lambda q: O.laplacian(q, h), shape)
    ref = O.dense_zero_mean_solve(mat, f)
    assert O.rel_linf(O.ppe_solve(f, LENGTHS), ref) < 1e-12


def _fields(n=(12, 8, 16), seed=5, **kw):
    nx, ny, nz = n
    return make_fields(nx, ny, nz, seed=seed, lx=LENGTHS[0], ly=LENGTHS[1], lz=LENGTHS[2], **kw)


@pytest.mark.parametrize("rule", [O.FACE_ARITHMETIC, O.FACE_HARMONIC])
def test_residual_and_divergence(rule):
    """O2 + O6 + O8 on generated two-phase fields."""
    fl = _fields()
    out = O.project_fields(fl, rule=rule)
    h = O.spacings(fl.shape, LENGTHS)
    r = out["f"] - out["f"].mean() - O.laplacian(out["p"], h)
    assert np.max(np.abs(r)) / np.max(np.abs(out["f"])) < 1e-13
    div_new = O.div(out["u"], out["v"], out["w"], h)
    div_old = O.div(fl.u, fl.v, fl.w, h)
    assert np.max(np.abs(div_new - fl.S)) < 1e-11 * np.max(np.abs(div_old))
    assert abs(out["p"].mean()) < 1e-15 * np.max(np.abs(out["p"])) * 10
    assert abs(out["f"].mean()) < 1e-12 * np.max(np.abs(out["f"]))
    assert np.all(out["v"][:, 0, :] == 0) and np.all(out["v"][:, -1, :] == 0)
    assert out["rho0"] == fl.rho.min()


def test_constant_density_limit():
    """O5: rho = rho_0 everywhere gives the classic projection, Eq. (29)-(30):
    f = (rho_0/dt)(D u* - S) whatever p_hat is, u = u* - dt G p / rho_0."""
    fl = _fields(seed=7)
    rho = np.full(fl.shape, 333.0)
    h = O.spacings(fl.shape, LENGTHS)
    a = O.ppe_project(fl.u, fl.v, fl.w, fl.S, rho, fl.p_n, fl.p_nm1, fl.dt, LENGTHS)
    b = O.ppe_project(fl.u, fl.v, fl.w, fl.S, rho, fl.p_nm1 * 3, fl.p_n, fl.dt, LENGTHS)
    assert O.rel_linf(a["p"], b["p"]) < 1e-14
    f_classic = (333.0 / fl.dt) * (O.div(fl.u, fl.v, fl.w, h) - fl.S)
    assert O.rel_linf(a["f"], f_classic) < 1e-14
    gx, gy, gz = O.grad(a["p"], h)
    assert O.rel_linf(a["u"], fl.u - fl.dt * gx / 333.0) < 1e-14
    assert O.rel_linf(a["v"], fl.v - fl.dt * gy / 333.0) < 1e-14


@pytest.mark.parametrize("rule", [O.FACE_ARITHMETIC, O.FACE_HARMONIC])
def test_split_exactness(rule):
    """O7: when grad p_hat = grad p^{n+1} the split (Eq. (32)) is exact.  Solve
    the unsplit variable-coefficient Eq. (30) for q by dense LU, set
    p^n = p^{n-1} = q; the split projection must return p = q and the unsplit
    corrected velocity of Eq. (29)."""
    fl = _fields(n=(8, 6, 10), seed=9, width=2.0)
    h = O.spacings(fl.shape, LENGTHS)
    src = (O.div(fl.u, fl.v, fl.w, h) - fl.S) / fl.dt
    q = O.var_coeff_solve_dense(src, fl.rho, LENGTHS, rule)
    out = O.ppe_project(fl.u, fl.v, fl.w, fl.S, fl.rho, q, q, fl.dt, LENGTHS, rule=rule)
    assert O.rel_linf(out["p"], q) < 1e-11
    gx, gy, gz = O.grad(q, h)
    rx, ry, rz = O.face_density(fl.rho, rule)
    assert O.rel_linf(out["u"], fl.u - fl.dt * gx / rx) < 1e-12
    assert O.rel_linf(out["v"], fl.v - fl.dt * gy / ry) < 1e-12
    assert O.rel_linf(out["w"], fl.w - fl.dt * gz / rz) < 1e-12


def test_symmetry_shift_and_reflection():
    """O9: a shift by one cell in x or z commutes with the projection; the
    reflection j -> Ny-1-j (v -> -v on mirrored faces) maps the solution."""
    fl = _fields(seed=15)
    base = O.project_fields(fl)
    for axis in (0, 2):
        sh = {k: np.roll(getattr(fl, k), 1, axis=axis) for k in ("u", "v", "w", "S", "rho", "p_n", "p_nm1")}
        out = O.ppe_project(sh["u"], sh["v"], sh["w"], sh["S"], sh["rho"], sh["p_n"], sh["p_nm1"],
                            fl.dt, LENGTHS)
        for key in ("p", "u", "v", "w"):
            assert O.rel_linf(out[key], np.roll(base[key], 1, axis=axis)) < 1e-13
    fy = {k: getattr(fl, k)[:, ::-1, :].copy() for k in ("u", "w", "S", "rho", "p_n", "p_nm1")}
    vy = -fl.v[:, ::-1, :].copy()
    out = O.ppe_project(fy["u"], vy, fy["w"], fy["S"], fy["rho"], fy["p_n"], fy["p_nm1"], fl.dt, LENGTHS)
    assert O.rel_linf(out["p"], base["p"][:, ::-1, :]) < 1e-13
    assert O.rel_linf(out["v"], -base["v"][:, ::-1, :]) < 1e-13
    assert O.rel_linf(out["u"], base["u"][:, ::-1, :]) < 1e-13


def test_generator_properties():
    fl = make_fields(16, 12, 8, seed=3, recipe="multimode", width=6.0)
    assert fl.v.shape == (8, 13, 16)
    assert np.all(fl.v[:, 0, :] == 0) and np.all(fl.v[:, 12, :] == 0)
    assert abs(fl.S.mean()) < 1e-17 * fl.S.size
    assert abs(fl.p_n.mean()) < 1e-15 and abs(fl.p_nm1.mean()) < 1e-15
    assert 120.0 <= fl.rho.min() < fl.rho.max() <= 640.0
    again = make_fields(16, 12, 8, seed=3, recipe="multimode", width=6.0)
    for k, a in fl.arrays().items():
        assert np.array_equal(a, again.arrays()[k])
    # liquid below the interface: density decreases upward in y on average
    prof = fl.rho.mean(axis=(0, 2))
    assert prof[0] > prof[-1]


# ----------------------------------------------------------------------------
# Planted mistakes: each plausible error in the oracle must trip a pin.
# ----------------------------------------------------------------------------

def test_planted_eigenvalue_mistake_is_caught(monkeypatch):
    """A y eigenvalue with pi k/N instead of pi k/(2N) must fail the dense-LU pin."""
    good = O.eigenvalues

    def bad(shape, lengths):
        lam = good(shape, lengths)
        nz, ny, nx = shape
        dy = lengths[1] / ny
        ky = np.arange(ny)
        wrong = -(4 / dy**2) * np.sin(math.pi * ky / ny) ** 2
        right = -(4 / dy**2) * np.sin(math.pi * ky / (2 * ny)) ** 2
        return lam + (wrong - right)[None, :, None]
    monkeypatch.setattr(O, "eigenvalues", bad)
    shape = (8, 8, 8)
    f = np.random.default_rng(1).standard_normal(shape)
    h = O.spacings(shape, LENGTHS)
    ref = O.dense_zero_mean_solve(O.dense_operator(lambda q: O.laplacian(q, h), shape), f)
    assert O.rel_linf(O.ppe_solve(f, LENGTHS), ref) > 1e-3


def test_planted_sign_mistake_is_caught(monkeypatch):
    """A flipped sign on S in Eq. (34) must fail the divergence identity."""
    good = O.ppe_rhs

    def bad(u, v, w, S, *a, **k):
        return good(u, v, w, -S, *a, **k)
    monkeypatch.setattr(O, "ppe_rhs", bad)
    fl = _fields(seed=4)
    out = O.project_fields(fl)
    h = O.spacings(fl.shape, LENGTHS)
    err = np.max(np.abs(O.div(out["u"], out["v"], out["w"], h) - fl.S))
    assert err > 1e-3 * np.max(np.abs(fl.S))


def test_planted_split_mistake_is_caught(monkeypatch):
    """Dropping the explicit split term of Eq. (34) must fail split exactness."""
    def bad(u, v, w, S, rho, p_n, p_nm1, rho0, dt, lengths, rule=O.FACE_ARITHMETIC, bc_top=O.BC_WALL):
        h = O.spacings(rho.shape, lengths)
        return (rho0 / dt) * (O.div(u, v, w, h) - S)
    fl = _fields(n=(8, 6, 10), seed=9, width=2.0)
    h = O.spacings(fl.shape, LENGTHS)
    q = O.var_coeff_solve_dense((O.div(fl.u, fl.v, fl.w, h) - fl.S) / fl.dt, fl.rho, LENGTHS)
    monkeypatch.setattr(O, "ppe_rhs", bad)
    out = O.ppe_project(fl.u, fl.v, fl.w, fl.S, fl.rho, q, q, fl.dt, LENGTHS)
    assert O.rel_linf(out["p"], q) > 1e-3


def _incompatible(fl, s_shift=0.05, v_top=0.3, v_bot=-0.1):
    """Fields with wall flux and a shifted S: sum of (D u* - S) no longer vanishes."""
    v = fl.v.copy()
    v[:, -1, :] = v_top
    v[:, 0, :] = v_bot
    return v, fl.S + s_shift


def test_compatibility_against_assembled_f():
    """The compatibility quantities predict mean(f) of the assembled Eq. (34)
    right-hand side (divergence theorem on the periodic/wall box), including
    wall flux and a non-zero mean of S; the solve then drops exactly that mean."""
    fl = _fields(seed=11)
    v, S = _incompatible(fl)
    rho0 = O.rho0_of(fl.rho)
    f = O.ppe_rhs(fl.u, v, fl.w, S, fl.rho, fl.p_n, fl.p_nm1, rho0, fl.dt, LENGTHS)
    c = O.compatibility(v, S, LENGTHS)
    predicted = (rho0 / fl.dt) * (c["wall_flux_mean"] - c["s_mean"])
    assert abs(f.mean() - predicted) <= 1e-12 * np.abs(f).max()
    assert abs(predicted) > 1e-3 * np.abs(f).max()   # the case is really incompatible
    assert c["wall_vmax"] == 0.3 and c["s_absmax"] == np.abs(S).max()
    # generated fields are compatible: no wall flux, S mean removed
    c0 = O.compatibility(fl.v, fl.S, LENGTHS)
    assert c0["wall_vmax"] == 0.0 and abs(c0["s_mean"]) <= 1e-15 * c0["s_absmax"]


def test_planted_wall_flux_sign_is_caught(monkeypatch):
    """A flipped wall-flux sign must disagree with the assembled f."""
    good = O.compatibility

    def bad(v, S, lengths):
        c = good(v, S, lengths)
        c["wall_flux_mean"] = -c["wall_flux_mean"]
        return c
    monkeypatch.setattr(O, "compatibility", bad)
    fl = _fields(seed=11)
    v, S = _incompatible(fl)
    rho0 = O.rho0_of(fl.rho)
    f = O.ppe_rhs(fl.u, v, fl.w, S, fl.rho, fl.p_n, fl.p_nm1, rho0, fl.dt, LENGTHS)
    c = O.compatibility(v, S, LENGTHS)
    predicted = (rho0 / fl.dt) * (c["wall_flux_mean"] - c["s_mean"])
    assert abs(f.mean() - predicted) > 1e-3 * np.abs(f).max()


@pytest.mark.parametrize("rule", [O.FACE_ARITHMETIC, O.FACE_HARMONIC])
def test_unsplit_projection_dense(rule):
    """Eqs. (29)-(30) by dense LU: the corrected velocity satisfies D u^{n+1} = S
    (zero-mean S), p has zero mean, the residual of Eq. (30) vanishes, and a
    brute-force loop of the variable-coefficient operator agrees with
    var_coeff_apply."""
    fl = _fields(n=(8, 6, 10), seed=21, width=2.0)
    h = O.spacings(fl.shape, LENGTHS)
    out = O.unsplit_project_dense(fl.u, fl.v, fl.w, fl.S, fl.rho, fl.dt, LENGTHS, rule)
    div_new = O.div(out["u"], out["v"], out["w"], h)
    assert np.max(np.abs(div_new - fl.S)) < 1e-11 * np.max(np.abs(O.div(fl.u, fl.v, fl.w, h)))
    assert abs(out["p"].mean()) < 1e-13 * np.max(np.abs(out["p"]))
    assert O.unsplit_residual(out["p"], out["g"], fl.rho, LENGTHS, rule) < 1e-12
    # brute-force A p at a few cells: sum over the 6 faces of (1/rho_f)(p_nbr - p)/h^2
    q, rho = out["p"], fl.rho
    nz, ny, nx = q.shape
    ap = O.var_coeff_apply(q, rho, LENGTHS, rule)

    def rf(a, b):
        return 0.5 * (a + b) if rule == O.FACE_ARITHMETIC else 2.0 / (1.0 / a + 1.0 / b)
    for (k, j, i) in [(0, 0, 0), (3, 2, 5), (nz - 1, ny - 1, nx - 1), (5, 3, 0)]:
        acc = 0.0
        for (dk, dj, di), hh in [((0, 0, 1), h[0]), ((0, 0, -1), h[0]), ((0, 1, 0), h[1]), ((0, -1, 0), h[1]),
                                 ((1, 0, 0), h[2]), ((-1, 0, 0), h[2])]:
            jj = j + dj
            if jj < 0 or jj >= ny:
                continue  # wall: no flux
            kk, ii = (k + dk) % nz, (i + di) % nx
            acc += (q[kk, jj, ii] - q[k, j, i]) / rf(rho[kk, jj, ii], rho[k, j, i]) / hh ** 2
        assert abs(acc - ap[k, j, i]) < 1e-12 * np.max(np.abs(ap))


def test_planted_unsplit_density_mistake_is_caught():
    """Using rho_0 instead of rho_f in Eq. (29) must break the divergence identity."""
    fl = _fields(n=(8, 6, 10), seed=22, width=2.0)
    h = O.spacings(fl.shape, LENGTHS)
    out = O.unsplit_project_dense(fl.u, fl.v, fl.w, fl.S, fl.rho, fl.dt, LENGTHS)
    gx, gy, gz = O.grad(out["p"], h)
    r0 = O.rho0_of(fl.rho)
    bad = O.div(fl.u - fl.dt * gx / r0, fl.v - fl.dt * gy / r0, fl.w - fl.dt * gz / r0, h)
    assert np.max(np.abs(bad - fl.S)) > 1e-3 * np.max(np.abs(fl.S))


def _eq31_inputs(shape=(6, 5, 4), seed=3):
    rng = np.random.default_rng(seed)
    C = rng.choice([0.0, 1.0, 0.3, 0.7], size=shape)
    comp_g = rng.normal(0.0, 2.0, shape)
    comp_l = rng.normal(0.0, 0.1, shape)
    mdot = np.where((C > 0) & (C < 1), rng.uniform(-1.0, 3.0, shape), 0.0)
    rho_g = rng.uniform(50.0, 130.0, shape)
    rho_l = rng.uniform(600.0, 700.0, shape)
    mask = (rng.random(shape) < 0.3).astype(np.uint8)
    return C, comp_g, comp_l, mdot, rho_g, rho_l, mask


def test_divergence_constraint_limits_and_loop():
    """Eq. (31): pure phases reduce to -(1/rho) D rho/Dt of that phase; no
    compressibility and equal densities give S = 0; evaporation (mdot > 0,
    rho_l > rho_g) expands (S > 0); the masked interface cells are zero and
    only those; a scalar loop agrees with the vectorised form."""
    C, cg, cl, md, rg, rl, mask = _eq31_inputs()
    S, rho = O.divergence_constraint(C, cg, cl, md, rg, rl, mask)
    gas, liq, itf = C == 0.0, C == 1.0, (C > 0) & (C < 1)
    assert np.array_equal(S[gas], -cg[gas]) and np.array_equal(S[liq], -cl[liq])
    assert np.all(S[itf & (mask != 0)] == 0.0)
    assert np.array_equal(rho[gas], rg[gas]) and np.array_equal(rho[liq], rl[liq])
    z = np.zeros_like(C)
    S0, _ = O.divergence_constraint(C, z, z, md, rg, rg)
    assert np.all(S0 == 0.0)
    Se, _ = O.divergence_constraint(np.full_like(C, 0.5), z, z, np.ones_like(C), rg, rl)
    assert np.all(Se > 0.0)
    for idx in np.ndindex(C.shape):
        c = C[idx]
        s = -(1 - c) * cg[idx] - c * cl[idx] + md[idx] * (1 / rg[idx] - 1 / rl[idx])
        if mask[idx] and 0 < c < 1:
            s = 0.0
        assert abs(s - S[idx]) <= 1e-15 * max(1.0, abs(s))
        assert abs(rg[idx] + (rl[idx] - rg[idx]) * c - rho[idx]) <= 1e-13 * rho[idx]


def test_planted_phase_change_sign_is_caught(monkeypatch):
    """Swapping 1/rho_g and 1/rho_l in the phase-change term must fail the
    expansion check."""
    good = O.divergence_constraint

    def bad(C, cg, cl, md, rg, rl, mask=None):
        return good(C, cg, cl, md, rl, rg, mask)
    monkeypatch.setattr(O, "divergence_constraint", bad)
    C, cg, cl, md, rg, rl, mask = _eq31_inputs()
    z = np.zeros_like(C)
    Se, _ = O.divergence_constraint(np.full_like(C, 0.5), z, z, np.ones_like(C), rg, rl)
    assert not np.all(Se > 0.0)



# ---------------------------------------------------------------------------
# outflow top boundary (p = 0 on the face y = Ly; the bottom stays a wall)
# ---------------------------------------------------------------------------
OUT = O.BC_OUTFLOW


@pytest.mark.parametrize("shape", [(6, 5, 4), (8, 7, 6)])
@pytest.mark.parametrize("abc", [(0, 0, 0), (1, 3, 2), (2, 0, 1)])
def test_outflow_eigenfunction_manufactured(shape, abc):
    """DCT-IV modes cos(pi (b + 1/2)(j + 1/2)/Ny) times Fourier modes in x, z
    are eigenfunctions of the 7-point operator with the outflow ghost value;
    the solve inverts them (including a = b = c = 0, which is no zero mode)."""
    nz, ny, nx = shape
    a, b, c = abc
    h = O.spacings(shape, LENGTHS)
    x = (np.arange(nx) + 0.5) * h[0]
    z = (np.arange(nz) + 0.5) * h[2]
    phi = (np.cos(2 * math.pi * a * x / LENGTHS[0] + 0.4)[None, None, :]
           * np.cos(math.pi * (b + 0.5) * (np.arange(ny) + 0.5) / ny)[None, :, None]
           * np.cos(2 * math.pi * c * z / LENGTHS[2] - 0.7)[:, None, None])
    lam = (-(4 / h[0] ** 2) * math.sin(math.pi * a / nx) ** 2
           - (4 / h[1] ** 2) * math.sin(math.pi * (b + 0.5) / (2 * ny)) ** 2
           - (4 / h[2] ** 2) * math.sin(math.pi * c / nz) ** 2)
    assert np.max(np.abs(O.laplacian(phi, h, OUT) - lam * phi)) < 1e-10 * abs(lam)
    assert O.rel_linf(O.ppe_solve(lam * phi, LENGTHS, OUT), phi) < 1e-12


def test_outflow_laplacian_brute_force_and_dense():
    """The top cell sees the ghost value -p_{Ny-1} (p = 0 on the face); the
    spectral solve equals a dense LU solve of the 7-point operator."""
    shape = (6, 5, 8)
    nz, ny, nx = shape
    h = O.spacings(shape, LENGTHS)
    q = np.random.default_rng(3).standard_normal(shape)
    lap = O.laplacian(q, h, OUT)
    for (k, j, i) in [(0, ny - 1, 0), (3, ny - 1, 5), (2, 0, 7), (5, 2, 3)]:
        up = q[k, j + 1, i] if j + 1 < ny else -q[k, j, i]
        dn = q[k, j - 1, i] if j > 0 else q[k, j, i]
        ref = ((q[k, j, (i + 1) % nx] - 2 * q[k, j, i] + q[k, j, i - 1]) / h[0] ** 2
               + (up - 2 * q[k, j, i] + dn) / h[1] ** 2
               + (q[(k + 1) % nz, j, i] - 2 * q[k, j, i] + q[k - 1, j, i]) / h[2] ** 2)
        assert abs(ref - lap[k, j, i]) < 1e-12 * np.max(np.abs(lap))
    f = np.random.default_rng(4).standard_normal(shape) + 3.0  # any mean: nothing is dropped
    mat = O.dense_operator(lambda p: O.laplacian(p, h, OUT), shape)
    dense = np.linalg.solve(mat, f.ravel()).reshape(shape)
    assert O.rel_linf(O.ppe_solve(f, LENGTHS, OUT), dense) < 1e-12


@pytest.mark.parametrize("rule", [O.FACE_ARITHMETIC, O.FACE_HARMONIC])
def test_outflow_divergence_identity_and_split_exactness(rule):
    """With an open top, D u^{n+1} = S holds for any S (no compatibility
    condition), the top-face velocity is corrected, and O7 holds: with
    p^n = p^{n-1} = q solving the unsplit Eq. (30) the split returns q."""
    fl = _fields(n=(8, 6, 10), seed=12, width=2.0)
    h = O.spacings(fl.shape, LENGTHS)
    S = fl.S + 0.3  # a net expansion, which walls could not absorb
    out = O.ppe_project(fl.u, fl.v, fl.w, S, fl.rho, fl.p_n, fl.p_nm1, fl.dt, LENGTHS, rule=rule, bc_top=OUT)
    div_new = O.div(out["u"], out["v"], out["w"], h)
    assert np.max(np.abs(div_new - S)) < 1e-11 * np.max(np.abs(O.div(fl.u, fl.v, fl.w, h)))
    assert np.all(out["v"][:, 0, :] == fl.v[:, 0, :])
    assert not np.allclose(out["v"][:, -1, :], fl.v[:, -1, :])
    src = (O.div(fl.u, fl.v, fl.w, h) - S) / fl.dt
    q = O.var_coeff_solve_dense(src, fl.rho, LENGTHS, rule, OUT)
    out2 = O.ppe_project(fl.u, fl.v, fl.w, S, fl.rho, q, q, fl.dt, LENGTHS, rule=rule, bc_top=OUT)
    assert O.rel_linf(out2["p"], q) < 1e-11


def test_planted_outflow_eigenvalue_mistake_is_caught(monkeypatch):
    """Solving the outflow problem with the wall (DCT-II) eigenvalues must fail
    the manufactured eigenfunction."""
    good = O.eigenvalues
    monkeypatch.setattr(O, "eigenvalues", lambda shape, lengths, bc_top=O.BC_WALL: good(shape, lengths))
    shape = (6, 5, 4)
    nz, ny, nx = shape
    h = O.spacings(shape, LENGTHS)
    phi = np.broadcast_to(np.cos(math.pi * 1.5 * (np.arange(ny) + 0.5) / ny)[None, :, None], shape).copy()
    lam = -(4 / h[1] ** 2) * math.sin(math.pi * 1.5 / (2 * ny)) ** 2
    with np.errstate(divide="ignore", invalid="ignore"):  # the wall table has a zero eigenvalue
        err = O.rel_linf(O.ppe_solve(lam * phi, LENGTHS, OUT), phi)
    assert not err < 1e-3
