"""FP64 oracle of the split pressure-gradient projection, Sec. 5.4 of
Poblador-Ibanez & Sirignano (arXiv 2103.01874).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may use this module.  It shares no code with the CUDA path.

The method reaches its result exactly (a direct, non-iterative solve of the
constant-coefficient Poisson equation, Sec. 5.4 text after Eq. (34)), so this
module is the plain definition of that discrete result, written with numpy and
scipy library transforms as steps:

  p_hat  = 2 p^n - p^{n-1}                                  Eq. (32)
  rho_0  = min(rho)                                          Eq. (32) text
  f      = D[(1 - rho_0/rho_f) G p_hat] + (rho_0/dt)(D u* - S)   Eq. (34)
  L p    = f,  L = D G,  mean(p) = 0                         Eq. (34)
  u^{n+1} = u* - dt [G p / rho_0 + (1/rho_f - 1/rho_0) G p_hat]   Eq. (33)

Discretisation ("standard finite-volume techniques" on the uniform staggered
mesh, Sec. 5 and the paragraph after Eq. (34)):
  G  cell -> face difference; zero on the two wall planes of y (Neumann);
  D  face -> cell divergence;  L = D G is the 7-point Laplacian;
  rho_f the face density, arithmetic mean of the two cells (default) or
        harmonic mean (option) -- the paper leaves the face rule for rho open.
Periodic in x and z, walls (homogeneous Neumann for p) in y.

The solve diagonalises L exactly: DFT in x and z (numpy.fft), DCT-II in y
(scipy.fft, orthonormal), divide by the eigenvalues
  lam = -(4/dx^2) sin^2(pi kx/Nx) - (4/dy^2) sin^2(pi ky/(2 Ny)) - (4/dz^2) sin^2(pi kz/Nz)
and drop the zero mode, which makes p the zero-mean least-squares solution.

Pins (tests/test_oracle_pins.py): discrete eigenfunctions, a brute-force
7-point stencil, dense LU of L on small grids, the divergence identity
D u^{n+1} = S, the constant-density limit, split exactness when
p^n = p^{n-1} solves Eq. (30), zero mean, and shift/reflection symmetry.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

FACE_ARITHMETIC = 0
FACE_HARMONIC = 1

# top boundary in y (the bottom, y = 0, is always a wall)
BC_WALL = 0      # no penetration, homogeneous Neumann for p
BC_OUTFLOW = 1   # open boundary: p = 0 on the top face (the paper's outflow
                 # condition of its jet cases, Sec. 6); v there is not fixed


def spacings(shape, lengths):
    nz, ny, nx = shape
    lx, ly, lz = lengths
    return lx / nx, ly / ny, lz / nz


# ----------------------------------------------------------------------------
# Discrete operators on the staggered mesh (Sec. 5, uniform MAC grid)
# ----------------------------------------------------------------------------

def grad(q, h, bc_top=BC_WALL):
    """G: cell field [Nz][Ny][Nx] -> face fields (gx [Nz][Ny][Nx],
    gy [Nz][Ny+1][Nx], gz [Nz][Ny][Nx]).  gx[..., i] = (q_i - q_{i-1})/dx with
    periodic wrap; gy on the walls j = 0, Ny is zero (homogeneous Neumann).
    With an outflow top, q = 0 on the face j = Ny, half a cell above the last
    centre: gy[Ny] = (0 - q_{Ny-1}) / (dy/2)."""
    dx, dy, dz = h
    nz, ny, nx = q.shape
    gx = (q - np.roll(q, 1, axis=2)) / dx
    gz = (q - np.roll(q, 1, axis=0)) / dz
    gy = np.zeros((nz, ny + 1, nx))
    gy[:, 1:ny, :] = (q[:, 1:, :] - q[:, :-1, :]) / dy
    if bc_top == BC_OUTFLOW:
        gy[:, ny, :] = -2.0 * q[:, ny - 1, :] / dy
    return gx, gy, gz


def div(a, b, c, h):
    """D: face fields -> cell field.  (a_{i+1} - a_i)/dx + (b_{j+1} - b_j)/dy
    + (c_{k+1} - c_k)/dz, periodic in i and k."""
    dx, dy, dz = h
    return ((np.roll(a, -1, axis=2) - a) / dx
            + (b[:, 1:, :] - b[:, :-1, :]) / dy
            + (np.roll(c, -1, axis=0) - c) / dz)


def laplacian(q, h, bc_top=BC_WALL):
    """L = D G, the 7-point operator of Eq. (34)'s left side."""
    return div(*grad(q, h, bc_top), h)


def face_density(rho, rule=FACE_ARITHMETIC):
    """rho on the faces.  Wall faces of y get the adjacent cell's value; they
    are never used because G = 0 there."""
    nz, ny, nx = rho.shape
    left_x = np.roll(rho, 1, axis=2)
    left_z = np.roll(rho, 1, axis=0)
    ry = np.empty((nz, ny + 1, nx))
    ry[:, 0, :] = rho[:, 0, :]
    ry[:, ny, :] = rho[:, ny - 1, :]
    lo, hi = rho[:, :-1, :], rho[:, 1:, :]
    if rule == FACE_ARITHMETIC:
        rx = 0.5 * (left_x + rho)
        rz = 0.5 * (left_z + rho)
        ry[:, 1:ny, :] = 0.5 * (lo + hi)
    elif rule == FACE_HARMONIC:
        rx = 2.0 / (1.0 / left_x + 1.0 / rho)
        rz = 2.0 / (1.0 / left_z + 1.0 / rho)
        ry[:, 1:ny, :] = 2.0 / (1.0 / lo + 1.0 / hi)
    else:
        raise ValueError("face rule")
    return rx, ry, rz


def rho0_of(rho):
    """rho_0 = min(rho), the text after Eq. (32)."""
    return float(np.min(rho))


# ----------------------------------------------------------------------------
# Eq. (34): right-hand side
# ----------------------------------------------------------------------------

def ppe_rhs(u, v, w, S, rho, p_n, p_nm1, rho0, dt, lengths, rule=FACE_ARITHMETIC, bc_top=BC_WALL):
    """f = D[(1 - rho_0/rho_f) G p_hat] + (rho_0/dt)(D u* - S), Eq. (34), with
    p_hat = 2 p^n - p^{n-1} (Eq. (32))."""
    h = spacings(rho.shape, lengths)
    p_hat = 2.0 * p_n - p_nm1
    gx, gy, gz = grad(p_hat, h, bc_top)
    rx, ry, rz = face_density(rho, rule)
    split = div((1.0 - rho0 / rx) * gx, (1.0 - rho0 / ry) * gy, (1.0 - rho0 / rz) * gz, h)
    return split + (rho0 / dt) * (div(u, v, w, h) - S)


# ----------------------------------------------------------------------------
# Eq. (34): direct solve of L p = f (the paper's FFT Poisson solver)
# ----------------------------------------------------------------------------

def compatibility(v, S, lengths):
    """Solvability of the Neumann problem L p = f (Sec. 5.4, Eq. (34)): the sum of
    f over the cells must vanish.  Summing D over the cells leaves only the wall
    faces of y (x and z are periodic), and G vanishes on the walls, so
    mean(f) = (rho_0/dt) (wall_flux_mean - mean(S)) with
    wall_flux_mean = sum over (i, k) of (v[:, Ny, :] - v[:, 0, :]) / (dy Nx Ny Nz).
    Returns the plain definitions: dict(s_mean, s_absmax, wall_flux_mean, wall_vmax)."""
    nz, ny, nx = S.shape
    dy = lengths[1] / ny
    wall = np.concatenate([v[:, 0, :].ravel(), v[:, ny, :].ravel()])
    return dict(s_mean=float(S.sum() / S.size), s_absmax=float(np.abs(S).max()),
                wall_flux_mean=float((v[:, ny, :] - v[:, 0, :]).sum() / (dy * S.size)),
                wall_vmax=float(np.abs(wall).max()))


def eigenvalues(shape, lengths, bc_top=BC_WALL):
    """Eigenvalues of L for the Fourier (x, z) x cosine (y) modes, shape
    [Nz][Ny][Nx//2+1] matching rfft in x, full fft in z, and in y DCT-II
    (walls: cos(pi k (j + 1/2)/Ny)) or DCT-IV (outflow top:
    cos(pi (k + 1/2)(j + 1/2)/Ny), which vanish on the top face)."""
    nz, ny, nx = shape
    dx, dy, dz = spacings(shape, lengths)
    kx = np.arange(nx // 2 + 1)
    ky = np.arange(ny) + (0.5 if bc_top == BC_OUTFLOW else 0.0)
    kz = np.arange(nz)
    lx = -(4.0 / dx**2) * np.sin(math.pi * kx / nx) ** 2
    ly = -(4.0 / dy**2) * np.sin(math.pi * ky / (2 * ny)) ** 2
    lz = -(4.0 / dz**2) * np.sin(math.pi * kz / nz) ** 2
    return lz[:, None, None] + ly[None, :, None] + lx[None, None, :]


def ppe_solve(f, lengths, bc_top=BC_WALL):
    """Walls: zero-mean p with L p = f - mean(f) (the zero mode is dropped).
    Outflow top: the unique p with L p = f (no zero mode)."""
    nz, ny, nx = f.shape
    fh = np.fft.rfft(f, axis=2)
    fh = np.fft.fft(fh, axis=0)
    if bc_top == BC_OUTFLOW:
        fh = sfft.dct(fh, type=4, axis=1, norm="ortho")
        ph = fh / eigenvalues(f.shape, lengths, bc_top)
        ph = sfft.idct(ph, type=4, axis=1, norm="ortho")
        ph = np.fft.ifft(ph, axis=0)
        return np.fft.irfft(ph, n=nx, axis=2)
    fh = sfft.dct(fh, type=2, axis=1, norm="ortho")
    lam = eigenvalues(f.shape, lengths)
    lam[0, 0, 0] = 1.0
    ph = fh / lam
    ph[0, 0, 0] = 0.0
    ph = sfft.idct(ph, type=2, axis=1, norm="ortho")
    ph = np.fft.ifft(ph, axis=0)
    return np.fft.irfft(ph, n=nx, axis=2)


def residual(f, p, lengths, bc_top=BC_WALL):
    h = spacings(f.shape, lengths)
    return f - laplacian(p, h, bc_top)


# ----------------------------------------------------------------------------
# Eq. (33): velocity correction
# ----------------------------------------------------------------------------

def ppe_correct(u, v, w, rho, p, p_n, p_nm1, rho0, dt, lengths, rule=FACE_ARITHMETIC, bc_top=BC_WALL):
    """u^{n+1} = u* - dt [G p / rho_0 + (1/rho_f - 1/rho_0) G p_hat] on every
    face, Eq. (33).  On the wall faces G = 0, so v is returned unchanged there;
    an outflow top face is corrected like an interior face."""
    h = spacings(rho.shape, lengths)
    p_hat = 2.0 * p_n - p_nm1
    gpx, gpy, gpz = grad(p, h, bc_top)
    ghx, ghy, ghz = grad(p_hat, h, bc_top)
    rx, ry, rz = face_density(rho, rule)
    u1 = u - dt * (gpx / rho0 + (1.0 / rx - 1.0 / rho0) * ghx)
    v1 = v - dt * (gpy / rho0 + (1.0 / ry - 1.0 / rho0) * ghy)
    w1 = w - dt * (gpz / rho0 + (1.0 / rz - 1.0 / rho0) * ghz)
    return u1, v1, w1


def ppe_project(u, v, w, S, rho, p_n, p_nm1, dt, lengths, rho0=None, rule=FACE_ARITHMETIC, bc_top=BC_WALL):
    """The whole projection step: returns dict(f, p, u, v, w, rho0)."""
    if rho0 is None or rho0 <= 0.0:
        rho0 = rho0_of(rho)
    f = ppe_rhs(u, v, w, S, rho, p_n, p_nm1, rho0, dt, lengths, rule, bc_top)
    p = ppe_solve(f, lengths, bc_top)
    u1, v1, w1 = ppe_correct(u, v, w, rho, p, p_n, p_nm1, rho0, dt, lengths, rule, bc_top)
    return dict(f=f, p=p, u=u1, v=v1, w=w1, rho0=rho0)


def project_fields(fl, rule=FACE_ARITHMETIC, rho0=None, bc_top=BC_WALL):
    """ppe_project on a paper_2103_01874_gb300.fields.Fields-like object."""
    return ppe_project(fl.u, fl.v, fl.w, fl.S, fl.rho, fl.p_n, fl.p_nm1, fl.dt,
                       (fl.lx, fl.ly, fl.lz), rho0=rho0, rule=rule, bc_top=bc_top)


# ----------------------------------------------------------------------------
# Eq. (30): the unsplit variable-coefficient equation (exactness reference)
# ----------------------------------------------------------------------------

def var_coeff_apply(q, rho, lengths, rule=FACE_ARITHMETIC, bc_top=BC_WALL):
    """A q = D[(1/rho_f) G q], the left side of Eq. (30)."""
    h = spacings(rho.shape, lengths)
    gx, gy, gz = grad(q, h, bc_top)
    rx, ry, rz = face_density(rho, rule)
    return div(gx / rx, gy / ry, gz / rz, h)


def dense_operator(apply, shape):
    """Columns of a linear cell-field operator, by applying it to unit cells."""
    n = int(np.prod(shape))
    mat = np.empty((n, n))
    e = np.zeros(n)
    for c in range(n):
        e[c] = 1.0
        mat[:, c] = apply(e.reshape(shape)).ravel()
        e[c] = 0.0
    return mat


def dense_zero_mean_solve(mat, rhs):
    """Solve mat x = rhs - mean(rhs) with sum(x) = 0 by dense LU of the system
    bordered with the constant vector (mat has the constants as null space)."""
    n = mat.shape[0]
    big = np.zeros((n + 1, n + 1))
    big[:n, :n] = mat
    big[:n, n] = 1.0
    big[n, :n] = 1.0
    b = np.zeros(n + 1)
    b[:n] = rhs.ravel() - rhs.mean()
    return np.linalg.solve(big, b)[:n].reshape(rhs.shape)


def var_coeff_solve_dense(rhs, rho, lengths, rule=FACE_ARITHMETIC, bc_top=BC_WALL):
    """q with D[(1/rho_f) G q] = rhs (Eq. (30)) by dense LU (small grids): the
    zero-mean solution for walls, the unique one for an outflow top."""
    mat = dense_operator(lambda q: var_coeff_apply(q, rho, lengths, rule, bc_top), rho.shape)
    if bc_top == BC_OUTFLOW:
        return np.linalg.solve(mat, rhs.ravel()).reshape(rhs.shape)
    return dense_zero_mean_solve(mat, rhs)


def unsplit_rhs(u, v, w, S, dt, lengths):
    """Right side of Eq. (30): (D u* - S) / dt."""
    h = spacings(S.shape, lengths)
    return (div(u, v, w, h) - S) / dt


def unsplit_correct(u, v, w, rho, p, dt, lengths, rule=FACE_ARITHMETIC):
    """u^{n+1} = u* - dt G p / rho_f on every face, Eq. (29) (G = 0 on the walls)."""
    h = spacings(rho.shape, lengths)
    gx, gy, gz = grad(p, h)
    rx, ry, rz = face_density(rho, rule)
    return u - dt * gx / rx, v - dt * gy / ry, w - dt * gz / rz


def unsplit_project_dense(u, v, w, S, rho, dt, lengths, rule=FACE_ARITHMETIC):
    """The unsplit projection, Eqs. (29)-(30), with the variable-coefficient
    equation solved exactly by dense LU (zero-mean p): small grids only.
    Returns dict(g, p, u, v, w), g the right side of Eq. (30)."""
    g = unsplit_rhs(u, v, w, S, dt, lengths)
    p = var_coeff_solve_dense(g, rho, lengths, rule)
    u1, v1, w1 = unsplit_correct(u, v, w, rho, p, dt, lengths, rule)
    return dict(g=g, p=p, u=u1, v=v1, w=w1)


def unsplit_residual(p, g, rho, lengths, rule=FACE_ARITHMETIC):
    """||(g - mean g) - A p||_inf / ||g - mean g||_inf for Eq. (30)."""
    gc = g - g.mean()
    r = gc - var_coeff_apply(p, rho, lengths, rule)
    return float(np.max(np.abs(r)) / np.max(np.abs(gc)))


# ----------------------------------------------------------------------------
# Eq. (31): the divergence constraint S from the phase-wise quantities
# ----------------------------------------------------------------------------

def divergence_constraint(C, comp_g, comp_l, mdot, rho_g, rho_l, under_resolved=None):
    """S = div u^{n+1} = -(1 - C) comp_g - C comp_l + mdot (1/rho_g - 1/rho_l),
    Eq. (31), with comp_f = (1/rho_f) D rho_f / Dt the phase compressibilities
    and mdot the volumetric phase-change rate (> 0 for liquid turning into gas).
    In under-resolved interface cells (mask set and 0 < C < 1) the one-fluid
    divergence is set to zero (the treatment of under-resolved regions in the
    extrapolation section of the paper).  Also returns the one-fluid density
    rho = rho_g (1 - C) + rho_l C of the volume-fraction substitution that
    precedes Eq. (31)."""
    S = -(1.0 - C) * comp_g - C * comp_l + mdot * (1.0 / rho_g - 1.0 / rho_l)
    if under_resolved is not None:
        S = np.where((under_resolved != 0) & (C > 0.0) & (C < 1.0), 0.0, S)
    rho = rho_g * (1.0 - C) + rho_l * C
    return S, rho


def rel_linf(a, b):
    """max|a - b| / max|b|."""
    a = np.asarray(a)
    b = np.asarray(b)
    den = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / (den if den > 0 else 1.0)
