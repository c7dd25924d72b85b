"""ctypes binding of the C++ FP64 oracle (oracle/ppe_oracle.cpp).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may use this module.  It shares no code with the CUDA path.

The library is compiled in-tree with g++ (-O3, single-threaded, no fast-math)
into oracle/_native/libppe_oracle.so on first use, or by build().  Arrays are
numpy FP64 in the layout of the paper's staggered mesh as the rest of the
project uses it: cells [nz][ny][nx], v [nz][ny+1][nx].
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ppe_oracle.cpp")
OUT = os.path.join(HERE, "_native")
LIB = os.path.join(OUT, "libppe_oracle.so")
FLAGS = ["-O3", "-std=c++17", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off"]

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT, exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    r = subprocess.run(["g++", *FLAGS, SRC, "-o", tmp], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("g++ failed on the oracle:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        d = ctypes.POINTER(ctypes.c_double)
        i, f64 = ctypes.c_int, ctypes.c_double
        L.oracle_project.argtypes = [i, i, i, f64, f64, f64, i, i, i, d, d, d, d, d, d, d, f64, f64, i,
                                     d, d, d, d, d, d]
        L.oracle_rhs.argtypes = [i, i, i, f64, f64, f64, i, i, d, d, d, d, d, d, d, f64, f64, d]
        L.oracle_solve.argtypes = [i, i, i, f64, f64, f64, i, i, d, d]
        L.oracle_laplacian.argtypes = [i, i, i, f64, f64, f64, i, d, d]
        for name in ("oracle_fft", "oracle_dft_direct"):
            getattr(L, name).argtypes = [i, i, d, d, d, d]
        L.oracle_dct2.argtypes = [i, d, d]
        L.oracle_dct3.argtypes = [i, d, d]
        L.oracle_thomas.argtypes = [i, d, d, d, d, d]
        for name in ("oracle_project", "oracle_rhs", "oracle_solve", "oracle_laplacian", "oracle_fft",
                     "oracle_dft_direct", "oracle_dct2", "oracle_dct3", "oracle_thomas", "oracle_version"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _in(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ok(rc, what):
    if rc != 0:
        raise ValueError(f"{what}: invalid arguments")


def project(u, v, w, S, rho, p_n, p_nm1, dt, lengths, rho0=None, rule=0, bc_top=0, y_method=0, mutation=0):
    """The whole projection: dict(f, p, u, v, w, rho0), like ppe_oracle.ppe_project."""
    nz, ny, nx = rho.shape
    ins = [_in(a) for a in (u, v, w, S, rho, p_n, p_nm1)]
    f = np.empty((nz, ny, nx))
    p = np.empty_like(f)
    u1, v1, w1 = np.empty_like(ins[0]), np.empty_like(ins[1]), np.empty_like(ins[2])
    r0 = ctypes.c_double(0.0)
    rc = lib().oracle_project(nx, ny, nz, lengths[0], lengths[1], lengths[2], rule, bc_top, y_method,
                              *[_p(a) for a in ins], -1.0 if rho0 is None else float(rho0), float(dt), mutation,
                              _p(f), _p(p), _p(u1), _p(v1), _p(w1), ctypes.byref(r0))
    _ok(rc, "oracle_project")
    return dict(f=f, p=p, u=u1, v=v1, w=w1, rho0=r0.value)


def project_fields(fl, rule=0, rho0=None, bc_top=0, y_method=0, mutation=0):
    """project() on a paper_2103_01874_gb300.fields.Fields-like object."""
    return project(fl.u, fl.v, fl.w, fl.S, fl.rho, fl.p_n, fl.p_nm1, fl.dt, (fl.lx, fl.ly, fl.lz), rho0=rho0,
                   rule=rule, bc_top=bc_top, y_method=y_method, mutation=mutation)


def rhs(u, v, w, S, rho, p_n, p_nm1, rho0, dt, lengths, rule=0, bc_top=0):
    nz, ny, nx = rho.shape
    ins = [_in(a) for a in (u, v, w, S, rho, p_n, p_nm1)]
    f = np.empty((nz, ny, nx))
    _ok(lib().oracle_rhs(nx, ny, nz, *lengths, rule, bc_top, *[_p(a) for a in ins], float(rho0), float(dt), _p(f)),
        "oracle_rhs")
    return f


def solve(f, lengths, bc_top=0, y_method=0):
    nz, ny, nx = f.shape
    f = _in(f)
    p = np.empty_like(f)
    _ok(lib().oracle_solve(nx, ny, nz, *lengths, bc_top, y_method, _p(f), _p(p)), "oracle_solve")
    return p


def laplacian(q, lengths, bc_top=0):
    nz, ny, nx = q.shape
    q = _in(q)
    out = np.empty_like(q)
    _ok(lib().oracle_laplacian(nx, ny, nz, *lengths, bc_top, _p(q), _p(out)), "oracle_laplacian")
    return out


def fft(x, inverse=False):
    """Unscaled complex DFT of x (exp(-2 pi i k n/N); +i for inverse) by the oracle's FFT."""
    x = np.asarray(x, dtype=np.complex128)
    re, im = _in(x.real), _in(x.imag)
    ore, oim = np.empty_like(re), np.empty_like(im)
    _ok(lib().oracle_fft(len(x), 1 if inverse else -1, _p(re), _p(im), _p(ore), _p(oim)), "oracle_fft")
    return ore + 1j * oim


def dft_direct(x, inverse=False):
    """The same DFT by the O(N^2) sum."""
    x = np.asarray(x, dtype=np.complex128)
    re, im = _in(x.real), _in(x.imag)
    ore, oim = np.empty_like(re), np.empty_like(im)
    _ok(lib().oracle_dft_direct(len(x), 1 if inverse else -1, _p(re), _p(im), _p(ore), _p(oim)),
        "oracle_dft_direct")
    return ore + 1j * oim


def dct2(x):
    """X_k = sum_j x_j cos(pi k (j + 1/2)/N), through the oracle's FFT of the even extension."""
    x = _in(x)
    X = np.empty_like(x)
    _ok(lib().oracle_dct2(len(x), _p(x), _p(X)), "oracle_dct2")
    return X


def dct3(X):
    """The inverse of dct2: x_j = X_0/N + (2/N) sum_{k>=1} X_k cos(pi k (j + 1/2)/N)."""
    X = _in(X)
    x = np.empty_like(X)
    _ok(lib().oracle_dct3(len(X), _p(X), _p(x)), "oracle_dct3")
    return x


def thomas(sub, diag, sup, d):
    """Tridiagonal solve sub[j] x_{j-1} + diag[j] x_j + sup[j] x_{j+1} = d_j."""
    sub, diag, sup, d = (_in(a) for a in (sub, diag, sup, d))
    x = np.empty_like(d)
    _ok(lib().oracle_thomas(len(d), _p(sub), _p(diag), _p(sup), _p(d), _p(x)), "oracle_thomas")
    return x
