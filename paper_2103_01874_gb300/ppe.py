"""ctypes binding of libppe (include/ppe.h): argument marshalling only.

Every step of the projection runs in the library's CUDA kernels; this module
checks tensor shapes, dtypes and devices, passes raw device pointers, and
raises PPEError on a non-zero status.  It loads the in-tree
paper_2103_01874_gb300/_native/libppe.so and raises RuntimeError if that
library is missing: there is no host fallback.

Field layout is that of the C ABI: torch float64 tensors, C-contiguous,
cell fields shaped (nz, ny, nx), v shaped (nz, ny + 1, nx).
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, c_double, c_int, c_size_t, c_void_p

from . import build as _build

FP64 = 0
FP32_REFINE = 1
FACE_ARITHMETIC = 0
FACE_HARMONIC = 1
BC_WALL = 0      # top boundary in y: wall (ppe_bc)
BC_OUTFLOW = 1   # open top, p = 0 on the face
# schedules of the spectral z and y steps (ppe_tuning.spectral)
SPECTRAL_LEGACY = 0  # three passes, spectrum [kz][j][kx]
SPECTRAL_FUSED = 1   # one cluster pass per kx plane
SPECTRAL_PENCIL = 2  # three bulk-copy-staged persistent passes, spectrum [kx][kz][j]
# y step of the LEGACY schedule (ppe_tuning.y_solve)
Y_COSINE = 0       # DCT-II, eigenvalue divide, DCT-III through FFTs
Y_TRIDIAGONAL = 1  # Thomas elimination as two affine scans (FP32 with walls, ny <= 512)
# forms of a batch (ppe_batch_options.form)
BATCH_AUTO = 0        # persistent where every plan qualifies, else graph
BATCH_GRAPH = 1       # graph branches, one per projection
BATCH_PERSISTENT = 2  # one persistent kernel over a device work queue

STATUS = {0: "PPE_OK", 1: "PPE_ERR_INVALID_ARG", 2: "PPE_ERR_UNSUPPORTED_SIZE", 3: "PPE_ERR_INCOMPATIBLE_RHS",
          4: "PPE_ERR_OUT_OF_MEMORY", 5: "PPE_ERR_NOT_CONVERGED", 6: "PPE_ERR_TIMEOUT", 7: "PPE_ERR_CUDA"}


class PPEError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({_strerror(code)})")


class Grid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("lx", c_double), ("ly", c_double), ("lz", c_double)]


class Options(ctypes.Structure):
    _fields_ = [("precision", c_int), ("face_rule", c_int), ("refine_tol", c_double), ("max_sweeps", c_int),
                ("compat_tol", c_double), ("bc_top", c_int)]


class Info(ctypes.Structure):
    _fields_ = [("sweeps", c_int), ("rel_residual", c_double), ("f_max", c_double), ("rho0", c_double),
                ("s_mean", c_double), ("s_absmax", c_double), ("wall_flux_mean", c_double), ("wall_vmax", c_double),
                ("f_mean_removed", c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("rhs_lines", c_int), ("rhs_planes", c_int), ("x_lines", c_int), ("z_cols", c_int),
                ("y_cols", c_int), ("spectral", c_int), ("y_solve", c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchOptions(ctypes.Structure):
    _fields_ = [("form", c_int), ("window", c_int), ("stagger", c_int), ("ctas_per_sm", c_int),
                ("wait_seconds", c_double), ("test_unset_wait", c_int), ("grain", c_int)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", c_int), ("total_ms", c_double)]


class FieldsC(ctypes.Structure):
    _fields_ = [("u", c_void_p), ("v", c_void_p), ("w", c_void_p), ("S", c_void_p), ("rho", c_void_p),
                ("p_n", c_void_p), ("p_nm1", c_void_p), ("rho0", c_double), ("dt", c_double),
                ("p", c_void_p), ("u_out", c_void_p), ("v_out", c_void_p), ("w_out", c_void_p), ("f", c_void_p)]


_LIB = None

# name -> (restype, argtypes), mirroring include/ppe.h
SIGNATURES = {
    "ppe_plan": (c_int, [POINTER(c_void_p), POINTER(Grid), POINTER(Options), c_void_p]),
    "ppe_set_stream": (c_int, [c_void_p, c_void_p]),
    "ppe_workspace_bytes": (c_size_t, [POINTER(Grid), POINTER(Options)]),
    "ppe_rhs": (c_int, [c_void_p] + [c_void_p] * 7 + [c_double, c_double, c_void_p]),
    "ppe_solve": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ppe_correct": (c_int, [c_void_p] + [c_void_p] * 7 + [c_double, c_double] + [c_void_p] * 3),
    "ppe_project": (c_int, [c_void_p, POINTER(FieldsC)]),
    "ppe_project_host": (c_int, [c_void_p, POINTER(FieldsC)]),
    "ppe_project_host_async": (c_int, [c_void_p, POINTER(FieldsC)]),
    "ppe_host_wait": (c_int, [c_void_p]),
    "ppe_get_info": (c_int, [c_void_p, POINTER(Info)]),
    "ppe_destroy": (None, [c_void_p]),
    "ppe_strerror": (ctypes.c_char_p, [c_int]),
    "ppe_size_supported": (c_int, [c_int, c_int, c_int]),
    "ppe_profile": (c_int, [c_void_p, c_int]),
    "ppe_rho0_noalloc": (c_int, [c_void_p, c_size_t, c_void_p, c_void_p]),
    "ppe_get_tuning": (c_int, [c_void_p, POINTER(Tuning)]),
    "ppe_batch_create": (c_int, [POINTER(c_void_p), c_int, POINTER(c_void_p), POINTER(FieldsC), c_void_p]),
    "ppe_batch_launch": (c_int, [c_void_p]),
    "ppe_batch_destroy": (None, [c_void_p]),
    "ppe_project_batched": (c_int, [c_int, POINTER(c_void_p), POINTER(FieldsC), c_void_p]),
    "ppe_batch_create_ex": (c_int, [POINTER(c_void_p), c_int, POINTER(c_void_p), POINTER(FieldsC), c_void_p,
                                    POINTER(BatchOptions)]),
    "ppe_batch_status": (c_int, [c_void_p, POINTER(c_int), POINTER(ctypes.c_longlong), POINTER(c_int),
                                 POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "ppe_batch_schedule": (ctypes.c_longlong, [c_int, POINTER(c_int), POINTER(c_int), c_int, c_int, c_int, c_int,
                                               POINTER(c_int), ctypes.c_longlong, POINTER(c_int), POINTER(c_int)]),
    "ppe_set_tuning": (c_int, [c_void_p, POINTER(Tuning)]),
    "ppe_profile_read": (c_int, [c_void_p, POINTER(KernelTime), c_int]),
    "ppe_project_unsplit": (c_int, [c_void_p, POINTER(FieldsC), c_double, c_int]),
    "ppe_unsplit_info": (c_int, [c_void_p, POINTER(c_int), POINTER(c_double)]),
    "ppe_divergence_constraint": (c_int, [c_void_p] + [c_void_p] * 9),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libppe.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libppe.so not found at {path}: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _strerror(code: int) -> str:
    try:
        return lib().ppe_strerror(code).decode()
    except Exception:  # pragma: no cover
        return "?"


def size_supported(nx: int, ny: int, nz: int) -> bool:
    return bool(lib().ppe_size_supported(nx, ny, nz))


def _check(code: int, where: str):
    if code != 0:
        raise PPEError(code, where)


def _ptr(t, shape, name):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name}: need a contiguous float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")
    return t.data_ptr()


def _hptr(a, shape, name):
    """Host buffer (numpy float64 C-contiguous or pinned torch CPU tensor)."""
    import numpy as np
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous or tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name}: need a C-contiguous float64 array of shape {shape}")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or a.is_cuda or not a.is_contiguous() or tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name}: need a contiguous float64 CPU tensor of shape {shape}")
        return a.data_ptr()
    raise TypeError(name)


RHO0_NOALLOC_MAX = 16384 * 4096


def rho0_noalloc(rho, out, stream=None):
    """ppe_rho0_noalloc: min(rho) into the one-element float64 CUDA tensor
    `out`, using the library's static scratch instead of any allocation (for
    callers that cannot allocate device memory).  Asynchronous on `stream`."""
    import torch
    if not (isinstance(rho, torch.Tensor) and rho.is_cuda and rho.dtype == torch.float64 and rho.is_contiguous()):
        raise ValueError("rho: need a contiguous float64 CUDA tensor")
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64 and out.numel() >= 1):
        raise ValueError("out: need a float64 CUDA tensor with at least one element")
    if rho.numel() > RHO0_NOALLOC_MAX:
        raise ValueError(f"rho has {rho.numel()} values; the static scratch of ppe_rho0_noalloc "
                         f"holds at most {RHO0_NOALLOC_MAX}")
    _check(lib().ppe_rho0_noalloc(rho.data_ptr(), rho.numel(), out.data_ptr(),
                                  c_void_p(_stream_handle(stream))), "ppe_rho0_noalloc")


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Batch:
    """ppe_batch_create / ppe_batch_launch: the projections of many plans (any
    grid sizes) captured once into one CUDA graph and replayed with one launch.
    `items` is a list of (plan, dict of tensors u, v, w, S, rho, p_n, p_nm1, p,
    u_out, v_out, w_out [, f], dt [, rho0])."""

    def __init__(self, items, stream=None, form=BATCH_GRAPH, window=0, stagger=-1, ctas_per_sm=0,
                 wait_seconds=0.0, test_unset_wait=False, grain=0):
        n = len(items)
        self._keep = items  # tensors must outlive the graph
        plans = (c_void_p * n)(*[pl._h.value for pl, _ in items])
        flds = (FieldsC * n)()
        for i, (pl, d) in enumerate(items):
            flds[i] = pl._fields(_ptr, d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], d["dt"],
                                 d["p"], d["u_out"], d["v_out"], d["w_out"], d.get("f"), d.get("rho0", -1.0))
        opt = BatchOptions(int(form), int(window), int(stagger), int(ctas_per_sm), float(wait_seconds),
                           1 if test_unset_wait else 0, int(grain))
        h = c_void_p()
        _check(lib().ppe_batch_create_ex(ctypes.byref(h), n, plans, flds, c_void_p(_stream_handle(stream)),
                                         ctypes.byref(opt)), "ppe_batch_create_ex")
        self._h = h
        self.n = n

    def launch(self):
        _check(lib().ppe_batch_launch(self._h), "ppe_batch_launch")

    def status(self, check=True):
        """Synchronise and read the last launch's status: a dict with form,
        items, ctas, launches, status (PPE_* code), err_grid, err_stage."""
        form, ctas, nl, eg, es = c_int(), c_int(), c_int(), c_int(), c_int()
        items = ctypes.c_longlong()
        code = lib().ppe_batch_status(self._h, ctypes.byref(form), ctypes.byref(items), ctypes.byref(ctas),
                                      ctypes.byref(nl), ctypes.byref(eg), ctypes.byref(es))
        if check and code not in (0, 6):
            _check(code, "ppe_batch_status")
        return {"form": form.value, "items": items.value, "ctas": ctas.value, "launches": nl.value,
                "status": code, "err_grid": eg.value, "err_stage": es.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ppe_batch_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Plan:
    """A libppe plan for one grid (ppe_plan / ppe_destroy)."""

    def __init__(self, nx, ny, nz, lx=2 * math.pi, ly=2 * math.pi, lz=2 * math.pi, precision=FP64,
                 face_rule=FACE_ARITHMETIC, refine_tol=1e-10, max_sweeps=6, stream=None, compat_tol=1e-12,
                 bc_top=None):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.lengths = (lx, ly, lz)
        self.precision = precision
        self.grid = Grid(nx, ny, nz, lx, ly, lz)
        self.bc_top = BC_WALL if bc_top is None else bc_top
        self.opts = Options(precision, face_rule, refine_tol, max_sweeps, compat_tol, self.bc_top)
        self._async_refs = []  # host buffers of enqueued project_host_async calls
        h = c_void_p()
        _check(lib().ppe_plan(ctypes.byref(h), ctypes.byref(self.grid), ctypes.byref(self.opts),
                              c_void_p(_stream_handle(stream))), "ppe_plan")
        self._h = h

    # shapes
    @property
    def cell_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def v_shape(self):
        return (self.nz, self.ny + 1, self.nx)

    def workspace_bytes(self) -> int:
        return int(lib().ppe_workspace_bytes(ctypes.byref(self.grid), ctypes.byref(self.opts)))

    def set_stream(self, stream):
        _check(lib().ppe_set_stream(self._h, c_void_p(_stream_handle(stream))), "ppe_set_stream")

    def rhs(self, u, v, w, S, rho, p_n, p_nm1, dt, f, rho0=-1.0):
        c, vs = self.cell_shape, self.v_shape
        _check(lib().ppe_rhs(self._h, _ptr(u, c, "u"), _ptr(v, vs, "v"), _ptr(w, c, "w"), _ptr(S, c, "S"),
                             _ptr(rho, c, "rho"), _ptr(p_n, c, "p_n"), _ptr(p_nm1, c, "p_nm1"),
                             float(rho0), float(dt), _ptr(f, c, "f")), "ppe_rhs")

    def solve(self, f, p):
        c = self.cell_shape
        _check(lib().ppe_solve(self._h, _ptr(f, c, "f"), _ptr(p, c, "p")), "ppe_solve")

    def correct(self, u, v, w, rho, p, p_n, p_nm1, dt, u_out, v_out, w_out, rho0=-1.0):
        c, vs = self.cell_shape, self.v_shape
        _check(lib().ppe_correct(self._h, _ptr(u, c, "u"), _ptr(v, vs, "v"), _ptr(w, c, "w"),
                                 _ptr(rho, c, "rho"), _ptr(p, c, "p"), _ptr(p_n, c, "p_n"),
                                 _ptr(p_nm1, c, "p_nm1"), float(rho0), float(dt),
                                 _ptr(u_out, c, "u_out"), _ptr(v_out, vs, "v_out"), _ptr(w_out, c, "w_out")),
               "ppe_correct")

    def _fields(self, conv, u, v, w, S, rho, p_n, p_nm1, dt, p, u_out, v_out, w_out, f=None, rho0=-1.0):
        c, vs = self.cell_shape, self.v_shape
        return FieldsC(conv(u, c, "u"), conv(v, vs, "v"), conv(w, c, "w"), conv(S, c, "S"), conv(rho, c, "rho"),
                       conv(p_n, c, "p_n"), conv(p_nm1, c, "p_nm1"), float(rho0), float(dt), conv(p, c, "p"),
                       conv(u_out, c, "u_out"), conv(v_out, vs, "v_out"), conv(w_out, c, "w_out"),
                       conv(f, c, "f"))

    def project(self, u, v, w, S, rho, p_n, p_nm1, dt, p, u_out, v_out, w_out, f=None, rho0=-1.0):
        fc = self._fields(_ptr, u, v, w, S, rho, p_n, p_nm1, dt, p, u_out, v_out, w_out, f, rho0)
        _check(lib().ppe_project(self._h, ctypes.byref(fc)), "ppe_project")

    def project_host(self, u, v, w, S, rho, p_n, p_nm1, dt, p, u_out, v_out, w_out, f=None, rho0=-1.0):
        fc = self._fields(_hptr, u, v, w, S, rho, p_n, p_nm1, dt, p, u_out, v_out, w_out, f, rho0)
        _check(lib().ppe_project_host(self._h, ctypes.byref(fc)), "ppe_project_host")

    def project_host_async(self, u, v, w, S, rho, p_n, p_nm1, dt, p, u_out, v_out, w_out, f=None, rho0=-1.0):
        """Enqueue a projection from host buffers (ppe_project_host_async); the
        buffers must stay untouched until host_wait()."""
        fc = self._fields(_hptr, u, v, w, S, rho, p_n, p_nm1, dt, p, u_out, v_out, w_out, f, rho0)
        _check(lib().ppe_project_host_async(self._h, ctypes.byref(fc)), "ppe_project_host_async")
        # the copies read and write these buffers until host_wait(): keep them alive
        self._async_refs.append((u, v, w, S, rho, p_n, p_nm1, p, u_out, v_out, w_out, f))

    def host_wait(self, allow_not_converged=False, allow_incompatible=False):
        """Wait for the enqueued host projections (ppe_host_wait)."""
        code = lib().ppe_host_wait(self._h)
        self._async_refs.clear()
        if (code == 5 and allow_not_converged) or (code == 3 and allow_incompatible):
            return code
        _check(code, "ppe_host_wait")
        return code

    def project_unsplit(self, u, v, w, S, rho, dt, p, u_out, v_out, w_out, tol=1e-10, max_iter=500):
        """The unsplit projection, Eqs. (29)-(30), by FFT-preconditioned CG (ppe_project_unsplit)."""
        fc = self._fields(_ptr, u, v, w, S, rho, None, None, dt, p, u_out, v_out, w_out)
        _check(lib().ppe_project_unsplit(self._h, ctypes.byref(fc), float(tol), int(max_iter)),
               "ppe_project_unsplit")

    def divergence_constraint(self, C, comp_g, comp_l, mdot, rho_g, rho_l, S, rho=None, under_resolved=None):
        """Eq. (31) into S (and the one-fluid density into rho); under_resolved a uint8 mask or None."""
        c = self.cell_shape
        mask = None
        if under_resolved is not None:
            import torch
            if under_resolved.dtype != torch.uint8 or not under_resolved.is_cuda or \
                    tuple(under_resolved.shape) != tuple(c) or not under_resolved.is_contiguous():
                raise ValueError("under_resolved: need a contiguous uint8 CUDA tensor of the cell shape")
            mask = under_resolved.data_ptr()
        _check(lib().ppe_divergence_constraint(self._h, _ptr(C, c, "C"), _ptr(comp_g, c, "comp_g"),
                                               _ptr(comp_l, c, "comp_l"), _ptr(mdot, c, "mdot"),
                                               _ptr(rho_g, c, "rho_g"), _ptr(rho_l, c, "rho_l"), mask,
                                               _ptr(S, c, "S"), _ptr(rho, c, "rho")), "ppe_divergence_constraint")

    def unsplit_info(self, allow_not_converged=False):
        """(iterations, relative residual) of the last unsplit projection."""
        it = c_int()
        rel = c_double()
        code = lib().ppe_unsplit_info(self._h, ctypes.byref(it), ctypes.byref(rel))
        if not (code == 5 and allow_not_converged):
            _check(code, "ppe_unsplit_info")
        return it.value, rel.value

    def info(self, allow_not_converged=False, allow_incompatible=False) -> Info:
        inf = Info()
        code = lib().ppe_get_info(self._h, ctypes.byref(inf))
        if (code == 5 and allow_not_converged) or (code == 3 and allow_incompatible):
            return inf
        _check(code, "ppe_get_info")
        return inf

    def get_tuning(self) -> dict:
        t = Tuning()
        _check(lib().ppe_get_tuning(self._h, ctypes.byref(t)), "ppe_get_tuning")
        return t.as_dict()

    def set_tuning(self, **kw):
        """Change launch shapes (ppe_set_tuning); unspecified fields keep their value."""
        cur = self.get_tuning()
        cur.update(kw)
        t = Tuning(**cur)
        _check(lib().ppe_set_tuning(self._h, ctypes.byref(t)), "ppe_set_tuning")

    def profile(self, enable: bool):
        _check(lib().ppe_profile(self._h, 1 if enable else 0), "ppe_profile")

    def profile_read(self) -> dict:
        """{kernel name: (launches, total_ms)} since the last read (synchronises)."""
        buf = (KernelTime * 32)()
        n = lib().ppe_profile_read(self._h, buf, 32)
        if n < 0:
            raise PPEError(7, "ppe_profile_read")
        return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(n)}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ppe_destroy(self._h)  # waits for the plan's streams
            self._h = c_void_p()
            self._async_refs = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def batch_schedule(dims, rho_given, window=0, stagger=-1, first=0, grain=0):
    """Host-side queue of the persistent batched form (ppe_batch_schedule; no
    device work): returns (items, need, tiles) with items a list of (grid,
    stage, first tile, tiles) in queue order (first = 0: the whole projection;
    8: a further sweep), need and tiles the items and tiles of the 15 stages of
    every grid, grid after grid; None if a grid does not qualify."""
    n = len(dims)
    d = (c_int * (3 * n))(*[int(v) for t in dims for v in t])
    rg = (c_int * n)(*[1 if v else 0 for v in rho_given])
    args = (int(window), int(stagger), int(grain), int(first))
    m = lib().ppe_batch_schedule(n, d, rg, *args, None, 0, None, None)
    if m < 0:
        return None
    out = (c_int * (4 * max(m, 1)))()
    need, tiles = (c_int * (15 * n))(), (c_int * (15 * n))()
    m2 = lib().ppe_batch_schedule(n, d, rg, *args, out, m, need, tiles)
    assert m2 == m
    items = [tuple(out[4 * i:4 * i + 4]) for i in range(m)]
    return items, list(need), list(tiles)
