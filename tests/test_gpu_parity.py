"""Parity of the CUDA projection (through the C ABI) with the FP64 oracle.

Bars: FP64 path rel L-inf <= 1e-12 on f, p, u, v, w; FP32 solve + FP64
refinement: rel residual ||f - L p||_inf / ||f||_inf <= 1e-10 (checked on the
host in FP64 from the returned f and p), and p, u, v, w within 1e-11 of the
oracle (one sweep measures ~3e-13), p zero-mean like the oracle's.
"""
import math

import numpy as np
import pytest

from oracle import cpp
from oracle import ppe_oracle as O
from paper_2103_01874_gb300 import fields, ppe

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL_RES = 1e-10
TOL_REF = 1e-11   # FP32 solve + refinement, fields against the oracle


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    ppe.lib()


def _compare(fl, res, ref, tol, keys=("f", "p", "u", "v", "w")):
    errs = {k: O.rel_linf(res[k], ref[k]) for k in keys}
    for k, e in errs.items():
        assert e <= tol, f"{k}: rel L-inf {e:.3e} > {tol:.1e} ({fl.shape})"
    return errs


SHAPES = [
    ((32, 32, 32), "single", 2.0, (2 * math.pi,) * 3),
    ((8, 8, 8), "single", 2.0, (2 * math.pi,) * 3),             # smallest supported
    ((48, 24, 36), "multimode", 6.0, (2 * math.pi, 3.0, 5.0)),   # anisotropic, ragged CTA tiles
    ((18, 27, 54), "single", 2.0, (1.0, 2.0, 3.0)),              # radix-3 heavy, odd ny
    ((96, 16, 12), "multimode", 6.0, (2 * math.pi, 1.0, 0.7)),
]


@pytest.mark.parametrize("shape,recipe,width,lengths", SHAPES)
def test_project_fp64(shape, recipe, width, lengths):
    nx, ny, nz = shape
    fl = fields.make_fields(nx, ny, nz, seed=nx + ny + nz, recipe=recipe, width=width,
                            lx=lengths[0], ly=lengths[1], lz=lengths[2])
    ref = O.project_fields(fl)
    res, info = project_gpu(fl)
    _compare(fl, res, ref, TOL64)
    _compare(fl, res, cpp.project_fields(fl), TOL64)  # the C++ oracle (own FFT and Thomas) too
    assert info.rho0 == ref["rho0"]
    assert abs(res["p"].mean()) <= 1e-13 * np.abs(res["p"]).max()


@pytest.mark.parametrize("shape", [(32, 32, 32), (48, 24, 36), (18, 27, 54)])
@pytest.mark.parametrize("rule", [ppe.FACE_ARITHMETIC, ppe.FACE_HARMONIC])
def test_project_fp32_refine_vs_cpp_oracle(shape, rule):
    """The refinement form against the C++ oracle, both face rules."""
    fl = fields.make_fields(*shape, seed=sum(shape), recipe="multimode", width=4.0, rho_g=60.0)
    ref = cpp.project_fields(fl, rule=rule)
    res, info = project_gpu(fl, precision=ppe.FP32_REFINE, face_rule=rule)
    assert info.rel_residual <= TOL_RES
    assert O.rel_linf(res["f"], ref["f"]) <= TOL64
    for k in ("p", "u", "v", "w"):
        assert O.rel_linf(res[k], ref[k]) <= TOL_REF, k


@pytest.mark.parametrize("rule", [ppe.FACE_ARITHMETIC, ppe.FACE_HARMONIC])
def test_face_rules_and_given_rho0(rule):
    fl = fields.make_fields(24, 16, 32, seed=4, recipe="multimode", width=3.0)
    ref = O.project_fields(fl, rule=rule, rho0=100.0)
    res, info = project_gpu(fl, face_rule=rule, rho0=100.0)
    _compare(fl, res, ref, TOL64)
    assert info.rho0 == 100.0


def test_separate_entry_points_match_project():
    """ppe_rhs -> ppe_solve -> ppe_correct (in place) equals the oracle."""
    import torch
    fl = fields.make_fields(32, 24, 16, seed=8, recipe="multimode", width=4.0)
    ref = O.project_fields(fl)
    d = dev_fields(fl)
    f = torch.empty(fl.shape, dtype=torch.float64, device="cuda")
    p = torch.empty_like(f)
    with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz) as plan:
        plan.rhs(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt, f)
        plan.solve(f, p)
        plan.correct(d["u"], d["v"], d["w"], d["rho"], p, d["p_n"], d["p_nm1"], fl.dt, d["u"], d["v"], d["w"])
        torch.cuda.synchronize()
    res = dict(f=f.cpu().numpy(), p=p.cpu().numpy(), u=d["u"].cpu().numpy(), v=d["v"].cpu().numpy(),
               w=d["w"].cpu().numpy())
    _compare(fl, res, ref, TOL64)


def test_solve_manufactured_eigenfunction():
    """The GPU solve of lam * phi returns phi for a discrete eigenfunction."""
    import torch
    nz, ny, nx = 24, 12, 16
    L = (2 * math.pi, 3.0, 5.0)
    dx, dy, dz = L[0] / nx, L[1] / ny, L[2] / nz
    a, b, c = 3, 2, 5
    x = (np.arange(nx) + 0.5) * dx
    z = (np.arange(nz) + 0.5) * dz
    phi = (np.cos(2 * math.pi * a * x / L[0] + 0.3)[None, None, :] * np.cos(math.pi * b * (np.arange(ny) + 0.5) / ny)
           [None, :, None] * np.cos(2 * math.pi * c * z / L[2] - 1.1)[:, None, None])
    lam = (-(4 / dx**2) * math.sin(math.pi * a / nx) ** 2 - (4 / dy**2) * math.sin(math.pi * b / (2 * ny)) ** 2
           - (4 / dz**2) * math.sin(math.pi * c / nz) ** 2)
    f = to_dev(lam * phi)
    p = torch.empty_like(f)
    with ppe.Plan(nx, ny, nz, *L) as plan:
        plan.solve(f, p)
    assert O.rel_linf(p.cpu().numpy(), phi) < 1e-13


@pytest.mark.parametrize("shape", [(32, 32, 32), (48, 24, 36)])
def test_project_fp32_refine(shape):
    nx, ny, nz = shape
    fl = fields.make_fields(nx, ny, nz, seed=3, recipe="multimode", width=6.0, rho_g=60.0)
    ref = O.project_fields(fl)
    res, info = project_gpu(fl, precision=ppe.FP32_REFINE)
    L = (fl.lx, fl.ly, fl.lz)
    r = O.residual(res["f"], res["p"], L)
    rel = np.abs(r - r.mean()).max() / np.abs(res["f"]).max()
    assert rel <= TOL_RES, rel
    assert info.rel_residual <= TOL_RES
    assert O.rel_linf(res["f"], ref["f"]) <= TOL64
    for k in ("p", "u", "v", "w"):
        assert O.rel_linf(res[k], ref[k]) <= TOL_REF, k
    assert abs(res["p"].mean()) <= 1e-13 * np.abs(res["p"]).max()


def test_project_128_fp64_full():
    """The 128^3 multimode workload, whole-field comparison with both oracles."""
    fl = fields.multimode_128()
    ref = O.project_fields(fl)
    res, _ = project_gpu(fl)
    _compare(fl, res, ref, TOL64)
    _compare(fl, res, cpp.project_fields(fl), TOL64)


def test_project_256_fp32_refine_full():
    """The 256^3, density ratio 640/60 workload in the mixed-precision form."""
    fl = fields.multimode_256()
    ref = O.project_fields(fl)
    res, info = project_gpu(fl, precision=ppe.FP32_REFINE)
    r = O.residual(res["f"], res["p"], (fl.lx, fl.ly, fl.lz))
    rel = np.abs(r - r.mean()).max() / np.abs(res["f"]).max()
    assert rel <= TOL_RES, rel
    assert O.rel_linf(res["f"], ref["f"]) <= TOL64
    for k in ("p", "u", "v", "w"):
        assert O.rel_linf(res[k], ref[k]) <= TOL_REF, k
    assert abs(res["p"].mean()) <= 1e-13 * np.abs(res["p"]).max()


def test_project_256_fp64_full():
    """The 256^3, 640/60 workload in the plain FP64 form, whole-field comparison."""
    fl = fields.multimode_256()
    ref = O.project_fields(fl)
    res, _ = project_gpu(fl)
    _compare(fl, res, ref, TOL64)
    assert abs(res["p"].mean()) <= 1e-13 * np.abs(res["p"]).max()


@pytest.mark.parametrize("precision", [ppe.FP64, ppe.FP32_REFINE])
def test_project_384x256x384_full(precision):
    """The largest served grid, 384 x 256 x 384 (nx = 384 takes the general
    right-hand-side kernel and radix-3 x transforms), multimode 640/60, whole
    fields against the oracle."""
    fl = fields.make_fields(384, 256, 384, seed=19, recipe="multimode", width=6.0, rho_g=60.0)
    ref = O.project_fields(fl)
    res, info = project_gpu(fl, precision=precision)
    if precision == ppe.FP64:
        _compare(fl, res, ref, TOL64)
    else:
        assert info.rel_residual <= TOL_RES
        assert O.rel_linf(res["f"], ref["f"]) <= TOL64
        for k in ("p", "u", "v", "w"):
            assert O.rel_linf(res[k], ref[k]) <= TOL_REF, k
    assert abs(res["p"].mean()) <= 1e-13 * np.abs(res["p"]).max()


def test_project_host_buffers():
    fl = fields.make_fields(32, 16, 24, seed=12, recipe="single")
    ref = O.project_fields(fl)
    c = fl.shape
    out = dict(p=np.empty(c), u=np.empty(c), v=np.empty(fl.v.shape), w=np.empty(c), f=np.empty(c))
    with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz) as plan:
        plan.project_host(fl.u, fl.v, fl.w, fl.S, fl.rho, fl.p_n, fl.p_nm1, fl.dt, out["p"], out["u"], out["v"],
                          out["w"], f=out["f"])
    _compare(fl, out, ref, TOL64)


def test_errors():
    import torch
    with pytest.raises(ppe.PPEError) as e:
        ppe.Plan(250, 32, 32)
    assert e.value.code == 2
    with pytest.raises(ppe.PPEError) as e:
        ppe.Plan(9, 32, 32)  # odd nx
    assert e.value.code == 2
    with ppe.Plan(8, 8, 8) as plan:
        f = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
        with pytest.raises(ValueError):
            plan.solve(f.float(), f)
        d = {k: torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda") for k in "uwSrab"}
        v = torch.zeros((8, 9, 8), dtype=torch.float64, device="cuda")
        with pytest.raises(ppe.PPEError) as e:
            plan.rhs(d["u"], v, d["w"], d["S"], d["r"], d["a"], d["b"], 0.0, f)
        assert e.value.code == 1


from _gpu_util import dev_fields, project_gpu, to_dev  # noqa: E402


@pytest.mark.parametrize("precision", [ppe.FP64, ppe.FP32_REFINE])
def test_repeated_projections_are_bit_identical(precision):
    """Determinism: sums are totalled in a fixed order and the maxima use
    integer atomics on bit patterns, so the same inputs give the same bits on
    every call (here three calls through the captured graph of one plan)."""
    import torch
    fl = fields.make_fields(64, 48, 64, seed=23, recipe="multimode", width=4.0, rho_g=60.0)
    d = dev_fields(fl)
    outs = []
    with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz, precision=precision) as plan:
        for _ in range(3):
            o = [torch.empty(fl.shape, dtype=torch.float64, device="cuda"), torch.empty_like(d["u"]),
                 torch.empty_like(d["v"]), torch.empty_like(d["w"])]
            plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt, *o)
            torch.cuda.synchronize()
            outs.append([t.cpu().numpy() for t in o])
            info = plan.info()
            outs[-1].append(np.array([info.rel_residual, info.f_max, info.sweeps]))
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [ppe.FP64, ppe.FP32_REFINE])
@pytest.mark.parametrize("grid", [(48, 24, 36), (64, 32, 64)])
def test_tuning_does_not_change_results(precision, grid):
    """Launch shapes (tile sizes, marching chunk) change no bit of the outputs,
    including ragged last tiles; invalid shapes are rejected.  The power-of-two
    grid takes the register-staged FP32 transforms in x, y and z."""
    import torch
    fl = fields.make_fields(*grid, seed=17, recipe="multimode", width=4.0)
    d = dev_fields(fl)
    shapes = [dict(rhs_lines=4, rhs_planes=16, x_lines=32, z_cols=8, y_cols=16),
              dict(rhs_lines=1, rhs_planes=5, x_lines=1, z_cols=1, y_cols=1),
              dict(rhs_lines=8, rhs_planes=36, x_lines=64, z_cols=16, y_cols=32),
              dict(rhs_lines=2, rhs_planes=7, x_lines=4, z_cols=2, y_cols=4)]
    outs = []
    with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz, precision=precision) as plan:
        for sh in shapes:
            plan.set_tuning(**sh)
            assert {k: plan.get_tuning()[k] for k in sh} == sh
            o = [torch.empty(fl.shape, dtype=torch.float64, device="cuda"), torch.empty_like(d["u"]),
                 torch.empty_like(d["v"]), torch.empty_like(d["w"])]
            plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt, *o)
            torch.cuda.synchronize()
            outs.append([t.cpu().numpy() for t in o])
        with pytest.raises(ppe.PPEError):
            plan.set_tuning(rhs_lines=3)
        with pytest.raises(ppe.PPEError):
            plan.set_tuning(rhs_planes=0)
        assert {k: plan.get_tuning()[k] for k in shapes[-1]} == shapes[-1]
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("spectral", [ppe.SPECTRAL_LEGACY, ppe.SPECTRAL_PENCIL])
def test_largest_tiles_on_long_lines(spectral):
    """The largest tile values on 256- and 512-point lines (the y pass with 32
    columns, the z pass with 16, the x passes with 64 lines) are capped inside
    the launchers at 256 threads per CTA and give the same bits as the default
    shapes; every value ppe_set_tuning accepts launches."""
    import torch
    fl = fields.make_fields(32, 256, 512 if spectral == ppe.SPECTRAL_LEGACY else 256, seed=23, recipe="multimode",
                            width=4.0)
    d = dev_fields(fl)
    outs = []
    with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz, precision=ppe.FP32_REFINE) as plan:
        plan.set_tuning(spectral=spectral)
        for sh in (None, dict(rhs_lines=8, rhs_planes=32, x_lines=64, z_cols=16, y_cols=32),
                   dict(rhs_lines=1, rhs_planes=1, x_lines=1, z_cols=1, y_cols=1)):
            if sh:
                plan.set_tuning(**sh)
            o = [torch.empty(fl.shape, dtype=torch.float64, device="cuda"), torch.empty_like(d["u"]),
                 torch.empty_like(d["v"]), torch.empty_like(d["w"])]
            plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt, *o)
            torch.cuda.synchronize()
            outs.append([t.cpu().numpy() for t in o])
            assert plan.info().rel_residual <= TOL_RES
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [ppe.FP64, ppe.FP32_REFINE])
def test_views_at_an_odd_double_offset(precision):
    """Device arrays that start 8 bytes past a 16-byte boundary (views into a
    larger allocation) give the same bits as aligned ones: the kernels that use
    16-byte accesses (the FP32 transform of a given f, an FP64 p out of the
    inverse transform) take their 8-byte forms there."""
    import torch
    fl = fields.make_fields(64, 32, 32, seed=29, recipe="multimode", width=4.0)
    d = dev_fields(fl)

    def view(t):
        buf = torch.empty(t.numel() + 1, dtype=t.dtype, device=t.device)
        v = buf[1:].view(t.shape)
        v.copy_(t)
        assert v.data_ptr() % 16 == 8
        return v

    outs = []
    for shift in (False, True):
        dd = {k: (view(t) if shift else t.clone()) for k, t in d.items()}
        o = [torch.empty(fl.shape, dtype=torch.float64, device="cuda"), torch.empty_like(d["u"]),
             torch.empty_like(d["v"]), torch.empty_like(d["w"])]
        if shift:
            o = [view(t) for t in o]
        f = view(torch.empty_like(d["rho"])) if shift else torch.empty_like(d["rho"])
        p2 = view(torch.empty_like(d["rho"])) if shift else torch.empty_like(d["rho"])
        with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz, precision=precision) as plan:
            plan.project(dd["u"], dd["v"], dd["w"], dd["S"], dd["rho"], dd["p_n"], dd["p_nm1"], fl.dt, *o, f=f)
            plan.solve(f, p2)
            torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in o + [f, p2]])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
