"""Compatibility of the right-hand side with the walls, and the mean of f that
the solve drops: the device sums (fixed-order reductions in the right-hand-side
kernel and the forward x transform) against the oracle's plain definitions,
the status codes, and the solution of an incompatible problem (the compatible
part, as the oracle computes it)."""
import ctypes
import math

import numpy as np
import pytest

from oracle import ppe_oracle as O
from paper_2103_01874_gb300 import fields, ppe

pytestmark = pytest.mark.gpu

PRECS = [ppe.FP64, ppe.FP32_REFINE]
F32_TRUNC = 2.0 ** -23  # maxima are reported from the float high part (truncated to 24 bits)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    ppe.lib()


def _incompatible(fl, s_shift=0.05, v_top=0.3, v_bot=-0.1):
    v = fl.v.copy()
    v[:, -1, :] = v_top
    v[:, 0, :] = v_bot
    return v, fl.S + s_shift


def _project(fl, precision, v=None, S=None, compat_tol=1e-12):
    import torch
    from _gpu_util import dev_fields, to_dev
    d = dev_fields(fl)
    if v is not None:
        d["v"] = to_dev(v)
    if S is not None:
        d["S"] = to_dev(S)
    out = dict(p=torch.empty_like(d["rho"]), u=torch.empty_like(d["u"]), v=torch.empty_like(d["v"]),
               w=torch.empty_like(d["w"]), f=torch.empty_like(d["rho"]))
    with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz, precision=precision, max_sweeps=8,
                  compat_tol=compat_tol) as plan:
        plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt,
                     out["p"], out["u"], out["v"], out["w"], f=out["f"])
        info = ppe.Info()
        code = ppe.lib().ppe_get_info(plan._h, ctypes.byref(info))
    return {k: t.cpu().numpy() for k, t in out.items()}, info, code


@pytest.mark.parametrize("precision", PRECS)
def test_compatible_fields_report(precision):
    fl = fields.make_fields(48, 24, 36, seed=21, recipe="multimode", width=6.0, rho_g=60.0)
    res, info, code = _project(fl, precision)
    assert code == 0
    c = O.compatibility(fl.v, fl.S, (fl.lx, fl.ly, fl.lz))
    assert abs(info.s_mean - c["s_mean"]) <= 1e-12 * c["s_absmax"]  # derived from the sum of f
    assert c["s_absmax"] * (1 - F32_TRUNC) <= info.s_absmax <= c["s_absmax"]
    assert info.wall_vmax == 0.0 and info.wall_flux_mean == 0.0
    fmax = np.abs(res["f"]).max()
    assert abs(info.f_mean_removed - res["f"].mean()) <= 1e-13 * fmax
    assert abs(info.f_mean_removed) <= 1e-12 * fmax


@pytest.mark.parametrize("precision", PRECS)
def test_incompatible_is_reported_and_the_compatible_part_solved(precision):
    fl = fields.make_fields(32, 16, 24, seed=22, recipe="single", width=2.0)
    L = (fl.lx, fl.ly, fl.lz)
    v, S = _incompatible(fl)
    res, info, code = _project(fl, precision, v=v, S=S)
    assert code == 3  # PPE_ERR_INCOMPATIBLE_RHS
    c = O.compatibility(v, S, L)
    dy = fl.ly / fl.ny
    assert abs(info.s_mean - c["s_mean"]) <= 1e-12 * c["s_absmax"]  # derived from the sum of f
    assert abs(info.wall_flux_mean - c["wall_flux_mean"]) <= 1e-14 * c["wall_vmax"] / dy
    assert abs(info.wall_vmax - 0.3) <= 0.3 * F32_TRUNC
    ref = O.ppe_project(fl.u, v, fl.w, S, fl.rho, fl.p_n, fl.p_nm1, fl.dt, L)
    fmax = np.abs(ref["f"]).max()
    assert abs(info.f_mean_removed - ref["f"].mean()) <= 1e-12 * fmax
    assert abs(info.f_mean_removed) > 1e-5 * fmax  # far above the 1e-12 test
    tol = 1e-12 if precision == ppe.FP64 else 1e-11
    for k in ("p", "u", "v", "w"):
        assert O.rel_linf(res[k], ref[k]) <= tol, k
    if precision == ppe.FP32_REFINE:
        # the residual leaves the dropped mean out, so the refinement converges
        assert 0 <= info.rel_residual <= 1e-10
        r = O.residual(res["f"], res["p"], L)
        assert np.abs(r - r.mean()).max() <= 1e-10 * fmax


@pytest.mark.parametrize("precision", PRECS)
def test_compat_tol_zero_removes_the_mean_silently(precision):
    fl = fields.make_fields(32, 16, 24, seed=23, recipe="single", width=2.0)
    v, S = _incompatible(fl)
    _, info, code = _project(fl, precision, v=v, S=S, compat_tol=0.0)
    assert code == 0
    assert math.isfinite(info.f_mean_removed) and info.f_mean_removed != 0.0


def test_balanced_wall_flux_is_compatible():
    """Equal flux through both walls, S with the matching zero mean: compatible."""
    fl = fields.make_fields(32, 16, 24, seed=24, recipe="single", width=2.0)
    v, S = _incompatible(fl, s_shift=0.0, v_top=0.3, v_bot=0.3)
    _, info, code = _project(fl, ppe.FP64, v=v, S=S)
    assert code == 0
    assert abs(info.wall_vmax - 0.3) <= 0.3 * F32_TRUNC
    assert abs(info.wall_flux_mean) <= 1e-15


def test_fp32_solve_of_f_with_a_mean_converges():
    """ppe_solve in the refinement form: f = lam * phi + 7 (a constant the solve
    drops) returns phi; before the residual left the mean out it stalled."""
    import torch
    from _gpu_util import to_dev
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
    f = to_dev(lam * phi + 7.0)
    p = torch.empty_like(f)
    with ppe.Plan(nx, ny, nz, *L, precision=ppe.FP32_REFINE, max_sweeps=8) as plan:
        plan.solve(f, p)
        with pytest.raises(ppe.PPEError) as e:
            plan.info()  # converged, but f has a mean: incompatible at the default compat_tol
        assert e.value.code == 3
        info = plan.info(allow_incompatible=True)
    assert 0 <= info.rel_residual <= 1e-10
    assert O.rel_linf(p.cpu().numpy(), phi) < 1e-11
    assert abs(info.f_mean_removed - (7.0 + (lam * phi).mean())) <= 1e-13 * abs(lam)
    assert math.isnan(info.s_mean)  # no right-hand side was assembled by this plan


def test_project_host_returns_the_device_status():
    fl = fields.make_fields(16, 8, 12, seed=25, recipe="single", width=2.0)
    v, S = _incompatible(fl)
    c = fl.shape
    out = dict(p=np.empty(c), u=np.empty(c), v=np.empty(fl.v.shape), w=np.empty(c))
    with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz) as plan:
        with pytest.raises(ppe.PPEError) as e:
            plan.project_host(fl.u, v, fl.w, S, fl.rho, fl.p_n, fl.p_nm1, fl.dt, out["p"], out["u"], out["v"],
                              out["w"])
        assert e.value.code == 3
        plan.project_host(fl.u, fl.v, fl.w, fl.S, fl.rho, fl.p_n, fl.p_nm1, fl.dt, out["p"], out["u"], out["v"],
                          out["w"])


def test_separate_rhs_then_solve_reports():
    """ppe_rhs alone reports the wall flux and max |S| (the sum of f is formed by
    the solve); the following ppe_solve adds the mean of f and the mean of S."""
    import torch
    from _gpu_util import dev_fields, to_dev
    fl = fields.make_fields(32, 16, 24, seed=26, recipe="single", width=2.0)
    L = (fl.lx, fl.ly, fl.lz)
    v, S = _incompatible(fl)
    d = dev_fields(fl)
    d["v"], d["S"] = to_dev(v), to_dev(S)
    f = torch.empty_like(d["rho"])
    p = torch.empty_like(d["rho"])
    c = O.compatibility(v, S, L)
    ref_f = O.ppe_rhs(fl.u, v, fl.w, S, fl.rho, fl.p_n, fl.p_nm1, O.rho0_of(fl.rho), fl.dt, L)
    dy = fl.ly / fl.ny
    with ppe.Plan(fl.nx, fl.ny, fl.nz, *L) as plan:
        plan.rhs(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt, f)
        info = plan.info()
        assert abs(info.wall_flux_mean - c["wall_flux_mean"]) <= 1e-14 * c["wall_vmax"] / dy
        assert c["s_absmax"] * (1 - F32_TRUNC) <= info.s_absmax <= c["s_absmax"]
        assert math.isnan(info.s_mean) and math.isnan(info.f_mean_removed)
        plan.solve(f, p)
        info = plan.info(allow_incompatible=True)
        fmax = np.abs(ref_f).max()
        assert abs(info.f_mean_removed - ref_f.mean()) <= 1e-12 * fmax
        assert abs(info.s_mean - c["s_mean"]) <= 1e-12 * c["s_absmax"]
        with pytest.raises(ppe.PPEError) as e:
            plan.info()
        assert e.value.code == 3
