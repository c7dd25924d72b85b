"""The spectral schedules of the FP32 solve (ppe_tuning.spectral) against the
FP64 oracle and against each other:

  LEGACY  z, y and inverse z passes on the [kz][j][kx] spectrum;
  FUSED   one pass per kx plane in a thread-block cluster (z DFT, y solve,
          inverse z DFT; tiles moved by bulk tensor copies, y lines read across
          the cluster's shared memory);
  PENCIL  persistent z, y and inverse z passes on the [kx][kz][j] spectrum, each
          32 KB tile moved by bulk copies while the previous one is transformed.

FUSED and PENCIL serve FP32-refinement plans with walls, ny and nz in
{32, 64, 128, 256} and a power-of-two nx/2; the fused cluster has 1, 2, 4 or 8
CTAs (64 KB tiles) depending on ny nz, and every cluster size is exercised.
"""
import math

import numpy as np
import pytest

from oracle import ppe_oracle as O
from paper_2103_01874_gb300 import fields, ppe

from _gpu_util import dev_fields

pytestmark = pytest.mark.gpu

TOL_RES = 1e-10
TOL_FIELD = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    ppe.lib()


def _project(plan, d, fl):
    import torch
    out = dict(p=torch.empty(fl.shape, dtype=torch.float64, device="cuda"), u=torch.empty_like(d["u"]),
               v=torch.empty_like(d["v"]), w=torch.empty_like(d["w"]),
               f=torch.empty(fl.shape, dtype=torch.float64, device="cuda"))
    plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt, out["p"], out["u"],
                 out["v"], out["w"], f=out["f"])
    info = plan.info(allow_not_converged=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}, info


def _host_residual(fl, f, p):
    h = O.spacings(fl.shape, (fl.lx, fl.ly, fl.lz))
    r = f - f.mean() - O.laplacian(p, h)
    return np.abs(r).max() / np.abs(f).max()


# (nx, ny, nz): cluster sizes ny nz / 8192 = 1, 1, 2, 4, 4, 8
GRIDS = [(32, 32, 32), (64, 32, 128), (32, 128, 128), (64, 128, 256), (128, 256, 128), (64, 256, 256)]


SCHEDULES = [ppe.SPECTRAL_FUSED, ppe.SPECTRAL_PENCIL]


@pytest.mark.parametrize("sched", SCHEDULES)
@pytest.mark.parametrize("grid", GRIDS)
def test_schedule_matches_oracle(grid, sched):
    nx, ny, nz = grid
    fl = fields.make_fields(nx, ny, nz, seed=nx + 2 * ny + 3 * nz, recipe="multimode", width=4.0, rho_g=60.0,
                            lx=2 * math.pi, ly=5.0, lz=5.0)
    ref = O.project_fields(fl)
    d = dev_fields(fl)
    with ppe.Plan(nx, ny, nz, fl.lx, fl.ly, fl.lz, precision=ppe.FP32_REFINE, refine_tol=1e-10) as plan:
        assert plan.get_tuning()["spectral"] == ppe.SPECTRAL_LEGACY, "the default schedule"
        plan.set_tuning(spectral=sched)
        assert plan.get_tuning()["spectral"] == sched
        res, info = _project(plan, d, fl)
    assert info.rel_residual <= TOL_RES
    assert _host_residual(fl, res["f"], res["p"]) <= TOL_RES
    assert O.rel_linf(res["f"], ref["f"]) <= 1e-12
    for k in ("p", "u", "v", "w"):
        assert O.rel_linf(res[k], ref[k]) <= TOL_FIELD, k
    assert abs(res["p"].mean()) <= 1e-13 * np.abs(res["p"]).max()


@pytest.mark.parametrize("grid", [(64, 64, 64), (32, 128, 256)])
def test_schedules_agree(grid):
    """The same plan under the three schedules: the refined results agree to the
    refinement's accuracy, and the FP32 solve alone (no sweep) agrees to FP32
    rounding."""
    nx, ny, nz = grid
    fl = fields.make_fields(nx, ny, nz, seed=5, recipe="multimode", width=4.0, rho_g=60.0)
    d = dev_fields(fl)
    for sweeps, tol in ((8, 1e-12), (0, 2e-6)):
        res = []
        with ppe.Plan(nx, ny, nz, fl.lx, fl.ly, fl.lz, precision=ppe.FP32_REFINE, refine_tol=1e-10 if sweeps else 0.0,
                      max_sweeps=sweeps) as plan:
            for sched in (ppe.SPECTRAL_LEGACY, ppe.SPECTRAL_FUSED, ppe.SPECTRAL_PENCIL):
                plan.set_tuning(spectral=sched)
                assert plan.get_tuning()["spectral"] == sched
                res.append(_project(plan, d, fl)[0])
        for other in res[1:]:
            for k in ("p", "u", "v", "w"):
                a, b = res[0][k], other[k]
                if k == "p" and not sweeps:
                    a, b = a - a.mean(), b - b.mean()  # the FP32 solve alone keeps a mean at its rounding
                assert O.rel_linf(a, b) <= tol, (sweeps, k, O.rel_linf(a, b))


def test_unavailable_schedules_are_refused():
    """The plane-layout schedules are refused where they do not apply (FP64
    plans, a non-power-of-two ny, an outflow top); those plans report LEGACY."""
    for kw, shape in ((dict(precision=ppe.FP64), (32, 32, 32)), (dict(precision=ppe.FP32_REFINE), (32, 48, 32)),
                      (dict(precision=ppe.FP32_REFINE, bc_top=ppe.BC_OUTFLOW), (32, 32, 32))):
        with ppe.Plan(*shape, 1.0, 1.0, 1.0, **kw) as plan:
            assert plan.get_tuning()["spectral"] == ppe.SPECTRAL_LEGACY
            for sched in (ppe.SPECTRAL_FUSED, ppe.SPECTRAL_PENCIL):
                with pytest.raises(ppe.PPEError):
                    plan.set_tuning(spectral=sched)


def test_plane_layout_solve_with_unaligned_f():
    """ppe_solve of a right-hand side that starts 8 bytes past a 16-byte
    boundary: the forward x pass of the plane layout reads it with 8-byte loads
    and gives the same bits as an aligned copy."""
    import torch
    fl = fields.make_fields(64, 64, 64, seed=31, recipe="multimode", width=4.0)
    d = dev_fields(fl)
    outs = []
    with ppe.Plan(64, 64, 64, fl.lx, fl.ly, fl.lz, precision=ppe.FP32_REFINE) as plan:
        plan.set_tuning(spectral=ppe.SPECTRAL_PENCIL)
        f = torch.empty_like(d["rho"])
        plan.rhs(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt, f)
        buf = torch.empty(f.numel() + 1, dtype=f.dtype, device=f.device)
        fv = buf[1:].view(f.shape)
        fv.copy_(f)
        assert fv.data_ptr() % 16 == 8
        for src in (f, fv):
            p = torch.empty_like(f)
            plan.solve(src, p)
            torch.cuda.synchronize()
            outs.append(p.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
