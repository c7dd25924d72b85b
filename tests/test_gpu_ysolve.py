"""The two y methods of the FP32 solve with walls (ppe_tuning.y_solve) against
the FP64 oracle and against each other:

  COSINE       DCT-II, eigenvalue divide, DCT-III through FFTs;
  TRIDIAGONAL  the Thomas elimination of the Neumann system with tabulated
               multipliers, as two affine scans over 16-element segments, the
               singular line kx = kz = 0 solved in FP64 from its flux form.

Both solve the same discrete system, so after refinement both meet the
oracle at the refinement form's tolerances; p stays zero-mean (the singular
line takes the mean the refinement asks for).  Lengths cover every
elements-per-thread instance (ny 8 .. 512), radix-3 ny and short last
segments.  Plans without the tridiagonal method refuse it."""
import numpy as np
import pytest

from oracle import ppe_oracle as O
from paper_2103_01874_gb300 import fields, ppe

pytestmark = pytest.mark.gpu

TOL_RES = 1e-10
TOL_FIELD = 1e-11


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


# ny = 8 (1 element per thread), 27 (radix 3, short segments), 48, 96, 128, 192,
# 256 (16), 512 (32); anisotropic boxes
GRIDS = [((32, 8, 16), (6.283185307179586, 1.0, 3.0)), ((18, 27, 12), (1.0, 4.0, 3.0)),
         ((24, 48, 32), (6.283185307179586, 5.0, 3.0)), ((32, 96, 16), (6.283185307179586,) * 3),
         ((16, 128, 24), (2.0, 7.0, 3.0)), ((24, 192, 16), (6.283185307179586,) * 3),
         ((32, 256, 32), (6.283185307179586,) * 3), ((16, 512, 16), (3.0, 9.0, 2.0))]


@pytest.mark.parametrize("shape,lengths", GRIDS)
def test_both_y_methods_meet_the_oracle(shape, lengths):
    import torch
    nx, ny, nz = shape
    fl = fields.make_fields(nx, ny, nz, seed=sum(shape), recipe="multimode", width=3.0, rho_g=60.0,
                            lx=lengths[0], ly=lengths[1], lz=lengths[2])
    ref = O.project_fields(fl)
    d = {k: torch.from_numpy(v.copy()).to("cuda") for k, v in fl.arrays().items()}
    res = {}
    # refined to 1e-12: the field bound holds on the anisotropic boxes too (a
    # 1e-10 residual allows ~1.3e-11 in v on 16 x 512 x 16 with dy = dx / 10)
    with ppe.Plan(nx, ny, nz, fl.lx, fl.ly, fl.lz, precision=ppe.FP32_REFINE, refine_tol=1e-12) as plan:
        assert plan.get_tuning()["y_solve"] == ppe.Y_COSINE, "the default"
        for method in (ppe.Y_TRIDIAGONAL, ppe.Y_COSINE):
            plan.set_tuning(y_solve=method)
            out, info = _project(plan, d, fl)
            assert info.rel_residual <= TOL_RES, (shape, method, info.rel_residual)
            assert _host_residual(fl, out["f"], out["p"]) <= TOL_RES
            for k in ("p", "u", "v", "w"):
                assert O.rel_linf(out[k], ref[k]) <= TOL_FIELD, (shape, method, k)
            assert abs(out["p"].mean()) <= 1e-13 * np.abs(out["p"]).max(), (shape, method)
            res[method] = out
    for k in ("p", "u", "v", "w"):
        assert O.rel_linf(res[ppe.Y_TRIDIAGONAL][k], res[ppe.Y_COSINE][k]) <= 2 * TOL_FIELD


def test_single_solve_of_a_discrete_eigenfunction():
    """ppe_solve of lam p* for a discrete eigenfunction p* of the 7-point
    operator (mode (3, 5, 2), and the kx = kz = 0 line's mode (0, 4, 0), which the
    FP64 flux-form solve carries) returns p* to the refinement tolerance."""
    import torch
    nx, ny, nz = 32, 64, 48
    L = (2 * np.pi, 3.0, 5.0)
    dx, dy, dz = L[0] / nx, L[1] / ny, L[2] / nz
    x = (np.arange(nx) + 0.5) * dx
    z = (np.arange(nz) + 0.5) * dz
    j = np.arange(ny)
    for a, b, c in ((3, 5, 2), (0, 4, 0)):
        Y = np.cos(np.pi * b * (j + 0.5) / ny)
        p = (np.cos(2 * np.pi * a * x / L[0] + 0.3)[None, None, :] * Y[None, :, None]
             * np.cos(2 * np.pi * c * z / L[2] - 1.1)[:, None, None])
        lam = (-(4 / dx**2) * np.sin(np.pi * a / nx) ** 2 - (4 / dy**2) * np.sin(np.pi * b / (2 * ny)) ** 2
               - (4 / dz**2) * np.sin(np.pi * c / nz) ** 2)
        with ppe.Plan(nx, ny, nz, *L, precision=ppe.FP32_REFINE) as plan:
            plan.set_tuning(y_solve=ppe.Y_TRIDIAGONAL)
            f = torch.from_numpy(lam * p).to("cuda")
            out = torch.empty_like(f)
            plan.solve(f, out)
            torch.cuda.synchronize()
            assert plan.info().rel_residual <= TOL_RES
            assert O.rel_linf(out.cpu().numpy(), p) <= 1e-11, (a, b, c)


def test_tridiagonal_refused_where_not_built():
    fl = fields.make_fields(16, 16, 16, seed=1, recipe="single", width=2.0)
    with ppe.Plan(16, 16, 16, fl.lx, fl.ly, fl.lz, precision=ppe.FP64) as plan:
        assert plan.get_tuning()["y_solve"] == ppe.Y_COSINE
        with pytest.raises(ppe.PPEError):
            plan.set_tuning(y_solve=ppe.Y_TRIDIAGONAL)
    with ppe.Plan(16, 16, 16, fl.lx, fl.ly, fl.lz, precision=ppe.FP32_REFINE, bc_top=ppe.BC_OUTFLOW) as plan:
        with pytest.raises(ppe.PPEError):
            plan.set_tuning(y_solve=ppe.Y_TRIDIAGONAL)
    with ppe.Plan(16, 1024, 8, 1.0, 1.0, 1.0, precision=ppe.FP32_REFINE) as plan:  # ny above 512
        assert plan.get_tuning()["y_solve"] == ppe.Y_COSINE
        with pytest.raises(ppe.PPEError):
            plan.set_tuning(y_solve=ppe.Y_TRIDIAGONAL)
        with pytest.raises(ppe.PPEError):
            plan.set_tuning(y_solve=2)
