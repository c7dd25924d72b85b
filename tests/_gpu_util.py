"""Helpers shared by the GPU tests: move seeded fields to the device, run the
C-ABI projection, pull results back."""
import numpy as np
import torch

from paper_2103_01874_gb300 import ppe


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def dev_fields(fl):
    return {k: to_dev(v) for k, v in fl.arrays().items()}


def project_gpu(fl, precision=ppe.FP64, face_rule=ppe.FACE_ARITHMETIC, rho0=-1.0, want_f=True,
                refine_tol=1e-10, max_sweeps=8, bc_top=None, S=None):
    d = dev_fields(fl)
    if S is not None:
        d["S"] = to_dev(S)
    c = fl.shape
    out = dict(p=torch.empty(c, dtype=torch.float64, device="cuda"),
               u=torch.empty_like(d["u"]), v=torch.empty_like(d["v"]), w=torch.empty_like(d["w"]),
               f=torch.empty(c, dtype=torch.float64, device="cuda") if want_f else None)
    with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz, precision=precision, face_rule=face_rule,
                  refine_tol=refine_tol, max_sweeps=max_sweeps, bc_top=bc_top) as plan:
        plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt,
                     out["p"], out["u"], out["v"], out["w"], f=out["f"], rho0=rho0)
        info = plan.info(allow_not_converged=True)
    torch.cuda.synchronize()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    return res, info
