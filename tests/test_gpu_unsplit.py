"""The unsplit projection, Eqs. (29)-(30), by FFT-preconditioned conjugate
gradients (ppe_project_unsplit) against the oracle: the exact discrete solution
by dense LU on small grids, and on larger grids the residual of Eq. (30) and
the divergence identity evaluated on the host in FP64."""
import math

import numpy as np
import pytest

from oracle import ppe_oracle as O
from paper_2103_01874_gb300 import fields, ppe

pytestmark = pytest.mark.gpu

PRECS = [ppe.FP64, ppe.FP32_REFINE]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    ppe.lib()


def _unsplit(fl, precision, face_rule=ppe.FACE_ARITHMETIC, tol=1e-12, max_iter=500):
    import torch
    from _gpu_util import dev_fields
    d = dev_fields(fl)
    out = dict(p=torch.empty_like(d["rho"]), u=torch.empty_like(d["u"]), v=torch.empty_like(d["v"]),
               w=torch.empty_like(d["w"]))
    with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz, precision=precision, face_rule=face_rule) as plan:
        plan.project_unsplit(d["u"], d["v"], d["w"], d["S"], d["rho"], fl.dt, out["p"], out["u"], out["v"],
                             out["w"], tol=tol, max_iter=max_iter)
        it, rel = plan.unsplit_info(allow_not_converged=True)
    return {k: t.cpu().numpy() for k, t in out.items()}, it, rel


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("rule", [ppe.FACE_ARITHMETIC, ppe.FACE_HARMONIC])
@pytest.mark.parametrize("shape", [(8, 8, 12), (12, 8, 16)])
def test_unsplit_matches_dense_solution(precision, rule, shape):
    nx, ny, nz = shape
    fl = fields.make_fields(nx, ny, nz, seed=31 + nx, recipe="single", width=2.0, lz=3.0)
    L = (fl.lx, fl.ly, fl.lz)
    ref = O.unsplit_project_dense(fl.u, fl.v, fl.w, fl.S, fl.rho, fl.dt, L, rule)
    res, it, rel = _unsplit(fl, precision, rule)
    assert 0 < it < 500 and rel <= 1e-12
    for k in ("p", "u", "v", "w"):
        assert O.rel_linf(res[k], ref[k]) <= 1e-9, k
    assert np.all(res["v"][:, 0, :] == fl.v[:, 0, :]) and np.all(res["v"][:, -1, :] == fl.v[:, -1, :])


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("shape", [(32, 32, 32), (48, 24, 36)])
def test_unsplit_residual_and_divergence(precision, shape):
    nx, ny, nz = shape
    fl = fields.make_fields(nx, ny, nz, seed=5, recipe="multimode", width=6.0, rho_g=60.0)
    L = (fl.lx, fl.ly, fl.lz)
    res, it, rel = _unsplit(fl, precision, tol=1e-10)
    assert 0 < it < 500 and rel <= 1e-10
    g = O.unsplit_rhs(fl.u, fl.v, fl.w, fl.S, fl.dt, L)
    # the true residual of Eq. (30), evaluated in FP64 on the host
    assert O.unsplit_residual(res["p"], g, fl.rho, L) <= 1e-9
    assert abs(res["p"].mean()) <= 1e-12 * np.abs(res["p"]).max()
    # Eq. (29) applied on the host to the GPU's p gives the GPU's velocity
    u1, v1, w1 = O.unsplit_correct(fl.u, fl.v, fl.w, fl.rho, res["p"], fl.dt, L)
    for a, b in ((res["u"], u1), (res["v"], v1), (res["w"], w1)):
        assert O.rel_linf(a, b) <= 1e-12
    h = O.spacings(fl.shape, L)
    div_new = O.div(res["u"], res["v"], res["w"], h)
    assert np.abs(div_new - fl.S).max() <= 1e-7 * np.abs(O.div(fl.u, fl.v, fl.w, h)).max()


def test_unsplit_zero_iterations_returns_the_predictor():
    fl = fields.make_fields(16, 8, 12, seed=7, recipe="single", width=2.0)
    res, it, rel = _unsplit(fl, ppe.FP64, max_iter=0)
    assert it == 0
    assert np.all(res["p"] == 0.0)
    # u* passes through the float-pair form (relative 2^-48)
    for k in ("u", "v", "w"):
        assert O.rel_linf(res[k], getattr(fl, k)) <= 1e-14, k


def test_unsplit_and_split_agree_when_the_split_is_exact():
    """With p^n = p^{n-1} = the unsplit p the split projection (Eq. (34)) returns
    the same p and velocity (O7 on the GPU: both paths through the C ABI)."""
    import torch
    from _gpu_util import project_gpu
    fl = fields.make_fields(24, 16, 18, seed=8, recipe="multimode", width=3.0)
    res, it, rel = _unsplit(fl, ppe.FP64, tol=1e-13, max_iter=1000)
    assert rel <= 1e-13
    fl.p_n = res["p"].copy()
    fl.p_nm1 = res["p"].copy()
    split, _ = project_gpu(fl, precision=ppe.FP64)
    assert O.rel_linf(split["p"], res["p"]) <= 1e-10
    for k in ("u", "v", "w"):
        assert O.rel_linf(split[k], res[k]) <= 1e-10, k
