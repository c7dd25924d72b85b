"""The projection with an open (outflow) top boundary, p = 0 on the face
y = Ly, through the C ABI against the oracle's outflow definitions."""
import math

import numpy as np
import pytest

from oracle import ppe_oracle as O
from paper_2103_01874_gb300 import fields, ppe

pytestmark = pytest.mark.gpu

OUT = ppe.BC_OUTFLOW
SHAPES = [
    ((32, 32, 32), "single", 2.0, (2 * math.pi,) * 3),
    ((48, 24, 36), "multimode", 6.0, (2 * math.pi, 3.0, 5.0)),
    ((18, 27, 54), "single", 2.0, (1.0, 2.0, 3.0)),   # radix 3, odd ny, S = 0 before the shift
    ((8, 8, 8), "single", 2.0, (2 * math.pi,) * 3),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    ppe.lib()


def _ref(fl, S, rule=O.FACE_ARITHMETIC):
    return O.ppe_project(fl.u, fl.v, fl.w, S, fl.rho, fl.p_n, fl.p_nm1, fl.dt, (fl.lx, fl.ly, fl.lz), rule=rule,
                         bc_top=O.BC_OUTFLOW)


@pytest.mark.parametrize("shape,recipe,width,lengths", SHAPES)
def test_outflow_fp64(shape, recipe, width, lengths):
    from _gpu_util import project_gpu
    nx, ny, nz = shape
    fl = fields.make_fields(nx, ny, nz, seed=nx + 2 * ny, recipe=recipe, width=width,
                            lx=lengths[0], ly=lengths[1], lz=lengths[2])
    S = fl.S + 0.3  # a net expansion: compatible with an open top
    ref = _ref(fl, S)
    res, info = project_gpu(fl, precision=ppe.FP64, bc_top=OUT, S=S)
    for k in ("f", "p", "u", "v", "w"):
        assert O.rel_linf(res[k], ref[k]) <= 1e-12, k
    assert np.array_equal(res["v"][:, 0, :], fl.v[:, 0, :])       # the bottom wall keeps v
    h = O.spacings(fl.shape, lengths)
    div_new = O.div(res["u"], res["v"], res["w"], h)
    assert np.abs(div_new - S).max() <= 1e-10 * np.abs(O.div(fl.u, fl.v, fl.w, h)).max()


@pytest.mark.parametrize("rule", [ppe.FACE_ARITHMETIC, ppe.FACE_HARMONIC])
@pytest.mark.parametrize("shape", [(32, 32, 32), (48, 24, 36)])
def test_outflow_fp32_refine(shape, rule):
    from _gpu_util import project_gpu
    nx, ny, nz = shape
    fl = fields.make_fields(nx, ny, nz, seed=3, recipe="multimode", width=6.0, rho_g=60.0)
    S = fl.S + 0.2
    L = (fl.lx, fl.ly, fl.lz)
    ref = _ref(fl, S, rule)
    res, info = project_gpu(fl, precision=ppe.FP32_REFINE, face_rule=rule, bc_top=OUT, S=S)
    r = O.residual(res["f"], res["p"], L, O.BC_OUTFLOW)
    assert np.abs(r).max() / np.abs(res["f"]).max() <= 1e-10  # nothing is dropped with an open top
    assert 0 <= info.rel_residual <= 1e-10
    assert O.rel_linf(res["f"], ref["f"]) <= 1e-12
    for k in ("p", "u", "v", "w"):
        assert O.rel_linf(res[k], ref[k]) <= 1e-11, k


def test_outflow_full_256():
    from _gpu_util import project_gpu
    fl = fields.multimode_256()
    S = fl.S + 0.1
    ref = _ref(fl, S)
    res, info = project_gpu(fl, precision=ppe.FP32_REFINE, bc_top=OUT, S=S)
    assert info.rel_residual <= 1e-10
    for k in ("p", "u", "v", "w"):
        assert O.rel_linf(res[k], ref[k]) <= 1e-11, k


def test_outflow_separate_entry_points_equal_fused():
    import torch
    from _gpu_util import dev_fields, to_dev
    fl = fields.make_fields(24, 16, 18, seed=9, recipe="multimode", width=3.0)
    S = fl.S + 0.25
    d = dev_fields(fl)
    d["S"] = to_dev(S)
    ref = _ref(fl, S)
    f = torch.empty_like(d["rho"])
    p = torch.empty_like(d["rho"])
    u, v, w = torch.empty_like(d["u"]), torch.empty_like(d["v"]), torch.empty_like(d["w"])
    with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz, bc_top=OUT) as plan:
        plan.rhs(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt, f)
        plan.solve(f, p)
        plan.correct(d["u"], d["v"], d["w"], d["rho"], p, d["p_n"], d["p_nm1"], fl.dt, u, v, w)
        plan.info()  # no compatibility condition with an open top
    out = dict(f=f, p=p, u=u, v=v, w=w)
    for k in ("f", "p", "u", "v", "w"):
        assert O.rel_linf(out[k].cpu().numpy(), ref[k]) <= 1e-12, k


def test_outflow_tuning_does_not_change_results():
    import torch
    from _gpu_util import dev_fields
    fl = fields.make_fields(48, 24, 36, seed=6, recipe="multimode", width=6.0)
    d = dev_fields(fl)
    outs = []
    with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz, precision=ppe.FP32_REFINE, bc_top=OUT) as plan:
        for lines, planes in ((2, 8), (1, 4), (4, 16)):
            plan.set_tuning(rhs_lines=lines, rhs_planes=planes)
            o = [torch.empty_like(d["rho"]), torch.empty_like(d["u"]), torch.empty_like(d["v"]),
                 torch.empty_like(d["w"])]
            plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt, *o)
            outs.append([t.cpu().numpy() for t in o])
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


def test_unsplit_rejects_an_open_top():
    import torch
    from _gpu_util import dev_fields
    fl = fields.make_fields(16, 8, 12, seed=1)
    d = dev_fields(fl)
    o = [torch.empty_like(d["rho"]), torch.empty_like(d["u"]), torch.empty_like(d["v"]), torch.empty_like(d["w"])]
    with ppe.Plan(fl.nx, fl.ny, fl.nz, bc_top=OUT) as plan:
        with pytest.raises(ppe.PPEError) as e:
            plan.project_unsplit(d["u"], d["v"], d["w"], d["S"], d["rho"], fl.dt, *o)
        assert e.value.code == 1
