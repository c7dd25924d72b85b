"""Programmatic dependent launch across plans and entry points.

The step's kernels are launched with programmatic stream serialisation and
each begins by waiting for the kernel before it on the stream.  Work of
different plans (and different entry points of one plan) queued back to back
on one stream must therefore give the same bits as each run alone; a kernel
that read its predecessor's output before that wait would break this."""
import numpy as np
import pytest

from paper_2103_01874_gb300 import fields, ppe

pytestmark = pytest.mark.gpu


def _dev(fl):
    import torch
    d = {k: torch.from_numpy(v.copy()).to("cuda") for k, v in fl.arrays().items()}
    d["out"] = dict(p=torch.empty(fl.shape, dtype=torch.float64, device="cuda"), u=torch.empty_like(d["u"]),
                    v=torch.empty_like(d["v"]), w=torch.empty_like(d["w"]))
    return d


def _project(plan, d, fl):
    o = d["out"]
    plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt, o["p"], o["u"], o["v"],
                 o["w"])


def _host(d):
    return {k: v.cpu().numpy() for k, v in d["out"].items()}


def test_interleaved_plans_on_one_stream_match_each_alone():
    import torch
    # FP32+refine (with and without the FP32 first-solve p: (nx/2) nz = 2048 and
    # 864) and FP64 plans of different shapes, all on the current stream (the
    # plans' default)
    specs = [((64, 64, 64), ppe.FP32_REFINE, 11), ((48, 32, 36), ppe.FP32_REFINE, 12), ((32, 48, 32), ppe.FP64, 13)]
    runs = []
    for shape, prec, seed in specs:
        fl = fields.make_fields(*shape, seed=seed, recipe="multimode", width=3.0, rho_g=60.0)
        plan = ppe.Plan(*shape, fl.lx, fl.ly, fl.lz, precision=prec)
        runs.append((plan, _dev(fl), fl))
    alone = []
    for plan, d, fl in runs:
        _project(plan, d, fl)
        torch.cuda.synchronize()
        alone.append(_host(d))
    for _, d, _ in runs:
        for v in d["out"].values():
            v.fill_(float("nan"))
    # back to back, three rounds, no synchronisation in between
    for _ in range(3):
        for plan, d, fl in runs:
            _project(plan, d, fl)
    torch.cuda.synchronize()
    for (plan, d, fl), ref in zip(runs, alone):
        got = _host(d)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), (fl.shape, k)
        plan.close()


def test_solve_and_project_interleaved_on_one_plan():
    import torch
    fl = fields.make_fields(64, 48, 32, seed=21, recipe="multimode", width=3.0, rho_g=60.0)
    d = _dev(fl)
    with ppe.Plan(64, 48, 32, fl.lx, fl.ly, fl.lz, precision=ppe.FP32_REFINE) as plan:
        f = torch.empty(fl.shape, dtype=torch.float64, device="cuda")
        plan.rhs(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt, f)
        p_alone = torch.empty_like(f)
        plan.solve(f, p_alone)
        _project(plan, d, fl)
        torch.cuda.synchronize()
        ref_solve, ref_proj = p_alone.cpu().numpy(), _host(d)
        p2 = torch.empty_like(f)
        for _ in range(2):
            plan.solve(f, p2)
            _project(plan, d, fl)
        torch.cuda.synchronize()
        assert np.array_equal(p2.cpu().numpy(), ref_solve)
        got = _host(d)
        for k in ref_proj:
            assert np.array_equal(got[k], ref_proj[k]), k
