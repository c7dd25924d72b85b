"""Batched projections (ppe_batch_create / ppe_batch_launch, ppe_project_batched):
uneven grids, both precisions and face rules in one CUDA graph.  Each result
must equal, bit for bit, the same plan's individual ppe_project (same kernels,
same plan), on two replays, and agree with the FP64 oracle."""
import ctypes

import numpy as np
import pytest

from oracle import ppe_oracle as O
from paper_2103_01874_gb300 import fields, ppe

pytestmark = pytest.mark.gpu

SHAPES = [((32, 48, 64), ppe.FP32_REFINE, ppe.FACE_ARITHMETIC), ((48, 32, 32), ppe.FP64, ppe.FACE_ARITHMETIC),
          ((64, 64, 32), ppe.FP32_REFINE, ppe.FACE_HARMONIC), ((96, 32, 48), ppe.FP32_REFINE, ppe.FACE_ARITHMETIC),
          ((32, 32, 32), ppe.FP64, ppe.FACE_HARMONIC), ((48, 48, 96), ppe.FP32_REFINE, ppe.FACE_ARITHMETIC)]


def _setup():
    import torch
    items, fls = [], []
    for n, (shape, prec, rule) in enumerate(SHAPES):
        nx, ny, nz = shape
        fl = fields.make_fields(nx, ny, nz, seed=100 + n, recipe="single", width=2.0)
        plan = ppe.Plan(nx, ny, nz, fl.lx, fl.ly, fl.lz, precision=prec, face_rule=rule)
        d = {k: torch.from_numpy(v.copy()).to("cuda") for k, v in fl.arrays().items()}
        d.update(p=torch.empty(fl.shape, dtype=torch.float64, device="cuda"), u_out=torch.empty_like(d["u"]),
                 v_out=torch.empty_like(d["v"]), w_out=torch.empty_like(d["w"]), dt=fl.dt)
        items.append((plan, d))
        fls.append(fl)
    return items, fls


def _outs(d):
    return [d[k].cpu().numpy() for k in ("p", "u_out", "v_out", "w_out")]


def test_batch_equals_individual_and_oracle():
    import torch
    items, fls = _setup()
    single = []
    for plan, d in items:
        plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], d["dt"], d["p"], d["u_out"],
                     d["v_out"], d["w_out"])
        torch.cuda.synchronize()
        single.append(_outs(d))
        for k in ("p", "u_out", "v_out", "w_out"):
            d[k].fill_(float("nan"))
    with ppe.Batch(items) as batch:
        for _ in range(2):
            batch.launch()
            torch.cuda.synchronize()
            for (plan, d), ref in zip(items, single):
                for a, b in zip(_outs(d), ref):
                    assert np.array_equal(a, b)
                for k in ("p", "u_out", "v_out", "w_out"):
                    d[k].fill_(float("nan"))
    # the same solves against the FP64 oracle
    batch2 = ppe.Batch(items)
    batch2.launch()
    torch.cuda.synchronize()
    for (shape, prec, rule), fl, (plan, d) in zip(SHAPES, fls, items):
        ref = O.project_fields(fl, rule=rule)
        tol = 1e-12 if prec == ppe.FP64 else 1e-11
        for k, key in (("p", "p"), ("u", "u_out"), ("v", "v_out"), ("w", "w_out")):
            assert O.rel_linf(d[key].cpu().numpy(), ref[k]) <= tol, (shape, k)
        if prec == ppe.FP32_REFINE:
            assert plan.info().rel_residual <= 1e-10
    batch2.close()
    for plan, _ in items:
        plan.close()


def test_batch_errors_and_one_shot():
    import torch
    items, _ = _setup()
    plan, d = items[0]
    with pytest.raises(ppe.PPEError) as e:
        ppe.Batch([items[0], items[0]])  # a plan may appear once
    assert e.value.code == 1
    # one-shot form through the raw C ABI
    n = 2
    plans = (ctypes.c_void_p * n)(*[pl._h.value for pl, _ in items[:n]])
    flds = (ppe.FieldsC * n)()
    for i, (pl, dd) in enumerate(items[:n]):
        flds[i] = pl._fields(ppe._ptr, dd["u"], dd["v"], dd["w"], dd["S"], dd["rho"], dd["p_n"], dd["p_nm1"],
                             dd["dt"], dd["p"], dd["u_out"], dd["v_out"], dd["w_out"])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert ppe.lib().ppe_project_batched(n, plans, flds, stream) == 0
    assert ppe.lib().ppe_project_batched(0, plans, flds, stream) == 1
    for pl, _ in items:
        pl.close()
