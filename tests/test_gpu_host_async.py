"""The pipelined host-buffer projection (ppe_project_host_async / ppe_host_wait):
several projections in flight through two staging sets give, bit for bit,
what ppe_project_host gives for each; the device-side status of every call
reaches ppe_host_wait; the staging sets are reused safely when more calls than
sets are enqueued."""
import numpy as np
import pytest

from paper_2103_01874_gb300 import fields, ppe

pytestmark = pytest.mark.gpu

SHAPE = (32, 24, 16)


def _host(fl, incompatible=False):
    import torch
    a = fl.arrays()
    if incompatible:
        a["v"] = a["v"].copy()
        a["v"][:, -1, :] = 0.3
        a["S"] = a["S"] + 0.05
    hin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in a.items()}
    c = fl.shape
    hout = dict(p=torch.empty(c, dtype=torch.float64).pin_memory(), u=torch.empty(c, dtype=torch.float64).pin_memory(),
                v=torch.empty(fl.v.shape, dtype=torch.float64).pin_memory(),
                w=torch.empty(c, dtype=torch.float64).pin_memory())
    return hin, hout


def _args(fl, hin, hout):
    return (hin["u"], hin["v"], hin["w"], hin["S"], hin["rho"], hin["p_n"], hin["p_nm1"], fl.dt, hout["p"], hout["u"],
            hout["v"], hout["w"])


@pytest.mark.parametrize("precision", [ppe.FP64, ppe.FP32_REFINE])
def test_pipelined_equals_one_at_a_time(precision):
    fls = [fields.make_fields(*SHAPE, seed=60 + s, recipe="multimode", width=3.0) for s in range(5)]
    with ppe.Plan(*SHAPE, fls[0].lx, fls[0].ly, fls[0].lz, precision=precision) as plan:
        ref = []
        for fl in fls:
            hin, hout = _host(fl)
            plan.project_host(*_args(fl, hin, hout))
            ref.append({k: t.numpy().copy() for k, t in hout.items()})
        bufs = [_host(fl) for fl in fls]
        for fl, (hin, hout) in zip(fls, bufs):  # five calls through two staging sets
            plan.project_host_async(*_args(fl, hin, hout))
        assert plan.host_wait() == 0
        for r, (_, hout) in zip(ref, bufs):
            for k in r:
                assert np.array_equal(hout[k].numpy(), r[k]), k
        # the plan's report describes the last projection
        info = plan.info()
        assert info.f_max > 0


def test_status_of_every_call_reaches_the_wait():
    fls = [fields.make_fields(*SHAPE, seed=70 + s, recipe="single", width=2.0) for s in range(3)]
    with ppe.Plan(*SHAPE, fls[0].lx, fls[0].ly, fls[0].lz) as plan:
        bufs = [_host(fl, incompatible=(s == 0)) for s, fl in enumerate(fls)]
        for fl, (hin, hout) in zip(fls, bufs):
            plan.project_host_async(*_args(fl, hin, hout))
        with pytest.raises(ppe.PPEError) as e:
            plan.host_wait()
        assert e.value.code == 3  # the first call's incompatible right-hand side
        # the status was consumed; the pipeline is clean again
        hin, hout = _host(fls[1])
        plan.project_host_async(*_args(fls[1], hin, hout))
        assert plan.host_wait() == 0


def test_missing_argument_is_refused():
    fl = fields.make_fields(*SHAPE, seed=80, recipe="single", width=2.0)
    with ppe.Plan(*SHAPE, fl.lx, fl.ly, fl.lz) as plan:
        hin, hout = _host(fl)
        with pytest.raises(ValueError):
            plan.project_host_async(hin["u"], hin["v"], hin["w"], hin["S"], hin["rho"], hin["p_n"], hin["p_nm1"],
                                    fl.dt, hout["p"], hout["u"], hout["u"], hout["w"])  # v_out of the wrong shape
        assert plan.host_wait() == 0


def test_plan_keeps_the_input_buffers_of_enqueued_calls():
    """Inputs passed as temporaries stay valid until host_wait: the binding
    holds them, so recycling pinned memory in between changes no result."""
    import torch
    fls = [fields.make_fields(*SHAPE, seed=90 + s, recipe="multimode", width=3.0) for s in range(3)]
    with ppe.Plan(*SHAPE, fls[0].lx, fls[0].ly, fls[0].lz, precision=ppe.FP32_REFINE) as plan:
        ref = []
        for fl in fls:
            hin, hout = _host(fl)
            plan.project_host(*_args(fl, hin, hout))
            ref.append({k: t.numpy().copy() for k, t in hout.items()})
        outs = []
        for fl in fls:
            hin, hout = _host(fl)
            plan.project_host_async(*_args(fl, hin, hout))
            outs.append(hout)
            del hin  # only the plan refers to the inputs now
            junk = [torch.full((fl.nz, fl.ny, fl.nx), 7.0, dtype=torch.float64).pin_memory() for _ in range(8)]
            del junk
        assert plan.host_wait() == 0
        for r, hout in zip(ref, outs):
            for k in r:
                assert np.array_equal(hout[k].numpy(), r[k]), k
