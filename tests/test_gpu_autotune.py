"""The autotuner on the GPU: it searches the spectral schedule and the tile
sizes of a real plan, applies a tuning the plan accepts, the tuned plan's
projection matches the default one (tile sizes change no bit; schedules agree
to the refinement's accuracy), and its cache gives a new plan of the same size
class the same tuning."""
import numpy as np
import pytest

from oracle import ppe_oracle as O
from paper_2103_01874_gb300 import autotune, fields, ppe

from _gpu_util import dev_fields

pytestmark = pytest.mark.gpu


def test_autotune_real_plan(tmp_path):
    import torch
    fl = fields.make_fields(64, 64, 64, seed=12, recipe="multimode", width=4.0, rho_g=60.0)
    d = dev_fields(fl)

    def make_out():
        return [torch.empty(fl.shape, dtype=torch.float64, device="cuda"), torch.empty_like(d["u"]),
                torch.empty_like(d["v"]), torch.empty_like(d["w"])]

    path = str(tmp_path / "tuning.json")
    outs = {}
    with ppe.Plan(64, 64, 64, fl.lx, fl.ly, fl.lz, precision=ppe.FP32_REFINE) as plan:
        o = make_out()

        def run(k):
            for _ in range(k):
                plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt, *o)

        run(1)
        torch.cuda.synchronize()
        outs["default"] = [t.cpu().numpy() for t in o]
        res = autotune.autotune(plan, run, reps=1, path=path)
        assert plan.get_tuning() == res["tuning"]
        assert set(res["kernel_us"]["spectral"]["tried"]) == {"0", "1", "2"}, "all three schedules ran"
        run(1)
        torch.cuda.synchronize()
        outs["tuned"] = [t.cpu().numpy() for t in o]
    for a, b in zip(outs["default"], outs["tuned"]):
        assert O.rel_linf(a, b) <= 1e-12
    with ppe.Plan(64, 64, 64, fl.lx, fl.ly, fl.lz, precision=ppe.FP32_REFINE) as fresh:
        assert autotune.apply_cached(fresh, path)
        assert fresh.get_tuning() == res["tuning"]
