"""The size limits of the plan: every direction at its maximum length (1024,
which takes the run-time radix plans and the smallest tiles), the minimum grid
(8^3), and strongly anisotropic grids, against the FP64 oracle in both
precisions."""
import numpy as np
import pytest

from oracle import ppe_oracle as O
from paper_2103_01874_gb300 import fields, ppe

pytestmark = pytest.mark.gpu

SHAPES = [(1024, 8, 8), (8, 1024, 8), (8, 8, 1024), (8, 8, 8), (512, 8, 96), (24, 384, 16)]


@pytest.mark.parametrize("precision", [ppe.FP64, ppe.FP32_REFINE])
@pytest.mark.parametrize("shape", SHAPES)
def test_limits_match_the_oracle(shape, precision):
    from _gpu_util import project_gpu
    assert ppe.size_supported(*shape)
    fl = fields.make_fields(*shape, seed=51, recipe="single", width=2.0)
    ref = O.project_fields(fl)
    # 1024-point lines make L's condition number ~1e5; the field error of the
    # refinement form is about that times its stopping residual, so these grids
    # refine to 1e-12 (one more sweep where the first stops above it)
    res, info = project_gpu(fl, precision=precision, refine_tol=1e-12)
    tol = 1e-12 if precision == ppe.FP64 else 1e-11
    for k in ("p", "u", "v", "w", "f"):
        err = np.abs(res[k] - ref[k]).max() / np.abs(ref[k]).max()
        assert err <= tol, (k, err)
    if precision == ppe.FP32_REFINE:
        assert info.rel_residual <= 1e-12


def test_one_past_the_limits_is_refused():
    assert not ppe.size_supported(2048, 8, 8)
    assert not ppe.size_supported(8, 8, 4)
    assert not ppe.size_supported(8, 10, 8)
    with pytest.raises(ppe.PPEError):
        ppe.Plan(8, 8, 2048, 1.0, 1.0, 1.0)
