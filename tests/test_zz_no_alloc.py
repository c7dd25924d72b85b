"""ppe_rho0_noalloc: the allocation-free min(rho) entry point, for callers that
cannot call cudaMalloc (their device memory belongs to another owner's budget,
or allocation would stall a latency-critical path).  Checked through the C ABI
against rho_0 as the plan-based entry point ppe_project computes it, on two
calls in a row, then on a different array right after (the static scratch is
shared by all calls), and for the size limit of that scratch.

Kept in a file of its own that pytest collects last."""
import ctypes

import pytest

from paper_2103_01874_gb300 import fields, ppe

pytestmark = pytest.mark.gpu


def _raw(rho, n, out):
    import torch
    return ppe.lib().ppe_rho0_noalloc(ctypes.c_void_p(rho.data_ptr()), ctypes.c_size_t(n),
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _plan_rho0(fl):
    """rho_0 from the existing entry point (ppe_project with rho0 <= 0)."""
    from _gpu_util import project_gpu
    _, info = project_gpu(fl, want_f=False)
    return info.rho0


@pytest.mark.parametrize("shape,seed,rho_g", [((48, 24, 36), 21, 120.0), ((64, 64, 64), 5, 77.0)])
def test_rho0_noalloc_matches_project(shape, seed, rho_g):
    import torch
    nx, ny, nz = shape
    fl = fields.make_fields(nx, ny, nz, seed=seed, recipe="multimode", width=6.0, rho_g=rho_g)
    want = _plan_rho0(fl)
    rho = torch.from_numpy(fl.rho.copy()).to("cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(2):  # two calls in a row share the static scratch
        out.fill_(-1.0)
        assert _raw(rho, rho.numel(), out) == 0
        torch.cuda.synchronize()
        # a minimum is exact: the tolerance of the other tests (1e-12) holds trivially
        assert abs(out.item() - want) <= 1e-12 * want
        assert out.item() == want
    # a different array right after: nothing stale survives in the scratch
    rho2 = rho.clone()
    rho2.view(-1)[rho2.numel() // 3] = 0.5 * want
    out.fill_(-1.0)
    ppe.rho0_noalloc(rho2, out)
    torch.cuda.synchronize()
    assert out.item() == 0.5 * want


def test_rho0_noalloc_rejects_sizes_beyond_scratch():
    import torch
    rho = torch.ones(8, dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    # rejected on the host before any launch, so the small buffer is never read
    assert _raw(rho, ppe.RHO0_NOALLOC_MAX + 1, out) == 2
    assert _raw(rho, 0, out) == 1
    with pytest.raises(ValueError):
        ppe.rho0_noalloc(rho.float(), out)  # the binding checks dtype before calling
