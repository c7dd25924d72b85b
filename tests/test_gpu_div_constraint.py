"""Eq. (31) on the GPU (ppe_divergence_constraint) against the oracle, and the
assembled S and one-fluid density fed to the projection."""
import numpy as np
import pytest

from oracle import ppe_oracle as O
from paper_2103_01874_gb300 import fields, ppe

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    ppe.lib()


def _inputs(shape, seed):
    rng = np.random.default_rng(seed)
    C = rng.choice([0.0, 1.0, 0.3, 0.7, 1e-300, 1.0 - 2.0 ** -52], size=shape)
    comp_g = rng.normal(0.0, 2.0, shape)
    comp_l = rng.normal(0.0, 0.1, shape)
    mdot = np.where((C > 0) & (C < 1), rng.uniform(-1.0, 3.0, shape), 0.0)
    rho_g = rng.uniform(50.0, 130.0, shape)
    rho_l = rng.uniform(600.0, 700.0, shape)
    mask = (rng.random(shape) < 0.3).astype(np.uint8)
    return C, comp_g, comp_l, mdot, rho_g, rho_l, mask


def _gpu(shape, arrays, mask, with_rho=True):
    import torch
    from _gpu_util import to_dev
    nz, ny, nx = shape
    dev = [to_dev(a) for a in arrays]
    S = torch.empty_like(dev[0])
    rho = torch.empty_like(dev[0]) if with_rho else None
    m = torch.from_numpy(mask).cuda() if mask is not None else None
    with ppe.Plan(nx, ny, nz) as plan:
        plan.divergence_constraint(*dev, S, rho=rho, under_resolved=m)
        torch.cuda.synchronize()
    return S.cpu().numpy(), (rho.cpu().numpy() if with_rho else None)


@pytest.mark.parametrize("shape", [(24, 16, 32), (12, 27, 18)])
@pytest.mark.parametrize("use_mask", [True, False])
def test_matches_oracle(shape, use_mask):
    C, cg, cl, md, rg, rl, mask = _inputs(shape, seed=sum(shape))
    mask = mask if use_mask else None
    S_ref, rho_ref = O.divergence_constraint(C, cg, cl, md, rg, rl, mask)
    S, rho = _gpu(shape, (C, cg, cl, md, rg, rl), mask)
    # a handful of lazy pair operations, each within ~2^-47 relative
    assert O.rel_linf(S, S_ref) <= 5e-14
    assert O.rel_linf(rho, rho_ref) <= 5e-14
    if use_mask:
        zero = (mask != 0) & (C > 0) & (C < 1)
        assert np.all(S[zero] == 0.0) and np.any(S[~zero] != 0.0)


def test_full_size_and_without_density():
    shape = (256, 256, 256)
    C, cg, cl, md, rg, rl, mask = _inputs(shape, seed=5)
    S_ref, _ = O.divergence_constraint(C, cg, cl, md, rg, rl, mask)
    S, rho = _gpu(shape, (C, cg, cl, md, rg, rl), mask, with_rho=False)
    assert rho is None
    assert O.rel_linf(S, S_ref) <= 5e-14


def test_assembled_constraint_drives_the_projection():
    """S and rho from Eq. (31) on the GPU, then ppe_project: the same result as
    the oracle's projection of the oracle's S and rho (compatible part, R5)."""
    import torch
    from _gpu_util import dev_fields, to_dev
    fl = fields.make_fields(32, 16, 24, seed=41, recipe="single", width=2.0)
    shape = fl.shape
    rng = np.random.default_rng(2)
    C = np.clip((fl.rho - 120.0) / (640.0 - 120.0), 0.0, 1.0)  # volume fraction from the tanh layer
    cg = rng.normal(0.0, 0.05, shape)
    cl = rng.normal(0.0, 0.005, shape)
    md = np.where((C > 0.01) & (C < 0.99), 0.2, 0.0)
    rg = np.full(shape, 120.0)
    rl = np.full(shape, 640.0)
    S_ref, rho_ref = O.divergence_constraint(C, cg, cl, md, rg, rl)
    d = dev_fields(fl)
    S = torch.empty_like(d["rho"])
    rho = torch.empty_like(d["rho"])
    out = dict(p=torch.empty_like(d["rho"]), u=torch.empty_like(d["u"]), v=torch.empty_like(d["v"]),
               w=torch.empty_like(d["w"]))
    with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz, compat_tol=0.0) as plan:
        plan.divergence_constraint(to_dev(C), to_dev(cg), to_dev(cl), to_dev(md), to_dev(rg), to_dev(rl), S, rho=rho)
        plan.project(d["u"], d["v"], d["w"], S, rho, d["p_n"], d["p_nm1"], fl.dt, out["p"], out["u"], out["v"],
                     out["w"])
        plan.info()
    ref = O.ppe_project(fl.u, fl.v, fl.w, S_ref, rho_ref, fl.p_n, fl.p_nm1, fl.dt, (fl.lx, fl.ly, fl.lz))
    for k in ("p", "u", "v", "w"):
        assert O.rel_linf(out[k].cpu().numpy(), ref[k]) <= 1e-12, k
