"""Serving loop on the GPU: requests that arrive while others run are admitted
and overlap on the slot streams; each request's result alone equals its
result in the mix, bit for bit; refinement requests meet their tolerance."""
import numpy as np
import pytest

from paper_2103_01874_gb300 import ppe, serve

pytestmark = pytest.mark.gpu


def test_alone_equals_in_mix():
    shapes = [(32, 32, 32), (48, 32, 64), (64, 64, 64), (96, 48, 32)]
    reqs = serve.poisson_requests(24, rate=5000.0, shapes=shapes, seed=9, fp64=ppe.FP64, fp32=ppe.FP32_REFINE)
    keep = {r.rid for r in reqs[:8]}
    ex = serve.CudaExecutor(slots=6)
    srv = serve.Server(ex, budget_bytes=8 << 30, slots=6)
    stats, mix = srv.run(reqs, keep=keep)
    srv.close()
    assert stats.completed == 24 and stats.rejected == 0
    assert stats.max_active > 1, "requests overlapped on the device"
    for r in reqs:
        if r.precision == ppe.FP32_REFINE:
            assert r.rel_residual <= 1e-10
    for r in reqs[:8]:
        ex1 = serve.CudaExecutor(slots=1, templates=ex.templates)
        one = serve.Server(ex1, budget_bytes=8 << 30, slots=1)
        st, res = one.run([serve.Request(r.rid, r.shape, r.precision, r.seed, 0.0)], keep={r.rid})
        one.close()
        assert st.completed == 1
        for k in ("p", "u", "v", "w"):
            assert np.array_equal(res[r.rid][k], mix[r.rid][k]), (r.rid, k)
