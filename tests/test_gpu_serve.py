"""Serving loop on the GPU: requests that arrive while others run are admitted
and overlap on the slot streams; every request projects its own seeded fields;
each request's result alone equals its result in the mix, bit for bit, and
matches the FP64 oracle on its own fields (FP64 requests to 1e-12, refinement
requests to 1e-11 with their residual at 1e-10)."""
import numpy as np
import pytest

from oracle import ppe_oracle as O
from paper_2103_01874_gb300 import ppe, serve

pytestmark = pytest.mark.gpu


def _overlap(a, b):
    return a.admitted < b.done and b.admitted < a.done


def test_alone_equals_in_mix_with_per_request_inputs():
    shapes = [(32, 32, 32), (48, 32, 64), (64, 64, 64), (96, 48, 32)]
    # a burst of same-shape requests with different seeds (so different fields)
    # at t = 0, both precisions, then a Poisson stream of mixed shapes
    burst = [serve.Request(i, (64, 64, 64), ppe.FP32_REFINE if i % 2 else ppe.FP64, 1000 + i, 0.0)
             for i in range(4)]
    rest = serve.poisson_requests(20, rate=5000.0, shapes=shapes, seed=9, fp64=ppe.FP64, fp32=ppe.FP32_REFINE)
    for r in rest:
        r.rid += 4
        r.seed += 4
        r.arrival += 1e-4
    reqs = burst + rest
    ex = serve.CudaExecutor(slots=6, pool=4)
    keep = {r.rid for r in reqs[:10]}
    srv = serve.Server(ex, budget_bytes=8 << 30, slots=6)
    stats, mix = srv.run(reqs, keep=keep)
    srv.close()
    assert stats.completed == 24 and stats.rejected == 0
    assert stats.max_active > 1, "requests overlapped on the device"
    # the four same-shape requests drew four different field sets, and at least
    # two of them were on the device at the same time
    assert len({ex.field_seed(r.shape, r.seed % ex.pool) for r in burst}) == 4
    assert any(_overlap(a, b) for i, a in enumerate(burst) for b in burst[i + 1:])
    for r in reqs:
        if r.precision == ppe.FP32_REFINE:
            assert r.rel_residual <= 1e-10
    for r in reqs[:10]:
        ex1 = serve.CudaExecutor(slots=1, pool=ex.pool, inputs=ex.inputs)
        one = serve.Server(ex1, budget_bytes=8 << 30, slots=1)
        st, res = one.run([serve.Request(r.rid, r.shape, r.precision, r.seed, 0.0)], keep={r.rid})
        one.close()
        assert st.completed == 1
        for k in ("p", "u", "v", "w"):
            assert np.array_equal(res[r.rid][k], mix[r.rid][k]), (r.rid, k)
        # and the oracle on the request's own fields
        _, fl = ex.fields_of(r.shape, r.seed)
        ref = O.project_fields(fl)
        tol = 1e-12 if r.precision == ppe.FP64 else 1e-11
        for k in ("p", "u", "v", "w"):
            assert O.rel_linf(mix[r.rid][k], ref[k]) <= tol, (r.rid, k)
    # requests of one shape with different seeds gave different results
    assert not np.array_equal(mix[0]["p"], mix[2]["p"])
