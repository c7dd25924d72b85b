"""The autotuner's search without a GPU: a fake plan whose per-kernel event
times follow a known cost model.  The tuner must take the schedule by the
whole projection's time and each tile size by its own kernel's time, skip the
values a plan refuses, apply the argmin, and round-trip its JSON cache."""
import json

import pytest

from paper_2103_01874_gb300 import autotune, ppe


class FakePlan:
    nx, ny, nz, precision = 64, 64, 64, 1

    class opts:
        face_rule = 0

    def __init__(self):
        self.t = dict(rhs_lines=2, rhs_planes=8, x_lines=16, z_cols=16, y_cols=8, spectral=0, y_solve=1)
        self.on = False
        self.rec = {}
        self.tri_us = 35  # the tridiagonal y method's time

    def get_tuning(self):
        return dict(self.t)

    def set_tuning(self, **kw):
        t = dict(self.t)
        t.update(kw)
        if t["spectral"] == 1 or t["rhs_lines"] == 8:  # a schedule this plan lacks; too much shared memory
            raise ppe.PPEError(1, "ppe_set_tuning")
        self.t = t

    def profile(self, on):
        self.on = on

    def profile_read(self):
        r, self.rec = self.rec, {}
        return r

    # cost model (us per launch): each tile size moves only its kernel; the
    # schedule changes which spectral kernels run
    def _costs(self):
        t = self.t
        c = {"k_rhs_march": 300 + 20 * abs(t["rhs_lines"] - 4) + abs(t["rhs_planes"] - 16),
             "k_xinv": 40 + abs(t["x_lines"] - 8)}
        if t["spectral"] == 0:
            ys = 60 + abs(t["y_cols"] - 16) if t["y_solve"] == 0 else self.tri_us
            c.update(k_zfft_fwd=30 + abs(t["z_cols"] - 4), k_ysolve=ys, k_zfft_inv=27)
        else:
            c.update(k_zfft_fwd=25, k_ysolve=55, k_zfft_inv=20)  # PENCIL: faster here
        return c

    def run(self, k):
        if not self.on:
            return
        for _ in range(k):
            for name, us in self._costs().items():
                n, ms = self.rec.get(name, (0, 0.0))
                self.rec[name] = (n + 1, ms + 1e-3 * us)


def test_search_picks_the_argmin_and_caches(tmp_path):
    path = str(tmp_path / "tuning.json")
    plan = FakePlan()
    res = autotune.autotune(plan, plan.run, reps=2, path=path)
    best = res["tuning"]
    assert best["spectral"] == 2, "the schedule by whole-step time (FUSED refused)"
    assert best["rhs_lines"] == 4 and best["rhs_planes"] == 16
    assert best["x_lines"] == 8
    assert plan.get_tuning() == best, "the best is applied"
    assert "1" not in res["kernel_us"]["spectral"]["tried"], "refused values are skipped"
    # under PENCIL the z and y column counts do not move any time: the first value tried stays
    assert best["z_cols"] == autotune.SEARCH["z_cols"][1][0]
    with open(path) as fh:
        doc = json.load(fh)
    assert autotune.cache_key(plan) in doc
    fresh = FakePlan()
    assert autotune.apply_cached(fresh, path)
    assert fresh.get_tuning() == best


def test_apply_cached_without_entry(tmp_path):
    assert not autotune.apply_cached(FakePlan(), str(tmp_path / "none.json"))


@pytest.mark.parametrize("field", list(autotune.SEARCH))
def test_every_search_field_is_a_tuning_field(field):
    assert field in dict(ppe.Tuning._fields_)


def test_tune_batch_coordinate_search():
    # a separable cost with its minimum at window=16, stagger=4, ctas=2; one
    # combination refused (None): the search must skip it
    cost = {"window": {0: 5.0, 32: 3.0, 16: 1.0, 8: 2.0}, "stagger": {1: 4.0, 2: 3.0, 4: 0.5, 8: 1.0},
            "ctas_per_sm": {0: 1.0, 2: 0.25}}
    calls = []

    def measure(o):
        calls.append(o)
        if o["window"] == 8 and o["stagger"] == 1:
            return None
        return sum(cost[k][o[k]] for k in cost)
    search = {k: v for k, v in autotune.BATCH_SEARCH.items() if k in cost}
    best, ms, trials = autotune.tune_batch(measure, search=search)
    assert best == {"window": 16, "stagger": 4, "ctas_per_sm": 2}
    assert ms == 1.0 + 0.5 + 0.25
    # every trial measured once, and the table lists them
    assert len(calls) == len({tuple(sorted(c.items())) for c in calls}) == len(trials)
    assert "window=16,stagger=4,ctas_per_sm=2" in trials


class LegacyOnly(FakePlan):
    def set_tuning(self, **kw):
        if kw.get("spectral", self.t["spectral"]) != 0:
            raise ppe.PPEError(1, "ppe_set_tuning")
        super().set_tuning(**kw)


@pytest.mark.parametrize("tri_us,expect", [(35, 1), (90, 0)])
def test_y_method_by_whole_step_time(tmp_path, tri_us, expect):
    plan = LegacyOnly()
    plan.tri_us = tri_us
    res = autotune.autotune(plan, plan.run, reps=2, path=str(tmp_path / "t.json"))
    assert res["tuning"]["spectral"] == 0
    assert res["tuning"]["y_solve"] == expect
    if expect == 0:  # with the cosine method the y column count matters again
        assert res["tuning"]["y_cols"] == 16
