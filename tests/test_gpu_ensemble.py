"""Ensemble driver and cycle tuner on the GPU: each field's estimate equals a separate trace_estimate run
with the same parameters (same seeds, same hierarchy), and the tuner returns one of its candidates."""
import numpy as np
import pytest

from synthetic import gauge

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2303_11512_gb300 import api
    return api


def test_ensemble_matches_single_runs(api):
    from paper_2303_11512_gb300 import ensemble as ens
    fields = [ens.Field(gauge.links(gauge.field(16, 3.0, 1)), 16, -0.05, "a"),
              ens.Field(gauge.links(gauge.field(32, 3.0, 2, sweeps=100)), 32, -0.03, "b"),
              ens.Field(gauge.links(gauge.field(16, 3.0, 3)), 16, -0.04, "c")]
    est = dict(d=4, k=1, nrhs_first=8, nrhs_max=32, seed=5)
    out = ens.run_ensemble(fields, eps=2e-2, est_params=est)
    assert not out["rejected"] and len(out["runs"]) == 3
    ctx = api.Context()
    for run in out["runs"]:
        f = next(x for x in fields if x.name == run["name"])
        U = torch.from_numpy(f.U).cuda()
        h = api.mg_setup(ctx, U, f.L, f.m0)
        r = api.trace_estimate(ctx, h, eps=2e-2, **est)
        h.close()
        assert r["tau"] == run["tau"] and r["N"] == run["N"]
        assert run["time_s"] > run["setup_s"] > 0
    ctx.close()
    assert out["fields_per_s"] > 0


def test_tune_cycle_returns_a_candidate(api):
    from paper_2303_11512_gb300 import ensemble as ens
    ctx = api.Context()
    U = torch.from_numpy(gauge.links(gauge.field(64, 3.0, 4, sweeps=60))).cuda()
    res = ens.tune_cycle(ctx, U, 64, -0.08, candidates=((1, 1), (2, 2)), nrhs=8)
    assert res["best"] in ((1, 1), (2, 2))
    assert all(t > 0 for t in res["times"].values())
    assert res["iters"][(2, 2)] <= res["iters"][(1, 1)]
    ctx.close()
