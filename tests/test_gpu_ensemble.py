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


def test_concurrent_ensemble_equals_sequential(api):
    """Two fields at a time on their own streams give the same estimates as one after another."""
    from paper_2303_11512_gb300 import ensemble as ens
    fields = [ens.Field(gauge.links(gauge.field(32, 3.0, 10 + i, sweeps=60)), 32, -0.04 - 0.01 * i, "g%d" % i)
              for i in range(4)]
    est = dict(d=4, k=1, nrhs_first=8, nrhs_max=32, seed=3)
    seq = ens.run_ensemble(fields, eps=2e-2, est_params=est, concurrency=1)
    par = ens.run_ensemble(fields, eps=2e-2, est_params=est, concurrency=2)
    assert max(len(g) for g in par["groups"]) == 2
    a = {r["name"]: r for r in seq["runs"]}
    for r in par["runs"]:
        assert r["tau"] == a[r["name"]]["tau"] and r["N"] == a[r["name"]]["N"]


def test_autotune_fills_the_table_and_keeps_results(api):
    """The tuned launch variants compute the same operator: applies before and after tuning agree to rounding,
    and every tunable kernel of the hierarchy has entries for the tuned batch sizes."""
    ctx = api.Context()
    U = torch.from_numpy(gauge.links(gauge.field(64, 3.0, 4, sweeps=60))).cuda()
    h = api.mg_setup(ctx, U, 64, -0.05)
    x1 = torch.randn((40, h.n[1]), dtype=torch.complex64, device="cuda")
    x0 = torch.randn((40, h.n[0]), dtype=torch.complex64, device="cuda")
    y1a, y0a = torch.empty_like(x1), torch.empty_like(x0)
    h.apply(1, x1, y1a, api.TF32)
    h.apply(0, x0, y0a, api.FP32)
    h.autotune((8, 64), force=True)
    rows = api.tune_table()
    kinds = {(r["kind"], r["side"], r["bucket"]) for r in rows}
    assert {(0, 64, 8), (0, 64, 64), (1, 16, 8), (1, 16, 64), (2, 16, 8), (2, 16, 64)} <= kinds
    y1b, y0b = torch.empty_like(x1), torch.empty_like(x0)
    h.apply(1, x1, y1b, api.TF32)
    h.apply(0, x0, y0b, api.FP32)
    assert torch.allclose(y1a, y1b, rtol=0, atol=1e-5 * float(y1a.abs().max()))
    assert torch.equal(y0a, y0b)
    assert h.tc_status() == 0
    h.close()
    ctx.close()
