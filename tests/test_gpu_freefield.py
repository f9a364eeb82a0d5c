"""End-to-end check at the benchmark size where the exact answer is known: for the free field (U = 1) the
trace of D^{-1} has a closed form (sum over the antiperiodic-in-t momenta of 2a / (a^2 + b^2), oracle
`free_field_trace_inverse`, itself pinned against dense LU at small L).  The GPU MG-MLMC++ estimate at L = 512
must lie within 3 sigma of it and reach the requested relative accuracy."""
import numpy as np
import pytest

from oracle import schwinger as osch

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_free_field_L512_estimate_within_3_sigma():
    import __graft_entry__ as g
    g.build()
    from paper_2303_11512_gb300 import api
    L, m0, eps = 512, -0.02, 1e-3
    exact = osch.free_field_trace_inverse(L, m0)
    ctx = api.Context()
    U = torch.ones((L, L, 2), dtype=torch.complex128, device="cuda")
    h = api.mg_setup(ctx, U, L, m0, bootstrap=1)
    r = api.trace_estimate(ctx, h, eps=eps, d=16, k=1, nrhs_first=16, seed=11)
    h.close()
    ctx.close()
    print("\n[free field L=512] exact %.6f  estimate %s  sigma %.4f  N %s"
          % (exact, r["tau"], r["sigma"], r["N"]))
    assert abs(r["tau"].real - exact) <= 3.0 * r["sigma"]
    assert abs(r["tau"].imag) <= 3.0 * r["sigma"]
    assert r["sigma"] <= 1.05 * eps * abs(r["tau"])
