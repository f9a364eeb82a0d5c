"""The Python binding checks every tensor's shape and device before a C-ABI call (the entry points receive bare
pointers and sizes, so a mismatch would become an out-of-bounds device access or a launch on another GPU's
memory).  Host-only: the library is replaced by a recorder, pointers by zeros, and the context's device is the
CPU, so the checks run without a GPU."""
import types

import pytest

torch = pytest.importorskip("torch")

from paper_2303_11512_gb300 import api  # noqa: E402

CPU = torch.device("cpu")


class Recorder:
    """Stands in for the loaded library: records (entry point, arguments) and returns status 0."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append((name, args))
            return 0
        return call


@pytest.fixture
def lib(monkeypatch):
    rec = Recorder()
    monkeypatch.setattr(api._lib, "load", lambda: rec)
    monkeypatch.setattr(api, "_ptr", lambda t, dtype=None: 0)
    return rec


def ctx(device=CPU):
    return types.SimpleNamespace(ptr=None, stream=types.SimpleNamespace(device=device))


def hier(c, n=(2 * 16 * 16, 16 * 4 * 4)):
    h = object.__new__(api.Hierarchy)
    h.ctx, h.ptr, h.L, h.m0 = c, None, 16, 0.0
    h.levels, h.n = len(n), list(n)
    h.side, h.dof = [16, 4][: len(n)], [2, 16][: len(n)]
    return h


def v(rows, n, dtype=torch.complex128, device=CPU):
    return torch.zeros((rows, n), dtype=dtype, device=device)


def last(rec, name):
    calls = [a for nm, a in rec.calls if nm == name]
    assert calls, name
    return calls[-1]


def test_schwinger_apply(lib):
    c, L = ctx(), 8
    U = torch.zeros((L, L, 2), dtype=torch.complex128)
    api.schwinger_apply(c, U, L, 0.1, v(3, 128), v(3, 128))
    assert last(lib, "schwinger_apply")[6] == 3
    one = torch.zeros(128, dtype=torch.complex128)
    api.schwinger_apply(c, U, L, 0.1, one, one.clone())
    assert last(lib, "schwinger_apply")[6] == 1
    for args in [(U, L, v(3, 128), v(3, 127)),                   # y too short
                 (U, L, v(3, 128), v(2, 128)),                   # fewer rows in y
                 (U, L, v(3, 130), v(3, 130)),                   # not 2 L^2
                 (torch.zeros((L, L - 1, 2), dtype=torch.complex128), L, v(3, 128), v(3, 128)),   # field shape
                 (U, L, v(3, 128), v(3, 128, device=torch.device("meta")))]:                      # device
        with pytest.raises(ValueError):
            api.schwinger_apply(c, args[0], args[1], 0.1, args[2], args[3])


def test_field_of_setup_and_net(lib):
    c = ctx()
    with pytest.raises(ValueError):
        api.mg_setup(c, torch.zeros((16, 16, 1), dtype=torch.complex128), 16, 0.0)
    api.mg_setup(c, torch.zeros((16, 16, 2), dtype=torch.complex128), 16, 0.0)
    assert last(lib, "mg_setup")[2] == 16
    with pytest.raises(ValueError):
        api.Net(c, torch.zeros((8, 8, 2), dtype=torch.complex128), 16)


def test_hierarchy_level_calls(lib):
    c = ctx()
    h = hier(c)
    n0, n1 = h.n
    h.apply(1, v(5, n1, torch.complex64), v(5, n1, torch.complex64), api.FP32)
    assert last(lib, "mg_apply")[5] == 5
    h.restrict(0, v(4, n0), v(4, n1))
    assert last(lib, "mg_restrict")[5] == 4
    h.prolong(0, v(2, n1), v(2, n0))
    assert last(lib, "mg_prolong")[5] == 2
    h.smooth(0, v(7, n0), v(7, n0))
    assert last(lib, "mg_smooth")[5] == 7
    h.vcycle(0, v(6, n0), v(6, n0))
    assert last(lib, "mg_vcycle")[5] == 6
    bad = [lambda: h.apply(1, v(5, n0), v(5, n0)),          # level-0 vectors on level 1
           lambda: h.apply(2, v(5, n1), v(5, n1)),          # no level 2
           lambda: h.restrict(1, v(4, n1), v(4, n1)),       # nothing below the coarsest level
           lambda: h.restrict(0, v(4, n0), v(3, n1)),       # rows differ
           lambda: h.prolong(0, v(2, n0), v(2, n1)),        # coarse and fine swapped
           lambda: h.smooth(0, v(7, n0), v(7, n0 - 2)),
           lambda: h.vcycle(-1, v(6, n0), v(6, n0)),
           lambda: h.vcycle(0, v(6, n0), v(6, n0, device=torch.device("meta")))]
    for f in bad:
        with pytest.raises(ValueError):
            f()


def test_solver_and_sample_calls(lib):
    c = ctx()
    h = hier(c)
    n0, n1 = h.n
    api.fgmres_batched(c, h, 1, v(9, n1), v(9, n1))
    assert last(lib, "fgmres_batched")[5] == 9
    api.mlmc_level_sample(c, h, 0, v(3, n0), v(3, n0), form=api.ACCUMULATED)
    assert last(lib, "mlmc_level_sample")[6] == 3
    out = api.mg_restrict_to_level(c, h, 1, v(3, n0))
    assert tuple(out.shape) == (3, n1) and last(lib, "mg_restrict_to_level")[5] == 3
    tau = api.hutchpp_project(c, None, v(4, n1), v(4, n1))
    assert tau.shape == (4,) and last(lib, "hutchpp_project")[5] == 4
    sk = types.SimpleNamespace(ptr=None, d=4, n=n1)
    api.hutchpp_project(c, sk, v(4, n1), v(4, n1))
    bad = [lambda: api.fgmres_batched(c, h, 0, v(9, n1), v(9, n1)),
           lambda: api.fgmres_batched(c, h, 1, v(9, n1), v(8, n1)),
           lambda: api.mlmc_level_sample(c, h, 0, v(3, n1), v(3, n1), form=api.ACCUMULATED),  # fine size needed
           lambda: api.mlmc_level_sample(c, h, 1, v(3, n1), v(3, n1), form=api.REDUCED),      # not a difference
           lambda: api.mg_restrict_to_level(c, h, 1, v(3, n1)),
           lambda: api.mg_restrict_to_level(c, h, 1, v(3, n0), out=v(2, n1)),
           lambda: api.hutchpp_project(c, None, v(4, n1), v(4, n0)),
           lambda: api.hutchpp_project(c, types.SimpleNamespace(ptr=None, d=4, n=n0), v(4, n1), v(4, n1)),
           lambda: api.mgmlmc_rademacher(c, 1, 0, 0, 0, n1, 3, out=v(3, n0)),
           lambda: api.mgmlmc_noise(c, 1, 1, 0, 0, 0, n1, 3, out=v(2, n1))]
    for f in bad:
        with pytest.raises(ValueError):
            f()


def test_network_vectors(lib):
    c = ctx()
    net = object.__new__(api.Net)
    net.ctx, net.ptr, net.L, net.nparams = c, None, 8, 10
    n = 2 * 8 * 8
    net.forward(v(3, n, torch.complex64))
    assert last(lib, "nn_forward")[4] == 3
    net.loss_grad(v(2, n, torch.complex64), v(2, n, torch.complex64))
    net.train_step(v(2, n, torch.complex64), v(2, n, torch.complex64))
    assert last(lib, "nn_train_step")[4] == 2
    bad = [lambda: net.forward(v(3, n - 2, torch.complex64)),
           lambda: net.forward(v(3, n, torch.complex64), v(2, n, torch.complex64)),
           lambda: net.loss_grad(v(2, n, torch.complex64), v(2, n + 2, torch.complex64)),
           lambda: net.train_step(v(2, n, torch.complex64), v(1, n, torch.complex64))]
    for f in bad:
        with pytest.raises(ValueError):
            f()
