"""CPU checks of the C ABI: the library loads, exports every function that
include/mgmlmc.h declares, and its host-only stop rule of Algorithm 2
(mlmc_update_active) agrees with the oracle's."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mgmlmc.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2303_11512_gb300 import _lib
    return _lib


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-zA-Z_][\w]*\s*\**\s*([a-zA-Z_]\w*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("schwinger_apply", "mg_setup", "mg_vcycle", "fgmres_batched", "mlmc_level_sample",
              "hutchpp_sketch_qr", "hutchpp_project", "trace_estimate"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if " T " in line)
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # and the ctypes table covers them
    assert set(declared_functions()) == set(lib.SIGNATURES)


def test_loaded_library_binds_all(lib):
    L = lib.load()
    assert L.mgmlmc_version() >= 100


def test_stop_rule_matches_oracle(lib):
    from oracle.estimators import update_active
    from paper_2303_11512_gb300 import api
    rs = np.random.default_rng(0)
    for trial in range(300):
        nd = int(rs.integers(1, 5))
        V = list(rs.uniform(0.1, 10, nd))
        N = [int(x) for x in rs.integers(1, 40, nd)]
        Cs = list(rs.uniform(0.5, 5, nd))
        act = list(rs.integers(0, 2, nd).astype(bool))
        eps = float(rs.uniform(0.01, 0.3))
        tau = float(rs.uniform(1, 50))
        for pol, name in ((api.OPTIMAL, "optimal"), (api.UNIFORM, "uniform")):
            a = api.mlmc_update_active(act, V, N, Cs, eps, tau, pol, 2)
            b = update_active(act, V, N, Cs, eps, tau, name, 2)
            assert a == b, (trial, V, N, Cs, act, eps, tau, name)


def test_noalloc_wrapper_rejects_mismatched_tensors():
    """hutchpp_project_noalloc's C entry point gets bare pointers; the binding checks shapes before any
    launch, so a mismatch raises ValueError instead of an out-of-bounds device access."""
    torch = pytest.importorskip("torch")
    from paper_2303_11512_gb300.api import check_noalloc_args
    z = torch.zeros((5, 64), dtype=torch.complex128)
    Q = torch.zeros((4, 64), dtype=torch.complex128)
    tau = torch.zeros(5, dtype=torch.complex128)
    assert check_noalloc_args(Q, z, z.clone(), tau) == (5, 64, 4)
    assert check_noalloc_args(None, z, z.clone(), tau) == (5, 64, 0)
    bad = [
        (Q, z, torch.zeros((5, 63), dtype=torch.complex128), tau),   # y shape
        (Q, z, torch.zeros((4, 64), dtype=torch.complex128), tau),   # y rows
        (torch.zeros((4, 32), dtype=torch.complex128), z, z, tau),   # Q columns
        (torch.zeros(64, dtype=torch.complex128), z, z, tau),        # Q rank
        (Q, z, z, torch.zeros(4, dtype=torch.complex128)),           # tau_out too short
        (Q, torch.zeros(64, dtype=torch.complex128), z, tau),        # zeta rank
    ]
    for args in bad:
        with pytest.raises(ValueError):
            check_noalloc_args(*args)
    with pytest.raises(ValueError):   # a tensor on another device than the launches
        check_noalloc_args(Q, z, z, tau, torch.device("meta"))
