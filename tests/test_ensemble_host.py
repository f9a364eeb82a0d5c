"""Host logic of the ensemble driver: level sizes, memory estimate and admission (no GPU)."""
import numpy as np
import pytest

pytest.importorskip("torch")
from paper_2303_11512_gb300 import ensemble as ens


def test_levels_match_the_library_rule():
    assert ens.levels_for(512) == [512, 128, 32, 8]
    assert ens.levels_for(128) == [128, 32, 8]
    assert ens.levels_for(64) == [64, 16, 4]
    assert ens.levels_for(16) == [16, 4]
    assert ens.levels_for(1024) == [1024, 256, 64, 16, 4]


def test_memory_estimate_grows_with_size_and_batch():
    a = ens.memory_estimate(128)
    assert ens.memory_estimate(256) > 3 * a
    assert ens.memory_estimate(128, nrhs_max=64) < a
    assert ens.memory_estimate(512) < 280e9   # the benchmark field fits a GB300


def test_admission_largest_first_and_rejection():
    f = [ens.Field(np.zeros((L, L, 2), complex), L, -0.05, "f%d" % L) for L in (64, 1024, 128, 512)]
    free = ens.memory_estimate(512) + 1
    ok, no = ens.admit(f, free)
    assert [x.L for x in ok] == [512, 128, 64]
    assert [x.L for x in no] == [1024]


def test_concurrent_groups_fit_memory_and_width():
    f = [ens.Field(np.zeros((L, L, 2), complex), L, -0.05, "f%d" % i) for i, L in enumerate((512, 512, 256, 128, 128))]
    m512, m256, m128 = ens.memory_estimate(512), ens.memory_estimate(256), ens.memory_estimate(128)
    g = ens.group_fields(f, m512 + m256 + 1, 2)
    assert [[x.name for x in grp] for grp in g] == [["f0"], ["f1", "f2"], ["f3", "f4"]]
    for grp in g:
        assert len(grp) <= 2 and sum(ens.memory_estimate(x.L) for x in grp) <= m512 + m256 + 1
    assert [len(grp) for grp in ens.group_fields(f, 10 ** 15, 1)] == [1] * 5


def test_tuning_table_round_trip():
    pytest.importorskip("torch")
    import __graft_entry__ as gentry
    gentry.build()
    from paper_2303_11512_gb300 import _lib, api
    api.tune_set([dict(kind=1, side=32, bucket=64, format=0, variant=5)])
    rows = [r for r in api.tune_table() if r["kind"] == 1 and r["side"] == 32 and r["bucket"] == 64]
    assert rows and rows[0]["variant"] == 5
    with pytest.raises(_lib.MgmlmcError):
        api.tune_set([dict(kind=0, side=32, bucket=64, format=0, variant=3)])   # 3 rhs per thread: no such variant
    with pytest.raises(_lib.MgmlmcError):
        api.tune_set([dict(kind=1, side=32, bucket=48, format=0, variant=0)])   # not a bucket
    api.tune_set([dict(kind=1, side=32, bucket=16, format=2, variant=16)])      # FP16 images: 2x2-block stencil
    rows = [r for r in api.tune_table() if r["kind"] == 1 and r["side"] == 32 and r["bucket"] == 16]
    assert rows and rows[0]["variant"] == 16 and rows[0]["format"] == 2
    with pytest.raises(_lib.MgmlmcError):
        api.tune_set([dict(kind=1, side=32, bucket=16, format=0, variant=16)])  # TF32 images: no block kernel
    with pytest.raises(_lib.MgmlmcError):
        api.tune_set([dict(kind=1, side=30, bucket=16, format=1, variant=16)])  # side not divisible by 4
    with pytest.raises(_lib.MgmlmcError):
        api.tune_set([dict(kind=2, side=32, bucket=16, format=1, variant=16)])  # SAP update has no such bit
