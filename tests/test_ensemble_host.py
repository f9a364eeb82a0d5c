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
