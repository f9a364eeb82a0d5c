"""Host-side check of the index tables of the 2x2-block tensor-core stencil (csrc/tc_block.cu), read from the
kernel source: for every block site j and stencil direction f the weight sub-tile W(j, f) sits in the MMA
window of the slab it multiplies (the site j + f) at the accumulator columns of site j; the windows stay in the
staged weight rows; the sub-tiles of a window that hold no weight block are the zero ones, which no copy
writes; and the first MMA of each site's columns overwrites them.  These are the invariants the kernel's
layout comment states; the GPU parity tests check the results, this checks the tables without a GPU."""
import ast
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2303_11512_gb300", "csrc",
                   "tc_block.cu")
SITES = [(0, 0), (0, 1), (1, 0), (1, 1)]                      # (dt, dx) of s00, s01, s10, s11 from the corner
DIRS = [(0, 0), (0, 1), (0, -1), (1, 0), (-1, 0)]             # self, +x, -x, +t, -t as (dt, dx)
SUB = 32                                                      # rows of one weight sub-tile (16 Re + 16 Im)


def tables():
    src = open(SRC).read()
    out = {}
    for name in ("c_rowpos", "c_brow", "c_ncol", "c_col0", "c_sdt", "c_sdx", "c_order"):
        m = re.search(r"__constant__\s+(?:short|signed char)\s+%s(?:\[[^\]]*\])+\s*=\s*(\{.*?\});" % name, src,
                      re.S)
        assert m, name
        out[name] = ast.literal_eval(m.group(1).replace("{", "[").replace("}", "]"))
    m = re.search(r"constexpr int TB_BROWS = (\d+);", src)
    out["rows"] = int(m.group(1))
    m = re.search(r"\(z \? (\d+) : (\d+)\) \* 64", src)       # the rows the kernel clears once
    out["cleared"] = {int(m.group(1)), int(m.group(2))}
    return out


@pytest.fixture(scope="module")
def T():
    return tables()


def slab_of(T, pos):
    qs = [q for q in range(12) if (T["c_sdt"][q], T["c_sdx"][q]) == pos]
    assert len(qs) == 1, pos
    return qs[0]


def test_slabs_are_the_block_and_its_halo(T):
    pos = {(T["c_sdt"][q], T["c_sdx"][q]) for q in range(12)}
    want = {(s[0] + d[0], s[1] + d[1]) for s in SITES for d in DIRS}
    assert len(pos) == 12 and pos == want
    assert [(T["c_sdt"][q], T["c_sdx"][q]) for q in range(4)] == SITES


def test_every_weight_block_lands_in_its_slab_window_at_its_site_columns(T):
    subs = set()
    for j, (tj, xj) in enumerate(SITES):
        for f, (dt, dx) in enumerate(DIRS):
            q = slab_of(T, (tj + dt, xj + dx))
            r = T["c_rowpos"][j][f]
            b, n, c0 = T["c_brow"][q], T["c_ncol"][q], T["c_col0"][q]
            assert r % SUB == 0 and b <= r and r + SUB <= b + n, (j, f, q)
            assert c0 + (r - b) == SUB * j, (j, f, q)            # the rows feed accumulator columns of site j
            subs.add(r)
    assert len(subs) == 20                                       # 20 distinct sub-tiles, one per (j, f)


def test_windows_fit_and_their_other_rows_are_the_zero_subtiles(T):
    rows = T["rows"]
    weights = {T["c_rowpos"][j][f] for j in range(4) for f in range(5)}
    zero = set()
    for q in range(12):
        b, n, c0 = T["c_brow"][q], T["c_ncol"][q], T["c_col0"][q]
        assert n % 16 == 0 and 16 <= n <= 256 and b % SUB == 0   # valid MMA N for M = 64
        assert 0 <= b and b + n <= rows and c0 + n <= 4 * SUB   # staged rows, 4 sites x 32 columns
        own = {T["c_rowpos"][j][f] for j, (tj, xj) in enumerate(SITES) for f, (dt, dx) in enumerate(DIRS)
               if slab_of(T, (tj + dt, xj + dx)) == q}
        for r in range(b, b + n, SUB):
            if r not in own:
                assert r not in weights, (q, r)                  # a row no bulk copy or converter writes
                zero.add(r)
    assert len(weights) + len(zero) == rows // SUB               # 20 weight + 2 zero sub-tiles fill the stage
    assert zero == T["cleared"]                                  # and those two are the ones the kernel clears


def test_first_mma_of_each_site_overwrites(T):
    order = T["c_order"]
    assert sorted(order) == list(range(12))
    cols = set()
    for q in order[:4]:                                          # issued with the accumulate flag off
        c = set(range(T["c_col0"][q], T["c_col0"][q] + T["c_ncol"][q]))
        assert not cols & c
        cols |= c
    assert cols == set(range(4 * SUB))
