"""The query streams of the two-query kernels, on the CPU (sw_query_streams:
host logic only, the layout sw_plan_search builds once it has chosen the
number of stream pairs).  Each half of a stream pair must walk its queries
strip by strip, every query exactly once, and the two streams of a pair must
be as even as any split of the pair's queries can make them."""
import itertools

import numpy as np
import pytest

from paper_2309_09609_gb300 import build as nvbuild
from paper_2309_09609_gb300 import swgb

END = np.int64(0x80000000)


@pytest.fixture(scope="module", autouse=True)
def built():
    nvbuild.build()
    swgb.lib()


def strips_of(m, rows):
    return max(1, -(-int(m) // rows))


def walk(strips, pairs, lens, rows):
    """Checks the table's structure; returns per pair the queries of each half."""
    nq = len(lens)
    seen = []
    halves = []
    at = 0
    for first, count in pairs:
        assert first == at and count >= 1                  # pairs tile the table in order
        at += count
        both = []
        for h in range(2):
            q_col, r_col = strips[first:first + count, 2 * h], strips[first:first + count, 2 * h + 1]
            r_col = r_col.astype(np.int64) & 0xFFFFFFFF
            queries, s = [], 0
            while s < count and q_col[s] >= 0:
                q = int(q_col[s])
                k = strips_of(lens[q], rows)
                assert s + k <= count
                for j in range(k):                          # rows 0, T, 2T, ... end bit on the last
                    assert q_col[s + j] == q
                    assert (r_col[s + j] & ~END) == j * rows
                    assert bool(r_col[s + j] & END) == (j == k - 1)
                queries.append(q)
                s += k
            assert (q_col[s:] == -1).all()                  # empty strips only at the tail
            both.append(queries)
        assert max(sum(strips_of(lens[q], rows) for q in hq) for hq in both) == count
        halves.append(both)
        seen += both[0] + both[1]
    assert at == len(strips)
    assert sorted(seen) == list(range(nq))                  # every query exactly once
    return halves


@pytest.mark.parametrize("rows", [16, 24, 32])
@pytest.mark.parametrize("seed", range(12))
def test_streams_are_well_formed_and_each_pair_evenly_split(rows, seed):
    rng = np.random.default_rng(seed)
    nq = int(rng.integers(2, 15))
    lens = rng.integers(0, 3000, nq).astype(np.int32)
    if seed % 3 == 0:
        lens[: nq // 2] = rng.integers(0, 40, nq // 2)      # many short queries
    n_pairs = int(rng.integers(1, nq // 2 + 1))
    strips, pairs = swgb.query_streams(lens, rows, n_pairs)
    halves = walk(strips, pairs, lens, rows)
    for (a, b), (_, count) in zip(halves, pairs):
        sizes = [strips_of(lens[q], rows) for q in a + b]
        total = sum(sizes)
        best = min(max(sum(c), total - sum(c))
                   for r in range(len(sizes) + 1) for c in itertools.combinations(sizes, r))
        assert count == best                                 # the best split of the pair's queries


def test_dealing_longest_first_then_the_exact_split():
    # one pair: dealing longest first leaves [954, 445, 227, 195] against
    # [754, 636, 410, 172] strips (1,821 against 1,972); the exact split of the
    # same eight queries is 1,903 against 1,890
    strips_each = [954, 754, 636, 445, 410, 227, 195, 172]
    lens = np.array([32 * s for s in strips_each], dtype=np.int32)
    strips, pairs = swgb.query_streams(lens, 32, 1)
    assert pairs.tolist() == [[0, 1903]]
    walk(strips, pairs, lens, 32)


def test_more_pairs_hold_fewer_queries_each():
    lens = np.full(16, 100, dtype=np.int32)
    for k in (1, 2, 4, 8):
        strips, pairs = swgb.query_streams(lens, 32, k)
        halves = walk(strips, pairs, lens, 32)
        assert len(pairs) == k
        assert all(len(a) + len(b) == 16 // k for a, b in halves)
        assert (pairs[:, 1] == 4 * (16 // k) // 2).all()    # 4 strips a query, evenly split


@pytest.mark.parametrize("lens,rows,n_pairs", [
    ([10], 32, 1),            # one query: no pair
    ([10, 20], 32, 2),        # more pairs than n_queries / 2
    ([10, 20], 32, 0),
    ([10, 20], 8, 1),         # not a compiled strip height
    ([10, -1], 32, 1),        # negative length
])
def test_bad_arguments_are_refused(lens, rows, n_pairs):
    with pytest.raises(swgb.SwError) as e:
        swgb.query_streams(np.array(lens, dtype=np.int32), rows, n_pairs)
    assert e.value.status == swgb.SW_EINVAL


def test_a_table_that_does_not_fit_is_refused():
    import ctypes
    lens = np.array([1000, 1000], dtype=np.int32)
    strips = np.zeros((4, 4), dtype=np.int32)
    pairs = np.zeros((1, 2), dtype=np.int32)
    n = ctypes.c_int64(-1)
    st = swgb.lib().sw_query_streams(swgb._ptr(lens), 2, 32, 1, swgb._ptr(strips), 4,
                                     swgb._ptr(pairs), ctypes.byref(n))
    assert st == swgb.SW_EBUSY and n.value == 0
