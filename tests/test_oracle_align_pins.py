"""Pins of the traceback oracle (oracle.align): the alignment it returns is
checked against brute-force enumeration, against the score oracle (itself
pinned in test_oracle_pins.py) and against a re-scoring of its transcript
written here, so that a wrong step, a wrong gap charge or a wrong end cell
fails a test.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle

ALPHA = 24


def gap_cost(k, gap_open, gap_extend):
    return 0 if k == 0 else gap_open + k * gap_extend


def rescore(q, d, a, sm, gap_open, gap_extend):
    """Score of a transcript: SM over the 'M' columns, open + k*extend per
    run of k 'I' (or 'D') columns; also checks that it walks exactly
    q[q_begin:q_end] and d[s_begin:s_end]."""
    i, j, s = a["q_begin"], a["s_begin"], 0
    for op, run in itertools.groupby(a["ops"]):
        k = len(list(run))
        if op == "M":
            for _ in range(k):
                assert i < len(q) and j < len(d), "transcript walks past a sequence"
                s += int(sm[q[i], d[j]])
                i += 1
                j += 1
        elif op == "I":
            s -= gap_cost(k, gap_open, gap_extend)
            i += k
        else:
            assert op == "D"
            s -= gap_cost(k, gap_open, gap_extend)
            j += k
    assert (i, j) == (a["q_end"], a["s_end"]) and i <= len(q) and j <= len(d)
    return s


def chains(m, n):
    """Every chain of aligned pairs (rows increasing, columns increasing)."""
    for k in range(1, min(m, n) + 1):
        for rows in itertools.combinations(range(m), k):
            for cols in itertools.combinations(range(n), k):
                yield rows, cols


def chain_score(q, d, rows, cols, sm, Go, Ge):
    s = sum(int(sm[q[r], d[c]]) for r, c in zip(rows, cols))
    for t in range(len(rows) - 1):
        for skip in (rows[t + 1] - rows[t] - 1, cols[t + 1] - cols[t] - 1):
            if skip:
                s -= Go + (skip - 1) * Ge
    return s


def m_pairs(a):
    """The aligned (query, subject) index pairs of a transcript."""
    i, j, out = a["q_begin"], a["s_begin"], []
    for op in a["ops"]:
        if op == "M":
            out.append((i, j))
            i += 1
            j += 1
        elif op == "I":
            i += 1
        else:
            j += 1
    return out


def rand_matrix(rng, lo=-6, hi=8):
    a = rng.integers(lo, hi + 1, size=(ALPHA, ALPHA))
    return a.astype(np.int32)


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_optimum_and_first_end_cell(seed):
    rng = np.random.default_rng(1000 + seed)
    for _ in range(25):
        m, n = int(rng.integers(0, 6)), int(rng.integers(0, 6))
        q = rng.integers(0, 4, size=m).astype(np.uint8)   # few letters: many ties
        d = rng.integers(0, 4, size=n).astype(np.uint8)
        sm = rand_matrix(rng)
        Ge = int(rng.integers(0, 4))
        Go = Ge + int(rng.integers(0, 5))
        a = oracle.align_paper(q, d, Go, Ge, sm)
        best, ends = 0, []
        for rows, cols in chains(m, n):
            s = chain_score(q, d, rows, cols, sm, Go, Ge)
            if s > best:
                best, ends = s, [(rows[-1], cols[-1])]
            elif s == best and s > 0:
                ends.append((rows[-1], cols[-1]))
        assert a["score"] == best
        if best == 0:
            assert a["ops"] == "" and a["q_end"] == a["q_begin"] == 0
            continue
        pairs = m_pairs(a)
        rows, cols = zip(*pairs)
        assert chain_score(q, d, rows, cols, sm, Go, Ge) == best   # an optimal chain
        assert pairs[-1] == min(ends)                              # rule 1: row-major first end
        assert a["ops"][0] == "M" and a["ops"][-1] == "M"
        assert (a["q_end"], a["s_end"]) == (pairs[-1][0] + 1, pairs[-1][1] + 1)


@pytest.mark.parametrize("gaps", [(10, 2), (5, 1), (0, 1), (11, 1), (3, 3)])
def test_transcript_rescores_to_the_score_oracle(gaps):
    rng = np.random.default_rng(sum(gaps))
    sm = oracle.blosum62()
    for _ in range(12):
        m, n = int(rng.integers(1, 260)), int(rng.integers(1, 260))
        q = rng.integers(0, 20, size=m).astype(np.uint8)
        d = rng.integers(0, 20, size=n).astype(np.uint8)
        if m > 40 and n > 40:   # a planted homologous stretch with an indel
            seg = q[10:40].copy()
            d[5:35] = seg
            d[20] = (d[20] + 1) % 20
        a = oracle.align(q, d, *gaps)
        s = oracle.sw_score(q, d, *gaps)
        assert a["score"] == s
        if s == 0:
            continue
        assert rescore(q, d, a, sm, *gaps) == s
        # the aligned stretches alone reach S
        assert oracle.sw_score(q[a["q_begin"]:a["q_end"]], d[a["s_begin"]:a["s_end"]], *gaps) == s
        # rule 1: no earlier row, and no earlier column of the end row, reaches S
        assert oracle.sw_score(q[:a["q_end"] - 1], d, *gaps) < s
        assert oracle.sw_score(q[:a["q_end"]], d[:a["s_end"] - 1], *gaps) < s


def test_textbook_shape():
    # HEAGAWGHEE vs PAWHEAE with a linear gap: AWGHE over AW-HE
    q, d = oracle.encode("HEAGAWGHEE"), oracle.encode("PAWHEAE")
    a = oracle.align_paper(q, d, 8, 8)
    assert (a["q_begin"], a["q_end"], a["s_begin"], a["s_end"], a["ops"]) == (4, 9, 1, 5, "MMIMM")


def test_self_alignment_is_the_diagonal():
    rng = np.random.default_rng(5)
    q = rng.integers(0, 20, size=300).astype(np.uint8)
    a = oracle.align(q, q, 10, 2)
    assert a["ops"] == "M" * 300 and (a["q_begin"], a["s_begin"]) == (0, 0)
    assert a["score"] == sum(int(oracle.blosum62()[c, c]) for c in q)


def test_gap_runs_are_charged_once():
    # a deletion of three residues in the subject copy: one run, open + 3*extend
    q = oracle.encode("WWWWWCCCCCWWWWW")
    d = oracle.encode("WWWWWCCWWWWW")
    a = oracle.align(q, d, 10, 2)
    assert a["ops"].count("I") == 3 and "III" in a["ops"] and "D" not in a["ops"]
    assert rescore(q, d, a, oracle.blosum62(), 10, 2) == a["score"]


def test_planted_traceback_mistakes_are_caught():
    # the re-scoring pin catches a transcript whose 'I' / 'D' meaning is
    # swapped, or whose begin is off by one
    q = oracle.encode("HEAGAWGHEEWWWKKKWWW")
    d = oracle.encode("PAWHEAEWWWWWW")
    a = oracle.align(q, d, 10, 2)
    sm = oracle.blosum62()
    assert rescore(q, d, a, sm, 10, 2) == a["score"]
    swapped = dict(a, ops=a["ops"].replace("I", "x").replace("D", "I").replace("x", "D"))
    if "I" in a["ops"] or "D" in a["ops"]:
        with pytest.raises(AssertionError):
            assert rescore(q, d, swapped, sm, 10, 2) == a["score"]
    shifted = dict(a, q_begin=a["q_begin"] + 1, q_end=a["q_end"] + 1)
    with pytest.raises(AssertionError):
        assert rescore(q, d, shifted, sm, 10, 2) == a["score"]
