"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test compares the oracle (Section II-B, Eq. 1-3) with something the
mathematics fixes independently: exhaustive enumeration of local alignments,
closed forms for special penalty settings, a textbook routine, or an
invariant every exact local-alignment score obeys.  A dropped term, a wrong
sign, a swapped index or a transposed operand in the oracle fails at least
one of them (``test_planted_mistakes_are_caught`` checks that claim).
"""
import difflib
import itertools

import numpy as np
import pytest

import oracle
from paper_2309_09609_gb300 import synth

BIG = 10 ** 6  # a gap penalty no alignment can afford


# ---- independent scorers (not the oracle's recurrence) ----------------------

def gap_cost(k, Go, Ge):
    """A gap of k >= 1 residues costs Go + (k-1)*Ge in Eq. 2-3's notation."""
    return 0 if k == 0 else Go + (k - 1) * Ge


def brute_force(q, d, sm, Go, Ge):
    """Best score over every local alignment, by enumeration.

    A local alignment is fixed by its chain of aligned residue pairs
    (i1 < i2 < ..., j1 < j2 < ...); between consecutive pairs the skipped
    query residues form one gap and the skipped subject residues another.
    Its score is the sum of SM over the pairs minus the gap costs; the empty
    alignment scores 0.  Valid for Go >= Ge (no gap is ever split).
    """
    m, n = len(q), len(d)
    best = 0
    for k in range(1, min(m, n) + 1):
        for rows in itertools.combinations(range(m), k):
            for cols in itertools.combinations(range(n), k):
                s = sum(int(sm[q[r], d[c]]) for r, c in zip(rows, cols))
                for a in range(k - 1):
                    s -= gap_cost(rows[a + 1] - rows[a] - 1, Go, Ge)
                    s -= gap_cost(cols[a + 1] - cols[a] - 1, Go, Ge)
                best = max(best, s)
    return best


def ungapped_best(q, d, sm):
    """Best ungapped segment: Kadane's maximum subarray along every diagonal."""
    m, n = len(q), len(d)
    best = 0
    for off in range(-(m - 1), n):
        run = 0
        for i in range(m):
            j = i + off
            if 0 <= j < n:
                run = max(0, run + int(sm[q[i], d[j]]))
                best = max(best, run)
    return best


def linear_gap_sw(q, d, sm, g):
    """Smith & Waterman (1981) with a linear gap (each gapped residue costs g)."""
    m, n = len(q), len(d)
    H = np.zeros((m + 1, n + 1), dtype=np.int64)
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            H[i, j] = max(0, H[i - 1, j - 1] + sm[q[i - 1], d[j - 1]],
                          H[i - 1, j] - g, H[i, j - 1] - g)
    return int(H.max())


def rand_seq(rng, lo, hi, alpha=24):
    return rng.integers(0, alpha, size=int(rng.integers(lo, hi + 1))).astype(np.uint8)


def rand_matrix(rng, alpha=24, lo=-6, hi=8, symmetric=True):
    a = rng.integers(lo, hi + 1, size=(alpha, alpha))
    if symmetric:
        a = np.triu(a) + np.triu(a, 1).T
    return a.astype(np.int32)


B62 = oracle.blosum62()


# ---- pins ---------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_enumeration(seed):
    rng = np.random.default_rng(1000 + seed)
    gaps = [(12, 2), (3, 1), (1, 1), (5, 0), (0, 0), (7, 3)]
    for t in range(60):
        q, d = rand_seq(rng, 1, 6), rand_seq(rng, 1, 6)
        sm = B62 if t % 3 == 0 else rand_matrix(rng, symmetric=(t % 2 == 0))
        Go, Ge = gaps[(seed + t) % len(gaps)]
        assert oracle.sw_score_paper(q, d, Go, Ge, sm) == brute_force(q, d, sm, Go, Ge)


def test_bruteforce_blosum62_library_gaps():
    # the library convention (open 10, extend 2) means Go = 12, Ge = 2
    rng = np.random.default_rng(7)
    for _ in range(150):
        q, d = rand_seq(rng, 1, 6, 20), rand_seq(rng, 1, 6, 20)
        assert oracle.sw_score(q, d, 10, 2) == brute_force(q, d, B62, 12, 2)


def test_huge_gaps_equal_ungapped_closed_form():
    rng = np.random.default_rng(11)
    for t in range(40):
        q, d = rand_seq(rng, 1, 60), rand_seq(rng, 1, 60)
        sm = B62 if t % 2 else rand_matrix(rng)
        assert oracle.sw_score_paper(q, d, BIG, BIG, sm) == ungapped_best(q, d, sm)


def test_equal_penalties_equal_linear_gap_sw():
    rng = np.random.default_rng(12)
    for t in range(40):
        q, d = rand_seq(rng, 1, 40), rand_seq(rng, 1, 40)
        g = int(rng.integers(1, 9))
        sm = B62 if t % 2 else rand_matrix(rng)
        assert oracle.sw_score_paper(q, d, g, g, sm) == linear_gap_sw(q, d, sm, g)


def test_identity_matrix_gives_longest_common_substring():
    rng = np.random.default_rng(13)
    ident = np.full((24, 24), -BIG, dtype=np.int32)
    np.fill_diagonal(ident, 1)
    for _ in range(40):
        a = rng.integers(0, 4, size=int(rng.integers(1, 80))).astype(np.uint8)
        b = rng.integers(0, 4, size=int(rng.integers(1, 80))).astype(np.uint8)
        sm_ = difflib.SequenceMatcher(None, list(a), list(b), autojunk=False)
        lcs = sm_.find_longest_match(0, len(a), 0, len(b)).size
        assert oracle.sw_score_paper(a, b, BIG, BIG, ident) == lcs


def test_invariants_random():
    rng = np.random.default_rng(14)
    for t in range(60):
        q, d = rand_seq(rng, 1, 120, 20), rand_seq(rng, 1, 120, 20)
        s = oracle.sw_score(q, d, 10, 2)
        assert s >= 0
        assert s == oracle.sw_score(d, q, 10, 2)                    # symmetry
        assert s >= ungapped_best(q, d, B62)                         # >= ungapped
        assert s <= min(len(q), len(d)) * int(B62.max())             # upper bound
        assert oracle.sw_score(q, d, 11, 2) <= s                     # monotone in open
        assert oracle.sw_score(q, d, 10, 3) <= s                     # monotone in extend
        d2 = rand_seq(rng, 1, 60, 20)
        cat = np.concatenate([d, d2])
        assert oracle.sw_score(q, cat, 10, 2) >= max(s, oracle.sw_score(q, d2, 10, 2))
        assert oracle.sw_score(q, q, 10, 2) >= int(B62[q, q].sum())  # self alignment


def test_trailing_padding_with_nonpositive_scores_is_neutral():
    rng = np.random.default_rng(15)
    sm = np.full((25, 25), -3, dtype=np.int32)
    sm[:24, :24] = B62
    sm[24, 24] = 0
    for _ in range(30):
        q, d = rand_seq(rng, 1, 50, 20), rand_seq(rng, 1, 50, 20)
        base = oracle.sw_score(q, d, 10, 2, sm)
        qp = np.concatenate([q, np.full(int(rng.integers(1, 9)), 24, np.uint8)])
        dp = np.concatenate([d, np.full(int(rng.integers(1, 9)), 24, np.uint8)])
        assert oracle.sw_score(qp, dp, 10, 2, sm) == base


def test_zero_and_minus_infinity_borders_agree():
    # the paper starts E and F at 0; the oracle at minus infinity (a reading)
    rng = np.random.default_rng(16)
    for t in range(80):
        q, d = rand_seq(rng, 1, 50), rand_seq(rng, 1, 50)
        sm = B62 if t % 2 else rand_matrix(rng)
        Go = int(rng.integers(0, 15))
        Ge = int(rng.integers(0, Go + 1))
        assert (oracle.sw_score_paper(q, d, Go, Ge, sm, zero_init=True)
                == oracle.sw_score_paper(q, d, Go, Ge, sm))


def test_gap_convention_mapping():
    # Eq. 2-3 read literally with "10/2" equals the library's (8, 2)
    rng = np.random.default_rng(17)
    for _ in range(40):
        q, d = rand_seq(rng, 1, 80, 20), rand_seq(rng, 1, 80, 20)
        assert oracle.sw_score_paper(q, d, 10, 2) == oracle.sw_score(q, d, 8, 2)


def test_empty_and_degenerate():
    e = np.zeros(0, np.uint8)
    q = oracle.encode("HEAGAWGHEE")
    assert oracle.sw_score(e, q) == 0 and oracle.sw_score(q, e) == 0
    assert oracle.sw_score(e, e) == 0
    # a single residue aligned with itself
    w = oracle.encode("W")
    assert oracle.sw_score(w, w) == 11
    # all-negative matrix: nothing is worth aligning
    neg = np.full((24, 24), -1, dtype=np.int32)
    assert oracle.sw_score(q, q, 10, 2, neg) == 0


def test_threaded_search_matches_single_pairs():
    rng = np.random.default_rng(18)
    qs = [rand_seq(rng, 0, 70, 20) for _ in range(5)]
    ds = [rand_seq(rng, 0, 90, 20) for _ in range(40)]
    S = oracle.search(qs, ds, 10, 2, nthreads=4)
    for a, q in enumerate(qs):
        for b, d in enumerate(ds):
            assert S[a, b] == oracle.sw_score(q, d, 10, 2)


def test_encode():
    assert list(oracle.encode("ARNDCQEGHILKMFPSTWYVBZX*")) == list(range(24))
    assert list(oracle.encode("uojaz?")) == [22, 22, 22, 0, 21, 22]


# ---- BLOSUM62 -----------------------------------------------------------------

def test_blosum62_structure():
    b = B62
    assert b.shape == (24, 24)
    assert (b == b.T).all()
    diag = np.diag(b)[:20]
    assert diag.min() >= 4 and diag.max() == 11
    W, C = oracle.ALPHABET.index("W"), oracle.ALPHABET.index("C")
    assert b[W, W] == 11 and b[C, C] == 9
    assert b.min() == -4 and b.max() == 11
    star = oracle.ALPHABET.index("*")
    assert (b[star, :23] == -4).all() and b[star, star] == 1


def _karlin_altschul(sm, p):
    from scipy.optimize import brentq
    P = np.outer(p, p)

    def f(lam):
        return float((P * np.exp(lam * sm)).sum()) - 1.0
    lam = brentq(f, 1e-6, 5.0)
    q = P * np.exp(lam * sm)
    H = float((q * lam * sm).sum())
    return lam, H


def test_blosum62_karlin_altschul_parameters():
    """Published ungapped BLOSUM62 statistics under Robinson & Robinson
    frequencies: lambda = 0.3176 nats, relative entropy H = 0.4012 nats
    (tests/golden/blosum62_karlin_altschul.txt).  Any single mistyped entry
    of the 20 x 20 core moves lambda or H beyond the tolerance below."""
    sm = B62[:20, :20].astype(np.float64)
    p = synth.BACKGROUND / synth.BACKGROUND.sum()
    assert float((np.outer(p, p) * sm).sum()) < 0  # local alignment needs E[s] < 0
    lam, H = _karlin_altschul(sm, p)
    gold = {}
    with open(__file__.replace("test_oracle_pins.py", "golden/blosum62_karlin_altschul.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                gold[k] = float(v)
    assert abs(lam - gold["lambda"]) < 2e-4
    assert abs(H - gold["H"]) < 2e-3


def test_planted_mistakes_are_caught():
    """Plausible slips in a Gotoh scorer each fail one of the pins above."""
    rng = np.random.default_rng(19)
    cases = [(rand_seq(rng, 1, 6), rand_seq(rng, 1, 6)) for _ in range(200)]

    def gotoh(q, d, sm, Go, Ge, slip):
        m, n = len(q), len(d)
        NEG = -10 ** 9
        H = np.zeros((m + 1, n + 1), np.int64)
        E = np.full((m + 1, n + 1), NEG, np.int64)
        F = np.full((m + 1, n + 1), NEG, np.int64)
        best = 0
        for i in range(1, m + 1):
            for j in range(1, n + 1):
                go_e = Go if slip != "open_as_extend" else Ge
                E[i, j] = max(H[i, j - 1] - go_e, E[i, j - 1] - Ge)
                F[i, j] = max(H[i - 1, j] - Go, F[i - 1, j] - Ge)
                s = sm[q[i - 1], d[j - 1]] if slip != "transposed" else sm[d[j - 1], q[i - 1]]
                diag = H[i - 1, j - 1] if slip != "wrong_diag" else H[i - 1, j]
                terms = [diag + s, E[i, j], F[i, j]]
                if slip != "no_zero":
                    terms.append(0)
                if slip == "no_F":
                    terms.remove(F[i, j])
                H[i, j] = max(terms)
                best = max(best, H[i, j]) if slip != "last_cell" else H[i, j]
        return int(best if slip != "no_zero" else max(best, 0))

    sm_asym = rand_matrix(rng, symmetric=False)
    for slip in ["open_as_extend", "transposed", "wrong_diag", "no_zero", "no_F", "last_cell"]:
        caught = False
        for q, d in cases:
            if gotoh(q, d, sm_asym, 7, 1, slip) != brute_force(q, d, sm_asym, 7, 1):
                caught = True
                break
        assert caught, slip
