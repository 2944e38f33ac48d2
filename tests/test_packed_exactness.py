"""The 16-bit exactness criterion, checked on the CPU against the oracle.

The packed kernels carry H, E, F and S with a bias of +Go in signed 16-bit
halves of a 32-bit word, two pairs per word, and add with wraparound (the
DPX add is ``add.s16x2``, without saturation).  The claim: a pair's 16-bit
score is exact unless S' >= 32767 - max(SM), and exactly the pairs whose true
biased score reaches that threshold are flagged for the int32 recompute.
Overflow in one half never reaches the other, because h' >= Go in both
halves, so the word-wide subtraction of (Go, Go) never borrows; the kernels
compiled for a fixed gap setting subtract (Go, Go) half by half instead,
which cannot cross halves at all, and both forms are modelled.

``packed_model`` below restates that arithmetic step by step (Eq. 1-3 with
the bias), independently of the CUDA sources; the oracle gives the exact
scores.  Inputs are long enough, and the matrices large enough, to push many
pairs past 32767.
"""
import numpy as np
import pytest

import oracle

LIMIT = 32767


def wrap16(x):
    """Signed 16-bit wraparound of int64 values."""
    return ((x + 32768) & 0xFFFF) - 32768


def packed_model(qs, ds, gap_open, gap_extend, sm, h_minus_go="word"):
    """16-bit biased scores and flags of pairs (qs[k], ds[k]), two per word.

    All queries share one length and all subjects another.  h' - Go is one
    32-bit subtraction of the packed word ("word") or a wrapping 16-bit
    subtraction per half ("half").  Returns (S' per pair, flagged per pair)."""
    B = len(qs)
    assert B % 2 == 0
    m, n = len(qs[0]), len(ds[0])
    Go, Ge = gap_open + gap_extend, gap_extend
    Q = np.stack(qs).astype(np.int64)
    D = np.stack(ds).astype(np.int64)

    def sub_go_word(h):
        # one 32-bit subtraction of (Go, Go) on the packed word of lanes 2k, 2k+1
        lo, hi = h[0::2] & 0xFFFF, h[1::2] & 0xFFFF
        word = (lo | (hi << 16)) - Go * 0x00010001
        word &= 0xFFFFFFFF
        t = np.empty_like(h)
        t[0::2] = wrap16(word & 0xFFFF)
        t[1::2] = wrap16((word >> 16) & 0xFFFF)
        return t

    def sub_go_half(h):
        return wrap16(h - Go)

    sub_go = sub_go_word if h_minus_go == "word" else sub_go_half

    h_up = np.full((B, n + 1), Go, np.int64)     # H' of the row above (row 0: H = 0)
    f_dn = np.zeros((B, n + 1), np.int64)        # F' entering this row (row 1: F = -Go)
    S = np.full(B, Go, np.int64)                 # S' (S = 0)
    for i in range(m):
        w_row = sm[Q[:, i][:, None], D]          # SM(q_i, d_j), j = 1..n
        h_row = np.empty_like(h_up)
        h_row[:, 0] = Go
        f_next = np.empty_like(f_dn)
        e = np.zeros(B, np.int64)                # E' entering column 1 (E = -Go)
        for j in range(1, n + 1):
            f = f_dn[:, j]
            h = np.maximum(wrap16(h_up[:, j - 1] + w_row[:, j - 1]),
                           np.maximum(np.maximum(e, f), Go))          # Eq. 1
            t = sub_go(h)
            e = np.maximum(wrap16(e - Ge), t)                          # Eq. 2
            f_next[:, j] = np.maximum(wrap16(f - Ge), t)               # Eq. 3
            h_row[:, j] = h
            S = np.maximum(S, h)
        h_up, f_dn = h_row, f_next
    return S, S >= LIMIT - int(sm.max())


def heavy_matrix(rng):
    """A matrix whose diagonal scores 95-127 per residue: a few hundred
    matching residues pass 32767."""
    a = rng.integers(-60, 21, size=(24, 24))
    a = np.triu(a) + np.triu(a, 1).T
    np.fill_diagonal(a, rng.integers(95, 128, size=24))
    return a.astype(np.int32)


def pairs_near_the_limit(rng, B, m, n, sm):
    """Subjects that share a mutated stretch of the query, from weak to
    strong, so the exact scores straddle the threshold."""
    qs, ds = [], []
    for k in range(B):
        q = rng.integers(0, 20, size=m).astype(np.uint8)
        d = rng.integers(0, 20, size=n).astype(np.uint8)
        L = min(m, n) - int(rng.integers(0, 40))
        seg = q[:L].copy()
        rate = [0.02, 0.08, 0.2, 0.5][k % 4]
        hit = rng.random(L) < rate
        seg[hit] = rng.integers(0, 20, size=int(hit.sum()))
        off = int(rng.integers(0, n - L + 1))
        d[off:off + L] = seg
        qs.append(q)
        ds.append(d)
    return qs, ds


def exact(qs, ds, gap_open, gap_extend, sm):
    return np.array([oracle.sw_score(q, d, gap_open, gap_extend, sm) for q, d in zip(qs, ds)])


@pytest.mark.parametrize("h_minus_go", ["word", "half"])
@pytest.mark.parametrize("seed,gaps", [(0, (10, 2)), (1, (40, 9)), (2, (0, 1)), (3, (11, 1))])
def test_flags_exactly_the_pairs_at_the_threshold_and_the_rest_is_exact(seed, gaps, h_minus_go):
    rng = np.random.default_rng(300 + seed)
    sm = heavy_matrix(rng)
    qs, ds = pairs_near_the_limit(rng, 16, 330, 360, sm)
    Sp, flagged = packed_model(qs, ds, *gaps, sm, h_minus_go)
    S = exact(qs, ds, *gaps, sm)
    Go = gaps[0] + gaps[1]
    thr = LIMIT - int(sm.max())
    assert (flagged == (S + Go >= thr)).all()
    assert (Sp[~flagged] - Go == S[~flagged]).all()
    # the case matters: some pairs overflow 16 bits outright, some stay exact,
    # and some words pair an overflowing lane with an exact one
    assert (S + Go > LIMIT).any() and (~flagged).any()
    lanes = flagged.reshape(-1, 2)
    assert (lanes[:, 0] != lanes[:, 1]).any()


def test_widest_gaps_of_the_packed_path():
    # Go + Ge = 16384 (Go = gap_open + gap_extend, Ge = gap_extend) is the
    # largest sum the packed path takes
    rng = np.random.default_rng(310)
    sm = heavy_matrix(rng)
    qs, ds = pairs_near_the_limit(rng, 8, 200, 240, sm)
    for gaps in [(16382, 1), (0, 8192), (5460, 5462)]:
        assert gaps[0] + 2 * gaps[1] == 16384
        Sp, flagged = packed_model(qs, ds, *gaps, sm)
        S = exact(qs, ds, *gaps, sm)
        Go = gaps[0] + gaps[1]
        assert (flagged == (S + Go >= LIMIT - int(sm.max()))).all(), gaps
        assert (Sp[~flagged] - Go == S[~flagged]).all(), gaps


def test_a_threshold_without_the_max_sm_margin_misses_wrapped_scores():
    # planted mistake: flag only S' >= 32767.  A pair whose true score passes
    # 32767 wraps, and its recorded S' stays below 32767: it would be kept.
    rng = np.random.default_rng(320)
    sm = heavy_matrix(rng)
    qs, ds = pairs_near_the_limit(rng, 16, 330, 360, sm)
    Sp, _ = packed_model(qs, ds, 10, 2, sm)
    S = exact(qs, ds, 10, 2, sm)
    wrong = (Sp < LIMIT) & (Sp - 12 != S)
    assert wrong.any()
