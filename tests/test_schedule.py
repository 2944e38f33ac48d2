"""The stage schedule of the block-cooperative int32 recompute (and of the
block-per-pair forward pass of the alignment, which uses the same one), by
enumeration on the CPU.

One (query, subject) pair runs on a block of W warps.  The query is cut into
passes of 32 x TI rows; pass p runs on warp p mod W and sweeps the subject's
n columns in n + 31 wavefront steps, 32 steps per stage, with a block-wide
barrier between stages.  Lane 31 of pass p writes the pass's bottom row at
column j (step j + 31) into its warp's border buffer; lane 0 of pass p + 1
reads it, fetched one stage ahead (stage k reads columns 32(k+1) .. 32(k+1)+31;
stage 0 also reads columns 0 .. 31).  Pass p starts at stage
(p div W) * period + (p mod W) * LAG with period = max(stages per pass, LAG * W).

Checked for every column of every pass, over a grid of sizes: the read of a
border value comes in a later stage than its write, the next pass on the
same warp overwrites it only in a later stage than that read, a warp's passes
never overlap, and the last pass ends at the block's last stage.  LAG = 3 is
the smallest lag with these properties; LAG = 2 puts a read and its write in
one stage.
"""
import itertools

import pytest


def schedule(npass, n, W, LAG):
    spass = (n + 31 + 31) // 32
    period = max(spass, LAG * W)
    start = [(p // W) * period + (p % W) * LAG for p in range(npass)]
    nstages = ((npass - 1) // W) * period + ((npass - 1) % W) * LAG + spass if npass else 0
    return spass, start, nstages


def write_stage(start_p, j):
    return start_p + (j + 31) // 32                  # lane 31 at step j + 31


def read_stage(start_p, j):
    return start_p + (0 if j < 32 else j // 32 - 1)  # fetched one stage ahead


def violations(npass, n, W, LAG):
    spass, start, nstages = schedule(npass, n, W, LAG)
    bad = []
    for p in range(npass):
        if p + W < npass and start[p + W] < start[p] + spass:
            bad.append(("warp passes overlap", p))
    if npass and start[-1] + spass != nstages:
        bad.append(("last stage", npass))
    for p in range(1, npass):
        for j in range(n):
            w = write_stage(start[p - 1], j)
            r = read_stage(start[p], j)
            if not r > w:
                bad.append(("read not after write", p, j, r, w))
            if p - 1 + W < npass:                    # the buffer's next writer
                w2 = write_stage(start[p - 1 + W], j)
                if not w2 > r:
                    bad.append(("overwritten before read", p, j, r, w2))
    return bad


@pytest.mark.parametrize("W", [2, 3, 5, 16])
def test_lag_three_orders_every_border_read_and_write(W):
    for npass, n in itertools.product([1, 2, W, W + 1, 2 * W + 3, 40],
                                      [1, 31, 32, 33, 63, 64, 65, 95, 200, 1000, 3000]):
        assert violations(npass, n, W, 3) == [], (npass, n, W)


def test_lag_two_races():
    bad = violations(4, 200, 16, 2)
    assert any(v[0] == "read not after write" and v[3] == v[4] for v in bad)


def test_short_subjects_wait_for_the_period():
    # when a pass is shorter than LAG * W stages, the warp waits a full period
    spass, start, _ = schedule(40, 33, 16, 3)
    assert spass == 2 and start[16] - start[0] == 48
    spass, start, _ = schedule(40, 5000, 16, 3)
    assert start[16] - start[0] == spass
