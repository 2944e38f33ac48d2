"""The integer-pipe microbenchmark runs every op and reports sane rates."""
import pytest

from paper_2309_09609_gb300 import intpeak, swgb

pytestmark = pytest.mark.gpu


def test_every_op_runs_with_a_plausible_rate():
    rows = intpeak.measure(blocks_per_sm=8, threads=256, iters=2000)
    assert [r["op"] for r in rows] == swgb.INTPEAK_OPS
    for r in rows:
        # an SM issues at most 4 warp-instructions (128 lane-ops) per clock
        assert 0.5 < r["lane_ops_per_clk_sm"] <= 130.0, r
        assert 500.0 < r["sm_mhz"] < 2500.0, r
    rate = {r["op"]: r["lane_ops_per_clk_sm"] for r in rows}
    # the packed search relies on DPX 16x2 max-plus at (at least) half rate
    assert rate["viaddmax_s16x2"] >= 30.0
