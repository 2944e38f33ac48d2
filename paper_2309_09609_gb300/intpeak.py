"""Integer-pipe throughput table: ``python -m paper_2309_09609_gb300.intpeak``.

Runs every op of the sw_intpeak microbenchmark (csrc/intpeak.cu) and prints
lane-operations per SM clock and the SM clock.  This is the measured
throughput term of the paper's capability model (Section III-B, Eq. 4) for
the instructions the alignment kernels use; bench.py takes its roofline peak
from the same measurement.
"""
from __future__ import annotations

import argparse
import json

from . import build, swgb


# cell-update ops: (lane-ops per update, cells per update); the update's
# throughput in cells per SM clock is lane-ops/clk/SM / ops * cells
CELL_SHAPE = {"cell_s16x2": (6, 2), "cell_s16x2_prmt": (7, 2), "cell_i32": (10, 1),
              "cell_biased": (6, 2), "cell_u8x4": (10, 4)}


def measure(blocks_per_sm: int = 8, threads: int = 256, iters: int = 20000) -> list[dict]:
    rows = []
    for op in swgb.INTPEAK_OPS:
        rate, mhz, secs = swgb.intpeak(op, blocks_per_sm, threads, iters)
        row = {"op": op, "lane_ops_per_clk_sm": round(rate, 2), "sm_mhz": round(mhz, 1),
               "ms": round(secs * 1e3, 3)}
        if op in CELL_SHAPE:
            ops, cells = CELL_SHAPE[op]
            row["cells_per_clk_sm"] = round(rate / ops * cells, 2)
        rows.append(row)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--blocks-per-sm", type=int, default=8)
    ap.add_argument("--json", action="store_true")
    a = ap.parse_args()
    build.build()
    rows = measure(a.blocks_per_sm)
    if a.json:
        print(json.dumps(rows))
        return
    print(f"{'op':22s} {'lane-ops/clk/SM':>16s} {'cells/clk/SM':>13s} {'SM MHz':>8s} {'ms':>8s}")
    for r in rows:
        cells = f"{r['cells_per_clk_sm']:13.1f}" if "cells_per_clk_sm" in r else " " * 13
        print(f"{r['op']:22s} {r['lane_ops_per_clk_sm']:16.1f} {cells} {r['sm_mhz']:8.0f} "
              f"{r['ms']:8.2f}")


if __name__ == "__main__":
    main()
