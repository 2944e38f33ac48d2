"""Peak-throughput model of Section III-B (Eq. 4-5) and architectural efficiency.

Eq. 4:  capability = clock rate x instruction throughput x lanes, summed over
        the device's cores (Table I multiplies by the core count).
Eq. 5:  theoretical peak (cell updates/s) = capability / instructions per cell.
Algorithm 1 counts 12 instructions per cell update (5 add/sub, 6 max, 1 move).
Architectural efficiency (Section II-C) = achieved / theoretical peak.
"""
from __future__ import annotations

#: instructions per cell update in the paper's int32 kernel (Algorithm 1)
PAPER_INSTRUCTIONS_PER_CELL = 12


def capability(cores: int, lanes: int, throughput: float, clock_mhz: float) -> float:
    """Eq. 4 in instructions per second for the whole device."""
    return float(cores) * lanes * throughput * clock_mhz * 1e6


def theoretical_peak_gcups(cores, lanes, throughput, clock_mhz,
                           instructions_per_cell=PAPER_INSTRUCTIONS_PER_CELL) -> float:
    """Eq. 5 in GCUPS."""
    return capability(cores, lanes, throughput, clock_mhz) / instructions_per_cell / 1e9


def arch_efficiency(achieved_gcups: float, peak_gcups: float) -> float:
    """Achieved / theoretical peak (Section II-C), as a fraction."""
    return achieved_gcups / peak_gcups


def gcups(cells: float, seconds: float) -> float:
    return cells / seconds / 1e9
