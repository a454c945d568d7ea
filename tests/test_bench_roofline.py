"""The bench's roofline arithmetic on the CPU.

The algorithmic bytes per right-hand side are read x once, write x~ once and read the
ensemble operand once per batch of R (bytes per element: 4 for x and x~ outside the FP64
path, 2 for the mixed path's ensemble operand).  The kept-mode counts L come from the
oracle's spectrum and the threshold tau = 1e-10; the expected totals below are written
out term by term for the three benchmark grids, so a change to the formula, to the
element sizes or to the workloads' shapes fails here.
"""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import basis  # noqa: E402
from paper_2609_13327_b300 import synth  # noqa: E402

# (workload, L, s_x (n + K L) + s_z n K / R with the terms spelled out)
CASES = [
    ("c2_128x128x10", 593, 4 * (10 * 128 * 128 + 32 * 593) + 4 * (10 * 128 * 128) * 32 // 256),
    ("c3_256x256x32", 949, 4 * (32 * 256 * 256 + 64 * 949) + 2 * (32 * 256 * 256) * 64 // 64),
    ("c5_512x512x16", 1669, 4 * (16 * 512 * 512 + 48 * 1669) + 4 * (16 * 512 * 512) * 48 // 8),
]


@pytest.mark.parametrize("name,L,expected", CASES, ids=[c[0] for c in CASES])
def test_kept_modes_and_algorithmic_bytes(name, L, expected):
    w = synth.WORKLOADS[name]
    lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
    assert len(basis.kept_modes(lam, w.tau)) == L
    assert bench.algorithmic_bytes_per_rhs(w, L, w.prec, w.R) == expected


def test_element_sizes():
    assert bench.element_sizes("fp64") == (8, 8)
    assert bench.element_sizes("fp32") == (4, 4)
    assert bench.element_sizes("mixed") == (4, 2)


def test_bytes_per_launch_and_peak_source():
    """The 64-rhs launch of the 256x256x32 workload counts 820.9 MB; the denominator is the
    measured copy bandwidth of MEASURED_PEAKS.json when the file is there, else 6.4 TB/s."""
    w = synth.WORKLOADS["c3_256x256x32"]
    assert bench.algorithmic_bytes_per_rhs(w, 949, w.prec, w.R) * w.R == 820854784
    peak, kind = bench.measured_peak_hbm()
    if kind == "fallback":
        assert peak == 6400.0
    else:
        assert kind == "measured" and 1000.0 < peak < 20000.0
