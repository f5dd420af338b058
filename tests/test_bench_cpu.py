"""Host-side helpers of bench.py: the phase-aligned object error that decides
"matched error" in the precision comparison, and the algorithmic work per
launch that the roofline figures divide by."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_object_error_ignores_a_global_phase_and_sees_a_local_change():
    import torch
    g = np.random.default_rng(0)
    O_true = torch.tensor(np.exp(1j * g.uniform(-0.5, 0.5, (64, 64))) * g.uniform(0.8, 1.0, (64, 64)),
                          dtype=torch.complex64)
    pos = torch.tensor([[20.0, 20.0], [40.0, 44.0]])
    shifted = O_true * np.exp(1j * 1.234)
    assert bench.object_error(shifted, O_true, pos, 16) < 1e-6
    bad = shifted.clone()
    bad[30, 30] += 0.5
    assert bench.object_error(bad, O_true, pos, 16) > 1e-3
    # pixels outside the scanned box (probe centres widened by N/4) do not count
    far = shifted.clone()
    far[0, 63] += 5.0
    assert bench.object_error(far, O_true, pos, 16) < 1e-6


def test_algorithmic_work_formulas():
    # FFT flops: forward and inverse 2-D transforms of every mode, 5 N^2 log2(N^2) each
    flops, nbytes = bench.pass1_work(128, 5, 1)
    assert flops == 2 * 5 * 5 * 128 ** 2 * math.log2(128 ** 2)
    assert abs(nbytes - 1.60e6) < 0.05e6            # 1.60 MB per position
    # split-BF16 DFT-GEMM: 100.7 MFLOP per 128^2 transform (88x the FFT's 1.15 MFLOP)
    per_transform = bench.far_tc_work(128, 1, 1) / 2
    assert abs(per_transform - 100.7e6) < 0.1e6
    assert 85 < per_transform / (5 * 128 ** 2 * math.log2(128 ** 2)) < 90
    assert bench.far_tc_work(128, 5, 256) == 256 * 2 * 5 * per_transform
