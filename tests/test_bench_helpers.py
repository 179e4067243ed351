"""The benchmark's own arithmetic, on CPU: algorithmic work per window, the
launch counts it claims, and the staleness rule of the committed ncu traffic
figures.  These numbers enter every roofline fraction the benchmark prints."""
import argparse
import dataclasses
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2504_10118_gb300 import synth  # noqa: E402


def test_fp32_flops_per_window_closed_form():
    # M (10 log2 M + 60): two 2-D FFTs at 5 M log2 M each plus 60 M element-wise
    assert bench.flops_per_window(128) == 16384 * (10 * 14 + 60) == 3_276_800
    assert bench.flops_per_window(32) == 1024 * (10 * 10 + 60)
    assert bench.flops_per_window(256) == pytest.approx(65536 * (10 * 16 + 60))


def test_hbm_bytes_per_window_are_the_amplitudes():
    assert bench.hbm_bytes_per_window(128) == 4 * 128 * 128


def test_tensor_flops_per_window_by_brute_count():
    """Count the real block-GEMM multiply-adds of one line's DFT directly:
    stage 1, the 32 x 32 DFT-16 block matrix times 32 x Qr; stage 2, m rows
    of depth 2 Qr (padded to a multiple of 16) times 2 Qr columns."""
    for m in (64, 128, 256):
        qr = m // 16
        depth2 = 16 * math.ceil(2 * qr / 16)
        stage1 = 2 * 32 * 32 * qr           # flops: 2 per multiply-add
        stage2 = 2 * 16 * depth2 * 2 * qr   # 16 rows of k1 per line
        per_window = 2 * m * (stage1 + stage2) * 2 * 3  # rows and columns, forward and inverse, three products
        assert bench.tc_flops_per_window(m) == per_window
    assert bench.tc_flops_per_window(256) == 201_326_592


def test_cnn_flops_per_window():
    h = 32
    layers = [(4, 32, 32), (32, 64, 16), (64, 128, 8), (128, 512, 4), (512, 64, 8), (64, 2, 32)]
    assert bench.cnn_flops_per_window(h) == sum(2 * 9 * a * b * s * s for a, b, s in layers)


@pytest.mark.parametrize("dft,levels,expected", [("fft", 3, 2), ("tc", 4, 5), ("tcgen05", 3, 5), ("tc", 2, 4),
                                                 ("tc", 1, 4)])
def test_launches_per_step(dft, levels, expected):
    """Window kernel + update for the FP32 path; for the precision form the
    three transform kernels, the coarse levels from three levels on, and the
    update (which forms the finest level itself)."""
    w = dataclasses.replace(synth.WORKLOADS["precision"], levels=levels)
    args = argparse.Namespace(learned=False, dft=dft)
    assert bench.launches_per_step(args, w) == expected


def test_committed_traffic_figures_match_the_running_source():
    """Both ncu summaries the roofline's traffic comes from were taken on the
    window kernel's current source (else the benchmark reports null)."""
    h = bench.kernel_source_hash()
    for det, path in bench.TRAFFIC_FILES.items():
        kv = dict(ln.split(":", 1) for ln in open(path).read().splitlines() if ":" in ln)
        assert kv["source_sha256"].strip() == h, path
        assert bench.measured_traffic(det) == float(kv["dram_bytes_per_launch"])


def test_traffic_is_null_once_the_source_changes(tmp_path, monkeypatch):
    edited = tmp_path / "window_body.inc"
    edited.write_text(open(bench.KERNEL_SOURCES[-1]).read() + "\n// edited\n")
    monkeypatch.setattr(bench, "KERNEL_SOURCES", bench.KERNEL_SOURCES[:-1] + [str(edited)])
    assert bench.measured_traffic(0) is None
    assert bench.measured_traffic(1) is None


def test_nrmse_lit_removes_the_global_phase_and_masks_unlit_pixels():
    import numpy as np
    rng = np.random.default_rng(0)
    n, m = 24, 8
    z_true = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    q2 = np.ones((m, m))
    pos = np.array([[0, 0], [0, 8], [8, 0]])  # pixels [8:, 8:] and [16:, :] etc. stay unlit
    assert bench.nrmse_lit(np.exp(0.7j) * z_true, z_true, q2, pos) == pytest.approx(0.0, abs=1e-12)
    z = z_true.copy()
    z[20:, 20:] += 100.0  # unlit: no effect
    assert bench.nrmse_lit(z, z_true, q2, pos) == pytest.approx(0.0, abs=1e-12)
    z = 2.0 * z_true  # |2b - b| / |b| = 1 on the lit pixels
    assert bench.nrmse_lit(z, z_true, q2, pos) == pytest.approx(1.0)
