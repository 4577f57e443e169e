"""Host logic of the benchmark's roofline bookkeeping (no GPU needed)."""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_stage_bytes_of_the_1e5_node_tangle():
    """384^3 grid, modes |m| <= 127, 2e5 sources, float32: the fused spread
    reads 32 B per source and writes 3 x 384 x 384 x 128 complex modes; the
    y passes move F1 (384 y-rows) and F2 (255 y-modes); the x pass reads and
    writes F2."""
    ms = {k: 1.0 for k in ("spread", "fft_fwd", "kspace", "fft_inv", "interp")}
    r = bench.stage_rooflines([384] * 3, [127] * 3, 200000, 100000, 6, 4, ms, 1000.0)
    full = 3 * 384 * 384 * 128 * 8
    half = 3 * 384 * 255 * 128 * 8
    assert r["spread"]["bytes"] == 32 * 200000 + full == 459384832
    assert r["fft_fwd"]["bytes"] == r["fft_inv"]["bytes"] == full + half
    assert r["kspace"]["bytes"] == 2 * half
    # 80-byte sorted node record (8 + 18 float weights, rounded to 16), sums, final float64 sum
    assert r["interp"]["bytes"] == full + 100000 * (80 + 12 + 12 + 72)
    assert r["spread"]["gbs"] == pytest.approx(459384832 / 1e-3 / 1e9)
    assert r["spread"]["frac"] == pytest.approx(r["spread"]["gbs"] / 1000.0)


def test_short_range_pair_estimate():
    # (4 pi / 3) r_c^3 NQ / V sources inside r_c per node
    L = [2 * math.pi] * 3
    n = bench.short_range_pairs(0.5, L, 10, 1000)
    assert n == pytest.approx(10 * 4 / 3 * math.pi * 0.125 * 1000 / (2 * math.pi) ** 3)


def test_source_digest_ignores_comments_and_layout(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("int f(int x) { return x + 1; }  // one\n")
    b.write_text("/* header */\nint f(int x)\n{\n    return x + 1;\n}\n")
    c.write_text("int f(int x) { return x + 2; }\n")
    assert bench.source_digest(str(a)) == bench.source_digest(str(b))
    assert bench.source_digest(str(a)) != bench.source_digest(str(c))
