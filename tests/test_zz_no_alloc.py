"""The allocation-free frame reduction (vca_reduce_frames_noalloc) against the analyzer.

The analyzer computes per-block values and, from them, the seven frame features (Section 2 of
the paper).  Here the same block values, read back from the analyzer, go through the
allocation-free entry point, whose scratch is a fixed array of the library: two calls in a row
(frames 0..5 without a previous frame, then 6..11 continuing h from the first call's last luma
energies) must give the analyzer's features within the feature tolerance, and repeating the pair
must give identical bits (the arrival counters return to zero after every call).  This file sorts
last so that it runs after the other GPU tests, and it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

from synth import frames_list, tiny_spec
from vca_testutil import FEATURES, assert_features_close, to_device

pytestmark = pytest.mark.gpu

ROWS = ("H_Y", "L_Y", "H_U", "L_U", "H_V", "L_V")


@pytest.fixture(scope="module")
def vca():
    import torch

    from paper_2304_12384_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2304_12384_gb300 import vca as v
    return v


def _analyzer_values(vca, frames):
    """Features and [frame][6][C] block values of the analyzer for a batch of frames."""
    y, u, v = to_device(frames)
    an = vca.Analyzer(width=640, height=352, bit_depth=8, block_size=32, low_pass=False, max_batch=len(frames))
    try:
        an.push(y, u, v)
        feats = [an.frame_features(t) for t in range(len(frames))]
        bv = np.stack([np.stack([an.block_values(t)[r] for r in ROWS]) for t in range(len(frames))])
    finally:
        an.close()
    return feats, bv


def _reduce(vca, bv_dev, first, count, prev, last, feats_dev, stream):
    C = bv_dev.shape[2]
    vca.vca_reduce_frames_noalloc(bv_dev[first].data_ptr(), C, 32, count,
                                  prev.data_ptr() if prev is not None else None, last.data_ptr(),
                                  feats_dev[first].data_ptr(), stream)


def test_noalloc_reduction_matches_analyzer(vca):
    import torch

    frames = frames_list(tiny_spec(11))[:12]
    exp, bv = _analyzer_values(vca, frames)
    bv_dev = torch.from_numpy(bv).cuda()
    C = bv.shape[2]
    stream = torch.cuda.Stream()
    runs = []
    for _ in range(2):
        feats_dev = torch.full((12, 8), float("nan"), dtype=torch.float64, device="cuda")
        last_a = torch.empty(C, dtype=torch.float32, device="cuda")
        last_b = torch.empty(C, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        _reduce(vca, bv_dev, 0, 6, None, last_a, feats_dev, stream.cuda_stream)
        _reduce(vca, bv_dev, 6, 6, last_a, last_b, feats_dev, stream.cuda_stream)
        stream.synchronize()
        got = feats_dev.cpu().numpy()
        assert np.array_equal(last_b.cpu().numpy(), bv[11, 0]), "last_H_Y must be the last frame's luma energies"
        for t in range(12):
            assert_features_close(dict(zip(FEATURES, got[t, :7])), exp[t], where=f"frame {t}")
            assert got[t, 7] == 0.0
        runs.append(got)
    assert np.array_equal(runs[0], runs[1]), "repeated calls must give identical features"


def test_noalloc_rejects_sizes_beyond_its_scratch(vca):
    import torch

    C = 4
    bv = torch.zeros((257, 6, C), dtype=torch.float32, device="cuda")
    last = torch.zeros(C, dtype=torch.float32, device="cuda")
    feats = torch.zeros((257, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(vca.VcaError) as ei:
        vca.vca_reduce_frames_noalloc(bv.data_ptr(), C, 32, 257, None, last.data_ptr(), feats.data_ptr(), 0)
    assert ei.value.status == vca.VCA_E_ARG
    assert "256" in str(ei.value)
    with pytest.raises(vca.VcaError) as ei:
        vca.vca_reduce_frames_noalloc(bv.data_ptr(), C, 8, 1, None, last.data_ptr(), feats.data_ptr(), 0)
    assert ei.value.status == vca.VCA_E_ARG
    with pytest.raises(vca.VcaError) as ei:
        vca.vca_reduce_frames_noalloc(bv.data_ptr(), C, 32, 1, last.data_ptr(), last.data_ptr(), feats.data_ptr(), 0)
    assert ei.value.status == vca.VCA_E_ARG


def _model_features(vals, prev, w):
    """Python-integer model of the documented reduction: each value truncated toward zero to a
    multiple of 2^-23 (values outside [0, 2^30) as 0), sums exact, rounded once to FP64, divided by
    the norm.  vals: [frames][6][C] float32; prev: C float32 or None."""
    import math

    def fx(v):
        v = float(v)
        if not (v >= 0.0) or math.copysign(1.0, v) < 0 or v >= 2.0 ** 30 or math.isinf(v):
            return 0
        return int(math.floor(v * 2 ** 23))

    C = vals.shape[2]
    nc = w // 2
    out = []
    for f in range(vals.shape[0]):
        s = [sum(fx(x) for x in vals[f, r]) for r in range(6)]
        if f > 0 or prev is not None:
            p = vals[f - 1, 0] if f > 0 else prev
            hsum = sum(abs(fx(a) - fx(b)) for a, b in zip(vals[f, 0], p))
            h = float(hsum) * 2.0 ** -23 / (C * w * w)
        else:
            h = 0.0
        g = [float(x) * 2.0 ** -23 for x in s]
        out.append([g[0] / (C * w * w), h, g[1] / C, g[2] / (C * nc * nc), g[4] / (C * nc * nc), g[3] / C, g[5] / C])
    return np.array(out)


def test_noalloc_hand_values_follow_the_documented_rounding(vca):
    import torch

    # Values that are not multiples of 2^-23, tiny values, and values the header says count as 0.
    nan, inf = float("nan"), float("inf")
    v = np.array([[[0.3, 1.5, 2.75, 0.0, 1e-9, 7.0e-8],
                   [1.25, 0.1, 3.0, 2.0 ** 29, 0.7, 0.0],
                   [0.3, -0.0, 9.5, 1.0, 4.0, 0.2],
                   [2.0, 2.0, 2.0, 2.0, 2.0, 2.0],
                   [-1.5, 0.125, 0.333, 5.0, nan, 1.0],
                   [inf, 2.0 ** 30, 6.0, 0.6, 1.0, 0.9]],
                  [[0.31, 1.4, 2.75, 0.5, 0.0, 7.0e-8],
                   [1.0, 0.1, 3.5, 1.0, 0.7, 0.0],
                   [0.4, 0.0, 9.0, 1.0, 4.5, 0.2],
                   [2.0, 1.0, 2.0, 3.0, 2.0, 2.0],
                   [1.5, 0.125, 0.333, 5.0, 0.5, 1.0],
                   [1.0, 2.0, 6.0, 0.6, 1.0, 0.9]]], dtype=np.float32)
    prev = np.array([0.2, 1.5, 3.25, 0.1, 0.0, 1.0], dtype=np.float32)
    C = v.shape[2]
    bv = torch.from_numpy(v).cuda()
    pv = torch.from_numpy(prev).cuda()
    last = torch.empty(C, dtype=torch.float32, device="cuda")
    last2 = torch.empty(C, dtype=torch.float32, device="cuda")
    feats = torch.zeros((2, 8), dtype=torch.float64, device="cuda")
    feats2 = torch.zeros((2, 8), dtype=torch.float64, device="cuda")
    vca.vca_reduce_frames_noalloc(bv.data_ptr(), C, 16, 2, pv.data_ptr(), last.data_ptr(), feats.data_ptr(), 0)
    # a later call with no previous frame and several frames: h of its frame 0 is 0
    vca.vca_reduce_frames_noalloc(bv.data_ptr(), C, 16, 2, None, last2.data_ptr(), feats2.data_ptr(), 0)
    torch.cuda.synchronize()
    assert np.array_equal(feats.cpu().numpy()[:, :7], _model_features(v, prev, 16))
    assert np.array_equal(feats2.cpu().numpy()[:, :7], _model_features(v, None, 16))
    assert np.array_equal(last.cpu().numpy(), v[1, 0]) and np.array_equal(last2.cpu().numpy(), v[1, 0])


def test_noalloc_rejects_overlapping_outputs(vca):
    import torch

    C = 8
    bv = torch.zeros((2, 6, C), dtype=torch.float32, device="cuda")
    buf = torch.zeros(3 * C, dtype=torch.float32, device="cuda")
    feats = torch.zeros((2, 8), dtype=torch.float64, device="cuda")
    fp = buf.data_ptr()
    cases = [
        (fp, fp + 4 * (C // 2)),       # last_H_Y half over prev_H_Y
        (fp + 4 * (C - 1), fp),        # prev_H_Y's last value under last_H_Y
    ]
    for prev, last in cases:
        with pytest.raises(vca.VcaError) as ei:
            vca.vca_reduce_frames_noalloc(bv.data_ptr(), C, 32, 2, prev, last, feats.data_ptr(), 0)
        assert ei.value.status == vca.VCA_E_ARG and "overlaps prev_H_Y" in str(ei.value)
    # last_H_Y inside the block values of the last frame
    with pytest.raises(vca.VcaError) as ei:
        vca.vca_reduce_frames_noalloc(bv.data_ptr(), C, 32, 2, None, bv[1, 3].data_ptr(), feats.data_ptr(), 0)
    assert ei.value.status == vca.VCA_E_ARG and "overlaps block_values" in str(ei.value)
    # adjacent, not overlapping: accepted
    vca.vca_reduce_frames_noalloc(bv.data_ptr(), C, 32, 2, fp, fp + 4 * C, feats.data_ptr(), 0)
    torch.cuda.synchronize()
