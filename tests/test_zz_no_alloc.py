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
