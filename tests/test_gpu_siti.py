"""SI / TI on the GPU (the paper's comparison features, Section 2) against the oracle.

SI sums an FP32 square root per pixel in 2^-16 fixed point (relative error of a term below
2^-23 + 2^-17 / magnitude), so SI is compared within 1e-6 relative (plus 1e-9 absolute for a
zero deviation); TI is formed from exact integer sums and compared within 1e-12.
"""

import numpy as np
import pytest

from oracle import siti_sequence
from synth import SequenceSpec, frames_list, uhd_spec
from vca_testutil import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vca():
    import torch

    from paper_2304_12384_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2304_12384_gb300 import vca as v
    return v


def _check(got, exp):
    assert got["SI"] == pytest.approx(exp["SI"], rel=1e-6, abs=1e-9)
    assert got["TI"] == pytest.approx(exp["TI"], rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("bit_depth", [8, 10, 12])
@pytest.mark.parametrize("size", [(640, 352), (203, 117)])
def test_siti_matches_oracle(vca, bit_depth, size):
    w, h = size
    frames = frames_list(SequenceSpec(w, h, 7, 61, bit_depth=bit_depth, sigma=4.0, cuts=(4,)))
    y = to_device(frames)[0]
    per, seq = siti_sequence([f[0] for f in frames])
    s = vca.Siti(w, h, bit_depth, max_batch=4)
    try:
        s.push(y[:3])   # TI of frame 3 uses frame 2 kept on the device from this push
        s.push(y[3:4])
        s.push(y[4:])
        for t in range(7):
            _check(s.frame_features(t), per[t])
        got = s.sequence_features()
        assert got["frames"] == 7
        _check(got, seq)
    finally:
        s.close()


def test_siti_host_frames_and_edge_cases(vca):
    import torch

    frames = frames_list(SequenceSpec(96, 64, 3, 62))
    host = torch.from_numpy(np.ascontiguousarray(np.stack([f[0] for f in frames])))
    per, _ = siti_sequence([f[0] for f in frames])
    with vca.Siti(96, 64, 8, max_batch=3) as s:
        s.push(host)
        for t in range(3):
            _check(s.frame_features(t), per[t])
    flat = torch.full((2, 8, 16), 77, dtype=torch.uint8, device="cuda")
    with vca.Siti(16, 8, 8, max_batch=2) as s:
        s.push(flat)
        assert s.frame_features(0) == {"SI": 0.0, "TI": 0.0} and s.frame_features(1) == {"SI": 0.0, "TI": 0.0}
    with pytest.raises(vca.VcaError):
        vca.Siti(2, 8, 8)


def test_siti_2160p_sample(vca):
    frames = frames_list(uhd_spec(3, 4), 0, 2)
    y = to_device(frames)[0]
    per, _ = siti_sequence([f[0] for f in frames])
    with vca.Siti(3840, 2160, 8, max_batch=2) as s:
        s.push(y)
        for t in range(2):
            _check(s.frame_features(t), per[t])
