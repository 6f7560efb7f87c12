"""Serving runtime: channels, segment submission, continuous batching on the native scheduler
thread, and admission by device memory.

Three channels of different frame sizes and bit depths submit segments of 4 frames; the
scheduler analyses one frame of every channel with a segment in progress per tick.  Each
channel's features must equal, bit for bit, those of a single analyzer fed the same frames (the
same kernel's arithmetic), match the oracle, and the h state must carry from one segment to the next.
"""

import time

import pytest

from synth import SequenceSpec, frames_list
from vca_testutil import assert_features_close, oracle_config, oracle_sequence, to_device

pytestmark = pytest.mark.gpu

CHANNELS = [(640, 352, 8), (320, 180, 10), (656, 368, 8)]
SEG = 4
NSEG = 3


@pytest.fixture(scope="module")
def vca():
    import torch

    from paper_2304_12384_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2304_12384_gb300 import vca as v
    return v


def _wait(srv, n, timeout=60.0):
    got = []
    t0 = time.monotonic()
    while len(got) < n:
        got += srv.poll()
        if time.monotonic() - t0 > timeout:
            raise TimeoutError(f"{len(got)} of {n} segments finished")
        time.sleep(0.001)
    return got


def test_server_segments_match_single_analyzers(vca):
    import torch

    frames = [frames_list(SequenceSpec(w, h, SEG * NSEG, 800 + i, bit_depth=bd, sigma=4.0, cuts=(5,)))
              for i, (w, h, bd) in enumerate(CHANNELS)]
    dev = [to_device(f) for f in frames]
    with vca.Server() as srv:
        ids = [srv.add_channel(w, h, bd, 32, True, max_segment_frames=SEG) for (w, h, bd) in CHANNELS]
        done = []
        pending = [(i, k) for k in range(NSEG) for i in range(len(CHANNELS))]
        t0 = time.monotonic()
        while pending:
            i, k = pending[0]
            y, u, v = dev[i]
            sl = slice(k * SEG, (k + 1) * SEG)
            st = srv.submit_frames(ids[i], y[sl], u[sl], v[sl], tag=100 * i + k)
            if st == vca.VCA_E_AGAIN:  # both slots of the channel busy: collect finished segments
                done += srv.poll()
                time.sleep(0.001)
                assert time.monotonic() - t0 < 60
                continue
            pending.pop(0)
        done += _wait(srv, len(CHANNELS) * NSEG - len(done))
        assert sorted(d["tag"] for d in done) == sorted(100 * i + k for i in range(len(CHANNELS)) for k in range(NSEG))
        for d in done:
            assert d["status"] == vca.VCA_OK
            assert d["n_frames"] == SEG and d["first_frame"] == SEG * (d["tag"] % 100)
            assert d["ready_ns"] >= d["submit_ns"]
        stats = srv.stats()
        assert stats["frames"] == SEG * NSEG * len(CHANNELS) and stats["channels"] == len(CHANNELS)
        assert stats["ticks"] <= stats["frames"]
        for i, (w, h, bd) in enumerate(CHANNELS):
            got = [srv.frame_features(ids[i], t) for t in range(SEG * NSEG)]
            single = vca.Analyzer(w, h, bd, 32, True, max_batch=SEG)  # the channel's kernel
            y, u, v = dev[i]
            for k in range(NSEG):
                sl = slice(k * SEG, (k + 1) * SEG)
                single.push(y[sl], u[sl], v[sl])
            exp = [single.frame_features(t) for t in range(SEG * NSEG)]
            single.close()
            assert got == exp, f"channel {i}"
            per, _ = oracle_sequence(frames[i], oracle_config(single))
            for t, e in enumerate(per):
                assert_features_close(got[t], e, where=f"channel {i} frame {t}")
    torch.cuda.synchronize()


def test_server_admission_by_device_memory(vca):
    with vca.Server(device_budget_bytes=256 << 20) as srv:
        with pytest.raises(vca.VcaError) as ei:
            srv.add_channel(3840, 2160, 10, 32, True, max_segment_frames=120)
        assert ei.value.status == vca.VCA_E_NOMEM
        assert "admission" in str(ei.value)
        cid = srv.add_channel(640, 360, 8, 32, True, max_segment_frames=8)
        st = srv.stats()
        assert st["channels"] == 1 and 0 < st["used_bytes"] <= st["budget_bytes"] == 256 << 20
        assert cid == 0
