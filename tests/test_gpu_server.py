"""Serving runtime: channels, segment submission, the native scheduler thread under both
policies (segments as multi-frame work items; frame-interleaved batched ticks), and admission by
device memory.

Three channels of different frame sizes and bit depths submit segments of 4 frames.  Each
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


@pytest.mark.parametrize("policy", ["segments", "ticks"])
def test_server_segments_match_single_analyzers(vca, policy):
    import torch

    frames = [frames_list(SequenceSpec(w, h, SEG * NSEG, 800 + i, bit_depth=bd, sigma=4.0, cuts=(5,)))
              for i, (w, h, bd) in enumerate(CHANNELS)]
    dev = [to_device(f) for f in frames]
    pol = vca.VCA_SERVE_SEGMENTS if policy == "segments" else vca.VCA_SERVE_TICKS
    with vca.Server(policy=pol) as srv:
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
        if policy == "segments":
            assert stats["ticks"] == NSEG * len(CHANNELS)  # one push per segment
        else:
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


def _run_channels(vca, srv, chans, frames, nseg, seg):
    """Submits nseg segments of seg frames per channel and waits for them; returns the channel ids."""
    ids = [srv.add_channel(**c, max_segment_frames=seg) for c in chans]
    dev = [to_device(f) for f in frames]
    pending = [(i, k) for k in range(nseg) for i in range(len(chans))]
    done = []
    t0 = time.monotonic()
    while pending:
        i, k = pending[0]
        y, u, v = dev[i]
        sl = slice(k * seg, (k + 1) * seg)
        if srv.submit_frames(ids[i], y[sl], u[sl], v[sl], tag=1000 * i + k) == vca.VCA_E_AGAIN:
            done += srv.poll()
            time.sleep(0.001)
            assert time.monotonic() - t0 < 120
            continue
        pending.pop(0)
    done += _wait(srv, len(chans) * nseg - len(done))
    assert all(d["status"] == vca.VCA_OK for d in done)
    return ids


def test_server_segments_policy_mixes_configurations(vca):
    # Under the segments policy channels need not share block size or chroma format: 32x32 and
    # 16x16 blocks, 4:2:0 and 4:2:2, low-pass and all coefficients side by side.
    chans = [dict(width=320, height=180, bit_depth=8, block_size=32, low_pass=True),
             dict(width=200, height=120, bit_depth=10, block_size=16, low_pass=False),
             dict(width=256, height=144, bit_depth=8, block_size=16, low_pass=True,
                  chroma_format=vca.VCA_CHROMA_422)]
    cf = {vca.VCA_CHROMA_422: "422"}
    frames = [frames_list(SequenceSpec(c["width"], c["height"], 6, 860 + i, bit_depth=c["bit_depth"], sigma=5.0,
                                       chroma_format=cf.get(c.get("chroma_format", 0), "420")))
              for i, c in enumerate(chans)]
    with vca.Server(policy=vca.VCA_SERVE_SEGMENTS) as srv:
        ids = _run_channels(vca, srv, chans, frames, 2, 3)
        for i, c in enumerate(chans):
            got = [srv.frame_features(ids[i], t) for t in range(6)]
            single = vca.Analyzer(c["width"], c["height"], c["bit_depth"], c["block_size"], c["low_pass"], max_batch=6,
                                  chroma_format=c.get("chroma_format", 0))
            single.push(*to_device(frames[i]))
            exp = [single.frame_features(t) for t in range(6)]
            per, _ = oracle_sequence(frames[i], oracle_config(single))
            single.close()
            assert got == exp, f"channel {i}"
            for t, e in enumerate(per):
                assert_features_close(got[t], e, where=f"channel {i} frame {t}")


def test_server_long_segment_takes_several_pushes(vca):
    # A 130-frame segment is pushed as 128 + 2 frames; the h chain crosses the push boundary.
    frames = frames_list(SequenceSpec(136, 72, 130, 870, sigma=4.0, cuts=(127,)))
    with vca.Server(policy=vca.VCA_SERVE_SEGMENTS) as srv:
        ids = _run_channels(vca, srv, [dict(width=136, height=72, bit_depth=8, block_size=32, low_pass=True)],
                            [frames], 1, 130)
        got = [srv.frame_features(ids[0], t) for t in range(130)]
        assert srv.stats()["ticks"] == 2
    single = vca.Analyzer(136, 72, 8, 32, True, max_batch=130)
    single.push(*to_device(frames))
    exp = [single.frame_features(t) for t in range(130)]
    single.close()
    assert got == exp
    per, _ = oracle_sequence(frames, oracle_config_for(vca, 136, 72))
    for t in (0, 1, 126, 127, 128, 129):
        assert_features_close(got[t], per[t], where=f"frame {t}")


def oracle_config_for(vca, w, h):
    an = vca.Analyzer(w, h, 8, 32, True, max_batch=1)
    try:
        return oracle_config(an)
    finally:
        an.close()


def test_server_policy_rules(vca):
    with vca.Server() as srv:
        with pytest.raises(vca.VcaError) as ei:
            vca.vca_server_set_policy(srv.handle, 7)
        assert ei.value.status == vca.VCA_E_ARG
        srv.add_channel(320, 180, 8, 32, True, max_segment_frames=4)
        with pytest.raises(vca.VcaError) as ei:
            vca.vca_server_set_policy(srv.handle, vca.VCA_SERVE_TICKS)
        assert ei.value.status == vca.VCA_E_STATE
