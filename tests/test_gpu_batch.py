"""Batched multi-stream ticks (one frame of every channel per tick, replayed from a CUDA graph:
on tensor cores one launch per sample size that also reduces each frame to its features, on CUDA
cores one launch of the block kernel and one of the reduction) against single analyzers and the
oracle.

Channels of one batch differ in frame size (ragged block grids included) and bit depth; some
ticks skip a channel.  Each channel's features must equal, bit for bit, those of its own
analyzer fed the same frames one at a time through the plain kernel (same arithmetic), and
match the oracle within the feature tolerance; the h state must carry across ticks, skipped
ticks and the batch's destruction.
"""

import pytest

from synth import SequenceSpec, frames_list
from vca_testutil import assert_features_close, oracle_config, oracle_sequence, to_device

pytestmark = pytest.mark.gpu

CHANNELS = [  # (width, height, bit depth)
    (640, 352, 8),
    (320, 180, 10),
    (656, 368, 8),
    (200, 120, 10),
]
TICKS = 6
SKIP = {(3, 2), (1, 0)}  # (tick, channel) pairs left out


@pytest.fixture(scope="module")
def vca():
    import torch

    from paper_2304_12384_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2304_12384_gb300 import vca as v
    return v


def _channel_frames(i, w, h, bd):
    spec = SequenceSpec(w, h, TICKS + 2, 700 + i, bit_depth=bd, sigma=4.0, cuts=(4,), motion=4)
    return frames_list(spec)


CHANNELS_8 = [(640, 352, 8), (656, 368, 8), (200, 120, 8)]
CHANNELS_10 = [(320, 180, 10), (200, 120, 10), (136, 72, 10)]
CASES = [  # (kernel, channels): the tensor-core batch with one sample size (bytes or words) and mixed
    ("plain", CHANNELS),
    ("tc", CHANNELS),
    ("tc", CHANNELS_8),
    ("tc", CHANNELS_10),
]


@pytest.mark.parametrize("block_size", [32, 16])
@pytest.mark.parametrize("low_pass", [True, False])
@pytest.mark.parametrize("kind,channels", CASES, ids=["plain", "tc-mixed", "tc-8bit", "tc-10bit"])
def test_batch_matches_single_analyzers_and_oracle(vca, block_size, low_pass, kind, channels):
    import torch

    kernel = vca.VCA_KERNEL_TC if kind == "tc" else vca.VCA_KERNEL_PLAIN
    frames = [_channel_frames(i, *c) for i, c in enumerate(channels)]
    dev = [to_device(f) for f in frames]
    members = [vca.Analyzer(w, h, bd, block_size, low_pass, kernel=kernel, max_batch=4) for (w, h, bd) in channels]
    singles = [vca.Analyzer(w, h, bd, block_size, low_pass, kernel=kernel, max_batch=4) for (w, h, bd) in channels]
    fed = [[] for _ in channels]
    try:
        batch = vca.Batch(members)
        assert batch.kernel == kernel
        for t in range(TICKS):
            refs = []
            for i in range(len(channels)):
                if (t, i) in SKIP:
                    refs.append(None)
                    continue
                y, u, v = dev[i]
                refs.append((y[t], u[t], v[t]))
                singles[i].push(y[t], u[t], v[t])
                fed[i].append(t)
            batch.tick(refs)
        batch.sync()
        # tensor cores: one launch per sample size, the reduction inside; CUDA cores: the block
        # kernel, then the reduction
        per_tick = len({bd > 8 for (_, _, bd) in channels}) if kind == "tc" else 2
        assert batch.launches() == per_tick * TICKS
        for i, (w, h, bd) in enumerate(channels):
            got = [members[i].frame_features(k) for k in range(len(fed[i]))]
            exp = [singles[i].frame_features(k) for k in range(len(fed[i]))]
            assert got == exp, f"channel {i}"
            cfg = oracle_config(members[i])
            per, seqf = oracle_sequence([frames[i][t] for t in fed[i]], cfg)
            for k, e in enumerate(per):
                assert_features_close(got[k], e, where=f"channel {i} frame {k}")
            assert_features_close(members[i].sequence_features(), seqf, where=f"channel {i} sequence")
        batch.close()
        # The h state continues after the batch is gone.
        for i in range(len(channels)):
            y, u, v = dev[i]
            members[i].push(y[TICKS], u[TICKS], v[TICKS])
            singles[i].push(y[TICKS], u[TICKS], v[TICKS])
            k = len(fed[i])
            assert members[i].frame_features(k) == singles[i].frame_features(k)
        torch.cuda.synchronize()
    finally:
        for a in members + singles:
            try:
                a.close()
            except vca.VcaError:
                pass


def test_batch_state_rules(vca):
    a = vca.Analyzer(640, 352, 8, 32, True, kernel=vca.VCA_KERNEL_PLAIN, max_batch=2)
    b = vca.Analyzer(320, 180, 10, 32, True, kernel=vca.VCA_KERNEL_PLAIN, max_batch=2)
    c = vca.Analyzer(320, 180, 8, 16, True, kernel=vca.VCA_KERNEL_PLAIN, max_batch=2)
    d = vca.Analyzer(320, 180, 8, 32, False, kernel=vca.VCA_KERNEL_PLAIN, max_batch=2)
    try:
        for bad in ([a, c], [a, d], [a, a]):
            with pytest.raises(vca.VcaError) as ei:
                vca.Batch(bad)
            assert ei.value.status == vca.VCA_E_ARG
        batch = vca.Batch([a, b])
        frames = to_device(frames_list(SequenceSpec(640, 352, 1, 9), 0, 1))
        with pytest.raises(vca.VcaError) as ei:
            a.push(frames[0][0], frames[1][0], frames[2][0])
        assert ei.value.status == vca.VCA_E_STATE
        with pytest.raises(vca.VcaError) as ei:
            vca.vca_close(a.handle)
        assert ei.value.status == vca.VCA_E_STATE
        with pytest.raises(vca.VcaError) as ei:
            vca.Batch([a])
        assert ei.value.status == vca.VCA_E_STATE
        # A misaligned plane pointer is rejected before anything is queued.
        y, u, v = frames
        with pytest.raises(vca.VcaError) as ei:
            batch.tick([(y[0][:, 1:], u[0], v[0]), None])
        assert ei.value.status == vca.VCA_E_ARG
        batch.tick([(y[0], u[0], v[0]), None])
        assert batch.kernel == vca.VCA_KERNEL_PLAIN
        batch.close()
        assert a.frame_features(0)["h"] == 0.0
        # One member off the tensor-core kernel puts the whole batch on the CUDA-core kernel.
        e = vca.Analyzer(640, 352, 8, 32, True, kernel=vca.VCA_KERNEL_TC, max_batch=2)
        try:
            with vca.Batch([e, b]) as mixed:
                assert mixed.kernel == vca.VCA_KERNEL_PLAIN
            with vca.Batch([e]) as alone:
                assert alone.kernel == vca.VCA_KERNEL_TC
        finally:
            e.close()
    finally:
        for x in (a, b, c, d):
            x.close()


@pytest.mark.parametrize("block_size", [32, 16])
def test_tc_batch_444(vca, block_size):
    # 4:4:4 channels (8- and 10-bit) tick on the tensor-core kernel, each plane of a tile a work item;
    # features equal the single analyzers' bit for bit and the oracle.
    chans = [(200, 120, 8), (136, 72, 10), (256, 144, 8)]
    frames = [frames_list(SequenceSpec(w, h, 3, 70 + i, bit_depth=bd, sigma=4.0, chroma_format="444"))
              for i, (w, h, bd) in enumerate(chans)]
    dev = [to_device(f) for f in frames]
    members = [vca.Analyzer(w, h, bd, block_size, True, max_batch=3, chroma_format=vca.VCA_CHROMA_444)
               for (w, h, bd) in chans]
    singles = [vca.Analyzer(w, h, bd, block_size, True, max_batch=3, chroma_format=vca.VCA_CHROMA_444)
               for (w, h, bd) in chans]
    try:
        with vca.Batch(members) as batch:
            assert batch.kernel == vca.VCA_KERNEL_TC
            for t in range(3):
                batch.tick([(y[t], u[t], v[t]) for (y, u, v) in dev])
                for s_, (y, u, v) in zip(singles, dev):
                    s_.push(y[t], u[t], v[t])
        for i, (m, s_) in enumerate(zip(members, singles)):
            got = [m.frame_features(t) for t in range(3)]
            assert got == [s_.frame_features(t) for t in range(3)], f"channel {i}"
            per, _ = oracle_sequence(frames[i], oracle_config(m))
            for t in range(3):
                assert_features_close(got[t], per[t], where=f"channel {i} frame {t}")
    finally:
        for a in members + singles:
            a.close()


def test_batch_444_422_and_block_8(vca):
    # Batches of 4:4:4 channels, of 4:2:2 channels and of 8 x 8-block channels match single
    # analyzers bit for bit.
    for kw in ({"chroma_format": vca.VCA_CHROMA_444, "block_size": 16}, {"chroma_format": 0, "block_size": 8},
               {"chroma_format": vca.VCA_CHROMA_422, "block_size": 32}, {"chroma_format": vca.VCA_CHROMA_422, "block_size": 8}):
        cf = {1: "444", 2: "422"}.get(kw["chroma_format"], "420")
        chans = [(200, 120, 8), (136, 72, 12)]
        frames = [frames_list(SequenceSpec(w, h, 3, 60 + i, bit_depth=bd, sigma=4.0, chroma_format=cf))
                  for i, (w, h, bd) in enumerate(chans)]
        dev = [to_device(f) for f in frames]
        members = [vca.Analyzer(w, h, bd, kw["block_size"], False, kernel=vca.VCA_KERNEL_PLAIN, max_batch=3,
                                chroma_format=kw["chroma_format"]) for (w, h, bd) in chans]
        singles = [vca.Analyzer(w, h, bd, kw["block_size"], False, kernel=vca.VCA_KERNEL_PLAIN, max_batch=3,
                                chroma_format=kw["chroma_format"]) for (w, h, bd) in chans]
        batch = vca.Batch(members)
        for t in range(3):
            batch.tick([(y[t], u[t], v[t]) for (y, u, v) in dev])
            for s_, (y, u, v) in zip(singles, dev):
                s_.push(y[t], u[t], v[t])
        batch.close()
        for m, s_ in zip(members, singles):
            assert [m.frame_features(t) for t in range(3)] == [s_.frame_features(t) for t in range(3)]
            m.close()
            s_.close()
    # 4:2:0 and 4:2:2 channels with the same block size do not share a batch
    a = vca.Analyzer(200, 120, 8, 32, False, kernel=vca.VCA_KERNEL_PLAIN)
    b = vca.Analyzer(200, 120, 8, 32, False, kernel=vca.VCA_KERNEL_PLAIN, chroma_format=vca.VCA_CHROMA_422)
    try:
        with pytest.raises(vca.VcaError) as ei:
            vca.Batch([a, b])
        assert ei.value.status == vca.VCA_E_ARG
    finally:
        a.close()
        b.close()


def test_batch_with_drop_in_matrices(vca):
    # Members sharing a drop-in matrix stay on the tensor-core kernel; members whose matrices differ
    # share a batch on the CUDA-core kernel.  Either way each channel matches its single analyzer.
    from vca_testutil import structured_dct_matrix

    m32 = structured_dct_matrix(32, (((32, 0, 0), -1), ((16, 3, 4), 1)))
    chans = [(640, 352, 8), (320, 180, 10)]
    frames = [frames_list(SequenceSpec(w, h, 3, 90 + i, bit_depth=bd, sigma=4.0)) for i, (w, h, bd) in enumerate(chans)]
    dev = [to_device(f) for f in frames]
    for same in (True, False):
        members = [vca.Analyzer(w, h, bd, 32, True, max_batch=3) for (w, h, bd) in chans]
        singles = [vca.Analyzer(w, h, bd, 32, True, max_batch=3) for (w, h, bd) in chans]
        for i, (a, s_) in enumerate(zip(members, singles)):
            if same or i == 0:
                a.set_dct_matrix(32, m32)
                s_.set_dct_matrix(32, m32)
        batch = vca.Batch(members)
        assert batch.kernel == (vca.VCA_KERNEL_TC if same else vca.VCA_KERNEL_PLAIN)
        for t in range(3):
            batch.tick([(y[t], u[t], v[t]) for (y, u, v) in dev])
            for s_, (y, u, v) in zip(singles, dev):
                s_.push(y[t], u[t], v[t])
        batch.close()
        for i, (m, s_) in enumerate(zip(members, singles)):
            got = [m.frame_features(t) for t in range(3)]
            if same:  # same kernel as the single analyzer: identical bits
                assert got == [s_.frame_features(t) for t in range(3)]
            per, _ = oracle_sequence(frames[i], oracle_config(m))
            for t, e in enumerate(per):
                assert_features_close(got[t], e, where=f"channel {i} frame {t} (same={same})")
            m.close()
            s_.close()


def test_batch_beyond_one_member_table_stays_on_tensor_cores(vca):
    # A tensor-core launch holds at most 64 members: 66 8-bit and 5 10-bit analyzers tick as three
    # launches (8-bit: 64 + 2 members, one after another; 10-bit: 5, beside them), each reducing
    # its members' frames, every member matching its single analyzer bit for bit and the oracle;
    # one member skips a tick.
    n8, n10 = 66, 5
    f8 = frames_list(SequenceSpec(64, 64, 3, 95, sigma=4.0))
    f10 = frames_list(SequenceSpec(64, 64, 3, 96, bit_depth=10, sigma=4.0))
    d8, d10 = to_device(f8), to_device(f10)
    members = [vca.Analyzer(64, 64, 8, 32, True, max_batch=1) for _ in range(n8)] + \
              [vca.Analyzer(64, 64, 10, 32, True, max_batch=1) for _ in range(n10)]
    single8 = vca.Analyzer(64, 64, 8, 32, True, max_batch=1)
    single10 = vca.Analyzer(64, 64, 10, 32, True, max_batch=1)
    try:
        assert members[0].kernel == vca.VCA_KERNEL_TC
        with vca.Batch(members) as batch:
            assert batch.kernel == vca.VCA_KERNEL_TC
            for t in range(3):
                refs = [(d8[0][t], d8[1][t], d8[2][t])] * n8 + [(d10[0][t], d10[1][t], d10[2][t])] * n10
                if t == 1:
                    refs[65] = None
                batch.tick(refs)
                single8.push(d8[0][t], d8[1][t], d8[2][t])
                single10.push(d10[0][t], d10[1][t], d10[2][t])
            batch.sync()
            assert batch.launches() == 3 * 3
        exp8 = [single8.frame_features(t) for t in range(3)]
        exp10 = [single10.frame_features(t) for t in range(3)]
        for i in (0, 1, 63, 64):
            assert [members[i].frame_features(t) for t in range(3)] == exp8, f"member {i}"
        for i in range(n8, n8 + n10):
            assert [members[i].frame_features(t) for t in range(3)] == exp10, f"member {i}"
        # member 65 skipped tick 1: its second frame is tick 2's frame, with h against tick 0's
        got = [members[65].frame_features(t) for t in range(2)]
        assert got[0] == exp8[0] and got[1]["E_Y"] == exp8[2]["E_Y"]
        for fr, single, lst in ((f8, single8, exp8), (f10, single10, exp10)):
            per, _ = oracle_sequence(fr, oracle_config(single))
            for t in range(3):
                assert_features_close(lst[t], per[t], where=f"frame {t}")
    finally:
        for a in members + [single8, single10]:
            a.close()


@pytest.mark.parametrize("ring", [3, 10])
def test_batch_ticks_from_a_ring_of_buffers(vca, ring):
    # Frames ticked from a ring of resident buffers rewritten in place, through tick arguments built
    # once per ring slot: the batch reuses each member's tensor maps by plane address (ring 3: every
    # tick after the first three hits; ring 10: more slots than a member keeps, so entries are
    # replaced).  Each channel matches its single analyzer fed the same frames, bit for bit.
    import torch

    ticks = 14
    chans = CHANNELS
    frames = [frames_list(SequenceSpec(w, h, ticks, 500 + i, bit_depth=bd, sigma=4.0, cuts=(7,), motion=3))
              for i, (w, h, bd) in enumerate(chans)]
    dev = [to_device(f) for f in frames]
    rings = [tuple(torch.empty((ring,) + tuple(p.shape[1:]), dtype=p.dtype, device=p.device) for p in d)
             for d in dev]
    members = [vca.Analyzer(w, h, bd, 32, True, max_batch=2) for (w, h, bd) in chans]
    singles = [vca.Analyzer(w, h, bd, 32, True, max_batch=2) for (w, h, bd) in chans]
    try:
        with vca.Batch(members) as batch:
            assert batch.kernel == vca.VCA_KERNEL_TC
            slots = [batch.frame_refs([(ry[s], ru[s], rv[s]) for (ry, ru, rv) in rings]) for s in range(ring)]
            with pytest.raises(ValueError):
                batch.frame_refs([(rings[0][0][0], rings[0][1][0], rings[0][2][0])])
            for t in range(ticks):
                s = t % ring
                for d, r in zip(dev, rings):
                    for p, rp in zip(d, r):
                        rp[s].copy_(p[t])
                torch.cuda.synchronize()
                batch.tick(slots[s])
                batch.sync()
                for a, (y, u, v) in zip(singles, dev):
                    a.push(y[t], u[t], v[t])
        for i, (m, a) in enumerate(zip(members, singles)):
            got = [m.frame_features(t) for t in range(ticks)]
            assert got == [a.frame_features(t) for t in range(ticks)], f"channel {i}"
    finally:
        for a in members + singles:
            a.close()


def test_batch_tick_without_one_sample_size(vca):
    # Ticks in which every 8-bit or every 10-bit member of a mixed tensor-core batch sits out (that
    # launch has no tiles) still match single analyzers fed the same frames, bit for bit.
    chans = [(640, 352, 8), (320, 180, 10), (200, 120, 10)]
    pattern = [(0, 1, 2), (0,), (1, 2), (), (2,), (0, 1, 2)]  # members taking part, per tick
    frames = [frames_list(SequenceSpec(w, h, len(pattern), 80 + i, bit_depth=bd, sigma=4.0, motion=2))
              for i, (w, h, bd) in enumerate(chans)]
    dev = [to_device(f) for f in frames]
    members = [vca.Analyzer(w, h, bd, 32, True, max_batch=2) for (w, h, bd) in chans]
    singles = [vca.Analyzer(w, h, bd, 32, True, max_batch=2) for (w, h, bd) in chans]
    try:
        with vca.Batch(members) as batch:
            assert batch.kernel == vca.VCA_KERNEL_TC
            for t, on in enumerate(pattern):
                refs = []
                for i, (y, u, v) in enumerate(dev):
                    if i in on:
                        refs.append((y[t], u[t], v[t]))
                        singles[i].push(y[t], u[t], v[t])
                    else:
                        refs.append(None)
                batch.tick(refs)
        for i, (m, a) in enumerate(zip(members, singles)):
            n = sum(i in on for on in pattern)
            assert [m.frame_features(k) for k in range(n)] == [a.frame_features(k) for k in range(n)], f"channel {i}"
    finally:
        for a in members + singles:
            a.close()


def test_ladder_size_batch_matches_single_analyzers(vca):
    # The batched tick at full size, in the launch configuration the ladder benchmark times: 24
    # channels from 640x360 to 3840x2160, half 10-bit (two tensor-core launches side by side, each
    # CTA on a run of 25-28 tiles).  Three ticks against single analyzers fed the same frames, bit
    # for bit; the 2160p 8-bit channel's first frame also against the oracle.
    from synth import ladder_specs

    specs = ladder_specs(4, n_frames=3)
    frames = [frames_list(sp, 0, 3) for sp in specs]
    dev = [to_device(f) for f in frames]
    members = [vca.Analyzer(sp.width, sp.height, sp.bit_depth, 32, True, max_batch=1) for sp in specs]
    singles = [vca.Analyzer(sp.width, sp.height, sp.bit_depth, 32, True, max_batch=1) for sp in specs]
    try:
        with vca.Batch(members) as batch:
            assert batch.kernel == vca.VCA_KERNEL_TC
            for t in range(3):
                batch.tick([(y[t], u[t], v[t]) for (y, u, v) in dev])
                for a, (y, u, v) in zip(singles, dev):
                    a.push(y[t], u[t], v[t])
        for i, (m, a) in enumerate(zip(members, singles)):
            assert [m.frame_features(t) for t in range(3)] == [a.frame_features(t) for t in range(3)], f"channel {i}"
        big = next(i for i, sp in enumerate(specs) if sp.width == 3840 and sp.bit_depth == 8)
        per, _ = oracle_sequence(frames[big][:1], oracle_config(members[big]))
        assert_features_close(members[big].frame_features(0), per[0], where="2160p 8-bit channel, frame 0")
    finally:
        for a in members + singles:
            a.close()


def test_batch_tail_over_several_passes_matches_single_analyzers(vca):
    # 24 channels at 1920x1080 with 16x16 blocks: 3,240 tiles on the device's CTAs, about 21 tiles
    # of 64 blocks per CTA, so each CTA's reduction tail takes its blocks in two passes of 1,024
    # and its run spans several members (some of whose blocks share a warp with the next
    # member's).  Half the channels 10-bit, one skips a tick; three ticks against single analyzers
    # fed the same frames, bit for bit, and one channel against the oracle.
    n = 24
    specs = [SequenceSpec(1920, 1080, 3, 900 + i, bit_depth=8 if i % 2 == 0 else 10, sigma=4.0, motion=3)
             for i in range(n)]
    frames = [frames_list(sp) for sp in specs]
    dev = [to_device(f) for f in frames]
    members = [vca.Analyzer(1920, 1080, sp.bit_depth, 16, True, max_batch=1) for sp in specs]
    singles = [vca.Analyzer(1920, 1080, sp.bit_depth, 16, True, max_batch=1) for sp in specs]
    fed = [[] for _ in range(n)]
    try:
        with vca.Batch(members) as batch:
            assert batch.kernel == vca.VCA_KERNEL_TC
            for t in range(3):
                refs = []
                for i, (y, u, v) in enumerate(dev):
                    if (t, i) == (1, 5):
                        refs.append(None)
                        continue
                    refs.append((y[t], u[t], v[t]))
                    singles[i].push(y[t], u[t], v[t])
                    fed[i].append(t)
                batch.tick(refs)
        for i, (m, a) in enumerate(zip(members, singles)):
            k = len(fed[i])
            assert [m.frame_features(j) for j in range(k)] == [a.frame_features(j) for j in range(k)], f"channel {i}"
        per, _ = oracle_sequence(frames[3][:3], oracle_config(members[3]))
        for t in range(3):
            assert_features_close(members[3].frame_features(t), per[t], where=f"channel 3 frame {t}")
    finally:
        for a in members + singles:
            a.close()
