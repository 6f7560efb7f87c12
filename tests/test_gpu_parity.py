"""GPU parity of the analyzer's CUDA path against the CPU oracle, through the C ABI.

Coefficients are compared bit-exactly (debug dump of the same kernel), per-block H/L and
per-frame features within the tolerances derived in vca_testutil.  Inputs are the seeded
synthetic workloads: the tiny 640x352 sequence, ragged small frames that leave partial
blocks on both edges, 1080p low-pass with its partial bottom block row, and sampled frames
of 2160p in the benchmark's launch configuration.
"""

import numpy as np
import pytest

from synth import SequenceSpec, frames_list, hd_spec, tiny_spec, uhd_spec
from vca_testutil import (BLOCK_H_RTOL, BLOCK_L_RTOL, assert_block_values_close, assert_features_close,
                          frame_block_values, oracle_coefficients, oracle_config, oracle_sequence, to_device,
                          to_host_pinned)

pytestmark = pytest.mark.gpu

KERNELS = {"plain": 1, "tc": 2}


@pytest.fixture(scope="session")
def vca():
    import torch

    from paper_2304_12384_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2304_12384_gb300 import vca as v
    return v


def open_analyzer(vca, kernel, **kw):
    try:
        return vca.Analyzer(kernel=KERNELS[kernel], **kw)
    except vca.VcaError as e:
        if e.status == vca.VCA_E_UNSUPPORTED and kernel == "tc":
            pytest.skip("the tensor-core kernel does not cover this configuration")
        raise


def run_and_compare(vca, kernel, frames, *, width, height, bit_depth=8, block_size=32, low_pass=False, pad_mode=0,
                    batch=None, dump_frames=(0,), block_frames=None, chroma_format=0, matrices=None):
    import torch

    an = open_analyzer(vca, kernel, width=width, height=height, bit_depth=bit_depth, block_size=block_size,
                       low_pass=low_pass, pad_mode=pad_mode, max_batch=max(len(frames), 1),
                       chroma_format=chroma_format)
    try:
        for n, m in (matrices or {}).items():
            an.set_dct_matrix(n, m)
        y, u, v = to_device(frames)
        assert an.kernel == KERNELS[kernel]
        an.push(y, u, v)
        cfg = oracle_config(an)
        per, seqf = oracle_sequence(frames, cfg)
        for t, exp in enumerate(per):
            assert_features_close(an.frame_features(t), exp, where=f"frame {t}")
        assert_features_close(an.sequence_features(), seqf, where="sequence")
        for t in (block_frames if block_frames is not None else range(len(frames))):
            assert_block_values_close(an.block_values(t), frame_block_values(*frames[t], cfg), where=f"frame {t}")
        for t in dump_frames:
            z = an.dump_coefficients(y[t], u[t], v[t])
            exp = oracle_coefficients(frames[t], cfg)
            for p in ("Y", "U", "V"):
                got = z[p].cpu().numpy().astype(np.int64)
                assert got.shape == exp[p].shape
                mism = np.argwhere(got != exp[p])
                assert mism.size == 0, f"{p} coefficients differ at {mism[:5].tolist()} (frame {t})"
        torch.cuda.synchronize()
        return an
    finally:
        an.close()


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_tiny_sequence(vca, kernel):
    frames = frames_list(tiny_spec(1))
    run_and_compare(vca, kernel, frames, width=640, height=352, dump_frames=(0, 8, 15))


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("block_size", [32, 16])
@pytest.mark.parametrize("low_pass", [False, True])
@pytest.mark.parametrize("bit_depth", [8, 10])
@pytest.mark.parametrize("pad_mode", [0, 1])
def test_ragged_frames(vca, kernel, block_size, low_pass, bit_depth, pad_mode):
    # 200 x 120 leaves partial blocks at the right and bottom edges of every plane.
    spec = SequenceSpec(200, 120, 3, seed=11 + block_size + bit_depth, bit_depth=bit_depth, sigma=6.0,
                        periods=(2.0, 16.0))
    frames = frames_list(spec)
    run_and_compare(vca, kernel, frames, width=200, height=120, bit_depth=bit_depth, block_size=block_size,
                    low_pass=low_pass, pad_mode=pad_mode, dump_frames=(0, 2))


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_hd_low_pass_around_scene_cut(vca, kernel):
    frames = frames_list(hd_spec(2), 38, 43)  # a scene cut at frame 40
    run_and_compare(vca, kernel, frames, width=1920, height=1080, low_pass=True, dump_frames=(0, 2),
                    block_frames=(0, 2, 4))


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("block_size,low_pass", [(32, True), (32, False), (16, True), (16, False)])
def test_uhd_sampled(vca, kernel, block_size, low_pass):
    # 2160p in the benchmark's launch configuration (one push of several frames); the oracle
    # checks every frame's features, and block values / coefficients on sampled frames.
    frames = frames_list(uhd_spec(3), 0, 4)
    run_and_compare(vca, kernel, frames, width=3840, height=2160, block_size=block_size, low_pass=low_pass,
                    dump_frames=(3,), block_frames=(0, 3))


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("block_size", [32, 16])
@pytest.mark.parametrize("bit_depth", [8, 10])
def test_extreme_blocks_are_exact(vca, kernel, block_size, bit_depth):
    # All-max, all-zero, checkerboards and sign-matched stripes: the largest intermediates of
    # both transform stages.
    W, H = 256, 128
    mx = (1 << bit_depth) - 1
    dt = np.uint16 if bit_depth > 8 else np.uint8
    yy, xx = np.indices((H, W))
    pats = [np.full((H, W), mx), np.zeros((H, W)), ((yy + xx) % 2) * mx, (xx % 2) * mx, (yy % 2) * mx,
            ((xx // 4) % 2) * mx, ((yy // 8) % 2) * mx, (((xx % 32) < 16) ^ ((yy % 32) < 16)) * mx]
    frames = []
    for i, p in enumerate(pats):
        cy, cx = np.indices((H // 2, W // 2))
        q = pats[(i + 3) % len(pats)]
        frames.append((p.astype(dt), q[:H // 2, :W // 2].astype(dt), (mx - q[:H // 2, :W // 2]).astype(dt)))
    for lp in (False, True):
        run_and_compare(vca, kernel, frames, width=W, height=H, bit_depth=bit_depth, block_size=block_size,
                        low_pass=lp, dump_frames=range(len(frames)))


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_frame_by_frame_equals_batch_and_is_deterministic(vca, kernel):
    import torch

    frames = frames_list(tiny_spec(5))[:10]
    y, u, v = to_device(frames)
    a = open_analyzer(vca, kernel, width=640, height=352, max_batch=10)
    b = open_analyzer(vca, kernel, width=640, height=352, max_batch=10)
    c = open_analyzer(vca, kernel, width=640, height=352, max_batch=10)
    try:
        a.push(y, u, v)
        for t in range(10):
            b.push(y[t], u[t], v[t])
        c.push(y[:3], u[:3], v[:3])
        c.push(y[3:], u[3:], v[3:])
        torch.cuda.synchronize()
        for t in range(10):
            fa, fb, fc = a.frame_features(t), b.frame_features(t), c.frame_features(t)
            assert fa == fb == fc, t
    finally:
        a.close()
        b.close()
        c.close()


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("size", [(640, 352), (200, 120)])  # rows and frames back to back; padded rows
def test_host_frames_equal_device_frames(vca, kernel, size):
    W, H = size
    frames = frames_list(tiny_spec(6))[:6] if size == (640, 352) else frames_list(SequenceSpec(W, H, 6, 61))
    y, u, v = to_device(frames)
    hy, hu, hv = to_host_pinned(frames)
    assert (hy.stride(-2) == W) == (size == (640, 352))
    a = open_analyzer(vca, kernel, width=W, height=H, max_batch=6)
    b = open_analyzer(vca, kernel, width=W, height=H, max_batch=6)
    try:
        a.push(y, u, v)
        b.push(hy, hu, hv)
        for t in range(6):
            assert a.frame_features(t) == b.frame_features(t)
        # pageable (non-pinned) host memory and a single-frame push
        b.push(hy[0].clone(), hu[0].clone(), hv[0].clone())
        assert b.frame_features(6)["h"] > 0
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_large_host_pushes_equal_device_pushes(vca, kernel):
    # 40 dense host frames (one copy per plane), then pushes of 6 and 37 frames on the same
    # staging buffer.
    frames = frames_list(SequenceSpec(640, 352, 40, 62, sigma=5.0, cuts=(17,), motion=3))
    y, u, v = to_device(frames)
    hy, hu, hv = to_host_pinned(frames)
    a = open_analyzer(vca, kernel, width=640, height=352, max_batch=40)
    b = open_analyzer(vca, kernel, width=640, height=352, max_batch=40)
    try:
        for sl in (slice(0, 40), slice(0, 6), slice(3, 40)):
            a.push(y[sl], u[sl], v[sl])
            b.push(hy[sl], hu[sl], hv[sl])
        n = 40 + 6 + 37
        assert [a.frame_features(t) for t in range(n)] == [b.frame_features(t) for t in range(n)]
        cfg = oracle_config(a)
        per, _ = oracle_sequence(frames, cfg)
        for t in (0, 16, 17, 39):
            assert_features_close(b.frame_features(t), per[t], where=f"frame {t}")
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_state_export_import_resumes_h(vca, kernel):
    frames = frames_list(tiny_spec(7))[:8]
    y, u, v = to_device(frames)
    a = open_analyzer(vca, kernel, width=640, height=352, max_batch=8)
    b = open_analyzer(vca, kernel, width=640, height=352, max_batch=8)
    c = open_analyzer(vca, kernel, width=640, height=352, max_batch=8)
    try:
        a.push(y, u, v)
        b.push(y[:4], u[:4], v[:4])
        state = b.export_state()
        c.import_state(state)
        c.push(y[4:], u[4:], v[4:])
        for t in range(4, 8):
            assert c.frame_features(t) == a.frame_features(t)
        assert c.sequence_features() == a.sequence_features()
        with pytest.raises(vca.VcaError):
            c.frame_features(3)
    finally:
        a.close()
        b.close()
        c.close()


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_argument_errors_on_device(vca, kernel):
    import torch

    an = open_analyzer(vca, kernel, width=640, height=352, max_batch=2)
    try:
        frames = frames_list(tiny_spec(8))[:3]
        y, u, v = to_device(frames)
        with pytest.raises(vca.VcaError) as e:
            an.push(y, u, v)  # 3 frames > max_batch
        assert e.value.status == vca.VCA_E_ARG
        raw = torch.zeros(640 * 352 + 64, dtype=torch.uint8, device="cuda")
        with pytest.raises(vca.VcaError) as e:
            vca.vca_push_frame(an.handle, raw.data_ptr() + 1, u.data_ptr(), v.data_ptr(), 640, 320, 1)
        assert e.value.status == vca.VCA_E_ARG
        with pytest.raises(vca.VcaError) as e:
            vca.vca_push_frame(an.handle, raw.data_ptr(), u.data_ptr(), v.data_ptr(), 600, 320, 1)
        assert e.value.status == vca.VCA_E_ARG
        with pytest.raises(vca.VcaError) as e:
            an.frame_features(0)  # nothing pushed
        assert e.value.status == vca.VCA_E_ARG
        an.push(y[:1], u[:1], v[:1])
        f = vca.VcaFrameFeatures()
        st = vca.lib().vca_read_frame_features(an.handle, 0, 0, vca.ctypes.byref(f))
        assert st in (vca.VCA_OK, vca.VCA_E_AGAIN)
        assert an.frame_features(0)["h"] == 0.0
    finally:
        an.close()


# Downsample reading of the low-pass option: halved planes (rounded 2x2 mean, odd edges
# repeated) analysed with 16 x 16 / 8 x 8 blocks on the 32-block grid.
@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("bit_depth", [8, 10])
@pytest.mark.parametrize("size", [(640, 352), (200, 120), (202, 118)])
def test_downsample_reading(vca, kernel, bit_depth, size):
    w, h = size
    frames = frames_list(SequenceSpec(w, h, 5, 41, bit_depth=bit_depth, sigma=4.0, cuts=(3,)))
    run_and_compare(vca, kernel, frames, width=w, height=h, bit_depth=bit_depth, low_pass="downsample",
                    dump_frames=(0, 3))


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_downsample_reading_hd(vca, kernel):
    frames = frames_list(hd_spec(2, 3))
    run_and_compare(vca, kernel, frames, width=1920, height=1080, low_pass="downsample", dump_frames=(2,),
                    block_frames=(0,))


def test_downsample_reading_rules(vca):
    # The halved planes take 16 x 16 / 8 x 8 blocks, which the tensor-core form covers at 8 and 10 bits.
    an = vca.Analyzer(640, 352, 8, 32, "downsample")
    assert an.kernel == vca.VCA_KERNEL_TC
    an.close()
    an = vca.Analyzer(640, 352, 12, 32, "downsample")
    assert an.kernel == vca.VCA_KERNEL_PLAIN
    an.close()
    with pytest.raises(vca.VcaError) as ei:
        vca.Analyzer(640, 352, 8, 16, "downsample")
    assert ei.value.status == vca.VCA_E_UNSUPPORTED


# Input variants: 8 x 8 blocks (4 x 4 chroma), 12-bit samples, 4:4:4 chroma (CUDA-core form).
@pytest.mark.parametrize("bit_depth", [8, 10, 12])
@pytest.mark.parametrize("low_pass", [False, True])
def test_block_8(vca, bit_depth, low_pass):
    frames = frames_list(SequenceSpec(200, 120, 4, 51, bit_depth=bit_depth, sigma=4.0, cuts=(2,)))
    run_and_compare(vca, "plain", frames, width=200, height=120, bit_depth=bit_depth, block_size=8,
                    low_pass=low_pass, dump_frames=(0, 2))


@pytest.mark.parametrize("block_size", [32, 16])
@pytest.mark.parametrize("low_pass", [False, True])
def test_12_bit(vca, block_size, low_pass):
    frames = frames_list(SequenceSpec(640, 352, 4, 52, bit_depth=12, sigma=4.0, cuts=(2,)))
    run_and_compare(vca, "plain", frames, width=640, height=352, bit_depth=12, block_size=block_size,
                    low_pass=low_pass, dump_frames=(1,))


CASES_444 = [("plain", bs, bd) for bs in (32, 16, 8) for bd in (8, 10, 12)] + \
            [("tc", bs, bd) for bs in (32, 16) for bd in (8, 10)]  # what the tensor-core form covers


@pytest.mark.parametrize("kernel,block_size,bit_depth", CASES_444)
def test_chroma_444(vca, kernel, block_size, bit_depth):
    # 4:4:4: full-size chroma planes with w x w blocks; the tensor-core form runs each plane of a tile
    # through its luma roles (8 and 10 bits, w 32 and 16).
    frames = frames_list(SequenceSpec(200, 120, 4, 53, bit_depth=bit_depth, sigma=4.0, cuts=(2,), chroma_format="444"))
    for low_pass in (False, True):
        run_and_compare(vca, kernel, frames, width=200, height=120, bit_depth=bit_depth, block_size=block_size,
                        low_pass=low_pass, dump_frames=(0, 3), chroma_format=1)


@pytest.mark.parametrize("kernel", list(KERNELS))
def test_chroma_444_hd_sampled(vca, kernel):
    frames = frames_list(SequenceSpec(1920, 1080, 3, 58, bit_depth=8, sigma=4.0, chroma_format="444"))
    run_and_compare(vca, kernel, frames, width=1920, height=1080, block_size=32, low_pass=True, dump_frames=(2,),
                    block_frames=(0, 2), chroma_format=1)


@pytest.mark.parametrize("block_size", [32, 16, 8])
@pytest.mark.parametrize("bit_depth", [8, 10, 12])
def test_chroma_422(vca, block_size, bit_depth):
    # 4:2:2: half-width, full-height chroma planes and chroma blocks of w rows by w/2 columns; 200 x 120
    # leaves partial blocks at the right and bottom edges of every plane, and the chroma planes'
    # 100-sample rows leave a ragged last block column at every block size.
    frames = frames_list(SequenceSpec(200, 120, 4, 54 + bit_depth, bit_depth=bit_depth, sigma=5.0, cuts=(2,),
                                      chroma_format="422", periods=(2.0, 24.0)))
    for low_pass in (False, True):
        run_and_compare(vca, "plain", frames, width=200, height=120, bit_depth=bit_depth, block_size=block_size,
                        low_pass=low_pass, dump_frames=(0, 3), chroma_format=vca.VCA_CHROMA_422)


@pytest.mark.parametrize("pad_mode", [0, 1])
def test_chroma_422_hd_sampled(vca, pad_mode):
    # 1080p 10-bit 4:2:2 (1080 = 33 * 32 + 24: a ragged block row) in one push of several frames.
    frames = frames_list(SequenceSpec(1920, 1080, 3, 57, bit_depth=10, sigma=4.0, chroma_format="422"))
    run_and_compare(vca, "plain", frames, width=1920, height=1080, bit_depth=10, block_size=32, pad_mode=pad_mode,
                    dump_frames=(2,), block_frames=(0, 2), chroma_format=vca.VCA_CHROMA_422)


def test_variant_rules(vca):
    # The tensor-core form covers 8- and 10-bit 4:2:0 and 4:4:4 with 32 x 32 or 16 x 16 blocks; the
    # others run on CUDA cores.
    for kw in ({"bit_depth": 12}, {"block_size": 8}, {"chroma_format": 2}):
        args = dict(width=640, height=352, bit_depth=8, block_size=32)
        args.update(kw)
        an = vca.Analyzer(**args)
        assert an.kernel == vca.VCA_KERNEL_PLAIN
        an.close()
    for kw in ({"chroma_format": 1}, {"chroma_format": 1, "block_size": 16, "bit_depth": 10}):
        args = dict(width=640, height=352, bit_depth=8, block_size=32)
        args.update(kw)
        an = vca.Analyzer(**args)
        assert an.kernel == vca.VCA_KERNEL_TC
        an.close()
    with pytest.raises(vca.VcaError) as ei:
        vca.Analyzer(640, 352, 8, 32, chroma_format=vca.VCA_CHROMA_422, kernel=vca.VCA_KERNEL_TC)
    assert ei.value.status == vca.VCA_E_UNSUPPORTED
    with pytest.raises(vca.VcaError) as ei:
        vca.Analyzer(640, 352, 8, 32, chroma_format=vca.VCA_CHROMA_422, low_pass=2)
    assert ei.value.status == vca.VCA_E_UNSUPPORTED
    with pytest.raises(vca.VcaError) as ei:
        vca.Analyzer(640, 352, 8, 32, chroma_format=3)
    assert ei.value.status == vca.VCA_E_ARG


# ---- drop-in DCT matrices (an encoder's own integer table in place of the round-cosine one) ----

def _drop_in_matrices():
    from vca_testutil import structured_dct_matrix
    return {32: structured_dct_matrix(32, (((32, 0, 0), -1), ((32, 7, 9), 2), ((16, 3, 4), 1), ((8, 1, 0), -1))),
            16: structured_dct_matrix(16, (((16, 0, 0), -1), ((16, 5, 3), 1), ((8, 2, 1), -2), ((4, 0, 1), 1)))}


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("low_pass", [True, False])
@pytest.mark.parametrize("bit_depth", [8, 10])
def test_drop_in_matrix(vca, kernel, low_pass, bit_depth):
    mats = _drop_in_matrices()
    for n, m in mats.items():
        assert vca.vca_check_dct_matrix(n, bit_depth, m) == 0
    frames = frames_list(SequenceSpec(200, 120, 4, 51, bit_depth=bit_depth, sigma=6.0, cuts=(2,)))
    run_and_compare(vca, kernel, frames, width=200, height=120, bit_depth=bit_depth, low_pass=low_pass,
                    dump_frames=(0, 3), matrices=mats)


def test_drop_in_matrix_rules(vca):
    import numpy as np

    mats = _drop_in_matrices()
    frames = to_device(frames_list(SequenceSpec(200, 120, 2, 52)))
    an = vca.Analyzer(200, 120, 8, 32, True, max_batch=2)
    try:
        with pytest.raises(vca.VcaError) as ei:  # not a transform size of this analyzer
            an.set_dct_matrix(8, np.full((8, 8), 64))
        assert ei.value.status == vca.VCA_E_ARG
        bad = mats[32].copy()
        bad[5, 0] += 1
        with pytest.raises(vca.VcaError) as ei:
            an.set_dct_matrix(32, bad)
        assert ei.value.status == vca.VCA_E_ARG and "symmetry" in str(ei.value)
        an.set_dct_matrix(32, mats[32])
        y, u, v = frames
        an.push(y[0:1], u[0:1], v[0:1])
        with pytest.raises(vca.VcaError) as ei:  # after the first push
            an.set_dct_matrix(16, mats[16])
        assert ei.value.status == vca.VCA_E_STATE
    finally:
        an.close()


# ---- per-feature error of the tensor-core path against the FP64 oracle ----

def _feature_error_table(vca, frames, width, height, bit_depth):
    """Max relative error per feature over the frames (h also relative to max(h, E_Y))."""
    from vca_testutil import FEATURES

    an = open_analyzer(vca, "tc", width=width, height=height, bit_depth=bit_depth, block_size=32, low_pass=True,
                       max_batch=len(frames))
    try:
        an.push(*to_device(frames))
        per, _ = oracle_sequence(frames, oracle_config(an))
        err = {k: 0.0 for k in FEATURES}
        err["h_vs_max(h,E_Y)"] = 0.0
        for t, exp in enumerate(per):
            got = an.frame_features(t)
            for k in FEATURES:
                if exp[k] != 0.0:
                    err[k] = max(err[k], abs(got[k] - exp[k]) / abs(exp[k]))
                else:
                    assert got[k] == 0.0, (t, k, got[k])
            err["h_vs_max(h,E_Y)"] = max(err["h_vs_max(h,E_Y)"],
                                         abs(got["h"] - exp["h"]) / max(abs(exp["h"]), abs(exp["E_Y"])))
        return err
    finally:
        an.close()


@pytest.mark.parametrize("case", ["2160p_8bit", "ladder_1080p_10bit"])
def test_feature_error_statement(vca, case):
    # The error of every feature against the FP64 oracle, measured and printed (pytest -s shows the
    # table), and bounded: E and L within 1e-6 relative; h within 1e-6 relative to max(h, E_Y) (h is a
    # sum of differences of FP32 block energies and cancels), and here also within 1e-5 of itself.
    if case == "2160p_8bit":
        frames = frames_list(uhd_spec(3), 0, 4)
        err = _feature_error_table(vca, frames, 3840, 2160, 8)
    else:
        from synth import ladder_specs
        spec = [s for s in ladder_specs(4, n_frames=6) if s.width == 1920 and s.bit_depth == 10][0]
        frames = frames_list(spec)
        err = _feature_error_table(vca, frames, 1920, 1080, 10)
    print(f"\nmax relative error per feature ({case}): " + ", ".join(f"{k} {v:.2e}" for k, v in err.items()))
    for k in ("E_Y", "L_Y", "E_U", "E_V", "L_U", "L_V"):
        assert err[k] <= 1e-6, (k, err[k])
    assert err["h_vs_max(h,E_Y)"] <= 1e-6
    assert err["h"] <= 1e-5


# ---- the largest frame vca_open accepts ----

@pytest.mark.parametrize("kernel,block_size,low_pass", [("tc", 32, True), ("tc", 16, False), ("plain", 32, True)])
def test_maximum_frame_size_sampled(vca, kernel, block_size, low_pass):
    # 16384 x 16384 8-bit 4:2:0, the largest frame vca_open accepts: 262,144 blocks of 32 x 32 per
    # plane (1,048,576 of 16 x 16) and 16,384 tiles of 128 x 128, the widest indices of every kernel.
    # Uniform noise drives the coefficients over their full range.  Block values are compared with
    # the oracle on sampled blocks (the four corners, the edges, random interior ones), cut by hand
    # from the planes; the frame features with exact sums of the kernel's own block values divided by
    # the oracle's norms (the reduction sums exactly and rounds once).
    import math

    from oracle import block_brightness, block_texture_energy, int_dct2

    W = H = 16384
    rng = np.random.default_rng(16384 + block_size)
    y = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    u = rng.integers(0, 256, size=(H // 2, W // 2), dtype=np.uint8)
    v = rng.integers(0, 256, size=(H // 2, W // 2), dtype=np.uint8)
    an = open_analyzer(vca, kernel, width=W, height=H, bit_depth=8, block_size=block_size, low_pass=low_pass,
                       max_batch=1)
    try:
        dy, du, dv = to_device([(y, u, v)])
        an.push(dy, du, dv)
        f = an.frame_features(0)
        bv = an.block_values(0)
    finally:
        an.close()
    w, nc = block_size, block_size // 2
    nbx = nby = W // w
    C = nbx * nby
    assert bv["H_Y"].shape == (C,)
    last = nbx - 1
    picks = {0, last, last * nbx, C - 1, nbx // 2, (nby // 2) * nbx + last}
    picks |= set(int(k) for k in rng.integers(0, C, size=40))
    ks = np.array(sorted(picks))
    bx, by = ks % nbx, ks // nbx
    for name, plane, n in (("Y", y, w), ("U", u, nc), ("V", v, nc)):
        blocks = np.stack([plane[j * n:(j + 1) * n, i * n:(i + 1) * n] for i, j in zip(bx, by)]).astype(np.int64)
        Z = int_dct2(blocks, 8, low_pass)
        eH, eL = block_texture_energy(Z, n), block_brightness(Z)
        gH, gL = bv["H_" + name][ks].astype(np.float64), bv["L_" + name][ks].astype(np.float64)
        bad = np.nonzero(np.abs(gH - eH) > BLOCK_H_RTOL * np.abs(eH))[0]
        assert bad.size == 0, f"H_{name} off at blocks {ks[bad[:5]]}: {gH[bad[:5]]} vs {eH[bad[:5]]}"
        bad = np.nonzero(np.abs(gL - eL) > BLOCK_L_RTOL * np.abs(eL))[0]
        assert bad.size == 0, f"L_{name} off at blocks {ks[bad[:5]]}: {gL[bad[:5]]} vs {eL[bad[:5]]}"
    exact = {k: math.fsum(bv[k].astype(np.float64)) for k in bv}
    assert f["E_Y"] == exact["H_Y"] / (C * w * w) and f["L_Y"] == exact["L_Y"] / C
    assert f["E_U"] == exact["H_U"] / (C * nc * nc) and f["E_V"] == exact["H_V"] / (C * nc * nc)
    assert f["L_U"] == exact["L_U"] / C and f["L_V"] == exact["L_V"] / C
    assert f["h"] == 0.0
