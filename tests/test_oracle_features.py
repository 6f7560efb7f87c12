"""Pins of the oracle's block and frame features (Section 2: E_Y, h, L_Y, E_U, E_V, L_U, L_V).

Each test checks a closed form, an invariant or a special case that a plausible
mistake (dropped DC exclusion, wrong weight index, missing |.|, wrong normaliser,
wrong padding, wrong h pairing) would break.
"""

import math

import numpy as np
import pytest

from oracle import (Config, analyze_sequence, block_brightness, block_grid, block_texture_energy, chroma_shape,
                    downsample_plane,
                    energy_weights,
                    frame_block_values, frame_features, int_dct2, int_dct_matrix, plane_blocks,
                    sequence_features, transform_shifts)


def test_weights_closed_form():
    for N in (4, 8, 16, 32):
        w = energy_weights(N)
        assert w[N - 1, N - 1] == 1.0
        assert w[0, 0] == pytest.approx(math.exp(1 - 1 / N ** 4), rel=1e-15)
        np.testing.assert_array_equal(w, w.T)
        assert np.all(w >= 1.0) and np.all(w <= math.e)
    # N = 4, (u, v) = (1, 1): ((2*2/16)^2 - 1) = -0.9375 -> e^0.9375
    assert energy_weights(4)[1, 1] == pytest.approx(math.exp(0.9375), rel=1e-15)
    # N = 4, (u, v) = (3, 1): (4*2/16)^2 = 0.25 -> e^0.75
    assert energy_weights(4)[3, 1] == pytest.approx(math.exp(0.75), rel=1e-15)


@pytest.mark.parametrize("N", [4, 8, 16, 32])
@pytest.mark.parametrize("low_pass", [False, True])
def test_flat_block_has_zero_energy_and_closed_form_brightness(N, low_pass):
    for B in (8, 10, 12):
        for v in (0, 16, 200):
            Z = int_dct2(np.full((1, N, N), v), B, low_pass)
            assert block_texture_energy(Z, N)[0] == 0.0
            assert block_brightness(Z)[0] == math.sqrt(v * 2 ** (15 - B))


def test_energy_of_column_pattern_closed_form():
    # x[r][c] = f(c): only row u = 0 of Z survives, so H = sum_{v>=1} w(0,v) |Z[0][v]|.
    N, B = 32, 8
    M = int_dct_matrix(N)
    s1, s2 = transform_shifts(N, B)
    f = np.random.default_rng(3).integers(0, 256, size=N)
    x = np.tile(f, (N, 1))[None]
    Z = int_dct2(x, B)
    z0 = [(64 * N * ((int(np.dot(M[v], f)) + (1 << (s1 - 1))) >> s1) + (1 << (s2 - 1))) >> s2 for v in range(N)]
    assert any(z < 0 for z in z0)  # |.| matters
    expect = sum(math.exp(abs(((1 * (v + 1)) / N ** 2) ** 2 - 1)) * abs(z0[v]) for v in range(1, N))
    assert block_texture_energy(Z, N)[0] == pytest.approx(expect, rel=1e-13)
    # low-pass keeps v < N/2 only
    Zlp = int_dct2(x, B, low_pass=True)
    expect_lp = sum(math.exp(abs(((v + 1) / N ** 2) ** 2 - 1)) * abs(z0[v]) for v in range(1, N // 2))
    assert block_texture_energy(Zlp, N)[0] == pytest.approx(expect_lp, rel=1e-13)


def test_energy_is_weighted_l1_of_ac():
    N = 16
    Z = np.zeros((1, N, N), dtype=np.int64)
    Z[0, 0, 0] = 999          # DC: excluded
    Z[0, 2, 5] = -7
    Z[0, 15, 15] = 3
    w = energy_weights(N)
    assert block_texture_energy(Z, N)[0] == pytest.approx(7 * w[2, 5] + 3 * 1.0, rel=1e-15)


def test_plane_blocks_replicate_equals_edge_padding():
    rng = np.random.default_rng(0)
    plane = rng.integers(0, 256, size=(45, 70))
    n = 16
    nbx, nby = -(-70 // n), -(-45 // n)
    padded = np.pad(plane, ((0, nby * n - 45), (0, nbx * n - 70)), mode="edge")
    blocks = plane_blocks(plane, n, nbx, nby)
    for by in range(nby):
        for bx in range(nbx):
            np.testing.assert_array_equal(blocks[by * nbx + bx], padded[by * n:(by + 1) * n, bx * n:(bx + 1) * n])


def test_block_grid_modes():
    assert block_grid(Config(1920, 1080, block_size=32)) == (60, 34)
    assert block_grid(Config(1920, 1080, block_size=32, pad_mode="skip")) == (60, 33)
    assert block_grid(Config(3840, 2160, block_size=32)) == (120, 68)
    assert block_grid(Config(3840, 2160, block_size=16)) == (240, 135)
    assert block_grid(Config(640, 352, block_size=32)) == (20, 11)


def _planes(cfg, seed, flat=None):
    rng = np.random.default_rng(seed)
    y = rng.integers(16, 236, size=(cfg.height, cfg.width))
    ch, cw = (cfg.height + 1) // 2, (cfg.width + 1) // 2
    u = rng.integers(16, 241, size=(ch, cw))
    v = rng.integers(16, 241, size=(ch, cw))
    if flat is not None:
        y[:] = flat
        u[:] = flat
        v[:] = flat
    return y, u, v


def test_skip_mode_equals_cropped_frame():
    cfg = Config(100, 70, block_size=32, pad_mode="skip")
    y, u, v = _planes(cfg, 1)
    a = frame_block_values(y, u, v, cfg)
    crop = Config(96, 64, block_size=32)
    b = frame_block_values(y[:64, :96], u[:32, :48], v[:32, :48], crop)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def test_frame_normalisation_single_textured_block():
    # Flat frame except one luma block and one U block: E_Y = H/(C w^2), E_U = H_U/(C (w/2)^2).
    cfg = Config(128, 64, block_size=32)
    C = 4 * 2
    y = np.full((64, 128), 100)
    u = np.full((32, 64), 120)
    v = np.full((32, 64), 130)
    rng = np.random.default_rng(2)
    blk = rng.integers(16, 236, size=(32, 32))
    y[32:64, 64:96] = blk
    ublk = rng.integers(16, 241, size=(16, 16))
    u[0:16, 16:32] = ublk
    vals = frame_block_values(y, u, v, cfg)
    f = frame_features(vals, None, cfg)
    H = block_texture_energy(int_dct2(blk[None], 8), 32)[0]
    Hu = block_texture_energy(int_dct2(ublk[None], 8), 16)[0]
    assert f["E_Y"] == pytest.approx(H / (C * 32 * 32), rel=1e-14)
    assert f["E_U"] == pytest.approx(Hu / (C * 16 * 16), rel=1e-14)
    assert f["E_V"] == 0.0
    Ly_flat = math.sqrt(100 * 128)
    Ly_blk = block_brightness(int_dct2(blk[None], 8))[0]
    assert f["L_Y"] == pytest.approx((7 * Ly_flat + Ly_blk) / C, rel=1e-14)
    assert f["L_V"] == pytest.approx(math.sqrt(130 * 128), rel=1e-14)
    assert f["h"] == 0.0


def test_h_pairs_consecutive_frames():
    cfg = Config(96, 64, block_size=32)
    C = 3 * 2
    f0 = _planes(cfg, 10)
    f1 = tuple(p.copy() for p in f0)
    # identical frames -> h = 0 exactly
    seq = analyze_sequence([f0, f1, f1], cfg)
    assert seq[0]["h"] == 0.0 and seq[1]["h"] == 0.0 and seq[2]["h"] == 0.0
    # change one luma block: h = |dH| / (C w^2)
    f2 = tuple(p.copy() for p in f1)
    f2[0][0:32, 32:64] = np.random.default_rng(11).integers(16, 236, size=(32, 32))
    seq = analyze_sequence([f1, f2], cfg)
    H1 = block_texture_energy(int_dct2(f1[0][None, 0:32, 32:64], 8), 32)[0]
    H2 = block_texture_energy(int_dct2(f2[0][None, 0:32, 32:64], 8), 32)[0]
    assert seq[1]["h"] == pytest.approx(abs(H2 - H1) / (C * 32 * 32), rel=1e-13)
    # chroma changes do not move h
    f3 = tuple(p.copy() for p in f1)
    f3[1][:] = 50
    seq = analyze_sequence([f1, f3], cfg)
    assert seq[1]["h"] == 0.0


def test_sequence_means():
    cfg = Config(64, 64, block_size=32)
    frames = [_planes(cfg, s) for s in range(4)]
    per = analyze_sequence(frames, cfg)
    seqf = sequence_features(per)
    assert seqf["frames"] == 4
    assert seqf["E_Y"] == pytest.approx(sum(p["E_Y"] for p in per) / 4, rel=1e-15)
    assert seqf["h"] == pytest.approx(sum(p["h"] for p in per[1:]) / 3, rel=1e-15)
    assert sequence_features(per[:1])["h"] == 0.0


def test_low_pass_features_use_quarter_coefficients():
    cfg_full = Config(64, 64, block_size=32)
    cfg_lp = Config(64, 64, block_size=32, low_pass=True)
    y, u, v = _planes(cfg_full, 5)
    full = frame_block_values(y, u, v, cfg_full)
    lp = frame_block_values(y, u, v, cfg_lp)
    np.testing.assert_array_equal(full["L_Y"], lp["L_Y"])
    assert np.all(lp["H_Y"] < full["H_Y"])
    blocks = plane_blocks(y, 32, 2, 2)
    Z = int_dct2(blocks, 8)[:, :16, :16]
    np.testing.assert_allclose(lp["H_Y"], block_texture_energy(Z, 32), rtol=1e-15)


# ---------------------------------------------------------------------------
# Downsample reading of the low-pass option (Section 2 item 3: "spatially
# downsampled by a factor of two"): 2x2 rounded mean, then half-size blocks.
# ---------------------------------------------------------------------------

def test_downsample_rounding_by_hand():
    # (a + b + c + d + 2) >> 2: 11 -> 3, 2 -> 1 (a half rounds up), 1 -> 0, 1020 -> 255.
    assert downsample_plane(np.array([[1, 2], [3, 5]])).tolist() == [[3]]
    assert downsample_plane(np.array([[0, 0], [0, 2]])).tolist() == [[1]]
    assert downsample_plane(np.array([[0, 0], [0, 1]])).tolist() == [[0]]
    assert downsample_plane(np.full((2, 2), 255)).tolist() == [[255]]


def test_downsample_odd_sizes_repeat_the_edge():
    # 3 x 3 -> 2 x 2; the last row and column pair with themselves.
    p = np.array([[0, 4, 8], [4, 8, 12], [8, 12, 16]])
    assert downsample_plane(p).tolist() == [[4, 10], [10, 16]]


def test_downsample_inverts_pixel_doubling():
    rng = np.random.default_rng(7)
    base = rng.integers(0, 1024, size=(9, 13))
    doubled = np.repeat(np.repeat(base, 2, axis=0), 2, axis=1)
    assert np.array_equal(downsample_plane(doubled), base)


@pytest.mark.parametrize("bit_depth", [8, 10])
def test_downsample_reading_equals_half_size_analysis_of_the_base_frame(bit_depth):
    # A frame made by pixel doubling a base frame, analysed with the downsample reading and
    # w = 32, is the base frame analysed with w = 16 on the same block grid (both pinned paths).
    rng = np.random.default_rng(11 + bit_depth)
    hi = (1 << bit_depth) - 1
    W, H = 96, 80  # base 48 x 40: luma grid 3 x 3 with a partial row
    base = [(rng.integers(0, hi + 1, size=(H // 2, W // 2)), rng.integers(0, hi + 1, size=(H // 4, W // 4)),
             rng.integers(0, hi + 1, size=(H // 4, W // 4))) for _ in range(3)]
    up = [tuple(np.repeat(np.repeat(p, 2, axis=0), 2, axis=1) for p in f) for f in base]
    got = analyze_sequence(up, Config(W, H, bit_depth, 32, downsample=True))
    exp = analyze_sequence(base, Config(W // 2, H // 2, bit_depth, 16))
    assert got == exp


def test_downsample_reading_normalises_with_half_size_blocks():
    # One textured block: E_Y = H / (C (w/2)^2) with H of the 16 x 16 transform of the
    # downsampled block.
    W = H = 64
    y = np.full((H, W), 100)
    y[:32, :32] = np.tile(np.array([100, 100, 140, 140]), (32, 8))  # alternates column by column after halving
    u = np.full((H // 2, W // 2), 128)
    cfg = Config(W, H, 8, 32, downsample=True)
    f = analyze_sequence([(y, u, u)], cfg)[0]
    d = downsample_plane(y)
    Z = int_dct2(plane_blocks(d, 16, 2, 2), 8)
    Hb = block_texture_energy(Z, 16)
    assert Hb[0] > 0 and Hb[1:].tolist() == [0.0, 0.0, 0.0]
    assert f["E_Y"] == pytest.approx(Hb[0] / (4 * 16 * 16), rel=1e-15)
    assert f["E_U"] == 0.0


# ---------------------------------------------------------------------------
# Variants of the input: 4:4:4 chroma, 8 x 8 blocks (4 x 4 chroma), 12-bit samples
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bit_depth", [8, 12])
def test_444_chroma_runs_the_luma_path(bit_depth):
    # In 4:4:4 a chroma block is w x w like a luma block: equal planes give equal features.
    rng = np.random.default_rng(3 + bit_depth)
    W, H = 72, 40
    frames = [tuple([rng.integers(0, 1 << bit_depth, size=(H, W))] * 3) for _ in range(2)]
    per = analyze_sequence(frames, Config(W, H, bit_depth, 16, chroma_format="444"))
    for f in per:
        assert f["E_U"] == f["E_Y"] and f["E_V"] == f["E_Y"]
        assert f["L_U"] == f["L_Y"] and f["L_V"] == f["L_Y"]
    assert chroma_shape(Config(W, H, chroma_format="444")) == (H, W)
    assert chroma_shape(Config(W + 2, H + 2)) == (H // 2 + 1, W // 2 + 1)


@pytest.mark.parametrize("bit_depth", [8, 10, 12])
def test_block_8_flat_frame_closed_forms(bit_depth):
    # 8 x 8 luma and 4 x 4 chroma blocks on a 3 x 2 grid with partial blocks: flat planes give
    # E = 0 and L = sqrt(v 2^(15 - B)) for both block sizes.
    W, H = 20, 12
    v, c = 37, 150
    y = np.full((H, W), v)
    u = np.full((H // 2, W // 2), c)
    f = analyze_sequence([(y, u, u)], Config(W, H, bit_depth, 8))[0]
    assert block_grid(Config(W, H, bit_depth, 8)) == (3, 2)
    assert f["E_Y"] == 0.0 and f["E_U"] == 0.0 and f["E_V"] == 0.0
    assert f["L_Y"] == pytest.approx(math.sqrt(v * 2 ** (15 - bit_depth)), rel=1e-15)  # mean of 6 equal values
    assert f["L_U"] == pytest.approx(math.sqrt(c * 2 ** (15 - bit_depth)), rel=1e-15)
