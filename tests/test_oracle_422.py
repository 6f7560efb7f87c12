"""Pins of the oracle's 4:2:2 chroma reading: rectangular blocks of Nv = w rows by Nh = w/2
columns (Section 2's transform applied to the co-located chroma area of a w x w luma block).

The rectangular transform runs rows first with the Nh-point matrix and the row shift of Nh, then
columns with the Nv-point matrix and the column shift of Nv.  These tests fix it against closed
forms (flat, row-only and column-only blocks, computed here one dimension at a time), the square
case, scipy's orthonormal DCT-II, and frames whose features follow by hand.
"""

import math

import numpy as np
import pytest
import scipy.fft

from oracle import (Config, analyze_sequence, block_texture_energy_rect, chroma_shape, energy_weights,
                    energy_weights_rect, frame_block_values, int_dct2, int_dct2_rect, int_dct2_rect_stages,
                    int_dct_matrix)
from synth import SequenceSpec, frames_list

SHAPES = [(8, 4), (16, 8), (32, 16), (4, 8), (16, 32)]


@pytest.mark.parametrize("N", [4, 8, 16, 32])
def test_square_case_is_the_square_transform(N):
    x = np.random.default_rng(N).integers(0, 1024, size=(12, N, N))
    for B in (8, 10):
        xb = x >> (10 - B)
        np.testing.assert_array_equal(int_dct2_rect(xb, B), int_dct2(xb, B))
        np.testing.assert_array_equal(int_dct2_rect(xb, B, True), int_dct2(xb, B, True))


@pytest.mark.parametrize("Nv,Nh", SHAPES)
@pytest.mark.parametrize("B", [8, 10, 12])
def test_flat_rect_block_closed_form(Nv, Nh, B):
    # The row sums of the matrices are 64 N for k = 0 and 0 otherwise, so both stages carry the DC
    # exactly: T[r][0] = Z[0][0] = v 2^(15-B), everything else 0.
    for v in (0, 1, 93, (1 << B) - 1):
        T, Z = int_dct2_rect_stages(np.full((Nv, Nh), v), B)
        assert T.shape == (Nv, Nh) and Z.shape == (Nv, Nh)
        assert np.all(T[:, 0] == v << (15 - B)) and np.all(T[:, 1:] == 0)
        assert Z[0, 0] == v << (15 - B)
        Z[0, 0] = 0
        assert np.all(Z == 0)


@pytest.mark.parametrize("Nv,Nh", SHAPES)
def test_row_only_and_column_only_patterns(Nv, Nh):
    # One dimension at a time with scalar arithmetic: a pattern that varies only along the columns
    # (x[r][c] = f(c)) runs the Nh-point row transform with shift log2 Nh + B - 9 and keeps u = 0;
    # one that varies only down the rows (x[r][c] = g(r)) runs the Nv-point column transform with
    # shift log2 Nv + 6 on T[r][0] = g(r) 2^(15-B) and keeps v = 0.
    B = 10
    rng = np.random.default_rng(Nv * 100 + Nh)
    Mh, Mv = int_dct_matrix(Nh), int_dct_matrix(Nv)
    s1 = int(math.log2(Nh)) + B - 9
    s2 = int(math.log2(Nv)) + 6
    f = rng.integers(0, 1 << B, size=Nh)
    Z = int_dct2_rect(np.tile(f, (Nv, 1)), B)
    t = [(sum(int(Mh[k][c]) * int(f[c]) for c in range(Nh)) + (1 << (s1 - 1))) >> s1 for k in range(Nh)]
    assert Z[0].tolist() == [(64 * Nv * tk + (1 << (s2 - 1))) >> s2 for tk in t]
    assert np.all(Z[1:] == 0)
    g = rng.integers(0, 1 << B, size=Nv)
    Z = int_dct2_rect(np.tile(g[:, None], (1, Nh)), B)
    T0 = [int(gr) << (15 - B) for gr in g]
    assert Z[:, 0].tolist() == [(sum(int(Mv[u][r]) * T0[r] for r in range(Nv)) + (1 << (s2 - 1))) >> s2
                                for u in range(Nv)]
    assert np.all(Z[:, 1:] == 0)


@pytest.mark.parametrize("Nv,Nh", SHAPES)
@pytest.mark.parametrize("B", [8, 10, 12])
def test_rect_transform_tracks_real_dct(Nv, Nh, B):
    # Each stage scales the orthonormal DCT by 64 sqrt(N) / 2^shift: together 2^(15-B) / sqrt(Nv Nh).
    scale = 2.0 ** (15 - B) / math.sqrt(Nv * Nh)
    x = np.random.default_rng(Nv + Nh + B).integers(0, 1 << B, size=(50, Nv, Nh))
    Z = int_dct2_rect(x, B).astype(np.float64)
    X = scipy.fft.dctn(x.astype(np.float64), type=2, norm="ortho", axes=(1, 2)) * scale
    err = np.abs(Z - X)
    assert np.sqrt(np.mean(err ** 2)) < 0.006 * np.sqrt(np.mean(X ** 2))
    assert err.max() < 0.005 * np.abs(X).max()


@pytest.mark.parametrize("Nv,Nh", SHAPES)
def test_rect_low_pass_is_top_left_quarter(Nv, Nh):
    x = np.random.default_rng(Nv * 7 + Nh).integers(0, 4096, size=(20, Nv, Nh))
    lp = int_dct2_rect(x, 12, low_pass=True)
    assert lp.shape == (20, Nv // 2, Nh // 2)
    np.testing.assert_array_equal(lp, int_dct2_rect(x, 12)[:, : Nv // 2, : Nh // 2])


def test_rect_intermediate_and_output_fit_int16():
    # 12-bit extremes through the largest 4:2:2 block (32 x 16): T and Z stay 16-bit signed.
    Nv, Nh, B = 32, 16, 12
    mx = (1 << B) - 1
    idx = np.indices((Nv, Nh))
    blocks = [np.full((Nv, Nh), mx), (idx.sum(0) % 2) * mx, (idx[1] % 2) * mx, (idx[0] % 2) * mx]
    Mh, Mv = int_dct_matrix(Nh), int_dct_matrix(Nv)
    for k in range(Nh):
        blocks.append(np.tile((Mh[k] > 0) * mx, (Nv, 1)))
    for u in range(Nv):
        blocks.append(np.tile((Mv[u] > 0)[:, None] * mx, (1, Nh)))
    T, Z = int_dct2_rect_stages(np.stack(blocks), B)
    assert T.max() <= 32767 and T.min() >= -32768
    assert Z.max() <= 32767 and Z.min() >= -32768


def test_rect_weights_closed_form():
    for Nv, Nh in SHAPES:
        w = energy_weights_rect(Nv, Nh)
        assert w.shape == (Nv, Nh)
        assert w[Nv - 1, Nh - 1] == 1.0
        assert w[0, 0] == pytest.approx(math.exp(1 - 1 / (Nv * Nh) ** 2), rel=1e-15)
        np.testing.assert_array_equal(w, energy_weights_rect(Nh, Nv).T)
    for N in (4, 8, 32):
        np.testing.assert_array_equal(energy_weights_rect(N, N), energy_weights(N))
    # (Nv, Nh) = (8, 4), (u, v) = (3, 1): (4 * 2 / 32)^2 = 1/16 -> e^(15/16)
    assert energy_weights_rect(8, 4)[3, 1] == pytest.approx(math.exp(15 / 16), rel=1e-15)
    # (u, v) = (7, 1): (8 * 2 / 32)^2 = 1/4 -> e^(3/4)
    assert energy_weights_rect(8, 4)[7, 1] == pytest.approx(math.exp(0.75), rel=1e-15)


def test_422_planes_and_grid():
    assert chroma_shape(Config(64, 48, chroma_format="422")) == (48, 32)
    assert chroma_shape(Config(66, 50, chroma_format="422")) == (50, 33)
    assert Config(64, 64, block_size=32, chroma_format="422").chroma_block() == (32, 16)
    assert Config(64, 64, block_size=16, low_pass=True, chroma_format="422").chroma_block() == (16, 8)
    sp = frames_list(SequenceSpec(66, 50, 2, 3, chroma_format="422"))
    assert sp[0][0].shape == (50, 66) and sp[0][1].shape == (50, 33) and sp[0][2].shape == (50, 33)


@pytest.mark.parametrize("bit_depth", [8, 12])
def test_422_flat_chroma_closed_form(bit_depth):
    # Flat chroma planes: E_U = E_V = 0, L = sqrt(c 2^(15-B)), including the partial blocks at the
    # right and bottom edges (3 x 2 grid of 16 x 16 luma blocks over a 40 x 20 frame).
    W, H = 40, 20
    rng = np.random.default_rng(bit_depth)
    y = rng.integers(0, 1 << bit_depth, size=(H, W))
    u = np.full((H, W // 2), 77 << (bit_depth - 8))
    v = np.full((H, W // 2), 200 << (bit_depth - 8))
    f = analyze_sequence([(y, u, v)], Config(W, H, bit_depth, 16, chroma_format="422"))[0]
    assert f["E_U"] == 0.0 and f["E_V"] == 0.0
    assert f["L_U"] == pytest.approx(math.sqrt((77 << (bit_depth - 8)) * 2 ** (15 - bit_depth)), rel=1e-15)
    assert f["L_V"] == pytest.approx(math.sqrt((200 << (bit_depth - 8)) * 2 ** (15 - bit_depth)), rel=1e-15)
    luma = analyze_sequence([(y, y[:H // 2, :W // 2], y[:H // 2, :W // 2])], Config(W, H, bit_depth, 16))[0]
    assert f["E_Y"] == luma["E_Y"] and f["L_Y"] == luma["L_Y"]


def test_422_column_pattern_energy_by_hand():
    # One 32 x 32 luma block; U varies only along its 16 columns, so only row u = 0 of its 32 x 16
    # coefficients survives: H_U = sum_{v >= 1} w(0, v) |Z[0][v]| with w(0, v) = exp(1 - ((v+1)/512)^2),
    # and E_U = H_U / (1 * 32 * 16).
    B = 8
    f = np.random.default_rng(12).integers(0, 256, size=16)
    u = np.tile(f, (32, 1))
    y = np.full((32, 32), 50)
    v = np.full((32, 16), 128)
    M = int_dct_matrix(16)
    s1 = 3                                                  # log2 16 + 8 - 9
    t = [(sum(int(M[k][c]) * int(f[c]) for c in range(16)) + (1 << (s1 - 1))) >> s1 for k in range(16)]
    z0 = [(64 * 32 * tk + (1 << 10)) >> 11 for tk in t]       # s2 = log2 32 + 6 = 11
    h = sum(math.exp(1 - ((k + 1) / 512) ** 2) * abs(z0[k]) for k in range(1, 16))
    fe = analyze_sequence([(y, u, v)], Config(32, 32, B, 32, chroma_format="422"))[0]
    assert fe["E_U"] == pytest.approx(h / (32 * 16), rel=1e-14)
    assert fe["L_U"] == pytest.approx(math.sqrt(z0[0]), rel=1e-15)
    assert fe["E_V"] == 0.0


def test_422_block_values_use_rect_blocks():
    # The per-block values of a 4:2:2 frame equal the rectangular transform of the co-located
    # (w x w/2) chroma areas taken by hand, edge rows and columns repeated.
    W, H, w = 72, 40, 16
    fr = frames_list(SequenceSpec(W, H, 1, 21, chroma_format="422"))[0]
    cfg = Config(W, H, 8, w, chroma_format="422")
    vals = frame_block_values(*fr, cfg)
    u = fr[1].astype(np.int64)
    nbx, nby = 5, 3
    for by in range(nby):
        for bx in range(nbx):
            rows = np.minimum(np.arange(by * 16, by * 16 + 16), H - 1)
            cols = np.minimum(np.arange(bx * 8, bx * 8 + 8), W // 2 - 1)
            blk = u[rows][:, cols]
            Z = int_dct2_rect(blk, 8)
            assert vals["H_U"][by * nbx + bx] == block_texture_energy_rect(Z, 16, 8)
            assert vals["L_U"][by * nbx + bx] == math.sqrt(Z[0, 0])
