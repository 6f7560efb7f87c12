"""Pins of the oracle's transforms against closed forms, scipy and brute force.

Section 2 item (2) of the paper: the analyzer's DCT is an integer encoder routine.
The real-valued DCT-II is the textbook transform it approximates.
"""

import math
import os

import numpy as np
import pytest
import scipy.fft

from oracle import (int_dct2, int_dct2_butterfly, int_dct2_stages, int_dct_matrix, real_dct2_definition,
                    real_dct2_separable, real_dct_matrix, real_idct2_separable, round_shift, transform_shifts)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "int_dct_n4_n8.txt")


def load_golden():
    sections, cur = {}, None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line[1:-1]
                sections[cur] = []
            else:
                sections[cur].append([int(t) for t in line.split()])
    return {k: np.array(v, dtype=np.int64) for k, v in sections.items()}


# --- real DCT-II -----------------------------------------------------------

@pytest.mark.parametrize("N", [4, 8])
def test_real_dct_definition_matches_separable_and_scipy(N):
    rng = np.random.default_rng(N)
    x = rng.uniform(-128, 128, size=(N, N))
    d = real_dct2_definition(x)
    assert np.max(np.abs(d - real_dct2_separable(x))) < 1e-9
    assert np.max(np.abs(d - scipy.fft.dctn(x, type=2, norm="ortho"))) < 1e-9


def test_real_dct_32_definition_matches_scipy():
    x = np.random.default_rng(32).integers(0, 256, size=(32, 32)).astype(np.float64)
    assert np.max(np.abs(real_dct2_definition(x) - scipy.fft.dctn(x, type=2, norm="ortho"))) < 1e-8


@pytest.mark.parametrize("N", [4, 8, 16, 32])
def test_real_dct_parseval_and_inverse(N):
    x = np.random.default_rng(100 + N).uniform(0, 255, size=(5, N, N))
    X = real_dct2_separable(x)
    np.testing.assert_allclose(np.sum(X ** 2, axis=(1, 2)), np.sum(x ** 2, axis=(1, 2)), rtol=1e-12)
    assert np.max(np.abs(real_idct2_separable(X) - x)) < 1e-11


@pytest.mark.parametrize("N", [4, 8])
def test_real_dct_basis_image_gives_single_coefficient(N):
    # The (u0, v0) basis image alpha_u0 alpha_v0 cos(.)cos(.) transforms to a unit impulse at (u0, v0).
    A = real_dct_matrix(N)
    for u0 in range(N):
        for v0 in range(N):
            basis = np.outer(A[u0], A[v0])
            X = real_dct2_definition(basis)
            expect = np.zeros((N, N))
            expect[u0, v0] = 1.0
            assert np.max(np.abs(X - expect)) < 1e-12


# --- integer matrix ---------------------------------------------------------

def test_int_matrix_small_sizes_match_hand_values():
    g = load_golden()
    np.testing.assert_array_equal(int_dct_matrix(4), g["M4"])
    np.testing.assert_array_equal(int_dct_matrix(8), g["M8"])


@pytest.mark.parametrize("N", [4, 8, 16, 32])
def test_int_matrix_structure(N):
    M = int_dct_matrix(N)
    assert np.all(M[0] == 64)
    assert np.abs(M).max() <= 90
    assert np.all(M[1:].sum(axis=1) == 0)                      # AC rows have zero sum
    assert np.all(M[0::2] == M[0::2, ::-1])                    # even rows symmetric
    assert np.all(M[1::2] == -M[1::2, ::-1])                   # odd rows antisymmetric
    if N > 4:
        np.testing.assert_array_equal(M[0::2, : N // 2], int_dct_matrix(N // 2))
    # near-orthogonality: M M^T ~ 64^2 N I
    G = M @ M.T
    assert np.max(np.abs(G - 4096 * N * np.eye(N))) < 0.02 * 4096 * N


@pytest.mark.parametrize("N", [4, 8, 16, 32])
def test_int_matrix_has_no_ambiguous_rounding(N):
    raw = 64 * math.sqrt(N) * real_dct_matrix(N)
    dist = np.abs(np.abs(raw) - np.floor(np.abs(raw)) - 0.5)
    assert dist.min() > 1e-3


def test_shift_table():
    assert transform_shifts(32, 8) == (4, 11)
    assert transform_shifts(16, 8) == (3, 10)
    assert transform_shifts(32, 10) == (6, 11)
    assert transform_shifts(8, 8) == (2, 9)
    assert transform_shifts(4, 8) == (1, 8)


def test_round_shift_is_floor_with_half_up():
    v = np.array([-3, -2, -1, 0, 1, 2, 3, 5, -5, 7, -7], dtype=np.int64)
    # (v + 1) >> 1 == floor(v/2 + 1/2)
    np.testing.assert_array_equal(round_shift(v, 1), np.floor(v / 2 + 0.5).astype(np.int64))
    np.testing.assert_array_equal(round_shift(v, 2), np.floor(v / 4 + 0.5).astype(np.int64))


# --- integer transform -----------------------------------------------------

def test_int_dct_worked_examples():
    g = load_golden()
    x = np.zeros((4, 4), dtype=np.int64)
    x[0, 0] = 3
    np.testing.assert_array_equal(int_dct2(x, 8), g["Z4_delta_r0c0_p3"])
    x = np.zeros((4, 4), dtype=np.int64)
    x[3, 3] = 3
    np.testing.assert_array_equal(int_dct2(x, 8), g["Z4_delta_r3c3_p3"])


@pytest.mark.parametrize("N", [4, 8, 16, 32])
@pytest.mark.parametrize("B", [8, 10, 12])
def test_matrix_form_equals_butterfly_form(N, B):
    rng = np.random.default_rng(N * 31 + B)
    x = rng.integers(0, 1 << B, size=(40, N, N))
    extremes = np.stack([np.full((N, N), (1 << B) - 1),
                         np.indices((N, N)).sum(0) % 2 * ((1 << B) - 1),
                         (np.indices((N, N))[1] % 2) * ((1 << B) - 1),
                         np.zeros((N, N), dtype=np.int64)])
    x = np.concatenate([x, extremes])
    np.testing.assert_array_equal(int_dct2(x, B), int_dct2_butterfly(x, B))


@pytest.mark.parametrize("N", [4, 8, 16, 32])
@pytest.mark.parametrize("B", [8, 10, 12])
def test_flat_block_closed_form(N, B):
    for v in (0, 1, 17, (1 << B) - 1):
        x = np.full((N, N), v, dtype=np.int64)
        T, Z = int_dct2_stages(x, B)
        assert np.all(T[:, 0] == v << (15 - B)) and np.all(T[:, 1:] == 0)
        assert Z[0, 0] == v << (15 - B)
        Z[0, 0] = 0
        assert np.all(Z == 0)


@pytest.mark.parametrize("N", [8, 32])
def test_orientation_rows_first(N):
    # Column-only pattern x[r][c] = f(c): stage 1 gives the same row for every r, so only u = 0 survives.
    B = 8
    M = int_dct_matrix(N)
    s1, s2 = transform_shifts(N, B)
    f = np.random.default_rng(5).integers(0, 256, size=N)
    x = np.tile(f, (N, 1))
    Z = int_dct2(x, B)
    t = [(int(np.dot(M[v], f)) + (1 << (s1 - 1))) >> s1 for v in range(N)]
    expect0 = [(64 * N * tv + (1 << (s2 - 1))) >> s2 for tv in t]
    np.testing.assert_array_equal(Z[0], expect0)
    assert np.all(Z[1:] == 0)
    # Row-only pattern x[r][c] = g(r): stage 1 keeps only k = 0, so only v = 0 survives.
    g = np.random.default_rng(6).integers(0, 256, size=N)
    x = np.tile(g[:, None], (1, N))
    Z = int_dct2(x, B)
    T0 = [(64 * N * int(gr) + (1 << (s1 - 1))) >> s1 for gr in g]
    expect = [(int(np.dot(M[u], T0)) + (1 << (s2 - 1))) >> s2 for u in range(N)]
    np.testing.assert_array_equal(Z[:, 0], expect)
    assert np.all(Z[:, 1:] == 0)


@pytest.mark.parametrize("N", [4, 8, 16, 32])
@pytest.mark.parametrize("B", [8, 10, 12])
def test_integer_transform_tracks_real_dct(N, B):
    # Z ~ 4096 / (N 2^(B-3)) * orthonormal DCT-II: the matrix is 64 sqrt(N) A rounded, and the
    # two shifts divide by 2^(2 log2 N + B - 3).
    scale = 4096.0 / (N * 2 ** (B - 3))
    x = np.random.default_rng(N + B).integers(0, 1 << B, size=(50, N, N))
    Z = int_dct2(x, B).astype(np.float64)
    X = scipy.fft.dctn(x.astype(np.float64), type=2, norm="ortho", axes=(1, 2)) * scale
    err = np.abs(Z - X)
    # The matrix rounding (|error| <= 1/2 per entry of a matrix with entries up to 90) leaves a
    # relative error of about 0.3 %; a transposed, mis-indexed or mis-shifted transform is off by O(1).
    assert np.sqrt(np.mean(err ** 2)) < 0.006 * np.sqrt(np.mean(X ** 2))
    assert err.max() < 0.005 * np.abs(X).max()


@pytest.mark.parametrize("N", [16, 32])
@pytest.mark.parametrize("B", [8, 10])
def test_intermediate_and_output_fit_int16(N, B):
    mx = (1 << B) - 1
    idx = np.indices((N, N))
    blocks = [np.full((N, N), mx), np.zeros((N, N), dtype=np.int64),
              (idx.sum(0) % 2) * mx, (idx[1] % 2) * mx, (idx[0] % 2) * mx]
    M = int_dct_matrix(N)
    for k in range(N):  # sign-matched patterns that maximise each stage-1 output
        blocks.append(np.tile((M[k] > 0) * mx, (N, 1)))
        blocks.append(np.tile((M[k] > 0)[:, None] * mx, (1, N)))
    rng = np.random.default_rng(9)
    blocks += list(rng.integers(0, mx + 1, size=(30, N, N)))
    T, Z = int_dct2_stages(np.stack(blocks), B)
    assert T.max() <= 32767 and T.min() >= -32768
    assert Z.max() <= 32767 and Z.min() >= -32768


@pytest.mark.parametrize("N", [8, 16, 32])
def test_low_pass_is_top_left_quarter(N):
    x = np.random.default_rng(N).integers(0, 256, size=(20, N, N))
    full = int_dct2(x, 8)
    lp = int_dct2(x, 8, low_pass=True)
    np.testing.assert_array_equal(lp, full[:, : N // 2, : N // 2])
