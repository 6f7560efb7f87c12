"""Caller-supplied integer DCT matrices in the oracle (the drop-in table of an encoder, such as a
hand-tuned standard table, in place of the round-cosine reading of Section 2 item (2)).

Pins: the structured-matrix builder reproduces the round-cosine matrix from its free entries; for
any matrix of that structure the recursive butterfly equals the matrix form bit for bit (the
identity the CUDA-core form relies on), while a matrix that breaks the structure makes them
differ; the configuration's matrices reach the per-block transform of every plane.
"""

import numpy as np
import pytest

from oracle import (Config, block_grid, frame_block_values, int_dct2, int_dct2_butterfly, int_dct_matrix,
                    plane_block_values, plane_blocks)
from vca_testutil import structured_dct_matrix

CHANGES = {  # a few free entries moved by one or two, at every level
    4: (((4, 0, 0), -1), ((4, 1, 1), 1), ((2, 0, 0), 1)),
    8: (((8, 0, 0), -1), ((8, 3, 2), 2), ((4, 1, 0), 1)),
    16: (((16, 0, 0), -1), ((16, 5, 3), 1), ((8, 2, 1), -2), ((4, 0, 1), 1)),
    32: (((32, 0, 0), -1), ((32, 7, 9), 2), ((16, 3, 4), 1), ((8, 1, 0), -1), ((2, 0, 0), -1)),
}


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32])
def test_builder_reproduces_round_cosine(N):
    assert np.array_equal(structured_dct_matrix(N), int_dct_matrix(N))


@pytest.mark.parametrize("N", [4, 8, 16, 32])
@pytest.mark.parametrize("B", [8, 10])
def test_butterfly_equals_matrix_form_for_structured_matrices(N, B):
    M = structured_dct_matrix(N, CHANGES[N])
    assert not np.array_equal(M, int_dct_matrix(N))
    assert np.all(M[0] == 64) and np.abs(M).max() <= 127
    rng = np.random.default_rng(N * 100 + B)
    x = rng.integers(0, 1 << B, size=(64, N, N))
    x[0] = (1 << B) - 1
    x[1] = np.where(np.add.outer(np.arange(N), np.arange(N)) % 2 == 0, (1 << B) - 1, 0)
    assert np.array_equal(int_dct2_butterfly(x, B, M), int_dct2(x, B, False, M))


@pytest.mark.parametrize("N", [8, 32])
def test_a_broken_structure_separates_the_forms(N):
    M = structured_dct_matrix(N, CHANGES[N])
    M[3, N - 1] += 1  # row 3 no longer odd about the middle
    rng = np.random.default_rng(7)
    x = rng.integers(0, 256, size=(16, N, N))
    assert not np.array_equal(int_dct2_butterfly(x, 8, M), int_dct2(x, 8, False, M))


def test_config_matrices_reach_every_plane():
    rng = np.random.default_rng(3)
    W, H = 96, 64
    y = rng.integers(0, 256, size=(H, W))
    u = rng.integers(0, 256, size=(H // 2, W // 2))
    v = rng.integers(0, 256, size=(H // 2, W // 2))
    My, Mc = structured_dct_matrix(32, CHANGES[32]), structured_dct_matrix(16, CHANGES[16])
    mats = ((16, tuple(map(tuple, Mc.tolist()))), (32, tuple(map(tuple, My.tolist()))))
    for lp in (False, True):
        cfg = Config(W, H, 8, 32, lp, dct_matrices=mats)
        assert np.array_equal(cfg.matrix(32), My) and np.array_equal(cfg.matrix(16), Mc)
        assert np.array_equal(cfg.matrix(8), int_dct_matrix(8))
        got = frame_block_values(y, u, v, cfg)
        nbx, nby = block_grid(cfg)
        for name, plane, n, M in (("Y", y, 32, My), ("U", u, 16, Mc), ("V", v, 16, Mc)):
            Hs, Ls, Z = plane_block_values(plane, n, nbx, nby, 8, lp, M)
            assert np.array_equal(Z, int_dct2(plane_blocks(plane, n, nbx, nby), 8, lp, M))
            assert np.array_equal(got["H_" + name], Hs) and np.array_equal(got["L_" + name], Ls)
        # and the default matrices give different values
        base = frame_block_values(y, u, v, Config(W, H, 8, 32, lp))
        assert not np.array_equal(base["H_Y"], got["H_Y"])
