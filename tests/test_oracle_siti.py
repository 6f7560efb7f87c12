"""Pins of the oracle's SI / TI (the paper's comparison features, Section 2: SI =
max std[Sobel(F)], TI = max std[F_t - F_{t-1}])."""

import math

import numpy as np
import pytest
import scipy.ndimage

from oracle import frame_si, frame_ti, siti_sequence, sobel_responses


def test_sobel_matches_scipy_on_the_interior():
    rng = np.random.default_rng(1)
    F = rng.integers(0, 1024, size=(23, 31))
    gx, gy = sobel_responses(F)
    sx = scipy.ndimage.sobel(F.astype(np.int64), axis=1)[1:-1, 1:-1]  # d/dx: across columns
    sy = scipy.ndimage.sobel(F.astype(np.int64), axis=0)[1:-1, 1:-1]
    assert np.array_equal(gx, sx) and np.array_equal(gy, sy)


def test_ramp_has_constant_gradient_and_zero_si():
    a, b = 3, -2
    y, x = np.indices((17, 19))
    F = a * x + b * y + 500
    gx, gy = sobel_responses(F)
    assert np.all(gx == 8 * a) and np.all(gy == 8 * b)
    assert frame_si(F) == pytest.approx(0.0, abs=1e-12)  # every magnitude is 8 sqrt(13)


def test_vertical_edge_closed_form():
    W, H, k = 20, 10, 7
    F = np.zeros((H, W), dtype=np.int64)
    F[:, k:] = 100
    # Two interior columns (k-1, k) see |Gx| = 400; the others 0.
    p = 2 / (W - 2)
    assert frame_si(F) == pytest.approx(400 * math.sqrt(p * (1 - p)), rel=1e-14)


def test_ti_closed_forms():
    F = np.zeros((8, 8), dtype=np.int64)
    assert frame_ti(F + 37, F) == 0.0
    G = F.copy()
    G[:, :4] = 5
    G[:, 4:] = -5
    assert frame_ti(G, F) == pytest.approx(5.0, rel=1e-15)
    assert frame_ti(F, None) == 0.0


def test_sequence_maxima():
    rng = np.random.default_rng(2)
    frames = [rng.integers(0, 256, size=(12, 14)) for _ in range(4)]
    per, seq = siti_sequence(frames)
    assert per[0]["TI"] == 0.0
    assert seq["SI"] == max(frame_si(f) for f in frames)
    assert seq["TI"] == max(frame_ti(frames[t], frames[t - 1]) for t in range(1, 4))
