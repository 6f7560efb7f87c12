"""Exact-integer / FP64 CPU oracle of the Video Complexity Analyzer (VCA) hot path.

TEST INFRASTRUCTURE.  This module is the slow, plain statement of what the CUDA
path must compute.  Only the tests, the smoke check and the CPU-baseline legs of
the benchmark may import it; the CUDA library shares no code, table or constant
with it (the library derives its own transform matrix and weights).

What the paper fixes
--------------------
Section 2 of the paper (Video complexity analyzer) says VCA computes seven
blockwise DCT-energy features per frame: the luma texture energy E_Y, its
temporal gradient h, the luminescence L_Y, the chroma texture energies E_U, E_V
and the chrominances L_U, L_V.  Section 2 item (1) says each block's DCT energy
is independent work; item (2) says the DCT is an integer SIMD encoder routine;
item (3) adds a low-pass DCT option that evaluates the features as if the video
were downsampled by two in each direction.  Section 3 measures UHD 8-bit video.

The formulas themselves sit in the VCA reference that the paper cites and does
not reproduce.  Every definition below is therefore a *reading*, stated where it
is used:

* input: planar Y, U, V, integer samples of bit depth B in {8, 10, 12}; chroma
  4:2:0 (planes of half width and height), 4:2:2 (half width, full height) or
  4:4:4 (full-size planes);
* block grid: luma w x w blocks, chroma blocks covering the same picture area
  ((w/2) x (w/2) samples in 4:2:0, (w/2) wide by w tall in 4:2:2, w x w in
  4:4:4) on the same (co-located) grid; partial blocks at the right/bottom edge
  are completed by repeating the last row/column ("replicate"), or dropped
  ("skip");
* integer DCT matrix M_N[k][n] = round_half_away(64 sqrt(N) alpha_k
  cos(pi (2n+1) k / 2N)) and the two-stage forward transform of HEVC encoders:
  rows first with shift s1 = log2 N + B - 9, then columns with s2 = log2 N + 6,
  each stage adding 2^(s-1) before an arithmetic right shift;
* low-pass: only coefficients with u, v < N/2 are computed (stage 1 keeps the
  first N/2 row outputs, stage 2 the first N/2 column outputs);
* rectangular (4:2:2 chroma) blocks of Nv rows and Nh columns: rows first with
  the Nh-point matrix and s1 = log2 Nh + B - 9, then columns with the Nv-point
  matrix and s2 = log2 Nv + 6 (each stage's shift from its own length, as the
  encoders' rectangular transforms do); low-pass keeps the first half of each
  dimension; weights w(u,v) = exp(|((u+1)(v+1)/(Nv Nh))^2 - 1|); E divides by
  C Nv Nh;
* low-pass, downsample reading: every plane is first downsampled by two in each
  direction (the rounded mean of each 2x2 group, (a + b + c + d + 2) >> 2, edges
  repeated for odd sizes); the downsampled frame is then analysed with half-size
  blocks (luma w/2, chroma w/4) on the same block grid, all coefficients, and the
  normalisations use the half-size blocks;
* block texture energy H = sum over computed (u,v) != (0,0) of
  w_N(u,v) |Z(u,v)| with w_N(u,v) = exp(|((u+1)(v+1)/N^2)^2 - 1|), N the full
  block size also under low-pass;
* block brightness L = sqrt(Z(0,0));
* frame features E_P = sum_k H_{P,k} / (C N_P^2), L_P = sum_k L_{P,k} / C,
  h_t = sum_k |H_{Y,k,t} - H_{Y,k,t-1}| / (C w^2) for t >= 1 and h_0 = 0;
* sequence features: arithmetic mean over frames (h over t >= 1).

Parity status: each function is pinned by the ``-m "not gpu"`` oracle tests
against closed forms, invariants, scipy's DCT or brute force.  Agreement with the
paper's own feature values is unpinned: the paper prints no feature value.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

FEATURES = ("E_Y", "h", "L_Y", "E_U", "E_V", "L_U", "L_V")


# ---------------------------------------------------------------------------
# Real-valued DCT-II (cross-check of the integer transform)
# ---------------------------------------------------------------------------

def dct_alpha(k: int, N: int) -> float:
    """Orthonormal DCT-II scale: sqrt(1/N) for k = 0, sqrt(2/N) otherwise."""
    return math.sqrt(1.0 / N) if k == 0 else math.sqrt(2.0 / N)


def real_dct_matrix(N: int) -> np.ndarray:
    """A[k][n] = alpha_k cos(pi (2n+1) k / (2N)), the orthonormal DCT-II basis."""
    A = np.empty((N, N), dtype=np.float64)
    for k in range(N):
        for n in range(N):
            A[k, n] = dct_alpha(k, N) * math.cos(math.pi * (2 * n + 1) * k / (2 * N))
    return A


def real_dct2_definition(x: np.ndarray) -> np.ndarray:
    """2-D DCT-II of one N x N block straight from its O(N^4) definition.

    X[u][v] = alpha_u alpha_v sum_r sum_c x[r][c] cos(pi(2r+1)u/2N) cos(pi(2c+1)v/2N),
    u indexing vertical frequency (rows r), v horizontal frequency (columns c).
    Pure Python loops: meant for N <= 8 (N = 32 takes about a second).
    """
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[0]
    out = np.empty((N, N), dtype=np.float64)
    for u in range(N):
        for v in range(N):
            s = 0.0
            for r in range(N):
                cu = math.cos(math.pi * (2 * r + 1) * u / (2 * N))
                for c in range(N):
                    s += x[r, c] * cu * math.cos(math.pi * (2 * c + 1) * v / (2 * N))
            out[u, v] = dct_alpha(u, N) * dct_alpha(v, N) * s
    return out


def real_dct2_separable(x: np.ndarray) -> np.ndarray:
    """Separable form of the same transform: A x A^T (any leading batch axes)."""
    x = np.asarray(x, dtype=np.float64)
    A = real_dct_matrix(x.shape[-1])
    return A @ x @ A.T


def real_idct2_separable(X: np.ndarray) -> np.ndarray:
    """Inverse of the orthonormal 2-D DCT-II: A^T X A."""
    X = np.asarray(X, dtype=np.float64)
    A = real_dct_matrix(X.shape[-1])
    return A.T @ X @ A


# ---------------------------------------------------------------------------
# Integer transform (Section 2 item (2): integer encoder DCT routines)
# ---------------------------------------------------------------------------

def round_half_away(x) -> np.ndarray:
    """Round to nearest, ties away from zero."""
    x = np.asarray(x, dtype=np.float64)
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def int_dct_matrix(N: int) -> np.ndarray:
    """Integer DCT matrix M_N[k][n] = round_half_away(64 sqrt(N) A[k][n]).

    Row 0 is 64 everywhere; for N = 16 and 32 the largest magnitude is 90.
    """
    return round_half_away(64.0 * math.sqrt(N) * real_dct_matrix(N)).astype(np.int64)


def transform_shifts(N: int, bit_depth: int) -> tuple[int, int]:
    """Stage shifts of the two-stage forward transform: s1 = log2 N + B - 9, s2 = log2 N + 6."""
    log2n = int(round(math.log2(N)))
    if (1 << log2n) != N:
        raise ValueError("block size must be a power of two")
    s1 = log2n + bit_depth - 9
    s2 = log2n + 6
    if s1 < 0:
        raise ValueError("unsupported block size / bit depth pair")
    return s1, s2


def round_shift(v, s: int) -> np.ndarray:
    """(v + 2^(s-1)) >> s on int64, '>>' an arithmetic (floor) shift; s = 0 is identity."""
    v = np.asarray(v, dtype=np.int64)
    if s == 0:
        return v
    return (v + (np.int64(1) << np.int64(s - 1))) >> np.int64(s)


def int_dct2_stages(blocks, bit_depth: int, low_pass: bool = False, M=None):
    """Two-stage integer forward DCT of blocks shaped (..., N, N).

    Stage 1 (rows):    T[r][k] = (sum_c x[r][c] M[k][c] + 2^(s1-1)) >> s1
    Stage 2 (columns): Z[u][v] = (sum_r M[u][r] T[r][v] + 2^(s2-1)) >> s2
    Low-pass (Section 2 item (3)): k and u run over the first N/2 rows of M only.
    M is the N x N integer matrix (default: the round-cosine matrix; a caller may supply another
    table of the same structure, such as an encoder's hand-tuned one).
    Returns (T, Z) as int64 arrays; T is (..., N, Nk) and Z is (..., Nk, Nk).
    """
    x = np.asarray(blocks, dtype=np.int64)
    N = x.shape[-1]
    M = int_dct_matrix(N) if M is None else np.asarray(M, dtype=np.int64)
    Nk = N // 2 if low_pass else N
    Mk = M[:Nk]
    s1, s2 = transform_shifts(N, bit_depth)
    T = round_shift(np.matmul(x, Mk.T), s1)
    Z = round_shift(np.matmul(Mk, T), s2)
    return T, Z


def int_dct2(blocks, bit_depth: int, low_pass: bool = False, M=None) -> np.ndarray:
    """Quantised coefficients Z of the two-stage integer transform (see int_dct2_stages)."""
    return int_dct2_stages(blocks, bit_depth, low_pass, M)[1]


def _butterfly_1d(x: np.ndarray, N: int, M=None) -> np.ndarray:
    """Raw 1-D integer transform y[k] = sum_n M_N[k][n] x[n] along the last axis.

    Even/odd decomposition: even outputs are the N/2-point transform of
    e[n] = x[n] + x[N-1-n] with the matrix of M's even rows on the first N/2 columns; odd outputs
    apply the odd rows of M (first half of the columns) to o[n] = x[n] - x[N-1-n].  Recurses
    down to the 1 x 1 matrix [[64]].  This equals the matrix form exactly when M has the DCT's
    structure (row 0 all 64, row k even / odd about the middle for even / odd k, and the even
    rows on the first half forming a matrix of the same structure).
    """
    if M is None:
        M = int_dct_matrix(N)
    M = np.asarray(M, dtype=np.int64)
    if N == 1:
        return 64 * x
    h = N // 2
    a = x[..., :h]
    b = x[..., ::-1][..., :h]
    e = a + b
    o = a - b
    y = np.empty(x.shape[:-1] + (N,), dtype=np.int64)
    y[..., 0::2] = _butterfly_1d(e, h, M[0::2, :h])
    y[..., 1::2] = np.matmul(o, M[1::2, :h].T)
    return y


def int_dct2_butterfly(blocks, bit_depth: int, M=None) -> np.ndarray:
    """Same two-stage integer transform computed with the recursive butterfly (full Z only)."""
    x = np.asarray(blocks, dtype=np.int64)
    N = x.shape[-1]
    s1, s2 = transform_shifts(N, bit_depth)
    T = round_shift(_butterfly_1d(x, N, M), s1)
    Zt = round_shift(_butterfly_1d(np.swapaxes(T, -1, -2), N, M), s2)
    return np.swapaxes(Zt, -1, -2)


# ---------------------------------------------------------------------------
# Block features (Section 2: E, L per block)
# ---------------------------------------------------------------------------

def int_dct2_rect_stages(blocks, bit_depth: int, low_pass: bool = False, Mh=None, Mv=None):
    """Two-stage integer forward transform of rectangular blocks shaped (..., Nv, Nh).

    Stage 1 (rows, Nh-point):    T[r][k] = (sum_c x[r][c] Mh[k][c] + 2^(s1-1)) >> s1, s1 = log2 Nh + B - 9
    Stage 2 (columns, Nv-point): Z[u][v] = (sum_r Mv[u][r] T[r][v] + 2^(s2-1)) >> s2, s2 = log2 Nv + 6
    Low-pass: k < Nh/2 and u < Nv/2.  Mh, Mv default to the round-cosine matrices.
    Returns (T, Z): T is (..., Nv, Nkh), Z is (..., Nkv, Nkh).
    """
    x = np.asarray(blocks, dtype=np.int64)
    Nv, Nh = x.shape[-2], x.shape[-1]
    Mh = int_dct_matrix(Nh) if Mh is None else np.asarray(Mh, dtype=np.int64)
    Mv = int_dct_matrix(Nv) if Mv is None else np.asarray(Mv, dtype=np.int64)
    Nkh = Nh // 2 if low_pass else Nh
    Nkv = Nv // 2 if low_pass else Nv
    s1 = transform_shifts(Nh, bit_depth)[0]
    s2 = transform_shifts(Nv, bit_depth)[1]
    T = round_shift(np.matmul(x, Mh[:Nkh].T), s1)
    Z = round_shift(np.matmul(Mv[:Nkv], T), s2)
    return T, Z


def int_dct2_rect(blocks, bit_depth: int, low_pass: bool = False, Mh=None, Mv=None) -> np.ndarray:
    """Quantised coefficients Z of the rectangular two-stage transform (see int_dct2_rect_stages)."""
    return int_dct2_rect_stages(blocks, bit_depth, low_pass, Mh, Mv)[1]


def energy_weights_rect(Nv: int, Nh: int) -> np.ndarray:
    """w(u,v) = exp(|((u+1)(v+1)/(Nv Nh))^2 - 1|) for 0 <= u < Nv, 0 <= v < Nh."""
    w = np.empty((Nv, Nh), dtype=np.float64)
    for u in range(Nv):
        for v in range(Nh):
            w[u, v] = math.exp(abs(((u + 1) * (v + 1) / (Nv * Nh)) ** 2 - 1.0))
    return w


def block_texture_energy_rect(Z: np.ndarray, Nv: int, Nh: int) -> np.ndarray:
    """H = sum_{(u,v) != (0,0)} w(u,v) |Z(u,v)| of rectangular blocks (FP64)."""
    Z = np.asarray(Z, dtype=np.int64)
    Nkv, Nkh = Z.shape[-2], Z.shape[-1]
    w = energy_weights_rect(Nv, Nh)[:Nkv, :Nkh].copy()
    w[0, 0] = 0.0
    return np.sum(np.abs(Z).astype(np.float64) * w, axis=(-2, -1))


def energy_weights(N: int) -> np.ndarray:
    """w_N(u,v) = exp(|((u+1)(v+1)/N^2)^2 - 1|) for 0 <= u, v < N."""
    w = np.empty((N, N), dtype=np.float64)
    for u in range(N):
        for v in range(N):
            w[u, v] = math.exp(abs(((u + 1) * (v + 1) / (N * N)) ** 2 - 1.0))
    return w


def block_texture_energy(Z: np.ndarray, N: int) -> np.ndarray:
    """H = sum_{(u,v) != (0,0)} w_N(u,v) |Z(u,v)| over the computed coefficients (FP64)."""
    Z = np.asarray(Z, dtype=np.int64)
    Nk = Z.shape[-1]
    w = energy_weights(N)[:Nk, :Nk].copy()
    w[0, 0] = 0.0  # DC is not texture
    return np.sum(np.abs(Z).astype(np.float64) * w, axis=(-2, -1))


def block_brightness(Z: np.ndarray) -> np.ndarray:
    """L = sqrt(Z(0,0)) (FP64)."""
    return np.sqrt(np.asarray(Z, dtype=np.int64)[..., 0, 0].astype(np.float64))


# ---------------------------------------------------------------------------
# Block grid and edge handling
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Config:
    width: int
    height: int
    bit_depth: int = 8
    block_size: int = 32
    low_pass: bool = False
    pad_mode: str = "replicate"  # or "skip"
    downsample: bool = False     # the downsample reading of the low-pass option (excludes low_pass)
    chroma_format: str = "420"   # or "422", "444"
    # Caller-supplied integer DCT matrices: ((N, rows), ...) with rows a tuple of N tuples of N
    # ints; a transform size without an entry uses the round-cosine matrix int_dct_matrix(N).
    dct_matrices: tuple = ()

    def matrix(self, n: int) -> np.ndarray:
        """The n x n integer DCT matrix of this configuration."""
        for size, rows in self.dct_matrices:
            if size == n:
                return np.asarray(rows, dtype=np.int64)
        return int_dct_matrix(n)

    def transform_sizes(self) -> tuple[int, int]:
        """(luma, chroma) block size of the transform: w and w/2 (4:2:0) or w (4:4:4), each
        halved when downsampling; for 4:2:2 the chroma block's width (w/2)."""
        w = self.block_size
        c = w if self.chroma_format == "444" else w // 2
        return (w // 2, c // 2) if self.downsample else (w, c)

    def chroma_block(self) -> tuple[int, int]:
        """(rows, columns) of a chroma block: (w/2, w/2) in 4:2:0, (w, w/2) in 4:2:2, (w, w) in
        4:4:4 (halved when downsampling, 4:2:0 only)."""
        w, c = self.transform_sizes()
        return (w, c) if self.chroma_format == "422" else (c, c)


def block_grid(cfg: Config) -> tuple[int, int]:
    """(blocks across, blocks down) of the luma grid, shared by the chroma planes."""
    w = cfg.block_size
    if cfg.pad_mode == "replicate":
        return -(-cfg.width // w), -(-cfg.height // w)
    if cfg.pad_mode == "skip":
        return cfg.width // w, cfg.height // w
    raise ValueError("pad_mode must be 'replicate' or 'skip'")


def chroma_shape(cfg: Config) -> tuple[int, int]:
    """(height, width) of a chroma plane: half size in 4:2:0, half width in 4:2:2, full size in
    4:4:4."""
    if cfg.chroma_format == "444":
        return cfg.height, cfg.width
    if cfg.chroma_format == "422":
        return cfg.height, (cfg.width + 1) // 2
    return (cfg.height + 1) // 2, (cfg.width + 1) // 2


def plane_blocks(plane: np.ndarray, n: int, nbx: int, nby: int, nh: int | None = None) -> np.ndarray:
    """Blocks of one plane in raster order, shaped (nby*nbx, n, nh): n rows and nh (default n)
    columns each.  Rows/columns past the plane's edge repeat its last row/column."""
    nh = n if nh is None else nh
    plane = np.asarray(plane)
    ph, pw = plane.shape
    ys = np.minimum(np.arange(nby * n), ph - 1)
    xs = np.minimum(np.arange(nbx * nh), pw - 1)
    padded = plane[ys][:, xs].astype(np.int64)
    return padded.reshape(nby, n, nbx, nh).transpose(0, 2, 1, 3).reshape(nby * nbx, n, nh)


def plane_block_values(plane, n: int, nbx: int, nby: int, bit_depth: int, low_pass: bool, M=None):
    """Per-block (H, L, Z) of one plane with n x n blocks (M: the n x n matrix, default round-cosine)."""
    Z = int_dct2(plane_blocks(plane, n, nbx, nby), bit_depth, low_pass, M)
    return block_texture_energy(Z, n), block_brightness(Z), Z


def downsample_plane(plane: np.ndarray) -> np.ndarray:
    """Halve a plane in each direction: each output sample is the rounded mean of a 2x2 group,
    (a + b + c + d + 2) >> 2; a plane of odd height or width repeats its last row or column."""
    p = np.asarray(plane).astype(np.int64)
    h, w = p.shape
    ys = np.minimum(np.arange(2 * ((h + 1) // 2)), h - 1)
    xs = np.minimum(np.arange(2 * ((w + 1) // 2)), w - 1)
    q = p[ys][:, xs]
    s = q[0::2, 0::2] + q[0::2, 1::2] + q[1::2, 0::2] + q[1::2, 1::2]
    return (s + 2) >> 2


def frame_block_values(y, u, v, cfg: Config) -> dict:
    """Per-block H and L of the Y, U and V planes of one frame."""
    nbx, nby = block_grid(cfg)
    ny, nc = cfg.transform_sizes()
    if cfg.downsample:
        y, u, v = downsample_plane(y), downsample_plane(u), downsample_plane(v)
    out = {}
    for name, plane, n in (("Y", y, ny), ("U", u, nc), ("V", v, nc)):
        if name != "Y" and cfg.chroma_format == "422":
            nv, nh = cfg.chroma_block()
            Z = int_dct2_rect(plane_blocks(plane, nv, nbx, nby, nh), cfg.bit_depth, cfg.low_pass, cfg.matrix(nh),
                              cfg.matrix(nv))
            H, L = block_texture_energy_rect(Z, nv, nh), block_brightness(Z)
        else:
            H, L, _ = plane_block_values(plane, n, nbx, nby, cfg.bit_depth, cfg.low_pass, cfg.matrix(n))
        out["H_" + name] = H
        out["L_" + name] = L
    return out


# ---------------------------------------------------------------------------
# Frame and sequence features (Section 2: the seven features)
# ---------------------------------------------------------------------------

def frame_features(values: dict, prev_HY, cfg: Config) -> dict:
    """Seven features of one frame from its per-block values (FP64).

    prev_HY is the previous frame's luma block energies, or None for the first
    frame of a sequence (then h = 0).
    """
    nbx, nby = block_grid(cfg)
    C = nbx * nby
    w, _ = cfg.transform_sizes()
    cv, ch = cfg.chroma_block()
    f = {
        "E_Y": float(np.sum(values["H_Y"])) / (C * w * w),
        "L_Y": float(np.sum(values["L_Y"])) / C,
        "E_U": float(np.sum(values["H_U"])) / (C * cv * ch),
        "E_V": float(np.sum(values["H_V"])) / (C * cv * ch),
        "L_U": float(np.sum(values["L_U"])) / C,
        "L_V": float(np.sum(values["L_V"])) / C,
    }
    if prev_HY is None:
        f["h"] = 0.0
    else:
        f["h"] = float(np.sum(np.abs(values["H_Y"] - prev_HY))) / (C * w * w)
    return f


def analyze_sequence(frames, cfg: Config, prev_HY=None) -> list[dict]:
    """Per-frame features of a sequence of (y, u, v) planes, in order."""
    out = []
    for (y, u, v) in frames:
        vals = frame_block_values(y, u, v, cfg)
        out.append(frame_features(vals, prev_HY, cfg))
        prev_HY = vals["H_Y"]
    return out


def sequence_features(per_frame: list[dict]) -> dict:
    """Mean of each feature over the frames; h averages frames t >= 1 (0 for one frame)."""
    n = len(per_frame)
    out = {"frames": n}
    for k in FEATURES:
        vals = [f[k] for f in per_frame]
        if k == "h":
            vals = vals[1:]
        out[k] = float(sum(vals) / len(vals)) if vals else 0.0
    return out


# ---------------------------------------------------------------------------
# SI / TI (the spatial and temporal information the paper compares VCA with,
# Section 2: SI = max over frames of std[Sobel(F)], TI = max over frames of
# std[F_t - F_{t-1}])
#
# Readings: F is the luma plane in raw sample values; Sobel(F) is the gradient
# magnitude sqrt(Gx^2 + Gy^2) of the 3x3 Sobel responses, evaluated on the interior
# pixels (the one-pixel border has no full neighbourhood); std is the population
# standard deviation over the pixels; the per-frame TI of the first frame is 0 and
# the sequence TI is the maximum over frames t >= 1.
# ---------------------------------------------------------------------------

def sobel_responses(plane) -> tuple[np.ndarray, np.ndarray]:
    """(Gx, Gy) on the interior pixels: Gx = right column - left column with weights 1, 2, 1
    down the rows, Gy = bottom row - top row with weights 1, 2, 1 across the columns (int64)."""
    F = np.asarray(plane).astype(np.int64)
    gx = (F[:-2, 2:] + 2 * F[1:-1, 2:] + F[2:, 2:]) - (F[:-2, :-2] + 2 * F[1:-1, :-2] + F[2:, :-2])
    gy = (F[2:, :-2] + 2 * F[2:, 1:-1] + F[2:, 2:]) - (F[:-2, :-2] + 2 * F[:-2, 1:-1] + F[:-2, 2:])
    return gx, gy


def frame_si(plane) -> float:
    """std over the interior pixels of sqrt(Gx^2 + Gy^2) (FP64)."""
    gx, gy = sobel_responses(plane)
    return float(np.std(np.sqrt((gx * gx + gy * gy).astype(np.float64))))


def frame_ti(plane, prev) -> float:
    """std over all pixels of F_t - F_{t-1} (FP64); 0 without a previous frame."""
    if prev is None:
        return 0.0
    d = np.asarray(plane).astype(np.int64) - np.asarray(prev).astype(np.int64)
    return float(np.std(d.astype(np.float64)))


def siti_sequence(lumas, prev=None) -> tuple[list, dict]:
    """Per-frame (SI, TI) of a sequence of luma planes and the sequence maxima."""
    per = []
    for F in lumas:
        per.append({"SI": frame_si(F), "TI": frame_ti(F, prev)})
        prev = F
    seq = {"SI": max(p["SI"] for p in per) if per else 0.0,
           "TI": max((p["TI"] for p in per[1:]), default=0.0)}
    return per, seq
