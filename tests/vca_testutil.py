"""Helpers shared by the GPU parity tests: device upload of synthetic frames, oracle
evaluation of the same frames, and the feature tolerance.

Tolerance (per feature, FP32 block arithmetic against the FP64 oracle):
  E_*, L_*: |got - exp| <= 1e-6 * |exp|;
  h:        |got - exp| <= 1e-6 * max(h, E_Y), because h is a difference of FP32 block
            energies and cancels (|H_t - H_{t-1}| << H);
  per-block H: relative 3e-6 -- 32 FMAs along u and a 5-level tree over v, each rounding
            by at most 2^-24 of a sum of non-negative terms, plus the FP32 weight rounding,
            bound the relative error by 38 * 2^-24 = 2.3e-6;
  per-block L: relative 2^-23 (one correctly rounded FP32 square root of an exact integer);
  coefficients: bit-exact.
"""

import numpy as np

from oracle import (Config, analyze_sequence, block_grid, downsample_plane, frame_block_values, int_dct2,
                    int_dct2_rect, int_dct_matrix, plane_blocks, sequence_features)
from synth import pack_planes

FEATURES = ("E_Y", "h", "L_Y", "E_U", "E_V", "L_U", "L_V")
FEATURE_RTOL = 1e-6
BLOCK_H_RTOL = 3e-6
BLOCK_L_RTOL = 2.0 ** -23


def to_device(frames, pitch_align=64):
    """(y, u, v) torch CUDA tensors shaped (F, rows, pitch_in_samples) from numpy planes."""
    import torch

    pk = pack_planes(frames, pitch_align)
    out = []
    for k in ("y", "u", "v"):
        a = pk[k]
        if a.dtype == np.uint16:
            a = a.view(np.int16)
        out.append(torch.from_numpy(np.ascontiguousarray(a)).cuda())
    return tuple(out)


def to_host_pinned(frames, pitch_align=64):
    import torch

    pk = pack_planes(frames, pitch_align)
    out = []
    for k in ("y", "u", "v"):
        a = pk[k]
        if a.dtype == np.uint16:
            a = a.view(np.int16)
        out.append(torch.from_numpy(np.ascontiguousarray(a)).pin_memory())
    return tuple(out)


def oracle_config(an) -> Config:
    c = an.cfg
    mats = tuple((n, tuple(tuple(int(v) for v in row) for row in m)) for n, m in sorted(an.dct_matrices.items()))
    return Config(c.width, c.height, c.bit_depth, c.block_size, c.low_pass == 1,
                  "skip" if c.pad_mode == 1 else "replicate", downsample=c.low_pass == 2,
                  chroma_format={1: "444", 2: "422"}.get(c.chroma_format, "420"), dct_matrices=mats)


def structured_dct_matrix(N, changes=()):
    """An N x N integer matrix with the structure of the DCT, built from its free entries.

    At each level L = N, N/2, ..., 2 the free entries are the odd rows of the level's matrix on
    its first L/2 columns; the other half of an odd row is its negated mirror image, the even rows
    are the level L/2 matrix and its mirror image, and level 1 is [[64]].  The free entries start
    from the round-cosine matrix's; `changes` adds ((L, j, n), delta) to odd row j (row 2j+1 of
    level L) at column n."""
    M0 = int_dct_matrix(N)
    free = {}
    L = N
    while L >= 2:
        free[L] = M0[::N // L, :L][1::2, :L // 2].copy()
        L //= 2
    for (L, j, n), d in changes:
        free[L][j, n] += d

    def build(L):
        if L == 1:
            return np.array([[64]], dtype=np.int64)
        h = L // 2
        E = build(h)
        M = np.zeros((L, L), dtype=np.int64)
        M[0::2, :h] = E
        M[0::2, h:] = E[:, ::-1]
        M[1::2, :h] = free[L]
        M[1::2, h:] = -free[L][:, ::-1]
        return M

    return build(N)


def oracle_coefficients(frame, cfg: Config):
    nbx, nby = block_grid(cfg)
    y, u, v = frame
    if cfg.downsample:
        y, u, v = downsample_plane(y), downsample_plane(u), downsample_plane(v)
    ny, _ = cfg.transform_sizes()
    nv, nh = cfg.chroma_block()
    return {
        "Y": int_dct2(plane_blocks(y, ny, nbx, nby), cfg.bit_depth, cfg.low_pass, cfg.matrix(ny)),
        "U": int_dct2_rect(plane_blocks(u, nv, nbx, nby, nh), cfg.bit_depth, cfg.low_pass, cfg.matrix(nh),
                           cfg.matrix(nv)),
        "V": int_dct2_rect(plane_blocks(v, nv, nbx, nby, nh), cfg.bit_depth, cfg.low_pass, cfg.matrix(nh),
                           cfg.matrix(nv)),
    }


def feature_errors(got: dict, exp: dict) -> dict:
    err = {}
    for k in FEATURES:
        if k == "h":
            denom = max(abs(exp["h"]), abs(exp["E_Y"]), 1e-300)
        else:
            denom = max(abs(exp[k]), 1e-300)
        err[k] = abs(got[k] - exp[k]) / denom
    return err


def assert_features_close(got: dict, exp: dict, rtol=FEATURE_RTOL, where=""):
    err = feature_errors(got, exp)
    bad = {k: (got[k], exp[k], e) for k, e in err.items() if e > rtol}
    assert not bad, f"{where}: features off (got, expected, rel err): {bad}"


def assert_block_values_close(got: dict, exp: dict, where=""):
    for p in ("Y", "U", "V"):
        gH, eH = got["H_" + p].astype(np.float64), exp["H_" + p]
        tolH = BLOCK_H_RTOL * np.abs(eH) + 1e-30
        bad = np.nonzero(np.abs(gH - eH) > tolH)[0]
        assert bad.size == 0, f"{where}: H_{p} off at blocks {bad[:5]}: {gH[bad[:5]]} vs {eH[bad[:5]]}"
        gL, eL = got["L_" + p].astype(np.float64), exp["L_" + p]
        bad = np.nonzero(np.abs(gL - eL) > BLOCK_L_RTOL * np.abs(eL) + 1e-30)[0]
        assert bad.size == 0, f"{where}: L_{p} off at blocks {bad[:5]}: {gL[bad[:5]]} vs {eL[bad[:5]]}"


def oracle_sequence(frames, cfg: Config, prev_HY=None):
    per = analyze_sequence(frames, cfg, prev_HY)
    return per, sequence_features(per)


__all__ = ["FEATURES", "to_device", "to_host_pinned", "oracle_config", "oracle_coefficients", "feature_errors",
           "assert_features_close", "assert_block_values_close", "oracle_sequence", "frame_block_values"]
