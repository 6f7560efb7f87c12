"""Host-side checks of the C-ABI library that need no GPU: it builds, loads, exports every
function include/vca.h declares, and rejects bad configurations before touching CUDA."""

import ctypes
import os
import re

import pytest

from paper_2304_12384_gb300 import build as vbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libvca():
    vbuild.build()
    from paper_2304_12384_gb300 import vca
    return vca


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(vca_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_header_declares_the_api():
    names = declared_functions()
    for required in ("vca_open", "vca_push_frame", "vca_push_frames", "vca_read_frame_features",
                     "vca_read_sequence_features", "vca_export_state", "vca_import_state", "vca_close",
                     "vca_status_str"):
        assert required in names


def test_library_exports_every_declared_symbol(libvca):
    L = libvca.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) <= set(libvca.exported_symbols()) | {"vca_status_str", "vca_last_error"}


def test_status_strings(libvca):
    assert libvca.vca_status_str(0) == "ok"
    assert libvca.vca_status_str(-1) == "invalid argument"


@pytest.mark.parametrize("cfg,status", [
    ((3841, 2160, 8, 32, 0, 0, 0, 64), -1),   # odd width
    ((0, 2160, 8, 32, 0, 0, 0, 64), -1),      # empty
    ((3840, 2160, 9, 32, 0, 0, 0, 64), -1),   # bit depth
    ((3840, 2160, 8, 24, 0, 0, 0, 64), -1),   # block size
    ((3840, 2160, 14, 32, 0, 0, 0, 64), -1),  # bit depth 14
    ((3840, 2160, 8, 32, 2, 0, 0, 64, 2), -2),  # 4:2:2 with the downsample reading
    ((3840, 2160, 8, 32, 0, 0, 0, 64, 5), -1),  # chroma format
    ((3840, 2160, 8, 32, 3, 0, 0, 64), -1),   # low_pass flag
    ((3840, 2160, 8, 16, 2, 0, 0, 64), -2),   # downsample reading needs block 32
    ((3840, 2160, 8, 32, 0, 5, 0, 64), -1),   # pad mode
    ((3840, 2160, 8, 32, 0, 0, 7, 64), -1),   # kernel selector
    ((3840, 2160, 8, 32, 0, 0, 0, 99999), -1),
    ((30, 30, 8, 32, 0, 1, 0, 64), -1),       # skip mode leaves no block
])
def test_config_validation(libvca, cfg, status):
    c = libvca.VcaConfig(*cfg)
    bx, by = ctypes.c_int64(), ctypes.c_int64()
    assert libvca.lib().vca_block_count(ctypes.byref(c), ctypes.byref(bx), ctypes.byref(by)) == status
    assert libvca.vca_last_error()
    h = ctypes.c_void_p()
    assert libvca.lib().vca_open(ctypes.byref(c), None, ctypes.byref(h)) == status
    assert h.value is None


@pytest.mark.parametrize("w,h,bs,mode,expect", [
    (3840, 2160, 32, 0, (120, 68)), (3840, 2160, 16, 0, (240, 135)), (1920, 1080, 32, 0, (60, 34)),
    (1920, 1080, 32, 1, (60, 33)), (640, 352, 32, 0, (20, 11)), (2, 2, 32, 0, (1, 1)),
])
def test_block_grid_matches_oracle(libvca, w, h, bs, mode, expect):
    from oracle import Config, block_grid
    c = libvca.VcaConfig(w, h, 8, bs, 0, mode, 0, 64)
    assert libvca.vca_block_count(c) == expect
    assert block_grid(Config(w, h, block_size=bs, pad_mode="skip" if mode else "replicate")) == expect


def test_null_arguments_are_rejected(libvca):
    L = libvca.lib()
    assert L.vca_open(None, None, None) == -1
    assert L.vca_push_frames(None, None, None, None, 0, 0, 0, 0, 1, 1) == -1
    assert L.vca_read_frame_features(None, 0, 1, None) == -1
    assert L.vca_close(None) == 0


# ---- drop-in DCT matrices: the library's structural check, pinned by what the oracle computes ----

def _matrix_cases():
    import numpy as np

    from oracle import int_dct_matrix
    from vca_testutil import structured_dct_matrix

    good = []
    for n in (4, 8, 16, 32):
        good.append(("round-cosine", n, int_dct_matrix(n)))
        good.append(("structured", n, structured_dct_matrix(n, (((n, 0, 0), -1), ((n // 2, 0, 0), -1)))))
    bad = []
    m = int_dct_matrix(8)
    m[3, 7] += 1
    bad.append(("odd row not odd", 8, m, "symmetry"))
    m = int_dct_matrix(16)
    m[2, 0] += 1  # even row of the top level, and odd row of level 8: both mirrors broken
    bad.append(("even row not even", 16, m, "symmetry"))
    m = int_dct_matrix(32)
    m[0, :] = 63
    bad.append(("row 0 not 64", 32, m, "not 64"))
    m = structured_dct_matrix(32)
    m[1::2, :16] = np.sign(m[1::2, :16]) * 127  # legal structure, but T leaves 16 bits
    m[1::2, 16:] = -m[1::2, 15::-1]
    bad.append(("T beyond 16 bits", 32, m, "limit"))
    return good, bad


def test_check_dct_matrix_accepts_structured_matrices(libvca):
    import numpy as np

    from oracle import int_dct2, int_dct2_butterfly
    good, _ = _matrix_cases()
    rng = np.random.default_rng(11)
    for name, n, m in good:
        for bd in (8, 10, 12):
            assert libvca.vca_check_dct_matrix(n, bd, m) == 0, (name, n, bd)
        # what acceptance promises: the butterfly and matrix forms agree
        x = rng.integers(0, 256, size=(8, n, n))
        assert np.array_equal(int_dct2_butterfly(x, 8, m), int_dct2(x, 8, False, m)), (name, n)


def test_check_dct_matrix_rejects_with_reasons(libvca):
    import numpy as np

    from oracle import int_dct2, int_dct2_butterfly
    _, bad = _matrix_cases()
    rng = np.random.default_rng(12)
    for name, n, m, reason in bad:
        with pytest.raises(libvca.VcaError) as ei:
            libvca.vca_check_dct_matrix(n, 8, m)
        assert ei.value.status == -1 and reason in str(ei.value), (name, str(ei.value))
        if reason == "symmetry":  # and the forms do disagree on some block
            x = rng.integers(0, 256, size=(16, n, n))
            assert not np.array_equal(int_dct2_butterfly(x, 8, m), int_dct2(x, 8, False, m)), name
    # the T bound binds only up to 10 bits (12-bit samples run on 32-bit integers)
    assert libvca.vca_check_dct_matrix(32, 12, bad[-1][2]) == 0
    m = np.full((6, 6), 64)
    with pytest.raises(libvca.VcaError):
        libvca.vca_check_dct_matrix(6, 8, m)


def test_batch_frame_refs_marshalling(libvca):
    # Batch.frame_refs builds the C tick argument on the host (no GPU involved): one entry per
    # analyzer, plane pointers and byte pitches from the tensors, zeros for a skipped channel, and
    # a length check so that the library never reads past the array.
    import torch

    vca = libvca
    batch = vca.Batch.__new__(vca.Batch)
    batch.analyzers = [object(), object()]
    batch.handle = None
    y8 = torch.zeros(2, 36, 64, dtype=torch.uint8)
    u8 = torch.zeros(2, 18, 48, dtype=torch.uint8)
    y16 = torch.zeros(2, 20, 32, dtype=torch.int16)
    u16 = torch.zeros(2, 10, 32, dtype=torch.int16)
    refs = batch.frame_refs([(y8[1], u8[1], u8[0]), (y16[0], u16[0], u16[1])])
    assert isinstance(refs, ctypes.Array) and len(refs) == 2
    assert (refs[0].y, refs[0].u, refs[0].v) == (y8[1].data_ptr(), u8[1].data_ptr(), u8[0].data_ptr())
    assert (refs[0].pitch_y, refs[0].pitch_uv) == (64, 48)
    assert (refs[1].pitch_y, refs[1].pitch_uv) == (64, 64)  # 16-bit samples: pitches in bytes
    skipped = batch.frame_refs([None, (y16[0], u16[0], u16[1])])
    assert skipped[0].y is None and skipped[0].pitch_y == 0
    with pytest.raises(ValueError):
        batch.frame_refs([(y8[0], u8[0], u8[1])])  # one frame for two analyzers
    with pytest.raises(ValueError):
        batch.frame_refs([(y8[0], u8[0], y16[0]), None])  # U and V pitches differ
    with pytest.raises(ValueError):
        batch.tick((vca.VcaFrameRef * 3)())  # a prepared argument of the wrong length
