"""ctypes binding of libvca.so (include/vca.h), argument marshalling only.

Every function keeps the C name and forwards to the library; all analysis runs in the
library's CUDA kernels.  If the library has not been built, loading fails loudly: there
is no Python or CPU fallback.  ``Analyzer`` is a small convenience wrapper that passes
torch tensors' device pointers and the current torch stream.
"""

from __future__ import annotations

import ctypes
import os

from .build import LIB_PATH

VCA_OK = 0
VCA_E_ARG = -1
VCA_E_UNSUPPORTED = -2
VCA_E_NOMEM = -3
VCA_E_CUDA = -4
VCA_E_AGAIN = -5
VCA_E_TIMEOUT = -6
VCA_E_STATE = -7

VCA_PAD_REPLICATE = 0
VCA_PAD_SKIP = 1
VCA_LOWPASS_OFF = 0
VCA_LOWPASS_QUARTER = 1
VCA_LOWPASS_DOWNSAMPLE = 2
VCA_CHROMA_420 = 0
VCA_CHROMA_444 = 1
VCA_CHROMA_422 = 2
VCA_SERVE_SEGMENTS, VCA_SERVE_TICKS = 0, 1
VCA_KERNEL_AUTO = 0
VCA_KERNEL_PLAIN = 1
VCA_KERNEL_TC = 2

FEATURES = ("E_Y", "h", "L_Y", "E_U", "E_V", "L_U", "L_V")


class VcaConfig(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("bit_depth", ctypes.c_int32),
                ("block_size", ctypes.c_int32), ("low_pass", ctypes.c_int32), ("pad_mode", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("chroma_format", ctypes.c_int32)]


class VcaFrameFeatures(ctypes.Structure):
    _fields_ = [("frame", ctypes.c_int64)] + [(k, ctypes.c_double) for k in FEATURES]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k in FEATURES}


class VcaSequenceFeatures(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_int64)] + [(k, ctypes.c_double) for k in FEATURES]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k in FEATURES}
        d["frames"] = self.frames
        return d


class VcaFrameRef(ctypes.Structure):
    _fields_ = [("y", ctypes.c_void_p), ("u", ctypes.c_void_p), ("v", ctypes.c_void_p),
                ("pitch_y", ctypes.c_int64), ("pitch_uv", ctypes.c_int64)]


class VcaTuneEntry(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("bit_depth", ctypes.c_int32),
                ("block_size", ctypes.c_int32), ("low_pass", ctypes.c_int32), ("chroma_format", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("plain_warps", ctypes.c_int32), ("tc_ctas", ctypes.c_int32),
                ("ms_per_frame", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class VcaSegmentDone(ctypes.Structure):
    _fields_ = [("channel", ctypes.c_int32), ("status", ctypes.c_int32), ("tag", ctypes.c_uint64),
                ("first_frame", ctypes.c_int64), ("n_frames", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("submit_ns", ctypes.c_int64), ("ready_ns", ctypes.c_int64)]


class VcaServerStats(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_int64), ("frames", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64), ("used_bytes", ctypes.c_int64), ("channels", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class VcaSitiFeatures(ctypes.Structure):
    _fields_ = [("frame", ctypes.c_int64), ("SI", ctypes.c_double), ("TI", ctypes.c_double)]


class VcaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


_lib = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64

_PROTOS = {
    "vca_block_count": (ctypes.POINTER(VcaConfig), ctypes.POINTER(_I64), ctypes.POINTER(_I64)),
    "vca_open": (ctypes.POINTER(VcaConfig), _P, ctypes.POINTER(_P)),
    "vca_push_frame": (_P, _P, _P, _P, _I64, _I64, _I32),
    "vca_push_frames": (_P, _P, _P, _P, _I64, _I64, _I64, _I64, _I32, _I32),
    "vca_read_frame_features": (_P, _I64, _I32, ctypes.POINTER(VcaFrameFeatures)),
    "vca_read_sequence_features": (_P, ctypes.POINTER(VcaSequenceFeatures)),
    "vca_read_block_values": (_P, _I32, _P, _P, _P, _P, _P, _P),
    "vca_dump_coefficients": (_P, _P, _P, _P, _I64, _I64, _P, _P, _P),
    "vca_sync": (_P,),
    "vca_stream_join": (_P,),
    "vca_export_state": (_P, _P, ctypes.POINTER(ctypes.c_size_t)),
    "vca_import_state": (_P, _P, ctypes.c_size_t),
    "vca_frames_pushed": (_P, ctypes.POINTER(_I64)),
    "vca_launch_count": (_P, ctypes.POINTER(_I64)),
    "vca_kernel_in_use": (_P, ctypes.POINTER(_I32)),
    "vca_set_kernel_timing": (_P, _I32),
    "vca_read_kernel_timing": (_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)),
    "vca_close": (_P,),
    "vca_reduce_frames_noalloc": (_P, _I64, _I32, _I32, _P, _P, _P, _P),
    "vca_autotune": (ctypes.POINTER(VcaConfig), _P, _P, _P, _I64, _I64, _I64, _I64, _I32, _I32, _P,
                     ctypes.POINTER(VcaTuneEntry), _I32, ctypes.POINTER(_I32), ctypes.POINTER(VcaTuneEntry)),
    "vca_tune_set": (ctypes.POINTER(VcaTuneEntry),),
    "vca_tune_lookup": (ctypes.POINTER(VcaConfig), ctypes.POINTER(VcaTuneEntry)),
    "vca_tune_clear": (),
    "vca_tune_save": (ctypes.c_char_p,),
    "vca_tune_load": (ctypes.c_char_p,),
    "vca_batch_split_weight": (_P, ctypes.c_float),
    "vca_debug_wait": (_P, _I64, _I32),
    "vca_batch_debug_wait": (_P, _I64, _I32),
    "vca_batch_autotune": (_P, ctypes.POINTER(VcaFrameRef), _I32, ctypes.POINTER(ctypes.c_float),
                           ctypes.POINTER(ctypes.c_float)),
    "vca_batch_create": (ctypes.POINTER(_P), _I32, ctypes.POINTER(_P)),
    "vca_batch_tick": (_P, ctypes.POINTER(VcaFrameRef)),
    "vca_batch_sync": (_P,),
    "vca_batch_launch_count": (_P, ctypes.POINTER(_I64)),
    "vca_batch_kernel": (_P, ctypes.POINTER(_I32)),
    "vca_set_dct_matrix": (_P, _I32, _P),
    "vca_check_dct_matrix": (_I32, _I32, _P),
    "vca_batch_destroy": (_P,),
    "vca_server_create": (ctypes.c_size_t, ctypes.POINTER(_P)),
    "vca_server_set_policy": (_P, ctypes.c_int32),
    "vca_server_add_channel": (_P, ctypes.POINTER(VcaConfig), _I32, ctypes.POINTER(_I32)),
    "vca_server_segment_buffer": (_P, _I32, _I32, ctypes.POINTER(VcaFrameRef), ctypes.POINTER(_I64),
                                  ctypes.POINTER(_I64)),
    "vca_server_submit": (_P, _I32, _I32, _I32, ctypes.c_uint64, _P),
    "vca_server_submit_frames": (_P, _I32, ctypes.POINTER(VcaFrameRef), _I64, _I64, _I32, ctypes.c_uint64, _P),
    "vca_server_poll": (_P, ctypes.POINTER(VcaSegmentDone), _I32, ctypes.POINTER(_I32)),
    "vca_server_read_features": (_P, _I32, _I64, ctypes.POINTER(VcaFrameFeatures)),
    "vca_server_stats": (_P, ctypes.POINTER(VcaServerStats)),
    "vca_server_destroy": (_P,),
    "vca_siti_open": (_I32, _I32, _I32, _I32, _P, ctypes.POINTER(_P)),
    "vca_siti_push": (_P, _P, _I64, _I64, _I32, _I32),
    "vca_siti_read": (_P, _I64, ctypes.POINTER(VcaSitiFeatures)),
    "vca_siti_sequence": (_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)),
    "vca_siti_launch_count": (_P, ctypes.POINTER(_I64)),
    "vca_siti_close": (_P,),
}


def lib():
    """The loaded library; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libvca.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _PROTOS.items():
            fn = getattr(L, name)
            fn.argtypes = list(args)
            fn.restype = ctypes.c_int
        L.vca_status_str.argtypes = [ctypes.c_int]
        L.vca_status_str.restype = ctypes.c_char_p
        L.vca_last_error.argtypes = []
        L.vca_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_PROTOS) + ["vca_status_str", "vca_last_error"]


def _check(status: int) -> int:
    if status != VCA_OK:
        L = lib()
        raise VcaError(status, (L.vca_last_error() or b"").decode() or L.vca_status_str(status).decode())
    return status


def vca_status_str(status: int) -> str:
    return lib().vca_status_str(status).decode()


def vca_last_error() -> str:
    return lib().vca_last_error().decode()


def vca_block_count(cfg: VcaConfig) -> tuple[int, int]:
    bx, by = _I64(), _I64()
    _check(lib().vca_block_count(ctypes.byref(cfg), ctypes.byref(bx), ctypes.byref(by)))
    return bx.value, by.value


def vca_reduce_frames_noalloc(block_values: int, blocks_per_plane: int, block_size: int, n_frames: int,
                              prev_H_Y: int | None, last_H_Y: int, features: int, stream: int = 0) -> int:
    """Frame features from device block values with no device allocation (device pointers)."""
    return _check(lib().vca_reduce_frames_noalloc(_P(block_values), blocks_per_plane, block_size, n_frames,
                                                  _P(prev_H_Y or 0), _P(last_H_Y), _P(features), _P(stream)))


def _config(width, height, bit_depth=8, block_size=32, low_pass=False, chroma_format=0, kernel=0,
            max_batch=0) -> "VcaConfig":
    c = VcaConfig()
    c.width, c.height, c.bit_depth, c.block_size = width, height, bit_depth, block_size
    c.low_pass = {False: 0, True: 1, "downsample": 2}.get(low_pass, low_pass)
    c.chroma_format, c.kernel, c.max_batch = chroma_format, kernel, max_batch
    return c


def vca_autotune(cfg: "VcaConfig", y, u, v, reps: int = 3, stream: int = 0):
    """Tunes the launch shape of cfg on (F, H, pitch) device frame tensors; returns (chosen entry,
    list of measured candidates) as dicts.  The chosen shape becomes cfg's table entry."""
    es = y.element_size()
    n = y.shape[0]
    cands = (VcaTuneEntry * 16)()
    ncand = _I32()
    chosen = VcaTuneEntry()
    _check(lib().vca_autotune(ctypes.byref(cfg), _P(y.data_ptr()), _P(u.data_ptr()), _P(v.data_ptr()),
                              y.stride(-2) * es, u.stride(-2) * es, y.stride(0) * es, u.stride(0) * es, n, reps,
                              _P(stream), cands, 16, ctypes.byref(ncand), ctypes.byref(chosen)))
    return chosen.as_dict(), [cands[i].as_dict() for i in range(min(ncand.value, 16))]


def vca_tune_set(**entry) -> None:
    e = VcaTuneEntry()
    for k, val in entry.items():
        setattr(e, k, val)
    _check(lib().vca_tune_set(ctypes.byref(e)))


def vca_tune_lookup(cfg: "VcaConfig"):
    """The table entry of cfg's configuration as a dict, or None."""
    e = VcaTuneEntry()
    st = lib().vca_tune_lookup(ctypes.byref(cfg), ctypes.byref(e))
    if st == VCA_E_AGAIN:
        return None
    _check(st)
    return e.as_dict()


def vca_debug_wait(handle: int, wait_limit_ns: int, withhold_tile: int = -1) -> None:
    _check(lib().vca_debug_wait(_P(handle), wait_limit_ns, withhold_tile))


def vca_batch_debug_wait(handle: int, wait_limit_ns: int, withhold_tile: int = -1) -> None:
    _check(lib().vca_batch_debug_wait(_P(handle), wait_limit_ns, withhold_tile))


def vca_tune_clear() -> None:
    _check(lib().vca_tune_clear())


def vca_tune_save(path: str) -> None:
    _check(lib().vca_tune_save(os.fsencode(path)))


def vca_tune_load(path: str) -> None:
    _check(lib().vca_tune_load(os.fsencode(path)))


def vca_server_set_policy(server: int, policy: int) -> None:
    _check(lib().vca_server_set_policy(_P(server), policy))


def vca_batch_create(handles) -> int:
    arr = (_P * len(handles))(*handles)
    h = _P()
    _check(lib().vca_batch_create(arr, len(handles), ctypes.byref(h)))
    return h.value


def vca_batch_tick(batch: int, refs) -> None:
    """refs: one VcaFrameRef per member of the batch (a sequence or a ctypes array of them)."""
    arr = refs if isinstance(refs, ctypes.Array) else (VcaFrameRef * len(refs))(*refs)
    _check(lib().vca_batch_tick(_P(batch), arr))


def vca_batch_sync(batch: int) -> None:
    _check(lib().vca_batch_sync(_P(batch)))


def vca_batch_launch_count(batch: int) -> int:
    n = _I64()
    _check(lib().vca_batch_launch_count(_P(batch), ctypes.byref(n)))
    return n.value


def vca_batch_kernel(batch: int) -> int:
    k = _I32()
    _check(lib().vca_batch_kernel(_P(batch), ctypes.byref(k)))
    return k.value


def vca_batch_destroy(batch: int) -> None:
    _check(lib().vca_batch_destroy(_P(batch)))


def vca_open(cfg: VcaConfig, stream: int = 0) -> int:
    h = _P()
    _check(lib().vca_open(ctypes.byref(cfg), _P(stream), ctypes.byref(h)))
    return h.value


def vca_push_frame(a, y, u, v, pitch_y, pitch_uv, on_device=1):
    return _check(lib().vca_push_frame(a, y, u, v, pitch_y, pitch_uv, on_device))


def vca_push_frames(a, y, u, v, pitch_y, pitch_uv, frame_stride_y, frame_stride_uv, n_frames, on_device=1):
    return _check(lib().vca_push_frames(a, y, u, v, pitch_y, pitch_uv, frame_stride_y, frame_stride_uv,
                                        n_frames, on_device))


def vca_read_frame_features(a, frame: int, blocking: int = 1) -> VcaFrameFeatures:
    out = VcaFrameFeatures()
    _check(lib().vca_read_frame_features(a, frame, blocking, ctypes.byref(out)))
    return out


def vca_read_sequence_features(a) -> VcaSequenceFeatures:
    out = VcaSequenceFeatures()
    _check(lib().vca_read_sequence_features(a, ctypes.byref(out)))
    return out


def vca_read_block_values(a, index: int, H_Y=None, L_Y=None, H_U=None, L_U=None, H_V=None, L_V=None):
    return _check(lib().vca_read_block_values(a, index, H_Y, L_Y, H_U, L_U, H_V, L_V))


def vca_dump_coefficients(a, y, u, v, pitch_y, pitch_uv, zy, zu, zv):
    return _check(lib().vca_dump_coefficients(a, y, u, v, pitch_y, pitch_uv, zy, zu, zv))


def vca_sync(a):
    return _check(lib().vca_sync(a))


def vca_stream_join(a):
    return _check(lib().vca_stream_join(a))


def vca_export_state(a) -> bytes:
    n = ctypes.c_size_t(0)
    _check(lib().vca_export_state(a, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().vca_export_state(a, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def vca_import_state(a, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    return _check(lib().vca_import_state(a, buf, len(state)))


def _int8_matrix(n, matrix):
    import numpy as np

    m = np.ascontiguousarray(np.asarray(matrix), dtype=np.int8)
    if m.shape != (n, n):
        raise ValueError(f"matrix must be {n} x {n}")
    return m


def vca_set_dct_matrix(a, n: int, matrix) -> int:
    """Drop-in n x n integer DCT matrix (int8 values, row k = basis function k)."""
    m = _int8_matrix(n, matrix)
    return _check(lib().vca_set_dct_matrix(_P(a), n, m.ctypes.data))


def vca_check_dct_matrix(n: int, bit_depth: int, matrix) -> int:
    """VCA_OK if the matrix meets the drop-in requirements, else raises VcaError with the reason."""
    m = _int8_matrix(n, matrix)
    return _check(lib().vca_check_dct_matrix(n, bit_depth, m.ctypes.data))


def vca_frames_pushed(a) -> int:
    n = _I64()
    _check(lib().vca_frames_pushed(a, ctypes.byref(n)))
    return n.value


def vca_launch_count(a) -> int:
    n = _I64()
    _check(lib().vca_launch_count(a, ctypes.byref(n)))
    return n.value


def vca_kernel_in_use(a) -> int:
    k = _I32()
    _check(lib().vca_kernel_in_use(a, ctypes.byref(k)))
    return k.value


def vca_set_kernel_timing(a, enable: int):
    return _check(lib().vca_set_kernel_timing(a, int(enable)))


def vca_read_kernel_timing(a) -> tuple[float, int]:
    ms, n = ctypes.c_double(), _I64()
    _check(lib().vca_read_kernel_timing(a, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def vca_close(a):
    return _check(lib().vca_close(a))


class Analyzer:
    """One analyzer (one video) on the current CUDA device and torch stream.

    Frames are torch tensors: device tensors are read in place; CPU tensors are copied by
    the library.  Planes are indexed (frame, row, column-in-samples) and may have a row
    pitch larger than the width.
    """

    def __init__(self, width, height, bit_depth=8, block_size=32, low_pass=False, pad_mode=VCA_PAD_REPLICATE,
                 kernel=VCA_KERNEL_AUTO, max_batch=64, stream=None, chroma_format=VCA_CHROMA_420):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        lp = VCA_LOWPASS_DOWNSAMPLE if low_pass in ("downsample", VCA_LOWPASS_DOWNSAMPLE) else int(bool(low_pass))
        self.cfg = VcaConfig(width, height, bit_depth, block_size, lp, pad_mode, kernel, max_batch, chroma_format)
        self.handle = vca_open(self.cfg, stream)
        self.blocks_x, self.blocks_y = vca_block_count(self.cfg)
        self.C = self.blocks_x * self.blocks_y
        self.dct_matrices = {}  # transform size -> drop-in matrix set through set_dct_matrix

    def set_dct_matrix(self, n, matrix):
        """Replace the n x n integer DCT matrix (before the first push)."""
        import numpy as np

        vca_set_dct_matrix(self.handle, n, matrix)
        self.dct_matrices[n] = np.asarray(matrix, dtype=np.int64).copy()

    def close(self):
        if self.handle:
            vca_close(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _plane_args(t):
        es = t.element_size()
        pitch = t.stride(-2) * es
        fstride = t.stride(0) * es if t.dim() == 3 else 0
        return t.data_ptr(), pitch, fstride

    def push(self, y, u, v):
        """Push frames given as (F, H, pitch) / (F, H/2, pitch) tensors or one (H, pitch) frame each."""
        on_device = 1 if y.is_cuda else 0
        n = y.shape[0] if y.dim() == 3 else 1
        py, pitch_y, fy = self._plane_args(y)
        pu, pitch_uv, fu = self._plane_args(u)
        pv, pitch_v, fv = self._plane_args(v)
        if pitch_v != pitch_uv or fv != fu:
            raise ValueError("U and V planes must share pitch and frame stride")
        vca_push_frames(self.handle, py, pu, pv, pitch_y, pitch_uv, fy, fu, n, on_device)
        return n

    def frame_features(self, frame, blocking=True) -> dict:
        return vca_read_frame_features(self.handle, frame, int(blocking)).as_dict()

    def sequence_features(self) -> dict:
        return vca_read_sequence_features(self.handle).as_dict()

    def block_values(self, index=0) -> dict:
        import numpy as np

        out = {k: np.zeros(self.C, dtype=np.float32) for k in ("H_Y", "L_Y", "H_U", "L_U", "H_V", "L_V")}
        vca_read_block_values(self.handle, index, *(out[k].ctypes.data for k in ("H_Y", "L_Y", "H_U", "L_U", "H_V",
                                                                                  "L_V")))
        return out

    def dump_coefficients(self, y, u, v):
        """Quantised coefficients of one device frame: dict plane -> int16 tensor (C, Nk, Nk)."""
        import torch

        w = self.cfg.block_size
        nk_y = w // 2 if self.cfg.low_pass else w  # quarter: N/2 coefficients; downsample: w/2 blocks
        nk_c = nk_y if self.cfg.chroma_format == VCA_CHROMA_444 else nk_y // 2
        nkv_c = nk_y if self.cfg.chroma_format == VCA_CHROMA_422 else nk_c  # 4:2:2: w rows, w/2 columns
        zy = torch.empty((self.C, nk_y, nk_y), dtype=torch.int16, device=y.device)
        zu = torch.empty((self.C, nkv_c, nk_c), dtype=torch.int16, device=y.device)
        zv = torch.empty_like(zu)
        py, pitch_y, _ = self._plane_args(y)
        pu, pitch_uv, _ = self._plane_args(u)
        pv, _, _ = self._plane_args(v)
        vca_dump_coefficients(self.handle, py, pu, pv, pitch_y, pitch_uv, zy.data_ptr(), zu.data_ptr(), zv.data_ptr())
        vca_sync(self.handle)
        return {"Y": zy, "U": zu, "V": zv}

    def sync(self):
        vca_sync(self.handle)

    def export_state(self) -> bytes:
        return vca_export_state(self.handle)

    def import_state(self, state: bytes):
        vca_import_state(self.handle, state)

    @property
    def frames_pushed(self) -> int:
        return vca_frames_pushed(self.handle)

    @property
    def launches(self) -> int:
        return vca_launch_count(self.handle)

    @property
    def kernel(self) -> int:
        return vca_kernel_in_use(self.handle)


class Batch:
    """Analyzers ticked together: one frame per analyzer per tick, replayed from a CUDA graph (on
    tensor cores one launch per sample size, the frame reduction inside)."""

    def __init__(self, analyzers):
        self.analyzers = list(analyzers)
        self.handle = vca_batch_create([a.handle for a in self.analyzers])

    def frame_refs(self, frames):
        """The tick argument for frames (as for tick), built once.  A caller that ticks from a ring
        of resident frame buffers can keep one per ring slot and pass it to tick unchanged."""
        if len(frames) != len(self.analyzers):
            raise ValueError(f"one frame (or None) per analyzer: {len(self.analyzers)} expected, got {len(frames)}")
        refs = (VcaFrameRef * len(frames))()
        for i, f in enumerate(frames):
            if f is None:
                continue
            y, u, v = f
            es = y.element_size()
            if u.stride(-2) != v.stride(-2):
                raise ValueError("U and V planes must share a pitch")
            refs[i] = VcaFrameRef(y.data_ptr(), u.data_ptr(), v.data_ptr(), y.stride(-2) * es, u.stride(-2) * es)
        return refs

    def tick(self, frames):
        """frames: one (y, u, v) device-tensor triple per analyzer (one frame each), or None to
        skip it; or the result of frame_refs."""
        if not isinstance(frames, ctypes.Array):
            frames = self.frame_refs(frames)
        elif len(frames) != len(self.analyzers) or frames._type_ is not VcaFrameRef:
            raise ValueError("a prepared tick argument must come from this batch's frame_refs")
        vca_batch_tick(self.handle, frames)

    def sync(self):
        vca_batch_sync(self.handle)

    def set_split_weight(self, weight: float) -> None:
        _check(lib().vca_batch_split_weight(_P(self.handle), ctypes.c_float(weight)))

    def autotune(self, frames, reps: int = 20):
        """Tunes the SM split of this batch's ticks on frames (as for tick); returns (weight, ms per tick)."""
        if not isinstance(frames, ctypes.Array):
            frames = self.frame_refs(frames)
        w, ms = ctypes.c_float(), ctypes.c_float()
        _check(lib().vca_batch_autotune(_P(self.handle), frames, reps, ctypes.byref(w), ctypes.byref(ms)))
        return w.value, ms.value

    def launches(self) -> int:
        return vca_batch_launch_count(self.handle)

    @property
    def kernel(self) -> int:
        return vca_batch_kernel(self.handle)

    def close(self):
        if self.handle:
            vca_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving runtime: live channels, segment submission, continuous batching on a native
    scheduler thread, admission by a device-memory budget."""

    def __init__(self, device_budget_bytes=0, policy=None):
        h = _P()
        _check(lib().vca_server_create(device_budget_bytes, ctypes.byref(h)))
        self.handle = h.value
        if policy is not None:
            _check(lib().vca_server_set_policy(_P(self.handle), policy))

    def add_channel(self, width, height, bit_depth=8, block_size=32, low_pass=True, max_segment_frames=120,
                    pad_mode=VCA_PAD_REPLICATE, chroma_format=VCA_CHROMA_420) -> int:
        cfg = VcaConfig(width, height, bit_depth, block_size, int(bool(low_pass)), pad_mode, VCA_KERNEL_AUTO, 1,
                        chroma_format)
        cid = _I32()
        _check(lib().vca_server_add_channel(_P(self.handle), ctypes.byref(cfg), max_segment_frames, ctypes.byref(cid)))
        return cid.value

    def submit_frames(self, channel, y, u, v, tag=0) -> int:
        """Copies (F, H, pitch) / (F, H/2, pitch) frames into a free slot and queues them (tag: the
        caller's number for the segment).
        Returns VCA_OK, or VCA_E_AGAIN when both slots of the channel are busy."""
        es = y.element_size()
        if u.stride(0) != v.stride(0) or u.stride(-2) != v.stride(-2):
            raise ValueError("U and V planes must share pitch and frame stride")
        ref = VcaFrameRef(y.data_ptr(), u.data_ptr(), v.data_ptr(), y.stride(-2) * es, u.stride(-2) * es)
        st = lib().vca_server_submit_frames(_P(self.handle), channel, ctypes.byref(ref), y.stride(0) * es,
                                            u.stride(0) * es, y.shape[0], tag, None)
        if st == VCA_E_AGAIN:
            return st
        return _check(st)

    def poll(self, max_items=256):
        arr = (VcaSegmentDone * max_items)()
        n = _I32()
        _check(lib().vca_server_poll(_P(self.handle), arr, max_items, ctypes.byref(n)))
        return [{"channel": d.channel, "status": d.status, "tag": d.tag, "first_frame": d.first_frame,
                 "n_frames": d.n_frames, "submit_ns": d.submit_ns, "ready_ns": d.ready_ns} for d in arr[:n.value]]

    def frame_features(self, channel, frame) -> dict:
        out = VcaFrameFeatures()
        _check(lib().vca_server_read_features(_P(self.handle), channel, frame, ctypes.byref(out)))
        return out.as_dict()

    def stats(self) -> dict:
        st = VcaServerStats()
        _check(lib().vca_server_stats(_P(self.handle), ctypes.byref(st)))
        return {k: getattr(st, k) for k in ("ticks", "frames", "launches", "budget_bytes", "used_bytes", "channels")}

    def close(self):
        if self.handle:
            _check(lib().vca_server_destroy(_P(self.handle)))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Siti:
    """SI / TI of a luma sequence (the paper's comparison features) on the current CUDA stream."""

    def __init__(self, width, height, bit_depth=8, max_batch=64, stream=None):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        h = _P()
        _check(lib().vca_siti_open(width, height, bit_depth, max_batch, _P(stream), ctypes.byref(h)))
        self.handle = h.value
        self.frames = 0

    def push(self, y):
        """(F, H, pitch) or (H, pitch) luma tensor, on the device or the host."""
        es = y.element_size()
        n = y.shape[0] if y.dim() == 3 else 1
        fs = y.stride(0) * es if y.dim() == 3 else 0
        _check(lib().vca_siti_push(_P(self.handle), _P(y.data_ptr()), y.stride(-2) * es, fs, n, 1 if y.is_cuda else 0))
        self.frames += n
        return n

    def frame_features(self, frame) -> dict:
        out = VcaSitiFeatures()
        _check(lib().vca_siti_read(_P(self.handle), frame, ctypes.byref(out)))
        return {"SI": out.SI, "TI": out.TI}

    def sequence_features(self) -> dict:
        si, ti, n = ctypes.c_double(), ctypes.c_double(), _I64()
        _check(lib().vca_siti_sequence(_P(self.handle), ctypes.byref(si), ctypes.byref(ti), ctypes.byref(n)))
        return {"SI": si.value, "TI": ti.value, "frames": n.value}

    def launches(self) -> int:
        n = _I64()
        _check(lib().vca_siti_launch_count(_P(self.handle), ctypes.byref(n)))
        return n.value

    def close(self):
        if self.handle:
            _check(lib().vca_siti_close(_P(self.handle)))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
