"""ctypes binding of libirfnr.so (the C ABI in include/ir_filter.h).

Every ``ir_*`` function here has the name and argument order of its C
counterpart; this module only converts arguments (torch tensors or integer
device addresses, streams) and turns non-OK statuses into exceptions. All
filtering happens in the library's CUDA kernels. If the library cannot be
loaded the first call raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libirfnr.so")

IR_OK, IR_EINVAL, IR_EALIGN, IR_ENOMEM, IR_ECUDA, IR_ETIMEOUT, IR_EBUSY, IR_EUNSUPPORTED, IR_ECHECK = range(9)
IR_U8, IR_U16, IR_U14 = 0, 1, 2
IR_ALGO_AUTO, IR_ALGO_DENSE3, IR_ALGO_NETWORK, IR_ALGO_BITPLANE, IR_ALGO_DENSE = 0, 1, 2, 3, 4
IR_BORDER_REPLICATE, IR_BORDER_MIRROR, IR_BORDER_ZERO = 0, 1, 2
BORDER_CODES = {"replicate": IR_BORDER_REPLICATE, "mirror": IR_BORDER_MIRROR, "zero": IR_BORDER_ZERO}
IR_DETECT_EXTREME, IR_DETECT_DIRECTIONAL = 0, 1
DETECTOR_CODES = {"extreme": IR_DETECT_EXTREME, "directional": IR_DETECT_DIRECTIONAL}
ALGO_NAMES = {IR_ALGO_AUTO: "auto", IR_ALGO_DENSE3: "dense3", IR_ALGO_NETWORK: "network",
              IR_ALGO_BITPLANE: "bitplane", IR_ALGO_DENSE: "dense"}

EXPORTED = (
    "ir_filter_create", "ir_filter_destroy", "ir_filter_run", "ir_filter_run2", "ir_filter_run_batch",
    "ir_batch_plan_create", "ir_batch_plan_launch", "ir_batch_plan_kernel_count", "ir_batch_plan_destroy",
    "ir_filter_sync_status", "ir_filter_autotune", "ir_filter_get_config", "ir_filter_set_config",
    "ir_filter_launch_count", "ir_status_string", "ir_filter_last_error", "ir_filter_version",
    "ir_filter_run_noalloc", "ir_filter_noalloc_status", "ir_filter_median_filter", "ir_filter_run_passes", "ir_filter_set_border",
    "ir_filter_get_border", "ir_filter_set_tile_fit", "ir_filter_set_detector", "ir_filter_get_detector", "ir_filter_set_strict_alignment",
    "ir_filter_run_host", "ir_filter_autotune_batch",
    "ir_server_create", "ir_server_destroy", "ir_server_filter", "ir_server_open_stream", "ir_server_close_stream",
    "ir_server_submit", "ir_server_poll", "ir_server_wait_idle", "ir_server_output", "ir_server_read",
    "ir_server_release", "ir_server_get_stats", "ir_server_clock", "ir_server_drive",
)


class IrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class ir_kernel_config(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("algo", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int)]


class ir_frame_desc(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("in_pitch", ctypes.c_size_t), ("out_pitch", ctypes.c_size_t), ("dtype", ctypes.c_int),
                ("k", ctypes.c_int), ("flagged_count", ctypes.c_void_p)]


class ir_tune_result(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("k", ctypes.c_int), ("frames", ctypes.c_int), ("candidates", ctypes.c_int),
                ("chosen", ir_kernel_config), ("chosen_ms", ctypes.c_float), ("defaults", ir_kernel_config),
                ("default_ms", ctypes.c_float)]


class ir_server_config(ctypes.Structure):
    _fields_ = [("max_streams", ctypes.c_int), ("ring_depth", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("exec_streams", ctypes.c_int), ("hbm_reserve_bytes", ctypes.c_size_t), ("poll_us", ctypes.c_int)]


class ir_completion(ctypes.Structure):
    _fields_ = [("stream_id", ctypes.c_int), ("slot", ctypes.c_int), ("tag", ctypes.c_ulonglong),
                ("t_submit", ctypes.c_double), ("t_launch", ctypes.c_double), ("t_done", ctypes.c_double),
                ("batch_frames", ctypes.c_int), ("status", ctypes.c_int)]


class ir_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_ulonglong), ("completed", ctypes.c_ulonglong),
                ("rejected_busy", ctypes.c_ulonglong), ("batches", ctypes.c_ulonglong),
                ("frames_in_batches", ctypes.c_ulonglong), ("open_streams", ctypes.c_int),
                ("max_inflight", ctypes.c_int), ("device_bytes", ctypes.c_size_t)]


class ir_drive_result(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_ulonglong), ("megapixels", ctypes.c_double), ("seconds", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    """The library this process loads: ``libirfnr.so``, or the file named by
    the IRFNR_LIBRARY environment variable (e.g. the debug-check build)."""
    return os.environ.get("IRFNR_LIBRARY") or LIB_PATH


def load(path: Optional[str] = None):
    """Load libirfnr.so (built by ``__graft_entry__.build()`` or ``_build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or library_path()
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library {p} is not built; run paper_1201_3972_gb300._build.build()")
        lib = ctypes.CDLL(p)
        vp, i32, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        sig = {
            "ir_filter_create": ([ctypes.POINTER(vp), i32], i32),
            "ir_filter_destroy": ([vp], None),
            "ir_filter_run": ([vp, vp, i32, i32, sz, i32, i32, vp], i32),
            "ir_filter_run2": ([vp, vp, sz, vp, sz, i32, i32, i32, i32, vp, vp], i32),
            "ir_filter_run_batch": ([vp, ctypes.POINTER(ir_frame_desc), i32, vp], i32),
            "ir_filter_run_host": ([vp, ctypes.POINTER(ir_frame_desc), i32, i32, vp], i32),
            "ir_batch_plan_create": ([vp, ctypes.POINTER(ir_frame_desc), i32, ctypes.POINTER(vp)], i32),
            "ir_batch_plan_launch": ([vp, vp], i32),
            "ir_batch_plan_kernel_count": ([vp], i32),
            "ir_batch_plan_destroy": ([vp], None),
            "ir_filter_sync_status": ([vp], i32),
            "ir_filter_autotune": ([vp, i32, i32, i32, i32, vp], i32),
            "ir_filter_autotune_batch": ([vp, ctypes.POINTER(ir_frame_desc), i32, i32, vp,
                                          ctypes.POINTER(ir_tune_result), i32, ctypes.POINTER(i32)], i32),
            "ir_filter_get_config": ([vp, i32, i32, ctypes.POINTER(ir_kernel_config)], i32),
            "ir_filter_set_config": ([vp, i32, i32, ctypes.POINTER(ir_kernel_config)], i32),
            "ir_filter_launch_count": ([vp], ctypes.c_ulonglong),
            "ir_status_string": ([i32], ctypes.c_char_p),
            "ir_filter_last_error": ([vp], ctypes.c_char_p),
            "ir_filter_version": ([], ctypes.c_char_p),
            "ir_filter_run_noalloc": ([vp, i32, i32, sz, i32, i32, vp], i32),
            "ir_filter_noalloc_status": ([], i32),
            "ir_filter_median_filter": ([vp, vp, sz, vp, sz, i32, i32, i32, i32, vp, vp], i32),
            "ir_filter_set_border": ([vp, i32], i32),
            "ir_filter_get_border": ([vp], i32),
            "ir_filter_set_detector": ([vp, i32], i32),
            "ir_filter_get_detector": ([vp], i32),
            "ir_filter_set_strict_alignment": ([vp, i32], i32),
            "ir_filter_set_tile_fit": ([vp, i32], i32),
            "ir_filter_run_passes": ([vp, vp, sz, vp, sz, i32, i32, i32, i32, i32, vp, vp], i32),
            "ir_server_create": ([i32, ctypes.POINTER(ir_server_config), ctypes.POINTER(vp)], i32),
            "ir_server_destroy": ([vp], None),
            "ir_server_filter": ([vp], vp),
            "ir_server_open_stream": ([vp, i32, i32, i32, i32, ctypes.POINTER(i32)], i32),
            "ir_server_close_stream": ([vp, i32], i32),
            "ir_server_submit": ([vp, i32, vp, sz, ctypes.c_ulonglong, ctypes.POINTER(i32)], i32),
            "ir_server_poll": ([vp, ctypes.POINTER(ir_completion), i32], i32),
            "ir_server_wait_idle": ([vp, ctypes.c_double], i32),
            "ir_server_output": ([vp, i32, i32, ctypes.POINTER(vp), ctypes.POINTER(sz)], i32),
            "ir_server_read": ([vp, i32, i32, vp, sz], i32),
            "ir_server_release": ([vp, i32, i32], i32),
            "ir_server_get_stats": ([vp, ctypes.POINTER(ir_server_stats)], i32),
            "ir_server_clock": ([], ctypes.c_double),
            "ir_server_drive": ([vp, ctypes.POINTER(i32), ctypes.POINTER(vp), ctypes.POINTER(sz), i32,
                                 ctypes.c_double, i32, i32, ctypes.POINTER(ir_drive_result)], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(lib, h, status: int) -> None:
    if status != IR_OK:
        msg = lib.ir_filter_last_error(h)
        raise IrError(status, (msg or b"").decode() or lib.ir_status_string(status).decode())


def _ptr(x) -> int:
    """Device address of a torch tensor, or an integer address as is."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def dtype_code(t, u14: bool = False) -> int:
    import torch
    if t.dtype == torch.uint8:
        return IR_U8
    if t.dtype in (torch.uint16, torch.int16):
        return IR_U14 if u14 else IR_U16
    raise TypeError(f"unsupported tensor dtype {t.dtype}: use uint8 or uint16")


def _frame_geometry(t):
    """(H, W, pitch_bytes) of a 2-D tensor with contiguous rows."""
    if t.dim() != 2:
        raise ValueError("frames are 2-D (H, W) tensors")
    if t.stride(1) != 1:
        raise ValueError("frame rows must be contiguous")
    H, W = t.shape
    pitch = t.stride(0) * t.element_size() if H > 1 else W * t.element_size()
    return int(H), int(W), int(pitch)


class Filter:
    """One library handle (``ir_filter``) on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        st = self.lib.ir_filter_create(ctypes.byref(h), int(device))
        _check(self.lib, None, st)
        self.h = h
        self.device = device

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.ir_filter_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- single frames ------------------------------------------------------
    def ir_filter_run(self, frame, H: int, W: int, pitch: int, dtype: int, k: int, stream=None) -> None:
        _check(self.lib, self.h, self.lib.ir_filter_run(self.h, _ptr(frame), H, W, pitch, dtype, k, _stream(stream)))

    def ir_filter_run2(self, src, in_pitch: int, dst, out_pitch: int, H: int, W: int, dtype: int, k: int,
                       stream=None, flagged_count=None) -> None:
        _check(self.lib, self.h, self.lib.ir_filter_run2(self.h, _ptr(src), in_pitch, _ptr(dst), out_pitch, H, W,
                                                         dtype, k, _stream(stream), _ptr(flagged_count) or None))

    def ir_filter_median_filter(self, src, in_pitch: int, dst, out_pitch: int, H: int, W: int, dtype: int, k: int,
                                stream=None, median_count=None) -> None:
        _check(self.lib, self.h, self.lib.ir_filter_median_filter(self.h, _ptr(src), in_pitch, _ptr(dst), out_pitch,
                                                                  H, W, dtype, k, _stream(stream),
                                                                  _ptr(median_count) or None))

    def ir_filter_run_passes(self, src, in_pitch: int, dst, out_pitch: int, H: int, W: int, dtype: int, k: int,
                             passes: int, stream=None, flagged_per_pass=None) -> None:
        _check(self.lib, self.h, self.lib.ir_filter_run_passes(self.h, _ptr(src), in_pitch, _ptr(dst), out_pitch, H,
                                                               W, dtype, k, passes, _stream(stream),
                                                               _ptr(flagged_per_pass) or None))

    def set_border(self, border) -> None:
        """Border reading for later calls: "replicate" (default), "mirror" or "zero"."""
        code = BORDER_CODES[border] if isinstance(border, str) else int(border)
        _check(self.lib, self.h, self.lib.ir_filter_set_border(self.h, code))

    def get_border(self) -> int:
        return int(self.lib.ir_filter_get_border(self.h))

    def set_detector(self, detector) -> None:
        """Noise detector for later calls: "extreme" (Eq. 3a/3b, default) or
        "directional" (Fig. 1)."""
        code = DETECTOR_CODES[detector] if isinstance(detector, str) else int(detector)
        _check(self.lib, self.h, self.lib.ir_filter_set_detector(self.h, code))

    def get_detector(self) -> int:
        return int(self.lib.ir_filter_get_detector(self.h))

    def set_tile_fit(self, on: bool) -> None:
        """Shrink the tile of launches that cannot fill the GPU (default on)."""
        _check(self.lib, self.h, self.lib.ir_filter_set_tile_fit(self.h, 1 if on else 0))

    def set_strict_alignment(self, on: bool) -> None:
        """Refuse (IR_EALIGN) frames whose base or pitch is not 16-byte aligned
        instead of staging them with plain loads."""
        _check(self.lib, self.h, self.lib.ir_filter_set_strict_alignment(self.h, 1 if on else 0))

    def median_filter(self, src, dst, k: int, u14: bool = False, stream=None, median_count=None) -> None:
        """Standard median filter (every pixel), the paper's MF baseline."""
        H, W, ip = _frame_geometry(src)
        _, _, op = _frame_geometry(dst)
        self.ir_filter_median_filter(src, ip, dst, op, H, W, dtype_code(src, u14), k, stream, median_count)

    def run_passes(self, src, dst, k: int, passes: int, u14: bool = False, stream=None, flagged_per_pass=None):
        """Iterative FNR: `passes` passes, the last written to dst."""
        H, W, ip = _frame_geometry(src)
        _, _, op = _frame_geometry(dst)
        self.ir_filter_run_passes(src, ip, dst, op, H, W, dtype_code(src, u14), k, passes, stream, flagged_per_pass)

    def run(self, frame, k: int, u14: bool = False, stream=None) -> None:
        """In-place filter of a 2-D uint8/uint16 CUDA tensor."""
        H, W, pitch = _frame_geometry(frame)
        self.ir_filter_run(frame, H, W, pitch, dtype_code(frame, u14), k, stream)

    def run2(self, src, dst, k: int, u14: bool = False, stream=None, flagged_count=None) -> None:
        """Out-of-place filter; ``flagged_count`` is an optional 1-element int64 CUDA tensor."""
        H, W, ip = _frame_geometry(src)
        H2, W2, op = _frame_geometry(dst)
        if (H, W) != (H2, W2) or src.dtype != dst.dtype:
            raise ValueError("src and dst must have the same shape and dtype")
        self.ir_filter_run2(src, ip, dst, op, H, W, dtype_code(src, u14), k, stream, flagged_count)

    # -- batches --------------------------------------------------------------
    @staticmethod
    def make_descs(frames):
        """frames: iterable of dicts with keys in, out, k and optional u14, flagged."""
        frames = list(frames)
        arr = (ir_frame_desc * len(frames))()
        for i, f in enumerate(frames):
            H, W, ip = _frame_geometry(f["in"])
            _, _, op = _frame_geometry(f["out"])
            arr[i].in_ = _ptr(f["in"])
            arr[i].out = _ptr(f["out"])
            arr[i].H, arr[i].W = H, W
            arr[i].in_pitch, arr[i].out_pitch = ip, op
            arr[i].dtype = dtype_code(f["in"], f.get("u14", False))
            arr[i].k = int(f["k"])
            arr[i].flagged_count = _ptr(f.get("flagged")) or None
        return arr

    def ir_filter_run_batch(self, descs, n: int, stream=None) -> None:
        _check(self.lib, self.h, self.lib.ir_filter_run_batch(self.h, descs, n, _stream(stream)))

    def ir_filter_run_host(self, descs, n: int, chunks: int = 0, stream=None) -> None:
        """Frames in host memory (descriptor in/out are host addresses)."""
        _check(self.lib, self.h, self.lib.ir_filter_run_host(self.h, descs, n, int(chunks), _stream(stream)))

    def run_batch(self, frames, stream=None) -> None:
        descs = self.make_descs(frames)
        self.ir_filter_run_batch(descs, len(descs), stream)

    def run_host(self, frames, chunks: int = 0, stream=None) -> None:
        """Frames in host memory: dicts as for ``run_batch`` whose ``in`` and
        ``out`` are CPU tensors (pinned for full speed); asynchronous on
        ``stream`` like every other call."""
        descs = self.make_descs(frames)
        self.ir_filter_run_host(descs, len(descs), chunks, stream)

    def plan(self, frames) -> "BatchPlan":
        descs = self.make_descs(frames)
        return BatchPlan(self, descs)

    # -- status, tuning ---------------------------------------------------------
    def ir_filter_sync_status(self) -> int:
        return self.lib.ir_filter_sync_status(self.h)

    def sync_status(self) -> None:
        _check(self.lib, self.h, self.ir_filter_sync_status())

    def launch_count(self) -> int:
        return int(self.lib.ir_filter_launch_count(self.h))

    def autotune(self, dtype: int, k: int, H: int, W: int, stream=None) -> None:
        _check(self.lib, self.h, self.lib.ir_filter_autotune(self.h, dtype, k, H, W, _stream(stream)))

    def autotune_batch(self, descs, reps: int = 20, stream=None) -> list:
        """Tune the table on these frames (an ``ir_frame_desc`` array, e.g. from
        ``make_descs``), class by class; returns one dict per (pixel size, k)
        class: the configuration chosen, its median ms, the default's, and the
        number of candidates timed."""
        out = (ir_tune_result * 64)()
        got = ctypes.c_int(0)
        _check(self.lib, self.h, self.lib.ir_filter_autotune_batch(self.h, descs, len(descs), int(reps),
                                                                   _stream(stream), out, 64, ctypes.byref(got)))

        def cfg(c):
            return {"tile_w": c.tile_w, "tile_h": c.tile_h, "algo": c.algo, "ctas_per_sm": c.ctas_per_sm}
        return [{"dtype": r.dtype, "k": r.k, "frames": r.frames, "candidates": r.candidates,
                 "chosen": cfg(r.chosen), "chosen_ms": float(r.chosen_ms), "defaults": cfg(r.defaults),
                 "default_ms": float(r.default_ms)} for r in out[:got.value]]

    def get_config(self, dtype: int, k: int) -> dict:
        c = ir_kernel_config()
        _check(self.lib, self.h, self.lib.ir_filter_get_config(self.h, dtype, k, ctypes.byref(c)))
        return {"tile_w": c.tile_w, "tile_h": c.tile_h, "algo": c.algo, "ctas_per_sm": c.ctas_per_sm}

    def set_config(self, dtype: int, k: int, tile_w: int, tile_h: int, algo: int, ctas_per_sm: int = 0) -> None:
        c = ir_kernel_config(tile_w, tile_h, algo, ctas_per_sm)
        _check(self.lib, self.h, self.lib.ir_filter_set_config(self.h, dtype, k, ctypes.byref(c)))

    # -- tuning table on disk -----------------------------------------------------
    def configs(self) -> dict:
        """The handle's (strategy, tile) table: {"<dtype>:<k>": config} for 8- and 16-bit pixels."""
        return {f"{dt}:{k}": self.get_config(dt, k) for dt in (IR_U8, IR_U16) for k in range(3, 22, 2)}

    def save_configs(self, path: str, device_name: str) -> None:
        """Store the table under ``device_name`` in a JSON file (other devices' tables are kept), e.g.
        after ``autotune`` runs, so that later processes on the same GPU model can reuse it."""
        import json
        import os
        table = {}
        if os.path.exists(path):
            with open(path) as fh:
                table = json.load(fh)
        table[device_name] = self.configs()
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)

    def load_configs(self, path: str, device_name: str) -> bool:
        """Apply the table stored under ``device_name``; False when the file or the entry is missing.
        An entry the library rejects raises IrError."""
        import json
        import os
        if not os.path.exists(path):
            return False
        with open(path) as fh:
            table = json.load(fh).get(device_name)
        if table is None:
            return False
        for key, c in table.items():
            dt, k = (int(v) for v in key.split(":"))
            self.set_config(dt, k, c["tile_w"], c["tile_h"], c["algo"], c.get("ctas_per_sm", 0))
        return True


class BatchPlan:
    """An uploaded descriptor set with its captured graph (``ir_batch_plan``)."""

    def __init__(self, flt: Filter, descs):
        self.flt = flt
        self.lib = flt.lib
        self.descs = descs
        p = ctypes.c_void_p()
        _check(self.lib, flt.h, self.lib.ir_batch_plan_create(flt.h, descs, len(descs), ctypes.byref(p)))
        self.p = p

    @property
    def kernel_count(self) -> int:
        return int(self.lib.ir_batch_plan_kernel_count(self.p))

    def launch(self, stream=None) -> None:
        _check(self.lib, self.flt.h, self.lib.ir_batch_plan_launch(self.p, _stream(stream)))

    def close(self) -> None:
        if getattr(self, "p", None):
            self.lib.ir_batch_plan_destroy(self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
