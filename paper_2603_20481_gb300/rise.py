"""Python binding of the RISE C ABI (include/rise.h): argument marshalling only.

Every step of the detection path runs in the CUDA library `_lib/librise.so`;
this module converts torch tensors / numpy arrays to pointers and sizes and
boxes back to arrays.  There is no fallback: if the library is missing the
first use raises.  PyTorch provides device memory and the current stream.

Boxes are returned as int64 arrays of shape (n, 8) with columns
(t0, t1, f0, f1, anchor, area, sum_q, energy_fx) in anchor order.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# RISE_CHECKED=1 selects the checked build (device index checks; see build.py)
LIB_PATH = (os.path.join(HERE, "_lib_checked", "librise_checked.so") if os.environ.get("RISE_CHECKED") == "1"
            else os.path.join(HERE, "_lib", "librise.so"))

RISE_OK, RISE_EINVAL, RISE_ENOMEM, RISE_ETRUNC = 0, -1, -2, -3
RISE_ECUDA, RISE_ETIMEOUT, RISE_EINTERNAL, RISE_ESCRATCH, RISE_EAGAIN = -4, -5, -6, -7, -8
NOALLOC_MAX_COLS = 4096
RANGE_AUTO_MAX, RANGE_FIXED = 0, 1
DBG_POWER_F32, DBG_IMAGE_U8, DBG_HIST, DBG_COLSTATS, DBG_FLOOR = 1, 2, 3, 4, 5
DBG_MASK0, DBG_MASK1, DBG_MASK2, DBG_MASK3, DBG_MAXPOW, DBG_LEVEL_EDGES = 6, 7, 8, 9, 10, 11
DBG_LAUNCHES, DBG_BATCH_INFO, DBG_GRAPHS, DBG_CCL = 12, 13, 14, 15
DBG_BATCH_IMAGES, DBG_BATCH_POWER, DBG_BATCH_ANCHORS = 16, 17, 18
STAGES = ("spectrum_pass1", "spectrum_pass2", "histogram", "column_stats", "morphology",
          "labelling", "readback", "total")
OPT_KEEP_POWER, OPT_KEEP_MASKS, OPT_TIMING, OPT_RANGE_PATH = 1, 2, 3, 4
OPT_GRAPH, OPT_AUTOTUNE, OPT_RUN_CAPACITY = 5, 6, 7
OPT_SCAN_WAIT_LIMIT, OPT_UNION_LIMIT, OPT_TEST_WITHHOLD, OPT_FFT_SCHEDULE = 8, 9, 10, 11
OPT_COPY_WAIT_LIMIT, OPT_TEST_WITHHOLD_COPY, OPT_BLOCKING_WAIT = 12, 13, 14
IQ_HOST, IQ_SC16 = 1, 2
OPT_BATCH_GRAPH = OPT_GRAPH
BATCH_MAX_ROWS = 524280
BOX_COLS = ("t0", "t1", "f0", "f1", "anchor", "area", "sum_q", "energy_fx")

# Functions the header declares; the ABI test checks the library exports them.
EXPORTS = ("rise_thresholds_default", "rise_create", "rise_destroy", "rise_strerror", "rise_boxes_widen",
           "rise_detect", "rise_detect_host", "rise_detect_image", "rise_debug_export",
           "rise_set_option", "rise_stage_times", "rise_column_stats_noalloc",
           "rise_detect_batch", "rise_submit", "rise_collect", "rise_match_boxes", "rise_contours",
           "rise_server_create", "rise_stream_submit", "rise_server_poll",
           "rise_server_drain", "rise_stream_export", "rise_stream_import", "rise_server_stats",
           "rise_server_result_image", "rise_server_destroy")


class RiseError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class Config(C.Structure):
    _fields_ = [("device", C.c_int), ("cuda_stream", C.c_void_p), ("max_samples", C.c_int64),
                ("max_fft", C.c_int), ("max_boxes", C.c_int64), ("mem_budget", C.c_size_t)]


class Thresholds(C.Structure):
    _fields_ = [("range_mode", C.c_int), ("hi_db", C.c_double), ("level_db", C.c_double),
                ("psd_offset_db", C.c_double), ("power_offset_db", C.c_double),
                ("sg_half_window", C.c_int), ("morph_order", C.c_int)]


class Capture(C.Structure):
    _fields_ = [("iq_dev", C.c_void_p), ("n", C.c_int64), ("fft_size", C.c_int), ("hop", C.c_int)]


class ServerConfig(C.Structure):
    _fields_ = [("device", C.c_int), ("fft_size", C.c_int), ("hop", C.c_int),
                ("max_chunk", C.c_int64), ("max_streams", C.c_int), ("lanes", C.c_int),
                ("max_batch", C.c_int), ("max_pending", C.c_int), ("mem_budget", C.c_size_t),
                ("thr", C.c_void_p), ("window_frames", C.c_int64), ("keep_images", C.c_int),
                ("spin_wait", C.c_int)]


class Result(C.Structure):
    _fields_ = [("stream", C.c_int), ("status", C.c_int), ("tag", C.c_uint64), ("seq", C.c_int64),
                ("first_frame", C.c_int64), ("frames", C.c_int64), ("box_offset", C.c_int64),
                ("n_boxes", C.c_int64), ("t_submit_ns", C.c_int64), ("t_start_ns", C.c_int64),
                ("t_done_ns", C.c_int64)]


class Box(C.Structure):
    _fields_ = [("t0", C.c_int32), ("t1", C.c_int32), ("f0", C.c_int32), ("f1", C.c_int32),
                ("anchor", C.c_int64), ("area", C.c_int64), ("sum_q", C.c_uint64),
                ("energy_fx", C.c_uint64)]


BOX_DTYPE = np.dtype([("t0", "<i4"), ("t1", "<i4"), ("f0", "<i4"), ("f1", "<i4"),
                      ("anchor", "<i8"), ("area", "<i8"), ("sum_q", "<u8"), ("energy_fx", "<u8")])
COLSTAT_DTYPE = np.dtype([("S", "<u8"), ("Shat", "<i8"), ("keep", "<i4"), ("otsu", "<i4"),
                          ("eff", "<i4"), ("pad", "<i4")])
assert C.sizeof(Box) == BOX_DTYPE.itemsize == 48

_lib = None


def lib() -> C.CDLL:
    """Load librise.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"RISE CUDA library not built: {LIB_PATH} is missing "
                           "(run paper_2603_20481_gb300/build.py)")
    L = C.CDLL(LIB_PATH)
    P, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    L.rise_thresholds_default.argtypes = [P]
    L.rise_thresholds_default.restype = None
    L.rise_create.argtypes = [C.POINTER(P), P]
    L.rise_create.restype = i32
    L.rise_destroy.argtypes = [P]
    L.rise_destroy.restype = None
    L.rise_strerror.argtypes = [i32]
    L.rise_strerror.restype = C.c_char_p
    L.rise_boxes_widen.argtypes = [P, i64, P]
    L.rise_boxes_widen.restype = None
    for name in ("rise_detect", "rise_detect_host"):
        f = getattr(L, name)
        f.argtypes = [P, P, i64, i32, i32, P, P, i64, P]
        f.restype = i32
    L.rise_detect_image.argtypes = [P, P, i64, i32, P, P, i64, P]
    L.rise_detect_image.restype = i32
    L.rise_debug_export.argtypes = [P, i32, P, C.c_size_t]
    L.rise_debug_export.restype = i32
    L.rise_set_option.argtypes = [P, i32, i64]
    L.rise_set_option.restype = i32
    L.rise_stage_times.argtypes = [P, P, i32]
    L.rise_stage_times.restype = i32
    L.rise_submit.argtypes = [P, P, i32, i64, i32, i32, P, i64]
    L.rise_submit.restype = i32
    L.rise_collect.argtypes = [P, P, i64, C.POINTER(i64)]
    L.rise_collect.restype = i32
    L.rise_contours.argtypes = [P, P, i64, C.POINTER(i64), P]
    L.rise_contours.restype = i32
    L.rise_match_boxes.argtypes = [P, P, i64, P, i64, P, i32, P, P, P, P]
    L.rise_match_boxes.restype = i32
    L.rise_detect_batch.argtypes = [P, P, i32, P, P, i64, P]
    L.rise_detect_batch.restype = i32
    L.rise_server_create.argtypes = [C.POINTER(P), P]
    L.rise_server_create.restype = i32
    L.rise_stream_submit.argtypes = [P, i32, P, i64, C.c_uint64]
    L.rise_stream_submit.restype = i32
    L.rise_server_poll.argtypes = [P, P, i32, P, i64, C.POINTER(i32), i32]
    L.rise_server_poll.restype = i32
    L.rise_server_drain.argtypes = [P, i32]
    L.rise_server_drain.restype = i32
    L.rise_stream_export.argtypes = [P, i32, P, C.c_size_t, C.POINTER(C.c_size_t)]
    L.rise_stream_export.restype = i32
    L.rise_stream_import.argtypes = [P, i32, P, C.c_size_t]
    L.rise_stream_import.restype = i32
    L.rise_server_stats.argtypes = [P, P, i32]
    L.rise_server_stats.restype = i32
    L.rise_server_result_image.argtypes = [P, i32, i64, P, C.c_size_t, C.POINTER(i64)]
    L.rise_server_result_image.restype = i32
    L.rise_server_destroy.argtypes = [P]
    L.rise_server_destroy.restype = None
    L.rise_column_stats_noalloc.argtypes = [P, i64, i32, P, P]
    L.rise_column_stats_noalloc.restype = i32
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return lib().rise_strerror(code).decode()
    except Exception:
        return "unknown"


def default_thresholds(**overrides) -> Thresholds:
    t = Thresholds()
    lib().rise_thresholds_default(C.byref(t))
    for k, v in overrides.items():
        setattr(t, k, v)
    return t


def boxes_from_raw(raw: np.ndarray, n: int) -> np.ndarray:
    """rise_box[n] -> int64 (n, 8): the four int32 fields, then the four 64-bit ones
    (sum_q and energy_fx stay below 2^63)."""
    out = np.empty((n, 8), np.int64)
    if n:
        lib().rise_boxes_widen(raw.ctypes.data, n, out.ctypes.data)
    return out


class Detector:
    """One library context bound to a device and a CUDA stream.

    By default the context gets a stream of its own (a torch.cuda.Stream);
    every call first makes that stream wait for the caller's current torch
    stream, so inputs produced by torch kernels are complete before the
    library reads them.
    """

    def __init__(self, device: int = 0, stream=None, mem_budget: int = 0,
                 max_boxes: int = 0, max_samples: int = 0):
        import torch
        self._torch = torch
        if stream is None:
            stream = torch.cuda.Stream(device)
        cfg = Config(device, C.c_void_p(stream.cuda_stream), max_samples, 0, max_boxes, mem_budget)
        h = C.c_void_p()
        rc = lib().rise_create(C.byref(h), C.byref(cfg))
        if rc != RISE_OK:
            raise RiseError(rc, "rise_create")
        self._h = h
        self.device = device
        self.stream = stream
        self._ev = torch.cuda.Event()
        self.cap = 1 << 16
        self._batch_caps = {}   # capture tables of recent batch calls, by their tensors

    def close(self):
        if getattr(self, "_h", None):
            lib().rise_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _order(self):
        cur = self._torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self._ev.record(cur)
            self.stream.wait_event(self._ev)

    # -- options ----------------------------------------------------------------
    def set_option(self, option: int, value: int):
        rc = lib().rise_set_option(self._h, option, int(value))
        if rc != RISE_OK:
            raise RiseError(rc, "rise_set_option")

    def stage_times(self) -> np.ndarray:
        ms = np.zeros(8, np.float32)
        lib().rise_stage_times(self._h, ms.ctypes.data, 8)
        return ms

    def launches(self) -> int:
        v = np.zeros(1, np.int64)
        rc = lib().rise_debug_export(self._h, DBG_LAUNCHES, v.ctypes.data, 8)
        if rc != RISE_OK:
            raise RiseError(rc, "rise_debug_export")
        return int(v[0])

    # -- detection --------------------------------------------------------------
    def _raw(self, cap: int) -> np.ndarray:
        buf = getattr(self, "_rawbuf", None)
        if buf is None or buf.shape[0] < cap:
            buf = np.empty(max(cap, 1), BOX_DTYPE)
            self._rawbuf = buf
        return buf

    def _run(self, fn, args, cap):
        cap = self.cap if cap is None else int(cap)
        while True:
            raw = self._raw(max(cap, 1))
            n = C.c_int64(0)
            rc = fn(*args, raw.ctypes.data if cap > 0 else None, cap, C.byref(n))
            if rc == RISE_ETRUNC and self._auto_grow:
                cap = int(n.value)
                self.cap = max(self.cap, cap)
                continue
            if rc not in (RISE_OK, RISE_ETRUNC):
                raise RiseError(rc, fn.__name__)
            self.last_status = rc
            return boxes_from_raw(raw, min(int(n.value), cap))

    _auto_grow = True

    def detect(self, iq, fft_size: int, hop: int, thr: Optional[Thresholds] = None,
               cap: Optional[int] = None) -> np.ndarray:
        """Boxes of one capture.  `iq`: CUDA complex64 tensor (1-D, contiguous)."""
        t = self._torch
        if not (isinstance(iq, t.Tensor) and iq.is_cuda and iq.dtype == t.complex64
                and iq.is_contiguous() and iq.dim() == 1):
            raise TypeError("iq must be a contiguous 1-D CUDA complex64 tensor")
        args = (self._h, C.c_void_p(iq.data_ptr()), iq.numel(), fft_size, hop,
                C.byref(thr) if thr is not None else None)
        self._order()
        return self._run(lib().rise_detect, args, cap)

    def detect_host(self, iq, fft_size: int, hop: int, thr: Optional[Thresholds] = None,
                    cap: Optional[int] = None) -> np.ndarray:
        """Boxes of one capture held in host memory (pinned tensor or numpy array)."""
        t = self._torch
        if isinstance(iq, t.Tensor):
            if iq.is_cuda or iq.dtype != t.complex64 or not iq.is_contiguous():
                raise TypeError("iq must be a contiguous host complex64 tensor")
            ptr, n = iq.data_ptr(), iq.numel()
        else:
            iq = np.ascontiguousarray(iq, dtype=np.complex64)
            ptr, n = iq.ctypes.data, iq.shape[0]
        args = (self._h, C.c_void_p(ptr), n, fft_size, hop,
                C.byref(thr) if thr is not None else None)
        self._order()
        return self._run(lib().rise_detect_host, args, cap)

    def contours(self, T: int, F: int, boundary: bool = True):
        """Shapes of the last call's blocks (rise_contours): runs int32 (n, 4) =
        box index, row, first, last column, in raster order; and the boundary
        mask unpacked to uint8 [T, F] (or None)."""
        n = C.c_int64(0)
        rc = lib().rise_contours(self._h, None, 0, C.byref(n), None)
        if rc not in (RISE_OK, RISE_ETRUNC):
            raise RiseError(rc, "rise_contours")
        runs = np.zeros((max(int(n.value), 1), 4), np.int32)
        words = np.zeros((T, F // 32), np.uint32) if boundary else None
        rc = lib().rise_contours(self._h, runs.ctypes.data, runs.shape[0], C.byref(n),
                                 words.ctypes.data if boundary else None)
        if rc != RISE_OK:
            raise RiseError(rc, "rise_contours")
        return runs[: int(n.value)], (unpack_mask(words, F) if boundary else None)

    def match(self, gt, det, thetas):
        """Detection quality on the GPU (rise_match_boxes): gt and det are
        arrays whose first four columns are t0, t1, f0, f1 (e.g. detect's
        output).  Returns n_t, n_f, p_d, p_fa per threshold and the best
        (intersection, union) pair of every box."""
        g = np.ascontiguousarray(np.asarray(gt)[:, :4], dtype=np.int32).reshape(-1, 4)
        d4 = np.asarray(det)[:, :4].reshape(-1, 4)
        d = np.zeros(d4.shape[0], BOX_DTYPE)
        for j, name in enumerate(("t0", "t1", "f0", "f1")):
            d[name] = d4[:, j]
        th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).reshape(-1))
        nt = np.zeros(th.shape[0], np.int64)
        nf = np.zeros(th.shape[0], np.int64)
        gb = np.zeros((g.shape[0], 2), np.int64)
        db = np.zeros((d.shape[0], 2), np.int64)
        rc = lib().rise_match_boxes(self._h, g.ctypes.data, g.shape[0], d.ctypes.data, d.shape[0],
                                    th.ctypes.data, th.shape[0], nt.ctypes.data, nf.ctypes.data,
                                    gb.ctypes.data, db.ctypes.data)
        if rc != RISE_OK:
            raise RiseError(rc, "rise_match_boxes")
        return {"n_t": nt, "n_f": nf, "gt_best": gb, "det_best": db,
                "p_d": nt / max(1, g.shape[0]), "p_fa": nf / max(1, d.shape[0])}

    # -- asynchronous calls ---------------------------------------------------
    def submit(self, iq, fft_size: int, hop: int, thr: Optional[Thresholds] = None,
               cap: Optional[int] = None):
        """Queues a capture (rise_submit), kept referenced until collected: a
        complex64 tensor or array (1-D), or 16-bit integer I/Q (sc16) as an
        int16 tensor or array of shape (n, 2); CUDA tensors are read in place,
        host ones (pinned tensors copy fastest) are copied in."""
        t = self._torch
        flags = 0
        if isinstance(iq, t.Tensor):
            if not iq.is_contiguous():
                raise TypeError("iq must be contiguous")
            if iq.dtype == t.int16 and iq.dim() == 2 and iq.shape[1] == 2:
                flags |= IQ_SC16
                n = iq.shape[0]
            elif iq.dtype == t.complex64 and iq.dim() == 1:
                n = iq.numel()
            else:
                raise TypeError("iq must be complex64 [n] or int16 [n, 2]")
            ptr = iq.data_ptr()
            if not iq.is_cuda:
                flags |= IQ_HOST
        else:
            iq = np.ascontiguousarray(iq)
            if iq.dtype == np.int16 and iq.ndim == 2 and iq.shape[1] == 2:
                flags |= IQ_SC16
            elif iq.dtype != np.complex64 or iq.ndim != 1:
                iq = np.ascontiguousarray(iq, dtype=np.complex64)
            ptr, n = iq.ctypes.data, iq.shape[0]
            flags |= IQ_HOST
        cap = self.cap if cap is None else int(cap)
        self._order()
        rc = lib().rise_submit(self._h, C.c_void_p(ptr), flags, n, fft_size, hop,
                               C.byref(thr) if thr is not None else None, cap)
        if rc != RISE_OK:
            raise RiseError(rc, "rise_submit")
        self._queued = getattr(self, "_queued", []) + [(iq, cap)]

    def collect(self) -> np.ndarray:
        """Boxes of the oldest queued call (rise_collect)."""
        _, cap = self._queued[0]
        raw = self._raw(max(cap, 1))
        n = C.c_int64(0)
        rc = lib().rise_collect(self._h, raw.ctypes.data, cap, C.byref(n))
        self._queued = self._queued[1:]
        if rc not in (RISE_OK, RISE_ETRUNC):
            raise RiseError(rc, "rise_collect")
        self.last_status = rc
        return boxes_from_raw(raw, min(int(n.value), cap))

    def detect_image(self, img, thr: Optional[Thresholds] = None,
                     cap: Optional[int] = None) -> np.ndarray:
        """Boxes of a given 8-bit image: CUDA uint8 tensor [T, F], contiguous."""
        t = self._torch
        if not (isinstance(img, t.Tensor) and img.is_cuda and img.dtype == t.uint8
                and img.is_contiguous() and img.dim() == 2):
            raise TypeError("img must be a contiguous 2-D CUDA uint8 tensor")
        T, F = img.shape
        args = (self._h, C.c_void_p(img.data_ptr()), T, F,
                C.byref(thr) if thr is not None else None)
        self._order()
        return self._run(lib().rise_detect_image, args, cap)

    def detect_batch(self, iqs, fft_sizes, hops, thr: Optional[Thresholds] = None,
                     cap: Optional[int] = None):
        """Boxes of many captures in one call (rise_detect_batch).

        `iqs`: list of contiguous 1-D CUDA complex64 tensors; `fft_sizes`,
        `hops`: one int each, or a list per capture.  Returns (boxes, offsets):
        boxes (total, 8) as for detect, capture c's rows being
        boxes[offsets[c]:offsets[c+1]].
        """
        t = self._torch
        k = len(iqs)
        if isinstance(fft_sizes, int):
            fft_sizes = [fft_sizes] * k
        if isinstance(hops, int):
            hops = [hops] * k
        # a recent call's capture table is reused when the same tensors (same
        # objects, storage, size and type) come again
        key = (tuple((id(x), x.data_ptr(), x.numel(), x.dtype) for x in iqs),
               tuple(fft_sizes), tuple(hops))
        caps = self._batch_caps.get(key)
        if caps is None:
            caps = (Capture * max(k, 1))()
            for i, x in enumerate(iqs):
                if not (isinstance(x, t.Tensor) and x.is_cuda and x.dtype == t.complex64
                        and x.is_contiguous() and x.dim() == 1):
                    raise TypeError("each capture must be a contiguous 1-D CUDA complex64 tensor")
                caps[i] = Capture(x.data_ptr(), x.numel(), int(fft_sizes[i]), int(hops[i]))
            if len(self._batch_caps) >= 4:
                self._batch_caps.pop(next(iter(self._batch_caps)))
            self._batch_caps[key] = caps
        offs = np.zeros(k + 1, np.int64)
        cap = self.cap if cap is None else int(cap)
        self._order()
        while True:
            raw = self._raw(max(cap, 1))
            rc = lib().rise_detect_batch(self._h, C.byref(caps), k,
                                         C.byref(thr) if thr is not None else None,
                                         raw.ctypes.data if cap > 0 else None, cap,
                                         offs.ctypes.data)
            if rc == RISE_ETRUNC and self._auto_grow:
                cap = int(offs[k])
                self.cap = max(self.cap, cap)
                continue
            if rc not in (RISE_OK, RISE_ETRUNC):
                raise RiseError(rc, "rise_detect_batch")
            self.last_status = rc
            return boxes_from_raw(raw, min(int(offs[k]), cap)), offs

    def graph_info(self) -> np.ndarray:
        v = np.zeros(4, np.int64)
        rc = lib().rise_debug_export(self._h, DBG_GRAPHS, v.ctypes.data, v.nbytes)
        if rc != RISE_OK:
            raise RiseError(rc, "rise_debug_export")
        return v

    def batch_info(self) -> np.ndarray:
        """The last batch's launch parameters (RISE_DBG_BATCH_INFO, int64[64])."""
        v = np.zeros(64, np.int64)
        rc = lib().rise_debug_export(self._h, DBG_BATCH_INFO, v.ctypes.data, v.nbytes)
        if rc != RISE_OK:
            raise RiseError(rc, "rise_debug_export")
        return v

    def batch_debug(self, shapes, what: int = DBG_BATCH_IMAGES):
        """Intermediates of the last detect_batch call: the captures' 8-bit
        images (DBG_BATCH_IMAGES) or float |X|^2 (DBG_BATCH_POWER) as a list of
        [T_c, F_c] arrays, given `shapes` = [(T_c, F_c), ...] in call order;
        DBG_BATCH_ANCHORS gives the float32 anchor power of every capture."""
        if what == DBG_BATCH_ANCHORS:
            out = np.zeros(len(shapes), np.float32)
        else:
            dt = np.float32 if what == DBG_BATCH_POWER else np.uint8
            out = np.zeros(sum(int(T) * int(F) for T, F in shapes), dt)
        rc = lib().rise_debug_export(self._h, what, out.ctypes.data, out.nbytes)
        if rc != RISE_OK:
            raise RiseError(rc, "rise_debug_export")
        if what == DBG_BATCH_ANCHORS:
            return out
        res, at = [], 0
        for T, F in shapes:
            res.append(out[at:at + int(T) * int(F)].reshape(int(T), int(F)))
            at += int(T) * int(F)
        return res

    # -- introspection ----------------------------------------------------------
    def debug(self, what: int, T: int, F: int) -> np.ndarray:
        shapes = {
            DBG_POWER_F32: ((T, F), np.float32), DBG_IMAGE_U8: ((T, F), np.uint8),
            DBG_HIST: ((F, 256), np.uint32), DBG_FLOOR: ((8,), np.int64), DBG_CCL: ((4,), np.int64),
            DBG_MASK0: ((T, F // 32), np.uint32), DBG_MASK1: ((T, F // 32), np.uint32),
            DBG_MASK2: ((T, F // 32), np.uint32), DBG_MASK3: ((T, F // 32), np.uint32),
            DBG_MAXPOW: ((1,), np.float32), DBG_LEVEL_EDGES: ((257,), np.float32),
        }
        if what == DBG_COLSTATS:
            out = np.zeros(F, COLSTAT_DTYPE)
        else:
            shape, dt = shapes[what]
            out = np.zeros(shape, dt)
        rc = lib().rise_debug_export(self._h, what, out.ctypes.data, out.nbytes)
        if rc != RISE_OK:
            raise RiseError(rc, "rise_debug_export")
        return out


def column_stats_noalloc(img, cols, stream=None) -> int:
    """Allocation-free column statistics (rise_column_stats_noalloc).

    `img`: contiguous 2-D CUDA uint8 tensor [T, F]; `cols`: CUDA tensor of at
    least F * 32 bytes (rise_colstat[F]) on the same device, which receives S
    and the Otsu threshold of every column.  Work is queued on `stream` (the
    current torch stream by default) and not waited for.  Returns the status
    code; the caller decides what to do with a non-zero one.
    """
    import torch
    if not (isinstance(img, torch.Tensor) and img.is_cuda and img.dtype == torch.uint8
            and img.is_contiguous() and img.dim() == 2):
        raise TypeError("img must be a contiguous 2-D CUDA uint8 tensor")
    if not (isinstance(cols, torch.Tensor) and cols.is_cuda and cols.is_contiguous()):
        raise TypeError("cols must be a contiguous CUDA tensor")
    if cols.numel() * cols.element_size() < img.shape[1] * COLSTAT_DTYPE.itemsize:
        raise ValueError("cols is smaller than rise_colstat[F]")
    if stream is None:
        stream = torch.cuda.current_stream(img.device)
    return int(lib().rise_column_stats_noalloc(C.c_void_p(img.data_ptr()), img.shape[0],
                                               img.shape[1], C.c_void_p(cols.data_ptr()),
                                               C.c_void_p(stream.cuda_stream)))


SERVER_STATS = ("submitted", "rejected", "completed", "batches", "largest_batch",
                "most_in_flight", "slots", "lanes", "graph_captures", "buffer_generations",
                "longest_batch_us", "relabels")


class Server:
    """Continuous-batching server over chunks from many radio streams
    (rise_server_*).  Host buffers passed to submit are kept referenced here
    until their result has been polled, as the library requires."""

    def __init__(self, fft_size: int, hop: int, max_chunk: int, max_streams: int,
                 device: int = 0, lanes: int = 0, max_batch: int = 0, max_pending: int = 0,
                 mem_budget: int = 0, thr: Optional[Thresholds] = None, window_frames: int = 0,
                 keep_images: bool = False, spin_wait: bool = False):
        self._thr = thr
        self.window = window_frames
        self.fft_size = fft_size
        cfg = ServerConfig(device, fft_size, hop, max_chunk, max_streams, lanes, max_batch,
                           max_pending, mem_budget,
                           C.cast(C.pointer(thr), C.c_void_p) if thr is not None else None,
                           window_frames, int(bool(keep_images)), int(bool(spin_wait)))
        h = C.c_void_p()
        rc = lib().rise_server_create(C.byref(h), C.byref(cfg))
        if rc != RISE_OK:
            raise RiseError(rc, "rise_server_create")
        self._h = h
        self._held = {}                 # (stream, seq) -> host buffer
        self._seq = [0] * max_streams
        self._arena = np.empty(1 << 16, BOX_DTYPE)
        self._res = (Result * 1024)()

    def result_image(self, stream: int, seq: int) -> np.ndarray:
        """The 8-bit image result (stream, seq) was detected on (servers made
        with keep_images=True), [T, fft_size] uint8; taken out of the server."""
        T = C.c_int64(0)
        rc = lib().rise_server_result_image(self._h, stream, seq, None, 0, C.byref(T))
        if rc != RISE_OK:
            raise RiseError(rc, "rise_server_result_image")
        out = np.zeros((int(T.value), self.fft_size), np.uint8)
        rc = lib().rise_server_result_image(self._h, stream, seq, out.ctypes.data, out.nbytes, C.byref(T))
        if rc != RISE_OK:
            raise RiseError(rc, "rise_server_result_image")
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().rise_server_destroy(self._h)
            self._h = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, stream: int, iq, tag: int = 0) -> bool:
        """Queues a chunk; False when the queue is full (RISE_EAGAIN)."""
        import torch
        if isinstance(iq, torch.Tensor):
            if iq.is_cuda or iq.dtype != torch.complex64 or not iq.is_contiguous():
                raise TypeError("iq must be a contiguous host complex64 tensor")
            ptr, n = iq.data_ptr(), iq.numel()
        else:
            if not (isinstance(iq, np.ndarray) and iq.dtype == np.complex64 and iq.flags.c_contiguous):
                raise TypeError("iq must be a contiguous complex64 array")
            ptr, n = iq.ctypes.data, iq.shape[0]
        rc = lib().rise_stream_submit(self._h, stream, C.c_void_p(ptr), n, tag)
        if rc == RISE_EAGAIN:
            return False
        if rc != RISE_OK:
            raise RiseError(rc, "rise_stream_submit")
        self._held[(stream, self._seq[stream])] = iq
        self._seq[stream] += 1
        return True

    def poll(self, timeout_ms: int = 0, max_results: int = 1024):
        """Finished chunks: list of (result fields dict, boxes (n, 8) int64).
        A result with more boxes than the host arena comes back alone with
        status RISE_ETRUNC and the arena's worth of boxes; the arena is then
        doubled for later polls."""
        n = C.c_int(0)
        rc = lib().rise_server_poll(self._h, self._res, min(max_results, 1024),
                                    self._arena.ctypes.data, self._arena.shape[0],
                                    C.byref(n), timeout_ms)
        if rc != RISE_OK:
            raise RiseError(rc, "rise_server_poll")
        out = []
        for i in range(n.value):
            r = self._res[i]
            d = {f[0]: getattr(r, f[0]) for f in Result._fields_}
            b = self._arena[r.box_offset:r.box_offset + r.n_boxes]
            out.append((d, boxes_from_raw(b, r.n_boxes)))
            if not self.window:   # window mode: results are per plot; buffers go at drain()
                self._held.pop((r.stream, r.seq), None)
        if n.value == 1 and self._res[0].status == RISE_ETRUNC:
            self._arena = np.empty(2 * self._arena.shape[0], BOX_DTYPE)
        return out

    def drain(self, timeout_ms: int = -1):
        rc = lib().rise_server_drain(self._h, timeout_ms)
        if rc != RISE_OK:
            raise RiseError(rc, "rise_server_drain")
        if self.window:
            self._held.clear()

    def export_stream(self, stream: int) -> bytes:
        need = C.c_size_t(0)
        rc = lib().rise_stream_export(self._h, stream, None, 0, C.byref(need))
        if rc != RISE_OK:
            raise RiseError(rc, "rise_stream_export")
        buf = (C.c_char * need.value)()
        rc = lib().rise_stream_export(self._h, stream, buf, need.value, C.byref(need))
        if rc != RISE_OK:
            raise RiseError(rc, "rise_stream_export")
        return bytes(buf)

    def import_stream(self, stream: int, state: bytes):
        rc = lib().rise_stream_import(self._h, stream, state, len(state))
        if rc != RISE_OK:
            raise RiseError(rc, "rise_stream_import")
        self._seq[stream] = int(np.frombuffer(state[24:32], np.int64)[0])

    def stats(self) -> dict:
        v = np.zeros(len(SERVER_STATS), np.int64)
        lib().rise_server_stats(self._h, v.ctypes.data, len(SERVER_STATS))
        return dict(zip(SERVER_STATS, (int(x) for x in v)))


def unpack_mask(words: np.ndarray, F: int) -> np.ndarray:
    """[T, F/32] uint32 bit-packed mask (bit f%32 of word f/32) -> [T, F] uint8."""
    b = np.unpackbits(words.view(np.uint8).reshape(words.shape[0], -1), axis=1, bitorder="little")
    return b[:, :F]
