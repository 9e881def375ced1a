"""Python binding of libbf.so, the GB300 plane-wave receive beamformer.

Argument marshalling only: every step of the beamforming path (ingest,
delays, interpolation, combiners, compounding, envelope, log compression)
runs in the library's CUDA kernels.  The functions keep the C names
(``bf_create``, ``bf_beamform``, ``bf_submit``, ``bf_poll``, ...).  Data
arguments may be numpy arrays (host memory) or torch tensors (host or CUDA);
PyTorch only provides device memory and streams.

There is no fallback: if libbf.so is missing or fails to load, importing the
binding's functions raises.  Build it with ``python -m paper_2311_00482_gb300.build``
(or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

BF_DAS, BF_DMAS, BF_CF, BF_PDAS, BF_MODE_MASK = 1, 2, 4, 8, 15
BF_IQDAS, BF_BBDMAS, BF_IQ_MASK = 1 << 12, 1 << 13, 3 << 12
BF_FK_STOLT = 1 << 16
BF_DEST_ONE_BUFFER = 1 << 17
BF_PREC_FP32, BF_PREC_FP16, BF_PREC_BF16, BF_PREC_MASK = 0, 1 << 4, 2 << 4, 3 << 4
BF_OUT_RF, BF_OUT_ENV, BF_OUT_LOGDB, BF_OUT_MASK = 0, 1 << 8, 2 << 8, 3 << 8
BF_OK, BF_PENDING = 0, 1
BF_EINVAL, BF_EAGAIN, BF_ENOMEM, BF_ECUDA, BF_ETIMEDOUT, BF_ENOTFOUND, BF_ENOSYS = (
    -1, -2, -3, -4, -5, -6, -7)
_NAMES = {-1: "BF_EINVAL", -2: "BF_EAGAIN", -3: "BF_ENOMEM", -4: "BF_ECUDA", -5: "BF_ETIMEDOUT",
          -6: "BF_ENOTFOUND", -7: "BF_ENOSYS"}

EXPORTED = ("bf_create", "bf_destroy", "bf_set_stream", "bf_set_pdas_order", "bf_output_bytes",
            "bf_beamform",
            "bf_beamform_plain", "bf_fkmig",
            "bf_submit", "bf_poll", "bf_submit_many", "bf_submit_many_into", "bf_poll_many", "bf_ticket_batch", "bf_ticket_times", "bf_engine_pause",
            "bf_engine_configure", "bf_sync",
            "bf_batch_create", "bf_batch_launch", "bf_batch_status", "bf_batch_timing",
            "bf_batch_destroy",
            "bf_host_tables", "bf_plan_info", "bf_autotune", "bf_logdb_static", "bf_selftest_wait",
            "bf_last_error", "bf_version")


class BFError(RuntimeError):
    def __init__(self, code, message):
        super().__init__("%s (%d): %s" % (_NAMES.get(code, "BF_?"), code, message))
        self.code = code


class bf_geometry(ctypes.Structure):
    _fields_ = [("n_elements", ctypes.c_int32), ("pitch_m", ctypes.c_double),
                ("x_elem_m", ctypes.POINTER(ctypes.c_double)), ("f_number", ctypes.c_double)]


class bf_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("nz", ctypes.c_int32), ("x0_m", ctypes.c_double),
                ("x1_m", ctypes.c_double), ("z0_m", ctypes.c_double), ("z1_m", ctypes.c_double)]


class bf_frame(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("rf_dev", ctypes.c_void_p), ("n_samples", ctypes.c_int32),
                ("angles_rad", ctypes.POINTER(ctypes.c_double)), ("n_angles", ctypes.c_int32),
                ("mode_and_flags", ctypes.c_uint32), ("out_dev", ctypes.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libbf.so (raises OSError if it is missing or does not load)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise OSError("libbf.so not built at %s (run paper_2311_00482_gb300.build.build())" % path)
    lib = ctypes.CDLL(path)
    vp, i32, u32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "bf_create": ([ctypes.POINTER(bf_geometry), ctypes.POINTER(bf_grid), ctypes.c_double,
                       ctypes.c_double, ctypes.c_double, ctypes.POINTER(vp)], ctypes.c_int),
        "bf_destroy": ([vp], ctypes.c_int),
        "bf_set_stream": ([vp, vp], ctypes.c_int),
        "bf_set_pdas_order": ([vp, ctypes.c_double], ctypes.c_int),
        "bf_output_bytes": ([vp, u32], ctypes.c_size_t),
        "bf_beamform": ([vp, vp, i32, dp, i32, u32, vp], ctypes.c_int),
        "bf_beamform_plain": ([vp, vp, i32, dp, i32, u32, vp], ctypes.c_int),
        "bf_fkmig": ([vp, vp, i32, dp, i32, u32, vp], ctypes.c_int),
        "bf_submit": ([vp, vp, i32, dp, i32, u32, ctypes.POINTER(u64)], ctypes.c_int),
        "bf_poll": ([vp, u64, vp, ctypes.c_size_t, i64], ctypes.c_int),
        "bf_submit_many": ([vp, i32, ctypes.POINTER(vp), i32, dp, i32, u32, ctypes.POINTER(u64),
                            ctypes.POINTER(i32)], ctypes.c_int),
        "bf_submit_many_into": ([vp, i32, ctypes.POINTER(vp), i32, dp, i32, u32, ctypes.POINTER(vp),
                                 ctypes.c_size_t, ctypes.POINTER(u64), ctypes.POINTER(i32)],
                                ctypes.c_int),
        "bf_poll_many": ([vp, i32, ctypes.POINTER(u64), ctypes.POINTER(vp), ctypes.c_size_t, i64],
                         ctypes.c_int),
        "bf_ticket_batch": ([vp, u64, ctypes.POINTER(i32), ctypes.POINTER(i32)], ctypes.c_int),
        "bf_engine_configure": ([i32, i32, u64], ctypes.c_int),
        "bf_engine_pause": ([i32], ctypes.c_int),
        "bf_ticket_times": ([vp, u64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                            ctypes.c_int),
        "bf_sync": ([vp], ctypes.c_int),
        "bf_batch_create": ([ctypes.POINTER(bf_frame), i32, ctypes.POINTER(vp)], ctypes.c_int),
        "bf_batch_launch": ([vp, vp], ctypes.c_int),
        "bf_batch_status": ([vp, vp], ctypes.c_int),
        "bf_batch_destroy": ([vp], ctypes.c_int),
        "bf_batch_timing": ([vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32)], ctypes.c_int),
        "bf_host_tables": ([ctypes.POINTER(bf_geometry), ctypes.POINTER(bf_grid), ctypes.c_double,
                            ctypes.c_double, ctypes.c_double, i32, dp, i32, vp, vp], ctypes.c_int),
        "bf_plan_info": ([vp, i32, dp, i32, u32, vp, vp, ctypes.c_size_t], ctypes.c_int),
        "bf_autotune": ([vp, i32, dp, i32, u32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                         ctypes.POINTER(ctypes.c_float), i32], ctypes.c_int),
        "bf_logdb_static": ([vp, i32, i32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, i32, vp, vp], ctypes.c_int),
        "bf_selftest_wait": ([i64], ctypes.c_int),
        "bf_last_error": ([], ctypes.c_char_p),
        "bf_version": ([], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def bf_last_error() -> str:
    return load().bf_last_error().decode()


def _check(code, allow=(BF_OK,)):
    if code in allow:
        return code
    raise BFError(code, bf_last_error())


def _ptr(x):
    """Raw address of a numpy array or torch tensor (must be contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    return int(x)


def _nbytes(x):
    """Bytes of a numpy array or torch tensor."""
    return x.nbytes


def _angles(angles):
    a = np.ascontiguousarray(np.atleast_1d(np.asarray(angles, dtype=np.float64)))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def bf_create(n_elements, pitch_m, f_number, grid, fs_hz, f0_hz, c_mps, x_elem_m=None):
    """grid = (nx, nz, x0, x1, z0, z1); returns an opaque handle (int)."""
    xe = None
    g = bf_geometry(int(n_elements), float(pitch_m), None, float(f_number))
    if x_elem_m is not None:
        xe = np.ascontiguousarray(x_elem_m, dtype=np.float64)
        g.x_elem_m = xe.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    nx, nz, x0, x1, z0, z1 = grid
    gr = bf_grid(int(nx), int(nz), float(x0), float(x1), float(z0), float(z1))
    h = ctypes.c_void_p()
    _check(load().bf_create(ctypes.byref(g), ctypes.byref(gr), float(fs_hz), float(f0_hz),
                            float(c_mps), ctypes.byref(h)))
    return h.value


def bf_host_tables(n_elements, pitch_m, f_number, grid, fs_hz, f0_hz, c_mps, n_samples, angles_rad,
                   x_elem_m=None):
    """Host-only decision tables: (valid_rows [A][nx][N][2] int32, aperture_count [nx][nz])."""
    g = bf_geometry(int(n_elements), float(pitch_m), None, float(f_number))
    xe = None
    if x_elem_m is not None:
        xe = np.ascontiguousarray(x_elem_m, dtype=np.float64)
        g.x_elem_m = xe.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    nx, nz, x0, x1, z0, z1 = grid
    gr = bf_grid(int(nx), int(nz), float(x0), float(x1), float(z0), float(z1))
    a, ap = _angles(angles_rad)
    valid = np.zeros((len(a), int(nx), int(n_elements), 2), np.int32)
    cnt = np.zeros((int(nx), int(nz)), np.uint16)
    _check(load().bf_host_tables(ctypes.byref(g), ctypes.byref(gr), float(fs_hz), float(f0_hz),
                                 float(c_mps), int(n_samples), ap, len(a), valid.ctypes.data,
                                 cnt.ctypes.data))
    return valid, cnt


def bf_destroy(h):
    return _check(load().bf_destroy(h))


def bf_set_stream(h, stream=None):
    """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    s = getattr(stream, "cuda_stream", stream)
    return _check(load().bf_set_stream(h, s))


def bf_set_pdas_order(h, p):
    """Order p of the handle's pDAS combiner (Eq. (2)-(3)), 1 <= p <= 16."""
    return _check(load().bf_set_pdas_order(h, float(p)))


def bf_output_bytes(h, flags) -> int:
    return int(load().bf_output_bytes(h, int(flags)))


def bf_beamform(h, rf_dev, n_samples, angles_rad, flags, out_dev):
    a, ap = _angles(angles_rad)
    return _check(load().bf_beamform(h, _ptr(rf_dev), int(n_samples), ap, len(a), int(flags),
                                     _ptr(out_dev)))


def bf_beamform_plain(h, rf_dev, n_samples, angles_rad, flags, out_dev):
    a, ap = _angles(angles_rad)
    return _check(load().bf_beamform_plain(h, _ptr(rf_dev), int(n_samples), ap, len(a), int(flags),
                                           _ptr(out_dev)))


def bf_fkmig(h, rf_dev, n_samples, angles_rad, flags, out_dev):
    """Plane-wave f-k migration onto the native grid [n_elements][n_samples] (see include/bf.h)."""
    a, ap = _angles(angles_rad)
    return _check(load().bf_fkmig(h, _ptr(rf_dev), int(n_samples), ap, len(a), int(flags),
                                  _ptr(out_dev)))


def bf_plan_info(h, n_samples, angles_rad, flags, with_windows=False):
    """Plan description dict; with_windows adds the [A][tiles][N] window table."""
    a, ap = _angles(angles_rad)
    info = np.zeros(8, np.int32)
    _check(load().bf_plan_info(h, int(n_samples), ap, len(a), int(flags), info.ctypes.data, None, 0))
    keys = ("wmax", "box", "group", "rows", "tiles_x", "tiles_z", "nsp", "entries")
    d = {k: int(v) for k, v in zip(keys, info)}
    if with_windows:
        w = np.zeros(d["entries"], np.int32)
        _check(load().bf_plan_info(h, int(n_samples), ap, len(a), int(flags), info.ctypes.data,
                                   w.ctypes.data, w.size))
        d["windows"] = w.reshape(len(a), d["tiles_x"] * d["tiles_z"], -1)
    return d


def bf_autotune(h, n_samples, angles_rad, flags, frames=8):
    """Pick the fastest tile configuration for this workload (kept by the handle).
    Returns {"rows", "stage_bytes", "candidates_us"}."""
    a, ap = _angles(angles_rad)
    rows, stage = ctypes.c_int32(), ctypes.c_int32()
    cand = (ctypes.c_float * 8)()
    _check(load().bf_autotune(h, int(n_samples), ap, len(a), int(flags), int(frames),
                              ctypes.byref(rows), ctypes.byref(stage), cand, 8))
    return {"rows": rows.value, "stage_bytes": stage.value,
            "candidates_us": [round(float(c), 2) for c in cand if c != 0.0]}


def bf_selftest_wait(timeout_us):
    """Device-side bounded-wait self-test (see include/bf.h): raises BFError with
    code BF_ETIMEDOUT when the wait ran out as designed."""
    return _check(load().bf_selftest_wait(ctypes.c_int64(int(timeout_us))))


def bf_logdb_static(y_dev, nx, nz, z0_m, z1_m, f0_hz, c_mps, bandpass, db_dev, stream=None):
    """Allocation-free envelope + log compression of one device image (see include/bf.h)."""
    s = getattr(stream, "cuda_stream", stream)
    return _check(load().bf_logdb_static(_ptr(y_dev), int(nx), int(nz), float(z0_m), float(z1_m),
                                         float(f0_hz), float(c_mps), int(bool(bandpass)),
                                         _ptr(db_dev), s))


def bf_sync(h):
    return _check(load().bf_sync(h))


def bf_submit(h, rf, n_samples, angles_rad, flags) -> int:
    """Returns the ticket; raises BFError (code BF_EAGAIN when admission is refused)."""
    a, ap = _angles(angles_rad)
    t = ctypes.c_uint64()
    _check(load().bf_submit(h, _ptr(rf), int(n_samples), ap, len(a), int(flags), ctypes.byref(t)))
    return t.value


def bf_poll(h, ticket, out=None, timeout_us=-1) -> int:
    """BF_OK once the result is in `out` (ticket released) or BF_PENDING; raises on errors."""
    nbytes = 0 if out is None else (out.nbytes if isinstance(out, np.ndarray)
                                    else out.numel() * out.element_size())
    return _check(load().bf_poll(h, int(ticket), _ptr(out), nbytes, int(timeout_us)),
                  allow=(BF_OK, BF_PENDING))


def bf_submit_many(h, rfs, n_samples, angles_rad, flags):
    """Submit several frames of one configuration; returns their tickets (raises
    BFError; on BF_EAGAIN the error's .submitted holds the tickets that got in)."""
    a, ap = _angles(angles_rad)
    n = len(rfs)
    ptrs = (ctypes.c_void_p * n)(*[_ptr(r) for r in rfs])
    t = (ctypes.c_uint64 * n)()
    done = ctypes.c_int32()
    rc = load().bf_submit_many(h, n, ptrs, int(n_samples), ap, len(a), int(flags), t,
                               ctypes.byref(done))
    if rc != BF_OK:
        err = BFError(rc, bf_last_error())
        err.submitted = [t[k] for k in range(done.value)]
        raise err
    return [t[k] for k in range(n)]


def bf_submit_many_into(h, rfs, n_samples, angles_rad, flags, outs):
    """bf_submit_many with a destination per frame (see include/bf.h): each result
    lands in outs[k] when its batch finishes; poll the tickets (without outs) to
    wait for them and release them."""
    a, ap = _angles(angles_rad)
    n = len(rfs)
    if len(outs) != n:
        raise ValueError("one destination per frame")
    ptrs = (ctypes.c_void_p * n)(*map(_ptr, rfs))
    optr = (ctypes.c_void_p * n)(*map(_ptr, outs))
    nbytes = min(map(_nbytes, outs)) if n else 0
    t = (ctypes.c_uint64 * n)()
    done = ctypes.c_int32()
    rc = load().bf_submit_many_into(h, n, ptrs, int(n_samples), ap, len(a), int(flags), optr,
                                    nbytes, t, ctypes.byref(done))
    if rc != BF_OK:
        err = BFError(rc, bf_last_error())
        err.submitted = [t[k] for k in range(done.value)]
        raise err
    return [t[k] for k in range(n)]


def bf_poll_many(h, tickets, outs=None, timeout_us=-1) -> int:
    """Wait for every ticket and copy each result into outs[k]; BF_OK or BF_PENDING."""
    n = len(tickets)
    tk = (ctypes.c_uint64 * n)(*[int(x) for x in tickets])
    nbytes = 0
    optr = None
    if outs is not None:
        optr = (ctypes.c_void_p * n)(*map(_ptr, outs))
        nbytes = min(map(_nbytes, outs))
    return _check(load().bf_poll_many(h, n, tk, optr, nbytes, int(timeout_us)),
                  allow=(BF_OK, BF_PENDING))


def bf_ticket_batch(h, ticket):
    bid, n = ctypes.c_int32(), ctypes.c_int32()
    rc = _check(load().bf_ticket_batch(h, int(ticket), ctypes.byref(bid), ctypes.byref(n)),
                allow=(BF_OK, BF_PENDING))
    return None if rc == BF_PENDING else (bid.value, n.value)


def bf_ticket_times(h, ticket):
    """(start_ms, end_ms) of the ticket's batch on the device, or None while pending."""
    t0, t1 = ctypes.c_double(), ctypes.c_double()
    rc = _check(load().bf_ticket_times(h, int(ticket), ctypes.byref(t0), ctypes.byref(t1)),
                allow=(BF_OK, BF_PENDING))
    return None if rc == BF_PENDING else (t0.value, t1.value)


def bf_engine_pause(paused=True):
    return _check(load().bf_engine_pause(int(bool(paused))))


def bf_engine_configure(max_batch=0, max_inflight=0, memory_budget_bytes=0):
    return _check(load().bf_engine_configure(int(max_batch), int(max_inflight),
                                             int(memory_budget_bytes)))


class Batch:
    """A prepared multi-frame launch (uneven grids, one CUDA graph)."""

    def __init__(self, frames):
        """frames: list of (handle, rf_dev, n_samples, angles_rad, flags, out_dev)."""
        self._keep = []
        arr = (bf_frame * len(frames))()
        for k, (h, rf, ns, ang, flags, out) in enumerate(frames):
            a, ap = _angles(ang)
            self._keep.append(a)
            arr[k] = bf_frame(h, _ptr(rf), int(ns), ap, len(a), int(flags), _ptr(out))
        b = ctypes.c_void_p()
        _check(load().bf_batch_create(arr, len(frames), ctypes.byref(b)))
        self.ptr = b.value

    def launch(self, stream=None):
        s = getattr(stream, "cuda_stream", stream)
        return _check(load().bf_batch_launch(self.ptr, s))

    def status(self, stream=None):
        s = getattr(stream, "cuda_stream", stream)
        return _check(load().bf_batch_status(self.ptr, s))

    def timing(self):
        """(ingest_ms, beamform_ms, envelope_log_ms) of the last replay, kernels per replay."""
        ms = (ctypes.c_float * 3)()
        n = ctypes.c_int32()
        _check(load().bf_batch_timing(self.ptr, ms, ctypes.byref(n)))
        return (ms[0], ms[1], ms[2]), n.value

    def close(self):
        if self.ptr:
            _check(load().bf_batch_destroy(self.ptr))
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def n_modes(flags) -> int:
    """Images one frame produces (one per selected RF or IQ combiner)."""
    return bin(int(flags) & (BF_MODE_MASK | BF_IQ_MASK)).count("1")
