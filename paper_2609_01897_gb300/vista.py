"""Python binding of libvista (include/vista.h): argument marshalling only.

Every step of the stacking runs in the library's CUDA kernels; this module
converts torch tensors into pointers and sizes, and C status codes into
exceptions.  It raises if libvista.so has not been built -- there is no
fallback implementation.
"""
import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

VISTA_OK, E_ARG, E_STATE, E_NOMEM, E_CUDA, E_RANGE, E_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
VIS_C64, VIS_C128, VIS_F16X2, VIS_BF16X2 = 0, 1, 2, 3
BIN_OVERLAP, BIN_NEAREST = 0, 1
PREC_MIXED, PREC_FP64 = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
MAX_BINS = 4

_CODES = {E_ARG: "VISTA_E_ARG", E_STATE: "VISTA_E_STATE", E_NOMEM: "VISTA_E_NOMEM",
          E_CUDA: "VISTA_E_CUDA", E_RANGE: "VISTA_E_RANGE", E_TIMEOUT: "VISTA_E_TIMEOUT"}


class CubeDesc(C.Structure):
    _fields_ = [("nu", C.c_int32), ("nv", C.c_int32), ("nrest", C.c_int32), ("npol", C.c_int32),
                ("du", C.c_double), ("dv", C.c_double), ("rest_f0", C.c_double),
                ("rest_df", C.c_double), ("central_freq", C.c_double),
                ("bin_mode", C.c_int32), ("precision", C.c_int32),
                ("hermitian_fold", C.c_int32), ("reserved0", C.c_int32), ("stream", C.c_void_p)]


class SourceDesc(C.Structure):
    _fields_ = [("nrow", C.c_int64), ("nchan", C.c_int32), ("npol", C.c_int32),
                ("uvw", C.c_void_p), ("freqs", C.c_void_p), ("vis", C.c_void_p),
                ("vis_type", C.c_int32), ("vis_scale", C.c_float),
                ("weights", C.c_void_p), ("flags", C.c_void_p), ("pol_map", C.c_void_p),
                ("l", C.c_double), ("m", C.c_double), ("z", C.c_double),
                ("mem", C.c_int32), ("reserved0", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("n_vis", C.c_uint64), ("n_flagged", C.c_uint64),
                ("n_dropped_uv", C.c_uint64), ("n_stacked", C.c_uint64),
                ("n_reductions", C.c_uint64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Tuning(C.Structure):
    _fields_ = [("rows_per_item", C.c_int32), ("chans_per_lane", C.c_int32),
                ("warps_per_cta", C.c_int32), ("sort_rows", C.c_int32), ("prefetch_rows", C.c_int32)]


class Timing(C.Structure):
    _fields_ = [("prepass_ms", C.c_double), ("stack_ms", C.c_double), ("other_ms", C.c_double),
                ("runs", C.c_int64), ("launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class VistaError(RuntimeError):
    def __init__(self, call, code, msg):
        super().__init__("%s failed: %s: %s" % (call, _CODES.get(code, code), msg))
        self.code = code


# Every symbol include/vista.h declares, with (restype, argtypes).
_P = C.c_void_p
SIGNATURES = {
    "vista_open_stack": (C.c_int, [C.POINTER(CubeDesc), C.POINTER(_P)]),
    "vista_add_source": (C.c_int, [_P, C.POINTER(SourceDesc)]),
    "vista_add_source_reproject": (C.c_int, [_P, C.POINTER(SourceDesc), C.c_double, C.c_double, C.c_double,
                                             C.c_double]),
    "vista_regrid_rows": (C.c_int, [_P, C.POINTER(SourceDesc), _P, _P, _P]),
    "vista_contsub": (C.c_int, [_P, _P, C.c_int32, _P, C.c_int]),
    "vista_set_wave_bytes": (C.c_int, [_P, C.c_int64]),
    "vista_get_waves": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "vista_get_h2d_bytes": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "vista_read_cube_async": (C.c_int, [_P, _P, _P, _P, _P]),
    "vista_wait_readback": (C.c_int, [_P]),
    "vista_read_cube_sparse": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, C.POINTER(C.c_int64), C.c_int]),
    "vista_run": (C.c_int, [_P]),
    "vista_read_cube": (C.c_int, [_P, _P, _P, _P, _P, C.c_int]),
    "vista_read_cube_f64": (C.c_int, [_P, _P, _P, _P, _P, C.c_int]),
    "vista_zero_cube": (C.c_int, [_P]),
    "vista_get_stats": (C.c_int, [_P, C.POINTER(Stats)]),
    "vista_get_lattice": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "vista_set_tuning": (C.c_int, [_P, C.POINTER(Tuning)]),
    "vista_get_tuning": (C.c_int, [_P, C.POINTER(Tuning)]),
    "vista_enable_timing": (C.c_int, [_P, C.c_int]),
    "vista_get_timing": (C.c_int, [_P, C.POINTER(Timing)]),
    "vista_close": (C.c_int, [_P]),
    "vista_last_error": (C.c_char_p, [_P]),
    "vista_abi_version": (C.c_int, []),
    "vista_plan_lattice": (C.c_int, [_P, _P, _P, C.c_int32, C.c_int32, C.c_double,
                                     C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "vista_plan_channels": (C.c_int, [_P, C.c_int32, C.c_double, C.c_double, C.c_double,
                                      C.c_int32, C.c_int32, _P, _P, _P]),
    "vista_debug_phasors": (C.c_int, [_P, C.c_int32, _P]),
    "vista_debug_cells": (C.c_int, [_P, C.c_int32, _P]),
    "vista_debug_order": (C.c_int, [_P, C.c_int32, _P]),
    "vista_stack_noalloc": (C.c_int, [C.POINTER(CubeDesc), C.POINTER(SourceDesc), _P, _P]),
    "vista_enable_graphs": (C.c_int, [_P, C.c_int]),
    "vista_autotune": (C.c_int, [_P, C.c_int32, C.c_int32, C.POINTER(Tuning)]),
    "vista_graph_runs": (C.c_int, [_P, C.POINTER(C.c_uint64)]),
}

_lib = None


def lib_path():
    return _build.LIB


def lib():
    """Load libvista.so (raises if it is missing: build it first)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libvista.so not found at %s: run paper_2609_01897_gb300.build.build() "
                               "(there is no CPU fallback)" % path)
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error(h=None):
    s = lib().vista_last_error(h)
    return s.decode() if s else ""


def _check(call, rc, h=None):
    if rc != VISTA_OK:
        raise VistaError(call, rc, last_error(h))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _vis_type(vis):
    if vis.dtype == torch.complex64:
        return VIS_C64
    if vis.dtype == torch.complex128:
        return VIS_C128
    if vis.dtype == torch.float16:
        return VIS_F16X2
    if vis.dtype == torch.bfloat16:
        return VIS_BF16X2
    raise TypeError("vis must be complex64, complex128, or float16/bfloat16 [..., 2]")


class Stack:
    """One stacking cube (vista_open_stack ... vista_close)."""

    def __init__(self, nu, nv, nrest, npol, du, dv, *, rest_f0=0.0, rest_df=0.0, central_freq=0.0,
                 bin_mode=BIN_OVERLAP, precision=PREC_MIXED, hermitian_fold=False, stream=None):
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream()
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        self.desc = CubeDesc(nu, nv, nrest, npol, du, dv, rest_f0, rest_df, central_freq,
                             bin_mode, precision, 1 if hermitian_fold else 0, 0, sp)
        h = _P()
        _check("vista_open_stack", lib().vista_open_stack(C.byref(self.desc), C.byref(h)))
        self.h = h
        self.shape = (nv, nu, nrest, npol)
        self._pending = []
        self._inflight = []

    # -- sources
    def add_source(self, uvw, freqs, vis, weights, flags=None, *, l=0.0, m=0.0, z, pol_map=None,
                   vis_scale=1.0, reproject=None):
        """uvw [nrow,3] f64, freqs [nchan] f64 (host), vis [nrow,nchan,npol] complex
        (or 16-bit [nrow,nchan,npol,2]), weights [nrow,npol] f32, flags u8 or None.
        CUDA tensors are borrowed device arrays; CPU tensors are host arrays
        (pin them for asynchronous copies).  reproject = (ra0, dec0, ra1, dec1),
        radians: the window's phase centre and the stacking position, for the
        full re-projection of Eq. 1 (l, m are then derived, not read)."""
        vt = _vis_type(vis)
        nrow, nchan, npol = int(vis.shape[0]), int(vis.shape[1]), int(vis.shape[2])
        if vt in (VIS_F16X2, VIS_BF16X2) and (vis.dim() != 4 or vis.shape[3] != 2):
            raise ValueError("16-bit visibilities are [nrow, nchan, npol, 2]")
        for name, t in (("uvw", uvw), ("vis", vis), ("weights", weights), ("flags", flags)):
            if t is not None and not t.is_contiguous():
                raise ValueError("%s must be contiguous" % name)
        dev = vis.is_cuda
        for name, t in (("uvw", uvw), ("weights", weights), ("flags", flags)):
            if t is not None and t.is_cuda != dev:
                raise ValueError("%s must live on the same side (host/device) as vis" % name)
        if uvw.dtype != torch.float64 or weights.dtype != torch.float32:
            raise TypeError("uvw must be float64 and weights float32")
        if flags is not None and flags.dtype != torch.uint8:
            raise TypeError("flags must be uint8")
        f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64))
        pm = None if pol_map is None else np.ascontiguousarray(np.asarray(pol_map, dtype=np.int32))
        d = SourceDesc(nrow, nchan, npol, _ptr(uvw), f.ctypes.data, _ptr(vis), vt, float(vis_scale),
                       _ptr(weights), _ptr(flags), None if pm is None else pm.ctypes.data,
                       float(l), float(m), float(z), MEM_DEVICE if dev else MEM_HOST, 0)
        if reproject is None:
            _check("vista_add_source", lib().vista_add_source(self.h, C.byref(d)), self.h)
        else:
            ra0, dec0, ra1, dec1 = (float(x) for x in reproject)
            _check("vista_add_source_reproject",
                   lib().vista_add_source_reproject(self.h, C.byref(d), ra0, dec0, ra1, dec1), self.h)
        self._pending.append((uvw, vis, weights, flags))

    def regrid_rows(self, uvw, freqs, vis, flags=None, *, l=0.0, m=0.0, z, vis_scale=1.0, with_uvw=False,
                    out=None):
        """The paper's per-row output (Eq. 3) of one window of device arrays:
        returns (vis_out complex64 [nrow, nrest, npol], wsum float32 [nrow,
        nrest, npol], uvw / (1 + z) float64 [nrow, 3] or None), on the device.
        The rest lattice must be fixed (rest_df at open, or after a run).
        `out` = (float32 [nrow, nrest, npol, 2], float32 [nrow, nrest, npol])
        contiguous device tensors are written in place instead of allocating,
        and returned as given (vis_out then as float pairs)."""
        vt = _vis_type(vis)
        nrow, nchan, npol = int(vis.shape[0]), int(vis.shape[1]), int(vis.shape[2])
        if not vis.is_cuda or not uvw.is_cuda or (flags is not None and not flags.is_cuda):
            raise ValueError("regrid_rows reads device arrays")
        for name, t in (("uvw", uvw), ("vis", vis), ("flags", flags)):
            if t is not None and not t.is_contiguous():
                raise ValueError("%s must be contiguous" % name)
        if uvw.dtype != torch.float64 or (flags is not None and flags.dtype != torch.uint8):
            raise TypeError("uvw must be float64 and flags uint8")
        nrest = self.shape[2]
        given = out is not None
        if out is None:   # every entry is written (0 where no channel contributes)
            out = torch.empty((nrow, nrest, npol, 2), dtype=torch.float32, device=vis.device)
            wsum = torch.empty((nrow, nrest, npol), dtype=torch.float32, device=vis.device)
        else:
            out, wsum = out
            for name, t, shp in (("out[0]", out, (nrow, nrest, npol, 2)), ("out[1]", wsum, (nrow, nrest, npol))):
                if (tuple(t.shape) != shp or t.dtype != torch.float32 or not t.is_cuda
                        or not t.is_contiguous()):
                    raise ValueError("%s must be a contiguous float32 device tensor of shape %s" % (name, shp))
        ruvw = torch.empty((nrow, 3), dtype=torch.float64, device=vis.device) if with_uvw else None
        f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64))
        d = SourceDesc(nrow, nchan, npol, _ptr(uvw), f.ctypes.data, _ptr(vis), vt, float(vis_scale),
                       None, _ptr(flags), None, float(l), float(m), float(z), MEM_DEVICE, 0)
        _check("vista_regrid_rows", lib().vista_regrid_rows(self.h, C.byref(d), _ptr(out), _ptr(wsum),
                                                            _ptr(ruvw)), self.h)
        return (out if given else torch.view_as_complex(out)), wsum, ruvw

    def run(self):
        _check("vista_run", lib().vista_run(self.h), self.h)
        # host-memory windows are copied by stream work that may still run
        # when run() returns: their arrays stay referenced until a sync
        self._inflight = self._inflight + self._pending
        self._pending = []

    # -- results
    def read_cube(self, device=True, f64=False, which=("sum_wv", "sum_w", "sum_wvv", "count"), out=None):
        """The cube's sums (ΣwV as [..., 2]) and counts, on the device or in
        pinned host memory.  `out` (a dict from an earlier call with the same
        device / f64 / which) is filled in place instead of allocating: pinning
        a host buffer of the cube's size costs more than the copy itself."""
        nv, nu, nrest, npol = self.shape
        dt = torch.float64 if f64 else torch.float32
        shapes = {"sum_wv": ((nv, nu, nrest, npol, 2), dt), "sum_w": ((nv, nu, nrest, npol), dt),
                  "sum_wvv": ((nv, nu, nrest, npol), dt), "count": ((nv, nu, nrest, npol), torch.int32)}
        if out is not None:
            for k in which:
                t = out.get(k)
                shp, tdt = shapes[k]
                if (t is None or tuple(t.shape) != shp or t.dtype != tdt or t.is_cuda != bool(device)
                        or not t.is_contiguous()):
                    raise ValueError("out[%r] must be a contiguous %s tensor of shape %s on the %s" % (
                        k, tdt, shp, "device" if device else "host"))
            out = {k: (out[k] if k in which else None) for k in shapes}
        else:
            kw = {"device": "cuda"} if device else {"pin_memory": torch.cuda.is_available()}
            out = {k: (torch.empty(shp, dtype=tdt, **kw) if k in which else None) for k, (shp, tdt) in shapes.items()}
        fn = lib().vista_read_cube_f64 if f64 else lib().vista_read_cube
        _check("vista_read_cube", fn(self.h, _ptr(out["sum_wv"]), _ptr(out["sum_w"]),
                                     _ptr(out["sum_wvv"]), _ptr(out["count"]), 1 if device else 0),
               self.h)
        self._inflight = []
        return {k: v for k, v in out.items() if v is not None}

    def read_cube_async(self, out):
        """vista_read_cube_async: queue the cube's readback into the pinned
        host tensors of `out` (a dict from read_cube(device=False)) and return
        at once; call wait_readback() before reading them."""
        nv, nu, nrest, npol = self.shape
        shapes = {"sum_wv": (nv, nu, nrest, npol, 2), "sum_w": (nv, nu, nrest, npol),
                  "sum_wvv": (nv, nu, nrest, npol), "count": (nv, nu, nrest, npol)}
        for k, t in out.items():
            if t is None:
                continue
            dt = torch.int32 if k == "count" else torch.float32
            if t.is_cuda or tuple(t.shape) != shapes[k] or t.dtype != dt or not t.is_contiguous():
                raise ValueError("out[%r] must be a contiguous host %s tensor of shape %s" % (k, dt, shapes[k]))
        _check("vista_read_cube_async", lib().vista_read_cube_async(
            self.h, _ptr(out.get("sum_wv")), _ptr(out.get("sum_w")), _ptr(out.get("sum_wvv")),
            _ptr(out.get("count"))), self.h)
        return out

    def read_cube_sparse(self, device=False, out=None):
        """The touched cube entries (count > 0) in entry order
        (vista_read_cube_sparse): index int64 [n] (the flat entry index into
        [nv][nu][nrest][npol]), sum_wv float32 [n, 2], sum_w and sum_wvv
        float32 [n], count int32 [n]; on the device, or in pinned host memory.
        `out` (a dict from an earlier call) is written in place when it holds
        at least n entries.  Returns the first n rows of each array."""
        L, n = lib(), C.c_int64(0)
        dev = 1 if device else 0

        def alloc(cap):
            kw = {"device": "cuda"} if device else {"pin_memory": torch.cuda.is_available()}
            return {"index": torch.empty(cap, dtype=torch.int64, **kw),
                    "sum_wv": torch.empty((cap, 2), dtype=torch.float32, **kw),
                    "sum_w": torch.empty(cap, dtype=torch.float32, **kw),
                    "sum_wvv": torch.empty(cap, dtype=torch.float32, **kw),
                    "count": torch.empty(cap, dtype=torch.int32, **kw)}

        if out is None or any(out[k].is_cuda != bool(device) for k in out):
            _check("vista_read_cube_sparse", L.vista_read_cube_sparse(self.h, 0, None, None, None, None, None,
                                                                      C.byref(n), dev), self.h)
            out = alloc(n.value)

        def call(o):
            return L.vista_read_cube_sparse(self.h, int(o["index"].shape[0]), _ptr(o["index"]), _ptr(o["sum_wv"]),
                                            _ptr(o["sum_w"]), _ptr(o["sum_wvv"]), _ptr(o["count"]), C.byref(n), dev)

        rc = call(out)
        if rc == E_RANGE and n.value > int(out["index"].shape[0]):
            out = alloc(n.value)
            rc = call(out)
        _check("vista_read_cube_sparse", rc, self.h)
        self._inflight = []
        return {k: v[:n.value] for k, v in out.items()}

    def wait_readback(self):
        _check("vista_wait_readback", lib().vista_wait_readback(self.h), self.h)
        self._inflight = []

    def contsub(self, line_free, order=1, device=True, out=None):
        """Continuum-subtracted sum W w V' of the cube (vista_contsub): a
        polynomial of degree <= order in rest channel, fitted per uv cell and
        plane over the line-free channels (line_free: [nrest] bools), is
        subtracted.  Returns a float32 tensor [nv, nu, nrest, npol, 2] on the
        device (or in pinned host memory)."""
        nv, nu, nrest, npol = self.shape
        lf = np.ascontiguousarray(np.asarray(line_free, dtype=np.uint8).reshape(-1))
        if lf.size != nrest:
            raise ValueError("line_free must have nrest = %d entries" % nrest)
        if out is None:
            kw = {"device": "cuda"} if device else {"pin_memory": torch.cuda.is_available()}
            out = torch.empty((nv, nu, nrest, npol, 2), dtype=torch.float32, **kw)
        _check("vista_contsub", lib().vista_contsub(self.h, lf.ctypes.data, int(order), _ptr(out),
                                                    1 if device else 0), self.h)
        return out

    def set_wave_bytes(self, nbytes):
        """Staged bytes per wave of host-memory windows (0 = the library's rule)."""
        _check("vista_set_wave_bytes", lib().vista_set_wave_bytes(self.h, int(nbytes)), self.h)

    def waves(self):
        """Waves the last run streamed its host-memory windows in."""
        n = C.c_int32(0)
        _check("vista_get_waves", lib().vista_get_waves(self.h, C.byref(n)), self.h)
        return int(n.value)

    def h2d_bytes(self):
        """Host-to-device bytes the last run copied for its host-memory windows."""
        n = C.c_int64(0)
        _check("vista_get_h2d_bytes", lib().vista_get_h2d_bytes(self.h, C.byref(n)), self.h)
        return int(n.value)

    def stats(self):
        s = Stats()
        _check("vista_get_stats", lib().vista_get_stats(self.h, C.byref(s)), self.h)
        self._inflight = []   # the call waited for the stream
        return s.as_dict()

    def lattice(self):
        f0, df = C.c_double(), C.c_double()
        _check("vista_get_lattice", lib().vista_get_lattice(self.h, C.byref(f0), C.byref(df)), self.h)
        return f0.value, df.value

    def zero(self):
        _check("vista_zero_cube", lib().vista_zero_cube(self.h), self.h)

    def set_tuning(self, rows_per_item=0, chans_per_lane=0, warps_per_cta=0, sort_rows=None,
                   prefetch_rows=0):
        """0 (or None for sort_rows) keeps the current value."""
        if sort_rows is None:
            sort_rows = self.tuning()["sort_rows"]
        t = Tuning(rows_per_item, chans_per_lane, warps_per_cta, int(sort_rows), prefetch_rows)
        _check("vista_set_tuning", lib().vista_set_tuning(self.h, C.byref(t)), self.h)

    def tuning(self):
        t = Tuning()
        _check("vista_get_tuning", lib().vista_get_tuning(self.h, C.byref(t)), self.h)
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def enable_timing(self, on=True):
        _check("vista_enable_timing", lib().vista_enable_timing(self.h, 1 if on else 0), self.h)

    def timing(self):
        t = Timing()
        _check("vista_get_timing", lib().vista_get_timing(self.h, C.byref(t)), self.h)
        return t.as_dict()

    def autotune(self, budget=0, reps=0):
        """Time the queued windows under candidate launch shapes and keep the
        fastest (the cube is zeroed afterwards; the queue is kept)."""
        t = Tuning()
        _check("vista_autotune", lib().vista_autotune(self.h, int(budget), int(reps), C.byref(t)), self.h)
        return {k: int(getattr(t, k)) for k, _ in Tuning._fields_}

    def enable_graphs(self, on=True):
        """Replay the device work of an unchanged source set from a CUDA graph (default on)."""
        _check("vista_enable_graphs", lib().vista_enable_graphs(self.h, 1 if on else 0), self.h)

    def graph_runs(self):
        n = C.c_uint64(0)
        _check("vista_graph_runs", lib().vista_graph_runs(self.h, C.byref(n)), self.h)
        return int(n.value)

    def debug_phasors(self, src, nrow, nchan):
        out = torch.zeros((nrow, nchan, 2), dtype=torch.float64, device="cuda")
        _check("vista_debug_phasors", lib().vista_debug_phasors(self.h, src, _ptr(out)), self.h)
        return out

    def debug_cells(self, src, nrow, nchan):
        out = torch.full((nrow, nchan, 2), -7, dtype=torch.int32, device="cuda")
        _check("vista_debug_cells", lib().vista_debug_cells(self.h, src, _ptr(out)), self.h)
        return out

    def debug_order(self, src, nrow):
        out = torch.full((nrow,), -1, dtype=torch.int32, device="cuda")
        _check("vista_debug_order", lib().vista_debug_order(self.h, src, _ptr(out)), self.h)
        return out

    def close(self):
        if self.h is not None:
            _check("vista_close", lib().vista_close(self.h))
            self.h = None
            self._inflight = []
            self._pending = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None:
                lib().vista_close(self.h)
        except Exception:
            pass


# -- host-only planner entry points

def plan_lattice(freq_list, z_list, nrest, central_freq):
    fs = [np.ascontiguousarray(f, dtype=np.float64) for f in freq_list]
    ptrs = (C.c_void_p * len(fs))(*[f.ctypes.data for f in fs])
    n = np.array([f.size for f in fs], dtype=np.int32)
    z = np.ascontiguousarray(z_list, dtype=np.float64)
    f0, df = C.c_double(), C.c_double()
    _check("vista_plan_lattice", lib().vista_plan_lattice(C.cast(ptrs, C.c_void_p), n.ctypes.data,
                                                          z.ctypes.data, len(fs), nrest, central_freq,
                                                          C.byref(f0), C.byref(df)))
    return f0.value, df.value


def plan_channels(freqs, z, f0, df, nrest, bin_mode=BIN_OVERLAP):
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    j0 = np.zeros(f.size, dtype=np.int32)
    nb = np.zeros(f.size, dtype=np.int32)
    w = np.zeros((f.size, MAX_BINS), dtype=np.float64)
    _check("vista_plan_channels", lib().vista_plan_channels(f.ctypes.data, f.size, z, f0, df, nrest,
                                                            bin_mode, j0.ctypes.data, nb.ctypes.data,
                                                            w.ctypes.data))
    return j0, nb, w
