"""ctypes front end of the FP64 CPU oracle (oracle/vista_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg; never by the GPU library.  Every function takes
and returns numpy arrays on the host.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrCube(C.Structure):
    _fields_ = [("nu", C.c_int32), ("nv", C.c_int32), ("nrest", C.c_int32), ("npol", C.c_int32),
                ("du", C.c_double), ("dv", C.c_double),
                ("rest_f0", C.c_double), ("rest_df", C.c_double),
                ("bin_mode", C.c_int32), ("hermitian_fold", C.c_int32)]


class OrSource(C.Structure):
    _fields_ = [("nrow", C.c_int64), ("nchan", C.c_int32), ("npol", C.c_int32),
                ("uvw", C.c_void_p), ("freqs", C.c_void_p), ("vis", C.c_void_p),
                ("vis_f64", C.c_int32), ("pad0", C.c_int32),
                ("weights", C.c_void_p), ("flags", C.c_void_p), ("pol_map", C.c_void_p),
                ("l", C.c_double), ("m", C.c_double), ("z", C.c_double),
                ("reproject", C.c_int32), ("pad1", C.c_int32),
                ("ra0", C.c_double), ("dec0", C.c_double), ("ra1", C.c_double), ("dec1", C.c_double)]


class OrStats(C.Structure):
    _fields_ = [("n_vis", C.c_uint64), ("n_flagged", C.c_uint64),
                ("n_dropped_uv", C.c_uint64), ("n_stacked", C.c_uint64),
                ("w_unflagged", C.c_double), ("w_cube", C.c_double),
                ("w_dropped_uv", C.c_double), ("w_dropped_rest", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_channel_widths.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
        L.or_auto_lattice.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                      C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.or_rest_weights.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_double,
                                      C.c_int32, C.c_int32, C.c_void_p]
        L.or_rotation.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p]
        L.or_rotation.restype = None
        L.or_offset.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p]
        L.or_offset.restype = None
        L.or_phasors.argtypes = [C.POINTER(OrSource), C.c_void_p]
        L.or_phasors.restype = None
        L.or_cells.argtypes = [C.POINTER(OrCube), C.POINTER(OrSource), C.c_void_p]
        L.or_cells.restype = None
        L.or_stack.argtypes = [C.POINTER(OrCube), C.POINTER(OrSource), C.c_int32, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.POINTER(OrStats), C.c_int32]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def channel_widths(freqs):
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    out = np.empty_like(f)
    if lib().or_channel_widths(_ptr(f), f.size, _ptr(out)) != 0:
        raise ValueError("need at least two channels")
    return out


def auto_lattice(freq_list, z_list, nrest, central_freq):
    fs = [np.ascontiguousarray(f, dtype=np.float64) for f in freq_list]
    ptrs = (C.c_void_p * len(fs))(*[f.ctypes.data for f in fs])
    n = np.array([f.size for f in fs], dtype=np.int32)
    z = np.ascontiguousarray(z_list, dtype=np.float64)
    f0, df = C.c_double(), C.c_double()
    rc = lib().or_auto_lattice(C.cast(ptrs, C.c_void_p), _ptr(n), _ptr(z), len(fs), nrest,
                               central_freq, C.byref(f0), C.byref(df))
    if rc != 0:
        raise ValueError("auto lattice failed (%d)" % rc)
    return f0.value, df.value


def rest_weights(freqs, z, f0, df, nrest, bin_mode=0):
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    out = np.zeros((f.size, nrest), dtype=np.float64)
    rc = lib().or_rest_weights(_ptr(f), f.size, z, f0, df, nrest, bin_mode, _ptr(out))
    if rc != 0:
        raise ValueError("rest weights failed (%d)" % rc)
    return out


class Source:
    """Host arrays of one (source, spectral window).  vis: complex64 or
    complex128 [nrow, nchan, npol]; the arrays are kept alive here.
    radec = (ra0, dec0, ra1, dec1), radians: re-project from the phase centre
    (ra0, dec0) to the stacking position (ra1, dec1) (Eq. 1); l, m are then
    ignored."""

    def __init__(self, uvw, freqs, vis, weights, flags, l, m, z, pol_map=None, radec=None):
        self.uvw = np.ascontiguousarray(uvw, dtype=np.float64)
        self.freqs = np.ascontiguousarray(freqs, dtype=np.float64)
        vis = np.asarray(vis)
        if vis.dtype == np.complex128:
            self.vis = np.ascontiguousarray(vis)
            f64 = 1
        else:
            self.vis = np.ascontiguousarray(vis, dtype=np.complex64)
            f64 = 0
        self.weights = np.ascontiguousarray(weights, dtype=np.float32)
        self.flags = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8)
        self.pol_map = None if pol_map is None else np.ascontiguousarray(pol_map, dtype=np.int32)
        nrow, nchan, npol = self.vis.shape
        assert self.uvw.shape == (nrow, 3) and self.freqs.shape == (nchan,)
        assert self.weights.shape == (nrow, npol)
        self.c = OrSource(nrow, nchan, npol, _ptr(self.uvw), _ptr(self.freqs), _ptr(self.vis),
                          f64, 0, _ptr(self.weights), _ptr(self.flags), _ptr(self.pol_map),
                          float(l), float(m), float(z), 0 if radec is None else 1, 0,
                          *((0.0, 0.0, 0.0, 0.0) if radec is None else tuple(float(x) for x in radec)))


def rotation(ra0, dec0, ra1, dec1):
    """Eq. 1's rotation R = M(ra1, dec1) M(ra0, dec0)^T as a 3 x 3 array."""
    R = np.empty(9, dtype=np.float64)
    lib().or_rotation(ra0, dec0, ra1, dec1, _ptr(R))
    return R.reshape(3, 3)


def offset(ra0, dec0, ra1, dec1):
    """Direction cosines (l, m) of (ra1, dec1) seen from (ra0, dec0)."""
    lm = np.empty(2, dtype=np.float64)
    lib().or_offset(ra0, dec0, ra1, dec1, _ptr(lm))
    return float(lm[0]), float(lm[1])


def regrid_rows(src, rest_f0, rest_df, nrest, bin_mode=0):
    """The paper's per-row output (Eq. 3): each row's shifted spectrum on the
    rest lattice, V_out(r, j, p) = sum_k V'(r, k, p) w_kj / sum_k w_kj over
    the unflagged channels k (0 where that sum is 0), and the sum itself.
    V' is the shifted visibility of Eq. 2 (phasors(): the same shift as the
    stack, re-projection included) and w_kj the Eq. 4 weights (rest_weights());
    the two sums are plain matrix products.  Returns (vis_out complex128
    [nrow, nrest, npol], wsum float64 [nrow, nrest, npol])."""
    vis = src.vis.astype(np.complex128) * phasors(src)[..., None]
    w = rest_weights(src.freqs, src.c.z, rest_f0, rest_df, nrest, bin_mode)     # [nchan, nrest]
    ok = np.ones(vis.shape, dtype=np.float64) if src.flags is None else (src.flags == 0).astype(np.float64)
    # [r, p, k] @ [k, j] -> [r, p, j] -> [r, j, p]
    num = np.moveaxis(np.matmul(np.moveaxis(vis * ok, 2, 1), w), 1, 2)
    den = np.moveaxis(np.matmul(np.moveaxis(ok, 2, 1), w), 1, 2)
    out = np.zeros_like(num)
    nz = den > 0
    out[nz] = num[nz] / den[nz]
    return out, den


def make_cube(nu, nv, nrest, npol, du, dv, rest_f0, rest_df, bin_mode=0, hermitian_fold=0):
    return OrCube(nu, nv, nrest, npol, du, dv, rest_f0, rest_df, bin_mode, hermitian_fold)


def phasors(src):
    out = np.empty((src.c.nrow, src.c.nchan, 2), dtype=np.float64)
    lib().or_phasors(C.byref(src.c), _ptr(out))
    return out[..., 0] + 1j * out[..., 1]


def cells(cube, src):
    out = np.empty((src.c.nrow, src.c.nchan, 2), dtype=np.int32)
    lib().or_cells(C.byref(cube), C.byref(src.c), _ptr(out))
    return out


def stack(cube, sources, iv_select=None, nthreads=1, with_abs=False):
    """Returns dict(sum_wv complex128, sum_w, sum_wvv, count uint64, stats, planes,
    and with with_abs=True sum_wabs = sum W w |V|, the scale of the sum_wv bound)."""
    nplanes = cube.nv
    sel = None
    if iv_select is not None:
        sel = np.zeros(cube.nv, dtype=np.uint8)
        sel[np.asarray(iv_select, dtype=np.int64)] = 1
        nplanes = int(sel.sum())
    shape = (nplanes, cube.nu, cube.nrest, cube.npol)
    sum_wv = np.zeros(shape + (2,), dtype=np.float64)
    sum_w = np.zeros(shape, dtype=np.float64)
    sum_wvv = np.zeros(shape, dtype=np.float64)
    count = np.zeros(shape, dtype=np.uint64)
    sum_wabs = np.zeros(shape, dtype=np.float64) if with_abs else None
    arr = (OrSource * max(1, len(sources)))(*[s.c for s in sources])
    st = OrStats()
    rc = lib().or_stack(C.byref(cube), arr, len(sources), _ptr(sel), _ptr(sum_wv), _ptr(sum_w),
                        _ptr(sum_wvv), _ptr(sum_wabs), _ptr(count), C.byref(st), int(nthreads))
    if rc != 0:
        raise ValueError("oracle stack failed (%d)" % rc)
    planes = np.arange(cube.nv) if sel is None else np.nonzero(sel)[0]
    return {"sum_wv": sum_wv[..., 0] + 1j * sum_wv[..., 1], "sum_w": sum_w, "sum_wvv": sum_wvv,
            "sum_wabs": sum_wabs, "count": count,
            "stats": st.as_dict() if iv_select is None else None, "planes": planes}


def default_threads():
    return os.cpu_count() or 1
