"""The full re-projection of Eq. 1 (vista_add_source_reproject): each window
names its phase centre (ra0, dec0) and the stacking position (ra1, dec1);
the shift uses the direction cosines of the stacking position and the uv
cells the baseline rotated into its frame.  Every case is compared with the
FP64 oracle, which derives the same quantities from the four angles itself:
counts and cells exact, sums within the path's tolerance."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from tests import gpu_helpers as H  # noqa: E402

DEC0 = math.radians(-30.0)   # the synthetic arrays observe at declination -30


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_01897_gb300 import build
    build.build()
    from paper_2609_01897_gb300 import vista
    vista.lib()
    return vista


@pytest.fixture(scope="module")
def tiny():
    from paper_2609_01897_gb300 import synth
    return synth.tiny("cuda")


def _position(ra0, dec0, l, m):
    """The sky position at direction cosines (l, m) from the phase centre
    (ra0, dec0), from the frame's unit vectors (east, north, centre)."""
    w = np.array([math.cos(dec0) * math.cos(ra0), math.cos(dec0) * math.sin(ra0), math.sin(dec0)])
    e = np.cross([0.0, 0.0, 1.0], w)
    e /= np.linalg.norm(e)
    nth = np.cross(w, e)
    s = l * e + m * nth + math.sqrt(1 - l * l - m * m) * w
    return math.atan2(s[1], s[0]), math.asin(s[2])


def _consistent(wl):
    """Each window's phase centre at ra 0.7 + 0.1 i, dec -30, and its
    stacking position where its synthetic source lies (its l, m)."""
    out = []
    for i, s in enumerate(wl.spws):
        ra0 = 0.7 + 0.1 * i
        out.append((ra0, DEC0) + _position(ra0, DEC0, s.l, s.m))
    return out


def _large(wl, deg):
    """Stacking positions `deg` degrees from the phase centres, in varied
    directions: the rotation moves most cells."""
    out = []
    for i, _ in enumerate(wl.spws):
        ra0, a = 0.2 + 0.3 * i, 2 * math.pi * i / len(wl.spws)
        l, m = math.radians(deg) * math.cos(a), math.radians(deg) * math.sin(a)
        out.append((ra0, DEC0) + _position(ra0, DEC0, l, m))
    return out


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_reprojection_at_the_sources(V, tiny, prec):
    rp = _consistent(tiny)
    precision = V.PREC_MIXED if prec == "mixed" else V.PREC_FP64
    g = H.run_gpu(tiny, precision=precision, reproject=rp)
    o = H.run_oracle(tiny, reproject=rp)
    H.compare(g, o, H.TOL_MIXED if prec == "mixed" else H.TOL_FP64, what="re-projected, " + prec)
    H.stats_equal(g, o)


@pytest.mark.parametrize("fold", [False, True])
def test_reprojection_by_degrees_moves_cells(V, tiny, fold):
    rp = _large(tiny, 1.5)
    g = H.run_gpu(tiny, reproject=rp, fold=fold)
    o = H.run_oracle(tiny, reproject=rp, fold=fold)
    H.compare(g, o, H.TOL_MIXED, what="re-projected by 1.5 deg, fold %s" % fold)
    plain = H.run_oracle(tiny, fold=fold)
    assert not np.array_equal(plain["count"], o["count"])   # the rotation does change the cells


def test_same_centre(V, tiny):
    """Re-projecting onto the phase centre itself: R = M M^T (the identity up
    to rounding) and no shift; still the oracle's cells, exactly."""
    rp = [(0.7 + 0.1 * i, DEC0, 0.7 + 0.1 * i, DEC0) for i in range(len(tiny.spws))]
    g = H.run_gpu(tiny, reproject=rp)
    o = H.run_oracle(tiny, reproject=rp)
    H.compare(g, o, H.TOL_MIXED, what="same centre")


def test_host_memory_and_mixed_sets(V, tiny):
    """Host-memory windows, and re-projected windows queued together with
    plain ones in one run."""
    rp = _large(tiny, 0.5)
    g = H.run_gpu(tiny, reproject=rp, host_mem=True)
    H.compare(g, H.run_oracle(tiny, reproject=rp), H.TOL_MIXED, what="host memory")
    half = [r if i % 2 == 0 else None for i, r in enumerate(rp)]
    g = H.run_gpu(tiny, reproject=half)
    H.compare(g, H.run_oracle(tiny, reproject=half), H.TOL_MIXED, what="half re-projected")


def test_changed_projection_is_planned_again(V, tiny):
    """An unchanged set replays its graph; a new stacking position is a new
    plan (not a stale replay)."""
    rp_a, rp_b = _large(tiny, 0.5), _large(tiny, 1.0)
    st = V.Stack(tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv, central_freq=tiny.central_freq)
    try:
        for _ in range(2):
            for s, r in zip(tiny.spws, rp_a):
                st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, z=s.z, reproject=r)
            st.run()
        assert st.graph_runs() == 1
        st.zero()
        for s, r in zip(tiny.spws, rp_b):
            st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, z=s.z, reproject=r)
        st.run()
        assert st.graph_runs() == 1
        c = {k: v.cpu().numpy() for k, v in st.read_cube(f64=True).items()}
        c["sum_wv"] = c["sum_wv"][..., 0] + 1j * c["sum_wv"][..., 1]
    finally:
        st.close()
    H.compare(c, H.run_oracle(tiny, reproject=rp_b), H.TOL_MIXED, what="changed projection")


def test_reprojection_errors(V, tiny):
    s = tiny.spws[0]
    st = V.Stack(tiny.nu, tiny.nv, tiny.nrest, tiny.npol, tiny.du, tiny.dv, central_freq=tiny.central_freq)
    try:
        for bad in [(0.0, 2.0, 0.0, 0.0), (0.0, 0.0, float("nan"), 0.0), (0.0, 0.0, math.pi / 2, 0.0),
                    (0.0, 0.0, math.pi, 0.0)]:
            with pytest.raises(V.VistaError) as ei:
                st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, z=s.z, reproject=bad)
            assert ei.value.code == V.E_ARG
        # the handle is unchanged: a valid run afterwards matches the oracle
        st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, z=s.z, reproject=_consistent(tiny)[0])
        st.run()
        assert st.stats()["n_vis"] > 0
    finally:
        st.close()
