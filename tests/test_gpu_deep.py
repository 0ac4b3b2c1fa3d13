"""Accuracy of the mixed-precision cube at depth: a reduced stack in which a
few cube entries each receive more than 10^5 contributions, against the FP64
oracle on every entry, once and stacked four times into one cube.  The FP32
cube entries are moved into the FP64 master at checkpoints, so the error
must not grow with the depth (the full batched stack at twice its depth is
in test_gpu_batched.py)."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from tests import gpu_helpers as H  # noqa: E402


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_01897_gb300 import build
    build.build()
    from paper_2609_01897_gb300 import vista
    vista.lib()
    return vista


def _deep_workload(nwin=4, nrow=80000, nchan=16, npol=2, seed=3, device="cuda"):
    """Short baselines (a few metres) on a coarse uv grid: every row falls in
    one of the four central cells, so each (cell, rest bin, pol) entry
    collects about nwin * nrow / 4 visibilities per channel it covers."""
    from paper_2609_01897_gb300 import synth
    rng = np.random.default_rng(seed)
    spws = []
    for w in range(nwin):
        uvw = rng.uniform(-3.0, 3.0, size=(nrow, 3))
        f = 100e9 + 31.25e6 * np.arange(nchan)
        g = torch.Generator(device=device)
        g.manual_seed(seed * 100 + w)
        vis = torch.complex(torch.randn((nrow, nchan, npol), generator=g, device=device) + 1.0,
                            torch.randn((nrow, nchan, npol), generator=g, device=device)).to(torch.complex64)
        wts = (torch.rand((nrow, npol), generator=g, device=device) + 0.5).to(torch.float32)
        flags = (torch.rand((nrow, nchan, npol), generator=g, device=device) < 0.02).to(torch.uint8)
        spws.append(synth.SourceSpw(torch.as_tensor(uvw, device=device), f, vis, wts, flags,
                                    2e-6 * (w + 1), -1e-6 * w, 0.3 + 0.002 * w))
    # cells of 4 m x 100 GHz / c wavelengths: |u| <= 3 m lands in the central 2 x 2
    du = 4.0 * 100.5e9 / H.C_LIGHT
    return synth.Workload("deep", 8, 8, 24, npol, du, du, (100e9 + 7.5 * 31.25e6) * 1.302, spws)


def test_deep_stack_against_oracle(V):
    wl = _deep_workload()
    g = H.run_gpu(wl)
    o = H.run_oracle(wl, nthreads=8)
    assert int(o["count"].max()) >= 100000, int(o["count"].max())
    errs = H.compare(g, o, H.TOL_MIXED, what="deep stack")
    H.stats_equal(g, o)
    print("deep stack: max count %d, worst errors %s" % (int(o["count"].max()),
                                                       {k: "%.2e" % v for k, v in errs.items()}))


def test_deep_stack_repeated_runs(V):
    """The same windows stacked in 4 successive runs into one cube: 4x the
    depth (counts above 2 x 10^5 per entry), 4x the oracle's sums."""
    wl = _deep_workload(nwin=2, nrow=80000)
    st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, central_freq=wl.central_freq)
    try:
        for _ in range(4):
            for s in wl.spws:
                st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z)
            st.run()
        cube = st.read_cube(device=True, f64=True)
        out = {k: v.cpu().numpy() for k, v in cube.items()}
    finally:
        st.close()
    out["sum_wv"] = out["sum_wv"][..., 0] + 1j * out["sum_wv"][..., 1]
    o = H.run_oracle(wl, nthreads=8)
    o4 = {"sum_wv": 4 * o["sum_wv"], "sum_w": 4 * o["sum_w"], "sum_wvv": 4 * o["sum_wvv"],
          "sum_wabs": 4 * o["sum_wabs"], "count": 4 * o["count"]}
    assert int(o4["count"].max()) >= 200000
    H.compare(out, o4, H.TOL_MIXED, what="deep stack x4")
