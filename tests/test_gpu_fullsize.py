"""Full-size parity: the ALMA-compact-like workload (64 sources x 2 windows,
3.3e9 visibilities) in the launch configuration bench.py times, compared with
the FP64 oracle on sampled cube planes.

The oracle accumulates only the sampled iv planes; every row whose v
coordinate could reach one of them at some channel (a conservative
interval test, since iv is monotone in frequency) is handed to it, so its
sums for those planes are complete.  Counters are checked against
properties computed independently from the inputs."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from tests import gpu_helpers as H  # noqa: E402

PLANES = [3, 97, 121, 128, 129, 140, 171, 250]


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
def alma():
    from paper_2609_01897_gb300 import synth
    wl = synth.alma_compact("cuda")
    yield wl
    del wl
    torch.cuda.empty_cache()


def _rows_reaching(s, planes, nv, dv):
    """Rows whose iv interval over the window's frequency range meets a plane."""
    g = 1.0 / (H.C_LIGHT * dv)
    v = s.uvw[:, 1]
    fmin, fmax = float(np.min(s.freqs)), float(np.max(s.freqs))
    a = torch.floor(v * (fmin * g)) + nv // 2
    b = torch.floor(v * (fmax * g)) + nv // 2
    lo, hi = torch.minimum(a, b) - 1, torch.maximum(a, b) + 1
    keep = torch.zeros_like(lo, dtype=torch.bool)
    for p in planes:
        keep |= (lo <= p) & (p <= hi)
    return torch.nonzero(keep).flatten()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_alma_full_size_sampled_planes(V, alma, prec):
    from paper_2609_01897_gb300 import synth
    p = V.PREC_MIXED if prec == "mixed" else V.PREC_FP64
    st = V.Stack(alma.nu, alma.nv, alma.nrest, alma.npol, alma.du, alma.dv, central_freq=alma.central_freq,
                 precision=p)
    for s in alma.spws:
        st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z)
    st.run()
    cube = st.read_cube(f64=True)
    stats = st.stats()
    f0, df = st.lattice()
    st.close()
    sel = torch.tensor(PLANES, device="cuda")
    g = {k: v.index_select(0, sel).cpu().numpy() for k, v in cube.items()}
    del cube
    g["sum_wv"] = g["sum_wv"][..., 0] + 1j * g["sum_wv"][..., 1]

    # the oracle on the rows that can reach the sampled planes
    sub = []
    for s in alma.spws:
        idx = _rows_reaching(s, PLANES, alma.nv, alma.dv)
        sub.append(synth.SourceSpw(s.uvw.index_select(0, idx), s.freqs, s.vis.index_select(0, idx),
                                   s.weights.index_select(0, idx), s.flags.index_select(0, idx),
                                   s.l, s.m, s.z))
    wl = synth.Workload(alma.name, alma.nu, alma.nv, alma.nrest, alma.npol, alma.du, alma.dv,
                        alma.central_freq, sub, rest_df=df, rest_f0=f0)
    o = H.run_oracle(wl, iv_select=PLANES, nthreads=16)
    errs = H.compare(g, o, H.TOL_MIXED if prec == "mixed" else H.TOL_FP64, what="alma " + prec)
    assert o["count"].sum() > 1e6
    print("alma %s worst errors %s" % (prec, errs))

    # counters against properties of the inputs
    n_vis = n_flag = 0
    for s in alma.spws:
        j0, nb, _ = V.plan_channels(s.freqs, s.z, f0, df, alma.nrest, V.BIN_OVERLAP)
        ch = torch.as_tensor(np.nonzero(nb > 0)[0], device="cuda")
        n_vis += int(s.vis.shape[0]) * int(ch.numel()) * int(s.vis.shape[2])
        n_flag += int(s.flags.index_select(1, ch).sum()) if ch.numel() else 0
    assert stats["n_vis"] == n_vis
    assert stats["n_flagged"] == n_flag
    assert stats["n_dropped_uv"] == 0
    assert stats["n_stacked"] == n_vis - n_flag
