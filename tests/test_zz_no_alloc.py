"""vista_stack_noalloc: stacking without any allocation, for callers that
cannot call cudaMalloc (device memory owned by another allocator, or no
allocation allowed once running).  Called through the C ABI twice in a row,
its output must match the FP64 oracle and the regular open/add/run/read path
on the same window within the tolerance the parity tests use; further cases
cover flags that are not whole words per row (copied into the scratch array
first), 16-bit storage and a single polarisation.

Collected last on purpose (file name): a failure here leaves every other
test already run."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_01897_gb300 import build
    build.build()
    from paper_2609_01897_gb300 import vista
    vista.lib()
    return vista


def _regular(V, wl, s, f0, df):
    st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, rest_f0=f0, rest_df=df)
    st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z)
    st.run()
    out = st.read_cube()
    st.close()
    return out


def _noalloc(V, wl, s, f0, df, vis=None, vis_type=None, scale=1.0):
    nv, nu, nrest, npol = wl.nv, wl.nu, wl.nrest, wl.npol
    cube4 = torch.zeros((nv, nu, nrest, npol, 4), dtype=torch.float32, device="cuda")
    count = torch.zeros((nv, nu, nrest, npol), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    cd = V.CubeDesc(nu, nv, nrest, npol, wl.du, wl.dv, f0, df, 0.0, V.BIN_OVERLAP, V.PREC_MIXED, 0, 0, stream)
    f = np.ascontiguousarray(s.freqs, dtype=np.float64)
    vis = s.vis if vis is None else vis
    sd = V.SourceDesc(int(s.vis.shape[0]), int(s.vis.shape[1]), int(s.vis.shape[2]), s.uvw.data_ptr(),
                      f.ctypes.data, vis.data_ptr(), V.VIS_C64 if vis_type is None else vis_type, scale,
                      s.weights.data_ptr(), s.flags.data_ptr(), None, s.l, s.m, s.z, V.MEM_DEVICE, 0)
    rc = V.lib().vista_stack_noalloc(C.byref(cd), C.byref(sd), cube4.data_ptr(), count.data_ptr())
    assert rc == V.VISTA_OK, V.last_error(None)
    return cube4, count


def _against_oracle(wl, s, f0, df, cube4, count, dequant=None):
    """The no-allocation cube against the FP64 oracle stacking the same
    window alone: counts exact, sums within the parity tolerance."""
    from oracle import oracle as O
    from tests import gpu_helpers as H
    vis = s.vis.cpu().numpy() if dequant is None else dequant
    src = O.Source(s.uvw.cpu().numpy(), s.freqs, vis, s.weights.cpu().numpy(), s.flags.cpu().numpy(),
                   s.l, s.m, s.z)
    cube = O.make_cube(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, f0, df, 0, 0)
    o = O.stack(cube, [src], with_abs=True)
    c4 = cube4.double().cpu().numpy()
    g = {"sum_wv": c4[..., 0] + 1j * c4[..., 1], "sum_w": c4[..., 2], "sum_wvv": c4[..., 3],
         "count": count.cpu().numpy().astype(np.uint64)}
    assert int(o["count"].sum()) > 0
    return H.compare(g, o, TOL, what="no-allocation vs oracle")


def test_noalloc_matches_regular_path_twice(V):
    from oracle import oracle as O
    from paper_2609_01897_gb300 import synth
    wl = synth.tiny("cuda")
    f0, df = O.auto_lattice([s.freqs for s in wl.spws], [s.z for s in wl.spws], wl.nrest, wl.central_freq)
    for s in wl.spws[:2]:                      # two calls in a row on the shared scratch
        ref = _regular(V, wl, s, f0, df)
        cube4, count = _noalloc(V, wl, s, f0, df)
        assert int(count.sum()) > 0
        _against_oracle(wl, s, f0, df, cube4, count)
        assert torch.equal(count, ref["count"])
        w_ref, w = ref["sum_w"].double(), cube4[..., 2].double()
        vv_ref, vv = ref["sum_wvv"].double(), cube4[..., 3].double()
        assert ((w - w_ref).abs() <= TOL * w_ref.abs()).all()
        assert ((vv - vv_ref).abs() <= TOL * vv_ref.abs()).all()
        # sum W w V: scale sqrt(sum W w * sum W w |V|^2) >= sum W w |V| (Cauchy-Schwarz)
        scale = (w_ref * vv_ref).sqrt()
        for c in (0, 1):
            d = (cube4[..., c].double() - ref["sum_wv"][..., c].double()).abs()
            assert (d <= TOL * scale + 1e-30).all()


def test_noalloc_rejects_what_it_cannot_hold(V):
    from oracle import oracle as O
    from paper_2609_01897_gb300 import synth
    wl = synth.tiny("cuda")
    f0, df = O.auto_lattice([s.freqs for s in wl.spws], [s.z for s in wl.spws], wl.nrest, wl.central_freq)
    s = wl.spws[0]
    big = synth.SourceSpw(s.uvw.repeat(200, 1), s.freqs, s.vis.repeat(200, 1, 1), s.weights.repeat(200, 1),
                          s.flags.repeat(200, 1, 1), s.l, s.m, s.z)
    nv, nu, nrest, npol = wl.nv, wl.nu, wl.nrest, wl.npol
    cube4 = torch.zeros((nv, nu, nrest, npol, 4), dtype=torch.float32, device="cuda")
    count = torch.zeros((nv, nu, nrest, npol), dtype=torch.int32, device="cuda")
    cd = V.CubeDesc(nu, nv, nrest, npol, wl.du, wl.dv, f0, df, 0.0, V.BIN_OVERLAP, V.PREC_MIXED, 0,
                    0, torch.cuda.current_stream().cuda_stream)
    f = np.ascontiguousarray(big.freqs, dtype=np.float64)
    sd = V.SourceDesc(int(big.vis.shape[0]), int(big.vis.shape[1]), int(big.vis.shape[2]), big.uvw.data_ptr(),
                      f.ctypes.data, big.vis.data_ptr(), V.VIS_C64, 1.0, big.weights.data_ptr(),
                      big.flags.data_ptr(), None, big.l, big.m, big.z, V.MEM_DEVICE, 0)
    # 180k rows x 2 channel chunks of row records alone exceed the 8 MiB array
    rc = V.lib().vista_stack_noalloc(C.byref(cd), C.byref(sd), cube4.data_ptr(), count.data_ptr())
    assert rc == V.E_RANGE
    assert "scratch" in V.last_error(None)
    assert int(count.sum()) == 0


def test_noalloc_unaligned_flags_half_storage_single_pol(V):
    """Windows whose flag rows are not whole 4-byte words (one pol, an odd
    channel count: the call first copies the flags it reads into the scratch
    array with a word-aligned pitch), then a 16-bit (FP16 pairs) window:
    each against the oracle, two calls in a row each."""
    from oracle import oracle as O
    from paper_2609_01897_gb300 import synth
    from tests import gpu_helpers as H
    wl = synth.random_case(71, "cuda", nsrc=3, max_rows=40, nchan_choices=(33, 63, 130), npol_choices=(1,),
                           flag_frac=0.1)
    wl.npol = 1
    f0, df = O.auto_lattice([s.freqs for s in wl.spws], [s.z for s in wl.spws], wl.nrest, wl.central_freq)
    odd = [s for s in wl.spws if s.vis.shape[0] > 0 and (s.vis.shape[1] * s.vis.shape[2]) % 4 != 0]
    assert odd, "the case must hold a window with flag rows that are not whole words"
    for s in odd[:2]:
        for _ in range(2):
            cube4, count = _noalloc(V, wl, s, f0, df)
            _against_oracle(wl, s, f0, df, cube4, count)
    # FP16 pairs with a per-window power-of-two scale, against the oracle on the stored values
    wl2 = synth.tiny("cuda")
    f0, df = O.auto_lattice([s.freqs for s in wl2.spws], [s.z for s in wl2.spws], wl2.nrest, wl2.central_freq)
    s = wl2.spws[3]
    q, scale, deq = H.quantise(s.vis, "f16")
    for _ in range(2):
        cube4, count = _noalloc(V, wl2, s, f0, df, vis=q, vis_type=V.VIS_F16X2, scale=scale)
        _against_oracle(wl2, s, f0, df, cube4, count, dequant=deq)
