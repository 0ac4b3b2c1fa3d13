"""The batched uneven stack (many sources of uneven rows, 1-4 windows of
128-3840 channels, 2 or 4 pols, windows aliased into a device pool):

* a reduced instance (30 sources, median 600 rows) against the FP64 oracle,
  every cube entry;
* the full instance (2000 sources, ~1.9e11 visibilities reach the cube, the
  launch configuration bench.py times) stacked twice into one cube (twice the
  depth: the accuracy of the mixed cube must not depend on it) against the
  plain FP64 GPU path doing the same, on every cube entry: counts identical,
  sums within 1e-5 of the Cauchy-Schwarz scale sqrt(sum_w * sum_wvv) >=
  sum W w |V| (the cancellation-aware bound, computed from the cube itself),
  and visibility counters that add up."""
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


def test_batched_reduced_against_oracle(V):
    from paper_2609_01897_gb300 import synth
    wl = synth.batched("cuda", n_sources=30, median_rows=600, pool_gb=0.5)
    g = H.run_gpu(wl)
    o = H.run_oracle(wl, nthreads=16)
    assert o["count"].sum() > 0
    H.compare(g, o, H.TOL_MIXED, what="batched reduced")
    H.stats_equal(g, o)


def test_batched_full_twice_mixed_against_fp64(V):
    from paper_2609_01897_gb300 import synth
    free, _ = torch.cuda.mem_get_info()
    if free < 150e9:
        pytest.skip("needs ~150 GB of free device memory")
    wl = synth.batched("cuda")
    cubes, stats = {}, {}
    for prec in (V.PREC_MIXED, V.PREC_FP64):
        st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, central_freq=wl.central_freq, precision=prec)
        try:
            for _ in range(2):
                for s in wl.spws:
                    st.add_source(s.uvw, s.freqs, s.vis, s.weights, s.flags, l=s.l, m=s.m, z=s.z,
                                  pol_map=s.pol_map)
                st.run()
            cubes[prec] = st.read_cube(device=True, f64=True)
            stats[prec] = st.stats()
        finally:
            st.close()
    m, d = cubes[V.PREC_MIXED], cubes[V.PREC_FP64]
    assert torch.equal(m["count"], d["count"])
    assert int(d["count"].sum()) > 0
    scale = torch.sqrt(d["sum_w"] * d["sum_wvv"])
    def worst(err, ref):
        rel = err / ref.clamp_min(1e-300)
        i = int(torch.argmax(rel))
        return "max rel err %.3g at entry %d (count %d, value %.6g)" % (
            float(rel.flatten()[i]), i, int(d["count"].flatten()[i]), float(ref.flatten()[i]))
    for key in ("sum_w", "sum_wvv"):
        err = (m[key] - d[key]).abs()
        print("batched full x2, %s: %s" % (key, worst(err, d[key].abs())))
        assert bool((err <= H.TOL_MIXED * d[key].abs() + 1e-300).all()), key + ": " + worst(err, d[key].abs())
    err = (m["sum_wv"] - d["sum_wv"]).abs().amax(dim=-1)
    print("batched full x2, sum_wv: %s" % worst(err, scale))
    assert bool((err <= H.TOL_MIXED * scale + 1e-300).all()), "sum_wv: " + worst(err, scale)
    sm, sd = stats[V.PREC_MIXED], stats[V.PREC_FP64]
    for k in ("n_vis", "n_flagged", "n_dropped_uv", "n_stacked"):
        assert int(sm[k]) == int(sd[k]), (k, sm[k], sd[k])
    # every stacked visibility adds 1 to the count of each of its 1..VISTA_MAX_BINS rest bins
    n_stk, n_cnt = int(sd["n_stacked"]), int(d["count"].sum())
    assert 0 < n_stk <= n_cnt <= 4 * n_stk
    assert int(sd["n_vis"]) == int(sd["n_flagged"]) + int(sd["n_dropped_uv"]) + n_stk
