"""Shared helpers of the GPU parity tests: run a synthetic workload through
libvista (C ABI via the Python binding) and through the FP64 oracle, and
compare with the tolerances the tests state."""
import math

import numpy as np
import torch

from oracle import oracle as O
from paper_2609_01897_gb300 import vista as V

C_LIGHT = 299792458.0

# Tolerances (relative, see the parity metric of the scope table):
#   counts and bins exact; sum_w, sum_wvv relative 1e-5; sum_wv scale-aware:
#   |d sum_wv| <= 1e-5 * sum W w |V| (the cancellation-aware form).
TOL_MIXED = 1e-5
TOL_FP64 = 1e-9
PHASE_TOL_MIXED = 1e-5   # rad
PHASE_TOL_FP64 = 1e-9


def oracle_sources(wl, dequant=None, reproject=None):
    """Host copies of a workload's windows as oracle sources.  dequant:
    optional dict id(spw) -> complex128 array replacing vis (16-bit inputs);
    reproject: optional per-window (ra0, dec0, ra1, dec1) (Eq. 1)."""
    out = []
    for i, s in enumerate(wl.spws):
        vis = s.vis.cpu().numpy() if dequant is None else dequant[id(s)]
        flags = None if s.flags is None else s.flags.cpu().numpy()
        out.append(O.Source(s.uvw.cpu().numpy(), s.freqs, vis, s.weights.cpu().numpy(), flags,
                            s.l, s.m, s.z, s.pol_map, radec=None if reproject is None else reproject[i]))
    return out


def lattice_of(wl):
    if wl.rest_df > 0:
        return wl.rest_f0, wl.rest_df
    return O.auto_lattice([s.freqs for s in wl.spws], [s.z for s in wl.spws], wl.nrest, wl.central_freq)


def run_gpu(wl, precision=V.PREC_MIXED, bin_mode=V.BIN_OVERLAP, fold=False, tuning=None,
            host_mem=False, vis_override=None, scales=None, f64=True, reproject=None):
    st = V.Stack(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, rest_f0=wl.rest_f0,
                 rest_df=wl.rest_df, central_freq=wl.central_freq, bin_mode=bin_mode,
                 precision=precision, hermitian_fold=fold)
    try:
        if tuning:
            st.set_tuning(**tuning)
        for i, s in enumerate(wl.spws):
            vis = s.vis if vis_override is None else vis_override[i]
            args = [s.uvw, s.freqs, vis, s.weights, s.flags]
            if host_mem:
                args = [a.cpu().pin_memory() if isinstance(a, torch.Tensor) else a for a in args]
            st.add_source(*args, l=s.l, m=s.m, z=s.z, pol_map=s.pol_map,
                          vis_scale=1.0 if scales is None else scales[i],
                          reproject=None if reproject is None else reproject[i])
        st.run()
        cube = st.read_cube(device=True, f64=f64)
        out = {k: v.cpu().numpy() for k, v in cube.items()}
        out["sum_wv"] = out["sum_wv"][..., 0] + 1j * out["sum_wv"][..., 1]
        out["stats"] = st.stats()
        out["lattice"] = st.lattice()
        return out
    finally:
        st.close()


def run_oracle(wl, bin_mode=V.BIN_OVERLAP, fold=False, iv_select=None, dequant=None, nthreads=4,
               reproject=None):
    f0, df = lattice_of(wl)
    cube = O.make_cube(wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, f0, df, bin_mode, 1 if fold else 0)
    srcs = oracle_sources(wl, dequant, reproject)
    out = O.stack(cube, srcs, iv_select=iv_select, nthreads=nthreads, with_abs=True)
    out["lattice"] = (f0, df)
    return out


def compare(gpu, orc, tol, planes=None, what=""):
    """Assert parity; returns a dict of the observed worst errors."""
    g = {k: (gpu[k] if planes is None else gpu[k][planes]) for k in ("sum_wv", "sum_w", "sum_wvv", "count")}
    cnt_o = orc["count"].astype(np.int64)
    cnt_g = g["count"].astype(np.int64)
    bad = np.argwhere(cnt_o != cnt_g)
    assert bad.size == 0, "%s: %d count mismatches, first %s (oracle %d, gpu %d)" % (
        what, len(bad), bad[0], cnt_o[tuple(bad[0])], cnt_g[tuple(bad[0])])
    errs = {}
    for key in ("sum_w", "sum_wvv"):
        o, x = orc[key], g[key]
        scale = np.abs(o)
        err = np.abs(x - o)
        ok = err <= tol * scale + 1e-300
        assert ok.all(), "%s: %s rel err %.3g > %.1g at %s" % (
            what, key, float((err / np.maximum(scale, 1e-300)).max()), tol, np.argwhere(~ok)[0])
        nz = scale > 0
        errs[key] = float((err[nz] / scale[nz]).max()) if nz.any() else 0.0
    o, x, sa = orc["sum_wv"], g["sum_wv"], orc["sum_wabs"]
    err = np.abs(x - o)
    ok = err <= tol * sa + 1e-300
    assert ok.all(), "%s: sum_wv scale-aware err %.3g > %.1g at %s" % (
        what, float((err / np.maximum(sa, 1e-300)).max()), tol, np.argwhere(~ok)[0])
    nz = sa > 0
    errs["sum_wv"] = float((err[nz] / sa[nz]).max()) if nz.any() else 0.0
    return errs


def stats_equal(gpu, orc):
    og = orc["stats"]
    for k in ("n_vis", "n_flagged", "n_dropped_uv", "n_stacked"):
        assert int(gpu["stats"][k]) == int(og[k]), (k, gpu["stats"][k], og[k])


def phase_error(p_gpu, p_orc):
    """Largest |arg(p_gpu conj(p_orc))| in radians."""
    z = p_gpu * np.conj(p_orc)
    return float(np.abs(np.angle(z)).max()) if z.size else 0.0


def quantise(vis, kind):
    """Per-window scaled 16-bit storage: returns (tensor [.., 2], scale, dequantised complex128)."""
    re = torch.view_as_real(vis)
    amax = float(re.abs().max()) if re.numel() else 1.0
    e = math.ceil(math.log2(amax)) if amax > 0 else 0
    # power-of-two scales are exact in FP32 and FP64 alike
    scale = 2.0 ** (e - 15) if kind == "f16" else 2.0 ** e
    q = (re / scale).to(torch.float16 if kind == "f16" else torch.bfloat16)
    deq = q.to(torch.float64) * scale
    deq_c = torch.view_as_complex(deq.contiguous()).cpu().numpy()
    return q.contiguous(), float(scale), deq_c
