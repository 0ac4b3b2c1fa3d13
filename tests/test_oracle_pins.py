"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics -- never against the oracle itself or the GPU library.

P1 point source -> real flux (sign of Eq. 2)     P5 Eq. 3 literal, one row
P2 z-invariance of phase and cell (Eq. 1/2 frame) P6 brute-force enumeration
P3 line stacking across redshifts (Sec. 3.1)      P7 zero offset is the identity
P4 weight conservation (Eq. 4 partition of unity) P8 all-flagged -> empty cube
plus the hand-derived Eq. 4 golden values, closed forms of the channel widths,
the auto lattice (Sec. 3.1) and the uv cell, and the Hermitian fold.
"""
import cmath
import math
import os
from fractions import Fraction

import numpy as np
import pytest

C = 299792458.0
HERE = os.path.dirname(os.path.abspath(__file__))
ARCSEC = math.pi / 180 / 3600


def _uvw(n, rng, scale=3000.0):
    return rng.uniform(-scale, scale, size=(n, 3))


def _point_vis(uvw, freqs, l0, m0, S, npol):
    """Measurement equation of a point source of flux S at (l0, m0), written
    out independently of the oracle: V = S exp(-2 pi i nu/c (u l + v m + w(n-1)))."""
    n0 = math.sqrt(1 - l0 * l0 - m0 * m0) - 1
    out = np.empty((uvw.shape[0], freqs.size, npol), dtype=np.complex128)
    for r in range(uvw.shape[0]):
        g = uvw[r, 0] * l0 + uvw[r, 1] * m0 + uvw[r, 2] * n0
        for k, f in enumerate(freqs):
            out[r, k, :] = S * cmath.exp(-2j * math.pi * g * f / C)
    return out


def _src(o, uvw, freqs, vis, l, m, z, weights=None, flags=None, pol_map=None):
    nrow, nchan, npol = vis.shape
    if weights is None:
        weights = np.ones((nrow, npol), dtype=np.float32)
    return o.Source(uvw, freqs, vis, weights, flags, l, m, z, pol_map)


# ----------------------------------------------------------------- Eq. 4 golden

def _golden_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "eq4_overlap_weights.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            case, freqs, z, f0, df, nrest, k, j, w = line.split()
            rows.append((case, [float(x) for x in freqs.split(",")], float(z), float(f0),
                         float(df), int(nrest), int(k), int(j), float(w)))
    return rows


def test_eq4_golden(oracle_mod):
    rows = _golden_rows()
    assert len(rows) == 15
    cases = {}
    for r in rows:
        cases.setdefault(r[0], []).append(r)
    for case, rs in cases.items():
        _, freqs, z, f0, df, nrest, _, _, _ = rs[0]
        W = oracle_mod.rest_weights(np.array(freqs), z, f0, df, nrest, 0)
        expect = np.zeros_like(W)
        for r in rs:
            expect[r[6], r[7]] = r[8]
        np.testing.assert_allclose(W, expect, rtol=1e-15, atol=0, err_msg="case " + case)


def test_channel_widths_closed_form(oracle_mod):
    f = 86e9 + 488281.25 * np.arange(33)
    np.testing.assert_array_equal(oracle_mod.channel_widths(f), np.full(33, 488281.25))
    np.testing.assert_array_equal(oracle_mod.channel_widths(f[::-1].copy()), np.full(33, 488281.25))
    g = np.array([1.0, 2.0, 4.0, 8.0, 16.0])
    np.testing.assert_array_equal(oracle_mod.channel_widths(g), [1.0, 1.5, 3.0, 6.0, 8.0])


def test_auto_lattice_closed_form(oracle_mod):
    fa = 100e9 + 15.625e6 * np.arange(10)
    fb = 200e9 + 31.25e6 * np.arange(5)
    f0, df = oracle_mod.auto_lattice([fa, fb], [2.0, 0.5], 64, 345e9)
    # widest rest-frame channel: max(15.625 MHz * 3, 31.25 MHz * 1.5) = 46.875 MHz
    assert df == 46.875e6
    assert f0 == 345e9 - 32 * 46.875e6


def test_partition_of_unity(oracle_mod):
    """Sum_j w_kj = 1 for every channel well inside the lattice (Eq. 4 with
    the rest-frame denominator), for random non-uniform axes and z."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        n = int(rng.integers(2, 40))
        f = 300e9 + np.cumsum(rng.uniform(1e6, 3e7, size=n))
        z = float(rng.uniform(0, 4))
        dnu = oracle_mod.channel_widths(f)
        df = float(dnu.max() * (1 + z) * rng.uniform(1.0, 3.0))
        f0 = f.min() * (1 + z) - 40 * df
        W = oracle_mod.rest_weights(f, z, f0, df, 200, 0)
        np.testing.assert_allclose(W.sum(axis=1), 1.0, rtol=1e-12)
        assert (np.count_nonzero(W, axis=1) <= 2).all()


# ----------------------------------------------------------------- P1 / P7 / P2

@pytest.mark.parametrize("offset", [10 * ARCSEC, 60 * ARCSEC])
def test_p1_point_source_becomes_real(oracle_mod, offset):
    rng = np.random.default_rng(1)
    uvw = _uvw(25, rng, 8000.0)
    freqs = 340e9 + 1.953125e6 * np.arange(16)
    l0, m0, S = offset, -0.7 * offset, 3.5e-3
    vis = _point_vis(uvw, freqs, l0, m0, S, 2)
    src = _src(oracle_mod, uvw, freqs, vis, l0, m0, 2.5)
    ph = oracle_mod.phasors(src)
    shifted = vis[..., 0] * ph
    np.testing.assert_allclose(shifted.real, S, rtol=1e-9)
    np.testing.assert_allclose(shifted.imag, 0.0, atol=1e-9 * S)
    # and through the stack: every cell's weighted mean is S + 0i
    f0, df = oracle_mod.auto_lattice([freqs], [2.5], 64, 340e9 * 3.5)
    du = 2 * 1.01 * np.abs(uvw[:, :2]).max() * freqs.max() / C / 32
    cube = oracle_mod.make_cube(32, 32, 64, 2, du, du, f0, df, 0, 0)
    out = oracle_mod.stack(cube, [src])
    m = out["sum_w"] > 0
    assert m.sum() > 50
    np.testing.assert_allclose((out["sum_wv"][m] / out["sum_w"][m]).real, S, rtol=1e-9)
    np.testing.assert_allclose((out["sum_wv"][m] / out["sum_w"][m]).imag, 0, atol=1e-9 * S)


def test_p1_wrong_sign_would_fail(oracle_mod):
    """The opposite sign convention leaves a phase of 2x the delay: make sure
    the point-source data are not trivially real (the pin has teeth)."""
    rng = np.random.default_rng(2)
    uvw = _uvw(5, rng, 2000.0)
    freqs = 230e9 + 15.625e6 * np.arange(4)
    vis = _point_vis(uvw, freqs, 10 * ARCSEC, 5 * ARCSEC, 1.0, 1)
    assert np.abs(vis.imag).max() > 0.1


def test_p7_zero_offset_identity(oracle_mod):
    rng = np.random.default_rng(3)
    uvw = _uvw(10, rng)
    freqs = 100e9 + 15.625e6 * np.arange(8)
    vis = rng.normal(size=(10, 8, 2)) + 1j * rng.normal(size=(10, 8, 2))
    src = _src(oracle_mod, uvw, freqs, vis, 0.0, 0.0, 1.0)
    ph = oracle_mod.phasors(src)
    assert (ph.real == 1.0).all() and (ph.imag == 0.0).all()


def test_p2_z_invariance(oracle_mod):
    rng = np.random.default_rng(4)
    uvw = _uvw(12, rng)
    freqs = 112e9 + 15.625e6 * np.arange(12)
    vis = np.ones((12, 12, 1), dtype=np.complex64)
    cube = oracle_mod.make_cube(64, 64, 32, 1, 40.0, 40.0, 300e9, 50e6, 0, 0)
    ref_ph = ref_cells = None
    for z in (0.0, 1.0, 3.0):
        src = _src(oracle_mod, uvw, freqs, vis, 20 * ARCSEC, -5 * ARCSEC, z)
        ph, cl = oracle_mod.phasors(src), oracle_mod.cells(cube, src)
        if ref_ph is None:
            ref_ph, ref_cells = ph, cl
        np.testing.assert_array_equal(ph, ref_ph)
        np.testing.assert_array_equal(cl, ref_cells)


def test_uv_cell_closed_form(oracle_mod):
    """cell = floor(u nu / (c du)) + N/2, checked with exact rational arithmetic
    wherever u nu/(c du) is not within 1e-9 of an integer."""
    rng = np.random.default_rng(6)
    uvw = _uvw(40, rng, 900.0)
    freqs = 230e9 + 15.625e6 * np.arange(7)
    du, N = 17000.0, 64
    cube = oracle_mod.make_cube(N, N, 8, 1, du, du, 1e9, 1e9, 0, 0)
    src = _src(oracle_mod, uvw, freqs, np.ones((40, 7, 1)), 0.0, 0.0, 0.0)
    cl = oracle_mod.cells(cube, src)
    checked = 0
    for r in range(40):
        for k in range(7):
            for ax in (0, 1):
                x = Fraction(uvw[r, ax]) * Fraction(freqs[k]) / (Fraction(C) * Fraction(du))
                fl = math.floor(x)
                if abs(x - fl) < 1e-9 or abs(x - fl - 1) < 1e-9:
                    continue
                inside = -N // 2 <= fl < N // 2
                other = cl[r, k, 1 - ax]
                if inside and other >= 0:
                    assert cl[r, k, ax] == fl + N // 2
                    checked += 1
                if not inside:
                    assert cl[r, k, ax] == -1
    assert checked > 300


# ----------------------------------------------------------------- P3 line stacking

def test_p3_line_lands_in_one_bin(oracle_mod):
    nu_L = 345.796e9
    df_obs = 15.625e6
    zs = [2.0, 2.37, 2.81, 3.0]
    srcs, freq_list = [], []
    for i, z in enumerate(zs):
        freqs = nu_L / (1 + z) + df_obs * (np.arange(21) - 10)   # channel 10 holds the line
        vis = np.zeros((3, 21, 1), dtype=np.complex128)
        vis[:, 10, 0] = 1.0
        uvw = np.array([[10.0, 20.0, 0.0], [30.0, -5.0, 1.0], [-7.0, 4.0, 0.5]])
        srcs.append(_src(oracle_mod, uvw, freqs, vis, 0.0, 0.0, z))
        freq_list.append(freqs)
    f0, df = oracle_mod.auto_lattice(freq_list, zs, 64, nu_L)
    f0 = f0 - 0.5 * df          # put nu_L at the centre of bin 32
    jL = 32
    for mode in (1, 0):
        cube = oracle_mod.make_cube(8, 8, 64, 1, 5000.0, 5000.0, f0, df, mode, 0)
        out = oracle_mod.stack(cube, srcs)
        per_j = np.abs(out["sum_wv"]).sum(axis=(0, 1, 3))
        if mode == 1:
            assert set(np.nonzero(per_j)[0]) == {jL}
            assert per_j[jL] == pytest.approx(12.0)
        else:
            # overlap mode: the line channel's rest-frame edges around nu_L
            # spread it over jL and at most one neighbour, with the Eq. 4
            # fractions computed here exactly.
            for s, z in zip(srcs, zs):
                one = oracle_mod.stack(cube, [s])
                pj = np.abs(one["sum_wv"]).sum(axis=(0, 1, 3))
                nz = set(np.nonzero(pj)[0])
                assert jL in nz and nz <= {jL - 1, jL, jL + 1}
                lo = (Fraction(nu_L / (1 + z)) - Fraction(df_obs) / 2) * Fraction(1 + z)
                hi = (Fraction(nu_L / (1 + z)) + Fraction(df_obs) / 2) * Fraction(1 + z)
                for j in nz:
                    ej, ej1 = Fraction(f0) + j * Fraction(df), Fraction(f0) + (j + 1) * Fraction(df)
                    w = max(Fraction(0), min(hi, ej1) - max(lo, ej)) / (hi - lo)
                    assert pj[j] == pytest.approx(3.0 * float(w), rel=1e-9)


# ----------------------------------------------------------------- P4 conservation

def test_p4_weight_conservation(oracle_mod):
    from paper_2609_01897_gb300 import synth
    w = synth.random_case(11, "cpu", nsrc=4, with_pol_map=False)
    srcs = [_src(oracle_mod, s.uvw.numpy(), s.freqs, s.vis.numpy(), s.l, s.m, s.z,
                 s.weights.numpy(), s.flags.numpy()) for s in w.spws]
    f0, df = oracle_mod.auto_lattice([s.freqs for s in w.spws], [s.z for s in w.spws],
                                     w.nrest, w.central_freq)
    cube = oracle_mod.make_cube(w.nu, w.nv, w.nrest, w.npol, w.du, w.dv, f0, df, 0, 0)
    out = oracle_mod.stack(cube, srcs)
    st = out["stats"]
    assert st["w_dropped_uv"] > 0 and st["w_dropped_rest"] > 0 and st["w_cube"] > 0
    total = st["w_cube"] + st["w_dropped_uv"] + st["w_dropped_rest"]
    assert total == pytest.approx(st["w_unflagged"], rel=1e-12)
    assert out["sum_w"].sum() == pytest.approx(st["w_cube"], rel=1e-12)
    # the unflagged weight is a plain sum over the inputs
    wu = 0.0
    for s in srcs:
        f = s.flags == 0
        wu += float((f * s.weights[:, None, :].astype(np.float64)).sum())
    assert st["w_unflagged"] == pytest.approx(wu, rel=1e-12)
    # thread count does not change anything
    out4 = oracle_mod.stack(cube, srcs, nthreads=4)
    for k in ("sum_wv", "sum_w", "sum_wvv", "count"):
        np.testing.assert_array_equal(out[k], out4[k])


# ----------------------------------------------------------------- P5 Eq. 3 literal

def test_p5_eq3_single_row(oracle_mod):
    """One row whose every channel falls in the same uv cell: the cube's
    sum_wv/sum_w per bin j is Eq. 3's V_out(j), computed here from Eqs. 3-4
    with the shifted visibilities taken from the point-source formula."""
    rng = np.random.default_rng(8)
    uvw = np.array([[3.0, -2.0, 0.7]])
    freqs = 100e9 + 15.625e6 * np.arange(9)
    vis = rng.normal(size=(1, 9, 1)) + 1j * rng.normal(size=(1, 9, 1))
    l0, m0, z = 8 * ARCSEC, 3 * ARCSEC, 2.3
    src = _src(oracle_mod, uvw, freqs, vis, l0, m0, z)
    df = 15.625e6 * (1 + z) * 1.7
    f0 = freqs[0] * (1 + z) - 2.3 * df
    cube = oracle_mod.make_cube(4, 4, 12, 1, 1e6, 1e6, f0, df, 0, 0)
    out = oracle_mod.stack(cube, [src])
    n1 = math.sqrt(1 - l0 * l0 - m0 * m0) - 1
    tau = 3.0 * l0 - 2.0 * m0 + 0.7 * n1
    Vs = [vis[0, k, 0] * cmath.exp(2j * math.pi * tau * freqs[k] / C) for k in range(9)]
    widths = [freqs[1] - freqs[0]] + [(freqs[k + 1] - freqs[k - 1]) / 2 for k in range(1, 8)] + [freqs[8] - freqs[7]]
    nz = np.nonzero(out["sum_w"][..., 0])
    assert len(set(zip(nz[0], nz[1]))) == 1
    iv, iu = nz[0][0], nz[1][0]
    for j in range(12):
        ej, ej1 = f0 + j * df, f0 + (j + 1) * df
        num = den = 0.0
        for k in range(9):
            lo = (freqs[k] - widths[k] / 2) * (1 + z)
            hi = (freqs[k] + widths[k] / 2) * (1 + z)
            w = max(0.0, min(hi, ej1) - max(lo, ej)) / (hi - lo)
            num += Vs[k] * w
            den += w
        if den == 0:
            assert out["sum_w"][iv, iu, j, 0] == 0
            continue
        got = out["sum_wv"][iv, iu, j, 0] / out["sum_w"][iv, iu, j, 0]
        assert abs(got - num / den) < 1e-10 * max(1.0, abs(num / den))


# ----------------------------------------------------------------- P6 brute force

@pytest.mark.parametrize("fold", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_p6_brute_force(oracle_mod, fold, mode):
    """<= 4 rows x 8 channels: direct enumeration with exp() of the full
    (unreduced) phase and Eq. 4 evaluated for every bin of the lattice."""
    rng = np.random.default_rng(9 + mode + 2 * fold)
    nrow, nchan, npol = 4, 8, 2
    uvw = _uvw(nrow, rng, 600.0)
    freqs = 230e9 + 31.25e6 * np.arange(nchan)
    vis = rng.normal(size=(nrow, nchan, npol)) + 1j * rng.normal(size=(nrow, nchan, npol))
    wts = rng.uniform(0.5, 2.0, size=(nrow, npol)).astype(np.float32)
    flags = (rng.random((nrow, nchan, npol)) < 0.15).astype(np.uint8)
    l0, m0, z = 12 * ARCSEC, -4 * ARCSEC, 1.7
    src = _src(oracle_mod, uvw, freqs, vis, l0, m0, z, wts, flags)
    N, nrest = 8, 24
    du = 2 * 1.05 * np.abs(uvw[:, :2]).max() * freqs.max() / C / N
    df = 31.25e6 * (1 + z) * 1.3
    f0 = freqs[0] * (1 + z) - 6.5 * df
    cube = oracle_mod.make_cube(N, N, nrest, npol, du, du, f0, df, mode, fold)
    out = oracle_mod.stack(cube, [src], with_abs=True)
    exp = np.zeros((N, N, nrest, npol), dtype=np.complex128)
    expw = np.zeros((N, N, nrest, npol))
    expa = np.zeros((N, N, nrest, npol))
    expc = np.zeros((N, N, nrest, npol), dtype=np.int64)
    n1 = math.sqrt(1 - l0 ** 2 - m0 ** 2) - 1
    widths = [freqs[1] - freqs[0]] + [(freqs[k + 1] - freqs[k - 1]) / 2 for k in range(1, nchan - 1)] + [freqs[-1] - freqs[-2]]
    for r in range(nrow):
        u, v, w = uvw[r]
        tau = u * l0 + v * m0 + w * n1
        flip = fold and (v < 0 or (v == 0 and u < 0))
        uu, vv = (-u, -v) if flip else (u, v)
        for k in range(nchan):
            iu = math.floor(uu * freqs[k] / C / du) + N // 2
            iv = math.floor(vv * freqs[k] / C / du) + N // 2
            if not (0 <= iu < N and 0 <= iv < N):
                continue
            ph = cmath.exp(2j * math.pi * tau * freqs[k] / C)
            for p in range(npol):
                if flags[r, k, p]:
                    continue
                Vs = vis[r, k, p] * ph
                if flip:
                    Vs = Vs.conjugate()
                for j in range(nrest):
                    if mode == 1:
                        rho = freqs[k] * (1 + z)
                        wk = 1.0 if f0 + j * df <= rho < f0 + (j + 1) * df else 0.0
                    else:
                        lo = (freqs[k] - widths[k] / 2) * (1 + z)
                        hi = (freqs[k] + widths[k] / 2) * (1 + z)
                        wk = max(0.0, min(hi, f0 + (j + 1) * df) - max(lo, f0 + j * df)) / (hi - lo)
                    if wk > 0:
                        exp[iv, iu, j, p] += wts[r, p] * wk * Vs
                        expw[iv, iu, j, p] += wts[r, p] * wk
                        expa[iv, iu, j, p] += wts[r, p] * wk * abs(vis[r, k, p])
                        expc[iv, iu, j, p] += 1
    np.testing.assert_array_equal(out["count"].astype(np.int64), expc)
    np.testing.assert_allclose(out["sum_w"], expw, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out["sum_wv"], exp, rtol=1e-9, atol=1e-9)
    # the scale of the sum_wv parity bound: sum of W w_kj |V| (|V'| = |V|)
    np.testing.assert_allclose(out["sum_wabs"], expa, rtol=1e-12, atol=1e-12)
    assert (out["sum_wabs"] >= np.abs(out["sum_wv"]) * (1 - 1e-12)).all()
    assert (out["sum_wabs"] > 0).sum() == (expc > 0).sum()


# ----------------------------------------------------------------- sampled planes

@pytest.mark.parametrize("fold", [0, 1])
@pytest.mark.parametrize("nthreads", [1, 3])
def test_iv_select_equals_full_cube_planes(oracle_mod, fold, nthreads):
    """Sampled mode (iv_select) accumulates exactly the chosen iv planes of the
    full cube: the same values bit for bit, in increasing iv, and nothing of
    the other planes.  The channel axis spans a 40 % fractional band, so a
    row's cell moves by several iv planes across its channels and many rows
    straddle a selected and an unselected plane."""
    rng = np.random.default_rng(77 + fold + 10 * nthreads)
    nchan, npol, N, nrest = 24, 2, 16, 20
    freqs = 100e9 + 1.75e9 * np.arange(nchan)
    srcs = []
    for s in range(3):
        nrow = 30
        uvw = _uvw(nrow, rng, 40.0)
        vis = rng.normal(size=(nrow, nchan, npol)) + 1j * rng.normal(size=(nrow, nchan, npol))
        wts = rng.uniform(0.5, 2.0, size=(nrow, npol)).astype(np.float32)
        flags = (rng.random((nrow, nchan, npol)) < 0.1).astype(np.uint8)
        srcs.append(_src(oracle_mod, uvw, freqs, vis, 3 * ARCSEC * s, -2 * ARCSEC, 0.3 + 0.1 * s, wts, flags))
    du = 2 * 1.01 * 40.0 * freqs.max() / C / N
    f0, df = oracle_mod.auto_lattice([freqs] * 3, [0.3, 0.4, 0.5], nrest, 140e9 * 1.4)
    cube = oracle_mod.make_cube(N, N, nrest, npol, du, du, f0, df, 0, fold)
    full = oracle_mod.stack(cube, srcs, nthreads=nthreads, with_abs=True)
    sel = [1, 4, 5, 8, 13]
    part = oracle_mod.stack(cube, srcs, iv_select=sel, nthreads=nthreads, with_abs=True)
    np.testing.assert_array_equal(part["planes"], sel)
    for k in ("sum_wv", "sum_w", "sum_wvv", "sum_wabs", "count"):
        assert part[k].shape[0] == len(sel)
        np.testing.assert_array_equal(part[k], full[k][sel])   # bit for bit
    assert part["count"].sum() > 0 and part["count"].sum() < full["count"].sum()
    # the sample has teeth: some rows put channels both in and out of the
    # selected planes
    straddle = 0
    gv = 1.0 / (C * du)
    for sc in srcs:
        for r in range(sc.uvw.shape[0]):
            v = sc.uvw[r, 1]
            u = sc.uvw[r, 0]
            if fold and (v < 0 or (v == 0 and u < 0)):
                v = -v
            ivs = {math.floor(v * (f * gv)) + N // 2 for f in freqs}
            straddle += bool(ivs & set(sel)) and bool(ivs - set(sel))
    assert straddle >= 10


# ----------------------------------------------------------------- Hermitian fold

def test_fold_conjugates(oracle_mod):
    """With the fold on, a sample from the lower half plane lands at -uv with
    the conjugate value: for a point source away from the shift centre the
    folded cell must hold the model evaluated at -uvw."""
    uvw = np.array([[120.0, -340.0, 5.0]])
    freqs = np.array([230e9, 230.03125e9])
    l0, m0 = 15 * ARCSEC, 9 * ARCSEC
    vis = _point_vis(uvw, freqs, l0, m0, 1.0, 1)
    src = _src(oracle_mod, uvw, freqs, vis, 0.0, 0.0, 0.0)
    du = 2000.0
    cube = oracle_mod.make_cube(512, 512, 4, 1, du, du, 229.99e9, 0.02e9, 1, 1)
    out = oracle_mod.stack(cube, [src])
    expect = _point_vis(-uvw, freqs, l0, m0, 1.0, 1)
    for k in range(2):
        iu = math.floor(-uvw[0, 0] * freqs[k] / C / du) + 256
        iv = math.floor(-uvw[0, 1] * freqs[k] / C / du) + 256
        assert iv >= 256
        j = math.floor((freqs[k] - 229.99e9) / 0.02e9)
        got = out["sum_wv"][iv, iu, j, 0] / out["sum_w"][iv, iu, j, 0]
        assert abs(got - expect[0, k, 0]) < 1e-9


# ----------------------------------------------------------------- P8 flags

def test_p8_all_flagged(oracle_mod):
    rng = np.random.default_rng(10)
    uvw = _uvw(6, rng, 100.0)
    freqs = 100e9 + 15.625e6 * np.arange(5)
    vis = np.ones((6, 5, 2))
    flags = np.ones((6, 5, 2), dtype=np.uint8)
    src = _src(oracle_mod, uvw, freqs, vis, 0.0, 0.0, 2.0, flags=flags)
    cube = oracle_mod.make_cube(16, 16, 8, 2, 1e3, 1e3, 299.9e9, 1e8, 0, 0)
    out = oracle_mod.stack(cube, [src])
    assert not out["sum_w"].any() and not out["count"].any() and not out["sum_wv"].any()
    assert out["stats"]["n_flagged"] == out["stats"]["n_vis"] > 0
    assert out["stats"]["n_stacked"] == 0


# ----------------------------------------------------------------- Eq. 1 re-projection

def _frame(ra, dec):
    """The uvw frame of a phase centre built without the oracle's closed form:
    w = the unit vector toward (ra, dec), u = the normalised cross product of
    the pole with w (east), v = w x u (north)."""
    w = np.array([math.cos(dec) * math.cos(ra), math.cos(dec) * math.sin(ra), math.sin(dec)])
    e = np.cross(np.array([0.0, 0.0, 1.0]), w)
    u = e / np.linalg.norm(e)
    v = np.cross(w, u)
    return np.stack([u, v, w])


def _centres(rng, n, spread):
    out = []
    for _ in range(n):
        ra0, dec0 = rng.uniform(0, 2 * math.pi), rng.uniform(-1.3, 1.3)
        out.append((ra0, dec0, ra0 + rng.uniform(-spread, spread), dec0 + rng.uniform(-spread, spread)))
    return out


def test_reprojection_rotation_against_numeric_frames(oracle_mod):
    """R = M(ra1, dec1) M(ra0, dec0)^T against frames built from cross
    products of unit vectors: orthonormal, det +1, the same matrix."""
    rng = np.random.default_rng(40)
    for ra0, dec0, ra1, dec1 in _centres(rng, 20, 0.3):
        R = oracle_mod.rotation(ra0, dec0, ra1, dec1)
        ref = _frame(ra1, dec1) @ _frame(ra0, dec0).T
        np.testing.assert_allclose(R, ref, atol=1e-14)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-14


def test_reprojection_offset_is_the_rotated_w_axis(oracle_mod):
    """(l, m) of the stacking position and R's last row are the same vector
    (two derivations), with n = sqrt(1 - l^2 - m^2): so w' - w is the delay
    of Eq. 2."""
    rng = np.random.default_rng(41)
    for ra0, dec0, ra1, dec1 in _centres(rng, 50, 0.05):
        l, m = oracle_mod.offset(ra0, dec0, ra1, dec1)
        R = oracle_mod.rotation(ra0, dec0, ra1, dec1)
        assert abs(R[2, 0] - l) < 1e-15 and abs(R[2, 1] - m) < 1e-15
        assert abs(R[2, 2] - math.sqrt(1 - l * l - m * m)) < 1e-14
        # the same offsets from the numerical frames
        s1 = _frame(ra1, dec1)[2]
        F0 = _frame(ra0, dec0)
        assert abs(F0[0] @ s1 - l) < 1e-14 and abs(F0[1] @ s1 - m) < 1e-14


def test_reprojection_same_centre_is_identity(oracle_mod):
    rng = np.random.default_rng(42)
    for ra0, dec0, _, _ in _centres(rng, 10, 0.0):
        assert oracle_mod.offset(ra0, dec0, ra0, dec0) == (0.0, 0.0)
        np.testing.assert_allclose(oracle_mod.rotation(ra0, dec0, ra0, dec0), np.eye(3), atol=1e-15)


def test_reprojected_point_source_is_real(oracle_mod):
    """A point source at (ra1, dec1) observed with phase centre (ra0, dec0)
    (visibilities from the numerically built frames) stacks to S + 0i when the
    oracle re-projects to (ra1, dec1)."""
    rng = np.random.default_rng(43)
    ra0, dec0 = 1.1, -0.5
    ra1, dec1 = ra0 + 40 * ARCSEC / math.cos(dec0), dec0 - 25 * ARCSEC
    s1 = _frame(ra1, dec1)[2]
    F0 = _frame(ra0, dec0)
    l0, m0 = float(F0[0] @ s1), float(F0[1] @ s1)
    uvw = _uvw(30, rng, 6000.0)
    freqs = 345e9 + 7.8125e6 * np.arange(12)
    S = 2e-3
    vis = _point_vis(uvw, freqs, l0, m0, S, 2)
    src = oracle_mod.Source(uvw, freqs, vis, np.ones((30, 2), np.float32), None, 0.0, 0.0, 2.0,
                            radec=(ra0, dec0, ra1, dec1))
    f0, df = oracle_mod.auto_lattice([freqs], [2.0], 64, 345e9 * 3.0)
    du = 2 * 1.01 * np.abs(uvw[:, :2]).max() * freqs.max() / C / 32
    cube = oracle_mod.make_cube(32, 32, 64, 2, du, du, f0, df, 0, 0)
    out = oracle_mod.stack(cube, [src])
    sel = out["sum_w"] > 0
    assert sel.sum() > 50
    np.testing.assert_allclose((out["sum_wv"][sel] / out["sum_w"][sel]).real, S, rtol=1e-8)
    np.testing.assert_allclose((out["sum_wv"][sel] / out["sum_w"][sel]).imag, 0, atol=1e-8 * S)


def test_reprojected_cells_use_the_rotated_baseline(oracle_mod):
    """The uv cell of a re-projected row is floor(u' nu/(c du)) + N/2 with
    (u', v') the baseline in the new frame, computed here from the numerical
    frames (rows away from a cell edge)."""
    rng = np.random.default_rng(44)
    ra0, dec0, ra1, dec1 = 0.3, 0.4, 0.3 + 0.02, 0.4 - 0.015
    uvw = _uvw(60, rng, 900.0)
    freqs = 230e9 + 15.625e6 * np.arange(5)
    du, N = 17000.0, 64
    cube = oracle_mod.make_cube(N, N, 8, 1, du, du, 1e9, 1e9, 0, 0)
    src = oracle_mod.Source(uvw, freqs, np.ones((60, 5, 1)), np.ones((60, 1), np.float32), None, 0.0, 0.0, 0.0,
                            radec=(ra0, dec0, ra1, dec1))
    cl = oracle_mod.cells(cube, src)
    R = _frame(ra1, dec1) @ _frame(ra0, dec0).T
    rot = uvw @ R.T
    moved = checked = 0
    for r in range(60):
        for k in range(5):
            xs = [rot[r, ax] * freqs[k] / (C * du) for ax in (0, 1)]
            if any(abs(x - math.floor(x) - 0.5) > 0.5 - 1e-6 for x in xs):
                continue
            want = [math.floor(x) + N // 2 for x in xs]
            if all(0 <= w < N for w in want):
                assert list(cl[r, k]) == want
                checked += 1
                plain = [math.floor(uvw[r, ax] * freqs[k] / (C * du)) + N // 2 for ax in (0, 1)]
                moved += plain != want
    assert checked > 150 and moved > 20   # the rotation changes cells


# ----------------------------------------------------------------- Eq. 3 per-row output

def test_regrid_rows_brute_force(oracle_mod):
    """Eq. 3 per row written as plain loops: the unreduced phase exp(2 pi i
    tau nu/c), the Eq. 4 weights, flagged channels left out of both sums."""
    rng = np.random.default_rng(50)
    uvw = _uvw(3, rng, 800.0)
    freqs = 115e9 + 7.8125e6 * np.arange(9)
    vis = rng.normal(size=(3, 9, 2)) + 1j * rng.normal(size=(3, 9, 2))
    flags = (rng.uniform(size=(3, 9, 2)) < 0.2).astype(np.uint8)
    l0, m0, z = 15 * ARCSEC, -8 * ARCSEC, 1.7
    src = _src(oracle_mod, uvw, freqs, vis, l0, m0, z, flags=flags)
    f0, df = oracle_mod.auto_lattice([freqs], [z], 40, 115e9 * 2.7)
    out, den = oracle_mod.regrid_rows(src, f0, df, 40)
    W = oracle_mod.rest_weights(freqs, z, f0, df, 40)
    n1 = math.sqrt(1 - l0 * l0 - m0 * m0) - 1
    for r in range(3):
        tau = uvw[r, 0] * l0 + uvw[r, 1] * m0 + uvw[r, 2] * n1
        for p in range(2):
            for j in range(40):
                num = 0j
                d = 0.0
                for k in range(9):
                    if flags[r, k, p] or W[k, j] == 0:
                        continue
                    num += vis[r, k, p] * cmath.exp(2j * math.pi * tau * freqs[k] / C) * W[k, j]
                    d += W[k, j]
                assert abs(den[r, j, p] - d) <= 1e-14
                want = num / d if d > 0 else 0j
                assert abs(out[r, j, p] - want) <= 1e-9 * max(1.0, abs(want))
    assert (den > 0).sum() > 40


def test_regrid_rows_flat_spectrum(oracle_mod):
    """No shift and a constant spectrum: every covered output channel holds
    the constant (Eq. 3 is a weighted mean)."""
    rng = np.random.default_rng(51)
    uvw = _uvw(5, rng)
    freqs = 100e9 + 15.625e6 * np.arange(16)
    vis = np.full((5, 16, 1), 0.3 - 0.4j)
    src = _src(oracle_mod, uvw, freqs, vis, 0.0, 0.0, 2.0)
    f0, df = oracle_mod.auto_lattice([freqs], [2.0], 48, 300e9)
    out, den = oracle_mod.regrid_rows(src, f0, df, 48)
    cov = den > 0
    assert cov.sum() >= 5 * 15
    np.testing.assert_allclose(out[cov], 0.3 - 0.4j, rtol=1e-14)
    np.testing.assert_allclose(den.sum(axis=1), 16.0, rtol=1e-12)   # every channel is inside the lattice


def test_regrid_rows_equals_one_row_stack(oracle_mod):
    """One row alone in its cells: the stack's sum_wv / sum_w (W = 1) is the
    row's Eq. 3 output -- the C stack and the per-row product agree."""
    rng = np.random.default_rng(52)
    uvw = _uvw(1, rng, 400.0)
    freqs = 230e9 + 15.625e6 * np.arange(12)
    vis = rng.normal(size=(1, 12, 2)) + 1j * rng.normal(size=(1, 12, 2))
    src = _src(oracle_mod, uvw, freqs, vis, 5 * ARCSEC, 3 * ARCSEC, 1.2)
    f0, df = oracle_mod.auto_lattice([freqs], [1.2], 32, 230e9 * 2.2)
    out, den = oracle_mod.regrid_rows(src, f0, df, 32)
    cube = oracle_mod.make_cube(8, 8, 32, 2, 1e6, 1e6, f0, df, 0, 0)   # one huge cell: every channel in it
    st = oracle_mod.stack(cube, [src])
    sw = st["sum_w"].sum(axis=(0, 1))          # [nrest, npol]
    swv = st["sum_wv"].sum(axis=(0, 1))
    cov = sw > 0
    np.testing.assert_allclose(swv[cov] / sw[cov], out[0][cov], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(sw, den[0], rtol=1e-12, atol=1e-15)
