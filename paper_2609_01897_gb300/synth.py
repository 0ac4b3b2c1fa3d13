"""Seeded synthetic interferometric inputs for stacking workloads.

This module only MAKES inputs (array layouts, Earth-rotation uvw tracks,
channel axes, model-plus-noise visibilities, weights and flags); it contains
none of the stacking arithmetic.  Both the GPU path and the CPU oracle are fed
from here, so the two are always compared on identical data.

Every workload stands in for archive data that is not available here (ALMA,
VLA and MeerKAT archive stacks, and the paper's own mock Measurement Sets):
shapes, channel setups, redshift ranges and noise levels follow the stated
workloads; the parameters marked "assumed" are choices made where the
workload statement is silent.

Conventions
  * uvw in metres, rows in Measurement Set order: time-major, baselines
    (i < j) inner.
  * visibilities [nrow, nchan, npol] complex64, weights [nrow, npol] float32
    (1/sigma^2), flags [nrow, nchan, npol] uint8 (1 = flagged).
  * Geometry and channel axes come from numpy PCG64 seeded with
    1000*config_id + source; visibilities, noise and flags from a torch
    generator seeded the same way on the target device.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import math
import numpy as np
import torch

C_LIGHT = 299792458.0
ARCSEC = math.pi / (180.0 * 3600.0)


@dataclass
class Spw:
    f0: float        # first channel centre, Hz
    df: float        # channel spacing, Hz (negative for a descending axis)
    nchan: int

    def freqs(self) -> np.ndarray:
        return self.f0 + np.arange(self.nchan, dtype=np.float64) * self.df


@dataclass
class SourceSpw:
    """One (source, spectral window) as handed to the stack."""
    uvw: torch.Tensor            # [nrow, 3] float64
    freqs: np.ndarray            # [nchan] float64, host
    vis: torch.Tensor            # [nrow, nchan, npol] complex64
    weights: torch.Tensor        # [nrow, npol] float32
    flags: Optional[torch.Tensor]  # [nrow, nchan, npol] uint8
    l: float
    m: float
    z: float
    pol_map: Optional[np.ndarray] = None
    source: int = 0
    vis_scale: float = 1.0       # 16-bit storage: stored value x vis_scale = visibility
    radec: Optional[tuple] = None  # (ra0, dec0, ra1, dec1): re-project (Eq. 1) instead of (l, m)


@dataclass
class Workload:
    name: str
    nu: int
    nv: int
    nrest: int
    npol: int
    du: float
    dv: float
    central_freq: float
    spws: List[SourceSpw] = field(default_factory=list)
    rest_df: float = 0.0
    rest_f0: float = 0.0

    def n_vis(self) -> int:
        return sum(s.vis.numel() for s in self.spws)


# --------------------------------------------------------------------------- geometry

def array_enu(n_ant: int, radius_m: float, rng: np.random.Generator) -> np.ndarray:
    """Antenna (E, N, U) positions uniform in a disc of the given radius, U = 0."""
    r = radius_m * np.sqrt(rng.random(n_ant))
    a = 2.0 * np.pi * rng.random(n_ant)
    return np.stack([r * np.cos(a), r * np.sin(a), np.zeros(n_ant)], axis=1)


def uvw_tracks(enu: np.ndarray, lat_deg: float, dec_deg: float, n_int: int,
               t_int_s: float, ha0_rad: float) -> np.ndarray:
    """Earth-rotation uvw of every baseline (i < j) at n_int hour angles,
    time-major.  Standard ENU -> equatorial XYZ -> (u, v, w) rotation."""
    n_ant = enu.shape[0]
    ii, jj = np.triu_indices(n_ant, k=1)
    b = enu[jj] - enu[ii]                          # [nbl, 3] ENU
    lat = np.deg2rad(lat_deg)
    dec = np.deg2rad(dec_deg)
    X = -np.sin(lat) * b[:, 1] + np.cos(lat) * b[:, 2]
    Y = b[:, 0]
    Z = np.cos(lat) * b[:, 1] + np.sin(lat) * b[:, 2]
    ha = ha0_rad + (np.arange(n_int) - 0.5 * (n_int - 1)) * t_int_s * (2.0 * np.pi / 86164.0905)
    sh, ch = np.sin(ha)[:, None], np.cos(ha)[:, None]
    u = sh * X + ch * Y
    v = -np.sin(dec) * ch * X + np.sin(dec) * sh * Y + np.cos(dec) * Z
    w = np.cos(dec) * ch * X - np.cos(dec) * sh * Y + np.sin(dec) * Z
    return np.stack([u, v, w], axis=-1).reshape(-1, 3)


# --------------------------------------------------------------------------- sky model

def model_vis(uvw: torch.Tensor, freqs: np.ndarray, l0: float, m0: float, flux: float,
              fwhm_rad: float, line_nu: float, line_peak: float, line_fwhm_kms: float,
              npol: int) -> torch.Tensor:
    """Visibilities of a circular Gaussian (or point, fwhm 0) source at (l0, m0)
    with a flat continuum plus a Gaussian line, under the measurement-equation
    sign convention V = S exp(-2 pi i nu/c (u l + v m + w (n - 1)))."""
    dev = uvw.device
    f = torch.as_tensor(freqs, dtype=torch.float64, device=dev)
    n0 = math.sqrt(1.0 - l0 * l0 - m0 * m0) - 1.0
    geo = uvw[:, 0:1] * l0 + uvw[:, 1:2] * m0 + uvw[:, 2:3] * n0          # [nrow, 1]
    turns = geo * (f[None, :] / C_LIGHT)                                   # [nrow, nchan]
    turns = turns - torch.floor(turns)
    ph = -2.0 * math.pi * turns
    spec = torch.full_like(f, flux)
    if line_peak != 0.0 and line_nu > 0.0:
        sig = line_nu * (line_fwhm_kms * 1e3 / C_LIGHT) / (2.0 * math.sqrt(2.0 * math.log(2.0)))
        spec = spec + line_peak * torch.exp(-0.5 * ((f - line_nu) / sig) ** 2)
    amp = spec[None, :].expand_as(turns)
    if fwhm_rad > 0.0:
        q2 = (uvw[:, 0:1] ** 2 + uvw[:, 1:2] ** 2) * (f[None, :] / C_LIGHT) ** 2
        amp = amp * torch.exp(-(math.pi * fwhm_rad) ** 2 * q2 / (4.0 * math.log(2.0)))
    v = torch.polar(amp, ph).to(torch.complex64)
    return v[:, :, None].expand(-1, -1, npol).contiguous()


def _noise_flags(shape, sigma: float, flag_frac: float, gen: torch.Generator, device):
    re = torch.randn(shape, generator=gen, device=device, dtype=torch.float32)
    im = torch.randn(shape, generator=gen, device=device, dtype=torch.float32)
    noise = torch.complex(re, im) * sigma
    flags = None
    if flag_frac > 0.0:
        flags = (torch.rand(shape, generator=gen, device=device) < flag_frac).to(torch.uint8)
    return noise, flags


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


# --------------------------------------------------------------------------- workloads

CONFIG_IDS = {"tiny": 0, "alma_compact": 1, "mixed": 2, "batched": 3, "wideband_hi": 4}


def _cube_du(spws: List[SourceSpw], n: int) -> float:
    """Cell size so the largest |u|,|v| in wavelengths fits with a 1e-4 margin."""
    m = 0.0
    for s in spws:
        fmax = float(np.max(np.abs(s.freqs)))
        m = max(m, float(s.uvw[:, :2].abs().max().item()) * fmax / C_LIGHT)
    return 2.0 * 1.0001 * m / n


def _make_sources(cid: int, n_src: int, *, n_ant, radius, n_int, t_int, lat, dec, spw_fn,
                  npol, flux_fn, fwhm, line_rest, line_peak_fn, line_fwhm, sigma,
                  flag_fn, offset_max, z_lo, z_hi, device, src_ids=None, meta_only=False,
                  storage="c64") -> List[SourceSpw]:
    """storage "f16" / "bf16": each window is converted to 16-bit pairs right
    after it is drawn (see half_pairs), so the complex form of the whole set
    never exists at once."""
    out = []
    ids = range(n_src) if src_ids is None else src_ids
    for s in ids:
        rng = np.random.default_rng(1000 * cid + s)
        enu = array_enu(n_ant, radius, rng)
        z = float(rng.uniform(z_lo, z_hi))
        l0 = float(rng.uniform(-offset_max, offset_max))
        m0 = float(rng.uniform(-offset_max, offset_max))
        ha0 = float(rng.uniform(-1.0, 1.0))
        flux = float(flux_fn(rng))
        line_peak = float(line_peak_fn(rng, flux))
        flag_frac = float(flag_fn(rng))
        uvw_np = uvw_tracks(enu, lat, dec, n_int, t_int, ha0)
        if meta_only:   # geometry and channel axes only (host uvw, no visibilities)
            for spw in spw_fn(rng, z):
                out.append(SourceSpw(torch.as_tensor(uvw_np), spw.freqs(), None, None, None, l0, m0, z,
                                     source=s))
            continue
        uvw = torch.as_tensor(uvw_np, dtype=torch.float64, device=device)
        gen = _gen(1000 * cid + s, device)
        for spw in spw_fn(rng, z):
            f = spw.freqs()
            v = model_vis(uvw, f, l0, m0, flux, fwhm, line_rest / (1.0 + z), line_peak,
                          line_fwhm, npol)
            noise, flags = _noise_flags(v.shape, sigma, flag_frac, gen, device)
            v = v + noise
            wts = torch.full((uvw.shape[0], npol), 1.0 / sigma ** 2, dtype=torch.float32,
                             device=device)
            scale = 1.0
            if storage != "c64":
                v, scale = half_pairs(v, storage)
            out.append(SourceSpw(uvw, f, v, wts, flags, l0, m0, z, source=s, vis_scale=scale))
    return out


def tiny(device="cpu") -> Workload:
    """8 sources, 10 antennas within 500 m, 20 x 30 s integrations at dec -30,
    lat -23; one 64 x 15.625 MHz window per source; 2 pols; 0.1 mJy Gaussian
    (FWHM 0.5") + line + 1 mJy noise; 1 % flags; offsets within +-10";
    z in [1, 3]; cube 64 x 64 x 128.  Assumed: the window is centred on the
    line's observed frequency 230.538 GHz/(1+z) (a fixed 230 GHz observed
    window could not hold a line emitted at 230.538 GHz from z in [1, 3]),
    line peak 1 mJy, FWHM 300 km/s, 30 s integrations."""
    nu_line = 230.538e9
    spws = _make_sources(
        0, 8, n_ant=10, radius=250.0, n_int=20, t_int=30.0, lat=-23.0, dec=-30.0,
        spw_fn=lambda rng, z: [Spw(nu_line / (1 + z) - 32 * 15.625e6, 15.625e6, 64)],
        npol=2, flux_fn=lambda rng: 1e-4, fwhm=0.5 * ARCSEC, line_rest=nu_line,
        line_peak_fn=lambda rng, f: 1e-3, line_fwhm=300.0, sigma=1e-3,
        flag_fn=lambda rng: 0.01, offset_max=10 * ARCSEC, z_lo=1.0, z_hi=3.0, device=device)
    n = 64
    du = _cube_du(spws, n)
    return Workload("tiny", n, n, 128, 2, du, du, nu_line, spws)


def alma_compact(device="cpu", n_sources=64, src_ids=None, meta_only=False, du=None) -> Workload:
    """64 sources, 43 antennas within 1 km, 120 integrations, two 120-channel
    windows at 100 and 112 GHz, 2 pols, point + line sources with flux
    lognormal(mean 0.05 mJy, sigma_ln 1), 0.5 mJy noise, z in [2, 3], cube
    256 x 256 x 512.  Assumed: 15.625 MHz channels, CO(3-2) line (rest
    345.796 GHz, also the cube's central frequency) with peak 2x the
    continuum and FWHM 300 km/s, offsets within +-10", 1 % flags, 30 s
    integrations, dec -30, lat -23."""
    nu_line = 345.796e9
    sig_ln = 1.0
    mu_ln = math.log(5e-5) - 0.5 * sig_ln ** 2
    spws = _make_sources(
        1, n_sources, n_ant=43, radius=500.0, n_int=120, t_int=30.0, lat=-23.0, dec=-30.0,
        spw_fn=lambda rng, z: [Spw(100e9 - 60 * 15.625e6, 15.625e6, 120),
                               Spw(112e9 - 60 * 15.625e6, 15.625e6, 120)],
        npol=2, flux_fn=lambda rng: rng.lognormal(mu_ln, sig_ln), fwhm=0.0, line_rest=nu_line,
        line_peak_fn=lambda rng, f: 2.0 * f, line_fwhm=300.0, sigma=5e-4,
        flag_fn=lambda rng: 0.01, offset_max=10 * ARCSEC, z_lo=2.0, z_hi=3.0, device=device,
        src_ids=src_ids, meta_only=meta_only)
    n = 256
    du = _cube_du(spws, n) if du is None else du
    return Workload("alma_compact", n, n, 512, 2, du, du, nu_line, spws)


CO10_9_REST = 1151.985452e9   # CO(10-9), Hz


def mixed(device="cpu", n_sources=64, src_ids=None, meta_only=False, du=None) -> Workload:
    """Precision workload: 64 sources, 43 antennas with baselines up to 16 km,
    120 integrations, 4 windows x 960 channels in 340-356 GHz, 2 pols,
    offsets up to 60" so that |tau nu / c| reaches ~5e3 turns (~3e4 rad).
    Assumed: window centres 341/343/353/355 GHz, 1.875 GHz wide; z in [2, 3];
    a CO(10-9) line (rest 1151.985 GHz, also the cube centre) with peak 2x
    the continuum and FWHM 300 km/s; flux lognormal(mean 0.05 mJy, sigma_ln
    1); 0.5 mJy noise; 1 % flags; 30 s integrations at dec -30, lat -23; cube
    256 x 256 x 512 x 2.  The whole set (5.3e10 visibilities, 426 GB as
    complex64) does not fit on one GPU: it is stacked in waves of sources
    into one cube (runs are additive)."""
    width, nchan = 1.875e9, 960
    df = width / nchan
    centres = (341e9, 343e9, 353e9, 355e9)
    sig_ln = 1.0
    mu_ln = math.log(5e-5) - 0.5 * sig_ln ** 2
    spws = _make_sources(
        CONFIG_IDS["mixed"], n_sources, n_ant=43, radius=8000.0, n_int=120, t_int=30.0, lat=-23.0, dec=-30.0,
        spw_fn=lambda rng, z: [Spw(c - 0.5 * (nchan - 1) * df, df, nchan) for c in centres],
        npol=2, flux_fn=lambda rng: rng.lognormal(mu_ln, sig_ln), fwhm=0.0, line_rest=CO10_9_REST,
        line_peak_fn=lambda rng, f: 2.0 * f, line_fwhm=300.0, sigma=5e-4,
        flag_fn=lambda rng: 0.01, offset_max=60 * ARCSEC, z_lo=2.0, z_hi=3.0, device=device,
        src_ids=src_ids, meta_only=meta_only)
    n = 256
    du = _cube_du(spws, n) if du is None else du
    return Workload("mixed", n, n, 512, 2, du, du, CO10_9_REST, spws)


def sky_position(ra0, dec0, l, m):
    """The sky position (ra, dec) at direction cosines (l, m) from the phase
    centre (ra0, dec0): l east, m north, from the frame's unit vectors."""
    w = np.array([math.cos(dec0) * math.cos(ra0), math.cos(dec0) * math.sin(ra0), math.sin(dec0)])
    e = np.cross([0.0, 0.0, 1.0], w)
    e /= np.linalg.norm(e)
    n = np.cross(w, e)
    s = l * e + m * n + math.sqrt(1.0 - l * l - m * m) * w
    return math.atan2(s[1], s[0]), math.asin(s[2])


def with_reprojection(wl: Workload, dec0: float) -> Workload:
    """Every window re-projected (Eq. 1): source s observed with phase centre
    (0.3 + 0.01 s, dec0) radians and stacked at the position of its synthetic
    source (its l, m), so the shift is the same and the cells are rotated."""
    for sp in wl.spws:
        ra0 = 0.3 + 0.01 * sp.source
        sp.radec = (ra0, dec0) + sky_position(ra0, dec0, sp.l, sp.m)
    wl.name += "+reproject"
    return wl


def half_pairs(vis: torch.Tensor, kind: str):
    """One window's complex visibilities as 16-bit (re, im) pairs,
    [nrow, nchan, npol, 2], with one power-of-two scale (exact in any
    precision): FP16 maps the largest |component| below 2^15, BF16 below 1.
    Returns (pairs, scale); pairs x scale = the stored visibility."""
    if kind not in ("f16", "bf16"):
        raise ValueError("kind is f16 or bf16")
    dt = torch.float16 if kind == "f16" else torch.bfloat16
    re_im = torch.view_as_real(vis)
    amax = float(re_im.abs().max()) if re_im.numel() else 1.0
    e = math.ceil(math.log2(amax)) if amax > 0 else 0
    scale = 2.0 ** (e - 15) if kind == "f16" else 2.0 ** e
    return (re_im / scale).to(dt).contiguous(), scale


def half_storage(wl: Workload, kind: str) -> Workload:
    """The workload with its visibilities stored as 16-bit pairs (half_pairs),
    converted one window at a time, the complex originals dropped."""
    out = []
    for s in wl.spws:
        q, scale = half_pairs(s.vis, kind)
        out.append(SourceSpw(s.uvw, s.freqs, q, s.weights, s.flags, s.l, s.m, s.z, s.pol_map, s.source, scale))
        s.vis = None
    return Workload(wl.name + "-" + kind, wl.nu, wl.nv, wl.nrest, wl.npol, wl.du, wl.dv, wl.central_freq, out,
                    rest_df=wl.rest_df, rest_f0=wl.rest_f0)


def wideband_hi(device="cpu", n_sources=24, src_ids=None, meta_only=False, du=None, storage="c64") -> Workload:
    """24 sources, 64 antennas within 8 km, 40 integrations, 856-1712 MHz in
    4096 channels, 2 pols, faint 21 cm line (rest 1420.405752 MHz, peak
    0.02 mJy, FWHM 200 km/s) under 2 mJy noise, z in [0.1, 0.5], cube
    512 x 512 x 2048.  Assumed: MeerKAT-like latitude -30.7, dec -30,
    no continuum, 8 s integrations, 1 % flags, offsets within +-10".
    The complex-half variant stacks 48 sources stored as 16-bit pairs
    (storage "f16" / "bf16", drawn window by window)."""
    nu_line = 1420.405752e6
    df = (1712e6 - 856e6) / 4096
    spws = _make_sources(
        4, n_sources, n_ant=64, radius=4000.0, n_int=40, t_int=8.0, lat=-30.7, dec=-30.0,
        spw_fn=lambda rng, z: [Spw(856e6 + 0.5 * df, df, 4096)],
        npol=2, flux_fn=lambda rng: 0.0, fwhm=0.0, line_rest=nu_line,
        line_peak_fn=lambda rng, f: 2e-5, line_fwhm=200.0, sigma=2e-3,
        flag_fn=lambda rng: 0.01, offset_max=10 * ARCSEC, z_lo=0.1, z_hi=0.5, device=device,
        src_ids=src_ids, meta_only=meta_only, storage=storage)
    n = 512
    du = _cube_du(spws, n) if du is None else du
    return Workload("wideband_hi", n, n, 2048, 2, du, du, nu_line, spws)


CII_REST = 1900.537e9   # [CII] 158 um, Hz


def batched(device="cpu", n_sources=2000, median_rows=20000, pool_gb=96.0, src_ids=None,
            meta_only=False, du=None, seed_pool=True, nrest=1024) -> Workload:
    """Batched uneven stack: per source, rows lognormal(median 20k, sigma_ln 1),
    1-4 windows of 1.875 GHz with 128/240/480/960/3840 channels in 84-950 GHz
    (window 0 centred on [CII] 1900.537 GHz/(1+z) when that falls in the
    band), 2 or 4 pols, z in [0.5, 4], flags 0-10 %; cube 256 x 256 x 1024 x 4
    centred on [CII].  The total (~5e11 visibilities) cannot be resident:
    every window's visibilities and flags are views at random offsets into
    two device pools (pool_gb of complex64 noise and a flag pool of the same
    element count in 11 segments with 0, 1, ..., 10 % flags; a window starts
    in its source's segment), so every read is a real HBM read, while each
    source's uvw and weights are its own.  Assumed: arrays of 10-50 antennas
    within 0.25-5 km, 30 s integrations at dec -30, lat -23 (rows = the first
    nrow of the baseline tracks), offsets within +-10", weights U[0.5, 1.5];
    a window's rows are capped so that it fits the pool (the far lognormal
    tail only).  nrest < 1024 narrows the rest range of the cube (same
    channel width and centre: a smaller cube for profiling captures)."""
    cid = CONFIG_IDS["batched"]
    nsrc_ids = range(n_sources) if src_ids is None else src_ids
    choices = np.array([128, 240, 480, 960, 3840])
    band_lo, band_hi, width = 84e9, 950e9, 1.875e9
    pool_elems = max(1 << 20, int(pool_gb * 1e9 / 8) // 16 * 16)
    plan = []
    for s in nsrc_ids:
        rng = np.random.default_rng(1000 * cid + s)
        nrow = max(1, int(round(rng.lognormal(math.log(median_rows), 1.0))))
        n_ant = int(rng.integers(10, 51))
        radius = float(rng.uniform(250.0, 5000.0))
        z = float(rng.uniform(0.5, 4.0))
        npol = int(rng.choice([2, 4]))
        flag_seg = int(rng.integers(0, 11))
        l0 = float(rng.uniform(-10 * ARCSEC, 10 * ARCSEC))
        m0 = float(rng.uniform(-10 * ARCSEC, 10 * ARCSEC))
        ha0 = float(rng.uniform(-1.0, 1.0))
        nspw = int(rng.integers(1, 5))
        wins = []
        nch_max = 0
        for k in range(nspw):
            nchan = int(rng.choice(choices))
            fc = CII_REST / (1.0 + z)
            if k > 0 or not (band_lo + 0.5 * width <= fc <= band_hi - 0.5 * width):
                fc = float(rng.uniform(band_lo + 0.5 * width, band_hi - 0.5 * width))
            df = width / nchan
            wins.append(Spw(fc - 0.5 * (nchan - 1) * df, df, nchan))
            nch_max = max(nch_max, nchan)
        nrow = min(nrow, pool_elems // (nch_max * npol))
        enu = array_enu(n_ant, radius, rng)
        nbl = n_ant * (n_ant - 1) // 2
        n_int = (nrow + nbl - 1) // nbl
        uvw_np = uvw_tracks(enu, -23.0, -30.0, n_int, 30.0, ha0)[:nrow]
        plan.append((s, nrow, npol, z, l0, m0, flag_seg, wins, uvw_np, rng))
    spws = []
    if meta_only:
        for s, nrow, npol, z, l0, m0, flag_seg, wins, uvw_np, rng in plan:
            for w in wins:
                spws.append(SourceSpw(torch.as_tensor(uvw_np), w.freqs(), None, None, None, l0, m0, z,
                                      source=s))
    else:
        g = _gen(1000 * cid + 999983, device)
        pool = torch.empty(pool_elems, dtype=torch.complex64, device=device)
        if seed_pool:
            torch.view_as_real(pool).normal_(generator=g)
        seg = pool_elems // 11 // 16 * 16
        fpool = torch.empty(pool_elems, dtype=torch.uint8, device=device)
        for k in range(11):
            lo, hi = k * seg, (k + 1) * seg if k < 10 else pool_elems
            fpool[lo:hi] = (torch.rand(hi - lo, generator=g, device=device) < 0.01 * k).to(torch.uint8)
        for s, nrow, npol, z, l0, m0, flag_seg, wins, uvw_np, rng in plan:
            uvw = torch.as_tensor(uvw_np, dtype=torch.float64, device=device)
            wts = torch.as_tensor(rng.uniform(0.5, 1.5, size=(nrow, npol)), dtype=torch.float32, device=device)
            for w in wins:
                n = nrow * w.nchan * npol
                off = int(rng.integers(0, (pool_elems - n) // 16 + 1)) * 16
                vis = pool[off:off + n].view(nrow, w.nchan, npol)
                foff = min(flag_seg * seg + int(rng.integers(0, seg // 16)) * 16, (pool_elems - n) // 16 * 16)
                flags = fpool[foff:foff + n].view(nrow, w.nchan, npol)
                spws.append(SourceSpw(uvw, w.freqs(), vis, wts, flags, l0, m0, z, source=s))
    n = 256
    du = _cube_du(spws, n) if du is None else du
    return Workload("batched", n, n, nrest, 4, du, du, CII_REST, spws)


def scaled(w: Workload, frac: float) -> Workload:
    """Same cube, only the first ceil(frac * nspw) windows (bounded samples)."""
    k = max(1, int(math.ceil(frac * len(w.spws))))
    return Workload(w.name, w.nu, w.nv, w.nrest, w.npol, w.du, w.dv, w.central_freq,
                    w.spws[:k], w.rest_df, w.rest_f0)


def random_case(seed: int, device="cpu", *, nsrc=3, max_rows=40, nchan_choices=(2, 3, 7, 33, 64, 130),
                npol_choices=(1, 2, 4), descending=False, offset_max=60 * ARCSEC,
                flag_frac=0.05, with_pol_map=False, nu=32, nv=32, nrest=48) -> Workload:
    """Small ragged workload for edge-case parity: ragged row counts (zero
    included), odd channel counts, 1/2/4 pols, optional descending axes and
    polarisation maps, some channels and rows outside the cube."""
    rng = np.random.default_rng(seed)
    enu = array_enu(8, 2000.0, rng)
    uvw_all = uvw_tracks(enu, -23.0, -30.0, 12, 60.0, 0.3)
    spws = []
    central = 230e9
    for s in range(nsrc):
        nrow = int(rng.integers(0, max_rows + 1)) if s > 0 else max_rows
        nchan = int(rng.choice(nchan_choices))
        npol = int(rng.choice(npol_choices))
        z = float(rng.uniform(0.2, 2.5))
        fc = central / (1 + z) * float(rng.uniform(0.995, 1.005))
        df = float(rng.choice([7.8125e6, 15.625e6, 31.25e6]))
        f0 = fc - 0.5 * (nchan - 1) * df
        spw = Spw(f0 + (nchan - 1) * df, -df, nchan) if descending and s % 2 == 0 else Spw(f0, df, nchan)
        sel = rng.integers(0, uvw_all.shape[0], size=nrow)
        uvw = torch.as_tensor(uvw_all[sel] * float(rng.uniform(0.5, 1.6)), dtype=torch.float64, device=device)
        g = _gen(seed * 7919 + s, device)
        shape = (nrow, nchan, npol)
        vis = torch.complex(torch.randn(shape, generator=g, device=device),
                            torch.randn(shape, generator=g, device=device)).to(torch.complex64)
        wts = (torch.rand((nrow, npol), generator=g, device=device) * 2.0).to(torch.float32)
        flags = (torch.rand(shape, generator=g, device=device) < flag_frac).to(torch.uint8)
        pm = None
        if with_pol_map:
            pm = rng.integers(-1, 2, size=npol).astype(np.int32)
            pm[0] = 0
        spws.append(SourceSpw(uvw, spw.freqs(), vis, wts, flags,
                              float(rng.uniform(-offset_max, offset_max)),
                              float(rng.uniform(-offset_max, offset_max)), z, pm, source=s))
    m = 0.0
    for s in spws:
        if s.uvw.shape[0]:
            m = max(m, float(s.uvw[:, :2].abs().max()) * float(np.max(s.freqs)) / C_LIGHT)
    du = 2.0 * m / nu * 0.8   # deliberately a little small: some rows fall off the grid
    return Workload("random%d" % seed, nu, nv, nrest, 4 if with_pol_map else max(
        int(s.vis.shape[2]) for s in spws), du, du, central, spws)
