"""Host-side pieces of bench.py and of the synthetic inputs, on the CPU: the
algorithmic byte count the roofline divides, the rank sharding, the
in-cube source selection, and the sky positions the re-projection inputs
are built from (checked with the oracle's own direction cosines)."""
import math

import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def bench():
    import bench as B
    return B


@pytest.fixture(scope="module")
def tiny():
    from paper_2609_01897_gb300 import synth
    return synth.tiny("cpu")


def test_algorithmic_bytes_by_hand(bench, tiny, oracle_mod):
    """9 B per in-cube visibility (complex64 + flag), 24 + 4 npol B per row
    of a window with an in-cube channel, 40 B per touched entry: recomputed
    here from the oracle's Eq. 4 weights."""
    f0, df = oracle_mod.auto_lattice([s.freqs for s in tiny.spws], [s.z for s in tiny.spws], tiny.nrest,
                                     tiny.central_freq)
    n_vis, alg = bench.algorithmic_bytes(tiny, f0, df, touched=1000)
    want_vis = want = 0
    for s in tiny.spws:
        W = oracle_mod.rest_weights(s.freqs, s.z, f0, df, tiny.nrest)
        nin = int((W.sum(axis=1) > 0).sum())
        nrow, _, npol = s.vis.shape
        want_vis += nrow * nin * npol
        want += nrow * nin * npol * 9 + (nrow * (24 + 4 * npol) if nin else 0)
    assert n_vis == want_vis and alg == want + 1000 * 40


def test_shards_are_disjoint_and_equal(bench):
    ids = [set(bench.shard_ids(64, r)) for r in range(8)]
    assert all(len(x) == 64 for x in ids)
    assert len(set().union(*ids)) == 8 * 64


def test_in_cube_sources_of_the_mixed_set(bench, oracle_mod):
    from paper_2609_01897_gb300 import synth
    meta = synth.mixed("cpu", meta_only=True)
    f0, df, ids = bench.in_cube_sources(meta, meta.nrest)
    assert ids and len(ids) < 64
    for s in meta.spws:
        W = oracle_mod.rest_weights(s.freqs, s.z, f0, df, meta.nrest)
        if W.sum() > 0:
            assert s.source in ids


def test_sky_positions_round_trip(oracle_mod):
    """synth.sky_position puts (l, m) on the sky; the oracle's direction
    cosines of that position, seen from the phase centre, give (l, m) back."""
    from paper_2609_01897_gb300 import synth
    rng = np.random.default_rng(60)
    for _ in range(50):
        ra0, dec0 = rng.uniform(0, 2 * math.pi), rng.uniform(-1.4, 1.4)
        l, m = rng.uniform(-0.02, 0.02, size=2)
        ra1, dec1 = synth.sky_position(ra0, dec0, l, m)
        lo, mo = oracle_mod.offset(ra0, dec0, ra1, dec1)
        assert abs(lo - l) < 1e-14 and abs(mo - m) < 1e-14


def test_half_pairs_scale_and_values():
    from paper_2609_01897_gb300 import synth
    g = torch.Generator().manual_seed(3)
    v = torch.complex(torch.randn(50, 8, 2, generator=g), torch.randn(50, 8, 2, generator=g)) * 7.0
    for kind, dt in (("f16", torch.float16), ("bf16", torch.bfloat16)):
        q, scale = synth.half_pairs(v, kind)
        assert q.dtype == dt and q.shape == (50, 8, 2, 2)
        assert math.log2(scale) == int(math.log2(scale))          # a power of two
        back = torch.view_as_complex(q.to(torch.float32).contiguous()) * scale
        rel = 2.0 ** -11 if kind == "f16" else 2.0 ** -8
        assert float((back - v).abs().max()) <= rel * float(v.abs().max()) * 2


def test_e2e_window_io_counts(bench, tiny, oracle_mod):
    """The end-to-end leg's per-window counts: in-cube visibilities sum to the
    step's count, and the bytes copied cover uvw, weights and the channels
    read (in-cube range rounded out to whole flag words) of vis and flags."""
    f0, df = oracle_mod.auto_lattice([s.freqs for s in tiny.spws], [s.z for s in tiny.spws], tiny.nrest,
                                     tiny.central_freq)
    n_vis, _ = bench.algorithmic_bytes(tiny, f0, df, touched=0)
    tot = 0
    for s in tiny.spws:
        nv, hb = bench.window_io(s, f0, df, tiny.nrest)
        tot += nv
        W = oracle_mod.rest_weights(s.freqs, s.z, f0, df, tiny.nrest)
        ks = np.nonzero(W.sum(axis=1) > 0)[0]
        nrow, nch, npol = s.vis.shape
        if ks.size == 0:
            assert hb == 0
            continue
        al = 4 // npol if npol < 4 else 1
        lo, hi = ks[0] // al * al, min(nch, -(-(ks[-1] + 1) // al) * al)
        flag_row = -(-(hi - lo) * npol // 4) * 4      # a word-aligned row of flag bytes
        assert hb == nrow * (24 + 4 * npol) + nrow * (hi - lo) * npol * 8 + nrow * flag_row
    assert tot == n_vis
