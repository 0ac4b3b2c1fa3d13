"""Pins of the oracle's continuum subtraction (oracle/contsub.py): the
post-processing step the paper names in Sec. 3.4, read as a weighted
least-squares polynomial fit over line-free rest channels per uv cell and
plane, subtracted from every channel.  Each pin states what the mathematics
fixes independently of the oracle's own code:

  flat-plus-line   a constant continuum plus a line confined to the masked
                   channels: the line survives exactly, the line-free
                   channels go to zero (any order)
  polynomial       a continuum of degree <= order is removed exactly; one of
                   degree order + 1 is not (the pin has teeth)
  order 0          the subtracted level is the weighted mean of the
                   line-free channels (closed form)
  normal eqs       the residual on the fit set is orthogonal to 1, x, .., x^d
                   under the weights (the defining property of the fit)
  edge cases       empty channels (sum_w = 0) are untouched and not fitted;
                   too few line-free channels lower the degree; no line-free
                   channel leaves the spectrum unchanged
"""
import numpy as np
import pytest

from oracle import contsub as CS


def _spectrum(rng, nrest, coeffs, line, wzero=0.0):
    x = CS.abscissa(nrest)
    cont = sum(c * x ** k for k, c in enumerate(coeffs))
    w = rng.uniform(0.2, 3.0, size=nrest)
    if wzero:
        w[rng.random(nrest) < wzero] = 0.0
    V = cont + line
    return V * w, w, cont


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_flat_plus_line_survives_exactly(order):
    rng = np.random.default_rng(1 + order)
    nrest = 40
    line = np.zeros(nrest, dtype=np.complex128)
    line[17:23] = rng.normal(size=6) + 1j * rng.normal(size=6)
    free = np.ones(nrest, dtype=bool)
    free[15:25] = False
    wv, w, _ = _spectrum(rng, nrest, [2.5 - 1.25j], line)
    out, c = CS.contsub_spectrum(wv, w, free, order)
    V = out / w
    np.testing.assert_allclose(V[free], 0.0, atol=1e-12)
    np.testing.assert_allclose(V[~free], line[~free], atol=1e-12)
    assert abs(c[0] - (2.5 - 1.25j)) < 1e-12


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_polynomial_continuum_removed_up_to_order(order):
    rng = np.random.default_rng(10 + order)
    nrest = 64
    free = rng.random(nrest) < 0.7
    line = np.where(free, 0.0, rng.normal(size=nrest)) + 0j
    coeffs = list(rng.normal(size=order + 1) + 1j * rng.normal(size=order + 1))
    wv, w, _ = _spectrum(rng, nrest, coeffs, line)
    out, c = CS.contsub_spectrum(wv, w, free, order)
    np.testing.assert_allclose(out / w, line, atol=1e-11)
    np.testing.assert_allclose(c, coeffs, atol=1e-11)
    # one degree more is not removed by this order
    wv2, w2, _ = _spectrum(rng, nrest, coeffs + [1.0], line)
    out2, _ = CS.contsub_spectrum(wv2, w2, free, order)
    assert np.abs(out2 / w2 - line)[free].max() > 1e-3


def test_order0_is_the_weighted_mean():
    rng = np.random.default_rng(3)
    nrest = 30
    V = rng.normal(size=nrest) + 1j * rng.normal(size=nrest)
    w = rng.uniform(0.1, 2.0, size=nrest)
    free = rng.random(nrest) < 0.6
    out, c = CS.contsub_spectrum(V * w, w, free, 0)
    mean = (w[free] * V[free]).sum() / w[free].sum()
    assert abs(c[0] - mean) < 1e-13
    np.testing.assert_allclose(out, (V - mean) * w, atol=1e-13)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_normal_equations_hold(order):
    rng = np.random.default_rng(20 + order)
    nrest = 50
    V = rng.normal(size=nrest) + 1j * rng.normal(size=nrest)
    w = rng.uniform(0.1, 2.0, size=nrest)
    free = rng.random(nrest) < 0.5
    out, c = CS.contsub_spectrum(V * w, w, free, order)
    x = CS.abscissa(nrest)
    r = out / w
    for k in range(order + 1):
        # sum over the fit set of w x^k (V - p) = 0
        s = (w[free] * x[free] ** k * r[free]).sum()
        assert abs(s) < 1e-11 * (w[free] * np.abs(V[free])).sum()


def test_edge_cases():
    rng = np.random.default_rng(5)
    nrest = 24
    V = rng.normal(size=nrest) + 1j * rng.normal(size=nrest)
    w = rng.uniform(0.5, 1.5, size=nrest)
    w[[2, 9, 10]] = 0.0
    wv = V * w
    free = np.ones(nrest, dtype=bool)
    out, c = CS.contsub_spectrum(wv, w, free, 2)
    assert (out[[2, 9, 10]] == 0).all()                      # empty channels stay empty
    # empty channels take no part in the fit: whatever they hold is neither
    # fitted nor changed
    wv_b = wv.copy()
    wv_b[[2, 9, 10]] = [5.0 + 1j, -3.0, 7j]
    out_b, _ = CS.contsub_spectrum(wv_b, w, free, 2)
    keep = np.ones(nrest, dtype=bool)
    keep[[2, 9, 10]] = False
    np.testing.assert_array_equal(out_b[keep], out[keep])
    np.testing.assert_array_equal(out_b[~keep], wv_b[~keep])
    # two line-free channels with data: the degree drops to 1 (a line through them)
    free2 = np.zeros(nrest, dtype=bool)
    free2[[0, 5]] = True
    out2, c2 = CS.contsub_spectrum(wv, w, free2, 3)
    assert c2.size == 2
    np.testing.assert_allclose(out2[[0, 5]] / w[[0, 5]], 0.0, atol=1e-12)
    # no line-free channel with data: nothing is subtracted
    out3, c3 = CS.contsub_spectrum(wv, w, np.zeros(nrest, dtype=bool), 1)
    assert c3.size == 0
    np.testing.assert_array_equal(out3, wv)


def test_cube_layout_per_cell_and_plane():
    """The cube form applies the per-spectrum fit to every (cell, plane) of a
    [nv][nu][nrest][npol] cube independently."""
    rng = np.random.default_rng(8)
    nv, nu, nrest, npol = 3, 2, 16, 2
    wv = rng.normal(size=(nv, nu, nrest, npol)) + 1j * rng.normal(size=(nv, nu, nrest, npol))
    w = rng.uniform(0.0, 2.0, size=(nv, nu, nrest, npol))
    free = rng.random(nrest) < 0.6
    out = CS.contsub(wv, w, free, 1)
    for iv in range(nv):
        for iu in range(nu):
            for p in range(npol):
                o, _ = CS.contsub_spectrum(wv[iv, iu, :, p], w[iv, iu, :, p], free, 1)
                np.testing.assert_array_equal(out[iv, iu, :, p], o)
