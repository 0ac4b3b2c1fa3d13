"""Continuum subtraction over the rest-frequency axis of a stacked cube, in
FP64 (numpy).

TEST INFRASTRUCTURE ONLY: imported by tests/ and by the benchmark's
CPU-baseline leg; never by the GPU library.

The paper names continuum subtraction as the first post-processing step of
the stacked output (Sec. 3.4, "Post-processing") and leaves its method to
CASA.  The reading taken here is the uv-plane form of that step: per uv cell
and polarisation plane, a low-order polynomial in rest frequency is fitted
to the cell's spectrum over channels the caller marks as free of line
emission, by weighted least squares, and subtracted from every channel.

On the cube's sums (sum_wv = sum W w V', sum_w = sum W w per entry):
  spectrum    V_j = sum_wv_j / sum_w_j, weight sum_w_j (channels with
              sum_w_j = 0 carry no data)
  abscissa    x_j = (2 j - (nrest - 1)) / nrest, in (-1, 1)
  fit set     F = { j : line_free[j] and sum_w_j > 0 }
  degree      d = min(order, |F| - 1); no fit when F is empty
  fit         p = argmin over polynomials of degree <= d of
                  sum_{j in F} sum_w_j |V_j - p(x_j)|^2
              (complex V: real and imaginary parts are fitted alike)
  output      sum_wv'_j = sum_wv_j - sum_w_j p(x_j) for every j
so that sum_wv'_j / sum_w_j is the continuum-subtracted spectrum and the
output stays a cube of sums (sum_w, sum_w|V|^2 and the counts are unchanged).

The fit is written as the textbook weighted least-squares problem and
solved by numpy's least-squares routine on the sqrt(weight)-scaled
Vandermonde system, one (cell, plane) at a time.
"""
import numpy as np


def abscissa(nrest):
    j = np.arange(nrest, dtype=np.float64)
    return (2.0 * j - (nrest - 1)) / nrest


def contsub_spectrum(wv, w, line_free, order):
    """One (cell, plane): wv complex [nrest], w float [nrest], line_free bool
    [nrest].  Returns (wv' complex [nrest], coefficients c_0..c_d, lowest
    power first; empty when no fit)."""
    nrest = w.shape[0]
    x = abscissa(nrest)
    fit = np.asarray(line_free, dtype=bool) & (w > 0)
    nf = int(fit.sum())
    if nf == 0:
        return wv.astype(np.complex128).copy(), np.zeros(0, dtype=np.complex128)
    d = min(int(order), nf - 1)
    xs, ws = x[fit], w[fit]
    y = wv[fit] / ws                         # the spectrum V_j on the fit set
    A = np.vander(xs, d + 1, increasing=True)
    sw = np.sqrt(ws)
    c, *_ = np.linalg.lstsq(A * sw[:, None], y * sw, rcond=None)
    model = np.vander(x, d + 1, increasing=True) @ c
    return wv - w * model, c


def contsub(sum_wv, sum_w, line_free, order):
    """The whole cube: sum_wv complex [..., nrest, npol], sum_w float
    [..., nrest, npol] (the layout [nv][nu][nrest][npol], or a subset of its
    planes).  Returns sum_wv' of the same shape (complex128)."""
    sum_wv = np.asarray(sum_wv)
    sum_w = np.asarray(sum_w, dtype=np.float64)
    out = np.empty(sum_wv.shape, dtype=np.complex128)
    lead = sum_wv.shape[:-2]
    for idx in np.ndindex(*lead):
        for p in range(sum_wv.shape[-1]):
            out[idx + (slice(None), p)], _ = contsub_spectrum(
                sum_wv[idx + (slice(None), p)].astype(np.complex128), sum_w[idx + (slice(None), p)],
                line_free, order)
    return out
