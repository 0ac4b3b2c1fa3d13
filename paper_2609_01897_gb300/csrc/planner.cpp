// Host planner of libvista: the FP64 channel tables and the rest lattice.
//
// Compiled with -ffp-contract=off so every FP64 expression is the separately
// rounded IEEE operations it is written as; the bin indices, and which bins
// a channel touches, are then a fixed function of the inputs.
//
//   Delta nu_k   centred finite difference of the channel centres, one-sided
//                at the two ends (Sec. 3.2, after Eq. 4).
//   rest edges   (nu_k -/+ Delta nu_k / 2) (1+z)  (the (1+z) frequency scaling
//                that goes with Eq. 1).
//   lattice      e_j = f0 + j df; df = max over windows of the rest-frame
//                channel width, f0 = central_freq - (nrest/2) df (Sec. 3.1).
//   weights      w_kj = overlap(rest edges of k, [e_j, e_j+1]) / rest width of k
//                (Eqs. 3-4); nearest mode: the bin holding nu_k (1+z).
#include "planner.h"

#include <cmath>
#include <cstdlib>
#include <vector>

#include "vista.h"

namespace vista {

int channel_widths(const double *f, int32_t n, double *dnu)
{
    if (n < 2) return -1;
    for (int32_t k = 0; k < n; ++k) {
        double d;
        if (k == 0)
            d = f[1] - f[0];
        else if (k == n - 1)
            d = f[n - 1] - f[n - 2];
        else
            d = (f[k + 1] - f[k - 1]) * 0.5;
        dnu[k] = std::fabs(d);
    }
    return 0;
}

double widest_rest_channel(const double *f, int32_t n, double z)
{
    std::vector<double> d((size_t)n);
    if (channel_widths(f, n, d.data()) != 0) return 0.0;
    double zf = 1.0 + z, best = 0.0;
    for (int32_t k = 0; k < n; ++k) {
        double w = d[(size_t)k] * zf;
        if (w > best) best = w;
    }
    return best;
}

double lattice_f0(double central_freq, int32_t nrest, double df)
{
    return central_freq - ((double)nrest / 2.0) * df;
}

static inline double edge(double f0, double df, int64_t j) { return f0 + (double)j * df; }

int channel_bins(const double *f, int32_t nchan, double z, double f0, double df, int32_t nrest,
                 int32_t bin_mode, int32_t *j0, int32_t *nb, double *w)
{
    std::vector<double> dnu((size_t)(nchan > 1 ? nchan : 1), 0.0);
    if (bin_mode == VISTA_BIN_OVERLAP && channel_widths(f, nchan, dnu.data()) != 0) return VISTA_E_ARG;
    const double zf = 1.0 + z;
    for (int32_t k = 0; k < nchan; ++k) {
        double *wk = w + (size_t)k * VISTA_MAX_BINS;
        for (int b = 0; b < VISTA_MAX_BINS; ++b) wk[b] = 0.0;
        j0[k] = 0;
        nb[k] = 0;
        if (bin_mode == VISTA_BIN_NEAREST) {
            double q = std::floor((f[k] * zf - f0) / df);
            if (q >= 0.0 && q < (double)nrest) {
                j0[k] = (int32_t)q;
                nb[k] = 1;
                wk[0] = 1.0;
            }
            continue;
        }
        double half = 0.5 * dnu[(size_t)k];
        double lo = (f[k] - half) * zf;
        double hi = (f[k] + half) * zf;
        double qa = std::floor((lo - f0) / df), qb = std::floor((hi - f0) / df);
        // Only bins inside the lattice matter here; clamp the candidate window
        // (two bins of slack either side of the ones holding lo and hi).
        double ca = qa - 2.0, cb = qb + 2.0;
        if (ca < 0.0) ca = 0.0;
        if (cb > (double)(nrest - 1)) cb = (double)(nrest - 1);
        if (!(ca <= cb)) continue;       // entirely outside (or NaN)
        int32_t n = 0, first = -1;
        for (int64_t j = (int64_t)ca; j <= (int64_t)cb; ++j) {
            double ej = edge(f0, df, j), ej1 = edge(f0, df, j + 1);
            double a = hi < ej1 ? hi : ej1;
            double bb = lo > ej ? lo : ej;
            double o = a - bb;
            if (!(o > 0.0)) continue;
            if (n == VISTA_MAX_BINS) return VISTA_E_RANGE;
            if (first < 0) first = (int32_t)j;
            if ((int32_t)j != first + n) return VISTA_E_RANGE;   // not contiguous: never expected
            wk[n++] = o / (hi - lo);
        }
        if (n > 0) {
            j0[k] = first;
            nb[k] = n;
        }
    }
    return VISTA_OK;
}

bool linear_axis(const double *f, int32_t n, double *step)
{
    if (n < 2) {
        *step = 0.0;
        return true;
    }
    double d = (f[n - 1] - f[0]) / (double)(n - 1);
    *step = d;
    for (int32_t k = 0; k < n; ++k) {
        double pred = f[0] + (double)k * d;
        if (std::fabs(f[k] - pred) > 1e-12 * std::fabs(f[k])) return false;
    }
    return true;
}

}  // namespace vista

extern "C" int vista_plan_lattice(const double *const *freqs, const int32_t *nchan, const double *z,
                                  int32_t nsrc, int32_t nrest, double central_freq,
                                  double *rest_f0, double *rest_df)
{
    if (!freqs || !nchan || !z || nsrc < 1 || nrest < 1 || !rest_f0 || !rest_df) return VISTA_E_ARG;
    double best = 0.0;
    for (int32_t s = 0; s < nsrc; ++s) {
        if (!freqs[s] || nchan[s] < 2) return VISTA_E_ARG;
        double w = vista::widest_rest_channel(freqs[s], nchan[s], z[s]);
        if (w > best) best = w;
    }
    if (!(best > 0.0)) return VISTA_E_ARG;
    *rest_df = best;
    *rest_f0 = vista::lattice_f0(central_freq, nrest, best);
    return VISTA_OK;
}

extern "C" int vista_plan_channels(const double *freqs, int32_t nchan, double z, double rest_f0,
                                   double rest_df, int32_t nrest, int32_t bin_mode,
                                   int32_t *j0, int32_t *nb, double *w)
{
    if (!freqs || nchan < 1 || !j0 || !nb || !w || nrest < 1 || !(rest_df > 0.0)) return VISTA_E_ARG;
    if (bin_mode != VISTA_BIN_OVERLAP && bin_mode != VISTA_BIN_NEAREST) return VISTA_E_ARG;
    if (bin_mode == VISTA_BIN_OVERLAP && nchan < 2) return VISTA_E_ARG;
    return vista::channel_bins(freqs, nchan, z, rest_f0, rest_df, nrest, bin_mode, j0, nb, w);
}
