// Host planner of libvista (FP64 channel tables and rest lattice).
#pragma once
#include <cstdint>

namespace vista {

// Delta nu_k: centred difference, one-sided at the ends, absolute value.
int channel_widths(const double *f, int32_t n, double *dnu);
// max_k Delta nu_k (1+z) of one window (0 if n < 2).
double widest_rest_channel(const double *f, int32_t n, double z);
// central_freq - (nrest/2) df.
double lattice_f0(double central_freq, int32_t nrest, double df);
// In-lattice rest bins of every channel (see vista_plan_channels).
int channel_bins(const double *f, int32_t nchan, double z, double f0, double df, int32_t nrest,
                 int32_t bin_mode, int32_t *j0, int32_t *nb, double *w);
// True if f_k = f_0 + k step to 1e-12 relative (the phasor recurrence then
// uses one step for the window); *step = (f_{n-1} - f_0)/(n-1).
bool linear_axis(const double *f, int32_t n, double *step);

}  // namespace vista
