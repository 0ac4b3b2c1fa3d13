/*
 * vista_oracle.c -- plain, slow, FP64 CPU oracle of visibility stacking in the
 * Fourier domain (ViSta, arxiv 2609.01897).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code, no
 * header and no table with the GPU library, and the GPU library never calls it.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread (see oracle/build.py).
 * -ffp-contract=off matters: every FP64 expression below is evaluated as the
 * individually rounded IEEE operations it is written as, so the bin indices
 * it produces are a fixed function of the inputs.
 *
 * What it computes (one pass over every source, row, channel, polarisation):
 *
 *   tau   = u*l + v*m + w*(sqrt(1 - l^2 - m^2) - 1)                [Eq. 2]
 *   V'    = V * exp(+2 pi i frac(tau*nu_k/c))                      [Eq. 2, sign read
 *           so that a point source at (l, m) becomes real, see the point-source pin]
 *   cell  = floor(u * s_k) + nu/2, s_k = nu_k * (1/(c*du))         [uv in wavelengths,
 *           u_obs*nu_obs/c = u_rf*nu_rest/c, the z-invariant form of Eq. 1]
 *   re-projected sources (Eq. 1 with a rotation): (l, m) are the direction
 *           cosines of the stacking position (ra1, dec1) seen from the phase
 *           centre (ra0, dec0), and the cell uses (u', v') = the first two
 *           rows of R (u, v, w), R = M(ra1, dec1) M(ra0, dec0)^T
 *   w_kj  = overlap of the input channel's rest-frame edges with output bin j,
 *           divided by the input channel's rest-frame width           [Eqs. 3-4]
 *   cube[iv][iu][j][plane] += (W w_kj V', W w_kj, W w_kj |V|^2, 1)
 *
 * Sums are plain FP64 (not compensated): with at most ~1e7 terms per cell the
 * FP64 rounding error is below 1e-9 relative, four orders under the 1e-5
 * parity tolerance it is used against.
 *
 * Parity pins for every function here live in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_C_LIGHT 299792458.0 /* m/s, exact by definition of the metre */

typedef struct {
    int32_t nu, nv, nrest, npol;
    double du, dv;          /* uv cell size, wavelengths */
    double rest_f0, rest_df;/* rest lattice lower edge and width, Hz */
    int32_t bin_mode;       /* 0 = channel overlap (Eqs. 3-4), 1 = nearest */
    int32_t hermitian_fold; /* 1: fold v<0 (or v==0, u<0) onto the upper half */
} or_cube;

typedef struct {
    int64_t nrow;
    int32_t nchan, npol;
    const double *uvw;      /* [nrow][3] metres */
    const double *freqs;    /* [nchan] Hz, observed channel centres */
    const void *vis;        /* [nrow][nchan][npol] complex, float or double pairs */
    int32_t vis_f64;        /* 0: float pairs, 1: double pairs */
    int32_t pad0;
    const float *weights;   /* [nrow][npol] */
    const uint8_t *flags;   /* [nrow][nchan][npol], nonzero = flagged, may be NULL */
    const int32_t *pol_map; /* [npol] -> cube plane or -1, may be NULL (identity) */
    double l, m, z;
    int32_t reproject;      /* 1: re-project (Eq. 1 rotation); l, m are then ignored */
    int32_t pad1;
    double ra0, dec0;       /* phase centre, radians */
    double ra1, dec1;       /* stacking position, radians */
} or_source;

typedef struct {
    uint64_t n_vis;         /* unflagged+flagged visibilities in channels that reach the cube */
    uint64_t n_flagged;     /* of those, flagged */
    uint64_t n_dropped_uv;  /* of those, unflagged but outside the uv grid */
    uint64_t n_stacked;     /* of those, unflagged and inside the uv grid */
    double w_unflagged;     /* sum of W over every unflagged visibility, all channels */
    double w_cube;          /* sum of W*w_kj that landed in the cube */
    double w_dropped_uv;    /* sum of W over unflagged visibilities outside the uv grid */
    double w_dropped_rest;  /* sum of W*w_kj over bins outside [0, nrest) */
} or_stats;

/* ------------------------------------------------------------------------ */
/* Channel width Delta nu_k: centred finite difference, one-sided at the two
 * ends (Eq. 4 and the sentence that follows it, Sec. 3.2).  Absolute value,
 * so that descending frequency axes give positive widths. */
int or_channel_widths(const double *f, int32_t n, double *dnu)
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
        dnu[k] = fabs(d);
    }
    return 0;
}

/* Rest-frame edges of input channel k: observed edges nu_k -/+ Delta nu_k/2,
 * multiplied by (1+z) (Eq. 1's frequency scaling, Sec. 3.1). */
static void rest_edges(double nu_k, double dnu_k, double zf, double *lo, double *hi)
{
    double half = 0.5 * dnu_k;
    *lo = (nu_k - half) * zf;
    *hi = (nu_k + half) * zf;
}

/* Output bin edge e_j of the common rest lattice. */
static double lattice_edge(double f0, double df, int64_t j)
{
    return f0 + (double)j * df;
}

/* Eq. 4: overlap of [lo, hi] with [e_j, e_{j+1}] over the channel's own
 * (rest-frame) width. */
static double overlap_weight(double lo, double hi, double ej, double ej1)
{
    double a = hi < ej1 ? hi : ej1;
    double b = lo > ej ? lo : ej;
    double o = a - b;
    if (!(o > 0.0)) return 0.0;
    return o / (hi - lo);
}

/* Common output channel width, Sec. 3.1: Delta nu_new = max over inputs of the
 * rest-frame channel width; the lattice is centred on central_freq.  nsrc
 * entries of freqs/nchan/z. */
int or_auto_lattice(const double *const *freqs, const int32_t *nchan, const double *z,
                    int32_t nsrc, int32_t nrest, double central_freq,
                    double *rest_f0, double *rest_df)
{
    double best = 0.0;
    for (int32_t s = 0; s < nsrc; ++s) {
        int32_t n = nchan[s];
        if (n < 2) return -1;
        double *d = (double *)malloc(sizeof(double) * (size_t)n);
        if (!d) return -2;
        or_channel_widths(freqs[s], n, d);
        double zf = 1.0 + z[s];
        for (int32_t k = 0; k < n; ++k) {
            double w = d[k] * zf;
            if (w > best) best = w;
        }
        free(d);
    }
    *rest_df = best;
    *rest_f0 = central_freq - ((double)nrest / 2.0) * best;
    return 0;
}

/* Every rest bin j (any integer, inside the lattice or not) with w_kj > 0 for
 * channel k, in increasing j.  Returns how many were written (<= cap), or -1
 * if cap is too small.  bin_mode 1 (nearest): the single bin holding
 * nu_k (1+z), weight 1. */
static int chan_bins(const double *f, const double *dnu, int32_t k, double zf,
                     double f0, double df, int32_t bin_mode,
                     int64_t *js, double *ws, int cap)
{
    if (bin_mode == 1) {
        double rho = f[k] * zf;
        double q = floor((rho - f0) / df);
        if (!(fabs(q) < 9.0e15)) return 0;
        js[0] = (int64_t)q;
        ws[0] = 1.0;
        return 1;
    }
    double lo, hi;
    rest_edges(f[k], dnu[k], zf, &lo, &hi);
    /* Candidate window: a few bins either side of the ones holding lo and hi;
     * the window ends are checked to carry zero weight. */
    double qa = floor((lo - f0) / df), qb = floor((hi - f0) / df);
    if (!(fabs(qa) < 9.0e15 && fabs(qb) < 9.0e15)) return 0;
    int64_t ja = (int64_t)qa - 2, jb = (int64_t)qb + 2;
    int n = 0;
    for (int64_t j = ja; j <= jb; ++j) {
        double w = overlap_weight(lo, hi, lattice_edge(f0, df, j), lattice_edge(f0, df, j + 1));
        if (w > 0.0) {
            if ((j == ja || j == jb)) return -2; /* window too small: never expected */
            if (n >= cap) return -1;
            js[n] = j;
            ws[n] = w;
            ++n;
        }
    }
    return n;
}

/* Dense Eq. 4 weights for one source: out[k][j] for j in [0, nrest). */
int or_rest_weights(const double *f, int32_t nchan, double z, double f0, double df,
                    int32_t nrest, int32_t bin_mode, double *out)
{
    double *dnu = (double *)calloc((size_t)(nchan > 1 ? nchan : 1), sizeof(double));
    if (!dnu) return -2;
    if (bin_mode == 0 && or_channel_widths(f, nchan, dnu) != 0) { free(dnu); return -1; }
    memset(out, 0, sizeof(double) * (size_t)nchan * (size_t)nrest);
    double zf = 1.0 + z;
    for (int32_t k = 0; k < nchan; ++k) {
        int64_t js[64];
        double ws[64];
        int n = chan_bins(f, dnu, k, zf, f0, df, bin_mode, js, ws, 64);
        if (n < 0) { free(dnu); return -3; }
        for (int i = 0; i < n; ++i)
            if (js[i] >= 0 && js[i] < nrest) out[(size_t)k * nrest + js[i]] = ws[i];
    }
    free(dnu);
    return 0;
}

/* Delay in metres: u l + v m + w (n - 1), n = sqrt(1 - l^2 - m^2)  (Eq. 2, with
 * the direction-cosine differences of a shift from the phase centre to (l, m)). */
static double delay_m(const double *uvw, double l, double m)
{
    double n1 = sqrt(1.0 - l * l - m * m) - 1.0;
    return uvw[0] * l + uvw[1] * m + uvw[2] * n1;
}

/* Eq. 1's frames: the rows of M(ra, dec) are the unit vectors u (east),
 * v (north) and w (toward (ra, dec)) in equatorial coordinates (x toward
 * ra = 0 on the equator, z toward the north pole). */
static void uvw_frame(double ra, double dec, double M[3][3])
{
    M[0][0] = -sin(ra);
    M[0][1] = cos(ra);
    M[0][2] = 0.0;
    M[1][0] = -sin(dec) * cos(ra);
    M[1][1] = -sin(dec) * sin(ra);
    M[1][2] = cos(dec);
    M[2][0] = cos(dec) * cos(ra);
    M[2][1] = cos(dec) * sin(ra);
    M[2][2] = sin(dec);
}

/* R = M(ra1, dec1) M(ra0, dec0)^T, row-major: a baseline's (u, v, w) for phase
 * centre 0 expressed for phase centre 1 (the rotation of Eq. 1). */
void or_rotation(double ra0, double dec0, double ra1, double dec1, double *R)
{
    double M0[3][3], M1[3][3];
    uvw_frame(ra0, dec0, M0);
    uvw_frame(ra1, dec1, M1);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            R[3 * i + j] = M1[i][0] * M0[j][0] + M1[i][1] * M0[j][1] + M1[i][2] * M0[j][2];
}

/* Direction cosines (l, m) of (ra1, dec1) seen from the phase centre
 * (ra0, dec0): the usual spherical offsets. */
void or_offset(double ra0, double dec0, double ra1, double dec1, double *lm)
{
    double da = ra1 - ra0;
    lm[0] = cos(dec1) * sin(da);
    lm[1] = sin(dec1) * cos(dec0) - cos(dec1) * sin(dec0) * cos(da);
}

/* Per-source geometry: the shift's (l, m) and, for a re-projected source,
 * the rotation applied to the baselines before the uv cell. */
typedef struct {
    double l, m;
    int rot;
    double R[9];
} src_geom;

static void source_geom(const or_source *s, src_geom *g)
{
    g->l = s->l;
    g->m = s->m;
    g->rot = s->reproject != 0;
    if (g->rot) {
        double lm[2];
        or_offset(s->ra0, s->dec0, s->ra1, s->dec1, lm);
        g->l = lm[0];
        g->m = lm[1];
        or_rotation(s->ra0, s->dec0, s->ra1, s->dec1, g->R);
    }
}

/* The (u, v) a row is gridded with: the stored ones, or the first two rows of
 * R (u, v, w) for a re-projected source. */
static void cell_uv(const src_geom *g, const double *uvw, double *u, double *v)
{
    if (g->rot) {
        *u = g->R[0] * uvw[0] + g->R[1] * uvw[1] + g->R[2] * uvw[2];
        *v = g->R[3] * uvw[0] + g->R[4] * uvw[1] + g->R[5] * uvw[2];
    } else {
        *u = uvw[0];
        *v = uvw[1];
    }
}

/* Phase turns of the shift for frequency nu, reduced to [0, 1). */
static double shift_turns(double tau, double nu)
{
    double t = tau * nu / OR_C_LIGHT;
    return t - floor(t);
}

/* uv cell along one axis: floor(x) + n/2 with x = coord * (nu * (1/(c*d))),
 * -1 when outside [0, n). */
static int32_t uv_cell(double coord, double s_k, int32_t n)
{
    double x = coord * s_k;
    double half = (double)(n / 2);
    if (!(x >= -half && x < half)) return -1;
    return (int32_t)floor(x) + n / 2;
}

/* Phasors exp(+2 pi i frac(tau nu_k / c)) of one source, out[r][k][2]. */
void or_phasors(const or_source *s, double *out)
{
    src_geom g;
    source_geom(s, &g);
    for (int64_t r = 0; r < s->nrow; ++r) {
        double tau = delay_m(s->uvw + 3 * r, g.l, g.m);
        for (int32_t k = 0; k < s->nchan; ++k) {
            double ph = 2.0 * M_PI * shift_turns(tau, s->freqs[k]);
            out[2 * (r * s->nchan + k)] = cos(ph);
            out[2 * (r * s->nchan + k) + 1] = sin(ph);
        }
    }
}

/* uv cells of one source, out[r][k][2] = (iu, iv), -1 where outside the grid
 * (both set to -1 when either axis is outside). */
void or_cells(const or_cube *c, const or_source *s, int32_t *out)
{
    double gu = 1.0 / (OR_C_LIGHT * c->du), gv = 1.0 / (OR_C_LIGHT * c->dv);
    src_geom g;
    source_geom(s, &g);
    for (int64_t r = 0; r < s->nrow; ++r) {
        double u, v;
        cell_uv(&g, s->uvw + 3 * r, &u, &v);
        if (c->hermitian_fold && (v < 0.0 || (v == 0.0 && u < 0.0))) { u = -u; v = -v; }
        for (int32_t k = 0; k < s->nchan; ++k) {
            int32_t iu = uv_cell(u, s->freqs[k] * gu, c->nu);
            int32_t iv = uv_cell(v, s->freqs[k] * gv, c->nv);
            if (iu < 0 || iv < 0) iu = iv = -1;
            out[2 * (r * s->nchan + k)] = iu;
            out[2 * (r * s->nchan + k) + 1] = iv;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* The stack. */

typedef struct {          /* per source, per channel: the nonzero Eq. 4 bins */
    int32_t nb;
    int32_t incube;       /* 1 if at least one bin lies in [0, nrest) */
    int64_t j[8];
    double w[8];
} chan_tab;

typedef struct {
    const or_cube *c;
    const or_source *srcs;
    int32_t nsrc;
    chan_tab *const *tabs;
    const int32_t *sel_map;  /* iv -> compact plane index, -1 = not selected */
    int32_t tid, nthreads;
    double *sum_wv, *sum_w, *sum_wvv, *sum_wabs;
    uint64_t *count;
    or_stats st;
} job_t;

static inline int owner_of(int32_t iv, int nthreads) { return iv < 0 ? 0 : iv % nthreads; }

static void *stack_worker(void *arg)
{
    job_t *jb = (job_t *)arg;
    const or_cube *c = jb->c;
    double gu = 1.0 / (OR_C_LIGHT * c->du), gv = 1.0 / (OR_C_LIGHT * c->dv);
    memset(&jb->st, 0, sizeof(jb->st));
    for (int32_t si = 0; si < jb->nsrc; ++si) {
        const or_source *s = &jb->srcs[si];
        const chan_tab *tab = jb->tabs[si];
        const float *vf = (const float *)s->vis;
        const double *vd = (const double *)s->vis;
        src_geom g;
        source_geom(s, &g);
        for (int64_t r = 0; r < s->nrow; ++r) {
            double u, v;
            cell_uv(&g, s->uvw + 3 * r, &u, &v);
            int fold = c->hermitian_fold && (v < 0.0 || (v == 0.0 && u < 0.0));
            if (fold) { u = -u; v = -v; }
            double tau = delay_m(s->uvw + 3 * r, g.l, g.m);
            for (int32_t k = 0; k < s->nchan; ++k) {
                const chan_tab *ct = &tab[k];
                int32_t iu = uv_cell(u, s->freqs[k] * gu, c->nu);
                int32_t iv = uv_cell(v, s->freqs[k] * gv, c->nv);
                int inuv = iu >= 0 && iv >= 0;
                if (owner_of(inuv ? iv : -1, jb->nthreads) != jb->tid) continue;
                int32_t plane_row = -1;
                if (inuv) plane_row = jb->sel_map ? jb->sel_map[iv] : iv;
                double cr = 0.0, ci = 0.0;
                int have_ph = 0;
                for (int32_t p = 0; p < s->npol; ++p) {
                    int32_t q = s->pol_map ? s->pol_map[p] : p;
                    if (q < 0) continue;
                    size_t vi = ((size_t)r * s->nchan + k) * s->npol + p;
                    int flagged = s->flags && s->flags[vi];
                    double W = (double)s->weights[(size_t)r * s->npol + p];
                    if (ct->incube && !jb->sel_map) {
                        jb->st.n_vis++;
                        if (flagged) jb->st.n_flagged++;
                        else if (!inuv) jb->st.n_dropped_uv++;
                        else jb->st.n_stacked++;
                    }
                    if (flagged) continue;
                    if (!jb->sel_map) jb->st.w_unflagged += W;
                    if (!inuv) { if (!jb->sel_map) jb->st.w_dropped_uv += W; continue; }
                    if (plane_row < 0) continue; /* not a sampled plane */
                    double vr, vim;
                    if (s->vis_f64) { vr = vd[2 * vi]; vim = vd[2 * vi + 1]; }
                    else { vr = (double)vf[2 * vi]; vim = (double)vf[2 * vi + 1]; }
                    if (!have_ph) {
                        double ph = 2.0 * M_PI * shift_turns(tau, s->freqs[k]);
                        cr = cos(ph); ci = sin(ph);
                        have_ph = 1;
                    }
                    double sr = vr * cr - vim * ci;   /* V' = V * exp(+i phi) */
                    double sim = vr * ci + vim * cr;
                    if (fold) sim = -sim;             /* V(-u) = conj V(u) */
                    double a2 = vr * vr + vim * vim;  /* |V'|^2 = |V|^2 */
                    for (int32_t b = 0; b < ct->nb; ++b) {
                        double ww = W * ct->w[b];
                        int64_t j = ct->j[b];
                        if (j < 0 || j >= c->nrest) {
                            if (!jb->sel_map) jb->st.w_dropped_rest += ww;
                            continue;
                        }
                        size_t ci_ = (((size_t)plane_row * c->nu + iu) * c->nrest + j) * c->npol + q;
                        jb->sum_wv[2 * ci_] += ww * sr;
                        jb->sum_wv[2 * ci_ + 1] += ww * sim;
                        jb->sum_w[ci_] += ww;
                        jb->sum_wvv[ci_] += ww * a2;
                        if (jb->sum_wabs) jb->sum_wabs[ci_] += ww * sqrt(a2);
                        jb->count[ci_] += 1;
                        if (!jb->sel_map) jb->st.w_cube += ww;
                    }
                }
            }
        }
    }
    return NULL;
}

/* Stack nsrc sources into zero-initialised FP64 outputs.
 *   iv_select: NULL for the whole cube, else [nv] bytes; only planes with a
 *              nonzero byte are accumulated, and the outputs hold only those
 *              planes, in increasing iv (sampled parity at large sizes).
 *   outputs:   sum_wv [planes][nu][nrest][npol][2], sum_w / sum_wvv / count
 *              [planes][nu][nrest][npol].
 *   sum_wabs:  optional (may be NULL): sum of W w_kj |V| per cell, the scale
 *              of the cancellation-aware error bound on sum_wv.
 *   stats:     filled only when iv_select is NULL.
 *   nthreads:  worker threads; thread t owns the planes iv with iv % T == t,
 *              so no two threads write the same output and the result does
 *              not depend on T.
 * Returns 0, or negative on bad input / allocation failure. */
int or_stack(const or_cube *c, const or_source *srcs, int32_t nsrc, const uint8_t *iv_select,
             double *sum_wv, double *sum_w, double *sum_wvv, double *sum_wabs, uint64_t *count,
             or_stats *stats, int32_t nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (c->nu < 2 || c->nv < 2 || (c->nu & 1) || (c->nv & 1) || c->nrest < 1 || c->npol < 1)
        return -1;
    if (!(c->rest_df > 0.0) || !(c->du > 0.0) || !(c->dv > 0.0)) return -1;
    chan_tab **tabs = (chan_tab **)calloc((size_t)(nsrc > 0 ? nsrc : 1), sizeof(chan_tab *));
    int32_t *sel_map = NULL;
    int rc = 0;
    if (!tabs) return -2;
    for (int32_t si = 0; si < nsrc && rc == 0; ++si) {
        const or_source *s = &srcs[si];
        if (s->nchan < 1 || (c->bin_mode == 0 && s->nchan < 2)) { rc = -1; break; }
        tabs[si] = (chan_tab *)calloc((size_t)s->nchan, sizeof(chan_tab));
        double *dnu = (double *)calloc((size_t)s->nchan, sizeof(double));
        if (!tabs[si] || !dnu) { free(dnu); rc = -2; break; }
        if (c->bin_mode == 0) or_channel_widths(s->freqs, s->nchan, dnu);
        double zf = 1.0 + s->z;
        for (int32_t k = 0; k < s->nchan; ++k) {
            chan_tab *ct = &tabs[si][k];
            int n = chan_bins(s->freqs, dnu, k, zf, c->rest_f0, c->rest_df, c->bin_mode,
                              ct->j, ct->w, 8);
            if (n < 0) { rc = -3; break; }
            ct->nb = n;
            for (int b = 0; b < n; ++b)
                if (ct->j[b] >= 0 && ct->j[b] < c->nrest) ct->incube = 1;
        }
        free(dnu);
    }
    if (rc == 0 && iv_select) {
        sel_map = (int32_t *)malloc(sizeof(int32_t) * (size_t)c->nv);
        if (!sel_map) rc = -2;
        else {
            int32_t n = 0;
            for (int32_t iv = 0; iv < c->nv; ++iv) sel_map[iv] = iv_select[iv] ? n++ : -1;
        }
    }
    if (rc == 0) {
        job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
        pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
        if (!jobs || !th) rc = -2;
        else {
            for (int t = 0; t < nthreads; ++t) {
                jobs[t] = (job_t){c, srcs, nsrc, tabs, sel_map, t, nthreads,
                                  sum_wv, sum_w, sum_wvv, sum_wabs, count, {0}};
            }
            for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, stack_worker, &jobs[t]);
            stack_worker(&jobs[0]);
            for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
            if (stats) {
                memset(stats, 0, sizeof(*stats));
                for (int t = 0; t < nthreads; ++t) {   /* fixed merge order */
                    stats->n_vis += jobs[t].st.n_vis;
                    stats->n_flagged += jobs[t].st.n_flagged;
                    stats->n_dropped_uv += jobs[t].st.n_dropped_uv;
                    stats->n_stacked += jobs[t].st.n_stacked;
                    stats->w_unflagged += jobs[t].st.w_unflagged;
                    stats->w_cube += jobs[t].st.w_cube;
                    stats->w_dropped_uv += jobs[t].st.w_dropped_uv;
                    stats->w_dropped_rest += jobs[t].st.w_dropped_rest;
                }
            }
        }
        free(jobs);
        free(th);
    }
    for (int32_t si = 0; si < nsrc; ++si) free(tabs[si]);
    free(tabs);
    free(sel_map);
    return rc;
}
