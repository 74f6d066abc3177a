/*
 * oracle.c -- plain FP64 CPU oracle for the time-domain Lienard-Wiechert (LW)
 * radiation path of Kan, Kaertner, Le Borne, Ruprecht, Zemke, "Parallel
 * Computation of Inverse Compton Scattering Radiation Spectra based on
 * Lienard-Wiechert Potentials" (arXiv 2206.03015).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header or constant with the CUDA library.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no -march flags,
 * no FMA contraction: every floating-point operation below is one IEEE-754
 * rounding in the order written).
 *
 * Units are SI throughout: t [s], r [m], beta [1], beta_dot [1/s].
 *
 * Trajectory layout: n_e electrons, n_s+1 samples each (steps i = 0..n_s).
 *   t        [n_s+1]            (t_per_electron == 0)  or [n_e][n_s+1]
 *   r        [n_e][n_s+1][3]
 *   beta     [n_e][n_s+1][3]
 *   beta_dot [n_e][n_s+1][3]
 * Detector: n_pix unit vectors n_hat [n_pix][3] at distance R.
 * Observer grid: t_j = t_min + j*dt_u, j = 0..n_bins-1.
 * Record: rec [n_pix][3][n_bins] (Cartesian components of the field with the
 *   constant q/(4 pi eps0 c0 R) removed; units 1/s).
 *
 * Status bits (OR-ed into *status):
 *   1  |beta| >= 1 or D = 1 - n.beta <= 0 at a sample (field set to 0 there)
 *   2  non-finite input value, or a bin coordinate beyond +-2^62
 *   4  lab time t not strictly increasing along a trajectory
 *   8  grid points outside [0, n_bins) were skipped (clipped)
 *  16  advanced time t_a not increasing between two samples
 *
 * Readings of the paper used here (each is also listed in the design notes):
 *  - The common constant |x|/c0 of Eq. (far_adv) is dropped from t_a; it shifts
 *    every arrival time and the grid alike and has no effect on |E(omega)|
 *    (the paper drops the matching phase after Eq. (const_phase_drop)).
 *  - Grid point j lies in the half-open interval (t_b, t_a] of Algorithm 2 iff
 *    floor(u_b) < j <= floor(u_a) with u = (t - t_min) * (1/dt_u), evaluated as
 *    one subtraction followed by one multiplication.
 *  - The first sample of each trajectory only fills the buffer of Algorithm 2
 *    (no deposit from the initial buffer value of zero).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_C0 299792458.0
#define OR_EPS0 8.8541878128e-12
#define OR_PI 3.14159265358979323846

#define ST_BETA 1
#define ST_NONFINITE 2
#define ST_TIME 4
#define ST_CLIP 8
#define ST_TA_ORDER 16

#define FLAG_ACCEL 1
#define FLAG_VELOCITY 2
#define FLAG_EXACT 4

typedef struct {
    int64_t n_e, n_s;
    const double *t;
    int t_per_electron;
    const double *r, *beta, *beta_dot;
} or_traj;

static double tr_time(const or_traj *tr, int64_t k, int64_t i) {
    return tr->t_per_electron ? tr->t[k * (tr->n_s + 1) + i] : tr->t[i];
}

static const double *tr_vec(const double *base, const or_traj *tr, int64_t k, int64_t i) {
    return base + 3 * (k * (tr->n_s + 1) + i);
}

static double dot3(const double *a, const double *b) {
    double s = a[0] * b[0];
    s = s + a[1] * b[1];
    s = s + a[2] * b[2];
    return s;
}

static void cross3(const double *a, const double *b, double *out) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* Far-field advanced time, Eq. (far_adv) without the constant |x|/c0:
 *   t_a = t - (n . x'(t)) / c0,
 * with n.x' summed x, y, z in that order and the division done as a
 * multiplication by the correctly rounded constant 1/c0. */
static double advanced_time_far(const double *n, const double *r, double t) {
    const double inv_c0 = 1.0 / OR_C0;
    double nr = n[0] * r[0];
    nr = nr + n[1] * r[1];
    nr = nr + n[2] * r[2];
    return t - nr * inv_c0;
}

/* Exact advanced time, Eq. (advanced_condition): t_a = t + |x - x'(t)| / c0,
 * observer at x = R n. */
static double advanced_time_exact(const double *n, double R, const double *r, double t) {
    double d[3] = {R * n[0] - r[0], R * n[1] - r[1], R * n[2] - r[2]};
    return t + sqrt(dot3(d, d)) / OR_C0;
}

/* Field sample with the constant q/(4 pi eps0 c0 R) removed.
 * Far field (flags without FLAG_EXACT), Eq. (far_efield):
 *   F = n x ((n - beta) x beta_dot) / (1 - n.beta)^3
 * plus, with FLAG_VELOCITY, the velocity field of the same LW solution
 * (the first term of the textbook LW field that the paper drops for the
 * radiation problem), in the same normalisation:
 *   c0 (n - beta) (1 - beta^2) / ((1 - n.beta)^3 R).
 * With FLAG_EXACT the unit vector and distance are the exact ones,
 * n(t) = (x - x')/|x - x'|, and both terms carry R/|x - x'|, i.e. the exact
 * LW field of Eq. (lw_fields_retarded) times 4 pi eps0 c0 R / q.
 * Returns 0 on success or ST_BETA when |beta| >= 1 or D <= 0 (F set to 0). */
static int lw_field(const double *n_obs, double R, int flags, const double *r,
                    const double *beta, const double *bdot, double *F) {
    double n[3];
    double scale = 1.0, dist = R;
    F[0] = F[1] = F[2] = 0.0;
    if (flags & FLAG_EXACT) {
        double d[3] = {R * n_obs[0] - r[0], R * n_obs[1] - r[1], R * n_obs[2] - r[2]};
        dist = sqrt(dot3(d, d));
        n[0] = d[0] / dist;
        n[1] = d[1] / dist;
        n[2] = d[2] / dist;
        scale = R / dist;
    } else {
        n[0] = n_obs[0];
        n[1] = n_obs[1];
        n[2] = n_obs[2];
    }
    double b2 = dot3(beta, beta);
    double D = 1.0 - dot3(n, beta);
    if (!(b2 < 1.0) || !(D > 0.0)) return ST_BETA;
    double D3 = D * D * D;
    double nmb[3] = {n[0] - beta[0], n[1] - beta[1], n[2] - beta[2]};
    if (flags & FLAG_ACCEL) {
        double inner[3], outer[3];
        cross3(nmb, bdot, inner);
        cross3(n, inner, outer);
        F[0] += scale * outer[0] / D3;
        F[1] += scale * outer[1] / D3;
        F[2] += scale * outer[2] / D3;
    }
    if (flags & FLAG_VELOCITY) {
        double g = OR_C0 * (1.0 - b2) / (D3 * dist);
        F[0] += scale * nmb[0] * g;
        F[1] += scale * nmb[1] * g;
        F[2] += scale * nmb[2] * g;
    }
    return 0;
}

static int finite3(const double *v) {
    return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}

/* Bounds of the uniform observer grid, Eqs. (tu_min) and (tu_max):
 *   t_u^min = min over (k, m) of t_a^{k,m}(t_start),
 *   t_u^max = max over (k, m) of t_a^{k,m}(t_end). */
/* Step 3-4 of oracle_tdm_grad for one sample: dL/d(r, beta, beta_dot) added from
 * dL/dE (gE) and dL/dt_a (gta) of the sample, E its far acceleration field. */
static void field_gradient(const double *n, const double *b, const double *a, const double *E,
                           const double *gE, double gta, double *o_r, double *o_b, double *o_a) {
    for (int d = 0; d < 3; ++d) o_r[d] += -gta * n[d] / OR_C0;
    const double D = 1.0 - dot3(n, b);
    if (!(dot3(b, b) < 1.0) || !(D > 0.0)) return;
    const double D3 = D * D * D;
    const double nmb[3] = {n[0] - b[0], n[1] - b[1], n[2] - b[2]};
    for (int d = 0; d < 3; ++d) {
        double e[3] = {0.0, 0.0, 0.0}, inner[3], dE[3];
        e[d] = 1.0;
        /* dE/dbeta_dot_d = n x ((n - beta) x e_d) / D^3 */
        cross3(nmb, e, inner);
        cross3(n, inner, dE);
        o_a[d] += (gE[0] * dE[0] + gE[1] * dE[1] + gE[2] * dE[2]) / D3;
        /* dE/dbeta_d = n x (-e_d x beta_dot) / D^3 + 3 n_d E / D */
        cross3(e, a, inner);
        cross3(n, inner, dE);
        double s = -(gE[0] * dE[0] + gE[1] * dE[1] + gE[2] * dE[2]) / D3;
        s += 3.0 * n[d] * dot3(gE, E) / D;
        o_b[d] += s;
    }
}

int oracle_grid_bounds(int64_t n_e, int64_t n_s, const double *t, int t_per_electron,
                       const double *r, const double *beta, const double *beta_dot,
                       int64_t n_pix, const double *n_hat, double R, int flags,
                       double *t_min_out, double *t_max_out) {
    or_traj tr = {n_e, n_s, t, t_per_electron, r, beta, beta_dot};
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t m = 0; m < n_pix; ++m) {
        const double *n = n_hat + 3 * m;
        for (int64_t k = 0; k < n_e; ++k) {
            double a0, a1;
            if (flags & FLAG_EXACT) {
                a0 = advanced_time_exact(n, R, tr_vec(r, &tr, k, 0), tr_time(&tr, k, 0));
                a1 = advanced_time_exact(n, R, tr_vec(r, &tr, k, n_s), tr_time(&tr, k, n_s));
            } else {
                a0 = advanced_time_far(n, tr_vec(r, &tr, k, 0), tr_time(&tr, k, 0));
                a1 = advanced_time_far(n, tr_vec(r, &tr, k, n_s), tr_time(&tr, k, n_s));
            }
            if (a0 < lo) lo = a0;
            if (a1 > hi) hi = a1;
        }
    }
    *t_min_out = lo;
    *t_max_out = hi;
    return 0;
}

/* All advanced times t_a[m][k][i] (far field or exact); for tests. */
int oracle_advanced_times(int64_t n_e, int64_t n_s, const double *t, int t_per_electron,
                          const double *r, int64_t n_pix, const double *n_hat, double R,
                          int flags, double *ta_out) {
    or_traj tr = {n_e, n_s, t, t_per_electron, r, NULL, NULL};
    for (int64_t m = 0; m < n_pix; ++m)
        for (int64_t k = 0; k < n_e; ++k)
            for (int64_t i = 0; i <= n_s; ++i) {
                const double *x = tr_vec(r, &tr, k, i);
                double tt = tr_time(&tr, k, i);
                ta_out[(m * n_e + k) * (n_s + 1) + i] =
                    (flags & FLAG_EXACT) ? advanced_time_exact(n_hat + 3 * m, R, x, tt)
                                         : advanced_time_far(n_hat + 3 * m, x, tt);
            }
    return 0;
}

/* Field samples F[m][k][i][3] (for tests). Returns OR of status bits. */
int oracle_fields(int64_t n_e, int64_t n_s, const double *r, const double *beta,
                  const double *beta_dot, int64_t n_pix, const double *n_hat, double R,
                  int flags, double *F_out) {
    or_traj tr = {n_e, n_s, NULL, 0, r, beta, beta_dot};
    int st = 0;
    for (int64_t m = 0; m < n_pix; ++m)
        for (int64_t k = 0; k < n_e; ++k)
            for (int64_t i = 0; i <= n_s; ++i)
                st |= lw_field(n_hat + 3 * m, R, flags, tr_vec(r, &tr, k, i),
                               tr_vec(beta, &tr, k, i), tr_vec(beta_dot, &tr, k, i),
                               F_out + 3 * ((m * n_e + k) * (n_s + 1) + i));
    return st;
}

/* Time-domain method, Algorithm 2, for every detector pixel (sensor).
 *
 * For one observation direction n the algorithm keeps, per particle k, a
 * buffer (t_b, E_b) holding the arrival time and field of the previous step.
 * In every simulation step i (outer loop) and for every particle k (inner
 * loop) it evaluates t_a (Eq. far_adv) and the field E (Eq. far_efield), adds
 * to every grid point t_u in (t_b, t_a] the linear interpolant
 *   E_b (t_a - t_u)/(t_a - t_b) + E (t_u - t_b)/(t_a - t_b),
 * and then stores (t_a, E) in the buffer.  Pixels are independent, which is
 * the paper's detector parallelization; they run as OpenMP threads here.
 *
 * rec must hold n_pix*3*n_bins doubles.  accumulate==0 zeroes it first. */
int oracle_tdm_deposit(int64_t n_e, int64_t n_s, const double *t, int t_per_electron,
                       const double *r, const double *beta, const double *beta_dot,
                       int64_t n_pix, const double *n_hat, double R, double t_min,
                       double dt_u, int64_t n_bins, int flags, int accumulate,
                       double *rec, int *status) {
    or_traj tr = {n_e, n_s, t, t_per_electron, r, beta, beta_dot};
    const double inv_dt_u = 1.0 / dt_u;
    int st_all = 0;
    if (!accumulate) memset(rec, 0, sizeof(double) * (size_t)(n_pix * 3 * n_bins));

    /* per-electron checks of the lab time */
    for (int64_t k = 0; k < (t_per_electron ? n_e : 1); ++k)
        for (int64_t i = 0; i <= n_s; ++i) {
            double ti = tr_time(&tr, k, i);
            if (!isfinite(ti)) st_all |= ST_NONFINITE;
            if (i > 0 && !(ti > tr_time(&tr, k, i - 1))) st_all |= ST_TIME;
        }

#pragma omp parallel for schedule(dynamic, 1) reduction(| : st_all)
    for (int64_t m = 0; m < n_pix; ++m) {
        const double *n = n_hat + 3 * m;
        double *out = rec + m * 3 * n_bins;
        double *tb = (double *)malloc(sizeof(double) * (size_t)n_e);
        double *Eb = (double *)malloc(sizeof(double) * 3 * (size_t)n_e);
        int st = 0;
        for (int64_t i = 0; i <= n_s; ++i) {
            for (int64_t k = 0; k < n_e; ++k) {
                const double *x = tr_vec(r, &tr, k, i);
                const double *b = tr_vec(beta, &tr, k, i);
                const double *bd = tr_vec(beta_dot, &tr, k, i);
                double tt = tr_time(&tr, k, i);
                if (!finite3(x) || !finite3(b) || !finite3(bd)) st |= ST_NONFINITE;
                double ta = (flags & FLAG_EXACT) ? advanced_time_exact(n, R, x, tt)
                                                 : advanced_time_far(n, x, tt);
                double E[3];
                st |= lw_field(n, R, flags, x, b, bd, E);
                if (i > 0) {
                    double ua = (ta - t_min) * inv_dt_u;
                    double ub = (tb[k] - t_min) * inv_dt_u;
                    if (!(fabs(ua) < 4.0e18) || !(fabs(ub) < 4.0e18)) {
                        st |= ST_NONFINITE;
                    } else {
                        int64_t j_hi = (int64_t)floor(ua);
                        int64_t j_lo = (int64_t)floor(ub) + 1;
                        if (!(ta > tb[k])) st |= ST_TA_ORDER;
                        if (j_lo <= j_hi) {
                            int64_t a = j_lo, z = j_hi;
                            if (a < 0) { a = 0; st |= ST_CLIP; }
                            if (z > n_bins - 1) { z = n_bins - 1; st |= ST_CLIP; }
                            for (int64_t j = a; j <= z; ++j) {
                                double tu = t_min + (double)j * dt_u;
                                double wa = (ta - tu) / (ta - tb[k]);
                                double wb = (tu - tb[k]) / (ta - tb[k]);
                                for (int c = 0; c < 3; ++c)
                                    out[c * n_bins + j] += Eb[3 * k + c] * wa + E[c] * wb;
                            }
                        }
                    }
                }
                tb[k] = ta;
                Eb[3 * k + 0] = E[0];
                Eb[3 * k + 1] = E[1];
                Eb[3 * k + 2] = E[2];
            }
        }
        free(tb);
        free(Eb);
        st_all |= st;
    }
    if (status) *status |= st_all;
    return 0;
}

/* In-place iterative radix-2 FFT with the paper's sign convention
 * (Eq. efield_xfrom uses exp(+j omega t)):
 *   X_l = sum_{j=0}^{n-1} x_j exp(+2 pi i j l / n),   n a power of two.
 * Twiddles are evaluated directly with cos/sin (no recurrence). */
int oracle_fft(int64_t n, double *re, double *im) {
    if (n < 1 || (n & (n - 1))) return -1;
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double tr_ = re[i]; re[i] = re[j]; re[j] = tr_;
            double ti_ = im[i]; im[i] = im[j]; im[j] = ti_;
        }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t half = len >> 1;
        for (int64_t q = 0; q < half; ++q) {
            double ang = 2.0 * OR_PI * (double)q / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int64_t s = 0; s < n; s += len) {
                int64_t a = s + q, b = s + q + half;
                double xr = re[b] * wr - im[b] * wi;
                double xi = re[b] * wi + im[b] * wr;
                re[b] = re[a] - xr;
                im[b] = im[a] - xi;
                re[a] = re[a] + xr;
                im[a] = im[a] + xi;
            }
        }
    }
    return 0;
}

/* Direct O(n^2) DFT with the same convention (any n); the FFT's checker. */
int oracle_dft(int64_t n, const double *re, const double *im, double *out_re, double *out_im) {
    for (int64_t l = 0; l < n; ++l) {
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            int64_t p = (j * l) % n;
            double ang = 2.0 * OR_PI * (double)p / (double)n;
            double c = cos(ang), s = sin(ang);
            sr += re[j] * c - im[j] * s;
            si += re[j] * s + im[j] * c;
        }
        out_re[l] = sr;
        out_im[l] = si;
    }
    return 0;
}

/* Spectral-angular distribution from the time records.
 * Substituting Eq. (far_efield) into the definition of d2I/domega dOmega
 * (Eq. efield_xfrom and the expression before it) and replacing the time
 * integral by the grid sum gives
 *   S_m(omega_l) = q^2 dt_u^2 / (16 pi^3 eps0 c0) * sum_c |X_{m,c}(l)|^2,
 *   X_{m,c}(l) = sum_j rec[m][c][j] exp(+2 pi i j l / n_bins),
 * at omega_l = 2 pi l / (n_bins dt_u), l = 0..n_bins/2 (the constant
 * prefactor is the one printed in Eq. const_phase_drop).
 * X_out (nullable) receives X as [n_pix][3][n_bins/2+1][2]. */
int oracle_spectrum(int64_t n_pix, int64_t n_bins, const double *rec, double dt_u, double q,
                    double *S, double *X_out) {
    if (n_bins < 2 || (n_bins & (n_bins - 1))) return -1;
    const int64_t nl = n_bins / 2 + 1;
    const double K = q * q / (16.0 * OR_PI * OR_PI * OR_PI * OR_EPS0 * OR_C0);
    const double scale = K * dt_u * dt_u;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t m = 0; m < n_pix; ++m) {
        double *re = (double *)malloc(sizeof(double) * (size_t)n_bins);
        double *im = (double *)malloc(sizeof(double) * (size_t)n_bins);
        for (int64_t l = 0; l < nl; ++l) S[m * nl + l] = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double *x = rec + (m * 3 + c) * n_bins;
            for (int64_t j = 0; j < n_bins; ++j) { re[j] = x[j]; im[j] = 0.0; }
            oracle_fft(n_bins, re, im);
            for (int64_t l = 0; l < nl; ++l) {
                S[m * nl + l] += scale * (re[l] * re[l] + im[l] * im[l]);
                if (X_out) {
                    X_out[2 * ((m * 3 + c) * nl + l) + 0] = re[l];
                    X_out[2 * ((m * 3 + c) * nl + l) + 1] = im[l];
                }
            }
        }
        free(re);
        free(im);
    }
    return 0;
}

/* Gradient of L = sum_m sum_{l=0}^{N/2} g[m][l] S[m][l] (S as oracle_spectrum with charge q)
 * of the far acceleration field's spectra, with respect to every sample's r, beta and
 * beta_dot (added to dr, dbeta, dbdot [n_e][n_s+1][3]), by the chain rule written out:
 *  1. the record of oracle_tdm_deposit (Algorithm 2) and its DFT X (Eq. efield_xfrom),
 *     S = K dt_u^2 sum_c |X_c|^2 (Eq. const_phase_drop), so
 *     dL/drec_c[j] = K dt_u^2 sum_{l=0}^{N/2} g_l 2 Re(conj(X_c(l)) exp(+2 pi i j l / N))
 *     (a direct sum over l);
 *  2. Algorithm 2's value at grid point t_j of the step (t_b, t_a],
 *     E_b (t_a - t_j)/(t_a - t_b) + E_a (t_j - t_b)/(t_a - t_b), differentiated with
 *     respect to E_b, E_a, t_a and t_b;
 *  3. t_a = t - n.r / c0 (Eq. far_adv): dL/dr = -(dL/dt_a) n / c0;
 *  4. E = n x ((n - beta) x beta_dot) / D^3, D = 1 - n.beta (Eq. far_efield):
 *     dE/dbeta_dot_d = n x ((n - beta) x e_d) / D^3,
 *     dE/dbeta_d = n x (-e_d x beta_dot) / D^3 + 3 n_d E / D
 *     (e_d the unit vector d), each applied with the cross products literally.
 * Samples with |beta| >= 1 or D <= 0 carry no field and get no field gradient. */
int oracle_tdm_grad(int64_t n_e, int64_t n_s, const double *t, int t_per_electron,
                    const double *r, const double *beta, const double *beta_dot,
                    int64_t n_pix, const double *n_hat, double t_min, double dt_u,
                    int64_t n_bins, const double *g, double q, double *dr, double *dbeta,
                    double *dbdot) {
    if (n_bins < 2 || (n_bins & (n_bins - 1))) return -1;
    or_traj tr = {n_e, n_s, t, t_per_electron, r, beta, beta_dot};
    const int64_t nl = n_bins / 2 + 1;
    const double K = q * q / (16.0 * OR_PI * OR_PI * OR_PI * OR_EPS0 * OR_C0);
    const double scale = K * dt_u * dt_u;
    const double inv_dt_u = 1.0 / dt_u;
    const size_t n_rec = (size_t)(n_pix * 3 * n_bins);
    double *rec = (double *)malloc(sizeof(double) * n_rec);
    double *drec = (double *)malloc(sizeof(double) * n_rec);
    int st = 0;
    oracle_tdm_deposit(n_e, n_s, t, t_per_electron, r, beta, beta_dot, n_pix, n_hat, 1.0, t_min,
                       dt_u, n_bins, FLAG_ACCEL, 0, rec, &st);
    /* step 1: dL/drec by direct sums */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t row = 0; row < n_pix * 3; ++row) {
        const int64_t m = row / 3;
        const double *x = rec + row * n_bins;
        double *Xre = (double *)malloc(sizeof(double) * (size_t)nl);
        double *Xim = (double *)malloc(sizeof(double) * (size_t)nl);
        for (int64_t l = 0; l < nl; ++l) {
            double re = 0.0, im = 0.0;
            for (int64_t j = 0; j < n_bins; ++j) {
                double ang = 2.0 * OR_PI * (double)((j * l) % n_bins) / (double)n_bins;
                re += x[j] * cos(ang);
                im += x[j] * sin(ang);
            }
            Xre[l] = re;
            Xim[l] = im;
        }
        for (int64_t j = 0; j < n_bins; ++j) {
            double acc = 0.0;
            for (int64_t l = 0; l < nl; ++l) {
                double ang = 2.0 * OR_PI * (double)((j * l) % n_bins) / (double)n_bins;
                /* Re(conj(X) e^{i ang}) = Xre cos + Xim sin */
                acc += g[m * nl + l] * 2.0 * (Xre[l] * cos(ang) + Xim[l] * sin(ang));
            }
            drec[row * n_bins + j] = scale * acc;
        }
        free(Xre);
        free(Xim);
    }
    /* steps 2-4, electron by electron (each writes only its own samples) */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n_e; ++k) {
        for (int64_t m = 0; m < n_pix; ++m) {
            const double *n = n_hat + 3 * m;
            const double *R = drec + m * 3 * n_bins;
            double tb = 0.0, Eb[3] = {0.0, 0.0, 0.0};
            double gEb[3] = {0.0, 0.0, 0.0}, gtb = 0.0;   /* dL/d(E, t_a) of sample i-1 */
            for (int64_t i = 0; i <= n_s; ++i) {
                const double *xi = tr_vec(r, &tr, k, i);
                const double *bi = tr_vec(beta, &tr, k, i);
                const double *ai = tr_vec(beta_dot, &tr, k, i);
                const double ta = advanced_time_far(n, xi, tr_time(&tr, k, i));
                double E[3];
                lw_field(n, 1.0, FLAG_ACCEL, xi, bi, ai, E);
                double gE[3] = {0.0, 0.0, 0.0}, gta = 0.0;   /* sample i */
                if (i > 0) {
                    const double ua = (ta - t_min) * inv_dt_u, ub = (tb - t_min) * inv_dt_u;
                    if (fabs(ua) < 4.0e18 && fabs(ub) < 4.0e18) {
                        int64_t a = (int64_t)floor(ub) + 1, z = (int64_t)floor(ua);
                        if (a < 0) a = 0;
                        if (z > n_bins - 1) z = n_bins - 1;
                        const double den = ta - tb;
                        for (int64_t j = a; j <= z; ++j) {
                            const double tu = t_min + (double)j * dt_u;
                            for (int c = 0; c < 3; ++c) {
                                const double Rc = R[c * n_bins + j];
                                gEb[c] += Rc * (ta - tu) / den;
                                gE[c] += Rc * (tu - tb) / den;
                                /* d/dt_a and d/dt_b of Eb (ta-tu)/den + E (tu-tb)/den */
                                gta += Rc * (Eb[c] - E[c]) * (tu - tb) / (den * den);
                                gtb += Rc * (Eb[c] - E[c]) * (ta - tu) / (den * den);
                            }
                        }
                    }
                    /* sample i-1 is complete */
                    double *o_r = dr + 3 * (k * (n_s + 1) + i - 1);
                    double *o_b = dbeta + 3 * (k * (n_s + 1) + i - 1);
                    double *o_a = dbdot + 3 * (k * (n_s + 1) + i - 1);
                    field_gradient(n, tr_vec(beta, &tr, k, i - 1), tr_vec(beta_dot, &tr, k, i - 1),
                                   Eb, gEb, gtb, o_r, o_b, o_a);
                }
                tb = ta;
                for (int c = 0; c < 3; ++c) {
                    Eb[c] = E[c];
                    gEb[c] = gE[c];
                }
                gtb = gta;
            }
            double *o_r = dr + 3 * (k * (n_s + 1) + n_s);
            double *o_b = dbeta + 3 * (k * (n_s + 1) + n_s);
            double *o_a = dbdot + 3 * (k * (n_s + 1) + n_s);
            field_gradient(n, tr_vec(beta, &tr, k, n_s), tr_vec(beta_dot, &tr, k, n_s), Eb, gEb,
                           gtb, o_r, o_b, o_a);
        }
    }
    free(rec);
    free(drec);
    return st;
}

/* Frequency-domain method, Eq. (inty_dft) / Algorithm 1:
 *   S(n, omega) = q^2 dt^2 / (16 pi^3 eps0 c0)
 *                 |sum_k sum_{i=0}^{n_s} A_k(n, t_i) exp(j omega (t_i - n.x'_k(t_i)/c0))|^2
 *   A_k = n x ((n - beta) x beta_dot) / (1 - n.beta)^2.
 * The phase uses the same far-field advanced time as the time-domain method
 * (constant |x|/c0 dropped).  Algorithm 1 accumulates E_bunch over particles
 * per step and then E_sum over steps; that order is kept.
 * S_out is [n_pix][n_omega]. */
int oracle_fdm(int64_t n_e, int64_t n_s, const double *t, int t_per_electron, const double *r,
               const double *beta, const double *beta_dot, int64_t n_pix, const double *n_hat,
               int64_t n_omega, const double *omega, double dt, double q, double *S_out) {
    or_traj tr = {n_e, n_s, t, t_per_electron, r, beta, beta_dot};
    const double K = q * q / (16.0 * OR_PI * OR_PI * OR_PI * OR_EPS0 * OR_C0);
    int st_all = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) reduction(| : st_all)
    for (int64_t m = 0; m < n_pix; ++m) {
        for (int64_t w = 0; w < n_omega; ++w) {
            const double *n = n_hat + 3 * m;
            double sum_re[3] = {0, 0, 0}, sum_im[3] = {0, 0, 0};
            for (int64_t i = 0; i <= n_s; ++i) {
                double bun_re[3] = {0, 0, 0}, bun_im[3] = {0, 0, 0};
                for (int64_t k = 0; k < n_e; ++k) {
                    const double *x = tr_vec(r, &tr, k, i);
                    const double *b = tr_vec(beta, &tr, k, i);
                    const double *bd = tr_vec(beta_dot, &tr, k, i);
                    double D = 1.0 - dot3(n, b);
                    if (!(D > 0.0) || !(dot3(b, b) < 1.0)) { st_all |= ST_BETA; continue; }
                    double nmb[3] = {n[0] - b[0], n[1] - b[1], n[2] - b[2]};
                    double inner[3], A[3];
                    cross3(nmb, bd, inner);
                    cross3(n, inner, A);
                    double phase = omega[w] * advanced_time_far(n, x, tr_time(&tr, k, i));
                    double cr = cos(phase), ci = sin(phase);
                    for (int c = 0; c < 3; ++c) {
                        double a = A[c] / (D * D);
                        bun_re[c] += a * cr;
                        bun_im[c] += a * ci;
                    }
                }
                for (int c = 0; c < 3; ++c) {
                    sum_re[c] += bun_re[c];
                    sum_im[c] += bun_im[c];
                }
            }
            double s = 0.0;
            for (int c = 0; c < 3; ++c) s += sum_re[c] * sum_re[c] + sum_im[c] * sum_im[c];
            S_out[m * n_omega + w] = K * dt * dt * s;
        }
    }
    return st_all;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
