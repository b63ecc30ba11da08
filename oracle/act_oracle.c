/*
 * FP64 CPU oracle for residual-projection matching pursuit over a
 * unit-normalised Gaussian-chirplet dictionary.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant with the CUDA implementation and never
 * includes or links anything of it.
 *
 * What it follows (all in double precision, plain loops, no blocking):
 *   - Eq. (1): the Gaussian chirplet g(t) with parameters (tc, fc, logDt, c),
 *     including its analytic prefactor (act_oracle_atom_complex).
 *   - Sec. III-A: every dictionary atom normalised to unit l2 norm before the
 *     search; the dictionary is a finite grid sampled from user ranges; the
 *     ranges of Table 2 are half-open (start, stop, step) sequences.
 *   - Eq. (4) and Fig. 1: r_0 = s; at every order k pick
 *     i* = argmax_i |<g_i, r_k>|, take c_k = <g*, r_k>, set
 *     r_{k+1} = r_k - c_k g*.
 *   - Fig. 1's refinement step theta* = argmax_theta |<g(theta), r_k>| by
 *     BFGS from the grid winner (Sec. III-A): the analytic gradient of the
 *     score and a plain BFGS with Armijo backtracking in grid-step-scaled
 *     coordinates (act_oracle_score_grad, act_oracle_refine,
 *     act_oracle_mp_refine).
 *   - Eq. (5): the normalised residue |r_k|^2 / |s|^2 is derived from the
 *     recorded residual energies.
 *
 * Readings where the paper is silent (each one also stated in the design
 * notes):
 *   - atoms are the real part of Eq. (1): signals are real, so coefficients
 *     and residuals stay real;
 *   - the prefactor of Eq. (1) is dropped for dictionary atoms, which are
 *     divided by their discrete l2 norm over the window instead;
 *   - tc is in samples, tau = (n - tc) / fs seconds, fc in Hz, c in Hz/s as
 *     it multiplies tau^2 in Eq. (1), Dt = exp(logDt) seconds;
 *   - ties in |score| go to the lowest flat index
 *     flat = ((i_tc * N_fc + i_fc) * N_logDt + i_logDt) * N_c + i_c;
 *   - an atom whose squared norm is below 1e-300 or not finite is
 *     degenerate: it is stored as zeros and scores 0;
 *   - with a zero residual every score is 0, index 0 is chosen with c_k = 0.
 *
 * Parallelism: the per-atom loops (generation, scoring) are split across
 * OpenMP threads; every reduction that decides a result (argmax, norms,
 * dot products) runs sequentially in index order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* ---------------------------------------------------------------------- */
/* Threads                                                                 */
/* ---------------------------------------------------------------------- */
void act_oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int act_oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Grid (Sec. III-A, Table 2)                                              */
/* ---------------------------------------------------------------------- */

/* Number of values of a half-open range start, start+step, ... < stop,
 * the way Table 2 ranges are enumerated: ceil((stop - start) / step). */
int64_t act_oracle_range_count(double start, double stop, double step) {
    if (!(step > 0.0)) return -1;
    double n = ceil((stop - start) / step);
    if (n < 0.0) n = 0.0;
    return (int64_t)n;
}

/* axes[8] = {tc_lo, tc_step, fc_lo, fc_step, ld_lo, ld_step, c_lo, c_step},
 * counts[4] = {N_tc, N_fc, N_logDt, N_c}.  Writes the parameters of one
 * flat index. */
void act_oracle_atom_params(const double *axes, const int64_t *counts, int64_t flat,
                            double *tc, double *fc, double *logdt, double *c) {
    int64_t ic = flat % counts[3];
    int64_t rest = flat / counts[3];
    int64_t il = rest % counts[2];
    rest /= counts[2];
    int64_t ifc = rest % counts[1];
    int64_t itc = rest / counts[1];
    *tc = axes[0] + (double)itc * axes[1];
    *fc = axes[2] + (double)ifc * axes[3];
    *logdt = axes[4] + (double)il * axes[5];
    *c = axes[6] + (double)ic * axes[7];
}

static int64_t grid_size(const int64_t *counts) {
    return counts[0] * counts[1] * counts[2] * counts[3];
}

/* ---------------------------------------------------------------------- */
/* Atoms (Eq. 1, Sec. III-A)                                               */
/* ---------------------------------------------------------------------- */

/* Eq. (1) as printed, sampled at t = n / fs for n = 0..n_samples-1:
 *   g(t) = (sqrt(pi) Dt)^(-1/2) exp(-1/2 ((t - tc)/Dt)^2)
 *          exp(i 2 pi [c (t - tc)^2 + fc (t - tc)]),   Dt = exp(logDt). */
void act_oracle_atom_complex(double tc, double fc, double logdt, double c, double fs,
                             int n_samples, double *re, double *im) {
    double dt = exp(logdt);
    double pref = 1.0 / sqrt(sqrt(ORACLE_PI) * dt);
    for (int n = 0; n < n_samples; ++n) {
        double tau = ((double)n - tc) / fs;
        double env = pref * exp(-0.5 * (tau / dt) * (tau / dt));
        double phase = 2.0 * ORACLE_PI * (c * tau * tau + fc * tau);
        re[n] = env * cos(phase);
        im[n] = env * sin(phase);
    }
}

/* Dictionary atom: the real part of Eq. (1) without its prefactor, divided
 * by its discrete l2 norm over the window.  Returns 1 (and zeros) for a
 * degenerate atom, 0 otherwise. */
int act_oracle_atom(double tc, double fc, double logdt, double c, double fs,
                    int n_samples, double *g) {
    double dt = exp(logdt);
    double energy = 0.0;
    for (int n = 0; n < n_samples; ++n) {
        double tau = ((double)n - tc) / fs;
        double env = exp(-0.5 * (tau / dt) * (tau / dt));
        double phase = 2.0 * ORACLE_PI * (c * tau * tau + fc * tau);
        g[n] = env * cos(phase);
        energy += g[n] * g[n];
    }
    if (!(energy >= 1e-300) || !isfinite(energy)) {
        for (int n = 0; n < n_samples; ++n) g[n] = 0.0;
        return 1;
    }
    double norm = sqrt(energy);
    for (int n = 0; n < n_samples; ++n) g[n] /= norm;
    return 0;
}

/* The whole dictionary D[K][n_samples], row = flat index.  degenerate may be
 * NULL.  Returns the number of degenerate atoms. */
int64_t act_oracle_dictionary(const double *axes, const int64_t *counts, int n_samples,
                              double fs, double *D, uint8_t *degenerate) {
    int64_t K = grid_size(counts);
    int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = 0; i < K; ++i) {
        double tc, fc, ld, c;
        act_oracle_atom_params(axes, counts, i, &tc, &fc, &ld, &c);
        int d = act_oracle_atom(tc, fc, ld, c, fs, n_samples, D + i * (int64_t)n_samples);
        if (degenerate) degenerate[i] = (uint8_t)d;
        bad += d;
    }
    return bad;
}

/* ---------------------------------------------------------------------- */
/* Search pieces                                                           */
/* ---------------------------------------------------------------------- */
static double dot(const double *a, const double *b, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* scores[i] = <D_i, r> for a stored dictionary. */
void act_oracle_scores(const double *D, int64_t K, int n_samples, const double *r,
                       double *scores) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < K; ++i) scores[i] = dot(D + i * (int64_t)n_samples, r, n_samples);
}

/* scores[i] = <g_i, r> with every atom regenerated from the grid. */
void act_oracle_scores_grid(const double *axes, const int64_t *counts, int n_samples, double fs,
                            const double *r, double *scores) {
    int64_t K = grid_size(counts);
#pragma omp parallel
    {
        double *g = (double *)malloc(sizeof(double) * (size_t)n_samples);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < K; ++i) {
            double tc, fc, ld, c;
            act_oracle_atom_params(axes, counts, i, &tc, &fc, &ld, &c);
            act_oracle_atom(tc, fc, ld, c, fs, n_samples, g);
            scores[i] = dot(g, r, n_samples);
        }
        free(g);
    }
}

/* Selection rule: the largest |score|, lowest index on ties.  Also reports
 * the runner-up (largest |score| among the other indices) for near-tie
 * checks; second is -1 when K < 2. */
void act_oracle_select(const double *scores, int64_t K, int64_t *best, int64_t *second) {
    int64_t b = 0, s2 = -1;
    for (int64_t i = 1; i < K; ++i) {
        if (fabs(scores[i]) > fabs(scores[b])) {
            s2 = b;
            b = i;
        } else if (s2 < 0 || fabs(scores[i]) > fabs(scores[s2])) {
            s2 = i;
        }
    }
    *best = b;
    *second = s2;
}

/* ---------------------------------------------------------------------- */
/* Matching pursuit (Eq. 4, Fig. 1)                                        */
/* ---------------------------------------------------------------------- */

/* One MP order given the chosen atom g: c = <g, r>, r <- r - c g.
 * Returns c. */
static double mp_update(const double *g, double *r, int n_samples) {
    double c = dot(g, r, n_samples);
    for (int n = 0; n < n_samples; ++n) r[n] -= c * g[n];
    return c;
}

/* MP over a stored dictionary D[K][n_samples] (any dictionary, not only
 * chirplets).  Outputs: idx[P], coef[P], r[n_samples] (final residual),
 * energy[P+1] = |r_k|^2 for k = 0..P (energy may be NULL).  Returns 0. */
int act_oracle_mp(const double *D, int64_t K, int n_samples, const double *s, int P,
                  int64_t *idx, double *coef, double *r, double *energy) {
    double *scores = (double *)malloc(sizeof(double) * (size_t)K);
    if (!scores) return -1;
    memcpy(r, s, sizeof(double) * (size_t)n_samples);
    if (energy) energy[0] = dot(r, r, n_samples);
    for (int k = 0; k < P; ++k) {
        int64_t best, second;
        act_oracle_scores(D, K, n_samples, r, scores);
        act_oracle_select(scores, K, &best, &second);
        idx[k] = best;
        coef[k] = mp_update(D + best * (int64_t)n_samples, r, n_samples);
        if (energy) energy[k + 1] = dot(r, r, n_samples);
    }
    free(scores);
    return 0;
}

/* MP over a chirplet grid with every atom regenerated at every order (for
 * grids whose FP64 dictionary would not fit in host memory).  Same outputs
 * as act_oracle_mp; gap[P] (may be NULL) receives the relative gap
 * (|s_best| - |s_second|) / |s_best| of each order (0 when |s_best| = 0). */
int act_oracle_mp_grid(const double *axes, const int64_t *counts, int n_samples, double fs,
                       const double *s, int P, int64_t *idx, double *coef, double *r,
                       double *energy, double *gap) {
    int64_t K = grid_size(counts);
    double *scores = (double *)malloc(sizeof(double) * (size_t)K);
    double *g = (double *)malloc(sizeof(double) * (size_t)n_samples);
    if (!scores || !g) {
        free(scores);
        free(g);
        return -1;
    }
    memcpy(r, s, sizeof(double) * (size_t)n_samples);
    if (energy) energy[0] = dot(r, r, n_samples);
    for (int k = 0; k < P; ++k) {
        int64_t best, second;
        act_oracle_scores_grid(axes, counts, n_samples, fs, r, scores);
        act_oracle_select(scores, K, &best, &second);
        if (gap) {
            double a = fabs(scores[best]);
            double b = second >= 0 ? fabs(scores[second]) : 0.0;
            gap[k] = a > 0.0 ? (a - b) / a : 0.0;
        }
        double tc, fc, ld, c;
        act_oracle_atom_params(axes, counts, best, &tc, &fc, &ld, &c);
        act_oracle_atom(tc, fc, ld, c, fs, n_samples, g);
        idx[k] = best;
        coef[k] = mp_update(g, r, n_samples);
        if (energy) energy[k + 1] = dot(r, r, n_samples);
    }
    free(scores);
    free(g);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Off-grid refinement (Fig. 1: theta* = argmax_theta |<g(theta), r_k>|,  */
/* started from the grid winner)                                           */
/* ---------------------------------------------------------------------- */

/* s(theta) = <r, g(theta)> for the unit-norm real atom of Eq. (1) at
 * continuous theta = (tc, fc, logDt, c), and its gradient.  With
 * u = E cos(phi), E = exp(-x^2/2), x = tau/Dt, phi = 2 pi (c tau^2 + fc tau),
 * tau = (n - tc)/fs and g = u/|u|:
 *   ds/dtheta_i = <r, du_i>/|u| - s <u, du_i>/|u|^2, where
 *   du/dtc    = (E x/Dt cos(phi) + E sin(phi) 2 pi (2 c tau + fc)) / fs,
 *   du/dfc    = -E sin(phi) 2 pi tau,
 *   du/dlogDt = E x^2 cos(phi),
 *   du/dc     = -E sin(phi) 2 pi tau^2.
 * Returns 1 for a degenerate atom (score and gradient 0). grad may be NULL. */
int act_oracle_score_grad(const double *theta, double fs, int n_samples, const double *r, double *score,
                          double *grad) {
    const double tc = theta[0], fc = theta[1], ld = theta[2], c = theta[3];
    const double dt = exp(ld);
    double ru = 0.0, uu = 0.0, rd[4] = {0, 0, 0, 0}, ud[4] = {0, 0, 0, 0};
    for (int n = 0; n < n_samples; ++n) {
        const double tau = ((double)n - tc) / fs;
        const double x = tau / dt;
        const double E = exp(-0.5 * x * x);
        const double phi = 2.0 * ORACLE_PI * (c * tau * tau + fc * tau);
        const double C = cos(phi), S = sin(phi);
        const double u = E * C;
        double du[4];
        du[0] = (E * x / dt * C + E * S * 2.0 * ORACLE_PI * (2.0 * c * tau + fc)) / fs;
        du[1] = -E * S * 2.0 * ORACLE_PI * tau;
        du[2] = E * x * x * C;
        du[3] = -E * S * 2.0 * ORACLE_PI * tau * tau;
        ru += r[n] * u;
        uu += u * u;
        for (int i = 0; i < 4; ++i) {
            rd[i] += r[n] * du[i];
            ud[i] += u * du[i];
        }
    }
    if (!(uu >= 1e-300) || !isfinite(uu)) {
        *score = 0.0;
        if (grad)
            for (int i = 0; i < 4; ++i) grad[i] = 0.0;
        return 1;
    }
    const double nu = sqrt(uu);
    const double s = ru / nu;
    *score = s;
    if (grad)
        for (int i = 0; i < 4; ++i) grad[i] = rd[i] / nu - s * ud[i] / uu;
    return 0;
}

/* Refinement by BFGS on f(z) = -|s(theta)|, theta = w (.) z (coordinates
 * scaled by w, the grid steps), from theta (updated in place), `steps`
 * iterations of:
 *   p = -H grad f              (H: inverse-Hessian estimate, starts at I;
 *                               reset to I when p is not a descent direction)
 *   alpha = min(1, 1/(2|p|))   (a first step of at most half a grid step)
 *   halve alpha (up to 20 times) until the Armijo condition
 *     f(z + alpha p) <= f(z) + 1e-4 alpha <grad f, p> holds
 *   z' = clamp(z + alpha p);  s = z' - z;  y = grad f(z') - grad f(z)
 *   if <y, s> > 0:  H = (I - s y^T / <y,s>) H (I - y s^T / <y,s>) + s s^T / <y,s>
 * stopping early when no step is accepted.  lo/hi[4] clamp theta.
 * Returns the final |s|. */
static void scaled_eval(const double *th, const double *w, double fs, int n, const double *r, double *f,
                        double *gz) {
    double s, g[4];
    act_oracle_score_grad(th, fs, n, r, &s, g);
    const double sg = s < 0.0 ? -1.0 : 1.0;
    *f = -fabs(s);
    for (int i = 0; i < 4; ++i) gz[i] = -sg * g[i] * w[i];
}

double act_oracle_refine(double *theta, double fs, int n_samples, const double *r, int steps, const double *w,
                         const double *lo, const double *hi) {
    /* z: scaled coordinates; theta itself is kept alongside, so a start
     * that is never improved is returned bit for bit */
    double z[4], gz[4], f, H[16];
    for (int i = 0; i < 4; ++i) z[i] = theta[i] / w[i];
    scaled_eval(theta, w, fs, n_samples, r, &f, gz);
    for (int i = 0; i < 16; ++i) H[i] = (i % 5 == 0) ? 1.0 : 0.0;
    for (int it = 0; it < steps; ++it) {
        double p[4], gp = 0.0, pn = 0.0;
        for (int i = 0; i < 4; ++i) {
            p[i] = 0.0;
            for (int j = 0; j < 4; ++j) p[i] -= H[4 * i + j] * gz[j];
            gp += gz[i] * p[i];
        }
        if (!(gp < 0.0)) {
            for (int i = 0; i < 16; ++i) H[i] = (i % 5 == 0) ? 1.0 : 0.0;
            gp = 0.0;
            for (int i = 0; i < 4; ++i) {
                p[i] = -gz[i];
                gp += gz[i] * p[i];
            }
            if (!(gp < 0.0)) break;  /* zero gradient */
        }
        for (int i = 0; i < 4; ++i) pn += p[i] * p[i];
        pn = sqrt(pn);
        double alpha = pn > 0.5 ? 0.5 / pn : 1.0;
        double z2[4], t2[4], f2 = 0.0, g2[4];
        int ok = 0;
        for (int ls = 0; ls < 20; ++ls) {
            for (int i = 0; i < 4; ++i) {
                double v = (z[i] + alpha * p[i]) * w[i];
                if (v < lo[i]) v = lo[i];
                if (v > hi[i]) v = hi[i];
                t2[i] = v;
                z2[i] = v / w[i];
            }
            scaled_eval(t2, w, fs, n_samples, r, &f2, g2);
            if (f2 <= f + 1e-4 * alpha * gp) {
                ok = 1;
                break;
            }
            alpha *= 0.5;
        }
        if (!ok) break;
        double sv[4], yv[4], ys = 0.0;
        for (int i = 0; i < 4; ++i) {
            sv[i] = z2[i] - z[i];
            yv[i] = g2[i] - gz[i];
            ys += yv[i] * sv[i];
        }
        if (ys > 1e-300) {
            /* H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T */
            const double rho = 1.0 / ys;
            double A[16], T[16];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) A[4 * i + j] = (i == j ? 1.0 : 0.0) - rho * sv[i] * yv[j];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < 4; ++k) acc += A[4 * i + k] * H[4 * k + j];
                    T[4 * i + j] = acc;
                }
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < 4; ++k) acc += T[4 * i + k] * A[4 * j + k];
                    H[4 * i + j] = acc + rho * sv[i] * sv[j];
                }
        }
        for (int i = 0; i < 4; ++i) {
            z[i] = z2[i];
            theta[i] = t2[i];
            gz[i] = g2[i];
        }
        f = f2;
    }
    return -f;
}

/* MP over a grid where every order's grid winner is refined off the grid
 * (act_oracle_refine with the grid steps as scales and the grid box
 * widened by one step) and the refined atom is subtracted.  Outputs as
 * act_oracle_mp_grid plus theta_out[P][4] (refined parameters). */
int act_oracle_mp_refine(const double *axes, const int64_t *counts, int n_samples, double fs, const double *s,
                         int P, int steps, int64_t *idx, double *coef, double *theta_out, double *r,
                         double *energy) {
    int64_t K = grid_size(counts);
    double *scores = (double *)malloc(sizeof(double) * (size_t)K);
    double *g = (double *)malloc(sizeof(double) * (size_t)n_samples);
    if (!scores || !g) {
        free(scores);
        free(g);
        return -1;
    }
    /* scales: the grid steps; box: the grid range widened by one step (an
     * axis with a zero step is held fixed) */
    double w[4], lo[4], hi[4];
    for (int i = 0; i < 4; ++i) {
        const double st = fabs(axes[2 * i + 1]);
        const double first = axes[2 * i], last = axes[2 * i] + (double)(counts[i] - 1) * axes[2 * i + 1];
        w[i] = st > 0.0 ? st : 1.0;
        lo[i] = st > 0.0 ? fmin(first, last) - st : first;
        hi[i] = st > 0.0 ? fmax(first, last) + st : first;
    }
    memcpy(r, s, sizeof(double) * (size_t)n_samples);
    if (energy) energy[0] = dot(r, r, n_samples);
    for (int k = 0; k < P; ++k) {
        int64_t best, second;
        act_oracle_scores_grid(axes, counts, n_samples, fs, r, scores);
        act_oracle_select(scores, K, &best, &second);
        double th[4];
        act_oracle_atom_params(axes, counts, best, &th[0], &th[1], &th[2], &th[3]);
        act_oracle_refine(th, fs, n_samples, r, steps, w, lo, hi);
        act_oracle_atom(th[0], th[1], th[2], th[3], fs, n_samples, g);
        idx[k] = best;
        for (int i = 0; i < 4; ++i) theta_out[4 * k + i] = th[i];
        coef[k] = mp_update(g, r, n_samples);
        if (energy) energy[k + 1] = dot(r, r, n_samples);
    }
    free(scores);
    free(g);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* LEM-inspired hierarchical search (Sec. VII-A, Fig. 7)                   */
/* ---------------------------------------------------------------------- */

/* The n-th output (n = 0, 1, ...) of SplitMix64 seeded with `seed`
 * (Steele, Lea and Flood, 2014): state advances by 0x9E3779B97F4A7C15 and
 * each output is the published mix of the state. */
uint64_t act_oracle_splitmix64_at(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Counter of one random draw: channel < 2^16, order < 2^12, axis < 4,
 * kind 0 (stratum key) or 1 (offset in the stratum), sample i < 2^20. */
static uint64_t lem_counter(int channel, int order, int axis, int kind, int i) {
    return (((((((uint64_t)channel << 12) | (uint64_t)order) << 2 | (uint64_t)axis) << 1) | (uint64_t)kind) << 20) |
           (uint64_t)i;
}

typedef struct {
    int n_coarse;          /* LHS samples of the coarse level */
    int top_k;             /* candidates kept per level */
    int levels;            /* refinement levels after the coarse level (<= 2) */
    double steps[3][4];    /* step of each level, (tc, fc, logDt, c) */
    int radius[4];         /* neighbourhood half-width in steps, per axis */
} act_oracle_lem;

/* Latin hypercube sample of n points in the box [lo, hi]: on every axis the
 * n strata of width (hi - lo)/n are each used exactly once, in a random
 * order (the ranks of SplitMix64 keys), and each point sits at a uniform
 * random offset inside its stratum:
 *   theta[i][a] = lo[a] + ((rank_a(i) + u) / n) * (hi[a] - lo[a]). */
void act_oracle_lhs(const double *lo, const double *hi, int n, uint64_t seed, int channel, int order,
                    double *theta) {
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    for (int a = 0; a < 4; ++a) {
        for (int i = 0; i < n; ++i) key[i] = act_oracle_splitmix64_at(seed, lem_counter(channel, order, a, 0, i));
        for (int i = 0; i < n; ++i) {
            int rank = 0;  /* number of keys below key[i] (keys are distinct) */
            for (int j = 0; j < n; ++j) rank += key[j] < key[i];
            const uint64_t h = act_oracle_splitmix64_at(seed, lem_counter(channel, order, a, 1, i));
            const double u = (double)(h >> 11) * 0x1.0p-53;
            const double t = ((double)rank + u) / (double)n;
            theta[4 * i + a] = lo[a] + t * (hi[a] - lo[a]);
        }
    }
    free(key);
}

static double lem_score(const double *th, double fs, int L, const double *r, double *g) {
    act_oracle_atom(th[0], th[1], th[2], th[3], fs, L, g);
    return dot(g, r, L);
}

/* The k best candidates by |score| (lowest candidate index on ties),
 * skipping candidates whose parameters equal an already kept one. */
int act_oracle_lem_topk(const double *cand, const double *score, int n, int k, double *kept, double *kept_score) {
    int m = 0;
    for (int round = 0; round < k; ++round) {
        int best = -1;
        for (int i = 0; i < n; ++i) {
            int dup = 0;
            for (int q = 0; q < m && !dup; ++q)
                dup = cand[4 * i] == kept[4 * q] && cand[4 * i + 1] == kept[4 * q + 1] &&
                      cand[4 * i + 2] == kept[4 * q + 2] && cand[4 * i + 3] == kept[4 * q + 3];
            if (dup) continue;
            if (best < 0 || fabs(score[i]) > fabs(score[best])) best = i;
        }
        if (best < 0) break;
        for (int a = 0; a < 4; ++a) kept[4 * m + a] = cand[4 * best + a];
        kept_score[m] = score[best];
        ++m;
    }
    return m;
}

/* Local neighbourhood dictionary of one level around the kept candidates:
 * for every parent (in kept order) and every offset o in
 * [-R_tc..R_tc] x [-R_fc..R_fc] x [-R_ld..R_ld] x [-R_c..R_c]
 * (c fastest), theta = clamp(parent + o * step, lo, hi).  Returns the
 * number of candidates written. */
int act_oracle_lem_neighbours(const double *kept, int m, const double *step, const int *R, const double *lo,
                              const double *hi, double *cand) {
    int n = 0;
    for (int j = 0; j < m; ++j)
        for (int o0 = -R[0]; o0 <= R[0]; ++o0)
            for (int o1 = -R[1]; o1 <= R[1]; ++o1)
                for (int o2 = -R[2]; o2 <= R[2]; ++o2)
                    for (int o3 = -R[3]; o3 <= R[3]; ++o3) {
                        const int o[4] = {o0, o1, o2, o3};
                        for (int a = 0; a < 4; ++a) {
                            double v = kept[4 * j + a] + (double)o[a] * step[a];
                            if (v < lo[a]) v = lo[a];
                            if (v > hi[a]) v = hi[a];
                            cand[4 * n + a] = v;
                        }
                        ++n;
                    }
    return n;
}

/* One hierarchical selection (Fig. 7 up to, not including, BFGS): LHS over
 * the box, projections onto r, keep top_k; then for each refinement level
 * build the neighbourhood dictionaries of the kept candidates with that
 * level's steps, project, pool and keep top_k.  Writes the best
 * candidate's parameters and score; returns 0 (or -1 on allocation
 * failure). */
int act_oracle_lem_select(const act_oracle_lem *p, const double *lo, const double *hi, double fs, int L,
                          const double *r, uint64_t seed, int channel, int order, double *theta_out,
                          double *score_out) {
    int per_parent = 1;
    for (int a = 0; a < 4; ++a) per_parent *= 2 * p->radius[a] + 1;
    int cap = p->n_coarse > p->top_k * per_parent ? p->n_coarse : p->top_k * per_parent;
    double *cand = (double *)malloc(sizeof(double) * 4 * (size_t)cap);
    double *score = (double *)malloc(sizeof(double) * (size_t)cap);
    double *g = (double *)malloc(sizeof(double) * (size_t)L);
    double *kept = (double *)malloc(sizeof(double) * 4 * (size_t)p->top_k);
    double *kept_score = (double *)malloc(sizeof(double) * (size_t)p->top_k);
    if (!cand || !score || !g || !kept || !kept_score) {
        free(cand);
        free(score);
        free(g);
        free(kept);
        free(kept_score);
        return -1;
    }
    act_oracle_lhs(lo, hi, p->n_coarse, seed, channel, order, cand);
    for (int i = 0; i < p->n_coarse; ++i) score[i] = lem_score(cand + 4 * i, fs, L, r, g);
    int m = act_oracle_lem_topk(cand, score, p->n_coarse, p->top_k, kept, kept_score);
    for (int lev = 1; lev <= p->levels; ++lev) {
        const int n = act_oracle_lem_neighbours(kept, m, p->steps[lev], p->radius, lo, hi, cand);
        for (int i = 0; i < n; ++i) score[i] = lem_score(cand + 4 * i, fs, L, r, g);
        m = act_oracle_lem_topk(cand, score, n, p->top_k, kept, kept_score);
    }
    for (int a = 0; a < 4; ++a) theta_out[a] = kept[a];
    *score_out = kept_score[0];
    free(cand);
    free(score);
    free(g);
    free(kept);
    free(kept_score);
    return 0;
}

/* MP whose every order is selected by the hierarchical search (no stored
 * dictionary), optionally refined by `steps` BFGS iterations (scales: the
 * level-0 LEM steps... see act_oracle_refine), then subtracted.
 * lo/hi: the parameter box; scale[4]: BFGS coordinate scales; box_lo/hi:
 * the BFGS clamp box.  Outputs theta_out[P][4], coef[P], r, energy[P+1]. */
int act_oracle_mp_lem(const act_oracle_lem *p, const double *lo, const double *hi, const double *scale,
                      const double *box_lo, const double *box_hi, double fs, int L, const double *s, int P,
                      int steps, uint64_t seed, int channel, double *theta_out, double *coef, double *r,
                      double *energy) {
    double *g = (double *)malloc(sizeof(double) * (size_t)L);
    if (!g) return -1;
    memcpy(r, s, sizeof(double) * (size_t)L);
    if (energy) energy[0] = dot(r, r, L);
    for (int k = 0; k < P; ++k) {
        double th[4], sc;
        if (act_oracle_lem_select(p, lo, hi, fs, L, r, seed, channel, k, th, &sc) != 0) {
            free(g);
            return -1;
        }
        if (steps > 0) act_oracle_refine(th, fs, L, r, steps, scale, box_lo, box_hi);
        act_oracle_atom(th[0], th[1], th[2], th[3], fs, L, g);
        for (int a = 0; a < 4; ++a) theta_out[4 * k + a] = th[a];
        coef[k] = mp_update(g, r, L);
        if (energy) energy[k + 1] = dot(r, r, L);
    }
    free(g);
    return 0;
}
