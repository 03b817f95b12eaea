/*
 * hermite6_oracle.c -- TEST INFRASTRUCTURE, not part of the product path.
 *
 * A plain, slow, single-threaded FP64 reference of the 6th-order Hermite
 * block-time-step integrator: the sixth-order extension of GraviDy's 4th-order
 * scheme (arXiv 1702.00440, Sec. 2.1 and Sec. 2.4) that the paper lists among
 * Hermite schemes of higher order it cites (Nitadori & Makino 2008, "nm08").
 * Only the test suite and the benchmark's CPU legs call it; it shares no code
 * with the CUDA library.  It reuses the 4th-order oracle's block bookkeeping
 * (or_active, or_quantise_init, or_quantise) and energy (or_energy).
 *
 * Steps (the same step list as Sec. 2.4, with one more derivative):
 *   - force, jerk and snap of the active particles from the predicted
 *     positions, velocities and accelerations of all particles (softened Eq. 1
 *     and its first two time derivatives);
 *   - prediction of x, v and a by their Taylor series to the 5th, 4th and 3rd
 *     power of dt (crackle c = the third derivative of a);
 *   - correction by the time-symmetric sixth-order formulas of nm08 from the
 *     end-point values (a, jerk, snap) at both ends of the step;
 *   - crackle, pop and the fifth derivative at the end of the step from the
 *     quintic Hermite interpolant of those end-point values;
 *   - the generalised Aarseth step of nm08 for a sixth-order scheme,
 *       dt = eta ( (|a||snap| + |jerk|^2) / (|crackle||a^(5)| + |pop|^2) )^(1/6),
 *     quantised to the power-of-two block steps exactly as in the 4th-order
 *     oracle.
 *
 * The same driver also runs the fourth-order scheme in its time-symmetric form
 * (order 4): the corrector of Hut, Makino & McMillan (1995), which is the
 * fourth-order member of the nm08 family,
 *     v1 = v0 + h (a1 + a0) - (h^2 / 3) (j1 - j0)
 *     x1 = x0 + h (v1 + v0) - (h^2 / 3) (a1 - a0),      h = dt / 2,
 * with GraviDy's cubic predictor, force and jerk, Aarseth step and block
 * quantisation (Sec. 2.1, 2.4); snap and crackle stay zero.  Either order may
 * iterate the evaluation and correction n_iter times per block step (P(EC)^n,
 * Kokubo, Yoshinaga & Makino 1998): after every pass but the last, the
 * corrected position and velocity and the new acceleration of each active
 * particle replace its prediction, and the next pass evaluates the active
 * particles against those values.  With shared constant steps and converged
 * passes the map is time-reversible.
 *
 * Readings where the sources are silent (listed in the design notes):
 *   - the initial step is eta_init |a| / |jerk| (quantised), crackle = 0 at t = 0;
 *     the first step's predictions miss the crackle term, so eta_init must be
 *     small (the wrappers default to 1e-3; 1e-2 leaves an energy error of about
 *     4e-9 at N = 1024 that no later step removes);
 *   - the initial snap uses the exact initial accelerations of all particles.
 *
 * Build: together with hermite_oracle.c, gcc -O2 -fno-fast-math -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* from hermite_oracle.c */
void or_hermite_derivs(const double a0[3], const double j0[3], const double a1[3],
                       const double j1[3], double dt, double a2[3], double a3[3]);
double or_aarseth_dt(const double a1[3], const double j1[3], const double a2e[3],
                     const double a3e[3], double eta);
void or_force(int64_t n, const double *m, const double *x, const double *v, double eps2,
              int64_t nact, const int32_t *idx, double *acc, double *jrk);
void or_energy(int64_t n, const double *m, const double *x, const double *v, double eps2,
               double *K, double *U);
int64_t or_active(int64_t n, const int64_t *tnext, int32_t *idx, int64_t *t_next);
int64_t or_quantise_init(double dt, double dt_min, int64_t dtau_max);
int64_t or_quantise(double dt_new, int64_t dtau_old, int64_t tick_now, double dt_min,
                    int64_t dtau_max);

/* ------------------------------------------------------------------------ */
/* Force, jerk and snap of one particle.                                     */
/* ------------------------------------------------------------------------ */

/* With r = x_j - x_i, v = v_j - v_i, w = a_j - a_i, s^2 = |r|^2 + eps^2, the
 * pair term A0 = m r / s^3 and its time derivatives are
 *   alpha = (r.v) / s^2,
 *   A1    = m v / s^3 - 3 alpha A0,
 *   beta  = (|v|^2 + r.w) / s^2 + alpha^2,
 *   A2    = m w / s^3 - 6 alpha A1 - 3 beta A0,
 * obtained by differentiating A0 once and twice (d s / dt = (r.v) / s). */
static void force6_on(int64_t n, const double *m, const double *x, const double *v,
                      const double *a, double eps2, int64_t i, double f0[3], double f1[3],
                      double f2[3])
{
    double s0[3] = {0, 0, 0}, s1[3] = {0, 0, 0}, s2[3] = {0, 0, 0};
    for (int64_t j = 0; j < n; j++) {
        if (j == i)
            continue;
        double r[3], u[3], w[3];
        for (int c = 0; c < 3; c++) {
            r[c] = x[3 * j + c] - x[3 * i + c];
            u[c] = v[3 * j + c] - v[3 * i + c];
            w[c] = a[3 * j + c] - a[3 * i + c];
        }
        double ss = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + eps2;
        double s = sqrt(ss);
        double mi3 = m[j] / (ss * s); /* m / s^3 */
        double alpha = (r[0] * u[0] + r[1] * u[1] + r[2] * u[2]) / ss;
        double beta = (u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + r[0] * w[0] + r[1] * w[1] +
                       r[2] * w[2]) / ss + alpha * alpha;
        for (int c = 0; c < 3; c++) {
            double A0 = mi3 * r[c];
            double A1 = mi3 * u[c] - 3.0 * alpha * A0;
            double A2 = mi3 * w[c] - 6.0 * alpha * A1 - 3.0 * beta * A0;
            s0[c] += A0;
            s1[c] += A1;
            s2[c] += A2;
        }
    }
    for (int c = 0; c < 3; c++) {
        f0[c] = s0[c];
        f1[c] = s1[c];
        f2[c] = s2[c];
    }
}

/* Force, jerk and snap for idx[0..nact) against all n (outputs [nact][3]). */
void or6_force(int64_t n, const double *m, const double *x, const double *v, const double *a,
               double eps2, int64_t nact, const int32_t *idx, double *acc, double *jrk,
               double *snp)
{
    for (int64_t k = 0; k < nact; k++)
        force6_on(n, m, x, v, a, eps2, idx[k], acc + 3 * k, jrk + 3 * k, snp + 3 * k);
}

/* ------------------------------------------------------------------------ */
/* Predictor, corrector, interpolation, step.                                */
/* ------------------------------------------------------------------------ */

/* Taylor prediction over dt: x to dt^5, v to dt^4, a to dt^3. */
void or6_predict_one(const double x[3], const double v[3], const double a[3], const double j[3],
                     const double s[3], const double c[3], double dt, double xp[3], double vp[3],
                     double ap[3])
{
    double dt2 = dt * dt, dt3 = dt2 * dt, dt4 = dt3 * dt, dt5 = dt4 * dt;
    for (int k = 0; k < 3; k++) {
        xp[k] = x[k] + v[k] * dt + a[k] * dt2 / 2.0 + j[k] * dt3 / 6.0 + s[k] * dt4 / 24.0 +
                c[k] * dt5 / 120.0;
        vp[k] = v[k] + a[k] * dt + j[k] * dt2 / 2.0 + s[k] * dt3 / 6.0 + c[k] * dt4 / 24.0;
        ap[k] = a[k] + j[k] * dt + s[k] * dt2 / 2.0 + c[k] * dt3 / 6.0;
    }
}

/* Time-symmetric sixth-order corrector (nm08): with h = dt / 2,
 *   v1 = v0 + h (a1 + a0) - (2/5) h^2 (j1 - j0) + (1/15) h^3 (s1 + s0)
 *   x1 = x0 + h (v1 + v0) - (2/5) h^2 (a1 - a0) + (1/15) h^3 (j1 + j0).
 * The velocity formula is the integral of the quintic Hermite interpolant of
 * (a, jerk, snap) at both ends; the position formula is the same quadrature of
 * the velocity. */
void or6_correct_one(const double x0[3], const double v0[3], const double a0[3],
                     const double j0[3], const double s0[3], const double a1[3],
                     const double j1[3], const double s1[3], double dt, double x1[3],
                     double v1[3])
{
    double h = dt / 2.0, h2 = h * h, h3 = h2 * h;
    for (int k = 0; k < 3; k++) {
        v1[k] = v0[k] + h * (a1[k] + a0[k]) - 0.4 * h2 * (j1[k] - j0[k]) +
                h3 * (s1[k] + s0[k]) / 15.0;
        x1[k] = x0[k] + h * (v1[k] + v0[k]) - 0.4 * h2 * (a1[k] - a0[k]) +
                h3 * (j1[k] + j0[k]) / 15.0;
    }
}

/* Time-symmetric fourth-order corrector (Hut, Makino & McMillan 1995): with
 * h = dt / 2,
 *   v1 = v0 + h (a1 + a0) - (1/3) h^2 (j1 - j0)
 *   x1 = x0 + h (v1 + v0) - (1/3) h^2 (a1 - a0).
 * The velocity formula integrates the cubic Hermite interpolant of (a, jerk)
 * at both ends; the position formula is the same quadrature of the velocity. */
void or4s_correct_one(const double x0[3], const double v0[3], const double a0[3],
                      const double j0[3], const double a1[3], const double j1[3], double dt,
                      double x1[3], double v1[3])
{
    double h = dt / 2.0, h2 = h * h;
    for (int k = 0; k < 3; k++) {
        v1[k] = v0[k] + h * (a1[k] + a0[k]) - h2 * (j1[k] - j0[k]) / 3.0;
        x1[k] = x0[k] + h * (v1[k] + v0[k]) - h2 * (a1[k] - a0[k]) / 3.0;
    }
}

/* The quintic a(tau) = sum_k c_k tau^k on tau in [-h, h] (h = dt / 2, tau = 0 at
 * the middle of the step) that matches a, jerk, snap at both ends.  With
 * plus/minus halves P = (q1 + q0)/2, M = (q1 - q0)/2 of each quantity:
 *   even part: c4 = (Sp h - Jm) / (8 h^3),   c2 = (3 Jm - Sp h) / (4 h),
 *   odd part:  c5 = (Sm h^2 - 3 Jp h + 3 Am) / (8 h^5),
 *              c3 = ((Jp h - Am) / 2 - 2 c5 h^5) / h^3.
 * Returns crackle a'''(h) = 6 c3 + 24 c4 h + 60 c5 h^2, pop a''''(h) =
 * 24 c4 + 120 c5 h and the fifth derivative 120 c5, all at the END of the step. */
void or6_derivs(const double a0[3], const double j0[3], const double s0[3], const double a1[3],
                const double j1[3], const double s1[3], double dt, double crk[3], double pop[3],
                double a5[3])
{
    double h = dt / 2.0, h2 = h * h, h3 = h2 * h, h5 = h3 * h2;
    for (int k = 0; k < 3; k++) {
        double Am = (a1[k] - a0[k]) / 2.0;
        double Jp = (j1[k] + j0[k]) / 2.0, Jm = (j1[k] - j0[k]) / 2.0;
        double Sp = (s1[k] + s0[k]) / 2.0, Sm = (s1[k] - s0[k]) / 2.0;
        double c4 = (Sp * h - Jm) / (8.0 * h3);
        double c5 = (Sm * h2 - 3.0 * Jp * h + 3.0 * Am) / (8.0 * h5);
        double c3 = ((Jp * h - Am) / 2.0 - 2.0 * c5 * h5) / h3;
        crk[k] = 6.0 * c3 + 24.0 * c4 * h + 60.0 * c5 * h2;
        pop[k] = 24.0 * c4 + 120.0 * c5 * h;
        a5[k] = 120.0 * c5;
    }
}

static double norm3(const double a[3]) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/* Generalised Aarseth criterion for the sixth-order scheme (nm08). */
double or6_aarseth_dt(const double a[3], const double j[3], const double s[3], const double c[3],
                      const double p[3], const double q[3], double eta)
{
    double num = norm3(a) * norm3(s) + norm3(j) * norm3(j);
    double den = norm3(c) * norm3(q) + norm3(p) * norm3(p);
    return eta * pow(num / den, 1.0 / 6.0);
}

/* ------------------------------------------------------------------------ */
/* The integrator.                                                           */
/* ------------------------------------------------------------------------ */

typedef struct or6_sim {
    int64_t n;
    double eps2, eta, dt_min;
    int64_t dtau_max, fixed_dtau;
    int order, n_iter;                 /* 4 (time-symmetric) or 6; evaluations per step */
    double *m, *x, *v, *a, *j, *s, *c; /* state at each particle's own time */
    double *xp, *vp, *ap;              /* predicted state of all particles */
    double *a1, *j1, *s1;              /* new force, jerk, snap of the active set */
    int64_t *tau, *dtau, *tnext;
    int32_t *act;
    int64_t tick, nblock, nsteps;
    double interactions;
} or6_sim;

void or6_sim_free(or6_sim *q)
{
    if (!q)
        return;
    free(q->m); free(q->x); free(q->v); free(q->a); free(q->j); free(q->s); free(q->c);
    free(q->xp); free(q->vp); free(q->ap); free(q->a1); free(q->j1); free(q->s1);
    free(q->tau); free(q->dtau); free(q->tnext); free(q->act);
    free(q);
}

/* Initial force, jerk (4th-order oracle) and, for order 6, snap (from the
 * exact initial accelerations); crackle 0; first steps eta_init |a| / |jerk|
 * (or fixed_dtau). */
or6_sim *or6_sim_new(int64_t n, const double *m, const double *x, const double *v, double eps,
                     double eta, double eta_init, double dt_min, double dt_max, int64_t fixed_dtau,
                     int order, int n_iter)
{
    if (n < 1 || !(eps >= 0) || !(eta > 0) || !(eta_init > 0) || !(dt_min > 0) ||
        !(dt_max >= dt_min) || (order != 4 && order != 6) || n_iter < 1)
        return NULL;
    or6_sim *q = (or6_sim *)calloc(1, sizeof(or6_sim));
    if (!q)
        return NULL;
    q->n = n;
    q->eps2 = eps * eps;
    q->eta = eta;
    q->dt_min = dt_min;
    q->dtau_max = (int64_t)(dt_max / dt_min);
    q->fixed_dtau = fixed_dtau;
    q->order = order;
    q->n_iter = n_iter;
    size_t v3 = (size_t)n * 3 * sizeof(double);
    q->m = malloc((size_t)n * sizeof(double));
    q->x = malloc(v3); q->v = malloc(v3); q->a = malloc(v3); q->j = malloc(v3);
    q->s = calloc((size_t)n * 3, sizeof(double)); q->c = calloc((size_t)n * 3, sizeof(double));
    q->xp = malloc(v3); q->vp = malloc(v3); q->ap = malloc(v3);
    q->a1 = malloc(v3); q->j1 = malloc(v3); q->s1 = malloc(v3);
    q->tau = calloc((size_t)n, sizeof(int64_t));
    q->dtau = malloc((size_t)n * sizeof(int64_t));
    q->tnext = malloc((size_t)n * sizeof(int64_t));
    q->act = malloc((size_t)n * sizeof(int32_t));
    if (!q->m || !q->x || !q->v || !q->a || !q->j || !q->s || !q->c || !q->xp || !q->vp ||
        !q->ap || !q->a1 || !q->j1 || !q->s1 || !q->tau || !q->dtau || !q->tnext || !q->act) {
        or6_sim_free(q);
        return NULL;
    }
    memcpy(q->m, m, (size_t)n * sizeof(double));
    memcpy(q->x, x, v3);
    memcpy(q->v, v, v3);
    for (int64_t i = 0; i < n; i++)
        q->act[i] = (int32_t)i;
    or_force(n, q->m, q->x, q->v, q->eps2, n, q->act, q->a, q->j);
    q->interactions += (double)n * (double)n;
    if (order == 6) {
        or6_force(n, q->m, q->x, q->v, q->a, q->eps2, n, q->act, q->a1, q->j1, q->s);
        q->interactions += (double)n * (double)n;
    }
    for (int64_t i = 0; i < n; i++) {
        if (fixed_dtau > 0) {
            q->dtau[i] = fixed_dtau;
        } else {
            double dt0 = eta_init * norm3(q->a + 3 * i) / norm3(q->j + 3 * i);
            q->dtau[i] = or_quantise_init(dt0, dt_min, q->dtau_max);
        }
        q->tnext[i] = q->dtau[i];
    }
    return q;
}

/* New force, jerk and (order 6) snap of the active set into a1, j1, s1. */
static void evaluate6(or6_sim *q, int64_t nact, const int32_t *idx)
{
    if (q->order == 6) {
        or6_force(q->n, q->m, q->xp, q->vp, q->ap, q->eps2, nact, idx, q->a1, q->j1, q->s1);
    } else {
        or_force(q->n, q->m, q->xp, q->vp, q->eps2, nact, idx, q->a1, q->j1);
        memset(q->s1, 0, (size_t)nact * 3 * sizeof(double));
    }
    q->interactions += (double)nact * (double)q->n;
}

/* Corrected x1, v1 of active slot k (particle i) from its state at its own time
 * and the slot's new force, jerk, snap. */
static void correct_slot6(const or6_sim *q, int64_t k, int64_t i, double dt, double x1[3],
                          double v1[3])
{
    if (q->order == 6)
        or6_correct_one(q->x + 3 * i, q->v + 3 * i, q->a + 3 * i, q->j + 3 * i, q->s + 3 * i,
                        q->a1 + 3 * k, q->j1 + 3 * k, q->s1 + 3 * k, dt, x1, v1);
    else
        or4s_correct_one(q->x + 3 * i, q->v + 3 * i, q->a + 3 * i, q->j + 3 * i, q->a1 + 3 * k,
                         q->j1 + 3 * k, dt, x1, v1);
}

static void block_step6(or6_sim *q, int64_t tick_next, int64_t nact, const int32_t *idx)
{
    int64_t n = q->n;
    for (int64_t i = 0; i < n; i++) {
        double dt = (double)(tick_next - q->tau[i]) * q->dt_min;
        or6_predict_one(q->x + 3 * i, q->v + 3 * i, q->a + 3 * i, q->j + 3 * i, q->s + 3 * i,
                        q->c + 3 * i, dt, q->xp + 3 * i, q->vp + 3 * i, q->ap + 3 * i);
    }
    /* P(EC)^n: every pass but the last puts the active particles' corrected
     * values in place of their predictions before the next evaluation */
    for (int pass = 1; pass < q->n_iter; pass++) {
        evaluate6(q, nact, idx);
        for (int64_t k = 0; k < nact; k++) {
            int64_t i = idx[k];
            double dt = (double)(tick_next - q->tau[i]) * q->dt_min;
            correct_slot6(q, k, i, dt, q->xp + 3 * i, q->vp + 3 * i);
            for (int c = 0; c < 3; c++)
                q->ap[3 * i + c] = q->a1[3 * k + c];
        }
    }
    evaluate6(q, nact, idx);
    for (int64_t k = 0; k < nact; k++) {
        int64_t i = idx[k];
        double dt = (double)(tick_next - q->tau[i]) * q->dt_min;
        double crk[3] = {0, 0, 0}, pop[3], a5[3], a2[3], a3[3], a2e[3];
        double *a1 = q->a1 + 3 * k, *j1 = q->j1 + 3 * k, *s1 = q->s1 + 3 * k;
        double x1[3], v1[3];
        correct_slot6(q, k, i, dt, x1, v1);
        if (q->order == 6)
            or6_derivs(q->a + 3 * i, q->j + 3 * i, q->s + 3 * i, a1, j1, s1, dt, crk, pop, a5);
        else
            or_hermite_derivs(q->a + 3 * i, q->j + 3 * i, a1, j1, dt, a2, a3);
        int64_t dtau;
        if (q->fixed_dtau > 0) {
            dtau = q->fixed_dtau;
        } else {
            double dtn;
            if (q->order == 6) {
                dtn = or6_aarseth_dt(a1, j1, s1, crk, pop, a5, q->eta);
            } else {
                for (int c = 0; c < 3; c++)
                    a2e[c] = a2[c] + dt * a3[c];
                dtn = or_aarseth_dt(a1, j1, a2e, a3, q->eta);
            }
            dtau = or_quantise(dtn, q->dtau[i], tick_next, q->dt_min, q->dtau_max);
        }
        for (int c = 0; c < 3; c++) {
            q->x[3 * i + c] = x1[c];
            q->v[3 * i + c] = v1[c];
            q->a[3 * i + c] = a1[c];
            q->j[3 * i + c] = j1[c];
            q->s[3 * i + c] = s1[c];
            q->c[3 * i + c] = crk[c];
        }
        q->tau[i] = tick_next;
        q->dtau[i] = dtau;
        q->tnext[i] = tick_next + dtau;
    }
    q->tick = tick_next;
    q->nblock += 1;
    q->nsteps += nact;
}

int64_t or6_sim_step(or6_sim *q, int64_t *tick_out, int32_t *idx_out)
{
    int64_t tick_next;
    int64_t nact = or_active(q->n, q->tnext, q->act, &tick_next);
    block_step6(q, tick_next, nact, q->act);
    if (tick_out)
        *tick_out = tick_next;
    if (idx_out)
        memcpy(idx_out, q->act, (size_t)nact * sizeof(int32_t));
    return nact;
}

void or6_sim_replay(or6_sim *q, int64_t tick_next, int64_t nact, const int32_t *idx)
{
    block_step6(q, tick_next, nact, idx);
}

int64_t or6_sim_evolve(or6_sim *q, int64_t tick_end)
{
    int64_t steps = 0;
    for (;;) {
        int64_t tmin = q->tnext[0];
        for (int64_t i = 1; i < q->n; i++)
            if (q->tnext[i] < tmin)
                tmin = q->tnext[i];
        if (tmin > tick_end)
            break;
        or6_sim_step(q, NULL, NULL);
        steps++;
    }
    return steps;
}

void or6_sim_energy(or6_sim *q, double *K, double *U)
{
    /* every particle predicted to the time of the last block step */
    int64_t n = q->n;
    for (int64_t i = 0; i < n; i++) {
        double dt = (double)(q->tick - q->tau[i]) * q->dt_min;
        or6_predict_one(q->x + 3 * i, q->v + 3 * i, q->a + 3 * i, q->j + 3 * i, q->s + 3 * i,
                        q->c + 3 * i, dt, q->xp + 3 * i, q->vp + 3 * i, q->ap + 3 * i);
    }
    or_energy(n, q->m, q->xp, q->vp, q->eps2, K, U);
}

void or6_sim_get(const or6_sim *q, double *x, double *v, double *a, double *j, double *s,
                 double *c, int64_t *tau, int64_t *dtau)
{
    size_t v3 = (size_t)q->n * 3 * sizeof(double);
    if (x) memcpy(x, q->x, v3);
    if (v) memcpy(v, q->v, v3);
    if (a) memcpy(a, q->a, v3);
    if (j) memcpy(j, q->j, v3);
    if (s) memcpy(s, q->s, v3);
    if (c) memcpy(c, q->c, v3);
    if (tau) memcpy(tau, q->tau, (size_t)q->n * sizeof(int64_t));
    if (dtau) memcpy(dtau, q->dtau, (size_t)q->n * sizeof(int64_t));
}

void or6_sim_stats(const or6_sim *q, int64_t *tick, int64_t *nblock, int64_t *nsteps,
                   double *interactions)
{
    *tick = q->tick;
    *nblock = q->nblock;
    *nsteps = q->nsteps;
    *interactions = q->interactions;
}
