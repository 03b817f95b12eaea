/*
 * hermite_oracle.c -- TEST INFRASTRUCTURE, not part of the product path.
 *
 * A plain, slow, single-threaded FP64 reference of the 4th-order Hermite
 * block-time-step integrator with Plummer softening described in GraviDy
 * (Maureira-Fredes & Amaro-Seoane, arXiv 1702.00440).  Only the test suite,
 * the smoke check and the CPU baseline leg of the benchmark call it.  It shares
 * no code, header or constant with the CUDA library.
 *
 * Sources of each step (section / equation of the paper, plus the published
 * Hermite scheme the paper defers to, Makino & Aarseth 1992, "ma92"):
 *   - softened acceleration ........ Sec. 2.4, softened form of Eq. 1
 *   - jerk (time derivative of it) . Sec. 2.4 step 3 ("the so-called jerk");
 *                                    derivative of the softened force
 *   - total energy ................. Sec. 2.1 Eq. 2 (with the same softening
 *                                    as the force, see the readings below)
 *   - active-particle search ....... Sec. 2.4 step 5
 *   - save old forces .............. Sec. 2.4 step 6
 *   - prediction of all N .......... Sec. 2.4 step 7a (Taylor series, ma92)
 *   - force of the active set ...... Sec. 2.4 step 7c, Sec. 2.5
 *   - correction ................... Sec. 2.4 step 7d (Hermite interpolation,
 *                                    ma92 Eq. 2 with the sign of the second
 *                                    term of the end-point jerk fixed, as the
 *                                    paper's footnote in Sec. 2.4 says)
 *   - time step criterion (eta) .... Sec. 3.2 (Aarseth criterion, ma92)
 *   - block time steps ............. Sec. 2.4 "Block time steps" (Press 1986)
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - G = 1; r_ij = x_j - x_i so the sum carries a plus sign.
 *   - the energy's potential term uses the softened distance sqrt(r^2+eps^2).
 *   - initial step dt = eta |a| / |jerk|, then quantised.
 *   - block quantisation: steps are powers of two times dt_min, clamped to
 *     [dt_min, dt_max]; a step may shrink to any smaller power of two; it may
 *     grow by a factor 2 only when the current time is a multiple of twice the
 *     old step; a step below dt_min is clamped (no error).
 *   - a non-finite step estimate (0/0 for an isolated particle) means "no
 *     constraint" and takes dt_max (initial step) or the growth branch.
 *   - active particles are listed in ascending index order.
 *   - the self term j = i is skipped.
 *
 * Layout: positions, velocities, accelerations and jerks are AoS [n][3]
 * doubles; times are integer ticks of dt_min (dt_min a power of two), so all
 * block-time arithmetic is exact.
 *
 * Build: gcc -O2 -fno-fast-math -ffp-contract=off -fPIC -shared (no FMA
 * contraction, IEEE round-to-nearest-even throughout).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Pairwise force and jerk (softened Eq. 1 and its time derivative).         */
/* ------------------------------------------------------------------------ */

/* Acceleration and jerk on particle i from every j != i:
 *   a_i    = sum_j m_j r / s^3
 *   jerk_i = sum_j m_j [ v / s^3 - 3 (r.v) r / s^5 ]
 * with r = x_j - x_i, v = v_j - v_i, s^2 = |r|^2 + eps^2. */
static void force_on(int64_t n, const double *m, const double *x, const double *v,
                     double eps2, int64_t i, double acc[3], double jrk[3])
{
    double ax = 0, ay = 0, az = 0, jx = 0, jy = 0, jz = 0;
    for (int64_t j = 0; j < n; j++) {
        if (j == i)
            continue;
        double rx = x[3 * j + 0] - x[3 * i + 0];
        double ry = x[3 * j + 1] - x[3 * i + 1];
        double rz = x[3 * j + 2] - x[3 * i + 2];
        double vx = v[3 * j + 0] - v[3 * i + 0];
        double vy = v[3 * j + 1] - v[3 * i + 1];
        double vz = v[3 * j + 2] - v[3 * i + 2];
        double s2 = rx * rx + ry * ry + rz * rz + eps2;
        double s = sqrt(s2);
        double s3 = s2 * s;
        double s5 = s3 * s2;
        double rv = rx * vx + ry * vy + rz * vz;
        ax += m[j] * rx / s3;
        ay += m[j] * ry / s3;
        az += m[j] * rz / s3;
        jx += m[j] * (vx / s3 - 3.0 * rv * rx / s5);
        jy += m[j] * (vy / s3 - 3.0 * rv * ry / s5);
        jz += m[j] * (vz / s3 - 3.0 * rv * rz / s5);
    }
    acc[0] = ax; acc[1] = ay; acc[2] = az;
    jrk[0] = jx; jrk[1] = jy; jrk[2] = jz;
}

/* Force and jerk for the listed particles idx[0..nact) against all n.
 * Outputs are [nact][3], in the order of idx. */
void or_force(int64_t n, const double *m, const double *x, const double *v, double eps2,
              int64_t nact, const int32_t *idx, double *acc, double *jrk)
{
    for (int64_t k = 0; k < nact; k++)
        force_on(n, m, x, v, eps2, idx[k], acc + 3 * k, jrk + 3 * k);
}

/* Sums of the magnitudes of the individual terms, used to scale round-off
 * tolerances:  an[k] = sum_j m_j |r|/s^3,
 *              jn[k] = sum_j m_j ( |v|/s^3 + 3 |r.v| |r| / s^5 ). */
void or_force_absnorm(int64_t n, const double *m, const double *x, const double *v,
                      double eps2, int64_t nact, const int32_t *idx, double *an,
                      double *jn)
{
    for (int64_t k = 0; k < nact; k++) {
        int64_t i = idx[k];
        double sa = 0, sj = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i)
                continue;
            double rx = x[3 * j + 0] - x[3 * i + 0];
            double ry = x[3 * j + 1] - x[3 * i + 1];
            double rz = x[3 * j + 2] - x[3 * i + 2];
            double vx = v[3 * j + 0] - v[3 * i + 0];
            double vy = v[3 * j + 1] - v[3 * i + 1];
            double vz = v[3 * j + 2] - v[3 * i + 2];
            double r = sqrt(rx * rx + ry * ry + rz * rz);
            double vv = sqrt(vx * vx + vy * vy + vz * vz);
            double s2 = r * r + eps2;
            double s = sqrt(s2);
            double s3 = s2 * s;
            double s5 = s3 * s2;
            double rv = fabs(rx * vx + ry * vy + rz * vz);
            sa += m[j] * r / s3;
            sj += m[j] * (vv / s3 + 3.0 * rv * r / s5);
        }
        an[k] = sa;
        jn[k] = sj;
    }
}

/* ------------------------------------------------------------------------ */
/* Energy (Eq. 2, softened potential).                                       */
/* ------------------------------------------------------------------------ */

/* K = 1/2 sum_i m_i |v_i|^2,  U = - sum_{i<j} m_i m_j / sqrt(|x_i-x_j|^2 + eps^2) */
void or_energy(int64_t n, const double *m, const double *x, const double *v, double eps2,
               double *K, double *U)
{
    double k = 0, u = 0;
    for (int64_t i = 0; i < n; i++)
        k += 0.5 * m[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] +
                           v[3 * i + 2] * v[3 * i + 2]);
    for (int64_t i = 0; i < n; i++) {
        for (int64_t j = i + 1; j < n; j++) {
            double rx = x[3 * j + 0] - x[3 * i + 0];
            double ry = x[3 * j + 1] - x[3 * i + 1];
            double rz = x[3 * j + 2] - x[3 * i + 2];
            u -= m[i] * m[j] / sqrt(rx * rx + ry * ry + rz * rz + eps2);
        }
    }
    *K = k;
    *U = u;
}

/* ------------------------------------------------------------------------ */
/* Active-particle search (Sec. 2.4 step 5).                                 */
/* ------------------------------------------------------------------------ */

/* t_next = min_i tnext[i]; writes the ascending indices i with
 * tnext[i] == t_next into idx and returns their count.  n >= 1. */
int64_t or_active(int64_t n, const int64_t *tnext, int32_t *idx, int64_t *t_next)
{
    int64_t tmin = tnext[0];
    for (int64_t i = 1; i < n; i++)
        if (tnext[i] < tmin)
            tmin = tnext[i];
    int64_t c = 0;
    for (int64_t i = 0; i < n; i++)
        if (tnext[i] == tmin)
            idx[c++] = (int32_t)i;
    *t_next = tmin;
    return c;
}

/* ------------------------------------------------------------------------ */
/* Hermite predictor / interpolation / corrector (ma92, Sec. 2.4 step 7).    */
/* ------------------------------------------------------------------------ */

/* Taylor prediction over dt of one particle (3 components). */
void or_predict_one(const double x[3], const double v[3], const double a[3],
                    const double j[3], double dt, double xp[3], double vp[3])
{
    double dt2 = dt * dt, dt3 = dt2 * dt;
    for (int c = 0; c < 3; c++) {
        xp[c] = x[c] + v[c] * dt + a[c] * dt2 / 2.0 + j[c] * dt3 / 6.0;
        vp[c] = v[c] + a[c] * dt + j[c] * dt2 / 2.0;
    }
}

/* Prediction of n particles, particle i over dt[i] (AoS [n][3] arrays). */
void or_predict_all(int64_t n, const double *x, const double *v, const double *a, const double *j,
                    const double *dt, double *xp, double *vp)
{
    for (int64_t i = 0; i < n; i++)
        or_predict_one(x + 3 * i, v + 3 * i, a + 3 * i, j + 3 * i, dt[i], xp + 3 * i, vp + 3 * i);
}

/* Second and third derivative of the acceleration at the START of an
 * interval of length dt from the end-point values (a0, j0) and (a1, j1): the
 * cubic a(t) = a0 + j0 t + a2 t^2/2 + a3 t^3/6 that matches a1 and j1 at
 * t = dt has
 *   a2 = ( -6 (a0 - a1) - dt (4 j0 + 2 j1) ) / dt^2
 *   a3 = ( 12 (a0 - a1) + 6 dt (j0 + j1) ) / dt^3 . */
void or_hermite_derivs(const double a0[3], const double j0[3], const double a1[3],
                       const double j1[3], double dt, double a2[3], double a3[3])
{
    double dt2 = dt * dt, dt3 = dt2 * dt;
    for (int c = 0; c < 3; c++) {
        double da = a0[c] - a1[c];
        a2[c] = (-6.0 * da - dt * (4.0 * j0[c] + 2.0 * j1[c])) / dt2;
        a3[c] = (12.0 * da + 6.0 * dt * (j0[c] + j1[c])) / dt3;
    }
}

/* Corrected position and velocity: the predicted values plus the 4th and
 * 5th order terms of the interpolating polynomial. */
void or_correct_one(const double xp[3], const double vp[3], const double a2[3],
                    const double a3[3], double dt, double x1[3], double v1[3])
{
    double dt2 = dt * dt, dt3 = dt2 * dt, dt4 = dt3 * dt, dt5 = dt4 * dt;
    for (int c = 0; c < 3; c++) {
        x1[c] = xp[c] + a2[c] * dt4 / 24.0 + a3[c] * dt5 / 120.0;
        v1[c] = vp[c] + a2[c] * dt3 / 6.0 + a3[c] * dt4 / 24.0;
    }
}

static double norm3(const double a[3]) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/* Aarseth's criterion at the END of the step, from the end-point acceleration
 * a1, jerk j1 and the end-point second and third derivatives a2e, a3e:
 *   dt = sqrt( eta (|a1||a2e| + |j1|^2) / (|j1||a3e| + |a2e|^2) ). */
double or_aarseth_dt(const double a1[3], const double j1[3], const double a2e[3],
                     const double a3e[3], double eta)
{
    double na = norm3(a1), nj = norm3(j1), n2 = norm3(a2e), n3 = norm3(a3e);
    return sqrt(eta * (na * n2 + nj * nj) / (nj * n3 + n2 * n2));
}

/* Largest power of two <= x, for 1 <= x (exact, via the binary exponent). */
static int64_t pow2_floor(double x)
{
    int e;
    frexp(x, &e); /* x = f 2^e, 0.5 <= f < 1 */
    return (int64_t)1 << (e - 1);
}

/* Initial block step: power of two times dt_min at most dt, clamped to
 * [1, dtau_max] ticks; a NaN or infinite dt takes dtau_max. */
int64_t or_quantise_init(double dt, double dt_min, int64_t dtau_max)
{
    if (!(dt < INFINITY))
        return dtau_max;
    double q = dt / dt_min;
    if (q < 1.0)
        return 1;
    if (q >= (double)dtau_max)
        return dtau_max;
    return pow2_floor(q);
}

/* Block step after a correction at tick `tick_now`: shrink to the largest
 * power of two not above dt_new; grow by 2 only if dt_new >= 2 dt_old, the
 * doubled step stays <= dtau_max and tick_now is a multiple of 2 dtau_old;
 * otherwise keep the old step.  A NaN dt_new is treated as +infinity. */
int64_t or_quantise(double dt_new, int64_t dtau_old, int64_t tick_now, double dt_min,
                    int64_t dtau_max)
{
    double dt_old = (double)dtau_old * dt_min;
    if (dt_new < dt_old) {
        double q = dt_new / dt_min;
        if (q < 1.0)
            return 1;
        return pow2_floor(q);
    }
    if (!(dt_new == dt_new) || dt_new >= 2.0 * dt_old) {
        if (2 * dtau_old <= dtau_max && tick_now % (2 * dtau_old) == 0)
            return 2 * dtau_old;
    }
    return dtau_old;
}

/* ------------------------------------------------------------------------ */
/* Post-Newtonian terms of one pair (Sec. 5: corrections for a binary with  */
/* eps = 0).  The paper prints no formulas; these are the relative          */
/* accelerations of the two-body problem in harmonic coordinates at 1PN,   */
/* 2PN and 2.5PN (radiation reaction) as published by Kidder (1995, Phys.   */
/* Rev. D 52, 821, Eq. 2.2) and Blanchet (2014, Living Rev. Relativ. 17, 2, */
/* A and B of its Eq. 219 at those orders).  With r = x_p - x_q,            */
/* v = v_p - v_q, M = m_p + m_q, eta = m_p m_q / M^2, n = r / |r|,          */
/* rdot = n.v and c the speed of light in code units (G = 1):               */
/*   1PN:   M / (c^2 r^2) { [(4 + 2 eta) M/r - (1 + 3 eta) v^2              */
/*                           + 3/2 eta rdot^2] n + (4 - 2 eta) rdot v }     */
/*   2PN:   M / (c^4 r^2) { [ -15/8 eta (1 - 3 eta) rdot^4                  */
/*                            + 3/2 eta (3 - 4 eta) v^2 rdot^2              */
/*                            - eta (3 - 4 eta) v^4                         */
/*                            + 1/2 eta (13 - 4 eta) (M/r) v^2              */
/*                            + (2 + 25 eta + 2 eta^2) (M/r) rdot^2         */
/*                            - 3/4 (12 + 29 eta) (M/r)^2 ] n               */
/*              + 1/2 rdot [ eta (15 + 4 eta) v^2                           */
/*                           - (4 + 41 eta + 8 eta^2) M/r                   */
/*                           - 3 eta (3 + 2 eta) rdot^2 ] v }               */
/*   2.5PN: 8/5 eta M^2 / (c^5 r^3) { rdot [18 v^2 + 2/3 M/r - 25 rdot^2] n */
/*                                    - [6 v^2 - 2 M/r - 15 rdot^2] v }     */
/* terms: bit 1 selects 1PN, bit 2 2PN, bit 4 2.5PN.  The                   */
/* pair's particles get m_q/M and -m_p/M of the relative term, which keeps  */
/* the pair's centre of mass at rest at this order.                         */
/* ------------------------------------------------------------------------ */

void or_pn_accel(double mp, double mq, const double r[3], const double v[3], double c, int terms,
                 double a[3])
{
    double M = mp + mq, eta = mp * mq / (M * M);
    double rr = norm3(r), n[3], v2 = 0.0, rd = 0.0;
    for (int k = 0; k < 3; k++) {
        n[k] = r[k] / rr;
        v2 += v[k] * v[k];
    }
    for (int k = 0; k < 3; k++)
        rd += n[k] * v[k];
    for (int k = 0; k < 3; k++)
        a[k] = 0.0;
    if (terms & 1) {
        double K = M / (c * c * rr * rr);
        double alpha = (4.0 + 2.0 * eta) * M / rr - (1.0 + 3.0 * eta) * v2 + 1.5 * eta * rd * rd;
        double beta = (4.0 - 2.0 * eta) * rd;
        for (int k = 0; k < 3; k++)
            a[k] += K * (alpha * n[k] + beta * v[k]);
    }
    if (terms & 2) {
        double K = M / (pow(c, 4.0) * rr * rr), Mr = M / rr, rd2 = rd * rd;
        double alpha = -15.0 / 8.0 * eta * (1.0 - 3.0 * eta) * rd2 * rd2
                       + 1.5 * eta * (3.0 - 4.0 * eta) * v2 * rd2
                       - eta * (3.0 - 4.0 * eta) * v2 * v2
                       + 0.5 * eta * (13.0 - 4.0 * eta) * Mr * v2
                       + (2.0 + 25.0 * eta + 2.0 * eta * eta) * Mr * rd2
                       - 0.75 * (12.0 + 29.0 * eta) * Mr * Mr;
        double beta = 0.5 * rd * (eta * (15.0 + 4.0 * eta) * v2 - (4.0 + 41.0 * eta + 8.0 * eta * eta) * Mr
                                  - 3.0 * eta * (3.0 + 2.0 * eta) * rd2);
        for (int k = 0; k < 3; k++)
            a[k] += K * (alpha * n[k] + beta * v[k]);
    }
    if (terms & 4) {
        double K = 1.6 * eta * M * M / (pow(c, 5.0) * rr * rr * rr);
        double alpha = rd * (18.0 * v2 + 2.0 / 3.0 * M / rr - 25.0 * rd * rd);
        double beta = -(6.0 * v2 - 2.0 * M / rr - 15.0 * rd * rd);
        for (int k = 0; k < 3; k++)
            a[k] += K * (alpha * n[k] + beta * v[k]);
    }
}

/* The time derivative of or_pn_accel along the relative motion, with
 * dr/dt = v and dv/dt = arel, by the chain rule written out term by term:
 * d|r|/dt = rdot, dn/dt = (v - rdot n)/|r|, d(v^2)/dt = 2 v.arel,
 * d(rdot)/dt = (v^2 - rdot^2)/|r| + n.arel. */
void or_pn_jerk(double mp, double mq, const double r[3], const double v[3], const double arel[3],
                double c, int terms, double j[3])
{
    double M = mp + mq, eta = mp * mq / (M * M);
    double rr = norm3(r), n[3], v2 = 0.0, rd = 0.0, va = 0.0, na = 0.0, dn[3];
    for (int k = 0; k < 3; k++) {
        n[k] = r[k] / rr;
        v2 += v[k] * v[k];
        va += v[k] * arel[k];
    }
    for (int k = 0; k < 3; k++) {
        rd += n[k] * v[k];
        na += n[k] * arel[k];
    }
    for (int k = 0; k < 3; k++)
        dn[k] = (v[k] - rd * n[k]) / rr;
    double drd = (v2 - rd * rd) / rr + na, dv2 = 2.0 * va;
    for (int k = 0; k < 3; k++)
        j[k] = 0.0;
    if (terms & 1) {
        double K = M / (c * c);
        double alpha = (4.0 + 2.0 * eta) * M / rr - (1.0 + 3.0 * eta) * v2 + 1.5 * eta * rd * rd;
        double beta = (4.0 - 2.0 * eta) * rd;
        double dalpha = -(4.0 + 2.0 * eta) * M * rd / (rr * rr) - (1.0 + 3.0 * eta) * dv2 + 3.0 * eta * rd * drd;
        double dbeta = (4.0 - 2.0 * eta) * drd;
        double i2 = 1.0 / (rr * rr), di2 = -2.0 * rd / (rr * rr * rr);
        for (int k = 0; k < 3; k++)
            j[k] += K * (di2 * (alpha * n[k] + beta * v[k]) +
                         i2 * (dalpha * n[k] + alpha * dn[k] + dbeta * v[k] + beta * arel[k]));
    }
    if (terms & 2) {
        double K = M / pow(c, 4.0);
        double Mr = M / rr, dMr = -M * rd / (rr * rr), rd2 = rd * rd, drd2 = 2.0 * rd * drd;
        double e1 = -15.0 / 8.0 * eta * (1.0 - 3.0 * eta), e2 = 1.5 * eta * (3.0 - 4.0 * eta);
        double e3 = -eta * (3.0 - 4.0 * eta), e4 = 0.5 * eta * (13.0 - 4.0 * eta);
        double e5 = 2.0 + 25.0 * eta + 2.0 * eta * eta, e6 = -0.75 * (12.0 + 29.0 * eta);
        double alpha = e1 * rd2 * rd2 + e2 * v2 * rd2 + e3 * v2 * v2 + e4 * Mr * v2 + e5 * Mr * rd2 + e6 * Mr * Mr;
        double dalpha = e1 * 2.0 * rd2 * drd2 + e2 * (dv2 * rd2 + v2 * drd2) + e3 * 2.0 * v2 * dv2
                        + e4 * (dMr * v2 + Mr * dv2) + e5 * (dMr * rd2 + Mr * drd2) + e6 * 2.0 * Mr * dMr;
        double f1 = eta * (15.0 + 4.0 * eta), f2 = -(4.0 + 41.0 * eta + 8.0 * eta * eta);
        double f3 = -3.0 * eta * (3.0 + 2.0 * eta);
        double Q = f1 * v2 + f2 * Mr + f3 * rd2, dQ = f1 * dv2 + f2 * dMr + f3 * drd2;
        double beta = 0.5 * rd * Q, dbeta = 0.5 * (drd * Q + rd * dQ);
        double i2 = 1.0 / (rr * rr), di2 = -2.0 * rd / (rr * rr * rr);
        for (int k = 0; k < 3; k++)
            j[k] += K * (di2 * (alpha * n[k] + beta * v[k]) +
                         i2 * (dalpha * n[k] + alpha * dn[k] + dbeta * v[k] + beta * arel[k]));
    }
    if (terms & 4) {
        double K = 1.6 * eta * M * M / pow(c, 5.0);
        double P = 18.0 * v2 + 2.0 / 3.0 * M / rr - 25.0 * rd * rd;
        double dP = 18.0 * dv2 - 2.0 / 3.0 * M * rd / (rr * rr) - 50.0 * rd * drd;
        double alpha = rd * P, dalpha = drd * P + rd * dP;
        double beta = -(6.0 * v2 - 2.0 * M / rr - 15.0 * rd * rd);
        double dbeta = -(6.0 * dv2 + 2.0 * M * rd / (rr * rr) - 30.0 * rd * drd);
        double i3 = 1.0 / (rr * rr * rr), di3 = -3.0 * rd / (rr * rr * rr * rr);
        for (int k = 0; k < 3; k++)
            j[k] += K * (di3 * (alpha * n[k] + beta * v[k]) +
                         i3 * (dalpha * n[k] + alpha * dn[k] + dbeta * v[k] + beta * arel[k]));
    }
}

/* ------------------------------------------------------------------------ */
/* The integrator (Sec. 2.4 steps 1-7).                                      */
/* ------------------------------------------------------------------------ */

typedef struct or_sim {
    int64_t n;
    double eps2, eta, dt_min;
    int64_t dtau_max, fixed_dtau;
    double *m, *x, *v, *a, *j;   /* state at each particle's own time */
    double *xp, *vp;             /* predicted state of all particles */
    double *a1, *j1;             /* new forces of the active set */
    int64_t *tau, *dtau, *tnext; /* particle time, step, next time (ticks) */
    int32_t *act;                /* active list */
    int64_t tick;                /* time of the last block step */
    int64_t nblock, nsteps;      /* block steps, particle steps */
    double interactions;         /* sum of nact * n over force evaluations */
    int32_t pn_p, pn_q;          /* post-Newtonian pair (pn_terms != 0) */
    double pn_c;
    int pn_terms;
} or_sim;

void or_sim_free(or_sim *s)
{
    if (!s)
        return;
    free(s->m); free(s->x); free(s->v); free(s->a); free(s->j);
    free(s->xp); free(s->vp); free(s->a1); free(s->j1);
    free(s->tau); free(s->dtau); free(s->tnext); free(s->act);
    free(s);
}

/* Steps 1-3: allocate, store the initial state, compute the initial force and
 * jerk of every particle (O(N^2)) and its first block step.
 * fixed_dtau > 0 switches to shared fixed steps of that many ticks (used by the
 * convergence-order tests); 0 selects the Aarseth criterion.  Returns NULL on
 * a bad argument or allocation failure. */
or_sim *or_sim_new(int64_t n, const double *m, const double *x, const double *v,
                   double eps, double eta, double dt_min, double dt_max, int64_t fixed_dtau)
{
    if (n < 1 || !(eps >= 0) || !(eta > 0) || !(dt_min > 0) || !(dt_max >= dt_min))
        return NULL;
    or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
    if (!s)
        return NULL;
    s->n = n;
    s->eps2 = eps * eps;
    s->eta = eta;
    s->dt_min = dt_min;
    s->dtau_max = (int64_t)(dt_max / dt_min);
    s->fixed_dtau = fixed_dtau;
    size_t v3 = (size_t)n * 3 * sizeof(double);
    s->m = malloc((size_t)n * sizeof(double));
    s->x = malloc(v3); s->v = malloc(v3); s->a = malloc(v3); s->j = malloc(v3);
    s->xp = malloc(v3); s->vp = malloc(v3); s->a1 = malloc(v3); s->j1 = malloc(v3);
    s->tau = calloc((size_t)n, sizeof(int64_t));
    s->dtau = malloc((size_t)n * sizeof(int64_t));
    s->tnext = malloc((size_t)n * sizeof(int64_t));
    s->act = malloc((size_t)n * sizeof(int32_t));
    if (!s->m || !s->x || !s->v || !s->a || !s->j || !s->xp || !s->vp || !s->a1 ||
        !s->j1 || !s->tau || !s->dtau || !s->tnext || !s->act) {
        or_sim_free(s);
        return NULL;
    }
    memcpy(s->m, m, (size_t)n * sizeof(double));
    memcpy(s->x, x, v3);
    memcpy(s->v, v, v3);
    for (int64_t i = 0; i < n; i++)
        s->act[i] = (int32_t)i;
    or_force(n, s->m, s->x, s->v, s->eps2, n, s->act, s->a, s->j);
    s->interactions += (double)n * (double)n;
    for (int64_t i = 0; i < n; i++) {
        if (fixed_dtau > 0) {
            s->dtau[i] = fixed_dtau;
        } else {
            double dt0 = eta * norm3(s->a + 3 * i) / norm3(s->j + 3 * i);
            s->dtau[i] = or_quantise_init(dt0, dt_min, s->dtau_max);
        }
        s->tnext[i] = s->dtau[i];
    }
    return s;
}

/* Adds the post-Newtonian terms of the pair (p, q) to particle i's force and
 * jerk, from positions x and velocities v of both (the same time); the jerk's
 * relative acceleration is the pair's Newtonian one, -M r / |r|^3. */
static void add_pn(const or_sim *s, int64_t i, const double *x, const double *v, double a[3], double j[3])
{
    int64_t p = s->pn_p, q = s->pn_q;
    double mp = s->m[p], mq = s->m[q], M = mp + mq;
    double r[3], vr[3], ar[3], apn[3], jpn[3];
    for (int c = 0; c < 3; c++) {
        r[c] = x[3 * p + c] - x[3 * q + c];
        vr[c] = v[3 * p + c] - v[3 * q + c];
    }
    double rr = norm3(r);
    for (int c = 0; c < 3; c++)
        ar[c] = -M * r[c] / (rr * rr * rr);
    or_pn_accel(mp, mq, r, vr, s->pn_c, s->pn_terms, apn);
    or_pn_jerk(mp, mq, r, vr, ar, s->pn_c, s->pn_terms, jpn);
    double w = i == p ? mq / M : -mp / M;
    for (int c = 0; c < 3; c++) {
        a[c] += w * apn[c];
        j[c] += w * jpn[c];
    }
}

/* Enables the post-Newtonian terms of the pair (p, q) (p != q, terms as for
 * or_pn_accel, c > 0).  Called before the first block step: the initial
 * forces and first steps of p and q are recomputed with the terms.  Returns 0,
 * or -1 for a bad argument or a call after the first step. */
int or_sim_set_pn(or_sim *s, int32_t p, int32_t q, double c, int terms)
{
    if (p < 0 || q < 0 || p >= s->n || q >= s->n || p == q || !(c > 0) || (terms & ~7) || s->nblock > 0)
        return -1;
    s->pn_p = p;
    s->pn_q = q;
    s->pn_c = c;
    s->pn_terms = terms;
    int32_t pq[2] = {p, q};
    or_force(s->n, s->m, s->x, s->v, s->eps2, 2, pq, s->a1, s->j1);
    for (int k = 0; k < 2; k++) {
        int64_t i = pq[k];
        add_pn(s, i, s->x, s->v, s->a1 + 3 * k, s->j1 + 3 * k);
        for (int cc = 0; cc < 3; cc++) {
            s->a[3 * i + cc] = s->a1[3 * k + cc];
            s->j[3 * i + cc] = s->j1[3 * k + cc];
        }
        if (s->fixed_dtau <= 0) {
            double dt0 = s->eta * norm3(s->a + 3 * i) / norm3(s->j + 3 * i);
            s->dtau[i] = or_quantise_init(dt0, s->dt_min, s->dtau_max);
            s->tnext[i] = s->dtau[i];
        }
    }
    return 0;
}

/* Steps 6-7 for a given block time and active list (idx ascending or not). */
static void block_step(or_sim *s, int64_t tick_next, int64_t nact, const int32_t *idx)
{
    int64_t n = s->n;
    /* 7a: predict every particle to the block time */
    for (int64_t i = 0; i < n; i++) {
        double dt = (double)(tick_next - s->tau[i]) * s->dt_min;
        or_predict_one(s->x + 3 * i, s->v + 3 * i, s->a + 3 * i, s->j + 3 * i, dt,
                       s->xp + 3 * i, s->vp + 3 * i);
    }
    /* 7c: new force and jerk of the active particles from predicted values */
    or_force(n, s->m, s->xp, s->vp, s->eps2, nact, idx, s->a1, s->j1);
    s->interactions += (double)nact * (double)n;
    if (s->pn_terms)
        for (int64_t k = 0; k < nact; k++)
            if (idx[k] == s->pn_p || idx[k] == s->pn_q)
                add_pn(s, idx[k], s->xp, s->vp, s->a1 + 3 * k, s->j1 + 3 * k);
    /* 7d + 6: correct, take the new step, and keep a1, j1 as the new a0, j0 */
    for (int64_t k = 0; k < nact; k++) {
        int64_t i = idx[k];
        double dt = (double)(tick_next - s->tau[i]) * s->dt_min;
        double a2[3], a3[3], a2e[3];
        double *a0 = s->a + 3 * i, *j0 = s->j + 3 * i;
        double *a1 = s->a1 + 3 * k, *j1 = s->j1 + 3 * k;
        or_hermite_derivs(a0, j0, a1, j1, dt, a2, a3);
        or_correct_one(s->xp + 3 * i, s->vp + 3 * i, a2, a3, dt, s->x + 3 * i, s->v + 3 * i);
        for (int c = 0; c < 3; c++)
            a2e[c] = a2[c] + dt * a3[c];
        int64_t dtau;
        if (s->fixed_dtau > 0) {
            dtau = s->fixed_dtau;
        } else {
            double dtn = or_aarseth_dt(a1, j1, a2e, a3, s->eta);
            dtau = or_quantise(dtn, s->dtau[i], tick_next, s->dt_min, s->dtau_max);
        }
        for (int c = 0; c < 3; c++) {
            a0[c] = a1[c];
            j0[c] = j1[c];
        }
        s->tau[i] = tick_next;
        s->dtau[i] = dtau;
        s->tnext[i] = tick_next + dtau;
    }
    s->tick = tick_next;
    s->nblock += 1;
    s->nsteps += nact;
}

/* One free-running block step (steps 5-7).  Writes the block time and the
 * active list (ascending) when the pointers are not NULL. */
int64_t or_sim_step(or_sim *s, int64_t *tick_out, int32_t *idx_out)
{
    int64_t tick_next;
    int64_t nact = or_active(s->n, s->tnext, s->act, &tick_next);
    block_step(s, tick_next, nact, s->act);
    if (tick_out)
        *tick_out = tick_next;
    if (idx_out)
        memcpy(idx_out, s->act, (size_t)nact * sizeof(int32_t));
    return nact;
}

/* One block step with a recorded block time and active list. */
void or_sim_replay(or_sim *s, int64_t tick_next, int64_t nact, const int32_t *idx)
{
    block_step(s, tick_next, nact, idx);
}

/* Advance until no particle's next time is <= tick_end.  Returns the number
 * of block steps taken. */
int64_t or_sim_evolve(or_sim *s, int64_t tick_end)
{
    int64_t steps = 0;
    for (;;) {
        int64_t tmin = s->tnext[0];
        for (int64_t i = 1; i < s->n; i++)
            if (s->tnext[i] < tmin)
                tmin = s->tnext[i];
        if (tmin > tick_end)
            break;
        or_sim_step(s, NULL, NULL);
        steps++;
    }
    return steps;
}

/* Energy of the system at the time of the last block step: every particle is
 * predicted to that time first (particles already there are unchanged). */
void or_sim_energy(or_sim *s, double *K, double *U)
{
    for (int64_t i = 0; i < s->n; i++) {
        double dt = (double)(s->tick - s->tau[i]) * s->dt_min;
        or_predict_one(s->x + 3 * i, s->v + 3 * i, s->a + 3 * i, s->j + 3 * i, dt,
                       s->xp + 3 * i, s->vp + 3 * i);
    }
    or_energy(s->n, s->m, s->xp, s->vp, s->eps2, K, U);
}

/* Copies of the state; any pointer may be NULL. */
void or_sim_get(const or_sim *s, double *x, double *v, double *a, double *j, int64_t *tau,
                int64_t *dtau)
{
    size_t v3 = (size_t)s->n * 3 * sizeof(double);
    if (x) memcpy(x, s->x, v3);
    if (v) memcpy(v, s->v, v3);
    if (a) memcpy(a, s->a, v3);
    if (j) memcpy(j, s->j, v3);
    if (tau) memcpy(tau, s->tau, (size_t)s->n * sizeof(int64_t));
    if (dtau) memcpy(dtau, s->dtau, (size_t)s->n * sizeof(int64_t));
}

void or_sim_stats(const or_sim *s, int64_t *tick, int64_t *nblock, int64_t *nsteps,
                  double *interactions)
{
    if (tick) *tick = s->tick;
    if (nblock) *nblock = s->nblock;
    if (nsteps) *nsteps = s->nsteps;
    if (interactions) *interactions = s->interactions;
}
