// hermite6.cu -- the sixth-order Hermite block-step integrator (gd_h6_* in
// include/gravidy.h), FP64, on the GPU.
//
// The block scheme is GraviDy's (Sec. 2.4: active set, prediction of all N,
// force of the active set from predicted values, correction, new block steps),
// raised to sixth order as in the sixth-order Hermite scheme the paper cites
// (Nitadori & Makino 2008): the force kernel also returns the snap (the second
// time derivative of the softened force), which needs the predicted
// accelerations of all particles; the predictor carries x to dt^5, v to dt^4
// and a to dt^3 with the crackle c; the corrector is the time-symmetric sixth-
// order formula; crackle, pop and the fifth derivative at the end of the step
// come from the quintic Hermite interpolant of (a, jerk, snap) at both ends;
// the step is the generalised Aarseth criterion
//     dt = eta ( (|a||snap| + |jerk|^2) / (|crackle||a^(5)| + |pop|^2) )^(1/6),
// quantised to power-of-two block steps by the same rules as the fourth-order
// path.  Every operation is FP64 (GB300 issues an FP64 warp instruction about
// once per 78 cycles per scheduler, so this path is about 70x slower per pair
// than the mixed fourth-order one; it is the accuracy-first form).
//
// The same engine runs the fourth-order scheme in its time-symmetric form
// (order 4: the corrector of Hut, Makino & McMillan 1995,
//     v1 = v0 + h (a1 + a0) - h^2 (j1 - j0) / 3,  x1 = x0 + h (v1 + v0) - h^2 (a1 - a0) / 3,
// h = dt / 2, with the cubic predictor, force and jerk only, and Aarseth's
// fourth-order step; snap and crackle stay zero), and either order can iterate
// evaluation and correction n_iter times per block step (P(EC)^n, Kokubo,
// Yoshinaga & Makino 1998): every pass but the last writes the corrected x, v
// and the new a of each active particle over its prediction, so the next pass
// sees them; with shared constant steps and n_iter >= 2 the map is reversible.
//
// Kernels per block step (1 + 2 n_iter, captured as a CUDA graph of G steps):
//   k6_select_predict  predict every particle to T_cur, append the active ones
//                      to the list (arrival order) and start the next-time
//                      minimum over the inactive ones;
//   k6_force           persistent CTAs over (active particle, j-chunk) items:
//                      each CTA sums force, jerk and snap of one active particle
//                      over one j-chunk with a fixed shared-memory tree; the
//                      split depends only on N_act and N, so a particle's sum
//                      does not depend on its slot;
//   k6_correct         one thread per active particle: the S partials summed in
//                      split order, interpolant derivatives, correction, step;
//                      the last CTA turns the minimum into the next block time.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gravidy.h"

namespace gdk6 {

constexpr int T6 = 128;   // threads per CTA
constexpr int NC = 9;     // force, jerk, snap components
constexpr int G6 = 16;    // block steps per graph launch

struct Ctrl6 {
    long long T_cur;       // block time of the next step (ticks)
    long long T_acc;       // running minimum of the next times
    long long T_last;      // block time of the last finished step
    long long tick_end;    // steps whose block time is above this are skipped
    long long nblock, nsteps;
    double interactions;
    int nact;              // active particles appended by the select kernel
    int last_nact;
    int err;
    unsigned done;         // finished-CTA counter of k6_correct
};

struct Dev6 {
    int n;
    int order;                       // 4 (time-symmetric fourth order) or 6
    int n_iter;                      // evaluation-correction passes per block step
    double dt_min, eps2, eta;
    long long dtau_max;
    double *m;
    double *x, *v, *a, *j, *s, *c;   // state at each particle's time, planes c*n + i
    double *xp, *vp, *ap;            // predicted to the block time
    long long *tau, *dtau, *tnext;
    int *act;
    double *part;                    // j-split partials, (sidx * NC + comp) * nact + k
    long long cap;                   // partial capacity per component (S * nact <= cap)
    double *fsum;                    // summed force of slot k: fsum[comp * n + k] (hooks, initial forces)
    double *eu, *ek;                 // per-particle energy terms
    Ctrl6 *ctrl;
};

struct Plan6 {
    int S;          // j-chunks per active particle
    int chunk;      // j per chunk, a multiple of T6
    long long items;
};

// Items fill about two waves of the persistent grid; the split depends only on
// (nact, n, grid, cap).
__host__ __device__ inline Plan6 plan6(int nact, int n, int grid, long long cap)
{
    Plan6 p;
    const int blocks = (n + T6 - 1) / T6;
    long long S = nact > 0 ? (2LL * grid + nact - 1) / nact : 1;
    if (S > blocks) S = blocks;
    if (S < 1) S = 1;
    if (nact > 0 && S * (long long)nact > cap) S = cap / nact;
    if (S < 1) S = 1;
    const int bpc = (int)((blocks + S - 1) / S);
    p.chunk = bpc * T6;
    p.S = (blocks + bpc - 1) / bpc;
    p.items = (long long)nact * p.S;
    return p;
}

__device__ __forceinline__ void set_err6(Ctrl6 *c, int code) { atomicCAS(&c->err, 0, code); }

// Taylor prediction of particle i over dt: x to dt^5, v to dt^4, a to dt^3.
__device__ __forceinline__ void predict6(const Dev6 &d, int i, double dt)
{
    const int n = d.n;
    const double dt2 = dt * dt, dt3 = dt2 * dt, dt4 = dt3 * dt, dt5 = dt4 * dt;
    for (int q = 0; q < 3; q++) {
        const int o = q * n + i;
        const double x = d.x[o], v = d.v[o], a = d.a[o], j = d.j[o], s = d.s[o], c = d.c[o];
        d.xp[o] = x + v * dt + a * dt2 / 2.0 + j * dt3 / 6.0 + s * dt4 / 24.0 + c * dt5 / 120.0;
        d.vp[o] = v + a * dt + j * dt2 / 2.0 + s * dt3 / 6.0 + c * dt4 / 24.0;
        d.ap[o] = a + j * dt + s * dt2 / 2.0 + c * dt3 / 6.0;
    }
}

__global__ void __launch_bounds__(T6) k6_select_predict(Dev6 d)
{
    Ctrl6 *ctrl = d.ctrl;
    const long long T = ctrl->T_cur;
    if (T > ctrl->tick_end) return;
    const int i = blockIdx.x * T6 + threadIdx.x;
    long long mn = LLONG_MAX;
    if (i < d.n) {
        const long long tn = d.tnext[i];
        if (tn == T) {
            const int pos = atomicAdd(&ctrl->nact, 1);
            if (pos < d.n) d.act[pos] = i;
        } else {
            mn = tn;
        }
        predict6(d, i, (double)(T - d.tau[i]) * d.dt_min);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long w = __shfl_xor_sync(0xffffffffu, mn, o);
        mn = w < mn ? w : mn;
    }
    if ((threadIdx.x & 31) == 0 && mn != LLONG_MAX) atomicMin((unsigned long long *)&ctrl->T_acc, (unsigned long long)mn);
}

// Every particle predicted to tick (hooks, energy, replay); no list.
__global__ void k6_predict_all(Dev6 d, long long tick)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < d.n) predict6(d, i, (double)(tick - d.tau[i]) * d.dt_min);
}

// The pair term with r = x_j - x_i, u = v_j - v_i, w = a_j - a_i, s^2 = r^2 + eps^2:
//   A0 = m r / s^3,  alpha = (r.u) / s^2,  A1 = m u / s^3 - 3 alpha A0,
//   beta = (u.u + r.w) / s^2 + alpha^2,  A2 = m w / s^3 - 6 alpha A1 - 3 beta A0.
// SNAP = false (order 4) evaluates A0 and A1 only and leaves the snap partials zero.
template <bool SNAP>
__global__ void __launch_bounds__(T6) k6_force(Dev6 d, int grid)
{
    constexpr int NQ = SNAP ? NC : 6;   // components reduced
    const int nact = min(d.ctrl->nact, d.n);
    if (nact <= 0) return;
    const Plan6 pl = plan6(nact, d.n, grid, d.cap);
    const int n = d.n, t = threadIdx.x;
    __shared__ double red[NC][T6];
    for (long long item = blockIdx.x; item < pl.items; item += gridDim.x) {
        const int k = (int)(item / pl.S), sidx = (int)(item % pl.S);
        const int i = d.act[k];
        const double xi = d.xp[i], yi = d.xp[n + i], zi = d.xp[2 * n + i];
        const double ui = d.vp[i], vi = d.vp[n + i], wi = d.vp[2 * n + i];
        double pi = 0.0, qi = 0.0, ri = 0.0;
        if (SNAP) {
            pi = d.ap[i];
            qi = d.ap[n + i];
            ri = d.ap[2 * n + i];
        }
        double f[NC];
#pragma unroll
        for (int q = 0; q < NC; q++) f[q] = 0.0;
        const int jb = sidx * pl.chunk, je = min(jb + pl.chunk, n);
        for (int jj = jb + t; jj < je; jj += T6) {
            if (jj == i) continue;
            const double rx = d.xp[jj] - xi, ry = d.xp[n + jj] - yi, rz = d.xp[2 * n + jj] - zi;
            const double ux = d.vp[jj] - ui, uy = d.vp[n + jj] - vi, uz = d.vp[2 * n + jj] - wi;
            const double ss = rx * rx + ry * ry + rz * rz + d.eps2;
            const double rinv = rsqrt(ss);
            const double rinv2 = rinv * rinv;
            const double mi3 = d.m[jj] * rinv * rinv2;
            const double alpha = (rx * ux + ry * uy + rz * uz) * rinv2;
            const double a0x = mi3 * rx, a0y = mi3 * ry, a0z = mi3 * rz;
            const double a1x = mi3 * ux - 3.0 * alpha * a0x, a1y = mi3 * uy - 3.0 * alpha * a0y,
                         a1z = mi3 * uz - 3.0 * alpha * a0z;
            f[0] += a0x;
            f[1] += a0y;
            f[2] += a0z;
            f[3] += a1x;
            f[4] += a1y;
            f[5] += a1z;
            if (SNAP) {
                const double wx = d.ap[jj] - pi, wy = d.ap[n + jj] - qi, wz = d.ap[2 * n + jj] - ri;
                const double beta =
                    (ux * ux + uy * uy + uz * uz + rx * wx + ry * wy + rz * wz) * rinv2 + alpha * alpha;
                f[6] += mi3 * wx - 6.0 * alpha * a1x - 3.0 * beta * a0x;
                f[7] += mi3 * wy - 6.0 * alpha * a1y - 3.0 * beta * a0y;
                f[8] += mi3 * wz - 6.0 * alpha * a1z - 3.0 * beta * a0z;
            }
        }
        // fixed pairwise tree over the CTA's threads
        __syncthreads();  // red[] of the previous item has been read
#pragma unroll
        for (int q = 0; q < NQ; q++) red[q][t] = f[q];
        __syncthreads();
        for (int h = T6 / 2; h >= 1; h >>= 1) {
            if (t < h)
#pragma unroll
                for (int q = 0; q < NQ; q++) red[q][t] += red[q][t + h];
            __syncthreads();
        }
        if (t < NC) d.part[((long long)sidx * NC + t) * nact + k] = t < NQ ? red[t][0] : 0.0;
    }
}

// The S partials of slot k, component q, in split order.
__device__ __forceinline__ double part_sum6(const Dev6 &d, int nact, int S, int q, int k)
{
    double acc = 0.0;
    for (int sidx = 0; sidx < S; sidx++) acc += d.part[((long long)sidx * NC + q) * nact + k];
    return acc;
}

// Summed force, jerk and snap of every active slot into fsum (hooks, initial forces).
__global__ void k6_sum(Dev6 d, int grid)
{
    const int nact = min(d.ctrl->nact, d.n);
    const Plan6 pl = plan6(nact, d.n, grid, d.cap);
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nact * NC) return;
    const int q = w / nact, k = w % nact;
    d.fsum[(long long)q * d.n + k] = part_sum6(d, nact, pl.S, q, k);
}

// Power-of-two block step after a correction at tick T from the estimate dt_new:
// shrink to the largest power of two of dt_min not above dt_new (at least 1 tick);
// grow by 2 only if dt_new >= 2 dt_old, the doubled step is within dtau_max and T
// is a multiple of twice the old step; a NaN estimate counts as unconstrained.
__device__ __forceinline__ long long quantise6(const Dev6 &d, double dt_new, long long dtau_old, long long T)
{
    const double dt_old = (double)dtau_old * d.dt_min;
    if (dt_new < dt_old) {
        const double q = dt_new / d.dt_min;
        if (q < 1.0) return 1;
        int e;
        frexp(q, &e);
        return 1LL << (e - 1);
    }
    if (!(dt_new == dt_new) || dt_new >= 2.0 * dt_old)
        if (2 * dtau_old <= d.dtau_max && T % (2 * dtau_old) == 0) return 2 * dtau_old;
    return dtau_old;
}

__device__ __forceinline__ double norm3(double x, double y, double z) { return sqrt(x * x + y * y + z * z); }

// Corrected position x1 and velocity v1 (component q) of particle i over dt
// from its state at its own time and the new a1, j1 (and s1 at order 6).
__device__ __forceinline__ void corrected(const Dev6 &d, int o, double dt, double a1, double j1, double s1,
                                          double &x1, double &v1)
{
    const double h = 0.5 * dt, h2 = h * h;
    const double x0 = d.x[o], v0 = d.v[o], a0 = d.a[o], j0 = d.j[o];
    if (d.order == 6) {
        const double h3 = h2 * h, s0 = d.s[o];
        v1 = v0 + h * (a1 + a0) - 0.4 * h2 * (j1 - j0) + h3 * (s1 + s0) / 15.0;
        x1 = x0 + h * (v1 + v0) - 0.4 * h2 * (a1 - a0) + h3 * (j1 + j0) / 15.0;
    } else {
        v1 = v0 + h * (a1 + a0) - h2 * (j1 - j0) / 3.0;
        x1 = x0 + h * (v1 + v0) - h2 * (a1 - a0) / 3.0;
    }
}

// A pass that is not the last: the corrected x, v and the new a of active slot k
// replace the particle's prediction (the next pass evaluates against them).
__device__ void trial6(const Dev6 &d, int k, long long T, const double a1[3], const double j1[3],
                       const double s1[3], int &bad)
{
    const int n = d.n;
    const int i = d.act[k];
    const double dt = (double)(T - d.tau[i]) * d.dt_min;
    for (int q = 0; q < 3; q++) {
        const int o = q * n + i;
        double x1, v1;
        corrected(d, o, dt, a1[q], j1[q], s1[q], x1, v1);
        if (!isfinite(x1) || !isfinite(v1)) bad = 1;
        d.xp[o] = x1;
        d.vp[o] = v1;
        d.ap[o] = a1[q];
    }
}

// Correct active slot k at block time T with its new force a1, jerk j1, snap s1
// (zero at order 4), take its new step and commit the state.
__device__ void correct6(const Dev6 &d, int k, long long T, const double a1[3], const double j1[3],
                         const double s1[3], long long &tn_out, int &bad)
{
    const int n = d.n;
    const int i = d.act[k];
    const long long dtick = T - d.tau[i];
    const double dt = (double)dtick * d.dt_min;
    double crk[3] = {0.0, 0.0, 0.0}, x1[3], v1[3];
    double dt_new;
    if (d.order == 6) {
        const double h = 0.5 * dt, h2 = h * h, h3 = h2 * h, h5 = h3 * h2;
        double pop[3], a5[3];
        for (int q = 0; q < 3; q++) {
            const int o = q * n + i;
            const double a0 = d.a[o], j0 = d.j[o], s0 = d.s[o];
            // the quintic interpolant on [-h, h] and its derivatives at +h
            const double Am = 0.5 * (a1[q] - a0), Jp = 0.5 * (j1[q] + j0), Jm = 0.5 * (j1[q] - j0);
            const double Sp = 0.5 * (s1[q] + s0), Sm = 0.5 * (s1[q] - s0);
            const double c4 = (Sp * h - Jm) / (8.0 * h3);
            const double c5 = (Sm * h2 - 3.0 * Jp * h + 3.0 * Am) / (8.0 * h5);
            const double c3 = (0.5 * (Jp * h - Am) - 2.0 * c5 * h5) / h3;
            crk[q] = 6.0 * c3 + 24.0 * c4 * h + 60.0 * c5 * h2;
            pop[q] = 24.0 * c4 + 120.0 * c5 * h;
            a5[q] = 120.0 * c5;
            corrected(d, o, dt, a1[q], j1[q], s1[q], x1[q], v1[q]);
        }
        const double na = norm3(a1[0], a1[1], a1[2]), nj = norm3(j1[0], j1[1], j1[2]);
        const double ns = norm3(s1[0], s1[1], s1[2]), nc = norm3(crk[0], crk[1], crk[2]);
        const double np = norm3(pop[0], pop[1], pop[2]), nq = norm3(a5[0], a5[1], a5[2]);
        dt_new = d.eta * pow((na * ns + nj * nj) / (nc * nq + np * np), 1.0 / 6.0);
    } else {
        // second and third derivative of the cubic interpolant of (a, jerk) at
        // both ends, taken to the end of the step for Aarseth's criterion
        const double dt2 = dt * dt, dt3 = dt2 * dt;
        double a2e[3], a3[3];
        for (int q = 0; q < 3; q++) {
            const int o = q * n + i;
            const double a0 = d.a[o], j0 = d.j[o];
            const double da = a0 - a1[q];
            const double a2 = (-6.0 * da - dt * (4.0 * j0 + 2.0 * j1[q])) / dt2;
            a3[q] = (12.0 * da + 6.0 * dt * (j0 + j1[q])) / dt3;
            a2e[q] = a2 + dt * a3[q];
            corrected(d, o, dt, a1[q], j1[q], 0.0, x1[q], v1[q]);
        }
        const double na = norm3(a1[0], a1[1], a1[2]), nj = norm3(j1[0], j1[1], j1[2]);
        const double n2 = norm3(a2e[0], a2e[1], a2e[2]), n3 = norm3(a3[0], a3[1], a3[2]);
        dt_new = sqrt(d.eta * (na * n2 + nj * nj) / (nj * n3 + n2 * n2));
    }
    const long long dtau = quantise6(d, dt_new, d.dtau[i], T);
    for (int q = 0; q < 3; q++) {
        const int o = q * n + i;
        if (!isfinite(x1[q]) || !isfinite(v1[q])) bad = 1;
        d.x[o] = x1[q];
        d.v[o] = v1[q];
        d.a[o] = a1[q];
        d.j[o] = j1[q];
        d.s[o] = s1[q];
        d.c[o] = crk[q];
    }
    d.tau[i] = T;
    d.dtau[i] = dtau;
    d.tnext[i] = T + dtau;
    tn_out = T + dtau;
}

// commit = 0: a pass that is not the last (trial6 per slot, no bookkeeping);
// commit = 1: correction, new steps, and the last CTA turns the minimum into
// the next block time.
__global__ void __launch_bounds__(T6) k6_correct(Dev6 d, int grid, int commit)
{
    Ctrl6 *ctrl = d.ctrl;
    const int nact = min(ctrl->nact, d.n);
    if (nact <= 0) return;
    const Plan6 pl = plan6(nact, d.n, grid, d.cap);
    const int ncta = min((int)gridDim.x, (nact + T6 - 1) / T6);
    if ((int)blockIdx.x >= ncta) return;
    const long long T = ctrl->T_cur;
    long long mn = LLONG_MAX;
    int bad = 0;
    for (int k = blockIdx.x * T6 + threadIdx.x; k < nact; k += ncta * T6) {
        double f[NC];
        for (int q = 0; q < NC; q++) f[q] = part_sum6(d, nact, pl.S, q, k);
        if (!commit) {
            trial6(d, k, T, f, f + 3, f + 6, bad);
            continue;
        }
        long long tn;
        correct6(d, k, T, f, f + 3, f + 6, tn, bad);
        mn = tn < mn ? tn : mn;
    }
    if (bad) set_err6(ctrl, GD_ENONFINITE);
    if (!commit) return;
    for (int o = 16; o > 0; o >>= 1) {
        const long long w = __shfl_xor_sync(0xffffffffu, mn, o);
        mn = w < mn ? w : mn;
    }
    if ((threadIdx.x & 31) == 0 && mn != LLONG_MAX) atomicMin((unsigned long long *)&ctrl->T_acc, (unsigned long long)mn);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&ctrl->done, 1u);
        if (prev == (unsigned)ncta - 1) {
            __threadfence();
            const long long next = (long long)atomicAdd((unsigned long long *)&ctrl->T_acc, 0ull);
            ctrl->T_last = T;
            ctrl->last_nact = nact;
            ctrl->T_cur = next;
            ctrl->T_acc = LLONG_MAX;
            ctrl->nblock += 1;
            ctrl->nsteps += nact;
            ctrl->interactions += (double)d.n_iter * (double)nact * (double)d.n;
            ctrl->nact = 0;
            ctrl->done = 0;
        }
    }
}

// Initial forces: a and jerk from pass 1 (fsum, predicted accelerations zero),
// snap from pass 2; first steps eta_init |a| / |jerk|, quantised; crackle 0.
__global__ void k6_take(Dev6 d, int pass)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int n = d.n;
    for (int q = 0; q < 3; q++) {
        if (pass == 1) {
            d.a[q * n + i] = d.fsum[(long long)q * n + i];
            d.j[q * n + i] = d.fsum[(long long)(3 + q) * n + i];
        } else {
            d.s[q * n + i] = d.fsum[(long long)(6 + q) * n + i];
        }
    }
}

__global__ void k6_init_steps(Dev6 d, double eta_init)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int n = d.n;
    const double na = norm3(d.a[i], d.a[n + i], d.a[2 * n + i]);
    const double nj = norm3(d.j[i], d.j[n + i], d.j[2 * n + i]);
    const double dt = eta_init * na / nj;
    long long dtau;
    if (!(dt < INFINITY)) {
        dtau = d.dtau_max;
    } else {
        const double q = dt / d.dt_min;
        if (q < 1.0) {
            dtau = 1;
        } else if (q >= (double)d.dtau_max) {
            dtau = d.dtau_max;
        } else {
            int e;
            frexp(q, &e);
            dtau = 1LL << (e - 1);
        }
    }
    d.tau[i] = 0;
    d.dtau[i] = dtau;
    d.tnext[i] = dtau;
}

// Next block time = minimum of all next times (after initialisation or a replayed step).
__global__ void k6_resync(Dev6 d)
{
    __shared__ long long s_m[32];
    long long mn = LLONG_MAX;
    for (int i = threadIdx.x; i < d.n; i += blockDim.x) mn = d.tnext[i] < mn ? d.tnext[i] : mn;
    for (int o = 16; o > 0; o >>= 1) {
        const long long w = __shfl_xor_sync(0xffffffffu, mn, o);
        mn = w < mn ? w : mn;
    }
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = mn;
    __syncthreads();
    if (threadIdx.x < 32) {
        mn = threadIdx.x < (int)(blockDim.x >> 5) ? s_m[threadIdx.x] : LLONG_MAX;
        for (int o = 16; o > 0; o >>= 1) {
            const long long w = __shfl_xor_sync(0xffffffffu, mn, o);
            mn = w < mn ? w : mn;
        }
        if (threadIdx.x == 0) {
            d.ctrl->T_cur = mn;
            d.ctrl->T_acc = LLONG_MAX;
            d.ctrl->nact = 0;
            d.ctrl->done = 0;
        }
    }
}

__global__ void k6_set_list(Dev6 d, long long tick, int nact)
{
    d.ctrl->T_cur = tick;
    d.ctrl->nact = nact;
}

__global__ void k6_set_tick_end(Ctrl6 *c, long long t) { c->tick_end = t; }

__global__ void k6_iota(int *p, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

// Energy terms of particle i from the predicted state: K_i and U_i (U counts
// each pair twice; the host halves it).
__global__ void __launch_bounds__(T6) k6_energy_terms(Dev6 d)
{
    const int n = d.n;
    const int i = blockIdx.x * T6 + threadIdx.x;
    if (i >= n) return;
    const double xi = d.xp[i], yi = d.xp[n + i], zi = d.xp[2 * n + i];
    double u = 0.0;
    for (int jj = 0; jj < n; jj++) {
        if (jj == i) continue;
        const double rx = d.xp[jj] - xi, ry = d.xp[n + jj] - yi, rz = d.xp[2 * n + jj] - zi;
        u -= d.m[jj] / sqrt(rx * rx + ry * ry + rz * rz + d.eps2);
    }
    d.eu[i] = 0.5 * d.m[i] * u;
    const double vx = d.vp[i], vy = d.vp[n + i], vz = d.vp[2 * n + i];
    d.ek[i] = 0.5 * d.m[i] * (vx * vx + vy * vy + vz * vz);
}

}  // namespace gdk6

using namespace gdk6;

struct gd_h6 {
    int dev;
    cudaStream_t stream;
    bool own_stream;
    Dev6 d;
    int grid;
    Ctrl6 *h_ctrl;       // pinned mirror
    double *h_stage;     // pinned staging: 9 n doubles
    cudaGraphExec_t graph;
    long long launches;
    std::vector<void *> allocs;
    std::string err;
    int sticky;
};

static thread_local std::string g_h6_err;

// allocation-failure injection of gd_test_fail_alloc (gravidy.cu)
bool gd_alloc_fails(int kind);

namespace {

int fail6(gd_h6 *s, int code, const std::string &msg)
{
    if (s)
        s->err = msg;
    else
        g_h6_err = msg;
    return code;
}

#define CK6(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return fail6(s, GD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int sync6(gd_h6 *s)
{
    CK6(cudaMemcpyAsync(s->h_ctrl, s->d.ctrl, sizeof(Ctrl6), cudaMemcpyDeviceToHost, s->stream));
    CK6(cudaStreamSynchronize(s->stream));
    if (s->h_ctrl->err != 0) {
        s->sticky = s->h_ctrl->err;
        return fail6(s, s->h_ctrl->err, "device reported a fault (non-finite state)");
    }
    return GD_OK;
}

int usable6(gd_h6 *s)
{
    if (!s) return fail6(nullptr, GD_EINVAL, "null context");
    if (s->sticky) return fail6(s, GD_ESTATE, "context is unusable after an earlier device fault");
    CK6(cudaSetDevice(s->dev));
    return GD_OK;
}

// kernel launches per block step
long long per_step6(const gd_h6 *s) { return 1 + 2LL * s->d.n_iter; }

void launch_force6(gd_h6 *s)
{
    if (s->d.order == 6)
        k6_force<true><<<s->grid, T6, 0, s->stream>>>(s->d, s->grid);
    else
        k6_force<false><<<s->grid, T6, 0, s->stream>>>(s->d, s->grid);
    s->launches += 1;
}

// the n_iter evaluation-correction passes of the current list; the last commits
void passes6(gd_h6 *s)
{
    for (int pass = 1; pass <= s->d.n_iter; pass++) {
        launch_force6(s);
        k6_correct<<<s->grid, T6, 0, s->stream>>>(s->d, s->grid, pass == s->d.n_iter ? 1 : 0);
        s->launches += 1;
    }
}

void step6(gd_h6 *s)
{
    const int gsel = (s->d.n + T6 - 1) / T6;
    k6_select_predict<<<gsel, T6, 0, s->stream>>>(s->d);
    s->launches += 1;
    passes6(s);
}

// force of the listed slots into fsum (plan of the current list)
void force_sum6(gd_h6 *s, int nact)
{
    launch_force6(s);
    k6_sum<<<(nact * NC + 255) / 256, 256, 0, s->stream>>>(s->d, s->grid);
    s->launches += 1;
}

// AoS host (n x 3) -> device planes, through the pinned stage
int upload6(gd_h6 *s, double *dst, const double *src)
{
    const int n = s->d.n;
    for (int i = 0; i < n; i++)
        for (int q = 0; q < 3; q++) s->h_stage[(size_t)q * n + i] = src[3 * i + q];
    CK6(cudaMemcpyAsync(dst, s->h_stage, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s->stream));
    CK6(cudaStreamSynchronize(s->stream));
    return GD_OK;
}

// device planes (rows x 3 with plane stride) -> AoS host
int download6(gd_h6 *s, double *dst, const double *src, long long stride, int rows)
{
    for (int q = 0; q < 3; q++)
        CK6(cudaMemcpyAsync(s->h_stage + (size_t)q * rows, src + q * stride, sizeof(double) * rows,
                            cudaMemcpyDeviceToHost, s->stream));
    CK6(cudaStreamSynchronize(s->stream));
    for (int i = 0; i < rows; i++)
        for (int q = 0; q < 3; q++) dst[3 * i + q] = s->h_stage[(size_t)q * rows + i];
    return GD_OK;
}

int build_graph6(gd_h6 *s)
{
    if (s->graph) return GD_OK;
    CK6(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    const long long before = s->launches;
    for (int k = 0; k < G6; k++) step6(s);
    s->launches = before;
    cudaGraph_t g;
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    if (e != cudaSuccess) return fail6(s, GD_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        s->graph = nullptr;
        return fail6(s, GD_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    return GD_OK;
}

bool pow2(double x)
{
    if (!(x > 0) || !std::isfinite(x)) return false;
    int e;
    return std::frexp(x, &e) == 0.5;
}

}  // namespace

extern "C" {

void gd_h6_free(gd_h6 *s)
{
    if (!s) return;
    cudaSetDevice(s->dev);
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->graph) cudaGraphExecDestroy(s->graph);
    for (void *p : s->allocs) cudaFree(p);
    if (s->h_ctrl) cudaFreeHost(s->h_ctrl);
    if (s->h_stage) cudaFreeHost(s->h_stage);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

const char *gd_h6_last_error(const gd_h6 *s) { return s ? s->err.c_str() : g_h6_err.c_str(); }

int gd_h6_init_scheme(gd_h6 **out, int64_t n, const double *m, const double *x, const double *v, double eps,
                      double eta, double eta_init, int32_t order, int32_t n_iter, const gd_opts *opt)
{
    if (!out) return fail6(nullptr, GD_EINVAL, "out is required");
    *out = nullptr;
    if (order != 4 && order != 6) return fail6(nullptr, GD_EINVAL, "order must be 4 or 6");
    if (n_iter < 1 || n_iter > 16) return fail6(nullptr, GD_EINVAL, "n_iter must be in [1, 16]");
    gd_opts o;
    gd_opts_default(&o);
    if (opt) o = *opt;
    if (n < 1 || n > (1 << 22)) return fail6(nullptr, GD_EINVAL, "n must be in [1, 2^22]");
    if (!m || !x || !v) return fail6(nullptr, GD_EINVAL, "m, x and v are required");
    if (!(eps >= 0) || !std::isfinite(eps)) return fail6(nullptr, GD_EINVAL, "eps must be finite and >= 0");
    if (!(eta > 0) || !std::isfinite(eta) || !(eta_init > 0) || !std::isfinite(eta_init))
        return fail6(nullptr, GD_EINVAL, "eta and eta_init must be finite and > 0");
    if (!pow2(o.dt_min) || !pow2(o.dt_max) || o.dt_max < o.dt_min || o.dt_max / o.dt_min > 4.0e15)
        return fail6(nullptr, GD_EINVAL, "dt_min and dt_max must be powers of two with dt_min <= dt_max");
    for (int64_t i = 0; i < n; i++) {
        if (!std::isfinite(m[i]) || m[i] < 0) return fail6(nullptr, GD_EINVAL, "masses must be finite and >= 0");
        for (int q = 0; q < 3; q++)
            if (!std::isfinite(x[3 * i + q]) || !std::isfinite(v[3 * i + q]))
                return fail6(nullptr, GD_EINVAL, "positions and velocities must be finite");
    }
    gd_h6 *s = gd_alloc_fails(0) ? nullptr : new (std::nothrow) gd_h6();
    if (!s) return fail6(nullptr, GD_ENOMEM, "host allocation failed");
    s->dev = o.device;
    auto bail = [&](int rc) {
        g_h6_err = s->err;
        gd_h6_free(s);
        return rc;
    };
    cudaError_t e = cudaSetDevice(s->dev);
    if (e != cudaSuccess) return bail(fail6(s, GD_ECUDA, "cudaSetDevice"));
    if (o.stream) {
        s->stream = (cudaStream_t)o.stream;
    } else {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(fail6(s, GD_ECUDA, "cudaStreamCreate"));
        s->own_stream = true;
    }
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k6_force<true>, T6, 0);
    s->grid = std::max(1, sms * std::max(1, occ));
    Dev6 &d = s->d;
    d.n = (int)n;
    d.order = order;
    d.n_iter = n_iter;
    d.dt_min = o.dt_min;
    d.eps2 = eps * eps;
    d.eta = eta;
    d.dtau_max = (long long)(o.dt_max / o.dt_min);
    d.cap = n + 2LL * s->grid + T6;
    auto al = [&](void **p, size_t bytes) {
        if (gd_alloc_fails(1) || cudaMalloc(p, bytes) != cudaSuccess) return false;
        s->allocs.push_back(*p);
        return true;
    };
    const size_t pl = sizeof(double) * 3 * n;
    bool ok = al((void **)&d.m, sizeof(double) * n) && al((void **)&d.x, pl) && al((void **)&d.v, pl) &&
              al((void **)&d.a, pl) && al((void **)&d.j, pl) && al((void **)&d.s, pl) && al((void **)&d.c, pl) &&
              al((void **)&d.xp, pl) && al((void **)&d.vp, pl) && al((void **)&d.ap, pl) &&
              al((void **)&d.tau, sizeof(long long) * n) && al((void **)&d.dtau, sizeof(long long) * n) &&
              al((void **)&d.tnext, sizeof(long long) * n) && al((void **)&d.act, sizeof(int) * n) &&
              al((void **)&d.part, sizeof(double) * NC * d.cap) && al((void **)&d.fsum, sizeof(double) * NC * n) &&
              al((void **)&d.eu, sizeof(double) * n) && al((void **)&d.ek, sizeof(double) * n) &&
              al((void **)&d.ctrl, sizeof(Ctrl6));
    if (!ok) return bail(fail6(s, GD_ENOMEM, "device allocation failed"));
    if (gd_alloc_fails(0) || cudaMallocHost((void **)&s->h_ctrl, sizeof(Ctrl6)) != cudaSuccess ||
        gd_alloc_fails(0) || cudaMallocHost((void **)&s->h_stage, sizeof(double) * 9 * n) != cudaSuccess)
        return bail(fail6(s, GD_ENOMEM, "pinned host allocation failed"));
    std::memset(s->h_ctrl, 0, sizeof(Ctrl6));
    s->h_ctrl->tick_end = LLONG_MAX;
    s->h_ctrl->T_acc = LLONG_MAX;
    e = cudaMemcpyAsync(d.ctrl, s->h_ctrl, sizeof(Ctrl6), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.m, m, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.a, 0, pl, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.j, 0, pl, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.s, 0, pl, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.c, 0, pl, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.tau, 0, sizeof(long long) * n, s->stream);
    if (e != cudaSuccess) return bail(fail6(s, GD_ECUDA, "upload"));
    int rc;
    if ((rc = upload6(s, d.x, x)) || (rc = upload6(s, d.v, v))) return bail(rc);
    // pass 1: force and jerk (predicted accelerations zero), pass 2 (order 6): snap
    const int gi = (int)((n + 255) / 256);
    const int npass = order == 6 ? 2 : 1;
    for (int pass = 1; pass <= npass; pass++) {
        k6_predict_all<<<gi, 256, 0, s->stream>>>(d, 0);
        k6_iota<<<gi, 256, 0, s->stream>>>(d.act, (int)n);
        k6_set_list<<<1, 1, 0, s->stream>>>(d, 0, (int)n);
        force_sum6(s, (int)n);
        k6_take<<<gi, 256, 0, s->stream>>>(d, pass);
        s->launches += 4;
    }
    k6_init_steps<<<gi, 256, 0, s->stream>>>(d, eta_init);
    k6_resync<<<1, 1024, 0, s->stream>>>(d);
    s->launches += 2;
    if (cudaGetLastError() != cudaSuccess) return bail(fail6(s, GD_ECUDA, "initial forces"));
    if ((rc = sync6(s))) return bail(rc);
    // the bookkeeping of the two passes is not a block step
    s->h_ctrl->nblock = 0;
    s->h_ctrl->nsteps = 0;
    s->h_ctrl->interactions = (double)npass * (double)n * (double)n;
    CK6(cudaMemcpyAsync(d.ctrl, s->h_ctrl, sizeof(Ctrl6), cudaMemcpyHostToDevice, s->stream));
    if ((rc = sync6(s))) return bail(rc);
    *out = s;
    return GD_OK;
}

int gd_h6_init(gd_h6 **out, int64_t n, const double *m, const double *x, const double *v, double eps, double eta,
               double eta_init, const gd_opts *opt)
{
    return gd_h6_init_scheme(out, n, m, x, v, eps, eta, eta_init, 6, 1, opt);
}

int gd_h6_step_block(gd_h6 *s, double *t_out, int64_t *nact_out)
{
    int rc = usable6(s);
    if (rc) return rc;
    step6(s);
    CK6(cudaGetLastError());
    if ((rc = sync6(s))) return rc;
    if (t_out) *t_out = (double)s->h_ctrl->T_last * s->d.dt_min;
    if (nact_out) *nact_out = s->h_ctrl->last_nact;
    return GD_OK;
}

int gd_h6_evolve(gd_h6 *s, double t_end)
{
    int rc = usable6(s);
    if (rc) return rc;
    if (!std::isfinite(t_end)) return fail6(s, GD_EINVAL, "t_end must be finite");
    const double q = std::floor(t_end / s->d.dt_min);
    if (q > 9.0e18) return fail6(s, GD_EINVAL, "t_end too large");
    const long long tick_end = (long long)q;
    if (tick_end < s->h_ctrl->T_last) return fail6(s, GD_EINVAL, "t_end is before the current time");
    if ((rc = build_graph6(s))) return rc;
    k6_set_tick_end<<<1, 1, 0, s->stream>>>(s->d.ctrl, tick_end);
    s->launches += 1;
    for (;;) {
        CK6(cudaGraphLaunch(s->graph, s->stream));
        s->launches += per_step6(s) * G6;
        if ((rc = sync6(s))) return rc;
        if (s->h_ctrl->T_cur > tick_end) break;
    }
    k6_set_tick_end<<<1, 1, 0, s->stream>>>(s->d.ctrl, LLONG_MAX);
    s->launches += 1;
    return sync6(s);
}

int gd_h6_replay_step(gd_h6 *s, int64_t tick_next, const int32_t *idx, int64_t nact)
{
    int rc = usable6(s);
    if (rc) return rc;
    const Dev6 &d = s->d;
    if (nact < 1 || nact > d.n || !idx) return fail6(s, GD_EINVAL, "nact must be in [1, n] and idx given");
    for (int64_t k = 0; k < nact; k++)
        if (idx[k] < 0 || idx[k] >= d.n || (k > 0 && idx[k] <= idx[k - 1]))
            return fail6(s, GD_EINVAL, "idx must be ascending, distinct and in range");
    if (tick_next <= 0) return fail6(s, GD_EINVAL, "tick_next must be > 0");
    CK6(cudaMemcpyAsync(d.act, idx, sizeof(int) * nact, cudaMemcpyHostToDevice, s->stream));
    const int gi = (d.n + 255) / 256;
    k6_predict_all<<<gi, 256, 0, s->stream>>>(d, tick_next);
    k6_set_list<<<1, 1, 0, s->stream>>>(d, tick_next, (int)nact);
    s->launches += 2;
    passes6(s);
    k6_resync<<<1, 1024, 0, s->stream>>>(d);
    s->launches += 1;
    CK6(cudaGetLastError());
    return sync6(s);
}

int gd_h6_force(gd_h6 *s, int64_t tick, const int32_t *idx, int64_t nact, double *acc, double *jerk, double *snap)
{
    int rc = usable6(s);
    if (rc) return rc;
    const Dev6 &d = s->d;
    if (nact < 1 || nact > d.n || !idx || !acc || !jerk || !snap)
        return fail6(s, GD_EINVAL, "nact must be in [1, n]; idx, acc, jerk and snap are required");
    for (int64_t k = 0; k < nact; k++)
        if (idx[k] < 0 || idx[k] >= d.n) return fail6(s, GD_EINVAL, "index out of range");
    if (tick < 0) return fail6(s, GD_EINVAL, "tick must be >= 0");
    const long long Tsave = s->h_ctrl->T_cur;
    CK6(cudaMemcpyAsync(d.act, idx, sizeof(int) * nact, cudaMemcpyHostToDevice, s->stream));
    k6_predict_all<<<(d.n + 255) / 256, 256, 0, s->stream>>>(d, tick);
    k6_set_list<<<1, 1, 0, s->stream>>>(d, Tsave, (int)nact);
    force_sum6(s, (int)nact);
    k6_set_list<<<1, 1, 0, s->stream>>>(d, Tsave, 0);
    s->launches += 3;
    CK6(cudaGetLastError());
    if ((rc = download6(s, acc, d.fsum, d.n, (int)nact))) return rc;
    if ((rc = download6(s, jerk, d.fsum + 3LL * d.n, d.n, (int)nact))) return rc;
    if ((rc = download6(s, snap, d.fsum + 6LL * d.n, d.n, (int)nact))) return rc;
    return sync6(s);
}

int gd_h6_energy(gd_h6 *s, double *K, double *U)
{
    int rc = usable6(s);
    if (rc) return rc;
    if (!K || !U) return fail6(s, GD_EINVAL, "K and U are required");
    const Dev6 &d = s->d;
    k6_predict_all<<<(d.n + 255) / 256, 256, 0, s->stream>>>(d, s->h_ctrl->T_last);
    k6_energy_terms<<<(d.n + T6 - 1) / T6, T6, 0, s->stream>>>(d);
    s->launches += 2;
    CK6(cudaGetLastError());
    CK6(cudaMemcpyAsync(s->h_stage, d.ek, sizeof(double) * d.n, cudaMemcpyDeviceToHost, s->stream));
    CK6(cudaMemcpyAsync(s->h_stage + d.n, d.eu, sizeof(double) * d.n, cudaMemcpyDeviceToHost, s->stream));
    CK6(cudaStreamSynchronize(s->stream));
    double k = 0.0, u = 0.0;
    for (int i = 0; i < d.n; i++) {
        k += s->h_stage[i];
        u += s->h_stage[d.n + i];
    }
    *K = k;
    *U = u;
    return GD_OK;
}

int gd_h6_get_state(gd_h6 *s, double *x, double *v, double *a, double *jerk, double *snap, double *crackle,
                    int64_t *tau, int64_t *dtau)
{
    int rc = usable6(s);
    if (rc) return rc;
    const Dev6 &d = s->d;
    const double *src[6] = {d.x, d.v, d.a, d.j, d.s, d.c};
    double *dst[6] = {x, v, a, jerk, snap, crackle};
    for (int q = 0; q < 6; q++)
        if (dst[q] && (rc = download6(s, dst[q], src[q], d.n, d.n))) return rc;
    if (tau) CK6(cudaMemcpy(tau, d.tau, sizeof(long long) * d.n, cudaMemcpyDeviceToHost));
    if (dtau) CK6(cudaMemcpy(dtau, d.dtau, sizeof(long long) * d.n, cudaMemcpyDeviceToHost));
    return GD_OK;
}

int gd_h6_get_stats(gd_h6 *s, gd_stats *st)
{
    int rc = usable6(s);
    if (rc) return rc;
    if (!st) return fail6(s, GD_EINVAL, "st is required");
    if ((rc = sync6(s))) return rc;
    std::memset(st, 0, sizeof(*st));
    st->tick = s->h_ctrl->T_last;
    st->block_steps = s->h_ctrl->nblock;
    st->particle_steps = s->h_ctrl->nsteps;
    st->interactions = s->h_ctrl->interactions;
    st->last_nact = s->h_ctrl->last_nact;
    st->kernel_launches = s->launches;
    return GD_OK;
}

}  // extern "C"
