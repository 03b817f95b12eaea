// kernels.cuh -- device code of the GB300 Hermite-4 block-time-step integrator
// (GraviDy, arXiv 1702.00440).  Included once, by gravidy.cu.
//
// One block step (Sec. 2.4 steps 5-7) is three kernels and no host round trip:
//   k_select_predict  predict every particle to the block time (step 7a) and list
//                     the active ones (step 5), each chunk of particles claiming
//                     its place with one atomic add; start the minimum of the
//                     next block time over the inactive ones.
//   k_force_*         force and jerk of the active set against all N predicted
//                     particles (step 7c, Sec. 2.5): a persistent kernel over
//                     (i-tile x j-chunk) work items; the j-range is split when the
//                     active set is small, and the last CTA to finish an i-tile
//                     sums its partials (step 7c-iii).
//   k_correct         correct (7d), take Aarseth's step (Sec. 3.2), quantise it to
//                     the block scheme, keep the new force (step 6), and finish the
//                     minimum that gives the next block time.
//
// Cost model that shapes the code: on this GPU an FP64 warp instruction holds an
// SMSP for about 78 cycles whether 1 or 32 lanes are active, while an FP32 one
// issues every cycle.  So the mixed path keeps positions and velocities as
// double-single values and predicts, corrects and chooses steps with FP32
// instructions (error-free transformations where the sums need more than 24
// bits), keeps its force sums in FP32 with compensated (two-sum) accumulation, and
// uses FP64 only for the energy totals and the host-facing conversions; the FP64
// path does everything in FP64, with every FP64 instruction working on as many
// particles or components as possible.
#pragma once

#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

namespace gdk {

// ---------------------------------------------------------------- constants

constexpr int FT = 128;                      // force kernel threads per CTA
constexpr int BJ = 128;                      // j-tile, and padding granule of the j-arrays
constexpr int BJ64 = 64;                     // FP64 i-parallel mode j-tile
constexpr int ITILE_A_MIX = 2 * FT;          // mixed i-parallel: 2 active particles per thread
constexpr int ITILE_A_64 = FT;               // FP64 i-parallel: 1 per thread
constexpr int ITILE_B_MIX = 2 * (FT / 32);   // mixed warp mode: 2 per warp, lanes split j
constexpr int ITILE_B_64 = FT / 32;          // FP64 warp mode: 1 per warp
constexpr int FOLD_B = 16;                   // warp mode: j-iterations per lane between folds
constexpr int ST = 128;                      // select/predict threads per CTA (= particles per chunk)
constexpr int CT = 128;                      // corrector threads per CTA
constexpr int ET = 128;                      // energy threads per CTA
constexpr int SPIN_LIMIT = 1 << 22;          // bounded device waits
constexpr float PAD_FAR_F = 1.0e18f;
constexpr double PAD_FAR_D = 1.0e30;

// status codes written to the device flag (same values as gd_status)
constexpr int ST_EINVAL = -1, ST_ENONFINITE = -4, ST_ETIMEOUT = -5, ST_ESTATE = -6;

// ---------------------------------------------------------------- control block

struct Ctrl {
    long long T_cur;       // block time of the next step (ticks)
    long long T_acc;       // running minimum of next times, for the step after it
    long long T_acc2[2];   // the same for the fused kernel, by step parity
    long long T_last;      // block time of the last finished step
    long long tick_end;    // steps whose block time is above this are skipped
    long long nblock;      // block steps
    long long nsteps;      // particle steps
    double interactions;   // sum of nact * n
    double K, U;           // energy results
    int nact;              // active count of the current step
    int last_nact;
    unsigned int epoch;    // step counter (parity slots of the fused kernel, look-back tag of the ensemble)
    unsigned int done;     // finished-CTA counter of k_correct
    int err;               // first device-side fault (gd_status), 0 = none
    unsigned sel_gen;      // launches of the ordered select kernel so far (mod 2^31), see k_select_predict
    unsigned long long ph_ns[3];  // fused kernel, CTA 0's clock: select, force, correct phases
    unsigned long long sel_acc;   // select: arrived chunks (high word), active count (low word); 0 between steps
    unsigned long long cl_cyc[12];  // small-step cluster, CTA 0's SM cycles per phase (see k_cluster_steps)
};

__device__ __forceinline__ void set_err(Ctrl *c, int code) { atomicCAS(&c->err, 0, code); }

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------- tuning table

// Force work decomposition, chosen by the autotuner (or defaults).
struct Tune {
    int mode_cut;             // N_act >= mode_cut: i-parallel mode, else warp mode
    int jchunk_min;           // smallest j-chunk of a split (multiple of BJ)
    int items_x4;             // target work items = grid * items_x4 / 4
    short s_fixed[32];        // per floor(log2 N_act): > 0 forces the j-split factor
    signed char mode_b[32];   // per floor(log2 N_act): 0 / 1 / 2 forces the mode (2: warp mode whose
                              // j-split sums are left to the corrector), -1 = mode_cut
};

// ---------------------------------------------------------------- device state

struct Dev {
    int n, npad;
    double dt_min, inv_dt_min, dt_min2;
    long long dtau_max;
    double eta;
    double eps2;
    float eps2f;
    float dt_min_f, inv_dt_min_f, eta_f;  // FP32 copies (dt_min is a power of two: exact)
    int tsym;                 // corrector: 0 the Hermite scheme's, 1 the time-symmetric form
    int n_iter;               // evaluation-correction passes per block step (P(EC)^n; 1 = PEC)
    int pn_terms;             // post-Newtonian terms of the pair (pn_p, pn_q): 0 none, bit 1 1PN, bit 4 2.5PN
    int pn_p, pn_q;
    double pn_c;              // speed of light in code units
    // FP64 state at each particle's own time, structure of arrays (plane c at +c*n);
    // on the mixed path these planes only stage the state in and out (k_state_to_ds,
    // k_state_from_ds)
    double *x, *v, *a, *jk, *m;
    // mixed-path state: x and v double-single, planes c = hi x, y, z and 3 + c = lo
    // (canonical: hi = the float nearest the value, hi + lo an FP64 number, see
    // ds_canon); a and jerk FP32 (the mixed forces carry FP32 accuracy); masses FP32
    float *xs, *vs, *af, *jf, *mf;
    long long *tau, *dtau, *tnext;
    // predicted j-records, mixed: A = (x_hi, y_hi, z_hi, m), B = (x_lo, y_lo, z_lo, vx),
    // C = (vy, vz); padded to npad with massless far-away particles
    float4 *jA, *jB;
    float2 *jC;
    // predicted j-records, FP64: 7 planes of npad (x, y, z, vx, vy, vz, m)
    double *pd;
    int *act;                 // active list
    void *part;               // j-split partials (float mixed, double FP64), (s*6 + c)*nact + k
    long long cap;            // partial capacity (entries per component)
    double *fsum;             // summed force of active slot k: fsum[c*n + k], c < 3 a, c >= 3 jerk
                              // (FP64 path; the mixed path stores floats, see fsum_f)
    unsigned int *tilecnt;    // per i-tile arrival counters (zero between launches)
    unsigned long long *status;  // ensemble look-back words, one per chunk of ST particles
    unsigned long long *selstat; // ordered select: (generation, active count) of each select CTA
    double *eu, *ek;          // per-particle energy terms
    int *nact_hist;           // nact of each step slot of a captured graph
    unsigned int *bar;        // grid-barrier counters of the fused kernel (see grid_sync)
    Ctrl *ctrl;
};

// ---------------------------------------------------------------- force plan

struct Plan {
    int mode;     // 0 = i-parallel, 1 = warp j-parallel
    int late;     // the j-split partials may be left to the corrector (i-parallel, or warp mode tuned 2)
    int itile;    // active particles per work item
    int itiles;
    int S;        // j-split factor
    int chunk;    // j per split (multiple of BJ)
    long long items;
};

__host__ __device__ inline int ilog2_floor(int x)
{
    int l = 0;
    while (x > 1) {
        x >>= 1;
        l++;
    }
    return l;
}

__host__ __device__ inline Plan make_plan(int nact, int npad, int grid, const Tune &tn, bool mixed, long long cap)
{
    Plan p;
    const int b = nact > 0 ? ilog2_floor(nact) : 0;
    const int mb = tn.mode_b[b < 32 ? b : 31];
    p.mode = mb >= 0 ? (mb == 0 ? 0 : 1) : (nact >= tn.mode_cut ? 0 : 1);
    p.late = p.mode == 0 || mb == 2;
    p.itile = p.mode == 0 ? (mixed ? ITILE_A_MIX : ITILE_A_64) : (mixed ? ITILE_B_MIX : ITILE_B_64);
    p.itiles = (nact + p.itile - 1) / p.itile;
    if (p.itiles < 1) p.itiles = 1;
    long long S = tn.s_fixed[b < 32 ? b : 31];
    if (S <= 0) {
        const long long target = (long long)grid * tn.items_x4 / 4;
        S = (target + p.itiles - 1) / p.itiles;
    }
    long long smax = npad / (tn.jchunk_min > BJ ? tn.jchunk_min : BJ);
    if (smax < 1) smax = 1;
    if (S > smax) S = smax;
    if (S < 1) S = 1;
    if (nact > 0 && S * (long long)nact > cap) S = cap / nact;
    if (S < 1) S = 1;
    const int tiles = npad / BJ;
    const int tpc = (int)((tiles + S - 1) / S);
    p.chunk = tpc * BJ;
    p.S = (tiles + tpc - 1) / tpc;
    p.items = (long long)p.itiles * p.S;
    return p;
}

// ---------------------------------------------------------------- small helpers

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned long long lb_pack(unsigned epoch, unsigned flag, unsigned val)
{
    return ((unsigned long long)(epoch & 0x3FFFFFFFu) << 34) | ((unsigned long long)flag << 32) | val;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p)
{
    return *(const volatile unsigned long long *)p;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the previous kernel in the stream still runs;
// pdl_wait() returns once that kernel has completed and its writes are visible
// (a no-op for an ordinary launch); pdl_trigger() lets the next such kernel start.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Loads of data that another CTA may have written earlier in the same launch go
// through L2 (the per-SM L1 is not coherent across SMs): ldc always, ldx<COH> in the
// fused kernel (COH = true); between kernels ordinary cached loads suffice.
template <class T>
__device__ __forceinline__ T ldc(const T *p)
{
    return __ldcg(p);
}

template <bool COH, class T>
__device__ __forceinline__ T ldx(const T *p)
{
    if (COH) return __ldcg(p);
    return *p;
}

// Asynchronous global -> shared copies of 16 bytes through L2 (cp.async.cg: no L1,
// so also coherent in the fused kernel), in commit groups; wait_group<N> returns once
// at most N of this thread's groups are still in flight.
__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ long long warp_min_ll(long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Compensated FP32 accumulator: h + l carries the running sum to about twice the
// float precision; each add is Knuth's two-sum of h and the addend, with the
// rounding error collected in l.
struct DS {
    float h, l;
    __device__ __forceinline__ void zero()
    {
        h = 0.f;
        l = 0.f;
    }
    __device__ __forceinline__ void add(float f)
    {
        const float s = h + f;
        const float bb = s - h;
        const float e = (h - (s - bb)) + (f - bb);
        l += e;
        h = s;
    }
    __device__ __forceinline__ float as_float() const { return h + l; }
    __device__ __forceinline__ double as_double() const { return (double)h + (double)l; }
};

// ---------------------------------------------------------------- double-single values
//
// The mixed path keeps positions and velocities as unevaluated sums h + l of two
// floats (about 48 significant bits) and does its updates with FP32 instructions:
// on this GPU one FP64 warp instruction costs as much issue time as about 78 FP32
// ones.  Error-free transformations: Knuth's two-sum (any magnitudes) and
// Dekker's fast two-sum (|a| >= |b|); products by an exact power of two are exact.
// Explicit __fadd_rn / __fmul_rn keep the compiler from contracting them.

struct F2 {
    float h, l;
};

__device__ __forceinline__ F2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    const float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
    return F2{s, e};
}

__device__ __forceinline__ F2 fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return F2{s, __fadd_rn(b, -__fadd_rn(s, -a))};
}

// (a.h + a.l) + b, normalised (h = the float nearest the sum)
__device__ __forceinline__ F2 ds_add_f(F2 a, float b)
{
    const F2 s = two_sum(a.h, b);
    return fast_two_sum(s.h, __fadd_rn(s.l, a.l));
}

// Canonical form of a normalised double-single value: lo rounded to a multiple of
// 2^(E - 51), E the binary exponent of hi, then renormalised.  The value is then
// an FP64 number (even if renormalising moves hi to the next binade), so FP64 ->
// double-single -> FP64 conversions are exact and a state read out and written
// back continues bit for bit.  Values below 2^-46 (and zero) are left as they are.
__device__ __forceinline__ F2 ds_canon(F2 a)
{
    const int eb = (int)((__float_as_uint(a.h) >> 23) & 0xFFu);  // biased exponent of hi
    if (eb < 81 || eb > 250) return a;
    const float g = __uint_as_float((unsigned)(eb - 51) << 23);    // 2^(E - 51)
    const float ig = __uint_as_float((unsigned)(305 - eb) << 23);  // 2^(51 - E)
    const float lq = __fmul_rn(rintf(__fmul_rn(a.l, ig)), g);
    return fast_two_sum(a.h, lq);
}

// FP64 -> canonical double-single (state upload) and back (exact for canonical values)
__device__ __forceinline__ F2 ds_from_double(double x)
{
    const float h = __double2float_rn(x);
    const float l = __double2float_rn(x - (double)h);
    return ds_canon(fast_two_sum(h, l));
}

__device__ __forceinline__ double ds_to_double(F2 a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ F2 ld_ds(const float *p, int n, int c, int i) { return F2{p[c * n + i], p[(3 + c) * n + i]}; }

template <bool COH>
__device__ __forceinline__ F2 ldx_ds(const float *p, int n, int c, int i)
{
    if (COH) return F2{__ldcg(p + c * n + i), __ldcg(p + (3 + c) * n + i)};
    return F2{p[c * n + i], p[(3 + c) * n + i]};
}

__device__ __forceinline__ void st_ds(float *p, int n, int c, int i, F2 a)
{
    p[c * n + i] = a.h;
    p[(3 + c) * n + i] = a.l;
}

// Step length in FP32 from ticks: exact for dtick < 2^24 (every step the
// integrator takes; dtau_max is at most 2^20 ticks here), with 1/dt exact when
// dtick is a power of two (always, in free-running steps).
__device__ __forceinline__ void step_f(const Dev &d, long long dtick, float &dt, float &idt)
{
    dt = __fmul_rn((float)dtick, d.dt_min_f);
    if (dtick > 0 && (dtick & (dtick - 1)) == 0) {
        const int e = 63 - __clzll(dtick);
        idt = __fmul_rn(d.inv_dt_min_f, __uint_as_float((unsigned)(127 - e) << 23));
    } else {
        idt = 1.0f / dt;
    }
}

// Taylor prediction (Sec. 2.4 step 7a) of one component on the mixed path:
//   xp = x + dt v + dt^2/2 a + dt^3/6 jerk,   vp = v + dt a + dt^2/2 jerk.
// dt v is formed exactly (dt * v.h as a product and its FMA residual); the a and
// jerk terms are FP32 like the forces they come from; the sum is double-single.
__device__ __forceinline__ F2 ds_pred_x(F2 x0, F2 v0, float a0, float j0, float dt, float h2, float h3)
{
    const float p = __fmul_rn(dt, v0.h);
    const float pe = fmaf(dt, v0.h, -p);
    const float small = fmaf(h3, j0, __fmul_rn(h2, a0));
    const F2 s = two_sum(x0.h, p);
    const float e = __fadd_rn(__fadd_rn(__fadd_rn(s.l, x0.l), fmaf(dt, v0.l, pe)), small);
    return two_sum(s.h, e);
}

__device__ __forceinline__ F2 ds_pred_v(F2 v0, float a0, float j0, float dt, float h2)
{
    const float t = fmaf(h2, j0, __fmul_rn(dt, a0));
    const F2 s = two_sum(v0.h, t);
    return two_sum(s.h, __fadd_rn(s.l, v0.l));
}

// The predicted velocity as the j-record's FP32 value: v.h + (v.l + dt a + dt^2/2 jerk).
__device__ __forceinline__ float ds_pred_v_rec(F2 v0, float a0, float j0, float dt, float h2)
{
    return __fadd_rn(v0.h, fmaf(h2, j0, fmaf(dt, a0, v0.l)));
}

// Predicts particle i to T on the mixed path and stores its j-record.
template <bool COH>
__device__ __forceinline__ void predict_store_ds(const Dev &d, int i, long long dtick)
{
    const int n = d.n;
    float dt, idt;
    step_f(d, dtick, dt, idt);
    const float h2 = __fmul_rn(0.5f, __fmul_rn(dt, dt));
    const float h3 = __fmul_rn(__fmul_rn(__fmul_rn(dt, dt), dt), 1.0f / 6.0f);
    F2 xp[3];
    float vp[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const F2 x0 = ldx_ds<COH>(d.xs, n, c, i), v0 = ldx_ds<COH>(d.vs, n, c, i);
        const float a0 = ldx<COH>(&d.af[c * n + i]), j0 = ldx<COH>(&d.jf[c * n + i]);
        xp[c] = ds_pred_x(x0, v0, a0, j0, dt, h2, h3);
        vp[c] = ds_pred_v_rec(v0, a0, j0, dt, h2);
    }
    d.jA[i] = make_float4(xp[0].h, xp[1].h, xp[2].h, d.mf[i]);
    d.jB[i] = make_float4(xp[0].l, xp[1].l, xp[2].l, vp[0]);
    d.jC[i] = make_float2(vp[1], vp[2]);
}

// Taylor prediction of particle i over dt (Sec. 2.4 step 7a), FP64.
template <bool COH>
__device__ __forceinline__ void predict64(const Dev &d, int i, double dt, double xp[3], double vp[3])
{
    const int n = d.n;
    const double h2 = 0.5 * dt * dt, h3 = dt * dt * dt * (1.0 / 6.0);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const double x0 = ldx<COH>(&d.x[c * n + i]), v0 = ldx<COH>(&d.v[c * n + i]),
                     a0 = ldx<COH>(&d.a[c * n + i]), j0 = ldx<COH>(&d.jk[c * n + i]);
        xp[c] = fma(j0, h3, fma(a0, h2, fma(v0, dt, x0)));
        vp[c] = fma(j0, h2, fma(a0, dt, v0));
    }
}

// The same FP64 prediction from the mixed path's state (hooks and energy).
__device__ __forceinline__ void predict64_ds(const Dev &d, int i, double dt, double xp[3], double vp[3])
{
    const int n = d.n;
    const double h2 = 0.5 * dt * dt, h3 = dt * dt * dt * (1.0 / 6.0);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const double x0 = ds_to_double(ld_ds(d.xs, n, c, i)), v0 = ds_to_double(ld_ds(d.vs, n, c, i));
        const double a0 = d.af[c * n + i], j0 = d.jf[c * n + i];
        xp[c] = fma(j0, h3, fma(a0, h2, fma(v0, dt, x0)));
        vp[c] = fma(j0, h2, fma(a0, dt, v0));
    }
}

// Store the predicted particle as the record the force kernel reads.
template <bool MIXED>
__device__ __forceinline__ void store_jrec(const Dev &d, int i, const double xp[3], const double vp[3], double mi)
{
    if (MIXED) {
        const float h0 = __double2float_rn(xp[0]), h1 = __double2float_rn(xp[1]), h2 = __double2float_rn(xp[2]);
        const float l0 = __double2float_rn(xp[0] - (double)h0);
        const float l1 = __double2float_rn(xp[1] - (double)h1);
        const float l2 = __double2float_rn(xp[2] - (double)h2);
        d.jA[i] = make_float4(h0, h1, h2, __double2float_rn(mi));
        d.jB[i] = make_float4(l0, l1, l2, __double2float_rn(vp[0]));
        d.jC[i] = make_float2(__double2float_rn(vp[1]), __double2float_rn(vp[2]));
    } else {
        const int np = d.npad;
        d.pd[0 * np + i] = xp[0];
        d.pd[1 * np + i] = xp[1];
        d.pd[2 * np + i] = xp[2];
        d.pd[3 * np + i] = vp[0];
        d.pd[4 * np + i] = vp[1];
        d.pd[5 * np + i] = vp[2];
        d.pd[6 * np + i] = mi;
    }
}

// ---------------------------------------------------------------- kernel: select + predict

// The fused kernel's selection: predicts every particle to T and writes the list
// of the particles whose next time equals T (Sec. 2.4 steps 5-6).  Each chunk of
// ST particles claims its place in the list with one 64-bit atomic add on
// ctrl->sel_acc: the low word counts active particles (the returned value is the
// chunk's offset), the high word counts arrived chunks, so the chunk that arrives
// last knows the total, publishes it as ctrl->nact and clears the word for the
// next step.  This list is in arrival order (k_select_predict writes the ascending
// one): every later per-particle computation (force sums over j in a fixed order,
// correction, step choice) is independent of a particle's slot, so the results do
// not depend on the order.  `slot` >= 0 records nact in nact_hist[slot].
template <bool MIXED, bool COH>
__device__ void phase_select(const Dev &d, long long T, int slot, int nchunks, unsigned long long *Tacc)
{
    Ctrl *ctrl = d.ctrl;
    __shared__ unsigned s_base;
    __shared__ unsigned s_wcnt[ST / 32];
    __shared__ long long s_wmin[ST / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long mn_all = LLONG_MAX;
    for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const int i = chunk * ST + threadIdx.x;
        bool act = false;
        if (i < d.n) {
            const long long tn = ldx<COH>(&d.tnext[i]);
            act = (tn == T);
            if (!act) mn_all = tn < mn_all ? tn : mn_all;
            const long long dtick = T - ldx<COH>(&d.tau[i]);
            if (MIXED) {
                predict_store_ds<COH>(d, i, dtick);
            } else {
                double xp[3], vp[3];
                predict64<COH>(d, i, (double)dtick * d.dt_min, xp, vp);
                store_jrec<false>(d, i, xp, vp, d.m[i]);
            }
        }
        const unsigned ballot = __ballot_sync(0xffffffffu, act);
        if (lane == 0) s_wcnt[warp] = __popc(ballot);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned tot = 0;
#pragma unroll
            for (int w = 0; w < ST / 32; w++) {
                const unsigned c = s_wcnt[w];
                s_wcnt[w] = tot;  // exclusive offset of warp w within the chunk
                tot += c;
            }
            const unsigned long long old = atomicAdd(&ctrl->sel_acc, (1ull << 32) | (unsigned long long)tot);
            s_base = (unsigned)old;
            if ((unsigned)(old >> 32) == (unsigned)(nchunks - 1)) {
                // every other chunk has added its count: the total is known
                unsigned long long na = (unsigned long long)(unsigned)old + tot;
                if (na > (unsigned long long)d.n) {
                    set_err(ctrl, ST_ETIMEOUT);
                    na = 0;
                }
                ctrl->nact = (int)na;
                if (slot >= 0) d.nact_hist[slot] = (int)na;
                atomicExch(&ctrl->sel_acc, 0ull);
            }
        }
        __syncthreads();
        if (act) {
            const unsigned pos = s_base + s_wcnt[warp] + __popc(ballot & ((1u << lane) - 1u));
            if (pos < (unsigned)d.n) d.act[pos] = i;
        }
        __syncthreads();
    }
    // minimum next time of the inactive particles -> next block time candidate
    long long mn = warp_min_ll(mn_all);
    if (lane == 0) s_wmin[warp] = mn;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < ST / 32; w++) mn = s_wmin[w] < mn ? s_wmin[w] : mn;
        if (mn != LLONG_MAX) atomicMin(Tacc, (unsigned long long)mn);
    }
    __syncthreads();
}

// The same prediction and selection with the active list in ascending particle
// order, as the oracle lists it (the fused kernel keeps phase_select's arrival
// order).  The G CTAs of the grid are co-resident (G is at most the SMs times the
// kernel's occupancy) and CTA b owns the contiguous chunks [b R, (b + 1) R), R =
// ceil(nchunks / G):
//   pass 1  predict the CTA's particles, count its active ones;
//   publish the count in selstat[b], tagged with this launch's generation;
//   sum the counts of CTAs 0 .. b-1 (each read with a bounded wait for its tag):
//           the CTA's offset in the list;
//   pass 2  chunk by chunk, warp ballots and a scan of the four warp counts give
//           each active particle its place, in particle order.
// CTA G - 1, whose wait saw every other CTA's count (so every CTA has read the
// generation by then), publishes N_act and advances the generation.  A wait that
// runs out records GD_ETIMEOUT and counts the missing CTA as empty.
template <bool MIXED>
__global__ void __launch_bounds__(ST) k_select_predict(Dev d, int slot, int nchunks)
{
    pdl_trigger();
    pdl_wait();
    Ctrl *ctrl = d.ctrl;
    const long long T = ctrl->T_cur;
    if (T > ctrl->tick_end) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctrl->nact = 0;
            if (slot >= 0) d.nact_hist[slot] = 0;
        }
        return;
    }
    __shared__ unsigned s_wcnt[ST / 32];
    __shared__ unsigned s_part[ST / 32];
    __shared__ long long s_wmin[ST / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned tag = (ctrl->sel_gen & 0x7FFFFFFFu) + 1u;  // never 0 (the words start at 0)
    const int G = gridDim.x, b = blockIdx.x;
    const int R = (nchunks + G - 1) / G;
    const int c0 = min(b * R, nchunks), c1 = min(c0 + R, nchunks);
    // pass 1: predict, count (lane 0 of each warp keeps its warp's running count)
    long long mn_all = LLONG_MAX;
    unsigned wc = 0;
    for (int ch = c0; ch < c1; ch++) {
        const int i = ch * ST + threadIdx.x;
        bool act = false;
        if (i < d.n) {
            const long long tn = d.tnext[i];
            act = (tn == T);
            if (!act) mn_all = tn < mn_all ? tn : mn_all;
            const long long dtick = T - d.tau[i];
            if (MIXED) {
                predict_store_ds<false>(d, i, dtick);
            } else {
                double xp[3], vp[3];
                predict64<false>(d, i, (double)dtick * d.dt_min, xp, vp);
                store_jrec<false>(d, i, xp, vp, d.m[i]);
            }
        }
        wc += __popc(__ballot_sync(0xffffffffu, act));
    }
    if (lane == 0) s_wcnt[warp] = wc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
#pragma unroll
        for (int w = 0; w < ST / 32; w++) tot += s_wcnt[w];
        __threadfence();
        atomicExch(&d.selstat[b], ((unsigned long long)tag << 32) | tot);
    }
    // this CTA's offset: the counts of CTAs 0 .. b-1
    unsigned part = 0;
    for (int q = threadIdx.x; q < b; q += ST) {
        unsigned long long w = ld_volatile_u64(&d.selstat[q]);
        int spins = 0;
        while ((unsigned)(w >> 32) != tag) {
            if (++spins > SPIN_LIMIT) {
                set_err(ctrl, ST_ETIMEOUT);
                w = (unsigned long long)tag << 32;
                break;
            }
            __nanosleep(32);
            w = ld_volatile_u64(&d.selstat[q]);
        }
        part += (unsigned)w;
    }
    __threadfence();
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) s_part[warp] = part;
    __syncthreads();
    unsigned base = 0;
#pragma unroll
    for (int w = 0; w < ST / 32; w++) base += s_part[w];
    // pass 2: places in particle order
    for (int ch = c0; ch < c1; ch++) {
        const int i = ch * ST + threadIdx.x;
        const bool act = i < d.n && d.tnext[i] == T;
        const unsigned ballot = __ballot_sync(0xffffffffu, act);
        __syncthreads();  // the previous chunk's reads of s_wcnt are done
        if (lane == 0) s_wcnt[warp] = __popc(ballot);
        __syncthreads();
        unsigned off = base, tot = 0;
#pragma unroll
        for (int w = 0; w < ST / 32; w++) {
            const unsigned cw = s_wcnt[w];
            off += w < warp ? cw : 0u;
            tot += cw;
        }
        if (act) {
            const unsigned pos = off + __popc(ballot & ((1u << lane) - 1u));
            if (pos < (unsigned)d.n) d.act[pos] = i;
        }
        base += tot;
    }
    if (b == G - 1 && threadIdx.x == 0) {
        unsigned long long na = base;
        if (na > (unsigned long long)d.n) {
            set_err(ctrl, ST_ETIMEOUT);
            na = 0;
        }
        ctrl->nact = (int)na;
        if (slot >= 0) d.nact_hist[slot] = (int)na;
        ctrl->sel_gen = tag & 0x7FFFFFFFu;
    }
    // minimum next time of the inactive particles -> next block time candidate
    long long mn = warp_min_ll(mn_all);
    if (lane == 0) s_wmin[warp] = mn;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < ST / 32; w++) mn = s_wmin[w] < mn ? s_wmin[w] : mn;
        if (mn != LLONG_MAX) atomicMin((unsigned long long *)&ctrl->T_acc, (unsigned long long)mn);
    }
}

// Predict all particles to `tick` (no selection): the hooks, gd_energy and the
// initial forces.  DS: the state is the mixed path's; RECS: mixed j-records (else
// the FP64 planes pd).
template <bool DS_STATE, bool RECS>
__global__ void k_predict_all(Dev d, long long tick)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const long long dtick = tick - d.tau[i];
    if (DS_STATE && RECS) {
        predict_store_ds<false>(d, i, dtick);
        return;
    }
    const double dt = (double)dtick * d.dt_min;
    double xp[3], vp[3];
    if (DS_STATE)
        predict64_ds(d, i, dt, xp, vp);
    else
        predict64<false>(d, i, dt, xp, vp);
    store_jrec<RECS>(d, i, xp, vp, d.m[i]);
}

// Mixed path: FP64 staging planes -> state (x, v double-single canonical, a and
// jerk FP32), and back.
__global__ void k_state_to_ds(Dev d, int with_aj)
{
    const int n = d.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < 3; c++) {
        st_ds(d.xs, n, c, i, ds_from_double(d.x[c * n + i]));
        st_ds(d.vs, n, c, i, ds_from_double(d.v[c * n + i]));
        if (with_aj) {
            d.af[c * n + i] = __double2float_rn(d.a[c * n + i]);
            d.jf[c * n + i] = __double2float_rn(d.jk[c * n + i]);
        }
    }
    d.mf[i] = __double2float_rn(d.m[i]);
}

// Mixed path: the FP32 summed forces of the first rows slots, widened into FP64
// planes dst[c * rows + k] (the force hook's download).
__global__ void k_fsum_widen(Dev d, int rows, double *dst)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= rows) return;
    const float *fs = (const float *)d.fsum;
    for (int c = 0; c < 6; c++) dst[(long long)c * rows + k] = (double)fs[(long long)c * d.n + k];
}

// Mixed path: the predicted j-records widened to FP64 planes dst (stride npad):
// x = hi + lo (exact), v the record's FP32 value (the predictor hook's download).
__global__ void k_jrec_widen(Dev d, double *dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int np = d.npad;
    const float4 A = d.jA[i], B = d.jB[i];
    const float2 C = d.jC[i];
    dst[0 * np + i] = (double)A.x + (double)B.x;
    dst[1 * np + i] = (double)A.y + (double)B.y;
    dst[2 * np + i] = (double)A.z + (double)B.z;
    dst[3 * np + i] = (double)B.w;
    dst[4 * np + i] = (double)C.x;
    dst[5 * np + i] = (double)C.y;
}

__global__ void k_state_from_ds(Dev d)
{
    const int n = d.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < 3; c++) {
        d.x[c * n + i] = ds_to_double(ld_ds(d.xs, n, c, i));
        d.v[c * n + i] = ds_to_double(ld_ds(d.vs, n, c, i));
        d.a[c * n + i] = (double)d.af[c * n + i];
        d.jk[c * n + i] = (double)d.jf[c * n + i];
    }
}

// Padding records: massless particles far away, so the inner loops need no tail test.
__global__ void k_init_pads(Dev d)
{
    const int i = d.n + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.npad) return;
    d.jA[i] = make_float4(PAD_FAR_F, PAD_FAR_F, PAD_FAR_F, 0.f);
    d.jB[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    d.jC[i] = make_float2(0.f, 0.f);
    const int np = d.npad;
    d.pd[0 * np + i] = PAD_FAR_D;
    d.pd[1 * np + i] = PAD_FAR_D;
    d.pd[2 * np + i] = PAD_FAR_D;
    d.pd[3 * np + i] = 0.0;
    d.pd[4 * np + i] = 0.0;
    d.pd[5 * np + i] = 0.0;
    d.pd[6 * np + i] = 0.0;
}

// ---------------------------------------------------------------- pair interactions

// One softened pair term (Sec. 2.4, softened Eq. 1, and its time derivative) in FP32
// on double-single positions: r = x_j - x_i from the hi and lo parts separately, so
// the difference keeps the bits of the FP64 positions.
//   a += m r / s^3,   jerk += m (v - 3 (r.v) r / s^2) / s^3,   s^2 = r^2 + eps^2
// m / s^3 takes one Newton step on rsqrt.approx (y^3 (1 + 3/2 (1 - s^2 y^2)), the
// residual from one FMA): without it the approximation's error, common to all six
// components of a term, sets the per-particle jerk error of particles whose terms
// cancel (measured p99 of |d jerk| / |jerk| 1.0-1.2e-6 without, 0.65-1.0e-6 with).
template <bool SOFT>
__device__ __forceinline__ void pair_mixed(const float4 A, const float4 B, const float2 C, const float xh,
                                           const float yh, const float zh, const float xl, const float yl,
                                           const float zl, const float vx, const float vy, const float vz,
                                           const float eps2, float f[6])
{
    const float dx = (A.x - xh) + (B.x - xl);
    const float dy = (A.y - yh) + (B.y - yl);
    const float dz = (A.z - zh) + (B.z - zl);
    const float dvx = B.w - vx, dvy = C.x - vy, dvz = C.y - vz;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    const float rv = fmaf(dx, dvx, fmaf(dy, dvy, dz * dvz));
    float rinv = rsqrt_approx(r2);
    if (!SOFT) rinv = r2 > 0.f ? rinv : 0.f;
    const float rinv2 = rinv * rinv;
    const float e = fmaf(-r2, rinv2, 1.0f);
    const float mr3 = fmaf(A.w * rinv * rinv2, 1.5f * e, A.w * rinv * rinv2);
    const float b = -3.f * rv * rinv2;
    f[0] = fmaf(mr3, dx, f[0]);
    f[1] = fmaf(mr3, dy, f[1]);
    f[2] = fmaf(mr3, dz, f[2]);
    f[3] = fmaf(mr3, fmaf(b, dx, dvx), f[3]);
    f[4] = fmaf(mr3, fmaf(b, dy, dvy), f[4]);
    f[5] = fmaf(mr3, fmaf(b, dz, dvz), f[5]);
}

template <bool SOFT>
__device__ __forceinline__ void pair_fp64(const double xj, const double yj, const double zj, const double vxj,
                                          const double vyj, const double vzj, const double mj, const double xi,
                                          const double yi, const double zi, const double vxi, const double vyi,
                                          const double vzi, const double eps2, double f[6])
{
    const double dx = xj - xi, dy = yj - yi, dz = zj - zi;
    const double dvx = vxj - vxi, dvy = vyj - vyi, dvz = vzj - vzi;
    const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    const double rv = fma(dx, dvx, fma(dy, dvy, dz * dvz));
    double rinv = rsqrt(r2);
    if (!SOFT) rinv = r2 > 0.0 ? rinv : 0.0;
    const double rinv2 = rinv * rinv;
    const double mr3 = mj * rinv * rinv2;
    const double b = -3.0 * rv * rinv2;
    f[0] = fma(mr3, dx, f[0]);
    f[1] = fma(mr3, dy, f[1]);
    f[2] = fma(mr3, dz, f[2]);
    f[3] = fma(mr3, fma(b, dx, dvx), f[3]);
    f[4] = fma(mr3, fma(b, dy, dvy), f[4]);
    f[5] = fma(mr3, fma(b, dz, dvz), f[5]);
}

struct FArgs {
    Dev d;
    int grid;
    Tune tn;
    int tail_ok;  // the host's choice of the TAIL kernel instance (the kernels use the template parameter)
    int defer;    // 1: plans with Plan::late leave their j-split partials to k_correct, unless
                  // their tiles are corrected in the force kernel's tails (see finish_item)
};

// ---------------------------------------------------------------- canonical sums of j-split partials

template <class P>
struct Acc;
template <>
struct Acc<float> {
    DS v;
    __device__ void zero() { v.zero(); }
    __device__ void add(float f) { v.add(f); }
    __device__ void add(const Acc &o)
    {
        v.add(o.v.h);
        v.add(o.v.l);
    }
    __device__ double value() const { return v.as_double(); }
    __device__ float result() const { return __fadd_rn(v.h, v.l); }
};
template <>
struct Acc<double> {
    double v;
    __device__ void zero() { v = 0.0; }
    __device__ void add(double f) { v += f; }
    __device__ void add(const Acc &o) { v += o.v; }
    __device__ double value() const { return v; }
    __device__ double result() const { return v; }
};

// Every (component, slot) sum of the S j-split partials is taken in one canonical
// order, whatever the tile's occupancy and whichever reduction routine runs: eight
// interleaved running sums q_r over s = r, r + 8, r + 16, ... (ascending), then
// ((q0 + q1) + (q2 + q3)) + ((q4 + q5) + (q6 + q7)).  A particle's force therefore
// does not depend on its slot in the active list, nor on which tile it shares.
constexpr int RED_R = 8;

template <class P>
__device__ __forceinline__ P combine8(Acc<P> q[RED_R])
{
    q[0].add(q[1]);
    q[2].add(q[3]);
    q[4].add(q[5]);
    q[6].add(q[7]);
    q[0].add(q[2]);
    q[4].add(q[6]);
    q[0].add(q[4]);
    return q[0].result();
}

// The canonical sum of the S partials of slot k, component c (partials at
// part[(s * 6 + c) * nact + k], written by other CTAs: read through L2).
template <class P>
__device__ __forceinline__ P part_sum(const Dev &d, int nact, int S, int c, int k)
{
    const P *p = (const P *)d.part + (long long)c * nact + k;
    const long long stride = 6LL * nact;
    Acc<P> q[RED_R];
#pragma unroll
    for (int r = 0; r < RED_R; r++) q[r].zero();
    for (int s0 = 0; s0 < S; s0 += RED_R) {
        P v[RED_R];
#pragma unroll
        for (int r = 0; r < RED_R; r++) v[r] = s0 + r < S ? __ldcg(p + (long long)(s0 + r) * stride) : P(0);
#pragma unroll
        for (int r = 0; r < RED_R; r++)
            if (s0 + r < S) q[r].add(v[r]);
    }
    return combine8<P>(q);
}

// ---------------------------------------------------------------- post-Newtonian pair terms
//
// Sec. 5's corrections for a binary: the 1PN, 2PN and 2.5PN relative accelerations of
// the two-body problem in harmonic coordinates (Kidder 1995, Eq. 2.2; Blanchet 2014,
// Eq. 219), with r = x_p - x_q, v = v_p - v_q, M = m_p + m_q, eta = m_p m_q / M^2,
// n = r / |r|, rdot = n.v:
//   1PN:   M / (c^2 r^2) {[(4 + 2 eta) M/r - (1 + 3 eta) v^2 + 3/2 eta rdot^2] n + (4 - 2 eta) rdot v}
//   2PN:   M / (c^4 r^2) {[-15/8 eta (1 - 3 eta) rdot^4 + 3/2 eta (3 - 4 eta) v^2 rdot^2
//                          - eta (3 - 4 eta) v^4 + 1/2 eta (13 - 4 eta) (M/r) v^2
//                          + (2 + 25 eta + 2 eta^2) (M/r) rdot^2 - 3/4 (12 + 29 eta) (M/r)^2] n
//                         + 1/2 rdot [eta (15 + 4 eta) v^2 - (4 + 41 eta + 8 eta^2) M/r
//                                     - 3 eta (3 + 2 eta) rdot^2] v}
//   2.5PN: 8/5 eta M^2 / (c^5 r^3) {rdot [18 v^2 + 2/3 M/r - 25 rdot^2] n - [6 v^2 - 2 M/r - 15 rdot^2] v}
// and their time derivative for the jerk, taken by carrying every quantity as a dual
// number (value, d/dt) along r' = v, v' = -M r / |r|^3 (the pair's Newtonian relative
// acceleration).  p gets m_q / M of the relative term, q gets -m_p / M.

template <class T>
struct Dual {
    T v, d;
};
template <class T>
__device__ __forceinline__ Dual<T> dadd(Dual<T> a, Dual<T> b) { return Dual<T>{a.v + b.v, a.d + b.d}; }
template <class T>
__device__ __forceinline__ Dual<T> dsub(Dual<T> a, Dual<T> b) { return Dual<T>{a.v - b.v, a.d - b.d}; }
template <class T>
__device__ __forceinline__ Dual<T> dmul(Dual<T> a, Dual<T> b) { return Dual<T>{a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class T>
__device__ __forceinline__ Dual<T> dscale(T s, Dual<T> a) { return Dual<T>{s * a.v, s * a.d}; }
template <class T>
__device__ __forceinline__ Dual<T> dinv(Dual<T> a) { const T i = T(1) / a.v; return Dual<T>{i, -a.d * i * i}; }
template <class T>
__device__ __forceinline__ Dual<T> dsqrt(Dual<T> a) { const T s = sqrt(a.v); return Dual<T>{s, a.d / (T(2) * s)}; }

// The pair's relative post-Newtonian acceleration (apn) and its time derivative (jpn)
// from the relative position r and velocity v.
template <class T>
__device__ void pn_pair_terms(int terms, T mp, T mq, T c, const T r[3], const T v[3], T apn[3], T jpn[3])
{
    const T M = mp + mq, eta = mp * mq / (M * M);
    const T r2v = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    const T rinv3 = T(1) / (r2v * sqrt(r2v));
    Dual<T> R[3], V[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        R[k] = Dual<T>{r[k], v[k]};
        V[k] = Dual<T>{v[k], -M * r[k] * rinv3};
    }
    Dual<T> r2 = dmul(R[0], R[0]), v2 = dmul(V[0], V[0]), rv = dmul(R[0], V[0]);
#pragma unroll
    for (int k = 1; k < 3; k++) {
        r2 = dadd(r2, dmul(R[k], R[k]));
        v2 = dadd(v2, dmul(V[k], V[k]));
        rv = dadd(rv, dmul(R[k], V[k]));
    }
    const Dual<T> rr = dsqrt(r2), ir = dinv(rr);
    const Dual<T> rd = dmul(rv, ir);  // rdot
    const Dual<T> Mr = dscale(M, ir);  // M / r
    Dual<T> acc[3] = {{T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}};
    if (terms & 1) {
        const Dual<T> alpha = dadd(dsub(dscale(T(4) + T(2) * eta, Mr), dscale(T(1) + T(3) * eta, v2)),
                                   dscale(T(1.5) * eta, dmul(rd, rd)));
        const Dual<T> beta = dscale(T(4) - T(2) * eta, rd);
        const Dual<T> K = dscale(M / (c * c), dmul(ir, ir));
#pragma unroll
        for (int k = 0; k < 3; k++)
            acc[k] = dadd(acc[k], dmul(K, dadd(dmul(alpha, dmul(R[k], ir)), dmul(beta, V[k]))));
    }
    if (terms & 2) {
        const Dual<T> rd2 = dmul(rd, rd), v4 = dmul(v2, v2), rd4 = dmul(rd2, rd2);
        const T e2 = eta * eta;
        Dual<T> alpha = dscale(T(-15) / T(8) * eta * (T(1) - T(3) * eta), rd4);
        alpha = dadd(alpha, dscale(T(1.5) * eta * (T(3) - T(4) * eta), dmul(v2, rd2)));
        alpha = dsub(alpha, dscale(eta * (T(3) - T(4) * eta), v4));
        alpha = dadd(alpha, dscale(T(0.5) * eta * (T(13) - T(4) * eta), dmul(Mr, v2)));
        alpha = dadd(alpha, dscale(T(2) + T(25) * eta + T(2) * e2, dmul(Mr, rd2)));
        alpha = dsub(alpha, dscale(T(0.75) * (T(12) + T(29) * eta), dmul(Mr, Mr)));
        Dual<T> Q = dscale(eta * (T(15) + T(4) * eta), v2);
        Q = dsub(Q, dscale(T(4) + T(41) * eta + T(8) * e2, Mr));
        Q = dsub(Q, dscale(T(3) * eta * (T(3) + T(2) * eta), rd2));
        const Dual<T> beta = dscale(T(0.5), dmul(rd, Q));
        const T c2 = c * c;
        const Dual<T> K = dscale(M / (c2 * c2), dmul(ir, ir));
#pragma unroll
        for (int k = 0; k < 3; k++)
            acc[k] = dadd(acc[k], dmul(K, dadd(dmul(alpha, dmul(R[k], ir)), dmul(beta, V[k]))));
    }
    if (terms & 4) {
        const Dual<T> rd2 = dmul(rd, rd);
        const Dual<T> alpha = dmul(rd, dadd(dsub(dscale(T(18), v2), dscale(T(25), rd2)), dscale(T(2) / T(3), Mr)));
        const Dual<T> beta = dsub(dadd(dscale(T(2), Mr), dscale(T(15), rd2)), dscale(T(6), v2));
        const T c2 = c * c;
        const Dual<T> K = dscale(T(1.6) * eta * M * M / (c2 * c2 * c), dmul(ir, dmul(ir, ir)));
#pragma unroll
        for (int k = 0; k < 3; k++)
            acc[k] = dadd(acc[k], dmul(K, dadd(dmul(alpha, dmul(R[k], ir)), dmul(beta, V[k]))));
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        apn[k] = acc[k].v;
        jpn[k] = acc[k].d;
    }
}

// Particle i's share of the pair terms, component c, from the predicted j-records
// (mixed: double-single positions, FP32 velocities; FP64: the planes pd) at the
// block time.  Adds to a and j when i is one of the pair.
// The pair terms' share of particle i (one of the pair), component c, from the two
// members' predicted mixed j-records (p's and q's), added to a and j.
__device__ __forceinline__ void pn_add_records(const Dev &d, int i, int c, float4 Ap, float4 Bp, float2 Cp,
                                               float4 Aq, float4 Bq, float2 Cq, float &a, float &j)
{
    float r[3], v[3];
    r[0] = (Ap.x - Aq.x) + (Bp.x - Bq.x);
    r[1] = (Ap.y - Aq.y) + (Bp.y - Bq.y);
    r[2] = (Ap.z - Aq.z) + (Bp.z - Bq.z);
    v[0] = Bp.w - Bq.w;
    v[1] = Cp.x - Cq.x;
    v[2] = Cp.y - Cq.y;
    const float mp = Ap.w, mq = Aq.w;
    float apn[3], jpn[3];
    pn_pair_terms<float>(d.pn_terms, mp, mq, (float)d.pn_c, r, v, apn, jpn);
    const float w = i == d.pn_p ? mq / (mp + mq) : -mp / (mp + mq);
    const float ac = c == 0 ? apn[0] : (c == 1 ? apn[1] : apn[2]);
    const float jc = c == 0 ? jpn[0] : (c == 1 ? jpn[1] : jpn[2]);
    a += w * ac;
    j += w * jc;
}

template <bool MIXED, bool COH, class T>
__device__ __forceinline__ void pn_add(const Dev &d, int i, int c, T &a, T &j)
{
    if (!d.pn_terms || (i != d.pn_p && i != d.pn_q)) return;
    const int p = d.pn_p, q = d.pn_q;
    if (MIXED) {
        const float4 Ap = ldx<COH>(&d.jA[p]), Bp = ldx<COH>(&d.jB[p]), Aq = ldx<COH>(&d.jA[q]), Bq = ldx<COH>(&d.jB[q]);
        const float2 Cp = ldx<COH>(&d.jC[p]), Cq = ldx<COH>(&d.jC[q]);
        float af = (float)a, jf = (float)j;
        pn_add_records(d, i, c, Ap, Bp, Cp, Aq, Bq, Cq, af, jf);
        a = (T)af;
        j = (T)jf;
        return;
    }
    T r[3], v[3], mp, mq;
    {
        const int np = d.npad;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            r[k] = (T)(ldx<COH>(&d.pd[k * np + p]) - ldx<COH>(&d.pd[k * np + q]));
            v[k] = (T)(ldx<COH>(&d.pd[(3 + k) * np + p]) - ldx<COH>(&d.pd[(3 + k) * np + q]));
        }
        mp = (T)d.pd[6 * np + p];
        mq = (T)d.pd[6 * np + q];
    }
    T apn[3], jpn[3];
    pn_pair_terms<T>(d.pn_terms, mp, mq, (T)d.pn_c, r, v, apn, jpn);
    const T w = i == p ? mq / (mp + mq) : -mp / (mp + mq);
    const T ac = c == 0 ? apn[0] : (c == 1 ? apn[1] : apn[2]);
    const T jc = c == 0 ? jpn[0] : (c == 1 ? jpn[1] : jpn[2]);
    a += w * ac;
    j += w * jc;
}

// Adds the pair terms to the summed forces of the first nact active slots (the
// initial forces and the force hook); one thread per slot.
template <bool MIXED>
__global__ void k_pn_fsum(Dev d, int nact)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nact) return;
    const int i = d.act[k];
    for (int c = 0; c < 3; c++) {
        if (MIXED) {
            float *fs = (float *)d.fsum;
            float a = fs[(long long)c * d.n + k], j = fs[(long long)(3 + c) * d.n + k];
            pn_add<true, false, float>(d, i, c, a, j);
            fs[(long long)c * d.n + k] = a;
            fs[(long long)(3 + c) * d.n + k] = j;
        } else {
            double a = d.fsum[(long long)c * d.n + k], j = d.fsum[(long long)(3 + c) * d.n + k];
            pn_add<false, false, double>(d, i, c, a, j);
            d.fsum[(long long)c * d.n + k] = a;
            d.fsum[(long long)(3 + c) * d.n + k] = j;
        }
    }
}

// ---------------------------------------------------------------- corrector + time step

// The power-of-two block step after a correction at tick T, from the Aarseth
// estimate dt_new^2 = num / den (Sec. 3.2) with num = eta (|a1||a2e| + |j1|^2) and
// den = |j1||a3| + |a2e|^2.  Rules (same as the initial quantisation): steps are
// powers of two of dt_min in [1, dtau_max] ticks; shrink to the largest power of two
// not above dt_new; grow by 2 only if dt_new >= 2 dt_old at a time that is a
// multiple of twice the old step.  dt_new = Inf or NaN (an isolated particle)
// counts as unconstrained.  The decisions compare num with den times exact powers
// of two, so no FP64 divide or square root is needed; floor(log2(num / D)) is read
// off the binary exponents and a mantissa comparison.
__device__ __forceinline__ long long next_block_step(const Dev &d, double num, double den, long long dtau_old,
                                                     long long T)
{
    const bool unconstrained = !(den > 0.0) || !(num == num) || isinf(num);
    if (!unconstrained) {
        if (!(num > 0.0)) return 1;  // dt_new = 0
        const double dto = (double)dtau_old * d.dt_min;
        const double lim = dto * dto * den;
        if (num < lim) {
            const double D = den * d.dt_min2;  // exact: dt_min^2 is a power of two
            int fl;
            if (D >= 2.2250738585072014e-308 && num >= 2.2250738585072014e-308) {
                const long long bn = __double_as_longlong(num), bd = __double_as_longlong(D);
                const int en = (int)((bn >> 52) & 0x7FF), ed = (int)((bd >> 52) & 0x7FF);
                const long long mn = bn & 0xFFFFFFFFFFFFFLL, md = bd & 0xFFFFFFFFFFFFFLL;
                fl = en - ed - (mn < md ? 1 : 0);
            } else {
                const double q = num / D;
                fl = (int)((__double_as_longlong(q) >> 52) & 0x7FF) - 1023;
            }
            const int lvl = fl >> 1;  // floor(fl / 2)
            if (lvl < 0) return 1;
            return 1LL << lvl;
        }
        if (!(num >= 4.0 * lim)) return dtau_old;
    }
    if (2 * dtau_old <= d.dtau_max && (T & (2 * dtau_old - 1)) == 0) return 2 * dtau_old;
    return dtau_old;
}

// ---------------------------------------------------------------- mixed-path time step
//
// The same rules as next_block_step, with the Aarseth estimate from FP32 norms.
// FP32 cannot hold the products of the criterion (|a3|^2 reaches 1e47 at the
// smallest steps), so every quantity is kept as m * 2^e with m in [1, 2) and an
// integer exponent: products and sums of the criterion never overflow, and the
// comparisons with powers of two stay exact.

struct XF {
    float m;  // 0, or in [1, 2)
    int e;
};

__device__ __forceinline__ XF xf_of(float x)  // x >= 0 finite
{
    if (!(x > 0.f)) return XF{0.f, 0};
    int sh = 0;
    if (x < 1.1754944e-38f) {  // subnormal: scale up exactly first
        x = __fmul_rn(x, 1.8446744e19f);  // 2^64
        sh = 64;
    }
    const unsigned b = __float_as_uint(x);
    return XF{__uint_as_float((b & 0x007FFFFFu) | 0x3F800000u), (int)((b >> 23) & 0xFFu) - 127 - sh};
}

__device__ __forceinline__ XF xf_norm(float m, int e)  // m in [0, 4)
{
    if (m >= 2.f) return XF{__fmul_rn(m, 0.5f), e + 1};
    return XF{m, e};
}

__device__ __forceinline__ XF xf_mul(XF a, XF b)
{
    if (a.m == 0.f || b.m == 0.f) return XF{0.f, 0};
    return xf_norm(__fmul_rn(a.m, b.m), a.e + b.e);
}

__device__ __forceinline__ XF xf_add(XF a, XF b)
{
    if (a.m == 0.f) return b;
    if (b.m == 0.f) return a;
    if (a.e < b.e) {
        const XF t = a;
        a = b;
        b = t;
    }
    const int k = a.e - b.e;
    if (k > 60) return a;
    return xf_norm(__fadd_rn(a.m, __fmul_rn(b.m, __uint_as_float((unsigned)(127 - k) << 23))), a.e);
}

// a < b for non-negative values
__device__ __forceinline__ bool xf_lt(XF a, XF b)
{
    if (a.m == 0.f) return b.m > 0.f;
    if (b.m == 0.f) return false;
    return a.e < b.e || (a.e == b.e && a.m < b.m);
}

// Euclidean norm of the 3-vector whose components sit on lanes 0-2 of each group of
// four (lane 3 passes 0), scaled by a power of two so the squares cannot overflow.
__device__ __forceinline__ float norm3_group(float x)
{
    float mx = fabsf(x);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    const int eb = (int)((__float_as_uint(mx) >> 23) & 0xFFu);
    const bool plain = !(mx > 0.f) || eb == 0 || eb > 253;  // zero, subnormal, huge, Inf or NaN
    const float sc = plain ? 1.f : __uint_as_float((unsigned)(254 - eb) << 23);  // 2^-(E)
    const float y = __fmul_rn(x, sc);
    float q = __fmul_rn(y, y);
    q = __fadd_rn(q, __shfl_xor_sync(0xffffffffu, q, 1));
    q = __fadd_rn(q, __shfl_xor_sync(0xffffffffu, q, 2));
    if (plain) return eb == 0 && mx > 0.f ? mx : (mx > 0.f ? __fsqrt_rn(q) : 0.f);
    return __fmul_rn(__fsqrt_rn(q), __uint_as_float((unsigned)eb << 23));  // * 2^E
}

__device__ __forceinline__ long long next_block_step_f(const Dev &d, float na1, float nj1, float na2, float na3,
                                                       long long dtau_old, long long T)
{
    const bool finite = isfinite(na1) && isfinite(nj1) && isfinite(na2) && isfinite(na3);
    // num = eta (|a1||a2e| + |j1|^2), den = |j1||a3| + |a2e|^2
    const XF A = xf_of(na1), J = xf_of(nj1), B = xf_of(na2), C = xf_of(na3);
    const XF num = xf_mul(xf_of(d.eta_f), xf_add(xf_mul(A, B), xf_mul(J, J)));
    const XF den = xf_add(xf_mul(J, C), xf_mul(B, B));
    const bool unconstrained = !finite || den.m == 0.f;
    if (!unconstrained) {
        if (num.m == 0.f) return 1;
        // dt_old^2 = 2^(2k), k = log2(dtau_old) + log2(dt_min)
        const int lt = 63 - __clzll(dtau_old);
        const int ldm = (int)((__float_as_uint(d.dt_min_f) >> 23) & 0xFFu) - 127;
        const XF lim{den.m, den.e + 2 * (lt + ldm)};
        if (xf_lt(num, lim)) {
            // floor(log2(num / (den dt_min^2)))
            const int fl = num.e - (den.e + 2 * ldm) - (num.m < den.m ? 1 : 0);
            const int lvl = fl >> 1;
            if (lvl < 0) return 1;
            return 1LL << lvl;
        }
        const XF lim4{den.m, lim.e + 2};
        if (xf_lt(num, lim4)) return dtau_old;
    }
    if (2 * dtau_old <= d.dtau_max && (T & (2 * dtau_old - 1)) == 0) return 2 * dtau_old;
    return dtau_old;
}

// (a.h + a.l) + (b.h + b.l), normalised
__device__ __forceinline__ F2 ds_add(F2 a, F2 b)
{
    const F2 s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

// The time-symmetric fourth-order corrector (Hut, Makino & McMillan 1995) of one
// component on the mixed path, with h = dt / 2:
//   v1 = v0 + h (a1 + a0) - (h^2 / 3) (j1 - j0),
//   x1 = x0 + h (v1 + v0) - (h^2 / 3) (a1 - a0).
// The velocity update is an FP32 term added to the double-single v0; the position
// update adds the exact product h * (v1 + v0).hi (product and FMA residual) and
// FP32 terms to the double-single x0.  Results canonical.
__device__ __forceinline__ void ds_correct_tsym(float dt, F2 x0, F2 v0, float a0, float j0, float a1, float j1,
                                                F2 &x1, F2 &v1)
{
    const float h = __fmul_rn(0.5f, dt);
    const float h2_3 = __fmul_rn(__fmul_rn(h, h), 1.0f / 3.0f);
    const float dv = fmaf(h, __fadd_rn(a1, a0), -__fmul_rn(h2_3, __fadd_rn(j1, -j0)));
    v1 = ds_canon(ds_add_f(v0, dv));
    const F2 sv = ds_add(v0, v1);
    const float p = __fmul_rn(h, sv.h);
    const float pe = fmaf(h, sv.h, -p);
    const float small = __fadd_rn(fmaf(h, sv.l, pe), -__fmul_rn(h2_3, __fadd_rn(a1, -a0)));
    const F2 t = two_sum(x0.h, p);
    x1 = ds_canon(two_sum(t.h, __fadd_rn(__fadd_rn(t.l, x0.l), small)));
}

// Correction (Sec. 2.4 step 7d, Hermite scheme) on the mixed path, laid out as
// correct_slots64 (four lanes per particle): FP32 Hermite derivatives and
// correction terms (the forces they come from are FP32-accurate), double-single
// position and velocity sums, canonical results, the step from next_block_step_f.
// One component of the mixed-path correction (lanes 0-2 of a group of four hold
// x, y, z; lane 3 repeats z and is ignored): prediction, Hermite derivatives from
// the end-point forces, corrected x and v (canonical double-single), and the new
// block step (every lane of the group gets the same).  dtick > 0.
__device__ __forceinline__ void ds_correct(const Dev &d, bool real, long long dtick, long long dtau_old, long long T,
                                           F2 x0, F2 v0, float a0, float j0, float a1, float j1, F2 &x1, F2 &v1,
                                           long long &dtau)
{
    float dt, idt;
    step_f(d, dtick, dt, idt);
    const float dt2 = __fmul_rn(dt, dt), dt3 = __fmul_rn(dt2, dt), dt4 = __fmul_rn(dt3, dt);
    const float dt5 = __fmul_rn(dt4, dt);
    const float idt2 = __fmul_rn(idt, idt), idt3 = __fmul_rn(idt2, idt);
    const float h2 = __fmul_rn(0.5f, dt2), h3 = __fmul_rn(dt3, 1.0f / 6.0f);
    const float h4 = __fmul_rn(dt4, 1.0f / 24.0f), h5 = __fmul_rn(dt5, 1.0f / 120.0f);
    // prediction of this component (Sec. 2.4 step 7a)
    const F2 xp = ds_pred_x(x0, v0, a0, j0, dt, h2, h3);
    const F2 vp = ds_pred_v(v0, a0, j0, dt, h2);
    // 2nd and 3rd derivative at the start of the step from the end-point values
    const float da = __fadd_rn(a0, -a1);
    const float a2 = __fmul_rn(fmaf(-6.0f, da, -__fmul_rn(dt, fmaf(4.0f, j0, __fmul_rn(2.0f, j1)))), idt2);
    const float a3 = __fmul_rn(fmaf(12.0f, da, __fmul_rn(__fmul_rn(6.0f, dt), __fadd_rn(j0, j1))), idt3);
    if (d.tsym) {
        ds_correct_tsym(dt, x0, v0, a0, j0, a1, j1, x1, v1);
    } else {
        x1 = ds_canon(ds_add_f(xp, fmaf(a3, h5, __fmul_rn(a2, h4))));
        v1 = ds_canon(ds_add_f(vp, fmaf(a3, h4, __fmul_rn(a2, h3))));
    }
    const float a2e = fmaf(dt, a3, a2);  // 2nd derivative at the end of the step
    const float na1 = norm3_group(real ? a1 : 0.f), nj1 = norm3_group(real ? j1 : 0.f);
    const float na2 = norm3_group(real ? a2e : 0.f), na3 = norm3_group(real ? a3 : 0.f);
    dtau = next_block_step_f(d, na1, nj1, na2, na3, dtau_old, T);
}

// S > 0: the new force of slot k is the canonical sum of its S j-split partials
// (part_sum, over nact slots); S = 0: it is read from fsum.
template <bool COH>
__device__ __forceinline__ void correct_slots_ds(const Dev &d, long long T, int k_lo, int k_hi, int w0, int ws,
                                                 long long &mymin, int &bad, int S, int nact, bool trial = false)
{
    const int n = d.n;
    const int lane = threadIdx.x & 31;
    const int q = lane & 3;
    const int c = q < 3 ? q : 2;
    const bool real = q < 3;
    const float *fs = (const float *)d.fsum;
    for (int kw = k_lo + w0 * 8; kw < k_hi; kw += ws * 8) {
        const int k = kw + (lane >> 2);
        const bool valid = k < k_hi;
        const int kk = valid ? k : k_hi - 1;
        const int i = ldx<COH>(&d.act[kk]);
        const long long tau0 = ldx<COH>(&d.tau[i]);
        const long long dtau_old = ldx<COH>(&d.dtau[i]);
        const long long dtick = T - tau0;
        const bool behind = dtick > 0;
        const F2 x0 = ldx_ds<COH>(d.xs, n, c, i), v0 = ldx_ds<COH>(d.vs, n, c, i);
        const float a0 = ldx<COH>(&d.af[c * n + i]), j0 = ldx<COH>(&d.jf[c * n + i]);
        float a1 = S > 0 ? part_sum<float>(d, nact, S, c, kk) : ldc(&fs[c * n + kk]);
        float j1 = S > 0 ? part_sum<float>(d, nact, S, 3 + c, kk) : ldc(&fs[(3 + c) * n + kk]);
        pn_add<true, COH, float>(d, i, c, a1, j1);
        F2 x1, v1;
        long long dtau;
        ds_correct(d, real, behind ? dtick : 1, dtau_old, T, x0, v0, a0, j0, a1, j1, x1, v1, dtau);
        const bool fin = isfinite(x1.h) && isfinite(v1.h) && isfinite(a1) && isfinite(j1);
        if (trial) {
            // a pass before the last (P(EC)^n): the corrected position and velocity
            // replace the particle's predicted j-record; the state stays
            if (valid && behind && real) {
                if (!fin) bad |= 1;
                ((float *)&d.jA[i])[c] = x1.h;
                ((float *)&d.jB[i])[c] = x1.l;
                const float vr = __fadd_rn(v1.h, v1.l);
                if (c == 0)
                    d.jB[i].w = vr;
                else
                    ((float *)&d.jC[i])[c - 1] = vr;
            }
            if (valid && !behind) bad |= 2;
            continue;
        }
        if (valid) {
            if (!behind) {
                bad |= 2;
            } else {
                if (real) {
                    if (!fin) bad |= 1;
                    st_ds(d.xs, n, c, i, x1);
                    st_ds(d.vs, n, c, i, v1);
                    d.af[c * n + i] = a1;
                    d.jf[c * n + i] = j1;
                }
                if (q == 0) {
                    d.tau[i] = T;
                    d.dtau[i] = dtau;
                    const long long tn = T + dtau;
                    d.tnext[i] = tn;
                    mymin = tn < mymin ? tn : mymin;
                }
            }
        }
    }
}

// Correction (Sec. 2.4 step 7d, Hermite scheme) of active slots [k_lo, k_hi) with
// the new force in fsum, at block time T: the calling warps w0, w0 + ws, ... take
// eight particles at a time, four lanes per particle -- lanes 0-2 the x, y, z
// components (prediction, Hermite derivatives, correction), the squared norms of
// the Aarseth criterion summed across the four lanes, lanes 0 and 1 its two square
// roots side by side.  mymin collects the new next times, bad the fault bits
// (1 non-finite, 2 a particle not behind T, which is left untouched).
template <bool COH>
__device__ __forceinline__ void correct_slots64(const Dev &d, long long T, int k_lo, int k_hi, int w0, int ws,
                                                long long &mymin, int &bad, int S, int nact, bool trial = false)
{
    const int n = d.n;
    const int lane = threadIdx.x & 31;
    const int q = lane & 3;
    const int c = q < 3 ? q : 2;
    const bool real = q < 3;
    for (int kw = k_lo + w0 * 8; kw < k_hi; kw += ws * 8) {
        const int k = kw + (lane >> 2);
        const bool valid = k < k_hi;
        const int kk = valid ? k : k_hi - 1;
        const int i = ldx<COH>(&d.act[kk]);
        const long long tau0 = ldx<COH>(&d.tau[i]);
        const long long dtau_old = ldx<COH>(&d.dtau[i]);
        const long long dtick = T - tau0;
        const bool behind = dtick > 0;
        const double dt = (double)dtick * d.dt_min;
        double idt;
        if (behind && (dtick & (dtick - 1)) == 0) {
            const int e = 63 - __clzll(dtick);
            idt = d.inv_dt_min * __longlong_as_double((long long)(1023 - e) << 52);
        } else {
            idt = 1.0 / dt;
        }
        const double dt2 = dt * dt, dt3 = dt2 * dt, dt4 = dt3 * dt, dt5 = dt4 * dt;
        const double idt2 = idt * idt, idt3 = idt2 * idt;
        const double h2 = 0.5 * dt2, h3 = dt3 * (1.0 / 6.0), h4 = dt4 * (1.0 / 24.0), h5 = dt5 * (1.0 / 120.0);
        const double x0 = ldx<COH>(&d.x[c * n + i]), v0 = ldx<COH>(&d.v[c * n + i]),
                     a0 = ldx<COH>(&d.a[c * n + i]), j0 = ldx<COH>(&d.jk[c * n + i]);
        double a1 = S > 0 ? part_sum<double>(d, nact, S, c, kk) : ldc(&d.fsum[(long long)c * n + kk]);
        double j1 = S > 0 ? part_sum<double>(d, nact, S, 3 + c, kk) : ldc(&d.fsum[(long long)(3 + c) * n + kk]);
        pn_add<false, COH, double>(d, i, c, a1, j1);
        // prediction of this component (Sec. 2.4 step 7a)
        const double xp = fma(j0, h3, fma(a0, h2, fma(v0, dt, x0)));
        const double vp = fma(j0, h2, fma(a0, dt, v0));
        // 2nd and 3rd derivative at the start of the step from the end-point values
        const double da = a0 - a1;
        const double a2 = (-6.0 * da - dt * (4.0 * j0 + 2.0 * j1)) * idt2;
        const double a3 = (12.0 * da + 6.0 * dt * (j0 + j1)) * idt3;
        double x1, v1;
        if (d.tsym) {  // time-symmetric form, h = dt / 2 (see ds_correct_tsym)
            const double h = 0.5 * dt, hh3 = h * h / 3.0;
            v1 = v0 + h * (a1 + a0) - hh3 * (j1 - j0);
            x1 = x0 + h * (v1 + v0) - hh3 * (a1 - a0);
        } else {
            x1 = xp + a2 * h4 + a3 * h5;
            v1 = vp + a2 * h3 + a3 * h4;
        }
        const double a2e = fma(dt, a3, a2);  // 2nd derivative at the end of the step
        // squared norms, summed over the group's lanes
        double sA = real ? a1 * a1 : 0.0, sJ = real ? j1 * j1 : 0.0;
        double sB = real ? a2e * a2e : 0.0, sC = real ? a3 * a3 : 0.0;
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            sA += __shfl_xor_sync(0xffffffffu, sA, o);
            sJ += __shfl_xor_sync(0xffffffffu, sJ, o);
            sB += __shfl_xor_sync(0xffffffffu, sB, o);
            sC += __shfl_xor_sync(0xffffffffu, sC, o);
        }
        // |a1||a2e| = sqrt(A B) on even lanes, |j1||a3| = sqrt(J C) on odd lanes
        const double r = sqrt((q & 1) ? sJ * sC : sA * sB);
        const double ro = __shfl_xor_sync(0xffffffffu, r, 1);
        const double sAB = (q & 1) ? ro : r, sJC = (q & 1) ? r : ro;
        const double num = d.eta * (sAB + sJ);
        const double den = sJC + sB;
        const long long dtau = next_block_step(d, num, den, dtau_old, T);
        const bool fin = isfinite(x1) && isfinite(v1) && isfinite(a1) && isfinite(j1);
        if (trial) {
            // a pass before the last (P(EC)^n): corrected x, v into the predicted record
            if (valid && behind && real) {
                if (!fin) bad |= 1;
                d.pd[c * d.npad + i] = x1;
                d.pd[(3 + c) * d.npad + i] = v1;
            }
            if (valid && !behind) bad |= 2;
            continue;
        }
        if (valid) {
            if (!behind) {
                bad |= 2;
            } else {
                if (real) {
                    if (!fin) bad |= 1;
                    d.x[c * n + i] = x1;
                    d.v[c * n + i] = v1;
                    d.a[c * n + i] = a1;
                    d.jk[c * n + i] = j1;
                }
                if (q == 0) {
                    d.tau[i] = T;
                    d.dtau[i] = dtau;
                    const long long tn = T + dtau;
                    d.tnext[i] = tn;
                    mymin = tn < mymin ? tn : mymin;
                }
            }
        }
    }
}

template <bool MIXED, bool COH>
__device__ __forceinline__ void correct_slots(const Dev &d, long long T, int k_lo, int k_hi, int w0, int ws,
                                              long long &mymin, int &bad, int S = 0, int nact = 0,
                                              bool trial = false)
{
    if (MIXED)
        correct_slots_ds<COH>(d, T, k_lo, k_hi, w0, ws, mymin, bad, S, nact, trial);
    else
        correct_slots64<COH>(d, T, k_lo, k_hi, w0, ws, mymin, bad, S, nact, trial);
}

// ---------------------------------------------------------------- j-split reduction

template <class P>
__device__ __forceinline__ void store_partial(const Dev &d, int nact, int s, int k, const P f[6])
{
    P *p = (P *)d.part + (long long)s * 6 * nact + k;
#pragma unroll
    for (int c = 0; c < 6; c++) p[(long long)c * nact] = f[c];
}

// The summed force of slot k, component c: FP64 on the FP64 path, FP32 on the
// mixed path (see fsum_f).
template <class P>
__device__ __forceinline__ void store_fsum(const Dev &d, int c, int k, P v)
{
    ((P *)d.fsum)[(long long)c * d.n + k] = v;
}

// Sums the S partials of slots [k0, k0 + nvalid) into fsum (large tiles): one
// thread per (component, slot) pair keeps the eight running sums, loading eight
// consecutive splits at a time.  Partials written by other CTAs are read through
// L2 (__ldcg).
template <class P>
__device__ void tile_reduce(const Dev &d, int nact, int S, int k0, int nvalid)
{
    const int npairs = nvalid * 6;
    for (int pidx = threadIdx.x; pidx < npairs; pidx += FT) {
        const int c = pidx / nvalid, k = k0 + pidx % nvalid;
        store_fsum<P>(d, c, k, part_sum<P>(d, nact, S, c, k));
    }
}

// The same sums for a small tile (at most MAXK slots, the warp-mode tiles): the
// (pair, residue) running sums are spread over the CTA's threads, so every load of
// a thread is independent and the latency is about one round trip per eight splits
// a residue holds; the eight sums of a pair meet in shared memory.
template <class P, int MAXK>
__device__ void tile_reduce_small(const Dev &d, int nact, int S, int k0, int nvalid)
{
    __shared__ Acc<P> s_q[6 * MAXK][RED_R];
    const P *part = (const P *)d.part;
    const int npairs = nvalid * 6;
    const long long stride = 6LL * nact;
    for (int w = threadIdx.x; w < npairs * RED_R; w += FT) {
        const int pidx = w / RED_R, r = w % RED_R;
        const int c = pidx / nvalid, k = k0 + pidx % nvalid;
        const P *p = part + (long long)c * nact + k;
        Acc<P> q;
        q.zero();
#pragma unroll 8
        for (int s = r; s < S; s += RED_R) q.add(__ldcg(p + (long long)s * stride));
        s_q[pidx][r] = q;
    }
    __syncthreads();
    if (threadIdx.x < npairs) {
        const int pidx = threadIdx.x;
        const int c = pidx / nvalid, k = k0 + pidx % nvalid;
        Acc<P> q[RED_R];
#pragma unroll
        for (int r = 0; r < RED_R; r++) q[r] = s_q[pidx][r];
        store_fsum<P>(d, c, k, combine8<P>(q));
    }
    __syncthreads();
}

// After a CTA has stored its partials for i-tile `it`: the last of the S CTAs of
// that tile sums them (the counter returns to zero for the next launch) and, with
// `tail`, corrects the tile's particles right away, adding their new next times
// to *Tacc.
//
// With `defer` an i-parallel plan (mode 0) stops after the partial stores: its
// tiles hold up to ITILE_A_MIX slots and S partials each, which one CTA would sum
// as a long chain of L2 round trips, while k_correct sums them spread over the GPU
// (part_sum, the same canonical order).  A warp-mode plan does the same where the
// tuning table asks for it (mode 2: chosen by the autotuner where it measured
// faster), unless it corrects its tiles in the tail.
template <class P, bool COH>
__device__ __forceinline__ void finish_item(const Dev &d, int nact, const Plan &pl, int it, bool tail, long long T,
                                            unsigned long long *Tacc, int defer = 0)
{
    __shared__ int s_last;
    // the barrier gathers this CTA's partial stores; thread 0's fence releases them
    // before the arrival is counted
    __syncthreads();
    if (defer && pl.late && !tail) return;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&d.tilecnt[it], 1u);
        s_last = prev == (unsigned)(pl.S - 1);
        if (s_last) d.tilecnt[it] = 0u;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        const int k0 = it * pl.itile;
        const int nvalid = min(pl.itile, nact - k0);
        constexpr int MAXK = sizeof(P) == 4 ? ITILE_B_MIX : ITILE_B_64;
        if (nvalid <= MAXK)
            tile_reduce_small<P, MAXK>(d, nact, pl.S, k0, nvalid);
        else
            tile_reduce<P>(d, nact, pl.S, k0, nvalid);
        if (tail) {
            __syncthreads();
            long long mymin = LLONG_MAX;
            int bad = 0;
            correct_slots<sizeof(P) == 4, COH>(d, T, k0, k0 + nvalid, threadIdx.x >> 5, FT / 32, mymin, bad);
            if (bad & 2) set_err(d.ctrl, ST_EINVAL);
            if (bad & 1) set_err(d.ctrl, ST_ENONFINITE);
            mymin = warp_min_ll(mymin);
            if ((threadIdx.x & 31) == 0 && mymin != LLONG_MAX) atomicMin(Tacc, (unsigned long long)mymin);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- force (mixed)

constexpr int BJB = 256;  // warp mode j-tile (2 records per thread)

// j-tiles of the force phases: nt records from jt (nt even) into buffer buf of the
// CTA's double-buffered shared-memory tile, by asynchronous copies (one commit group
// per tile, so the next tile loads while the warps work on the current one); the
// C fields travel two records per 16-byte copy.
struct JTile {
    float4 A[2][BJB], B[2][BJB];
    float2 C[2][BJB];
};

__device__ __forceinline__ void stage_jtile(const Dev &d, JTile &s, int buf, int jt, int nt)
{
    for (int q = threadIdx.x; q < nt; q += FT) {
        cp_async16(&s.A[buf][q], &d.jA[jt + q]);
        cp_async16(&s.B[buf][q], &d.jB[jt + q]);
    }
    for (int q = threadIdx.x; q < nt / 2; q += FT) cp_async16(&s.C[buf][2 * q], &d.jC[jt + 2 * q]);
    cp_async_commit();
}

// Waits for the tile in the current buffer, first putting the next one (if any) in
// flight; ends with a CTA barrier so every warp sees the current tile.
__device__ __forceinline__ void next_jtile(const Dev &d, JTile &s, int buf, int jt, int tile, int jend)
{
    const int jn = jt + tile;
    if (jn < jend) {
        stage_jtile(d, s, buf ^ 1, jn, min(tile, jend - jn));
        cp_async_wait<1>();
    } else {
        cp_async_wait<0>();
    }
    __syncthreads();
}

template <bool SOFT, bool COH>
__device__ void phase_force_mixed(const Dev &d, int nact, const Plan &pl, bool tail, long long T,
                                  unsigned long long *Tacc, int defer = 0)
{
    const float eps2 = d.eps2f;
    __shared__ __align__(16) JTile sj;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (long long item = blockIdx.x; item < pl.items; item += gridDim.x) {
        const int it = (int)(item / pl.S), s = (int)(item % pl.S);
        const int jbeg = s * pl.chunk;
        const int jend = min(jbeg + pl.chunk, d.npad);
        // the j-range [jbeg, jend) comes in tiles of BJ (i-parallel) or BJB (warp mode)
        // records, a multiple of BJ each; the first is put in flight here
        const int tile = pl.mode == 0 ? BJ : BJB;
        __syncthreads();  // the previous item's warps are done with both buffers
        if (jbeg < jend) stage_jtile(d, sj, 0, jbeg, min(tile, jend - jbeg));
        if (pl.mode == 0) {
            // i-parallel: thread t owns active slots k0 and k1
            const int k0 = it * ITILE_A_MIX + t, k1 = k0 + FT;
            const int i0 = ldx<COH>(&d.act[min(k0, nact - 1)]), i1 = ldx<COH>(&d.act[min(k1, nact - 1)]);
            const float4 A0 = ldx<COH>(&d.jA[i0]), B0 = ldx<COH>(&d.jB[i0]);
            const float2 C0 = ldx<COH>(&d.jC[i0]);
            const float4 A1 = ldx<COH>(&d.jA[i1]), B1 = ldx<COH>(&d.jB[i1]);
            const float2 C1 = ldx<COH>(&d.jC[i1]);
            const bool busy = it * ITILE_A_MIX + warp * 32 < nact;  // the warp has a real slot
            DS g0[6], g1[6];
#pragma unroll
            for (int c = 0; c < 6; c++) {
                g0[c].zero();
                g1[c].zero();
            }
            int buf = 0;
            for (int jt = jbeg; jt < jend; jt += BJ, buf ^= 1) {
                next_jtile(d, sj, buf, jt, BJ, jend);
                if (busy) {
                    const float4 *sA = sj.A[buf], *sB = sj.B[buf];
                    const float2 *sC = sj.C[buf];
                    float f0[6] = {0, 0, 0, 0, 0, 0}, f1[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 8
                    for (int jj = 0; jj < BJ; jj++) {
                        const float4 A = sA[jj], B = sB[jj];
                        const float2 C = sC[jj];
                        pair_mixed<SOFT>(A, B, C, A0.x, A0.y, A0.z, B0.x, B0.y, B0.z, B0.w, C0.x, C0.y, eps2, f0);
                        pair_mixed<SOFT>(A, B, C, A1.x, A1.y, A1.z, B1.x, B1.y, B1.z, B1.w, C1.x, C1.y, eps2, f1);
                    }
#pragma unroll
                    for (int c = 0; c < 6; c++) {
                        g0[c].add(f0[c]);
                        g1[c].add(f1[c]);
                    }
                }
                __syncthreads();  // every warp is done with this buffer before it is refilled
            }
            float r0[6], r1[6];
#pragma unroll
            for (int c = 0; c < 6; c++) {
                r0[c] = g0[c].as_float();
                r1[c] = g1[c].as_float();
            }
            if (k0 < nact) store_partial<float>(d, nact, s, k0, r0);
            if (k1 < nact) store_partial<float>(d, nact, s, k1, r1);
        } else {
            // warp j-parallel: warp w owns slots k0, k0+1; the warp's lanes split each
            // staged tile of BJB records
            const int k0 = it * ITILE_B_MIX + 2 * warp;
            const bool busy = k0 < nact;
            const bool has1 = k0 + 1 < nact;
            const int i0 = ldx<COH>(&d.act[min(k0, nact - 1)]), i1 = ldx<COH>(&d.act[min(has1 ? k0 + 1 : k0, nact - 1)]);
            const float4 A0 = ldx<COH>(&d.jA[i0]), B0 = ldx<COH>(&d.jB[i0]);
            const float2 C0 = ldx<COH>(&d.jC[i0]);
            const float4 A1 = ldx<COH>(&d.jA[i1]), B1 = ldx<COH>(&d.jB[i1]);
            const float2 C1 = ldx<COH>(&d.jC[i1]);
            DS g0[6], g1[6];
#pragma unroll
            for (int c = 0; c < 6; c++) {
                g0[c].zero();
                g1[c].zero();
            }
            // FP32 sums over 32 * FOLD_B = 2 BJB j's (each lane: FOLD_B of them), folded
            // into the compensated sums
            static_assert(32 * FOLD_B == 2 * BJB, "fold blocks span two staged tiles");
            float f0[6] = {0, 0, 0, 0, 0, 0}, f1[6] = {0, 0, 0, 0, 0, 0};
            int buf = 0;
            for (int jt = jbeg; jt < jend; jt += BJB, buf ^= 1) {
                const int nt = min(BJB, jend - jt);  // a multiple of BJ
                next_jtile(d, sj, buf, jt, BJB, jend);
                if (busy) {
                    const float4 *sA = sj.A[buf], *sB = sj.B[buf];
                    const float2 *sC = sj.C[buf];
#pragma unroll 8
                    for (int jj = lane; jj < nt; jj += 32) {
                        const float4 A = sA[jj], B = sB[jj];
                        const float2 C = sC[jj];
                        pair_mixed<SOFT>(A, B, C, A0.x, A0.y, A0.z, B0.x, B0.y, B0.z, B0.w, C0.x, C0.y, eps2, f0);
                        pair_mixed<SOFT>(A, B, C, A1.x, A1.y, A1.z, B1.x, B1.y, B1.z, B1.w, C1.x, C1.y, eps2, f1);
                    }
                    if (((jt - jbeg) / BJB) % 2 == 1 || jt + BJB >= jend) {
#pragma unroll
                        for (int c = 0; c < 6; c++) {
                            g0[c].add(f0[c]);
                            g1[c].add(f1[c]);
                            f0[c] = 0.f;
                            f1[c] = 0.f;
                        }
                    }
                }
                __syncthreads();  // every warp is done with this buffer before it is refilled
            }
            if (busy) {
                float r0[6], r1[6];
#pragma unroll
                for (int c = 0; c < 6; c++) {
                    r0[c] = g0[c].as_float();
                    r1[c] = g1[c].as_float();
                    for (int o = 16; o > 0; o >>= 1) {
                        r0[c] += __shfl_xor_sync(0xffffffffu, r0[c], o);
                        r1[c] += __shfl_xor_sync(0xffffffffu, r1[c], o);
                    }
                }
                if (lane == 0) {
                    store_partial<float>(d, nact, s, k0, r0);
                    if (has1) store_partial<float>(d, nact, s, k0 + 1, r1);
                }
            }
        }
        finish_item<float, COH>(d, nact, pl, it, tail, T, Tacc, defer);
    }
}

// The last CTA to finish a kernel that corrected in its tile tails turns the
// running minimum into the next block time and counts the step.
// Only the CTAs that took work items (the first min(grid, items)) count in.
__device__ __forceinline__ void finalize_step(const Dev &d, int nact, long long T, long long items)
{
    Ctrl *ctrl = d.ctrl;
    const unsigned nin = (unsigned)min((long long)gridDim.x, items);
    if (blockIdx.x >= nin) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&ctrl->done, 1u);
        if (prev == nin - 1) {
            __threadfence();
            const long long next = (long long)atomicAdd((unsigned long long *)&ctrl->T_acc, 0ull);
            ctrl->T_last = T;
            ctrl->last_nact = nact;
            ctrl->T_cur = next;
            ctrl->T_acc = LLONG_MAX;
            ctrl->nblock += 1;
            ctrl->nsteps += nact;
            ctrl->interactions += (double)nact * (double)d.n;
            ctrl->epoch += 1;
            ctrl->done = 0;
        }
    }
}

// TAIL (compile time, so the plain force kernel carries no corrector code): small
// tiles are corrected in their reduction tails and the step is finalized here.
template <bool SOFT, bool TAIL>
__global__ void __launch_bounds__(FT, 4) k_force_mixed(FArgs fa)
{
    pdl_trigger();
    pdl_wait();
    const Dev &d = fa.d;
    const int nact = min(d.ctrl->nact, d.n);
    if (nact <= 0) return;
    const Plan pl = make_plan(nact, d.npad, fa.grid, fa.tn, true, d.cap);
    if (TAIL && pl.mode == 1) {
        const long long T = d.ctrl->T_cur;
        phase_force_mixed<SOFT, false>(d, nact, pl, true, T, (unsigned long long *)&d.ctrl->T_acc, fa.defer);
        finalize_step(d, nact, T, pl.items);
    } else {
        phase_force_mixed<SOFT, false>(d, nact, pl, false, 0, nullptr, fa.defer);
    }
}

// ---------------------------------------------------------------- kernel: force (FP64)

template <bool SOFT, bool TAIL>
__global__ void __launch_bounds__(FT, 4) k_force_fp64(FArgs fa)
{
    pdl_trigger();
    pdl_wait();
    const Dev &d = fa.d;
    const int nact = min(d.ctrl->nact, d.n);
    if (nact <= 0) return;
    const long long T = d.ctrl->T_cur;
    const Plan pl = make_plan(nact, d.npad, fa.grid, fa.tn, false, d.cap);
    const bool tail = TAIL && pl.mode == 1;
    const double eps2 = d.eps2;
    const int np = d.npad;
    const double *P = d.pd;
    __shared__ double sP[7][BJ64];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (long long item = blockIdx.x; item < pl.items; item += gridDim.x) {
        const int it = (int)(item / pl.S), s = (int)(item % pl.S);
        const int jbeg = s * pl.chunk;
        const int jend = min(jbeg + pl.chunk, np);
        if (pl.mode == 0) {
            const int k = it * ITILE_A_64 + t;
            const int i = d.act[min(k, nact - 1)];
            const double xi = P[i], yi = P[np + i], zi = P[2 * np + i];
            const double vxi = P[3 * np + i], vyi = P[4 * np + i], vzi = P[5 * np + i];
            const bool busy = it * ITILE_A_64 + warp * 32 < nact;
            double g[6] = {0, 0, 0, 0, 0, 0};
            for (int jt = jbeg; jt < jend; jt += BJ64) {
                __syncthreads();
                for (int q = t; q < 7 * BJ64; q += FT) {
                    const int c = q / BJ64, jj = q % BJ64;
                    sP[c][jj] = P[(long long)c * np + jt + jj];
                }
                __syncthreads();
                if (busy) {
#pragma unroll 2
                    for (int jj = 0; jj < BJ64; jj++)
                        pair_fp64<SOFT>(sP[0][jj], sP[1][jj], sP[2][jj], sP[3][jj], sP[4][jj], sP[5][jj], sP[6][jj],
                                        xi, yi, zi, vxi, vyi, vzi, eps2, g);
                }
            }
            if (k < nact) store_partial<double>(d, nact, s, k, g);
        } else {
            const int k = it * ITILE_B_64 + warp;
            if (k < nact) {
                const int i = d.act[k];
                const double xi = P[i], yi = P[np + i], zi = P[2 * np + i];
                const double vxi = P[3 * np + i], vyi = P[4 * np + i], vzi = P[5 * np + i];
                double g[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 2
                for (int j = jbeg + lane; j < jend; j += 32)
                    pair_fp64<SOFT>(__ldg(&P[j]), __ldg(&P[np + j]), __ldg(&P[2 * np + j]), __ldg(&P[3 * np + j]),
                                    __ldg(&P[4 * np + j]), __ldg(&P[5 * np + j]), __ldg(&P[6 * np + j]), xi, yi, zi,
                                    vxi, vyi, vzi, eps2, g);
#pragma unroll
                for (int c = 0; c < 6; c++)
                    for (int o = 16; o > 0; o >>= 1) g[c] += __shfl_xor_sync(0xffffffffu, g[c], o);
                if (lane == 0) store_partial<double>(d, nact, s, k, g);
            }
        }
        finish_item<double, false>(d, nact, pl, it, tail, T, (unsigned long long *)&d.ctrl->T_acc, fa.defer);
    }
    if (tail) finalize_step(d, nact, T, pl.items);
}

struct CArgs {
    Dev d;
    int grid;      // the force plan's parameters: with tail_ok and a warp-mode plan the
    Tune tn;       // force kernel has already corrected and finalized the step
    int tail_ok;
    int mixed;
    int defer;     // the force kernel ran with FArgs::defer: its deferred plans are summed here
    int commit;    // 1: the block step's last pass (state, steps, next block time); 0: a pass
                   // before it (P(EC)^n), which only writes the corrected active records
};

// Corrects every active particle and (last CTA) turns the running minimum into the
// next block time.
template <bool MIXED>
__global__ void __launch_bounds__(CT) k_correct(CArgs ca)
{
    pdl_trigger();
    pdl_wait();
    const Dev &d = ca.d;
    Ctrl *ctrl = d.ctrl;
    const int nact = min(ctrl->nact, d.n);
    if (nact <= 0) return;
    const Plan pl = make_plan(nact, d.npad, ca.grid, ca.tn, ca.mixed != 0, d.cap);
    if (ca.tail_ok && pl.mode == 1) return;
    const int S = ca.defer && pl.late ? pl.S : 0;
    // only the CTAs that have particles to correct take part (eight per warp); the
    // others leave at once, so a small active set costs a few CTAs, not the grid
    constexpr int PER_CTA = (CT / 32) * 8;
    const int ncta = min((int)gridDim.x, (nact + PER_CTA - 1) / PER_CTA);
    if ((int)blockIdx.x >= ncta) return;
    const long long T = ctrl->T_cur;
    const int n = d.n;
    const int lane = threadIdx.x & 31;
    const int gwarp = (blockIdx.x * CT + threadIdx.x) >> 5;
    const int nwarps = (ncta * CT) >> 5;
    long long mymin = LLONG_MAX;
    int bad = 0;
    correct_slots<MIXED, false>(d, T, 0, nact, gwarp, nwarps, mymin, bad, S, nact, ca.commit == 0);
    if (bad & 2) set_err(ctrl, ST_EINVAL);
    if (bad & 1) set_err(ctrl, ST_ENONFINITE);
    if (!ca.commit) return;
    mymin = warp_min_ll(mymin);
    if (lane == 0 && mymin != LLONG_MAX) atomicMin((unsigned long long *)&ctrl->T_acc, (unsigned long long)mymin);
    // the barrier orders this CTA's minimum updates before thread 0's release fence
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
            ctrl->interactions += (double)nact * (double)n * d.n_iter;  // every pass evaluated the forces
            ctrl->epoch += 1;
            ctrl->done = 0;
        }
    }
}

// The sums k_correct takes for a deferred i-parallel plan (slot k, components c and
// 3 + c per thread), stored to fsum: the autotuner times a deferred plan's force
// launch together with this kernel, so both work decompositions are compared with
// their reductions.
template <class P>
__global__ void k_part_sum(Dev d, int nact, int S)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= 3 * nact) return;
    const int c = w / nact, k = w % nact;
    store_fsum<P>(d, c, k, part_sum<P>(d, nact, S, c, k));
    store_fsum<P>(d, 3 + c, k, part_sum<P>(d, nact, S, 3 + c, k));
}

// Initial steps after the first full force evaluation (Sec. 2.4 steps 3-4 and the
// initial step dt = eta |a| / |jerk|), and a = fsum, jerk = fsum.
// Reads the summed force of slot i into a[], jerk[] and stores it as the state's
// a and jerk (FP64 planes, or the mixed path's FP32 ones).
template <bool MIXED>
__device__ __forceinline__ void take_force(const Dev &d, int slot, int i, double a[3], double j[3])
{
    const int n = d.n;
    for (int c = 0; c < 3; c++) {
        if (MIXED) {
            const float *fs = (const float *)d.fsum;
            const float af = fs[(long long)c * n + slot], jf = fs[(long long)(3 + c) * n + slot];
            d.af[c * n + i] = af;
            d.jf[c * n + i] = jf;
            a[c] = af;
            j[c] = jf;
        } else {
            a[c] = d.fsum[(long long)c * n + slot];
            j[c] = d.fsum[(long long)(3 + c) * n + slot];
            d.a[c * n + i] = a[c];
            d.jk[c * n + i] = j[c];
        }
    }
}

template <bool MIXED>
__global__ void k_init_steps(Dev d)
{
    const int n = d.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a[3], j[3];
    take_force<MIXED>(d, i, i, a, j);
    const double na = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const double nj = sqrt(j[0] * j[0] + j[1] * j[1] + j[2] * j[2]);
    const double dt0 = d.eta * na / nj;
    long long dtau;
    if (!(dt0 < INFINITY)) {
        dtau = d.dtau_max;
    } else {
        const double q = dt0 / d.dt_min;
        if (q < 1.0) {
            dtau = 1;
        } else if (q >= (double)d.dtau_max) {
            dtau = d.dtau_max;
        } else {
            dtau = 1LL << ((int)((__double_as_longlong(q) >> 52) & 0x7FF) - 1023);
        }
    }
    d.tau[i] = 0;
    d.dtau[i] = dtau;
    d.tnext[i] = dtau;
    bool ok = true;
    for (int c = 0; c < 3; c++) ok = ok && isfinite(a[c]) && isfinite(j[c]);
    if (!ok) set_err(d.ctrl, ST_ENONFINITE);
}

// Minimum next time from scratch (after init, set_state and replayed steps).
__global__ void k_resync(Dev d)
{
    __shared__ long long s_m[32];
    long long mn = LLONG_MAX;
    for (int i = threadIdx.x; i < d.n; i += blockDim.x) mn = d.tnext[i] < mn ? d.tnext[i] : mn;
    mn = warp_min_ll(mn);
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = mn;
    __syncthreads();
    if (threadIdx.x < 32) {
        mn = threadIdx.x < (blockDim.x >> 5) ? s_m[threadIdx.x] : LLONG_MAX;
        mn = warp_min_ll(mn);
        if (threadIdx.x == 0) {
            Ctrl *c = d.ctrl;
            c->T_cur = mn;
            c->T_acc = LLONG_MAX;
            c->T_acc2[0] = LLONG_MAX;
            c->T_acc2[1] = LLONG_MAX;
            c->epoch += 1;
            c->done = 0;
            c->sel_acc = 0ull;
        }
    }
}

__global__ void k_iota(int *p, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

// ---------------------------------------------------------------- energy

// FP64 path: eu[i] = m_i sum_{j != i} m_j / sqrt(r_ij^2 + eps^2) in FP64 pairs, and
// ek[i] = m_i |v_i|^2 / 2, from the FP64 predicted planes.
__global__ void __launch_bounds__(ET) k_energy_fp64(Dev d)
{
    const int np = d.npad, n = d.n;
    const double *P = d.pd;
    __shared__ double sx[ET], sy[ET], sz[ET], sm[ET];
    const int i = blockIdx.x * ET + threadIdx.x;
    const int ii = i < n ? i : n - 1;
    const double xi = P[ii], yi = P[np + ii], zi = P[2 * np + ii];
    double phi = 0.0;
    for (int jt = 0; jt < n; jt += ET) {
        __syncthreads();
        const int j = jt + threadIdx.x;
        if (j < n) {
            sx[threadIdx.x] = P[j];
            sy[threadIdx.x] = P[np + j];
            sz[threadIdx.x] = P[2 * np + j];
            sm[threadIdx.x] = P[6 * np + j];
        }
        __syncthreads();
        const int jn = min(ET, n - jt);
        for (int jj = 0; jj < jn; jj++) {
            const double dx = sx[jj] - xi, dy = sy[jj] - yi, dz = sz[jj] - zi;
            const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, d.eps2)));
            const double term = (jt + jj == ii) ? 0.0 : sm[jj] * rsqrt(r2);
            phi += term;
        }
    }
    if (i < n) {
        const double mi = P[6 * np + i];
        const double vx = P[3 * np + i], vy = P[4 * np + i], vz = P[5 * np + i];
        d.eu[i] = mi * phi;
        d.ek[i] = 0.5 * mi * (vx * vx + vy * vy + vz * vz);
    }
}

// Mixed path: the same sums with FP32 pair arithmetic on the double-single
// j-records (one Newton step refines rsqrt.approx to about one float ulp) and a
// compensated accumulator per term, so the sum adds no error beyond the terms'
// own rounding; FP64 result; kinetic terms from the FP64 prediction of the state
// in the planes pd (k_predict_all<true, false>).
__global__ void __launch_bounds__(ET) k_energy_mixed(Dev d)
{
    const int n = d.n, np = d.npad;
    __shared__ float4 sA[ET], sB[ET];
    const int i = blockIdx.x * ET + threadIdx.x;
    const int ii = i < n ? i : n - 1;
    const float4 Ai = d.jA[ii], Bi = d.jB[ii];
    const float eps2 = d.eps2f;
    DS phi;
    phi.zero();
    for (int jt = 0; jt < np; jt += ET) {
        __syncthreads();
        sA[threadIdx.x] = d.jA[jt + threadIdx.x];
        sB[threadIdx.x] = d.jB[jt + threadIdx.x];
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < ET; jj++) {
            const float4 A = sA[jj], B = sB[jj];
            const float dx = (A.x - Ai.x) + (B.x - Bi.x);
            const float dy = (A.y - Ai.y) + (B.y - Bi.y);
            const float dz = (A.z - Ai.z) + (B.z - Bi.z);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
            float y = rsqrt_approx(r2);
            y = y * fmaf(-0.5f * r2 * y, y, 1.5f);
            const float term = (jt + jj == ii) ? 0.f : A.w * y;
            phi.add(term);
        }
    }
    if (i < n) {
        const double mi = d.m[i];
        const double vx = d.pd[3 * np + i], vy = d.pd[4 * np + i], vz = d.pd[5 * np + i];
        d.eu[i] = mi * phi.as_double();
        d.ek[i] = 0.5 * mi * (vx * vx + vy * vy + vz * vz);
    }
}

// Deterministic sums of eu and ek (one CTA, fixed order).
__global__ void k_energy_sum(Dev d)
{
    __shared__ double su[1024], sk[1024];
    double u = 0.0, k = 0.0;
    for (int i = threadIdx.x; i < d.n; i += blockDim.x) {
        u += d.eu[i];
        k += d.ek[i];
    }
    su[threadIdx.x] = u;
    sk[threadIdx.x] = k;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            su[threadIdx.x] += su[threadIdx.x + o];
            sk[threadIdx.x] += sk[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        d.ctrl->K = sk[0];
        d.ctrl->U = -0.5 * su[0];
    }
}

// Sets the block time and active count of a caller-given step.
__global__ void k_set_step(Ctrl *c, long long T, int nact)
{
    c->T_cur = T;
    c->nact = nact;
}

__global__ void k_set_tick_end(Ctrl *c, long long tick_end) { c->tick_end = tick_end; }


// ---------------------------------------------------------------- fused block steps

constexpr int BAR_WORDS = 32;            // the barrier counter sits alone in a 128-byte line
constexpr int BAR_SPIN_LIMIT = 1 << 24;  // bounded wait

// Polls *ctr until it reaches target, at most `limit` times; false if it gave up.
// The bounded wait of the grid barrier (and of the failure-detection probe).
__device__ __forceinline__ bool wait_counter_ge(const unsigned long long *ctr, unsigned long long target, int limit)
{
    int spins = 0;
    while (*(volatile const unsigned long long *)ctr < target)
        if (++spins > limit) return false;
    return true;
}

// Grid-wide barrier for a co-resident (cooperative) grid of nb CTAs: one 64-bit
// counter that only grows; the k-th barrier is passed when the counter reaches
// nb * k, so each CTA waits for the multiple of nb above the value its own arrival
// returned.  Thread 0's fences release the CTA's writes before arriving and
// acquire the others' after passing.  The wait is bounded: on time-out the device
// flag records GD_ETIMEOUT and the CTA goes on (the results are then void, but the
// kernel ends).
__device__ __forceinline__ void grid_sync(unsigned int *bar, Ctrl *ctrl)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long *ctr = (unsigned long long *)bar;
        const unsigned long long nb = gridDim.x;
        __threadfence();
        const unsigned long long old = atomicAdd(ctr, 1ull);
        const unsigned long long target = (old / nb + 1) * nb;
        if (!wait_counter_ge(ctr, target, BAR_SPIN_LIMIT)) set_err(ctrl, ST_ETIMEOUT);
        __threadfence();
    }
    __syncthreads();
}

// Failure-detection probe: one thread waits, with the grid barrier's bounded
// wait, for a counter that nothing advances (the upper half of the barrier
// array, which the barrier does not use), so the wait runs out after `limit`
// polls and the device flag records GD_ETIMEOUT; the kernel then ends normally.
__global__ void k_wait_probe(Dev d, int limit)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned long long *ctr = (const unsigned long long *)(d.bar + BAR_WORDS / 2);
    const unsigned long long target = *(volatile const unsigned long long *)ctr + 1ull;
    if (!wait_counter_ge(ctr, target, limit)) set_err(d.ctrl, ST_ETIMEOUT);
}

struct SArgs {
    Dev d;
    int plan_grid;  // grid size the force plan assumes (the same as the three-kernel path)
    Tune tn;
    int nchunks;
    int max_steps;
};

// Up to max_steps block steps in one cooperative launch (all CTAs resident).  Per
// step: select + predict, grid barrier, force -- with the correction done by the
// last CTA of each i-tile when the tiles are small (warp mode) -- grid barrier, and
// in i-parallel mode a separate correction pass and a third barrier.  The block
// time of the next step is the atomic minimum gathered during the step (slot by
// step parity), read after the last barrier.  Stops early once the block time
// passes tick_end.  Computes exactly what the three-kernel step computes.
template <bool SOFT>
__global__ void __launch_bounds__(FT, 4) k_steps(SArgs a)
{
    const Dev &d = a.d;
    Ctrl *ctrl = d.ctrl;
    const unsigned base = ctrl->epoch;
    const long long tick_end = ctrl->tick_end;
    long long T = ctrl->T_cur;
    int s = 0;
    bool capped = true;
    for (; s < a.max_steps; s++) {
        const unsigned g = base + (unsigned)s;
        unsigned long long *acc = (unsigned long long *)&ctrl->T_acc2[g & 1];
        if (s > 0) T = (long long)ldc((const unsigned long long *)&ctrl->T_acc2[(g - 1) & 1]);
        if (T > tick_end) {
            capped = false;
            break;
        }
        const unsigned long long t0 = global_ns();
        phase_select<true, true>(d, T, -1, a.nchunks, acc);
        grid_sync(d.bar, ctrl);
        const unsigned long long t1 = global_ns();
        const int nact = min(ldc(&ctrl->nact), d.n);
        if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->T_acc2[(g - 1) & 1] = LLONG_MAX;
        const Plan pl = make_plan(nact, d.npad, a.plan_grid, a.tn, true, d.cap);
        const bool tail = pl.mode == 1;
        if (nact > 0) phase_force_mixed<SOFT, true>(d, nact, pl, tail, T, acc);
        grid_sync(d.bar, ctrl);
        const unsigned long long t2 = global_ns();
        if (!tail && nact > 0) {
            long long mymin = LLONG_MAX;
            int bad = 0;
            const int gwarp = (blockIdx.x * FT + threadIdx.x) >> 5;
            const int nwarps = (gridDim.x * FT) >> 5;
            correct_slots<true, true>(d, T, 0, nact, gwarp, nwarps, mymin, bad);
            if (bad & 2) set_err(ctrl, ST_EINVAL);
            if (bad & 1) set_err(ctrl, ST_ENONFINITE);
            mymin = warp_min_ll(mymin);
            if ((threadIdx.x & 31) == 0 && mymin != LLONG_MAX) atomicMin(acc, (unsigned long long)mymin);
            grid_sync(d.bar, ctrl);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const unsigned long long t3 = global_ns();
            ctrl->ph_ns[0] += t1 - t0;
            ctrl->ph_ns[1] += t2 - t1;
            ctrl->ph_ns[2] += t3 - t2;
            ctrl->T_last = T;
            ctrl->last_nact = nact;
            ctrl->nblock += 1;
            ctrl->nsteps += nact;
            ctrl->interactions += (double)nact * (double)d.n;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (s > 0) {
            const unsigned gl = base + (unsigned)s - 1;
            if (capped) T = (long long)ldc((const unsigned long long *)&ctrl->T_acc2[gl & 1]);
            ctrl->T_acc2[gl & 1] = LLONG_MAX;
        }
        ctrl->T_cur = T;
        ctrl->epoch = base + (unsigned)s + 1;
    }
}

}  // namespace gdk
