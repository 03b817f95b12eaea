// gravidy.cu -- GB300 (sm_103a) kernels and C ABI of the Hermite-4 block-time-step
// N-body integrator of GraviDy (arXiv 1702.00440).  The ABI is declared in
// include/gravidy.h.
//
// One block step (Sec. 2.4 steps 5-7) is three kernels with no host round trip:
//   k_select_predict  predict every particle to the block time (step 7a) and
//                     compact the active ones in ascending index order (step 5)
//                     with a single-pass decoupled look-back scan; also start the
//                     minimum of the next block time over the inactive ones.
//   k_force           force and jerk of the active set against all N predicted
//                     particles (step 7c, Sec. 2.5): a persistent kernel over
//                     (i-tile x j-chunk) work items; the j-range is split when the
//                     active set is small and partial sums go to scratch.
//   k_correct         sum the j-split partials (step 7c-iii), correct (7d), take
//                     Aarseth's step (Sec. 3.2), quantise it to the block scheme,
//                     keep the new force as the old one (step 6), and finish the
//                     minimum that gives the next block time.
// The block time, active count and all bookkeeping stay on the device, so a run
// of block steps can be captured once in a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gravidy.h"

namespace {

// ---------------------------------------------------------------- constants

constexpr int FT = 128;            // force kernel threads per CTA
constexpr int BJ = 128;            // j-tile (mixed) and padding granule of the j-arrays
constexpr int BJ64 = 64;           // j-tile of the FP64 i-parallel mode
constexpr int ITILE_A_MIX = 2 * FT;  // i-parallel mode: 2 active particles per thread
constexpr int ITILE_A_64 = FT;       // FP64 i-parallel mode: 1 per thread
constexpr int ITILE_B_MIX = 2 * (FT / 32);  // warp mode: 2 per warp, lanes split j
constexpr int ITILE_B_64 = FT / 32;         // FP64 warp mode: 1 per warp
constexpr int JCHUNK_MIN = 256;    // smallest j-chunk of a split
constexpr int FOLD_B = 16;         // warp mode: j-iterations per lane between FP64 folds
constexpr int ST = 128;            // select/predict kernel threads per CTA
constexpr int CT = 128;            // corrector threads per CTA
constexpr int ET = 128;            // energy kernel threads per CTA
constexpr int SPIN_LIMIT = 1 << 22;  // bounded device waits
constexpr float PAD_FAR_F = 1.0e18f;
constexpr double PAD_FAR_D = 1.0e30;

// ---------------------------------------------------------------- device control block

struct Ctrl {
    long long T_cur;       // block time of the next step (ticks)
    long long T_acc;       // running minimum of next times for the step after it
    long long T_last;      // block time of the last finished step
    long long tick_end;    // steps whose block time is above this are skipped
    long long nblock;      // block steps
    long long nsteps;      // particle steps
    double interactions;   // sum of nact * n
    double K, U;           // energy results
    int nact;              // active count of the current step
    int last_nact;
    unsigned int epoch;    // look-back tag, advanced once per step
    unsigned int ticket;   // logical CTA counter of k_select_predict
    unsigned int done;     // finished-CTA counter of k_correct
    int err;               // first device-side fault (gd_status), 0 = none
};

__device__ __forceinline__ void set_err(Ctrl *c, int code) { atomicCAS(&c->err, 0, code); }

// ---------------------------------------------------------------- device state

struct Dev {
    int n, npad;
    double dt_min;
    long long dtau_max;
    double eta;
    double eps2;
    float eps2f;
    // FP64 state at each particle's own time, structure of arrays (plane c at +c*n)
    double *x, *v, *a, *jk, *m;
    long long *tau, *dtau, *tnext;
    // predicted j-records, mixed: A = (x_hi, y_hi, z_hi, m), B = (x_lo, y_lo, z_lo, vx),
    // C = (vy, vz); padded to npad with massless far-away particles
    float4 *jA, *jB;
    float2 *jC;
    // predicted j-records, FP64: 7 planes of npad (x, y, z, vx, vy, vz, m)
    double *pd;
    int *act;                 // active list
    double *part;             // j-split partial sums, (s*6 + c) * nact + k
    long long cap;            // partial capacity (entries per component)
    unsigned long long *status;  // look-back words of k_select_predict
    double *eu, *ek;          // per-particle energy terms
    double *fout;             // 6 * n summed forces for the gd_force hook
    int *nact_hist;           // nact of each step slot of a captured graph
    Ctrl *ctrl;
};

// ---------------------------------------------------------------- force plan

struct Plan {
    int mode;     // 0 = i-parallel, 1 = warp j-parallel
    int itile;    // active particles per work item
    int itiles;
    int S;        // j-split factor
    int chunk;    // j per split (multiple of BJ)
    long long items;
};

__host__ __device__ inline Plan make_plan(int nact, int npad, int grid, int mode_cut, int jsplit,
                                          bool mixed, long long cap)
{
    Plan p;
    p.mode = nact >= mode_cut ? 0 : 1;
    p.itile = p.mode == 0 ? (mixed ? ITILE_A_MIX : ITILE_A_64) : (mixed ? ITILE_B_MIX : ITILE_B_64);
    p.itiles = (nact + p.itile - 1) / p.itile;
    if (p.itiles < 1) p.itiles = 1;
    long long S;
    if (jsplit > 0) {
        S = jsplit;
    } else {
        long long target = 2LL * grid;
        S = (target + p.itiles - 1) / p.itiles;
    }
    long long smax = npad / JCHUNK_MIN;
    if (smax < 1) smax = 1;
    if (S > smax) S = smax;
    if (S < 1) S = 1;
    if (nact > 0 && S * (long long)nact > cap) S = cap / nact;
    if (S < 1) S = 1;
    int tiles = npad / BJ;
    int tpc = (int)((tiles + S - 1) / S);
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

__device__ __forceinline__ long long warp_min_ll(long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Taylor prediction of particle i over dt (Sec. 2.4 step 7a), FP64.
__device__ __forceinline__ void predict64(const Dev &d, int i, double dt, double xp[3], double vp[3])
{
    const int n = d.n;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        double x0 = d.x[c * n + i], v0 = d.v[c * n + i], a0 = d.a[c * n + i], j0 = d.jk[c * n + i];
        xp[c] = x0 + dt * (v0 + dt * (0.5 * a0 + dt * (j0 * (1.0 / 6.0))));
        vp[c] = v0 + dt * (a0 + dt * (0.5 * j0));
    }
}

// Store the predicted particle as the record the force kernel reads.
template <bool MIXED>
__device__ __forceinline__ void store_jrec(const Dev &d, int i, const double xp[3], const double vp[3],
                                           double mi)
{
    if (MIXED) {
        float h0 = __double2float_rn(xp[0]), h1 = __double2float_rn(xp[1]), h2 = __double2float_rn(xp[2]);
        float l0 = __double2float_rn(xp[0] - (double)h0);
        float l1 = __double2float_rn(xp[1] - (double)h1);
        float l2 = __double2float_rn(xp[2] - (double)h2);
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

// Predicts every particle to T = ctrl->T_cur and writes the ascending list of the
// particles whose next time equals T.  Logical CTA order comes from a ticket so a
// CTA only ever waits on CTAs that are already running; every wait is bounded.
// `slot` >= 0 records nact in nact_hist[slot] (timed graph runs).
template <bool MIXED>
__global__ void __launch_bounds__(ST) k_select_predict(Dev d, int slot)
{
    Ctrl *ctrl = d.ctrl;
    const long long T = ctrl->T_cur;
    if (T > ctrl->tick_end) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctrl->nact = 0;
            if (slot >= 0) d.nact_hist[slot] = 0;
        }
        return;
    }
    __shared__ unsigned s_blk, s_excl;
    __shared__ unsigned s_wcnt[ST / 32];
    __shared__ long long s_wmin[ST / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_blk = atomicAdd(&ctrl->ticket, 1u);
    __syncthreads();
    const unsigned blk = s_blk;
    if (blk >= gridDim.x) {  // stale ticket counter: record and leave (uniform per CTA)
        if (threadIdx.x == 0) set_err(ctrl, GD_ESTATE);
        return;
    }
    const unsigned epoch = ctrl->epoch;
    const int i = (int)blk * ST + threadIdx.x;
    bool act = false;
    long long tn = LLONG_MAX;
    if (i < d.n) {
        tn = d.tnext[i];
        act = (tn == T);
        double dt = (double)(T - d.tau[i]) * d.dt_min;
        double xp[3], vp[3];
        predict64(d, i, dt, xp, vp);
        store_jrec<MIXED>(d, i, xp, vp, d.m[i]);
    }
    // minimum next time of the inactive particles -> next block time candidate
    long long mn = warp_min_ll(act ? LLONG_MAX : tn);
    const unsigned ballot = __ballot_sync(0xffffffffu, act);
    if (lane == 0) {
        s_wcnt[warp] = __popc(ballot);
        s_wmin[warp] = mn;
    }
    __syncthreads();
    if (warp == 0) {
        unsigned cnt = lane < ST / 32 ? s_wcnt[lane] : 0u;
        long long wm = lane < ST / 32 ? s_wmin[lane] : LLONG_MAX;
        // inclusive scan of the warp counts
        unsigned incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
        if (lane < ST / 32) s_wcnt[lane] = incl - cnt;  // exclusive offsets
        wm = warp_min_ll(wm);
        if (lane == 0 && wm != LLONG_MAX) atomicMin((unsigned long long *)&ctrl->T_acc, (unsigned long long)wm);
        // decoupled look-back over the logical predecessors
        const unsigned ep = epoch & 0x3FFFFFFFu;
        unsigned excl = 0;
        if (blk == 0) {
            if (lane == 0) atomicExch(&d.status[0], lb_pack(ep, 2u, total));
        } else {
            if (lane == 0) atomicExch(&d.status[blk], lb_pack(ep, 1u, total));
            int base = (int)blk - 1;
            int spins = 0;
            for (;;) {
                const int p = base - lane;
                unsigned f = 2u, val = 0u;
                if (p >= 0) {
                    unsigned long long w = ld_volatile_u64(&d.status[p]);
                    f = ((unsigned)(w >> 34) == ep) ? (unsigned)((w >> 32) & 3u) : 0u;
                    val = (unsigned)w;
                }
                const unsigned notready = __ballot_sync(0xffffffffu, f == 0u);
                const unsigned prefix = __ballot_sync(0xffffffffu, f == 2u);
                const int first = prefix ? __ffs(prefix) - 1 : 31;
                const unsigned need = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
                if (notready & need) {
                    if (++spins > SPIN_LIMIT) {
                        if (lane == 0) set_err(ctrl, GD_ETIMEOUT);
                        break;
                    }
                    __nanosleep(64);
                    continue;
                }
                unsigned contrib = lane <= first ? val : 0u;
                for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
                excl += contrib;
                if (prefix) break;
                base -= 32;
            }
            if (lane == 0) atomicExch(&d.status[blk], lb_pack(ep, 2u, excl + total));
        }
        if (lane == 0) {
            s_excl = excl;
            if (blk == gridDim.x - 1) {
                int na = (int)(excl + total);
                if (excl + total > (unsigned)d.n) {
                    set_err(ctrl, GD_ETIMEOUT);
                    na = 0;
                }
                ctrl->nact = na;
                if (slot >= 0) d.nact_hist[slot] = na;
            }
        }
    }
    __syncthreads();
    if (act) {
        unsigned pos = s_excl + s_wcnt[warp] + __popc(ballot & ((1u << lane) - 1u));
        if (pos < (unsigned)d.n) d.act[pos] = i;
    }
}

// Predict all particles to `tick` (no selection).  Used by the hooks and by gd_energy.
template <bool MIXED>
__global__ void k_predict_all(Dev d, long long tick)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    double dt = (double)(tick - d.tau[i]) * d.dt_min;
    double xp[3], vp[3];
    predict64(d, i, dt, xp, vp);
    store_jrec<MIXED>(d, i, xp, vp, d.m[i]);
}

// Padding records: massless particles far away, so the inner loops need no tail test.
__global__ void k_init_pads(Dev d)
{
    int i = d.n + blockIdx.x * blockDim.x + threadIdx.x;
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
// on double-single positions: r = x_j - x_i from hi and lo parts separately, so
// the difference keeps the bits of the FP64 positions.
//   a += m r / s^3,   jerk += m (v - 3 (r.v) r / s^2) / s^3,   s^2 = r^2 + eps^2
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
    const float mr3 = A.w * rinv * rinv2;
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
    int mode_cut;
    int jsplit;
};

__device__ __forceinline__ void store_partial(const Dev &d, int nact, int s, int k, const double f[6])
{
    double *p = d.part + (long long)s * 6 * nact + k;
#pragma unroll
    for (int c = 0; c < 6; c++) p[(long long)c * nact] = f[c];
}

__device__ __forceinline__ void warp_sum6(double f[6])
{
#pragma unroll
    for (int c = 0; c < 6; c++)
        for (int o = 16; o > 0; o >>= 1) f[c] += __shfl_xor_sync(0xffffffffu, f[c], o);
}

// ---------------------------------------------------------------- kernel: force (mixed)

template <bool SOFT>
__global__ void __launch_bounds__(FT, 4) k_force_mixed(FArgs fa)
{
    const Dev &d = fa.d;
    const int nact = min(d.ctrl->nact, d.n);
    if (nact <= 0) return;
    const Plan pl = make_plan(nact, d.npad, fa.grid, fa.mode_cut, fa.jsplit, true, d.cap);
    const float eps2 = d.eps2f;
    __shared__ float4 sA[BJ], sB[BJ];
    __shared__ float2 sC[BJ];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (long long item = blockIdx.x; item < pl.items; item += gridDim.x) {
        const int it = (int)(item / pl.S), s = (int)(item % pl.S);
        const int jbeg = s * pl.chunk;
        const int jend = min(jbeg + pl.chunk, d.npad);
        if (pl.mode == 0) {
            // i-parallel: thread t owns active slots k0 and k1; j-tiles staged in shared memory
            const int k0 = it * ITILE_A_MIX + t, k1 = k0 + FT;
            const int i0 = d.act[min(k0, nact - 1)], i1 = d.act[min(k1, nact - 1)];
            const float4 A0 = d.jA[i0], B0 = d.jB[i0];
            const float2 C0 = d.jC[i0];
            const float4 A1 = d.jA[i1], B1 = d.jB[i1];
            const float2 C1 = d.jC[i1];
            const bool busy = it * ITILE_A_MIX + warp * 32 < nact;  // warp has a real slot
            double g0[6] = {0, 0, 0, 0, 0, 0}, g1[6] = {0, 0, 0, 0, 0, 0};
            for (int jt = jbeg; jt < jend; jt += BJ) {
                __syncthreads();
                sA[t] = d.jA[jt + t];
                sB[t] = d.jB[jt + t];
                sC[t] = d.jC[jt + t];
                __syncthreads();
                if (busy) {
                    float f0[6] = {0, 0, 0, 0, 0, 0}, f1[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 4
                    for (int jj = 0; jj < BJ; jj++) {
                        const float4 A = sA[jj], B = sB[jj];
                        const float2 C = sC[jj];
                        pair_mixed<SOFT>(A, B, C, A0.x, A0.y, A0.z, B0.x, B0.y, B0.z, B0.w, C0.x, C0.y, eps2, f0);
                        pair_mixed<SOFT>(A, B, C, A1.x, A1.y, A1.z, B1.x, B1.y, B1.z, B1.w, C1.x, C1.y, eps2, f1);
                    }
#pragma unroll
                    for (int c = 0; c < 6; c++) {
                        g0[c] += (double)f0[c];
                        g1[c] += (double)f1[c];
                    }
                }
            }
            if (k0 < nact) store_partial(d, nact, s, k0, g0);
            if (k1 < nact) store_partial(d, nact, s, k1, g1);
        } else {
            // warp j-parallel: warp w owns slots k0, k0+1; its lanes split the j-chunk
            const int k0 = it * ITILE_B_MIX + 2 * warp;
            if (k0 < nact) {
                const bool has1 = k0 + 1 < nact;
                const int i0 = d.act[k0], i1 = d.act[has1 ? k0 + 1 : k0];
                const float4 A0 = d.jA[i0], B0 = d.jB[i0];
                const float2 C0 = d.jC[i0];
                const float4 A1 = d.jA[i1], B1 = d.jB[i1];
                const float2 C1 = d.jC[i1];
                double g0[6] = {0, 0, 0, 0, 0, 0}, g1[6] = {0, 0, 0, 0, 0, 0};
                for (int jb = jbeg; jb < jend; jb += 32 * FOLD_B) {
                    const int je = min(jb + 32 * FOLD_B, jend);
                    float f0[6] = {0, 0, 0, 0, 0, 0}, f1[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 4
                    for (int j = jb + lane; j < je; j += 32) {
                        const float4 A = __ldg(&d.jA[j]), B = __ldg(&d.jB[j]);
                        const float2 C = __ldg(&d.jC[j]);
                        pair_mixed<SOFT>(A, B, C, A0.x, A0.y, A0.z, B0.x, B0.y, B0.z, B0.w, C0.x, C0.y, eps2, f0);
                        pair_mixed<SOFT>(A, B, C, A1.x, A1.y, A1.z, B1.x, B1.y, B1.z, B1.w, C1.x, C1.y, eps2, f1);
                    }
#pragma unroll
                    for (int c = 0; c < 6; c++) {
                        g0[c] += (double)f0[c];
                        g1[c] += (double)f1[c];
                    }
                }
                warp_sum6(g0);
                warp_sum6(g1);
                if (lane == 0) {
                    store_partial(d, nact, s, k0, g0);
                    if (has1) store_partial(d, nact, s, k0 + 1, g1);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- kernel: force (FP64)

template <bool SOFT>
__global__ void __launch_bounds__(FT, 4) k_force_fp64(FArgs fa)
{
    const Dev &d = fa.d;
    const int nact = min(d.ctrl->nact, d.n);
    if (nact <= 0) return;
    const Plan pl = make_plan(nact, d.npad, fa.grid, fa.mode_cut, fa.jsplit, false, d.cap);
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
            if (k < nact) store_partial(d, nact, s, k, g);
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
                warp_sum6(g);
                if (lane == 0) store_partial(d, nact, s, k, g);
            }
        }
    }
}

// ---------------------------------------------------------------- partial sums

struct RArgs {
    Dev d;
    int grid;
    int mode_cut;
    int jsplit;
    bool mixed;
};

// Sum of the S partials of active slot k (FP64, fixed order).
__device__ __forceinline__ void sum_partials(const Dev &d, int nact, int S, int k, double f[6])
{
#pragma unroll
    for (int c = 0; c < 6; c++) f[c] = 0.0;
    for (int s = 0; s < S; s++) {
        const double *p = d.part + (long long)s * 6 * nact + k;
#pragma unroll
        for (int c = 0; c < 6; c++) f[c] += p[(long long)c * nact];
    }
}

// out[c * ostride + k] = summed component c of slot k (c < 3: a, c >= 3: jerk at o2)
__global__ void k_reduce_partials(RArgs ra, double *oa, double *oj, int ostride)
{
    const Dev &d = ra.d;
    const int nact = min(d.ctrl->nact, d.n);
    if (nact <= 0) return;
    const Plan pl = make_plan(nact, d.npad, ra.grid, ra.mode_cut, ra.jsplit, ra.mixed, d.cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nact; k += gridDim.x * blockDim.x) {
        double f[6];
        sum_partials(d, nact, pl.S, k, f);
        for (int c = 0; c < 3; c++) {
            oa[(long long)c * ostride + k] = f[c];
            oj[(long long)c * ostride + k] = f[c + 3];
        }
    }
}

// ---------------------------------------------------------------- corrector + time step

__device__ __forceinline__ double norm3(const double a[3]) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

// Power-of-two block step after a correction at tick T (same rules as the initial
// quantisation: steps are powers of two of dt_min in [1, dtau_max] ticks; a step may
// shrink to any smaller power of two, and grow by 2 only at a time that is a
// multiple of twice the old step).  A NaN estimate counts as +infinity.
__device__ __forceinline__ long long next_block_step(double dtn, long long dtau_old, long long T, double dt_min,
                                                     long long dtau_max)
{
    const double dt_old = (double)dtau_old * dt_min;
    if (dtn < dt_old) {
        const double q = dtn / dt_min;
        if (q < 1.0) return 1;
        const int e = (int)((__double_as_longlong(q) >> 52) & 0x7FF) - 1023;  // floor(log2 q), q normal
        return 1LL << e;
    }
    if (!(dtn == dtn) || dtn >= 2.0 * dt_old) {
        if (2 * dtau_old <= dtau_max && (T & (2 * dtau_old - 1)) == 0) return 2 * dtau_old;
    }
    return dtau_old;
}

__device__ __forceinline__ long long first_block_step(double dt, double dt_min, long long dtau_max)
{
    if (!(dt < INFINITY)) return dtau_max;
    const double q = dt / dt_min;
    if (q < 1.0) return 1;
    if (q >= (double)dtau_max) return dtau_max;
    const int e = (int)((__double_as_longlong(q) >> 52) & 0x7FF) - 1023;
    return 1LL << e;
}

__device__ __forceinline__ bool finite6(const double *a, const double *b)
{
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; c++) ok = ok && isfinite(a[c]) && isfinite(b[c]);
    return ok;
}

// Correction of one active particle (Sec. 2.4 step 7d, ma92 Hermite scheme) with the
// new force a1/j1 at block time T; returns its new next time.
// bad |= 1: non-finite result; bad |= 2: the particle is not behind T.
__device__ __forceinline__ long long correct_one(const Dev &d, int i, long long T, const double f[6], int &bad)
{
    const int n = d.n;
    const long long tau0 = d.tau[i];
    if (tau0 >= T) {
        bad |= 2;
        return d.tnext[i];
    }
    const double dt = (double)(T - tau0) * d.dt_min;
    double xp[3], vp[3];
    predict64(d, i, dt, xp, vp);
    const double a1[3] = {f[0], f[1], f[2]}, j1[3] = {f[3], f[4], f[5]};
    double a2[3], a3[3], a2e[3], x1[3], v1[3];
    const double dt2 = dt * dt, dt3 = dt2 * dt, dt4 = dt3 * dt, dt5 = dt4 * dt;
    const double idt2 = 1.0 / dt2, idt3 = idt2 / dt;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const double a0 = d.a[c * n + i], j0 = d.jk[c * n + i];
        const double da = a0 - a1[c];
        // derivatives at the start of the step from the end-point values
        a2[c] = (-6.0 * da - dt * (4.0 * j0 + 2.0 * j1[c])) * idt2;
        a3[c] = (12.0 * da + 6.0 * dt * (j0 + j1[c])) * idt3;
        x1[c] = xp[c] + a2[c] * (dt4 * (1.0 / 24.0)) + a3[c] * (dt5 * (1.0 / 120.0));
        v1[c] = vp[c] + a2[c] * (dt3 * (1.0 / 6.0)) + a3[c] * (dt4 * (1.0 / 24.0));
        a2e[c] = a2[c] + dt * a3[c];  // second derivative at the end of the step
    }
    // Aarseth criterion at the end of the step
    const double na = norm3(a1), nj = norm3(j1), n2 = norm3(a2e), n3 = norm3(a3);
    const double dtn = sqrt(d.eta * (na * n2 + nj * nj) / (nj * n3 + n2 * n2));
    const long long dtau = next_block_step(dtn, d.dtau[i], T, d.dt_min, d.dtau_max);
    if (!finite6(x1, v1) || !finite6(a1, j1)) bad |= 1;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        d.x[c * n + i] = x1[c];
        d.v[c * n + i] = v1[c];
        d.a[c * n + i] = a1[c];
        d.jk[c * n + i] = j1[c];
    }
    d.tau[i] = T;
    d.dtau[i] = dtau;
    const long long tn = T + dtau;
    d.tnext[i] = tn;
    return tn;
}

// Reduces the j-split partials, corrects every active particle, and (last CTA)
// turns the running minimum into the next block time.  finalize = false leaves the
// block-time bookkeeping alone (replayed steps resynchronise it afterwards).
__global__ void __launch_bounds__(CT) k_correct(RArgs ra)
{
    const Dev &d = ra.d;
    Ctrl *ctrl = d.ctrl;
    const int nact = min(ctrl->nact, d.n);
    if (nact <= 0) return;
    const long long T = ctrl->T_cur;
    const Plan pl = make_plan(nact, d.npad, ra.grid, ra.mode_cut, ra.jsplit, ra.mixed, d.cap);
    const int lane = threadIdx.x & 31;
    long long mymin = LLONG_MAX;
    int bad = 0;
    if (pl.S <= 8) {
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nact; k += gridDim.x * blockDim.x) {
            double f[6];
            sum_partials(d, nact, pl.S, k, f);
            long long tn = correct_one(d, d.act[k], T, f, bad);
            mymin = tn < mymin ? tn : mymin;
        }
    } else {
        const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int nw = (gridDim.x * blockDim.x) >> 5;
        for (int k = wid; k < nact; k += nw) {
            double f[6] = {0, 0, 0, 0, 0, 0};
            for (int s = lane; s < pl.S; s += 32) {
                const double *p = d.part + (long long)s * 6 * nact + k;
#pragma unroll
                for (int c = 0; c < 6; c++) f[c] += p[(long long)c * nact];
            }
            warp_sum6(f);
            if (lane == 0) {
                long long tn = correct_one(d, d.act[k], T, f, bad);
                mymin = tn < mymin ? tn : mymin;
            }
        }
    }
    if (bad & 2) set_err(ctrl, GD_EINVAL);
    if (bad & 1) set_err(ctrl, GD_ENONFINITE);
    mymin = warp_min_ll(mymin);
    if (lane == 0 && mymin != LLONG_MAX) {
        atomicMin((unsigned long long *)&ctrl->T_acc, (unsigned long long)mymin);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&ctrl->done, 1u);
        if (prev == gridDim.x - 1) {
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
            ctrl->ticket = 0;
            ctrl->done = 0;
        }
    }
}

// Initial steps after the first full force evaluation (Sec. 2.4 steps 3-4 and the
// initial step dt = eta |a| / |jerk|).
__global__ void k_init_steps(Dev d)
{
    const int n = d.n;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a[3] = {d.a[i], d.a[n + i], d.a[2 * n + i]};
    const double j[3] = {d.jk[i], d.jk[n + i], d.jk[2 * n + i]};
    const double dt0 = d.eta * norm3(a) / norm3(j);
    const long long dtau = first_block_step(dt0, d.dt_min, d.dtau_max);
    d.tau[i] = 0;
    d.dtau[i] = dtau;
    d.tnext[i] = dtau;
    if (!finite6(a, j)) set_err(d.ctrl, GD_ENONFINITE);
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
            c->epoch += 1;
            c->ticket = 0;
            c->done = 0;
        }
    }
}

__global__ void k_iota(int *p, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

// ---------------------------------------------------------------- energy (FP64 pairs)

// eu[i] = m_i sum_{j != i} m_j / sqrt(r_ij^2 + eps^2), ek[i] = m_i |v_i|^2 / 2, from
// the FP64 predicted planes.
__global__ void __launch_bounds__(ET) k_energy_terms(Dev d)
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

}  // namespace

// ================================================================ host side

struct gd_ctx {
    gd_opts opt;
    int dev;
    cudaStream_t stream;
    bool own_stream;
    Dev d;
    int grid_force, grid_sel, grid_corr;
    bool mixed, soft;
    Ctrl *h_ctrl;  // pinned mirror
    Ctrl *h_snap;  // two pinned snapshots for the pipelined gd_evolve
    cudaEvent_t ev_snap[2];
    double *h_stage;  // pinned staging: 12 n doubles then 3 n int64
    long long launches;  // kernels launched by this context
    cudaGraphExec_t graph;
    int graph_steps;
    std::vector<cudaEvent_t> ev;  // force timing pairs, one per graph slot (or eager)
    int *h_hist;                  // pinned copy of nact_hist
    double force_ms;
    long long force_launches;
    double force_interactions;
    std::string err;
    int sticky;
};

static thread_local std::string g_init_err;

namespace {

int fail(gd_ctx *c, int code, const std::string &msg)
{
    if (c) {
        c->err = msg;
    } else {
        g_init_err = msg;
    }
    return code;
}

int cuda_fail(gd_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, GD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);       \
    } while (0)

bool is_pow2(double x)
{
    if (!(x > 0) || !std::isfinite(x)) return false;
    int e;
    double f = std::frexp(x, &e);
    return f == 0.5;
}

RArgs rargs(const gd_ctx *c) { return RArgs{c->d, c->grid_force, c->opt.mode_cut, c->opt.jsplit, c->mixed}; }
FArgs fargs(const gd_ctx *c) { return FArgs{c->d, c->grid_force, c->opt.mode_cut, c->opt.jsplit}; }

int launch_force(gd_ctx *c)
{
    FArgs fa = fargs(c);
    c->launches += 1;
    if (c->mixed) {
        if (c->soft)
            k_force_mixed<true><<<c->grid_force, FT, 0, c->stream>>>(fa);
        else
            k_force_mixed<false><<<c->grid_force, FT, 0, c->stream>>>(fa);
    } else {
        if (c->soft)
            k_force_fp64<true><<<c->grid_force, FT, 0, c->stream>>>(fa);
        else
            k_force_fp64<false><<<c->grid_force, FT, 0, c->stream>>>(fa);
    }
    return GD_OK;
}

void launch_predict_all(gd_ctx *c, long long tick, bool mixed_records)
{
    const int g = (c->d.n + 255) / 256;
    c->launches += 1;
    if (mixed_records)
        k_predict_all<true><<<g, 256, 0, c->stream>>>(c->d, tick);
    else
        k_predict_all<false><<<g, 256, 0, c->stream>>>(c->d, tick);
}

// One free-running block step: select+predict, force, correct.
void launch_step(gd_ctx *c, int slot, cudaEvent_t e0, cudaEvent_t e1, bool capturing)
{
    c->launches += 2;  // select + correct (launch_force counts itself)
    if (c->mixed)
        k_select_predict<true><<<c->grid_sel, ST, 0, c->stream>>>(c->d, slot);
    else
        k_select_predict<false><<<c->grid_sel, ST, 0, c->stream>>>(c->d, slot);
    if (e0) cudaEventRecordWithFlags(e0, c->stream, capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
    launch_force(c);
    if (e1) cudaEventRecordWithFlags(e1, c->stream, capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
    k_correct<<<c->grid_corr, CT, 0, c->stream>>>(rargs(c));
}

int sync_ctrl(gd_ctx *c)
{
    CK(cudaMemcpyAsync(c->h_ctrl, c->d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->h_ctrl->err != 0) {
        c->sticky = c->h_ctrl->err;
        return fail(c, c->sticky, c->sticky == GD_ENONFINITE ? "non-finite value in the integration state"
                                  : c->sticky == GD_ETIMEOUT ? "bounded device wait gave up"
                                  : c->sticky == GD_EINVAL   ? "invalid replayed step"
                                                             : "device fault");
    }
    return GD_OK;
}

int check_usable(gd_ctx *c)
{
    if (!c) return fail(nullptr, GD_EINVAL, "null context");
    if (c->sticky) return fail(c, c->sticky, "context is in an error state: " + c->err);
    cudaError_t e = cudaSetDevice(c->dev);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return GD_OK;
}

template <class T>
int dalloc(gd_ctx *c, T **p, size_t count)
{
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T) + 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(c, GD_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return GD_OK;
}

void free_all(gd_ctx *c)
{
    Dev &d = c->d;
    void *ps[] = {d.x, d.v, d.a, d.jk, d.m, d.tau, d.dtau, d.tnext, d.jA, d.jB, d.jC, d.pd,
                  d.act, d.part, d.status, d.eu, d.ek, d.fout, d.nact_hist, d.ctrl};
    for (void *p : ps)
        if (p) cudaFree(p);
    if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
    if (c->h_snap) cudaFreeHost(c->h_snap);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    for (int k = 0; k < 2; k++)
        if (c->ev_snap[k]) cudaEventDestroy(c->ev_snap[k]);
    if (c->h_hist) cudaFreeHost(c->h_hist);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

// AoS (n,3) host -> SoA planes on the device through pinned staging slot `slot`
// (0..3); the copy is queued on the stream, the caller synchronises.
int upload_aos(gd_ctx *c, double *dst, const double *src, int slot)
{
    const int n = c->d.n;
    double *t = c->h_stage + (size_t)slot * 3 * n;
    for (int i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) t[(size_t)k * n + i] = src[3 * (size_t)i + k];
    CK(cudaMemcpyAsync(dst, t, (size_t)3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    return GD_OK;
}

// Device SoA planes (stride plane_stride) -> pinned staging slot; transpose later
// with unstage_aos after a synchronise.
int download_planes(gd_ctx *c, const double *src, int plane_stride, int slot)
{
    const int n = c->d.n;
    double *t = c->h_stage + (size_t)slot * 3 * n;
    for (int k = 0; k < 3; k++)
        CK(cudaMemcpyAsync(t + (size_t)k * n, src + (size_t)k * plane_stride, (size_t)n * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
    return GD_OK;
}

void unstage_aos(gd_ctx *c, double *dst, int slot)
{
    const int n = c->d.n;
    const double *t = c->h_stage + (size_t)slot * 3 * n;
    for (int i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) dst[3 * (size_t)i + k] = t[(size_t)k * n + i];
}

long long *stage_i64(gd_ctx *c, int k) { return (long long *)(c->h_stage + (size_t)12 * c->d.n) + (size_t)k * c->d.n; }

int first_forces(gd_ctx *c)
{
    Dev &d = c->d;
    const int n = d.n;
    // a = jerk = 0 and tau = 0, so the prediction to tick 0 is exact
    CK(cudaMemsetAsync(d.a, 0, sizeof(double) * 3 * n, c->stream));
    CK(cudaMemsetAsync(d.jk, 0, sizeof(double) * 3 * n, c->stream));
    CK(cudaMemsetAsync(d.tau, 0, sizeof(long long) * n, c->stream));
    launch_predict_all(c, 0, c->mixed);
    k_iota<<<(n + 255) / 256, 256, 0, c->stream>>>(d.act, n);
    k_set_step<<<1, 1, 0, c->stream>>>(d.ctrl, 0, n);
    launch_force(c);
    k_reduce_partials<<<(n + 255) / 256, 256, 0, c->stream>>>(rargs(c), d.a, d.jk, n);
    k_init_steps<<<(n + 255) / 256, 256, 0, c->stream>>>(d);
    k_resync<<<1, 1024, 0, c->stream>>>(d);
    c->launches += 5;
    CK(cudaGetLastError());
    return sync_ctrl(c);
}

int build_graph(gd_ctx *c)
{
    if (c->graph) return GD_OK;
    const int G = c->graph_steps;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    for (int s = 0; s < G; s++) {
        cudaEvent_t e0 = c->opt.time_force ? c->ev[2 * s] : nullptr;
        cudaEvent_t e1 = c->opt.time_force ? c->ev[2 * s + 1] : nullptr;
        launch_step(c, s, e0, e1, true);
    }
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph = nullptr;
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    return GD_OK;
}

// Adds the timed force launches of the last chunk (slots with nact > 0).
int harvest_times(gd_ctx *c, int slots)
{
    if (!c->opt.time_force) return GD_OK;
    CK(cudaMemcpyAsync(c->h_hist, c->d.nact_hist, sizeof(int) * slots, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int s = 0; s < slots; s++) {
        if (c->h_hist[s] <= 0) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev[2 * s], c->ev[2 * s + 1]));
        c->force_ms += ms;
        c->force_launches += 1;
        c->force_interactions += (double)c->h_hist[s] * (double)c->d.n;
    }
    return GD_OK;
}

}  // namespace

extern "C" {

void gd_opts_default(gd_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->dt_min = std::ldexp(1.0, -22);
    o->dt_max = 0.125;
    o->precision = GD_MIXED;
    o->device = 0;
    o->stream = nullptr;
    o->use_graph = 1;
    o->graph_steps = 16;
    o->jsplit = 0;
    o->mode_cut = 0;
    o->time_force = 0;
}

int gd_init(gd_ctx **out, int64_t n, const double *m, const double *x, const double *v, double eps, double eta,
            const gd_opts *opt)
{
    if (!out) return fail(nullptr, GD_EINVAL, "out is null");
    *out = nullptr;
    if (n < 1 || n > (int64_t)(INT_MAX / 2)) return fail(nullptr, GD_EINVAL, "n out of range");
    if (!m || !x || !v) return fail(nullptr, GD_EINVAL, "m, x, v are required");
    if (!(eps >= 0) || !std::isfinite(eps)) return fail(nullptr, GD_EINVAL, "eps must be finite and >= 0");
    if (!(eta > 0) || !std::isfinite(eta)) return fail(nullptr, GD_EINVAL, "eta must be finite and > 0");
    gd_opts o;
    gd_opts_default(&o);
    if (opt) o = *opt;
    if (o.mode_cut <= 0) o.mode_cut = o.precision == GD_MIXED ? 192 : 96;
    if (o.graph_steps <= 0) o.graph_steps = 16;
    if (o.graph_steps > 64) return fail(nullptr, GD_EINVAL, "graph_steps must be <= 64");
    if (!is_pow2(o.dt_min) || !is_pow2(o.dt_max) || o.dt_max < o.dt_min)
        return fail(nullptr, GD_EINVAL, "dt_min and dt_max must be powers of two with dt_min <= dt_max");
    if (o.dt_max / o.dt_min > std::ldexp(1.0, 40)) return fail(nullptr, GD_EINVAL, "dt_max/dt_min too large");
    if (o.precision != GD_FP64 && o.precision != GD_MIXED) return fail(nullptr, GD_EINVAL, "bad precision");
    for (int64_t i = 0; i < n; i++) {
        if (!std::isfinite(m[i]) || m[i] < 0) return fail(nullptr, GD_EINVAL, "masses must be finite and >= 0");
        for (int k = 0; k < 3; k++)
            if (!std::isfinite(x[3 * i + k]) || !std::isfinite(v[3 * i + k]))
                return fail(nullptr, GD_EINVAL, "positions and velocities must be finite");
    }

    gd_ctx *c = new (std::nothrow) gd_ctx();
    if (!c) return fail(nullptr, GD_ENOMEM, "host allocation failed");
    c->opt = o;
    c->dev = o.device;
    c->mixed = o.precision == GD_MIXED;
    c->soft = eps > 0;
    c->graph_steps = o.graph_steps;
    int rc = GD_OK;
    auto bail = [&](int code) {
        g_init_err = c->err;
        free_all(c);
        delete c;
        return code;
    };
    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaSetDevice"));
    if (o.stream) {
        c->stream = (cudaStream_t)o.stream;
        c->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamCreate"));
        c->own_stream = true;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o.device);
    int occ = 0;
    if (c->mixed)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c->soft ? k_force_mixed<true> : k_force_mixed<false>,
                                                          FT, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c->soft ? k_force_fp64<true> : k_force_fp64<false>,
                                                          FT, 0);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "occupancy query"));
    if (occ < 1) occ = 1;
    c->grid_force = sms * occ;

    Dev &d = c->d;
    d.n = (int)n;
    d.npad = (int)((n + BJ - 1) / BJ * BJ);
    d.dt_min = o.dt_min;
    d.dtau_max = (long long)(o.dt_max / o.dt_min);
    d.eta = eta;
    d.eps2 = eps * eps;
    d.eps2f = (float)(eps * eps);
    c->grid_sel = (d.n + ST - 1) / ST;
    c->grid_corr = std::max(1, std::min((d.n + CT - 1) / CT, sms * 8));
    // partial capacity: S * nact entries per component, see make_plan
    d.cap = std::max<long long>((long long)d.npad, (2LL * c->grid_force + 1) * ITILE_A_MIX) + d.npad;
    const size_t n3 = (size_t)3 * d.n;
    if ((rc = dalloc(c, &d.x, n3)) || (rc = dalloc(c, &d.v, n3)) || (rc = dalloc(c, &d.a, n3)) ||
        (rc = dalloc(c, &d.jk, n3)) || (rc = dalloc(c, &d.m, (size_t)d.n)) || (rc = dalloc(c, &d.tau, (size_t)d.n)) ||
        (rc = dalloc(c, &d.dtau, (size_t)d.n)) || (rc = dalloc(c, &d.tnext, (size_t)d.n)) ||
        (rc = dalloc(c, &d.jA, (size_t)d.npad)) || (rc = dalloc(c, &d.jB, (size_t)d.npad)) ||
        (rc = dalloc(c, &d.jC, (size_t)d.npad)) || (rc = dalloc(c, &d.pd, (size_t)7 * d.npad)) ||
        (rc = dalloc(c, &d.act, (size_t)d.n)) || (rc = dalloc(c, &d.part, (size_t)6 * d.cap)) ||
        (rc = dalloc(c, &d.status, (size_t)c->grid_sel)) || (rc = dalloc(c, &d.eu, (size_t)d.n)) ||
        (rc = dalloc(c, &d.ek, (size_t)d.n)) || (rc = dalloc(c, &d.fout, (size_t)6 * d.n)) ||
        (rc = dalloc(c, &d.nact_hist, (size_t)64)) ||
        (rc = dalloc(c, &d.ctrl, (size_t)1)))
        return bail(rc);
    e = cudaMallocHost((void **)&c->h_ctrl, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_hist, sizeof(int) * 64);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_snap, 2 * sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_stage, (size_t)15 * d.n * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_snap[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_snap[1], cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(fail(c, GD_ENOMEM, "pinned host allocation failed"));
    if (o.time_force) {
        c->ev.resize(2 * 64);
        for (auto &ev : c->ev) {
            e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaEventCreate"));
        }
    }
    Ctrl h;
    std::memset(&h, 0, sizeof(h));
    h.T_acc = LLONG_MAX;
    h.tick_end = LLONG_MAX;
    h.epoch = 1;
    h.interactions = (double)n * (double)n;  // the initial full force evaluation
    e = cudaMemcpyAsync(d.ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.status, 0, sizeof(unsigned long long) * c->grid_sel, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.nact_hist, 0, sizeof(int) * 64, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.act, 0, sizeof(int) * d.n, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.m, m, sizeof(double) * d.n, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "upload"));
    if ((rc = upload_aos(c, d.x, x, 0)) || (rc = upload_aos(c, d.v, v, 1))) return bail(rc);
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "upload"));
    if (d.npad > d.n) k_init_pads<<<(d.npad - d.n + 127) / 128, 128, 0, c->stream>>>(d);
    if ((rc = first_forces(c))) return bail(rc);
    *out = c;
    return GD_OK;
}

int gd_evolve(gd_ctx *c, double t_end)
{
    int rc = check_usable(c);
    if (rc) return rc;
    if (!std::isfinite(t_end)) return fail(c, GD_EINVAL, "t_end must be finite");
    const double q = std::floor(t_end / c->d.dt_min);
    if (q > 9.0e18) return fail(c, GD_EINVAL, "t_end too large");
    const long long tick_end = (long long)q;
    if (tick_end < c->h_ctrl->T_last) return fail(c, GD_EINVAL, "t_end is before the current time");
    const int G = c->graph_steps;
    if (c->opt.use_graph) {
        if ((rc = build_graph(c))) return rc;
    }
    k_set_tick_end<<<1, 1, 0, c->stream>>>(c->d.ctrl, tick_end);
    c->launches += 1;
    auto chunk = [&]() -> int {
        if (c->opt.use_graph) {
            CK(cudaGraphLaunch(c->graph, c->stream));
            c->launches += 3LL * G;
        } else {
            for (int s = 0; s < G; s++) {
                cudaEvent_t e0 = c->opt.time_force ? c->ev[2 * s] : nullptr;
                cudaEvent_t e1 = c->opt.time_force ? c->ev[2 * s + 1] : nullptr;
                launch_step(c, s, e0, e1, false);
            }
        }
        CK(cudaGetLastError());
        return GD_OK;
    };
    if (c->opt.time_force) {
        // timed runs read the per-slot events after every chunk: no overlap
        for (;;) {
            if ((rc = chunk())) return rc;
            if ((rc = sync_ctrl(c))) return rc;
            if ((rc = harvest_times(c, G))) return rc;
            if (c->h_ctrl->T_cur > tick_end) break;
        }
    } else {
        // keep one chunk in flight while the host looks at the previous one's snapshot
        if ((rc = chunk())) return rc;
        CK(cudaMemcpyAsync(&c->h_snap[0], c->d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaEventRecord(c->ev_snap[0], c->stream));
        for (long long k = 0;; k++) {
            const int cur = (int)(k & 1), nxt = 1 - cur;
            if ((rc = chunk())) return rc;
            CK(cudaMemcpyAsync(&c->h_snap[nxt], c->d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaEventRecord(c->ev_snap[nxt], c->stream));
            CK(cudaEventSynchronize(c->ev_snap[cur]));
            if (c->h_snap[cur].err != 0 || c->h_snap[cur].T_cur > tick_end) break;
        }
    }
    k_set_tick_end<<<1, 1, 0, c->stream>>>(c->d.ctrl, LLONG_MAX);
    c->launches += 1;
    return sync_ctrl(c);
}

int gd_step_block(gd_ctx *c, double *t_out, int64_t *nact_out)
{
    int rc = check_usable(c);
    if (rc) return rc;
    launch_step(c, 0, c->opt.time_force ? c->ev[0] : nullptr, c->opt.time_force ? c->ev[1] : nullptr, false);
    CK(cudaGetLastError());
    if ((rc = sync_ctrl(c))) return rc;
    if ((rc = harvest_times(c, 1))) return rc;
    if (t_out) *t_out = (double)c->h_ctrl->T_last * c->d.dt_min;
    if (nact_out) *nact_out = c->h_ctrl->last_nact;
    return GD_OK;
}

int gd_energy(gd_ctx *c, double *K, double *U)
{
    int rc = check_usable(c);
    if (rc) return rc;
    launch_predict_all(c, c->h_ctrl->T_last, false);
    k_energy_terms<<<(c->d.n + ET - 1) / ET, ET, 0, c->stream>>>(c->d);
    k_energy_sum<<<1, 1024, 0, c->stream>>>(c->d);
    c->launches += 2;
    CK(cudaGetLastError());
    if ((rc = sync_ctrl(c))) return rc;
    if (K) *K = c->h_ctrl->K;
    if (U) *U = c->h_ctrl->U;
    return GD_OK;
}

int gd_get_state(gd_ctx *c, double *x, double *v, double *a, double *jerk, int64_t *tau, int64_t *dtau)
{
    int rc = check_usable(c);
    if (rc) return rc;
    const Dev &d = c->d;
    if (x && (rc = download_planes(c, d.x, d.n, 0))) return rc;
    if (v && (rc = download_planes(c, d.v, d.n, 1))) return rc;
    if (a && (rc = download_planes(c, d.a, d.n, 2))) return rc;
    if (jerk && (rc = download_planes(c, d.jk, d.n, 3))) return rc;
    if (tau) CK(cudaMemcpyAsync(stage_i64(c, 0), d.tau, sizeof(long long) * d.n, cudaMemcpyDeviceToHost, c->stream));
    if (dtau) CK(cudaMemcpyAsync(stage_i64(c, 1), d.dtau, sizeof(long long) * d.n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (x) unstage_aos(c, x, 0);
    if (v) unstage_aos(c, v, 1);
    if (a) unstage_aos(c, a, 2);
    if (jerk) unstage_aos(c, jerk, 3);
    if (tau) std::memcpy(tau, stage_i64(c, 0), sizeof(long long) * d.n);
    if (dtau) std::memcpy(dtau, stage_i64(c, 1), sizeof(long long) * d.n);
    return GD_OK;
}

int gd_set_state(gd_ctx *c, const double *x, const double *v, const double *a, const double *jerk,
                 const int64_t *tau, const int64_t *dtau)
{
    int rc = check_usable(c);
    if (rc) return rc;
    if (!x || !v || !a || !jerk || !tau || !dtau) return fail(c, GD_EINVAL, "all state arrays are required");
    const Dev &d = c->d;
    long long tmax = 0;
    std::vector<long long> tn((size_t)d.n);
    for (int i = 0; i < d.n; i++) {
        const long long dt = dtau[i], t = tau[i];
        if (dt < 1 || dt > d.dtau_max || (dt & (dt - 1)) != 0)
            return fail(c, GD_EINVAL, "dtau must be a power of two in [1, dt_max/dt_min]");
        if (t < 0 || t % dt != 0) return fail(c, GD_EINVAL, "tau must be a non-negative multiple of dtau");
        for (int k = 0; k < 3; k++)
            if (!std::isfinite(x[3 * i + k]) || !std::isfinite(v[3 * i + k]) || !std::isfinite(a[3 * i + k]) ||
                !std::isfinite(jerk[3 * i + k]))
                return fail(c, GD_EINVAL, "state values must be finite");
        tn[i] = t + dt;
        tmax = std::max(tmax, t);
    }
    CK(cudaStreamSynchronize(c->stream));  // the staging buffer is free
    if ((rc = upload_aos(c, d.x, x, 0)) || (rc = upload_aos(c, d.v, v, 1)) || (rc = upload_aos(c, d.a, a, 2)) ||
        (rc = upload_aos(c, d.jk, jerk, 3)))
        return rc;
    std::memcpy(stage_i64(c, 0), tau, sizeof(long long) * d.n);
    std::memcpy(stage_i64(c, 1), dtau, sizeof(long long) * d.n);
    std::memcpy(stage_i64(c, 2), tn.data(), sizeof(long long) * d.n);
    CK(cudaMemcpyAsync(d.tau, stage_i64(c, 0), sizeof(long long) * d.n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(d.dtau, stage_i64(c, 1), sizeof(long long) * d.n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(d.tnext, stage_i64(c, 2), sizeof(long long) * d.n, cudaMemcpyHostToDevice, c->stream));
    k_resync<<<1, 1024, 0, c->stream>>>(c->d);
    c->launches += 1;
    // the time of the last block step becomes the latest particle time
    Ctrl *h = c->h_ctrl;
    if ((rc = sync_ctrl(c))) return rc;
    h->T_last = tmax;
    CK(cudaMemcpyAsync(&c->d.ctrl->T_last, &h->T_last, sizeof(long long), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return GD_OK;
}

int gd_get_stats(gd_ctx *c, gd_stats *s)
{
    int rc = check_usable(c);
    if (rc) return rc;
    if (!s) return fail(c, GD_EINVAL, "null stats");
    if ((rc = sync_ctrl(c))) return rc;
    const Ctrl *h = c->h_ctrl;
    s->tick = h->T_last;
    s->block_steps = h->nblock;
    s->particle_steps = h->nsteps;
    s->interactions = h->interactions;
    s->last_nact = h->last_nact;
    s->kernel_launches = c->launches;
    return GD_OK;
}

int gd_kernel_time(gd_ctx *c, double *ms_total, int64_t *launches, double *interactions)
{
    if (!c) return fail(nullptr, GD_EINVAL, "null context");
    if (!c->opt.time_force) return fail(c, GD_ESTATE, "time_force was not enabled");
    if (ms_total) *ms_total = c->force_ms;
    if (launches) *launches = c->force_launches;
    if (interactions) *interactions = c->force_interactions;
    c->force_ms = 0;
    c->force_launches = 0;
    c->force_interactions = 0;
    return GD_OK;
}

void gd_free(gd_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->dev);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

const char *gd_last_error(const gd_ctx *c)
{
    if (!c) return g_init_err.c_str();
    return c->err.c_str();
}

int gd_force(gd_ctx *c, int64_t tick, const int32_t *idx, int64_t nact, double *acc, double *jerk)
{
    int rc = check_usable(c);
    if (rc) return rc;
    const Dev &d = c->d;
    if (nact < 1 || nact > d.n) return fail(c, GD_EINVAL, "nact must be in [1, n]");
    if (!idx || !acc || !jerk) return fail(c, GD_EINVAL, "idx, acc and jerk are required");
    if (tick < 0) return fail(c, GD_EINVAL, "tick must be >= 0");
    for (int64_t k = 0; k < nact; k++)
        if (idx[k] < 0 || idx[k] >= d.n) return fail(c, GD_EINVAL, "index out of range");
    CK(cudaMemcpyAsync(d.act, idx, sizeof(int) * nact, cudaMemcpyHostToDevice, c->stream));
    const long long Tsave = c->h_ctrl->T_cur;
    launch_predict_all(c, tick, c->mixed);
    k_set_step<<<1, 1, 0, c->stream>>>(d.ctrl, Tsave, (int)nact);
    c->launches += 2;
    if (c->opt.time_force) CK(cudaEventRecord(c->ev[0], c->stream));
    launch_force(c);
    if (c->opt.time_force) CK(cudaEventRecord(c->ev[1], c->stream));
    double *out = d.fout;
    k_reduce_partials<<<(int)((nact + 255) / 256), 256, 0, c->stream>>>(rargs(c), out, out + 3 * nact, (int)nact);
    std::vector<double> h((size_t)6 * nact);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), out, sizeof(double) * 6 * nact, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "gd_force");
    for (int64_t k = 0; k < nact; k++)
        for (int q = 0; q < 3; q++) {
            acc[3 * k + q] = h[(size_t)q * nact + k];
            jerk[3 * k + q] = h[(size_t)(3 + q) * nact + k];
        }
    if (c->opt.time_force) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
        c->force_ms += ms;
        c->force_launches += 1;
        c->force_interactions += (double)nact * (double)d.n;
    }
    // the free-running step recomputes act and nact
    return sync_ctrl(c);
}

int gd_predict(gd_ctx *c, int64_t tick, double *xp, double *vp)
{
    int rc = check_usable(c);
    if (rc) return rc;
    if (tick < 0) return fail(c, GD_EINVAL, "tick must be >= 0");
    launch_predict_all(c, tick, false);
    CK(cudaGetLastError());
    if ((rc = download_planes(c, c->d.pd, c->d.npad, 0))) return rc;
    if ((rc = download_planes(c, c->d.pd + 3 * (size_t)c->d.npad, c->d.npad, 1))) return rc;
    CK(cudaStreamSynchronize(c->stream));
    if (xp) unstage_aos(c, xp, 0);
    if (vp) unstage_aos(c, vp, 1);
    return GD_OK;
}

int gd_active(gd_ctx *c, int32_t *idx, int64_t *nact, int64_t *tick_next)
{
    int rc = check_usable(c);
    if (rc) return rc;
    if (!idx || !nact || !tick_next) return fail(c, GD_EINVAL, "idx, nact and tick_next are required");
    const Dev &d = c->d;
    if (c->mixed)
        k_select_predict<true><<<c->grid_sel, ST, 0, c->stream>>>(d, -1);
    else
        k_select_predict<false><<<c->grid_sel, ST, 0, c->stream>>>(d, -1);
    CK(cudaGetLastError());
    if ((rc = sync_ctrl(c))) return rc;
    const int na = c->h_ctrl->nact;
    *nact = na;
    *tick_next = c->h_ctrl->T_cur;
    CK(cudaMemcpyAsync(idx, d.act, sizeof(int) * na, cudaMemcpyDeviceToHost, c->stream));
    k_resync<<<1, 1024, 0, c->stream>>>(d);
    c->launches += 2;
    return sync_ctrl(c);
}

int gd_replay_step(gd_ctx *c, int64_t tick_next, const int32_t *idx, int64_t nact)
{
    int rc = check_usable(c);
    if (rc) return rc;
    const Dev &d = c->d;
    if (nact < 1 || nact > d.n) return fail(c, GD_EINVAL, "nact must be in [1, n]");
    if (!idx) return fail(c, GD_EINVAL, "idx is required");
    for (int64_t k = 0; k < nact; k++) {
        if (idx[k] < 0 || idx[k] >= d.n) return fail(c, GD_EINVAL, "index out of range");
        if (k > 0 && idx[k] <= idx[k - 1]) return fail(c, GD_EINVAL, "idx must be ascending and distinct");
    }
    if (tick_next <= 0) return fail(c, GD_EINVAL, "tick_next must be > 0");
    CK(cudaMemcpyAsync(d.act, idx, sizeof(int) * nact, cudaMemcpyHostToDevice, c->stream));
    launch_predict_all(c, tick_next, c->mixed);
    k_set_step<<<1, 1, 0, c->stream>>>(d.ctrl, tick_next, (int)nact);
    launch_force(c);
    k_correct<<<c->grid_corr, CT, 0, c->stream>>>(rargs(c));
    k_resync<<<1, 1024, 0, c->stream>>>(d);
    c->launches += 3;
    CK(cudaGetLastError());
    return sync_ctrl(c);
}

}  // extern "C"

// ================================================================ allocation-free force evaluation
//
// gd_force_noalloc: the mixed-precision force/jerk evaluation (k_force_mixed with
// its j-split partial sums) for callers that cannot allocate device memory.  Its
// scratch -- control block, a sanitised copy of the index list, the predicted
// j-records and the j-split partials -- lives in one file-scope __device__ array
// of fixed size, so the call allocates nothing.  Host code must not use the
// array's name as an address: the per-device set-up below asks the runtime for
// the array's device address once, with that device current, and passes it to
// the kernels.

namespace {

constexpr int NOALLOC_NMAX = 32768;                        // largest n accepted
constexpr long long NOALLOC_CAP = 2LL * NOALLOC_NMAX;      // partial entries per component
constexpr size_t NA_OFF_ACT = 256;
constexpr size_t NA_OFF_JA = NA_OFF_ACT + sizeof(int) * (size_t)NOALLOC_NMAX;
constexpr size_t NA_OFF_JB = NA_OFF_JA + sizeof(float4) * (size_t)NOALLOC_NMAX;
constexpr size_t NA_OFF_JC = NA_OFF_JB + sizeof(float4) * (size_t)NOALLOC_NMAX;
constexpr size_t NA_OFF_PART = NA_OFF_JC + sizeof(float2) * (size_t)NOALLOC_NMAX;
constexpr size_t NOALLOC_BYTES = NA_OFF_PART + sizeof(double) * 6 * (size_t)NOALLOC_CAP;  // about 4.4 MiB
static_assert(sizeof(Ctrl) <= NA_OFF_ACT, "control block must fit its slot");
static_assert(NOALLOC_NMAX % BJ == 0, "the j-records are padded to whole tiles");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

struct NoAllocDevice {
    bool ready;
    unsigned char *scratch;  // device address of g_noalloc_scratch on this device
    int grid;                // force-kernel grid (SMs x resident CTAs)
};
constexpr int NOALLOC_MAX_DEVICES = 64;
NoAllocDevice g_noalloc_dev[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mu;

// Packs the caller's FP64 particles (AoS, device) into the scratch j-records with
// massless far-away padding, copies the index list with out-of-range entries
// replaced by 0 (and remembered), and resets the control block.
__global__ void k_noalloc_pack(Dev d, const double *m, const double *x, const double *v, const int *idx, int nact,
                               int *bad_flags)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < d.npad) {
        if (i < d.n) {
            double xp[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
            double vp[3] = {v[3 * i], v[3 * i + 1], v[3 * i + 2]};
            store_jrec<true>(d, i, xp, vp, m[i]);
        } else {
            d.jA[i] = make_float4(PAD_FAR_F, PAD_FAR_F, PAD_FAR_F, 0.f);
            d.jB[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            d.jC[i] = make_float2(0.f, 0.f);
        }
    }
    if (i < nact) {
        const int k = idx[i];
        const bool ok = k >= 0 && k < d.n;
        d.act[i] = ok ? k : 0;
        bad_flags[i] = ok ? 0 : 1;
    }
    if (i == 0) {
        Ctrl c;
        memset(&c, 0, sizeof(c));
        c.nact = nact;
        *d.ctrl = c;
    }
}

// Sums the j-split partials of every slot into the caller's AoS outputs; slots
// whose index was out of range get NaN.
__global__ void k_noalloc_out(RArgs ra, const int *bad_flags, double *acc, double *jerk)
{
    const Dev &d = ra.d;
    const int nact = d.ctrl->nact;
    const Plan pl = make_plan(nact, d.npad, ra.grid, ra.mode_cut, ra.jsplit, true, d.cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nact; k += gridDim.x * blockDim.x) {
        double f[6];
        sum_partials(d, nact, pl.S, k, f);
        if (bad_flags[k]) {
            for (int c = 0; c < 6; c++) f[c] = __longlong_as_double(0x7ff8000000000000LL);
        }
        for (int c = 0; c < 3; c++) {
            acc[3 * (long long)k + c] = f[c];
            jerk[3 * (long long)k + c] = f[3 + c];
        }
    }
}

// Once per device, with that device current: the device address of the scratch
// array and the force-kernel grid.
int noalloc_setup(int dev, NoAllocDevice **out)
{
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(nullptr, GD_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocDevice &s = g_noalloc_dev[dev];
    if (!s.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        int sms = 0, occ_s = 0, occ_u = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, k_force_mixed<true>, FT, 0);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_u, k_force_mixed<false>, FT, 0);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "device query");
        s.scratch = (unsigned char *)p;
        s.grid = sms * std::max(1, std::min(occ_s, occ_u));
        s.ready = true;
    }
    *out = &s;
    return GD_OK;
}

}  // namespace

extern "C" int gd_force_noalloc(int64_t n, const double *m, const double *x, const double *v, double eps,
                                const int32_t *idx, int64_t nact, double *acc, double *jerk, void *stream)
{
    if (n < 1 || n > NOALLOC_NMAX)
        return fail(nullptr, GD_EINVAL,
                    "gd_force_noalloc: n must be in [1, " + std::to_string(NOALLOC_NMAX) + "], got " +
                        std::to_string((long long)n));
    if (nact < 1 || nact > n)
        return fail(nullptr, GD_EINVAL, "gd_force_noalloc: nact must be in [1, n], got " + std::to_string((long long)nact));
    if (!m || !x || !v || !idx || !acc || !jerk) return fail(nullptr, GD_EINVAL, "gd_force_noalloc: null pointer");
    if (!(eps >= 0) || !std::isfinite(eps)) return fail(nullptr, GD_EINVAL, "gd_force_noalloc: eps must be finite and >= 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    NoAllocDevice *s = nullptr;
    int rc = noalloc_setup(dev, &s);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Dev d;
    std::memset(&d, 0, sizeof(d));
    d.n = (int)n;
    d.npad = (int)((n + BJ - 1) / BJ * BJ);
    d.eps2f = (float)(eps * eps);
    d.eps2 = eps * eps;
    d.ctrl = (Ctrl *)s->scratch;
    d.act = (int *)(s->scratch + NA_OFF_ACT);
    d.jA = (float4 *)(s->scratch + NA_OFF_JA);
    d.jB = (float4 *)(s->scratch + NA_OFF_JB);
    d.jC = (float2 *)(s->scratch + NA_OFF_JC);
    d.part = (double *)(s->scratch + NA_OFF_PART);
    // the partial area's tail holds the per-slot out-of-range flags: the plan keeps
    // S * nact <= cap - nact, so they never overlap a partial in use
    d.cap = NOALLOC_CAP - (long long)n;
    int *bad = (int *)(d.part + 6 * (size_t)d.cap);
    const int mode_cut = 192;
    const int g = (d.npad + 255) / 256;
    k_noalloc_pack<<<g, 256, 0, st>>>(d, m, x, v, idx, (int)nact, bad);
    FArgs fa{d, s->grid, mode_cut, 0};
    if (eps > 0)
        k_force_mixed<true><<<s->grid, FT, 0, st>>>(fa);
    else
        k_force_mixed<false><<<s->grid, FT, 0, st>>>(fa);
    RArgs ra{d, s->grid, mode_cut, 0, true};
    k_noalloc_out<<<(int)((nact + 255) / 256), 256, 0, st>>>(ra, bad, acc, jerk);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "gd_force_noalloc launch");
    return GD_OK;
}
