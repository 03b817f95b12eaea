// cluster.cuh -- small block steps inside one thread-block cluster (mixed path).
// Included once, by gravidy.cu, after kernels.cuh.
//
// Most block steps of a collisional system move only a handful of particles
// (Sec. 2.2: the active set at a block time is the set of particles whose next
// time equals it), and for those the three full-GPU kernels of a step cost far more
// in launch and memory round trips than in arithmetic.  k_cluster_steps runs such
// steps with the whole system resident in the shared memory of one cluster of C
// CTAs (C = 16 where the GPU allows it): CTA r owns particles [r P, (r + 1) P).
// Per block step T (Sec. 2.4 steps 5-7):
//   1. every CTA predicts its own particles to T into its j-records (shared
//      memory) and lists its active ones;                      cluster barrier
//   2. every CTA reads the C active counts (the same total everywhere), gathers
//      the active particles' j-records from their owners, and sums the force of
//      every active particle over its own j-range; the partial sums go to the
//      owner's shared memory (distributed shared memory);      cluster barrier
//   3. owners add the C partials in rank order, correct, choose the new steps
//      (the same arithmetic as the mixed three-kernel path), and post their
//      minimum next time;                                      cluster barrier
//   4. every CTA takes the minimum over the C posts: the next block time; owners
//      write their corrected particles through to global memory.
// The loop stops, with the same decision in every CTA, when a step has more than
// `ns` active particles (then the full-GPU kernels take that step), when the block
// time passes tick_end, after max_steps steps, or on a fault.  With `handoff` the
// step the cluster leaves to the full GPU is handed over already selected: every
// CTA writes its predicted j-records and its active particles' places in the
// (ascending) active list to global memory and starts the running minimum of the
// next block time with its inactive particles, i.e. the work of k_select_predict,
// so that the force kernel runs next; a launch that ends at tick_end hands over an
// empty step.  All cluster
// barriers are unconditional in the loop body, so every CTA passes the same
// sequence of them; a last barrier keeps every CTA's shared memory alive until no
// CTA can still read it.
#pragma once

#include <cooperative_groups.h>

namespace gdk {

namespace cgx = cooperative_groups;

constexpr int CL_T = 512;     // threads per CTA (one CTA per SM)
constexpr int CL_W = CL_T / 32;
constexpr int CL_MAXC = 16;   // largest cluster
constexpr int CL_NS = 128;    // most active particles a cluster step takes
constexpr int CL_ROUNDS = 3;  // particles per thread at most (P <= CL_ROUNDS * CL_T)
constexpr int CL_PS = CL_MAXC * 6 + 4;  // floats of one active's partials (padded: no bank conflicts)

// Shared-memory layout of a CTA owning up to P particles (P a multiple of 32).
struct ClLayout {
    int P;
    size_t xh, xl, vh, vl, af, jf, tau, dtau, jA, jB, jC, lact, iA, iB, iC, aown, oA, oB, oC, aloc, part, tp, bytes;
    __host__ __device__ ClLayout(int P_) : P(P_)
    {
        size_t o = 0;
        auto take = [&](size_t bytes) {
            const size_t at = o;
            o += (bytes + 15) / 16 * 16;
            return at;
        };
        jA = take(sizeof(float4) * P);
        jB = take(sizeof(float4) * P);
        iA = take(sizeof(float4) * CL_NS);
        iB = take(sizeof(float4) * CL_NS);
        tau = take(sizeof(long long) * P);
        dtau = take(sizeof(long long) * P);
        jC = take(sizeof(float2) * P);
        iC = take(sizeof(float2) * CL_NS);
        xh = take(sizeof(float) * 3 * P);
        xl = take(sizeof(float) * 3 * P);
        vh = take(sizeof(float) * 3 * P);
        vl = take(sizeof(float) * 3 * P);
        af = take(sizeof(float) * 3 * P);
        jf = take(sizeof(float) * 3 * P);
        lact = take(sizeof(int) * CL_NS);
        aown = take(sizeof(int) * CL_NS);
        oA = take(sizeof(float4) * CL_NS);
        oB = take(sizeof(float4) * CL_NS);
        oC = take(sizeof(float2) * CL_NS);
        aloc = take(sizeof(int) * CL_NS);
        part = take(sizeof(float) * CL_NS * CL_PS);
        tp = take(sizeof(float) * 2 * CL_W * 6);
        bytes = o;
    }
};

struct ClArgs {
    Dev d;
    int P;          // particles per CTA
    int ns;         // largest active count taken here (<= CL_NS)
    int max_steps;  // block steps per launch
    int handoff;    // 1: hand the next step over selected (see above); 0: leave it to k_select_predict
    int slot;       // handoff: >= 0 records the handed-over N_act in nact_hist[slot]
};


// EXTRA: the instance that takes P(EC)^n passes and a post-Newtonian pair (the
// other compiles to the plain single-pass step).
template <bool SOFT, bool EXTRA>
__global__ void __launch_bounds__(CL_T, 1) k_cluster_steps(ClArgs a)
{
    cgx::cluster_group cl = cgx::this_cluster();
    const int C = (int)cl.num_blocks();
    const int r = (int)cl.block_rank();
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const Dev &d = a.d;
    const int n = d.n, P = a.P;
    const ClLayout L(P);
    const long long K0 = clock64();
    extern __shared__ __align__(16) unsigned char smem[];
    float *xh = (float *)(smem + L.xh), *xl = (float *)(smem + L.xl);
    float *vh = (float *)(smem + L.vh), *vl = (float *)(smem + L.vl);
    float *af = (float *)(smem + L.af), *jf = (float *)(smem + L.jf);
    long long *tau = (long long *)(smem + L.tau), *dtau = (long long *)(smem + L.dtau);
    float4 *jA = (float4 *)(smem + L.jA), *jB = (float4 *)(smem + L.jB);  // own j-records; jA[p].w
    float2 *jC = (float2 *)(smem + L.jC);                                 // holds the mass throughout
    int *lact = (int *)(smem + L.lact), *aown = (int *)(smem + L.aown), *aloc = (int *)(smem + L.aloc);
    float4 *oA = (float4 *)(smem + L.oA), *oB = (float4 *)(smem + L.oB);  // outbox: own active
    float2 *oC = (float2 *)(smem + L.oC);                                 // particles' j-records
    float4 *iA = (float4 *)(smem + L.iA), *iB = (float4 *)(smem + L.iB);
    float2 *iC = (float2 *)(smem + L.iC);
    float *part = (float *)(smem + L.part);  // [slot][rank][6], slot stride CL_PS
    float *tp = (float *)(smem + L.tp);      // [active][segment][6]
    // inboxes the other CTAs write (distributed shared memory) before a cluster barrier:
    // active counts of the step (before B1), minimum next time and fault bits (before B3)
    __shared__ int s_cnt_in[CL_MAXC];
    __shared__ long long s_mn_in[CL_MAXC];
    __shared__ int s_bad_in[CL_MAXC];
    __shared__ int s_off[CL_MAXC + 1];
    __shared__ int s_wc[CL_ROUNDS * CL_W];
    __shared__ int s_base;
    __shared__ long long s_wmin[CL_W];
    __shared__ int s_wbad[CL_W];
    __shared__ long long s_T;
    __shared__ int s_bad;

    const int p0 = r * P;
    const int Pr = max(0, min(P, n - p0));
    for (int p = t; p < Pr; p += CL_T) {
        const int i = p0 + p;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            xh[c * P + p] = d.xs[c * n + i];
            xl[c * P + p] = d.xs[(3 + c) * n + i];
            vh[c * P + p] = d.vs[c * n + i];
            vl[c * P + p] = d.vs[(3 + c) * n + i];
            af[c * P + p] = d.af[c * n + i];
            jf[c * P + p] = d.jf[c * n + i];
        }
        jA[p] = make_float4(0.f, 0.f, 0.f, d.mf[i]);
        tau[p] = d.tau[i];
        dtau[p] = d.dtau[i];
    }
    Ctrl *ctrl = d.ctrl;
    long long T = ctrl->T_cur;
    const long long tick_end = ctrl->tick_end;
    long long T_last = 0, psteps = 0;
    int last_n = 0, steps = 0;
    unsigned long long ph[3] = {0ull, 0ull, 0ull};  // CTA 0's clock: predict, force, correct
    // CTA 0's SM cycles of every finished small step's phases: predict and list, count
    // push + B1 + offsets, gather, force tasks, segment tree + partial push, B2,
    // correction, post + B3, next time; then the launch's prologue and epilogue and
    // the number of finished small steps (only CTA 0's thread 0 publishes them)
    unsigned long long cyc[12] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    bool handed = false;  // the next step was handed over selected
    const float eps2 = d.eps2f;
    __syncthreads();

    const long long L0 = clock64();
    for (;;) {
        // the exit tests read values every CTA holds identically
        if (T > tick_end || (!a.handoff && steps >= a.max_steps)) break;

        // ---- 1. predict own particles, list own active ones (ascending local index)
        const unsigned long long t0 = global_ns();
        const long long P0 = clock64();
        long long mn = LLONG_MAX;
        unsigned bal[CL_ROUNDS];
        float4 rA[CL_ROUNDS], rB[CL_ROUNDS];
        float2 rC[CL_ROUNDS];
#pragma unroll
        for (int rd = 0; rd < CL_ROUNDS; rd++) {
            const int p = rd * CL_T + t;
            bool act = false;
            if (p < Pr) {
                const long long tn = tau[p] + dtau[p];
                act = tn == T;
                if (!act) mn = tn < mn ? tn : mn;
                float dt, idt;
                step_f(d, T - tau[p], dt, idt);
                const float h2 = __fmul_rn(0.5f, __fmul_rn(dt, dt));
                const float h3 = __fmul_rn(__fmul_rn(__fmul_rn(dt, dt), dt), 1.0f / 6.0f);
                F2 xp[3];
                float vp[3];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const F2 x0{xh[c * P + p], xl[c * P + p]}, v0{vh[c * P + p], vl[c * P + p]};
                    xp[c] = ds_pred_x(x0, v0, af[c * P + p], jf[c * P + p], dt, h2, h3);
                    vp[c] = ds_pred_v_rec(v0, af[c * P + p], jf[c * P + p], dt, h2);
                }
                rA[rd] = make_float4(xp[0].h, xp[1].h, xp[2].h, jA[p].w);
                rB[rd] = make_float4(xp[0].l, xp[1].l, xp[2].l, vp[0]);
                rC[rd] = make_float2(vp[1], vp[2]);
                jA[p] = rA[rd];
                jB[p] = rB[rd];
                jC[p] = rC[rd];
            }
            bal[rd] = __ballot_sync(0xffffffffu, act);
            if (lane == 0) s_wc[rd * CL_W + warp] = __popc(bal[rd]);
        }
        __syncthreads();
        if (warp == 0) {  // exclusive scan of the (round, warp) counts: ascending particle order
            static_assert(CL_ROUNDS * CL_W <= 64, "two counts per lane");
            const int c0 = s_wc[lane], c1 = lane + 32 < CL_ROUNDS * CL_W ? s_wc[lane + 32] : 0;
            // entries 0-31 on the lanes in order, then entries 32-47
            int e0 = c0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, e0, o);
                if (lane >= o) e0 += y;
            }
            const int tot0 = __shfl_sync(0xffffffffu, e0, 31);
            int e1 = c1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, e1, o);
                if (lane >= o) e1 += y;
            }
            __syncwarp();
            s_wc[lane] = e0 - c0;
            if (lane + 32 < CL_ROUNDS * CL_W) s_wc[lane + 32] = tot0 + e1 - c1;
            if (lane == 31) s_base = tot0 + e1;
        }
        __syncthreads();
#pragma unroll
        for (int rd = 0; rd < CL_ROUNDS; rd++) {
            if ((bal[rd] >> lane) & 1u) {
                const int pos = s_wc[rd * CL_W + warp] + __popc(bal[rd] & ((1u << lane) - 1u));
                if (pos < CL_NS) {
                    lact[pos] = rd * CL_T + t;
                    oA[pos] = rA[rd];
                    oB[pos] = rB[rd];
                    oC[pos] = rC[rd];
                }
            }
        }
        const long long P2 = clock64();
        if (t < C) cl.map_shared_rank(s_cnt_in, t)[r] = s_base;  // this CTA's count, into every inbox
        cl.sync();  // B1: j-records, active lists and counts of every CTA are visible

        // ---- 2. the step's active set: counts of all CTAs, prefix offsets
        if (warp == 0) {  // lane q holds CTA q's count; a shuffle scan gives the offsets
            const int cq = lane < C ? s_cnt_in[lane] : 0;
            int inc = cq;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane < C) s_off[lane] = inc - cq;
            if (lane == 31) s_off[C] = inc;
            // owner table of the step's active slots (only needed if the cluster takes it)
            if (__shfl_sync(0xffffffffu, inc, 31) <= a.ns)
                for (int k = inc - cq; k < inc; k++) {
                    aown[k] = lane;
                    aloc[k] = k - (inc - cq);
                }
        }
        __syncthreads();
        const int nact = s_off[C];
        const unsigned long long t1 = global_ns();
        const long long P4 = clock64();
        ph[0] += t1 - t0;
        if (nact > a.ns || (a.handoff && steps >= a.max_steps)) {
            // a large step (or the last of this launch): the full-GPU kernels take it
            if (a.handoff) {
                for (int p = t; p < Pr; p += CL_T) {
                    d.jA[p0 + p] = jA[p];
                    d.jB[p0 + p] = jB[p];
                    d.jC[p0 + p] = jC[p];
                }
#pragma unroll
                for (int rd = 0; rd < CL_ROUNDS; rd++)
                    if ((bal[rd] >> lane) & 1u)
                        d.act[s_off[r] + s_wc[rd * CL_W + warp] + __popc(bal[rd] & ((1u << lane) - 1u))] =
                            p0 + rd * CL_T + t;
                const long long m = warp_min_ll(mn);  // the inactive particles' next times
                if (lane == 0 && m != LLONG_MAX) atomicMin((unsigned long long *)&ctrl->T_acc, (unsigned long long)m);
                if (r == 0 && t == 0) {
                    ctrl->nact = nact;
                    if (a.slot >= 0) d.nact_hist[a.slot] = nact;
                }
                handed = true;
            }
            break;
        }
        // gather the active particles' j-records (i-records of this step)
        for (int k = t; k < nact; k += CL_T) {
            const int q = aown[k], kl = aloc[k];
            iA[k] = cl.map_shared_rank(oA, q)[kl];
            iB[k] = cl.map_shared_rank(oB, q)[kl];
            iC[k] = cl.map_shared_rank(oC, q)[kl];
        }
        __syncthreads();
        int bad = 0;
        long long P5 = 0, P6 = 0, P7 = 0, P8 = 0;
        unsigned long long t2 = 0;
        // evaluation-correction passes (P(EC)^n): each pass but the last writes the
        // owners' corrected positions and velocities over the active particles'
        // records, which the next pass evaluates against
        for (int pass = 1;; pass++) {
        const bool last = !EXTRA || pass >= d.n_iter;
        P5 = clock64();
        // forces over this CTA's j-range: tasks (pair of active particles, j-segment),
        // so every j-record loaded from shared memory serves two pair terms; with
        // fewer than CL_W pairs each pair's j-range is cut into Sw = 2^lgS segments
        const int npair = (nact + 1) >> 1;
        int lgS = 0;
        if (npair < CL_W) lgS = 31 - __clz(CL_W / npair);
        const int Sw = 1 << lgS;
        const int seg = (((Pr + Sw - 1) >> lgS) + 31) & ~31;
        const int ntask = npair << lgS;
        for (int task = warp; task < ntask; task += CL_W) {
            const int kp = task >> lgS, sg = task & (Sw - 1);
            const int k0 = 2 * kp;
            const bool has1 = k0 + 1 < nact;
            const int k1 = has1 ? k0 + 1 : k0;
            const int jb = sg * seg, je = min(jb + seg, Pr);
            const float4 A0 = iA[k0], B0 = iB[k0], A1 = iA[k1], B1 = iB[k1];
            const float2 C0 = iC[k0], C1 = iC[k1];
            float f0[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, f1[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (has1) {
#pragma unroll 8
                for (int j = jb + lane; j < je; j += 32) {
                    const float4 A = jA[j], B = jB[j];
                    const float2 Cj = jC[j];
                    pair_mixed<SOFT>(A, B, Cj, A0.x, A0.y, A0.z, B0.x, B0.y, B0.z, B0.w, C0.x, C0.y, eps2, f0);
                    pair_mixed<SOFT>(A, B, Cj, A1.x, A1.y, A1.z, B1.x, B1.y, B1.z, B1.w, C1.x, C1.y, eps2, f1);
                }
            } else {
#pragma unroll 4
                for (int j = jb + lane; j < je; j += 32)
                    pair_mixed<SOFT>(jA[j], jB[j], jC[j], A0.x, A0.y, A0.z, B0.x, B0.y, B0.z, B0.w, C0.x, C0.y, eps2,
                                     f0);
            }
#pragma unroll
            for (int c = 0; c < 6; c++)
                for (int o = 16; o > 0; o >>= 1) {
                    f0[c] = __fadd_rn(f0[c], __shfl_xor_sync(0xffffffffu, f0[c], o));
                    f1[c] = __fadd_rn(f1[c], __shfl_xor_sync(0xffffffffu, f1[c], o));
                }
            // lane q < 12 stores component q % 6 of active k0 (q < 6) or k1 (selected
            // without indexing the arrays)
            float mine_c = f0[0];
#pragma unroll
            for (int c = 1; c < 6; c++) mine_c = lane == c ? f0[c] : mine_c;
#pragma unroll
            for (int c = 0; c < 6; c++) mine_c = lane == 6 + c ? f1[c] : mine_c;
            const bool store = lane < 6 || (has1 && lane < 12);
            const int k = lane < 6 ? k0 : k1, c = lane < 6 ? lane : lane - 6;
            if (store) {
                if (Sw == 1) {
                    float *dst = cl.map_shared_rank(part, aown[k]);
                    dst[aloc[k] * CL_PS + r * 6 + c] = mine_c;
                } else {
                    tp[((k << lgS) + sg) * 6 + c] = mine_c;
                }
            }
        }
        P6 = clock64();
        if (Sw > 1) {
            // this CTA's partial of active k: a pairwise tree over its Sw segment sums
            for (int lh = lgS - 1; lh >= 0; lh--) {
                const int h = 1 << lh;
                __syncthreads();
                for (int w = t; w < (nact * 6) << lh; w += CL_T) {
                    const int c = w % 6, ks = w / 6, k = ks >> lh, sg = ks & (h - 1);
                    const int at = (((k << lgS) + sg) * 6) + c;
                    tp[at] = __fadd_rn(tp[at], tp[at + h * 6]);
                }
            }
            __syncthreads();
            for (int w = t; w < nact * 6; w += CL_T) {
                const int k = w / 6, c = w % 6;
                float *dst = cl.map_shared_rank(part, aown[k]);
                dst[aloc[k] * CL_PS + r * 6 + c] = tp[((k << lgS) * 6) + c];
            }
        }
        P7 = clock64();
        cl.sync();  // B2: every partial has reached its owner
        t2 = global_ns();
        P8 = clock64();
        ph[1] += t2 - t1;

        // ---- 3. owners: sum the C partials (rank order), correct, new steps
        const int mine = s_off[r + 1] - s_off[r];
        {
            const int q4 = lane & 3;
            const int c = q4 < 3 ? q4 : 2;
            const bool real = q4 < 3;
            const int k = warp * 8 + (lane >> 2);
            if (warp * 8 < mine) {
                const bool valid = k < mine;
                const int kk = valid ? k : mine - 1;
                const int p = lact[kk];
                // the C partials in a fixed pairwise tree (absent ranks count zero)
                float pa[CL_MAXC], pj[CL_MAXC];
#pragma unroll
                for (int q = 0; q < CL_MAXC; q++) {
                    pa[q] = q < C ? part[kk * CL_PS + q * 6 + c] : 0.f;
                    pj[q] = q < C ? part[kk * CL_PS + q * 6 + 3 + c] : 0.f;
                }
#pragma unroll
                for (int h = CL_MAXC / 2; h >= 1; h >>= 1)
#pragma unroll
                    for (int q = 0; q < h; q++) {
                        pa[q] = __fadd_rn(pa[q], pa[q + h]);
                        pj[q] = __fadd_rn(pj[q], pj[q + h]);
                    }
                float a1 = pa[0], j1 = pj[0];
                if (EXTRA && d.pn_terms) {
                    // a post-Newtonian pair member: the pair terms from both members'
                    // predicted records, wherever in the cluster they are held
                    const int gi = p0 + p;
                    if (gi == d.pn_p || gi == d.pn_q) {
                        const int op = d.pn_p / P, lp = d.pn_p % P, oq = d.pn_q / P, lq = d.pn_q % P;
                        pn_add_records(d, gi, c, cl.map_shared_rank(jA, op)[lp], cl.map_shared_rank(jB, op)[lp],
                                       cl.map_shared_rank(jC, op)[lp], cl.map_shared_rank(jA, oq)[lq],
                                       cl.map_shared_rank(jB, oq)[lq], cl.map_shared_rank(jC, oq)[lq], a1, j1);
                    }
                }
                const F2 x0{xh[c * P + p], xl[c * P + p]}, v0{vh[c * P + p], vl[c * P + p]};
                const float a0 = af[c * P + p], j0 = jf[c * P + p];
                const long long dtau_old = dtau[p];
                F2 x1, v1;
                long long dtn;
                ds_correct(d, real, T - tau[p], dtau_old, T, x0, v0, a0, j0, a1, j1, x1, v1, dtn);
                const bool fin = isfinite(x1.h) && isfinite(v1.h) && isfinite(a1) && isfinite(j1);
                __syncwarp();
                if (!last) {
                    // a trial pass: the corrected x, v into the particle's j-record and
                    // its outbox copy; the state stays
                    if (valid && real) {
                        if (!fin) bad |= 1;
                        const float vr = __fadd_rn(v1.h, v1.l);
                        ((float *)&jA[p])[c] = x1.h;
                        ((float *)&jB[p])[c] = x1.l;
                        ((float *)&oA[kk])[c] = x1.h;
                        ((float *)&oB[kk])[c] = x1.l;
                        if (c == 0) {
                            jB[p].w = vr;
                            oB[kk].w = vr;
                        } else {
                            ((float *)&jC[p])[c - 1] = vr;
                            ((float *)&oC[kk])[c - 1] = vr;
                        }
                    }
                } else if (valid) {
                    if (real) {
                        if (!fin) bad |= 1;
                        xh[c * P + p] = x1.h;
                        xl[c * P + p] = x1.l;
                        vh[c * P + p] = v1.h;
                        vl[c * P + p] = v1.l;
                        af[c * P + p] = a1;
                        jf[c * P + p] = j1;
                    }
                    if (q4 == 0) {
                        tau[p] = T;
                        dtau[p] = dtn;
                        mn = T + dtn < mn ? T + dtn : mn;
                    }
                }
            }
        }
        if (last) break;
        cl.sync();  // the trial records are written; the owners have read the partials
        for (int k = t; k < nact; k += CL_T) {  // the active particles' corrected records
            const int q = aown[k], kl = aloc[k];
            iA[k] = cl.map_shared_rank(oA, q)[kl];
            iB[k] = cl.map_shared_rank(oB, q)[kl];
            iC[k] = cl.map_shared_rank(oC, q)[kl];
        }
        __syncthreads();
        }
        mn = warp_min_ll(mn);
        bad = __reduce_or_sync(0xffffffffu, bad);
        if (lane == 0) {
            s_wmin[warp] = mn;
            s_wbad[warp] = bad;
        }
        __syncthreads();
        const long long P9 = clock64();
        if (warp == 0) {
            long long m = lane < CL_W ? s_wmin[lane] : LLONG_MAX;
            int b = lane < CL_W ? s_wbad[lane] : 0;
            m = warp_min_ll(m);
            b = __reduce_or_sync(0xffffffffu, b);
            if (lane < C) {  // this CTA's post, into every inbox
                cl.map_shared_rank(s_mn_in, lane)[r] = m;
                cl.map_shared_rank(s_bad_in, lane)[r] = b;
            }
        }
        cl.sync();  // B3: corrected state and the posts of every CTA are visible
        const long long P10 = clock64();

        // ---- 4. next block time: minimum over the C posts
        if (warp == 0) {  // lane q holds CTA q's post
            long long m = LLONG_MAX;
            int b = 0;
            if (lane < C) {
                m = s_mn_in[lane];
                b = s_bad_in[lane];
            }
            m = warp_min_ll(m);
            b = __reduce_or_sync(0xffffffffu, b);
            if (lane == 0) {
                s_T = m;
                s_bad = b;
            }
        }
        __syncthreads();
        ph[2] += global_ns() - t2;
        T_last = T;
        last_n = nact;
        psteps += nact;
        steps++;
        T = s_T;
        const bool stop = s_bad != 0;
        __syncthreads();  // s_T, s_bad are rewritten next step
        {
            const long long P11 = clock64();
            const long long pt[12] = {P0, P2, P4, P5, P6, P7, P8, P9, P10, P11, 0, 0};
#pragma unroll
            for (int k = 0; k < 9; k++) cyc[k] += (unsigned long long)(pt[k + 1] - pt[k]);
            cyc[11] += 1;
        }
        if (stop) {
            if (t == 0 && r == 0) set_err(ctrl, ST_ENONFINITE);
            break;
        }
    }
    const long long L1 = clock64();
    // the particles this launch corrected (their time moved on), written back to
    // global memory once
    for (int p = t; p < Pr; p += CL_T) {
        const int i = p0 + p;
        if (tau[p] == d.tau[i]) continue;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            d.xs[c * n + i] = xh[c * P + p];
            d.xs[(3 + c) * n + i] = xl[c * P + p];
            d.vs[c * n + i] = vh[c * P + p];
            d.vs[(3 + c) * n + i] = vl[c * P + p];
            d.af[c * n + i] = af[c * P + p];
            d.jf[c * n + i] = jf[c * P + p];
        }
        d.tau[i] = tau[p];
        d.dtau[i] = dtau[p];
        d.tnext[i] = tau[p] + dtau[p];
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
    if (r == 0 && t == 0) {
        cyc[9] += (unsigned long long)(L0 - K0);
        cyc[10] += (unsigned long long)(clock64() - L1);
#pragma unroll
        for (int k = 0; k < 12; k++) ctrl->cl_cyc[k] += cyc[k];
        ctrl->T_cur = T;
        if (a.handoff && !handed) {  // tick_end passed, or a fault: nothing to hand over
            ctrl->nact = 0;
            if (a.slot >= 0) d.nact_hist[a.slot] = 0;
        }
        ctrl->ph_ns[0] += ph[0];
        ctrl->ph_ns[1] += ph[1];
        ctrl->ph_ns[2] += ph[2];
        if (steps > 0) {
            ctrl->T_last = T_last;
            ctrl->last_nact = last_n;
            ctrl->nblock += steps;
            ctrl->nsteps += psteps;
            ctrl->interactions += (double)psteps * (double)n * d.n_iter;  // every pass evaluated the forces
            ctrl->epoch += (unsigned)steps;
        }
    }
}

}  // namespace gdk
