// Independent systems of an ensemble, each integrated to the end time inside one
// thread-block cluster (the paper's block-step scheme, Sec. 2.4 steps 5-7, per
// system; its many-system use is the ensemble of independent clusters).
//
// A system's block steps depend on no other system, so no global block time is
// needed: k_ens_systems is a persistent launch whose thread-block clusters of CE
// CTAs each take a whole system from a work queue (largest first), load its
// particles into shared memory (CE CTAs x up to ES_P particles), run every one of
// its block steps up to tick_end, write it back and take the next.  A block step is
// the small-step cluster's (cluster.cuh) generalised to any number of active
// particles:
//   1. every CTA predicts its particles to T into its j-records and lists its
//      active ones (ascending local index); counts go to every CTA;   barrier B1
//   2. the step's active slots (ascending owner, then local index) in batches of
//      up to ES_NS: gather the batch's j-records from their owners, sum their
//      forces over this CTA's j-range, push the partials to the owners;
//                                                                       barrier B2
//      owners add the CE partials (rank order), correct (the mixed path's
//      arithmetic), choose the new steps;  (barrier B2b before the next batch)
//   3. every CTA's minimum next time (inactive and corrected particles) to every
//      CTA;                                                             barrier B3
//      the next block time is the minimum.
// The arithmetic per particle is that of the three-kernel mixed path and the
// small-step cluster; only the j-split of the force sums (CE CTAs) differs.

#include <cooperative_groups.h>

namespace gdk {

namespace cgx = cooperative_groups;

constexpr int ES_T = 512;           // threads per CTA
constexpr int ES_W = ES_T / 32;
constexpr int ES_ROUNDS = 3;        // particles per thread at most
constexpr int ES_P = 1280;          // particles per CTA at most (fuller CTAs measured faster)
constexpr int ES_NS = 96;           // active particles per batch (at most 16 warps x 8 in the correction)
constexpr int ES_NO = 96;           // outbox records per CTA (later active ones are read from the j-records)
static_assert(ES_P <= ES_ROUNDS * ES_T && ES_NS <= 16 * 8, "capacities");
constexpr int ES_MAXC = 16;         // largest cluster
constexpr int ES_CLASSES = 5;       // cluster sizes 1, 2, 4, 8, 16
constexpr int ES_PS = ES_MAXC * 6 + 4;  // floats of one batch slot's partials (padded: no bank conflicts)

struct EsLayout {
    size_t jA, jB, jC, tau, dtau, xh, xl, vh, vl, af, jf, lact, oA, oB, oC, iA, iB, iC, aown, aloc, part, tp, bytes;
    __host__ __device__ EsLayout()
    {
        size_t o = 0;
        auto take = [&](size_t b) {
            const size_t at = o;
            o += (b + 15) / 16 * 16;
            return at;
        };
        jA = take(sizeof(float4) * ES_P);
        jB = take(sizeof(float4) * ES_P);
        jC = take(sizeof(float2) * ES_P);
        tau = take(sizeof(long long) * ES_P);
        dtau = take(sizeof(long long) * ES_P);
        xh = take(sizeof(float) * 3 * ES_P);
        xl = take(sizeof(float) * 3 * ES_P);
        vh = take(sizeof(float) * 3 * ES_P);
        vl = take(sizeof(float) * 3 * ES_P);
        af = take(sizeof(float) * 3 * ES_P);
        jf = take(sizeof(float) * 3 * ES_P);
        lact = take(sizeof(int) * ES_P);
        oA = take(sizeof(float4) * ES_NO);
        oB = take(sizeof(float4) * ES_NO);
        oC = take(sizeof(float2) * ES_NO);
        iA = take(sizeof(float4) * ES_NS);
        iB = take(sizeof(float4) * ES_NS);
        iC = take(sizeof(float2) * ES_NS);
        aown = take(sizeof(int) * ES_NS);
        aloc = take(sizeof(int) * ES_NS);
        part = take(sizeof(float) * ES_NS * ES_PS);
        tp = take(sizeof(float) * 2 * ES_W * 6);
        bytes = o;
    }
};

struct EsArgs {
    Dev d;
    Ens e;
    const int *order;        // this launch's systems, largest first
    int nsys;                // how many
    unsigned int *queue;     // next position in order (zero at launch)
    long long tick_end;
};

template <bool SOFT>
__global__ void __launch_bounds__(ES_T, 1) k_ens_systems(EsArgs a)
{
    cgx::cluster_group cl = cgx::this_cluster();
    const int C = (int)cl.num_blocks();
    const int r = (int)cl.block_rank();
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const Dev &d = a.d;
    const int n = d.n;  // plane stride of the ensemble's (padded) arrays
    const EsLayout L;
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *jA = (float4 *)(smem + L.jA), *jB = (float4 *)(smem + L.jB);  // own j-records (jA.w: mass)
    float2 *jC = (float2 *)(smem + L.jC);
    long long *tau = (long long *)(smem + L.tau), *dtau = (long long *)(smem + L.dtau);
    float *xh = (float *)(smem + L.xh), *xl = (float *)(smem + L.xl);
    float *vh = (float *)(smem + L.vh), *vl = (float *)(smem + L.vl);
    float *af = (float *)(smem + L.af), *jf = (float *)(smem + L.jf);
    int *lact = (int *)(smem + L.lact);
    float4 *oA = (float4 *)(smem + L.oA), *oB = (float4 *)(smem + L.oB);  // outbox: the first ES_NO
    float2 *oC = (float2 *)(smem + L.oC);                                 // own active j-records
    float4 *iA = (float4 *)(smem + L.iA), *iB = (float4 *)(smem + L.iB);  // the batch's records
    float2 *iC = (float2 *)(smem + L.iC);
    int *aown = (int *)(smem + L.aown), *aloc = (int *)(smem + L.aloc);   // the batch's owners
    float *part = (float *)(smem + L.part);  // [batch slot][rank][6], slot stride ES_PS
    float *tp = (float *)(smem + L.tp);      // [active][segment][6]
    // inboxes the other CTAs write before a cluster barrier
    __shared__ int s_cnt_in[ES_MAXC];
    __shared__ long long s_mn_in[ES_MAXC];
    __shared__ int s_bad_in[ES_MAXC];
    __shared__ int s_sys;
    __shared__ int s_off[ES_MAXC + 1];
    __shared__ int s_wc[ES_ROUNDS * ES_W];
    __shared__ int s_base;
    __shared__ long long s_wmin[ES_W];
    __shared__ int s_wbad[ES_W];
    Ctrl *ctrl = d.ctrl;
    const float eps2 = d.eps2f;
    // CTA 0's counters over every system the cluster integrates
    long long steps_all = 0, psteps_all = 0;
    double inter_all = 0.0;

    for (;;) {
        // ---- the next system from the queue (CTA 0 takes it, every CTA learns it)
        if (r == 0 && t == 0) {
            const unsigned k = atomicAdd(a.queue, 1u);
            const int q = k < (unsigned)a.nsys ? a.order[k] : -1;
            for (int c = 0; c < C; c++) cl.map_shared_rank(&s_sys, c)[0] = q;
        }
        cl.sync();
        const int q = s_sys;
        if (q < 0) break;
        const int base = a.e.cs[q], nq = a.e.cn[q];
        const int Pq = (nq + C - 1) / C;  // particles per CTA of this system (<= ES_P)
        const int p0 = r * Pq;
        const int Pr = max(0, min(Pq, nq - p0));
        long long mn0 = LLONG_MAX;
        for (int p = t; p < Pr; p += ES_T) {
            const int i = base + p0 + p;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                xh[c * ES_P + p] = d.xs[c * n + i];
                xl[c * ES_P + p] = d.xs[(3 + c) * n + i];
                vh[c * ES_P + p] = d.vs[c * n + i];
                vl[c * ES_P + p] = d.vs[(3 + c) * n + i];
                af[c * ES_P + p] = d.af[c * n + i];
                jf[c * ES_P + p] = d.jf[c * n + i];
            }
            jA[p] = make_float4(0.f, 0.f, 0.f, d.mf[i]);
            tau[p] = d.tau[i];
            dtau[p] = d.dtau[i];
            const long long tn = tau[p] + dtau[p];
            mn0 = tn < mn0 ? tn : mn0;
        }
        // the system's first block time: the minimum over every CTA's particles
        mn0 = warp_min_ll(mn0);
        if (lane == 0) s_wmin[warp] = mn0;
        __syncthreads();
        if (warp == 0) {
            long long m = lane < ES_W ? s_wmin[lane] : LLONG_MAX;
            m = warp_min_ll(m);
            if (lane < C) cl.map_shared_rank(s_mn_in, lane)[r] = m;
        }
        cl.sync();
        long long T = LLONG_MAX;
        for (int c = 0; c < C; c++) T = s_mn_in[c] < T ? s_mn_in[c] : T;
        __syncthreads();  // s_mn_in is rewritten at the end of the first step

        bool stop = false;
        long long T_done = -1;  // the system's last block time
        while (T <= a.tick_end && !stop) {
            // ---- 1. predict own particles, list own active ones (ascending local index)
            long long mn = LLONG_MAX;
            unsigned bal[ES_ROUNDS];
            float4 rA[ES_ROUNDS], rB[ES_ROUNDS];
            float2 rC[ES_ROUNDS];
#pragma unroll
            for (int rd = 0; rd < ES_ROUNDS; rd++) {
                const int p = rd * ES_T + t;
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
                        const F2 x0{xh[c * ES_P + p], xl[c * ES_P + p]}, v0{vh[c * ES_P + p], vl[c * ES_P + p]};
                        xp[c] = ds_pred_x(x0, v0, af[c * ES_P + p], jf[c * ES_P + p], dt, h2, h3);
                        vp[c] = ds_pred_v_rec(v0, af[c * ES_P + p], jf[c * ES_P + p], dt, h2);
                    }
                    rA[rd] = make_float4(xp[0].h, xp[1].h, xp[2].h, jA[p].w);
                    rB[rd] = make_float4(xp[0].l, xp[1].l, xp[2].l, vp[0]);
                    rC[rd] = make_float2(vp[1], vp[2]);
                    jA[p] = rA[rd];
                    jB[p] = rB[rd];
                    jC[p] = rC[rd];
                }
                bal[rd] = __ballot_sync(0xffffffffu, act);
                if (lane == 0) s_wc[rd * ES_W + warp] = __popc(bal[rd]);
            }
            __syncthreads();
            if (warp == 0) {  // exclusive scan of the (round, warp) counts: entries 0-31, then 32-47
                static_assert(ES_ROUNDS * ES_W <= 64, "two counts per lane");
                const int c0 = s_wc[lane], c1 = lane + 32 < ES_ROUNDS * ES_W ? s_wc[lane + 32] : 0;
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
                if (lane + 32 < ES_ROUNDS * ES_W) s_wc[lane + 32] = tot0 + e1 - c1;
                if (lane == 31) s_base = tot0 + e1;
            }
            __syncthreads();
#pragma unroll
            for (int rd = 0; rd < ES_ROUNDS; rd++) {
                if ((bal[rd] >> lane) & 1u) {
                    const int pos = s_wc[rd * ES_W + warp] + __popc(bal[rd] & ((1u << lane) - 1u));
                    lact[pos] = rd * ES_T + t;
                    if (pos < ES_NO) {
                        oA[pos] = rA[rd];
                        oB[pos] = rB[rd];
                        oC[pos] = rC[rd];
                    }
                }
            }
            if (t < C) cl.map_shared_rank(s_cnt_in, t)[r] = s_base;
            cl.sync();  // B1: j-records, active lists and counts of every CTA are visible

            if (warp == 0) {  // prefix offsets of the CTAs' active counts
                const int cq = lane < C ? s_cnt_in[lane] : 0;
                int inc = cq;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                if (lane < C) s_off[lane] = inc - cq;
                if (lane == 31) s_off[C] = inc;
            }
            __syncthreads();
            const int nact = s_off[C];
            int bad = 0;

            // ---- 2. the active slots in batches
            for (int b0 = 0; b0 < nact; b0 += ES_NS) {
                const int nb = min(ES_NS, nact - b0);
                if (b0 > 0) cl.sync();  // B2b: the owners have read the previous batch's partials
                if (warp == 0 && lane < C) {  // owners of the batch's slots
                    const int lo = max(s_off[lane], b0), hi = min(s_off[lane + 1], b0 + nb);
                    for (int k = lo; k < hi; k++) {
                        aown[k - b0] = lane;
                        aloc[k - b0] = k - s_off[lane];
                    }
                }
                __syncthreads();
                // gather the batch's j-records (the outbox, else through the owner's list)
                for (int kb = t; kb < nb; kb += ES_T) {
                    const int o = aown[kb], kl = aloc[kb];
                    if (kl < ES_NO) {
                        iA[kb] = cl.map_shared_rank(oA, o)[kl];
                        iB[kb] = cl.map_shared_rank(oB, o)[kl];
                        iC[kb] = cl.map_shared_rank(oC, o)[kl];
                    } else {
                        const int p = cl.map_shared_rank(lact, o)[kl];
                        iA[kb] = cl.map_shared_rank(jA, o)[p];
                        iB[kb] = cl.map_shared_rank(jB, o)[p];
                        iC[kb] = cl.map_shared_rank(jC, o)[p];
                    }
                }
                __syncthreads();
                // forces over this CTA's j-range: (pair of actives, j-segment) tasks
                const int npair = (nb + 1) >> 1;
                int lgS = 0;
                if (npair < ES_W) lgS = 31 - __clz(ES_W / npair);
                const int Sw = 1 << lgS;
                const int seg = (((Pr + Sw - 1) >> lgS) + 31) & ~31;
                const int ntask = npair << lgS;
                for (int task = warp; task < ntask; task += ES_W) {
                    const int kp = task >> lgS, sg = task & (Sw - 1);
                    const int k0 = 2 * kp;
                    const bool has1 = k0 + 1 < nb;
                    const int k1 = has1 ? k0 + 1 : k0;
                    const int jb = sg * seg, je = min(jb + seg, Pr);
                    const float4 A0 = iA[k0], B0 = iB[k0], A1 = iA[k1], B1 = iB[k1];
                    const float2 C0 = iC[k0], C1 = iC[k1];
                    float f0[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, f1[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
                    for (int j = jb + lane; j < je; j += 32) {
                        const float4 A = jA[j], B = jB[j];
                        const float2 Cj = jC[j];
                        pair_mixed<SOFT>(A, B, Cj, A0.x, A0.y, A0.z, B0.x, B0.y, B0.z, B0.w, C0.x, C0.y, eps2, f0);
                        pair_mixed<SOFT>(A, B, Cj, A1.x, A1.y, A1.z, B1.x, B1.y, B1.z, B1.w, C1.x, C1.y, eps2, f1);
                    }
#pragma unroll
                    for (int c = 0; c < 6; c++)
                        for (int o = 16; o > 0; o >>= 1) {
                            f0[c] = __fadd_rn(f0[c], __shfl_xor_sync(0xffffffffu, f0[c], o));
                            f1[c] = __fadd_rn(f1[c], __shfl_xor_sync(0xffffffffu, f1[c], o));
                        }
                    float mine_c = f0[0];
#pragma unroll
                    for (int c = 1; c < 6; c++) mine_c = lane == c ? f0[c] : mine_c;
#pragma unroll
                    for (int c = 0; c < 6; c++) mine_c = lane == 6 + c ? f1[c] : mine_c;
                    const bool store = lane < 6 || (has1 && lane < 12);
                    const int k = lane < 6 ? k0 : k1, c = lane < 6 ? lane : lane - 6;
                    if (store) {
                        if (Sw == 1)
                            cl.map_shared_rank(part, aown[k])[k * ES_PS + r * 6 + c] = mine_c;
                        else
                            tp[((k << lgS) + sg) * 6 + c] = mine_c;
                    }
                }
                if (Sw > 1) {
                    for (int lh = lgS - 1; lh >= 0; lh--) {
                        const int h = 1 << lh;
                        __syncthreads();
                        for (int w = t; w < (nb * 6) << lh; w += ES_T) {
                            const int c = w % 6, ks = w / 6, k = ks >> lh, sg = ks & (h - 1);
                            const int at = (((k << lgS) + sg) * 6) + c;
                            tp[at] = __fadd_rn(tp[at], tp[at + h * 6]);
                        }
                    }
                    __syncthreads();
                    for (int w = t; w < nb * 6; w += ES_T) {
                        const int k = w / 6, c = w % 6;
                        cl.map_shared_rank(part, aown[k])[k * ES_PS + r * 6 + c] = tp[((k << lgS) * 6) + c];
                    }
                }
                cl.sync();  // B2: every partial of the batch has reached its owner

                // owners: this CTA's slots of the batch, eight per warp, four lanes each
                const int klo = max(s_off[r], b0) - b0, khi = min(s_off[r + 1], b0 + nb) - b0;
                const int mine = max(0, khi - klo);
                {
                    const int q4 = lane & 3;
                    const int c = q4 < 3 ? q4 : 2;
                    const bool real = q4 < 3;
                    const int kw = warp * 8 + (lane >> 2);
                    if (warp * 8 < mine) {
                        const bool valid = kw < mine;
                        const int kb = klo + (valid ? kw : mine - 1);
                        const int p = lact[kb + b0 - s_off[r]];
                        float pa[ES_MAXC], pj[ES_MAXC];
#pragma unroll
                        for (int o = 0; o < ES_MAXC; o++) {
                            pa[o] = o < C ? part[kb * ES_PS + o * 6 + c] : 0.f;
                            pj[o] = o < C ? part[kb * ES_PS + o * 6 + 3 + c] : 0.f;
                        }
#pragma unroll
                        for (int h = ES_MAXC / 2; h >= 1; h >>= 1)
#pragma unroll
                            for (int o = 0; o < h; o++) {
                                pa[o] = __fadd_rn(pa[o], pa[o + h]);
                                pj[o] = __fadd_rn(pj[o], pj[o + h]);
                            }
                        const float a1 = pa[0], j1 = pj[0];
                        const F2 x0{xh[c * ES_P + p], xl[c * ES_P + p]}, v0{vh[c * ES_P + p], vl[c * ES_P + p]};
                        const float a0 = af[c * ES_P + p], j0 = jf[c * ES_P + p];
                        F2 x1, v1;
                        long long dtn;
                        ds_correct(d, real, T - tau[p], dtau[p], T, x0, v0, a0, j0, a1, j1, x1, v1, dtn);
                        const bool fin = isfinite(x1.h) && isfinite(v1.h) && isfinite(a1) && isfinite(j1);
                        __syncwarp();
                        if (valid) {
                            if (real) {
                                if (!fin) bad |= 1;
                                xh[c * ES_P + p] = x1.h;
                                xl[c * ES_P + p] = x1.l;
                                vh[c * ES_P + p] = v1.h;
                                vl[c * ES_P + p] = v1.l;
                                af[c * ES_P + p] = a1;
                                jf[c * ES_P + p] = j1;
                            }
                            if (q4 == 0) {
                                tau[p] = T;
                                dtau[p] = dtn;
                                mn = T + dtn < mn ? T + dtn : mn;
                            }
                        }
                    }
                }
            }

            // ---- 3. next block time: every CTA's minimum and fault bits to every CTA
            mn = warp_min_ll(mn);
            bad = __reduce_or_sync(0xffffffffu, bad);
            if (lane == 0) {
                s_wmin[warp] = mn;
                s_wbad[warp] = bad;
            }
            __syncthreads();
            if (warp == 0) {
                long long m = lane < ES_W ? s_wmin[lane] : LLONG_MAX;
                int b = lane < ES_W ? s_wbad[lane] : 0;
                m = warp_min_ll(m);
                b = __reduce_or_sync(0xffffffffu, b);
                if (lane < C) {
                    cl.map_shared_rank(s_mn_in, lane)[r] = m;
                    cl.map_shared_rank(s_bad_in, lane)[r] = b;
                }
            }
            cl.sync();  // B3
            long long Tn = LLONG_MAX;
            int bn = 0;
            for (int c = 0; c < C; c++) {
                Tn = s_mn_in[c] < Tn ? s_mn_in[c] : Tn;
                bn |= s_bad_in[c];
            }
            __syncthreads();  // s_mn_in, s_bad_in and s_off are rewritten next step
            steps_all += 1;
            psteps_all += nact;
            inter_all += (double)nact * (double)nq;
            T_done = T;
            T = Tn;
            if (bn) {
                if (r == 0 && t == 0) set_err(ctrl, ST_ENONFINITE);
                stop = true;
            }
        }
        // the system's state back to global memory
        for (int p = t; p < Pr; p += ES_T) {
            const int i = base + p0 + p;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                d.xs[c * n + i] = xh[c * ES_P + p];
                d.xs[(3 + c) * n + i] = xl[c * ES_P + p];
                d.vs[c * n + i] = vh[c * ES_P + p];
                d.vs[(3 + c) * n + i] = vl[c * ES_P + p];
                d.af[c * n + i] = af[c * ES_P + p];
                d.jf[c * n + i] = jf[c * ES_P + p];
            }
            d.tau[i] = tau[p];
            d.dtau[i] = dtau[p];
            d.tnext[i] = tau[p] + dtau[p];
        }
        if (r == 0 && t == 0 && T_done >= 0) atomicMax(&ctrl->T_last, T_done);
        cl.sync();  // no CTA takes the next system while another may read its shared memory
    }
    if (r == 0 && t == 0 && steps_all > 0) {
        atomicAdd((unsigned long long *)&ctrl->nblock, (unsigned long long)steps_all);
        atomicAdd((unsigned long long *)&ctrl->nsteps, (unsigned long long)psteps_all);
        atomicAdd(&ctrl->interactions, inter_all);
    }
}

}  // namespace gdk
