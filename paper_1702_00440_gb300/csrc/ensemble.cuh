// ensemble.cuh -- device code for an ensemble of independent N-body clusters
// advanced together (GraviDy's Hermite-4 block-step scheme, Sec. 2.4, applied to
// every cluster; each cluster only feels its own particles).  Included once, by
// gravidy.cu, after kernels.cuh.
//
// Layout: the clusters' particles are concatenated, each cluster padded to a
// multiple of ST (= BJ) slots with massless particles that are never active.  The
// single-system Dev describes the whole padded array (n = npad = total slots), so
// prediction, j-records, the corrector and the state arrays are shared with the
// single-system path; the cluster bookkeeping lives in Ens.
//
// A global block step takes the smallest next time over all clusters; the
// particles of every cluster whose next time equals it are active.  Each cluster's
// active list is compacted into its own segment of the active array (starting at
// the cluster's first slot), so clusters never need a global prefix.  Two kernels
// per block step:
//   k_ens_select  predict all slots, compact per cluster (look-back stops at the
//                 cluster's first chunk), start the next-time minimum;
//   k_ens_force   every CTA derives the same work plan from the per-cluster active
//                 counts (tiles of 8 active particles, a j-split per tile that
//                 fills the GPU), computes FP32 partials over j-chunks of the
//                 tile's own cluster, and the last CTA of each tile sums them,
//                 corrects the tile's particles and adds their new next times; the
//                 last CTA to finish turns the minimum into the next block time.
#pragma once

namespace gdk {

constexpr int ENS_CMAX = 2048;   // clusters per ensemble (plan tables live in shared memory)
constexpr int ENS_TILE = 8;      // active particles per tile: 4 warps x 2
constexpr int ENS_PART = ENS_TILE * 6;

struct Ens {
    int C;
    const int *cs;      // first slot of cluster c (multiple of ST)
    const int *cnp;     // padded slot count of cluster c (multiple of ST)
    const int *cn;      // real particle count of cluster c
    int *cnact;         // active count of cluster c in the current step
    const int *pcl;     // cluster of each slot
    unsigned int *tilecnt;  // per global tile arrival counters
    float *part;        // FP32 partials: (item * ENS_TILE + slot) * 6 + component
    double *K, *U;      // per-cluster energies
    int target_items;   // work items the plan aims for
};

struct EArgs {
    Dev d;
    Ens e;
    int correct;        // 1: correct in the tile tails and finalize the step; 0: forces only
};

// Selection + prediction with per-cluster compaction (see k_select_predict) at
// block time T with look-back tag ep.  COH: the state was written earlier in the
// same launch (the fused kernel), so it is read through L2.
template <bool COH>
__device__ void ens_select_phase(const Dev &d, const Ens &e, int nchunks, long long T, unsigned ep)
{
    Ctrl *ctrl = d.ctrl;
    __shared__ unsigned s_excl;
    __shared__ unsigned s_wcnt[ST / 32];
    __shared__ long long s_wmin[ST / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long mn_all = LLONG_MAX;
    for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const int i = chunk * ST + threadIdx.x;
        const int c = e.pcl[chunk * ST];
        const int cf = e.cs[c] / ST;                 // the cluster's first chunk
        const int cl = cf + e.cnp[c] / ST - 1;       // and its last
        const long long tn = ldc(&d.tnext[i]);
        const bool act = (tn == T);
        if (!act) mn_all = tn < mn_all ? tn : mn_all;
        predict_store_ds<COH>(d, i, T - ldc(&d.tau[i]));
        const unsigned ballot = __ballot_sync(0xffffffffu, act);
        if (lane == 0) s_wcnt[warp] = __popc(ballot);
        __syncthreads();
        if (warp == 0) {
            const unsigned cnt = lane < ST / 32 ? s_wcnt[lane] : 0u;
            unsigned incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
            if (lane < ST / 32) s_wcnt[lane] = incl - cnt;
            unsigned excl = 0;
            if (chunk == cf) {
                if (lane == 0) atomicExch(&d.status[chunk], lb_pack(ep, 2u, total));
            } else {
                if (lane == 0) atomicExch(&d.status[chunk], lb_pack(ep, 1u, total));
                int base = chunk - 1;
                int spins = 0;
                for (;;) {
                    const int p = base - lane;
                    unsigned f = 2u, val = 0u;
                    if (p >= cf) {
                        const unsigned long long w = ld_volatile_u64(&d.status[p]);
                        f = ((unsigned)(w >> 34) == ep) ? (unsigned)((w >> 32) & 3u) : 0u;
                        val = (unsigned)w;
                    }
                    const unsigned notready = __ballot_sync(0xffffffffu, f == 0u);
                    const unsigned prefix = __ballot_sync(0xffffffffu, f == 2u);
                    const int first = prefix ? __ffs(prefix) - 1 : 31;
                    const unsigned need = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
                    if (notready & need) {
                        if (++spins > SPIN_LIMIT) {
                            if (lane == 0) set_err(ctrl, ST_ETIMEOUT);
                            break;
                        }
                        __nanosleep(32);
                        continue;
                    }
                    unsigned contrib = lane <= first ? val : 0u;
                    for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
                    excl += contrib;
                    if (prefix) break;
                    base -= 32;
                }
                if (lane == 0) atomicExch(&d.status[chunk], lb_pack(ep, 2u, excl + total));
            }
            if (lane == 0) {
                s_excl = excl;
                if (chunk == cl) {
                    int na = (int)(excl + total);
                    if (na > e.cn[c]) {
                        set_err(ctrl, ST_ETIMEOUT);
                        na = 0;
                    }
                    e.cnact[c] = na;
                }
            }
        }
        __syncthreads();
        if (act) {
            const unsigned pos = s_excl + s_wcnt[warp] + __popc(ballot & ((1u << lane) - 1u));
            if (pos < (unsigned)e.cnp[c]) d.act[e.cs[c] + pos] = i;
        }
        __syncthreads();
    }
    long long mn = warp_min_ll(mn_all);
    if (lane == 0) s_wmin[warp] = mn;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < ST / 32; w++) mn = s_wmin[w] < mn ? s_wmin[w] : mn;
        if (mn != LLONG_MAX) atomicMin((unsigned long long *)&ctrl->T_acc, (unsigned long long)mn);
    }
    __syncthreads();  // shared memory is reused by the next phase or step
}

__global__ void __launch_bounds__(ST) k_ens_select(Dev d, Ens e, int nchunks)
{
    Ctrl *ctrl = d.ctrl;
    const long long T = ctrl->T_cur;
    if (T > ctrl->tick_end) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->nact = 0;
        return;
    }
    ens_select_phase<false>(d, e, nchunks, T, ctrl->epoch & 0x3FFFFFFFu);
}

// The work plan, the same in every CTA: per cluster, tiles of ENS_TILE active
// particles and a j-split S_c (at least one chunk of 2 BJ particles), item and tile
// offsets by exclusive scans.  Also the step's active and interaction counts.
struct EnsPlanSmem {
    int item_base[ENS_CMAX + 1];
    int tile_base[ENS_CMAX + 1];
    int S[ENS_CMAX];
    long long nact_total;
    double inter_total;
};

__device__ void ens_plan(const Ens &e, EnsPlanSmem &p)
{
    __shared__ int s_wt[FT / 32], s_wi[FT / 32];
    __shared__ long long s_wn[FT / 32];
    __shared__ double s_wx[FT / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (e.C + FT - 1) / FT;  // consecutive clusters per thread
    const int c_lo = min(t * per, e.C), c_hi = min(c_lo + per, e.C);
    // pass 1: tiles, active particles and interactions of the step
    int tiles = 0;
    long long na = 0;
    double inter = 0.0;
    for (int c = c_lo; c < c_hi; c++) {
        const int nc = ldc(&e.cnact[c]);
        tiles += (nc + ENS_TILE - 1) / ENS_TILE;
        na += nc;
        inter += (double)nc * (double)e.cn[c];
    }
    for (int o = 16; o > 0; o >>= 1) {
        tiles += __shfl_xor_sync(0xffffffffu, tiles, o);
        na += __shfl_xor_sync(0xffffffffu, na, o);
        inter += __shfl_xor_sync(0xffffffffu, inter, o);
    }
    if (lane == 0) {
        s_wt[warp] = tiles;
        s_wn[warp] = na;
        s_wx[warp] = inter;
    }
    __syncthreads();
    int total_tiles = 0;
    long long nn = 0;
    double xx = 0.0;
    for (int w = 0; w < FT / 32; w++) {
        total_tiles += s_wt[w];
        nn += s_wn[w];
        xx += s_wx[w];
    }
    if (t == 0) {
        p.nact_total = nn;
        p.inter_total = xx;
    }
    if (total_tiles < 1) total_tiles = 1;
    const int S_target = (e.target_items + total_tiles - 1) / total_tiles;
    // pass 2: per-cluster split and item count, then a block-wide exclusive scan
    int my_items = 0, my_tiles = 0;
    for (int c = c_lo; c < c_hi; c++) {
        const int nc = ldc(&e.cnact[c]);
        const int tl = (nc + ENS_TILE - 1) / ENS_TILE;
        int smax = e.cnp[c] / (2 * BJ);
        if (smax < 1) smax = 1;
        int S = S_target < smax ? S_target : smax;
        if (S < 1) S = 1;
        p.S[c] = S;
        my_items += tl * S;
        my_tiles += tl;
    }
    int ii = my_items, it = my_tiles;  // inclusive warp scans
    for (int o = 1; o < 32; o <<= 1) {
        const int yi = __shfl_up_sync(0xffffffffu, ii, o), yt = __shfl_up_sync(0xffffffffu, it, o);
        if (lane >= o) {
            ii += yi;
            it += yt;
        }
    }
    __syncthreads();  // s_wt / s_wi reuse
    if (lane == 31) {
        s_wi[warp] = ii;
        s_wt[warp] = it;
    }
    __syncthreads();
    int bi = ii - my_items, bt = it - my_tiles;
    for (int w = 0; w < warp; w++) {
        bi += s_wi[w];
        bt += s_wt[w];
    }
    for (int c = c_lo; c < c_hi; c++) {
        const int nc = ldc(&e.cnact[c]);
        const int tl = (nc + ENS_TILE - 1) / ENS_TILE;
        p.item_base[c] = bi;
        p.tile_base[c] = bt;
        bi += tl * p.S[c];
        bt += tl;
    }
    if (t == FT - 1) {
        p.item_base[e.C] = bi;
        p.tile_base[e.C] = bt;
    }
    __syncthreads();
}

// Sums the S partials of the ENS_TILE slots of a tile into fsum: every thread takes
// the items s = t, t + FT, ... (all 48 values of an item are contiguous: twelve
// float4 loads at once), then a warp-shuffle tree and a four-warp sum in a fixed
// order.
__device__ void ens_tile_reduce(const Dev &d, const Ens &e, int item0, int S, int slot0, int nvalid)
{
    __shared__ float s_w[FT / 32][ENS_PART];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float acc[ENS_PART];
#pragma unroll
    for (int q = 0; q < ENS_PART; q++) acc[q] = 0.f;
    for (int s = t; s < S; s += FT) {
        const float4 *p4 = (const float4 *)(e.part + (long long)(item0 + s) * ENS_PART);
        float4 v[ENS_PART / 4];
#pragma unroll
        for (int q = 0; q < ENS_PART / 4; q++) v[q] = __ldcg(p4 + q);
#pragma unroll
        for (int q = 0; q < ENS_PART / 4; q++) {
            acc[4 * q] += v[q].x;
            acc[4 * q + 1] += v[q].y;
            acc[4 * q + 2] += v[q].z;
            acc[4 * q + 3] += v[q].w;
        }
    }
#pragma unroll
    for (int q = 0; q < ENS_PART; q++)
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < ENS_PART; q++) s_w[warp][q] = acc[q];
    }
    __syncthreads();
    if (t < ENS_PART) {
        const int k = t / 6, comp = t % 6;
        if (k < nvalid) {
            DS sum;
            sum.zero();
            for (int w = 0; w < FT / 32; w++) sum.add(s_w[w][t]);
            store_fsum<float>(d, comp, slot0 + k, __fadd_rn(sum.h, sum.l));
        }
    }
    __syncthreads();
}

// Force (and, with a.correct, correction and the step's end) of the active
// particles of every cluster at block time T: the work plan, the (tile, j-chunk)
// items, the tile sums by the last of a tile's items, and the last CTA turning the
// running minimum into the next block time.  COH as for ens_select_phase.
template <bool SOFT, bool COH>
__device__ void ens_force_phase(const EArgs &a, long long T, EnsPlanSmem &p)
{
    const Dev &d = a.d;
    const Ens &e = a.e;
    Ctrl *ctrl = d.ctrl;
    __shared__ float4 sA[2 * BJ], sB[2 * BJ];
    __shared__ float2 sC[2 * BJ];
    __shared__ int s_last;
    ens_plan(e, p);
    const int total_items = p.item_base[e.C];
    const float eps2 = d.eps2f;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    long long mymin = LLONG_MAX;
    int bad = 0;
    for (int item = blockIdx.x; item < total_items; item += gridDim.x) {
        // the cluster of this item: the last c with item_base[c] <= item
        int lo = 0, hi = e.C;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (p.item_base[mid] <= item) lo = mid; else hi = mid;
        }
        const int c = lo;
        const int S = p.S[c];
        const int rem = item - p.item_base[c];
        const int tl = rem / S, s = rem % S;
        const int nact_c = ldc(&e.cnact[c]);
        const int cs = e.cs[c], cnp = e.cnp[c];
        const int slot0 = cs + tl * ENS_TILE;
        const int nvalid = min(ENS_TILE, nact_c - tl * ENS_TILE);
        const int tiles_chunk = (cnp / BJ + S - 1) / S;
        const int jbeg = cs + s * tiles_chunk * BJ;
        const int jend = min(jbeg + tiles_chunk * BJ, cs + cnp);
        // warp w owns tile slots 2w and 2w+1
        const int k0 = 2 * warp;
        const bool busy = k0 < nvalid;
        const bool has1 = k0 + 1 < nvalid;
        const int i0 = ldc(&d.act[slot0 + min(k0, nvalid - 1)]);
        const int i1 = ldc(&d.act[slot0 + min(has1 ? k0 + 1 : k0, nvalid - 1)]);
        const float4 A0 = ldc(&d.jA[i0]), B0 = ldc(&d.jB[i0]);
        const float2 C0 = ldc(&d.jC[i0]);
        const float4 A1 = ldc(&d.jA[i1]), B1 = ldc(&d.jB[i1]);
        const float2 C1 = ldc(&d.jC[i1]);
        DS g0[6], g1[6];
#pragma unroll
        for (int q = 0; q < 6; q++) {
            g0[q].zero();
            g1[q].zero();
        }
        for (int jt = jbeg; jt < jend; jt += 2 * BJ) {
            const int nt = min(2 * BJ, jend - jt);
            __syncthreads();
            for (int q = t; q < nt; q += FT) {
                sA[q] = ldc(&d.jA[jt + q]);
                sB[q] = ldc(&d.jB[jt + q]);
                sC[q] = ldc(&d.jC[jt + q]);
            }
            __syncthreads();
            if (busy) {
                float f0[6] = {0, 0, 0, 0, 0, 0}, f1[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll 4
                for (int jj = lane; jj < nt; jj += 32) {
                    const float4 A = sA[jj], B = sB[jj];
                    const float2 C = sC[jj];
                    pair_mixed<SOFT>(A, B, C, A0.x, A0.y, A0.z, B0.x, B0.y, B0.z, B0.w, C0.x, C0.y, eps2, f0);
                    pair_mixed<SOFT>(A, B, C, A1.x, A1.y, A1.z, B1.x, B1.y, B1.z, B1.w, C1.x, C1.y, eps2, f1);
                }
#pragma unroll
                for (int q = 0; q < 6; q++) {
                    g0[q].add(f0[q]);
                    g1[q].add(f1[q]);
                }
            }
        }
        if (busy) {
            float r0[6], r1[6];
#pragma unroll
            for (int q = 0; q < 6; q++) {
                r0[q] = g0[q].as_float();
                r1[q] = g1[q].as_float();
                for (int o = 16; o > 0; o >>= 1) {
                    r0[q] += __shfl_xor_sync(0xffffffffu, r0[q], o);
                    r1[q] += __shfl_xor_sync(0xffffffffu, r1[q], o);
                }
            }
            if (lane == 0) {
                float *pp = e.part + ((long long)item * ENS_TILE + k0) * 6;
#pragma unroll
                for (int q = 0; q < 6; q++) pp[q] = r0[q];
                if (has1) {
#pragma unroll
                    for (int q = 0; q < 6; q++) pp[6 + q] = r1[q];
                }
            }
        }
        // the last of the tile's S items sums, corrects and records the new next times
        __syncthreads();
        const int gtile = p.tile_base[c] + tl;
        if (t == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(&e.tilecnt[gtile], 1u);
            s_last = prev == (unsigned)(S - 1);
            if (s_last) e.tilecnt[gtile] = 0u;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            ens_tile_reduce(d, e, p.item_base[c] + tl * S, S, slot0, nvalid);
            if (a.correct) correct_slots<true, COH>(d, T, slot0, slot0 + nvalid, warp, FT / 32, mymin, bad);
        }
        __syncthreads();
    }
    if (!a.correct) return;
    if (bad & 2) set_err(ctrl, ST_EINVAL);
    if (bad & 1) set_err(ctrl, ST_ENONFINITE);
    mymin = warp_min_ll(mymin);
    if (lane == 0 && mymin != LLONG_MAX) atomicMin((unsigned long long *)&ctrl->T_acc, (unsigned long long)mymin);
    __syncthreads();
    if (t == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&ctrl->done, 1u);
        if (prev == gridDim.x - 1) {
            __threadfence();
            const long long next = (long long)atomicAdd((unsigned long long *)&ctrl->T_acc, 0ull);
            ctrl->T_last = T;
            ctrl->last_nact = (int)p.nact_total;
            ctrl->nact = (int)p.nact_total;
            ctrl->T_cur = next;
            ctrl->T_acc = LLONG_MAX;
            ctrl->nblock += 1;
            ctrl->nsteps += p.nact_total;
            ctrl->interactions += p.inter_total;
            ctrl->epoch += 1;
            ctrl->done = 0;
        }
    }
    __syncthreads();  // the plan in shared memory is rebuilt by the next step
}

template <bool SOFT>
__global__ void __launch_bounds__(FT, 2) k_ens_force(EArgs a)
{
    Ctrl *ctrl = a.d.ctrl;
    const long long T = ctrl->T_cur;
    if (a.correct && T > ctrl->tick_end) return;
    __shared__ EnsPlanSmem p;
    ens_force_phase<SOFT, false>(a, T, p);
}

// Up to max_steps global block steps in one cooperative launch (every CTA
// resident): select + predict, grid barrier, force + correction + the step's end,
// grid barrier.  The block time and the look-back tag of the next step are read
// through L2 after the barrier; every CTA sees the same values, so all leave the
// loop together once the block time passes tick_end.  Computes what the
// two-kernel step computes, bit for bit.
template <bool SOFT>
__global__ void __launch_bounds__(FT, 2) k_ens_steps(EArgs a, int nchunks, int max_steps)
{
    const Dev &d = a.d;
    Ctrl *ctrl = d.ctrl;
    __shared__ EnsPlanSmem p;
    const long long tick_end = ldc(&ctrl->tick_end);
    for (int s = 0; s < max_steps; s++) {
        const long long T = ldc(&ctrl->T_cur);
        if (T > tick_end) break;
        const unsigned ep = ldc(&ctrl->epoch) & 0x3FFFFFFFu;
        ens_select_phase<true>(d, a.e, nchunks, T, ep);
        grid_sync(d.bar, ctrl);
        ens_force_phase<SOFT, true>(a, T, p);
        grid_sync(d.bar, ctrl);
    }
}

// First steps of the real particles (pads keep next time +inf).
__global__ void k_ens_init_steps(Dev d, Ens e)
{
    const int n = d.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = e.pcl[i];
    const bool real = i - e.cs[c] < e.cn[c];
    if (!real) {
        d.tau[i] = 0;
        d.dtau[i] = d.dtau_max;
        d.tnext[i] = LLONG_MAX;
        return;
    }
    double a[3], j[3];
    take_force<true>(d, i, i, a, j);
    const double na = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const double nj = sqrt(j[0] * j[0] + j[1] * j[1] + j[2] * j[2]);
    const double dt0 = d.eta * na / nj;
    long long dtau;
    if (!(dt0 < INFINITY)) {
        dtau = d.dtau_max;
    } else {
        const double q = dt0 / d.dt_min;
        if (q < 1.0)
            dtau = 1;
        else if (q >= (double)d.dtau_max)
            dtau = d.dtau_max;
        else
            dtau = 1LL << ((int)((__double_as_longlong(q) >> 52) & 0x7FF) - 1023);
    }
    d.tau[i] = 0;
    d.dtau[i] = dtau;
    d.tnext[i] = dtau;
    bool ok = true;
    for (int q = 0; q < 3; q++) ok = ok && isfinite(a[q]) && isfinite(j[q]);
    if (!ok) set_err(d.ctrl, ST_ENONFINITE);
}

// Per-slot energy terms with j over the slot's own cluster (mixed pair
// arithmetic, see k_energy_mixed).
__global__ void __launch_bounds__(ET) k_ens_energy_terms(Dev d, Ens e)
{
    __shared__ float4 sA[ET], sB[ET];
    const int np = d.npad;
    const int i = blockIdx.x * ET + threadIdx.x;   // all CTA slots are in one cluster (ET = ST)
    const int c = e.pcl[blockIdx.x * ET];
    const int cs = e.cs[c], cnp = e.cnp[c];
    const float4 Ai = d.jA[i], Bi = d.jB[i];
    const float eps2 = d.eps2f;
    DS phi;
    phi.zero();
    for (int jt = cs; jt < cs + cnp; jt += ET) {
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
            const float term = (jt + jj == i) ? 0.f : A.w * y;
            phi.add(term);
        }
    }
    const double mi = d.m[i];
    const double vx = d.pd[3 * np + i], vy = d.pd[4 * np + i], vz = d.pd[5 * np + i];
    d.eu[i] = mi * phi.as_double();
    d.ek[i] = 0.5 * mi * (vx * vx + vy * vy + vz * vz);
}

// One CTA per cluster: fixed-order sums of its slots' terms.
__global__ void k_ens_energy_sum(Dev d, Ens e)
{
    __shared__ double su[256], sk[256];
    const int c = blockIdx.x;
    const int cs = e.cs[c], cnp = e.cnp[c];
    double u = 0.0, k = 0.0;
    for (int i = cs + threadIdx.x; i < cs + cnp; i += blockDim.x) {
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
        e.K[c] = sk[0];
        e.U[c] = -0.5 * su[0];
    }
}

__global__ void k_ens_set_counts(Ens e)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < e.C) e.cnact[c] = e.cn[c];
}

}  // namespace gdk
