// segmerge.cu -- kernels of the time-segment-parallel merge (see segmerge.cuh).
#include "internal.h"
#include "segmerge.cuh"

namespace hull3d {

__device__ __forceinline__ void seg_status(int32_t *status, int code) { atomicCAS(status, 0, code); }

struct SegArgs {
    Points pts;
    Span sp;
    SegGeom geo;
    PassBufs pb[2];
    SegBufs sb[2];
    uint64_t *pairs;                 // keys; sorted in place between the kernels
    uint32_t *pair_vals;
    unsigned long long *npairs;
    int *overflow;
    int *nseg_merges;  // merges of this level that are merged in windows
    // device work lists (entries: pass << 31 | index)
    unsigned *wlist, *flist, *mlist;  // windows, windows to retry, merges in windows
    int *wcount, *fcount;
    unsigned *flist2;  // windows for the largest shared-memory table
    int *f2count;
    // windows too large for the biggest shared-memory table: a last round
    // with per-CTA slot tables of gcap slots in global memory (gtab, gstride
    // bytes apart); none when gtab is null
    unsigned *glist;
    int *gcount;
    int *nserial;  // merges of this level run by the serial fallback
    int *refit;    // window length multiplier of the second attempt (0: none)
    char *gtab;
    int64_t gstride;
    int gcap;
    int64_t S_cap, M_cap;
    int rbits;  // bits of a rank in a start-hull entry's key
    int32_t *status;
};

// ---- bounds: one thread per (merge, window) --------------------------------
__global__ void k_seg_bounds(SegArgs a, int second)
{
    if (*a.status) return;
    const int f = second ? *a.refit : 1;  // the second attempt runs only after a refit
    if (f <= 1 && second) return;
    const int pass = blockIdx.y;
    const SegGeom &G = a.geo;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t m = t / G.smax;
    const int s = (int)(t % G.smax);
    const int64_t half = 1ll << (G.level - 1);
    const int64_t lo = m << G.level;
    int64_t hi;
    if (!node_span(a.sp, G.level, lo, hi)) return;
    const int64_t mid = lo + half;
    if (mid >= hi) return;
    const PassBufs &pb = a.pb[pass];
    const SegBufs &sb = a.sb[pass];
    const int src = (G.level - 1) & 1;
    const int nl = pb.cnt[src][lo], nr = pb.cnt[src][mid];
    // small merges are done by the compacted kernel: no windows
    int len = seg_window_len(nl + nr, G.K, G.Kmin);
    if (f > 1) len = min(len * f, max(len, SEG_EVCAP_BIG));
    const int S = (nl + nr > G.min_events) ? seg_count(nl, nr, len, G.smax) : 0;
    if (s == 0) {
        sb.nseg[m] = S;
        sb.nofit[m] = 0;
        if (S) a.mlist[atomicAdd(a.nseg_merges, 1)] = ((unsigned)pass << 31) | (unsigned)m;
    }
    if (s >= S) return;
    const int64_t g = m * G.smax + s;
    a.wlist[atomicAdd(a.wcount, 1)] = ((unsigned)pass << 31) | (unsigned)g;
    int kL = 0;
    const int j = (int)(((int64_t)s * (nl + nr)) / S);
    if (s > 0) {
        GPts gp{ a.pts.P };
        const unsigned *W = pb.W[src];
        const int *A = pb.A[src], *B = pb.B[src];
        kL = merge_path(gp, W + 2 * lo, A + 2 * lo, B + 2 * lo, nl, W + 2 * mid, A + 2 * mid, B + 2 * mid, nr, j,
                        pass != 0);
    }
    sb.bound[g] = make_int2(kL, j - kL);
    // the x-extremes of both children are on their hulls at every time
    int ext[4] = { (int)lo, (int)mid - 1, (int)mid, (int)hi - 1 };
    int cnt = 2 + (ext[1] != ext[0]) + (ext[3] != ext[2]);
    unsigned long long pos = atomicAdd(a.npairs, (unsigned long long)cnt);
    if (pos + cnt > (unsigned long long)G.pair_cap) { atomicExch(a.overflow, 1); return; }
    a.pairs[pos++] = seg_key(pass, g, 0, ext[0], a.S_cap, a.rbits);
    if (ext[1] != ext[0]) a.pairs[pos++] = seg_key(pass, g, 0, ext[1], a.S_cap, a.rbits);
    a.pairs[pos++] = seg_key(pass, g, 1, ext[2], a.S_cap, a.rbits);
    if (ext[3] != ext[2]) a.pairs[pos++] = seg_key(pass, g, 1, ext[3], a.S_cap, a.rbits);
}

// Maps a position q of the level's source movie buffer to its child movie:
// returns false when q holds no event of a merged child.
__device__ __forceinline__ bool seg_locate(const Span &sp, const SegGeom &G, const PassBufs &pb, int64_t q,
                                           int64_t &clo, int64_t &plo, int &k, int &E)
{
    const int64_t half = 1ll << (G.level - 1);
    const int64_t r = q >> 1;
    if (r >= sp.n) return false;
    clo = r & ~(half - 1);
    plo = r & ~(2 * half - 1);
    const int64_t pmid = plo + half;
    int64_t phi;
    if (!node_span(sp, G.level, plo, phi)) return false;
    if (pmid >= phi) return false;  // pass-through node
    k = (int)(q - 2 * clo);
    E = pb.cnt[(G.level - 1) & 1][clo];
    return k < E;
}

// The child event positions of the merges that are cut into windows (the
// work list written by k_seg_bounds): when the list is shorter than the grid,
// several blocks share a merge; f(pass, q, valid) gets each position q once
// with valid = true (and is also called with valid = false to keep the lanes
// of a warp together).
template <class F>
__device__ __forceinline__ void for_windowed_events(const SegArgs &a, F &&f)
{
    const SegGeom &G = a.geo;
    const int nm = (int)*a.nseg_merges;
    if (nm == 0) return;
    const int bpm = (int)gridDim.x >= nm ? (int)gridDim.x / nm : 1;  // blocks per merge
    const int slots = (int)gridDim.x / bpm;                           // merges in flight
    if ((int)blockIdx.x / bpm >= slots) return;
    const int src = (G.level - 1) & 1;
    const int64_t half = 1ll << (G.level - 1);
    for (int idx = (int)blockIdx.x / bpm; idx < nm; idx += slots) {
        const unsigned e = a.mlist[idx];
        const int pass = (int)(e >> 31);
        const int64_t m = e & 0x7fffffffu;
        const int64_t lo = m << G.level, mid = lo + half;
        const PassBufs &pb = a.pb[pass];
        const int nl = pb.cnt[src][lo], nr = pb.cnt[src][mid];
        // warp-uniform trip count: every lane of a warp calls f in each round
        // (valid = false past the end), so f may use warp collectives
        const int64_t lane = threadIdx.x & 31;
        for (int64_t t = ((int)blockIdx.x % bpm) * (int64_t)blockDim.x + threadIdx.x; t - lane < nl + nr;
             t += (int64_t)bpm * blockDim.x)
            f(pass, t < nl ? 2 * lo + t : 2 * mid + (t - nl), t < nl + nr);
    }
}

// ---- idx: every event records its index under its point --------------------
__global__ void k_seg_idx(SegArgs a)
{
    if (*a.status) return;
    const int src = (a.geo.level - 1) & 1;
    const int64_t half = 1ll << (a.geo.level - 1);
    for_windowed_events(a, [&](int pass, int64_t q, bool valid) {
        if (!valid) return;
        const unsigned w = a.pb[pass].W[src][q];
        const int rk = (int)(w & RANK_MASK);
        const int k = (int)(q - 2 * ((q >> 1) & ~(half - 1)));  // index in the child movie
        if (w & INS_BIT) a.sb[pass].ins_idx[rk] = k;
        else a.sb[pass].del_idx[rk] = k;
    });
}

// ---- pairs: each event point joins the start hulls of the windows it spans --
__device__ void seg_pairs_one(const SegArgs &a, int pass, int64_t q, bool valid);

__global__ void k_seg_pairs(SegArgs a, int second)
{
    if (*a.status) return;
    if (second && *a.refit <= 1) return;
    for_windowed_events(a, [&](int pass, int64_t q, bool valid) { seg_pairs_one(a, pass, q, valid); });
}

// ---- refit: longer windows when the start hulls overflowed their buffer --
// The start-hull entries of a level are (windows) x (child hull sizes).  On
// the workloads the hulls grow as the square root of the points, but points on
// a convex surface in lattice order (a planar lattice lifted to the
// paraboloid: every column of equal x lies on one parabola) keep most of an
// extreme column on the hull, and the entries can exceed the buffer.  The
// counter still holds the level's whole demand, so one thread picks the
// smallest power-of-two multiplier f of the window lengths (at most 64, windows
// up to SEG_EVCAP_BIG events) that brings the demand under three quarters of
// the buffer, clears the level's lists, and the bounds and pairs run again
// with windows f times longer.  The windows that no longer fit the first
// round's tables take the retry rounds.
__global__ void k_seg_refit(SegArgs a)
{
    if (*a.status || !*a.overflow) return;
    const unsigned long long demand = *a.npairs;
    const unsigned long long room = (unsigned long long)(a.geo.pair_cap - a.geo.pair_cap / 4);
    int f = 2;
    while (f < 64 && demand > room * (unsigned long long)f) f <<= 1;
    *a.refit = f;
    *a.npairs = 0;
    *a.overflow = 0;
    *a.nseg_merges = 0;
    *a.wcount = 0;
}

__device__ void seg_pairs_one(const SegArgs &a, int pass, int64_t q, bool valid)
{
    // Called by all 32 lanes of a warp together.  Each lane finds the windows
    // whose start hull holds its event point; the warp then reserves room for
    // all of its entries with one atomic (a single counter serves the level).
    const SegGeom &G = a.geo;
    int64_t clo = 0, plo = 0;
    int k = 0, E = 0, cnt = 0, s_first = 0, rk = 0, child = 0;
    int64_t m = 0;
    const PassBufs &pb = a.pb[pass];
    const SegBufs &sb = a.sb[pass];
    if (valid && seg_locate(a.sp, G, pb, q, clo, plo, k, E)) {
        const unsigned *CW = pb.W[(G.level - 1) & 1] + 2 * clo;
        const unsigned w = CW[k];
        rk = (int)(w & RANK_MASK);
        int lo_p = 0, hi_p = -1;  // alive after i child events iff lo_p < i <= hi_p
        bool counted = true;
        if (w & INS_BIT) {
            lo_p = k;
            const int dd = sb.del_idx[rk];
            hi_p = (dd > k && dd < E && (int)(CW[dd] & RANK_MASK) == rk && !(CW[dd] & INS_BIT)) ? dd : E;
        } else {
            const int ii = sb.ins_idx[rk];
            // a point inserted before its delete is counted at its insert
            counted = !(ii >= 0 && ii < k && (int)(CW[ii] & RANK_MASK) == rk && (CW[ii] & INS_BIT));
            lo_p = -1;
            hi_p = k;
        }
        if (counted) {
            child = clo == plo ? 0 : 1;
            m = plo >> G.level;
            const int S = sb.nseg[m];
            const int2 *bd = sb.bound + m * G.smax;
            // windows s with lo_p < kC_s <= hi_p (kC_s is nondecreasing in s)
            int b0 = 0, b1 = S;
            while (b0 < b1) {
                int c = (b0 + b1) >> 1;
                int kc = child ? bd[c].y : bd[c].x;
                if (kc > lo_p) b1 = c; else b0 = c + 1;
            }
            s_first = b0;
            b0 = s_first; b1 = S;
            while (b0 < b1) {
                int c = (b0 + b1) >> 1;
                int kc = child ? bd[c].y : bd[c].x;
                if (kc <= hi_p) b0 = c + 1; else b1 = c;
            }
            cnt = b0 - s_first;
        }
    }
    // exclusive prefix of cnt over the warp, one atomic for the warp's total
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += y;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total > 0) base = atomicAdd(a.npairs, (unsigned long long)total);
    base = __shfl_sync(FULL, base, 31);
    if (total == 0) return;
    if (base + (unsigned long long)total > (unsigned long long)G.pair_cap) {
        if (lane == 0) atomicExch(a.overflow, 1);
        return;
    }
    unsigned long long pos = base + (unsigned long long)(incl - cnt);
    for (int s = s_first; s < s_first + cnt; s++) a.pairs[pos++] = seg_key(pass, m * G.smax + s, child, rk, a.S_cap, a.rbits);
}

// ---- merge: one warp per window ---------------------------------------------
struct SegOut {  // slots in, ranks out
    unsigned *W;
    int *A, *B;
    const int *RK;
    __device__ __forceinline__ void put(int k, unsigned w, int a, int b)
    {
        W[k] = (unsigned)RK[w & RANK_MASK] | (w & INS_BIT);
        A[k] = RK[a];
        B[k] = RK[b];
    }
};

struct SegIn {
    const unsigned *W;
    __device__ __forceinline__ unsigned w(int i) const { return W[i]; }
};

constexpr int SEG_THREADS = 32;

// first index in [0, cnt) of keys >= key
__device__ __forceinline__ int64_t lower_key(const uint64_t *keys, int64_t cnt, uint64_t key)
{
    int64_t lo = 0, hi = cnt;
    while (lo < hi) {
        int64_t m = (lo + hi) >> 1;
        if (keys[m] < key) lo = m + 1; else hi = m;
    }
    return lo;
}

// retry = 0: every window, slot table of geo.scap in shared memory; a window
// that does not fit goes to the retry list.  retry = 1: those windows, with a
// shared-memory table of `cap` slots (two CTAs per SM); retry = 2: the ones
// that still did not fit, with the largest shared-memory table (one CTA per
// SM); retry = 3: the rest, with a table of `cap` slots in global memory.  A
// window that fits none sends its merge to the serial fallback.
__device__ void seg_window(const SegArgs &a, int pass, int64_t g, int retry, int cap);

__global__ void __launch_bounds__(SEG_THREADS) k_seg_merge(SegArgs a, int retry, int cap)
{
    if (*a.status) return;
    const unsigned *list = retry == 3 ? a.glist : retry == 2 ? a.flist2 : retry ? a.flist : a.wlist;
    const int cnt = retry == 3 ? *a.gcount : retry == 2 ? *a.f2count : retry ? *a.fcount : *a.wcount;
    for (int it = blockIdx.x; it < cnt; it += gridDim.x) {
        const unsigned e = list[it];
        seg_window(a, (int)(e >> 31), (int64_t)(e & 0x7fffffffu), retry, cap);
        __syncthreads();
    }
}

// One window: its start hulls and inserted points in a slot table, the start
// bridge, the event loop.  All threads of the (one-warp) CTA call it.
__device__ void seg_window(const SegArgs &a, int pass, int64_t g, int retry, int cap)
{
    extern __shared__ int sm[];
    __shared__ int s_bad, s_nins;
    const bool upper = pass != 0;
    const SegGeom &G = a.geo;
    const int64_t m = g / G.smax;
    const int s = (int)(g % G.smax);
    const int64_t half = 1ll << (G.level - 1);
    const int64_t lo = m << G.level;
    int64_t hi;
    if (!node_span(a.sp, G.level, lo, hi)) return;
    const int64_t mid = lo + half;
    if (mid >= hi) return;
    const PassBufs &pb = a.pb[pass];
    const SegBufs &sb = a.sb[pass];
    const int S = sb.nseg[m];
    if (s >= S) return;
    if (*a.overflow) { if (threadIdx.x == 0) sb.nofit[m] = 1; return; }
    const int scap = retry ? cap : G.scap;
    const int evcap = retry ? SEG_EVCAP_BIG : G.K;  // child events the window's table holds
    const int tid = threadIdx.x;
    const int src = (G.level - 1) & 1;
    const int nl = pb.cnt[src][lo], nr = pb.cnt[src][mid];
    const int2 b0 = sb.bound[g];
    const int2 b1 = (s + 1 < S) ? sb.bound[g + 1] : make_int2(nl, nr);
    const unsigned *LW = pb.W[src] + 2 * lo, *RW = pb.W[src] + 2 * mid;
    const int wl = b1.x - b0.x, wr = b1.y - b0.y;
    // start hulls
    const int64_t np = (int64_t)*a.npairs;
    const int64_t aL0 = lower_key(a.pairs, np, seg_key(pass, g, 0, 0, a.S_cap, a.rbits));
    const int64_t aR0 = lower_key(a.pairs, np, seg_key(pass, g, 1, 0, a.S_cap, a.rbits));
    const int64_t aR1 = lower_key(a.pairs, np, seg_key(pass, g + 1, 0, 0, a.S_cap, a.rbits));
    const int aL = (int)(aR0 - aL0), aR = (int)(aR1 - aR0);
    // inserted points of the window
    if (tid == 0) { s_bad = 0; s_nins = 0; }
    __syncthreads();
    int nins_local = 0;
    for (int e = tid; e < wl + wr; e += SEG_THREADS) {
        unsigned w = e < wl ? LW[b0.x + e] : RW[b0.y + e - wl];
        nins_local += (w & INS_BIT) ? 1 : 0;
    }
    atomicAdd(&s_nins, nins_local);
    __syncthreads();
    const int nins = s_nins;
    const int base_ins = aL + aR;
    const int tsize = base_ins + nins + 3;  // + the three points of the window's boundary event
    if (wl + wr > SEG_EVCAP_BIG + 1 || aL < 1 || aR < 1) {  // cannot happen for valid movies
        if (tid == 0) sb.nofit[m] = 1;
        return;
    }
    if (tsize > scap || wl + wr > evcap + 1) {
        if (tid == 0) {
            const unsigned e = ((unsigned)pass << 31) | (unsigned)g;
            if (retry == 0) a.flist[atomicAdd(a.fcount, 1)] = e;
            else if (retry == 1) a.flist2[atomicAdd(a.f2count, 1)] = e;
            else if (retry == 2 && a.gtab) a.glist[atomicAdd(a.gcount, 1)] = e;
            else sb.nofit[m] = 1;
        }
        return;
    }
    // the slot table: this CTA's region of global memory in the last round
    int4 *sPt = retry == 3 ? (int4 *)(a.gtab + (int64_t)blockIdx.x * a.gstride) : (int4 *)sm;
    int2 *sLk = (int2 *)(sPt + scap);
    int *sRK = (int *)(sLk + scap);
    unsigned *sIn = (unsigned *)(sRK + scap);  // window movies as slots: left then right
    // start hulls, linked in x-order
    for (int i = tid; i < aL + aR; i += SEG_THREADS) {
        const bool left = i < aL;
        const int r = (int)(a.pairs[aL0 + i] & ((1ull << a.rbits) - 1));
        sRK[i] = r;
        sPt[i] = a.pts.P[r];
        const int first = left ? 0 : aL, last = left ? aL - 1 : aL + aR - 1;
        sLk[i] = make_int2(i > first ? i - 1 : NIL, i < last ? i + 1 : NIL);
    }
    // slots of the inserted points, in window order (warp prefix over ballots)
    {
        int run = 0;
        for (int e0 = 0; e0 < wl + wr; e0 += SEG_THREADS) {
            const int e = e0 + tid;
            unsigned w = 0;
            if (e < wl + wr) w = e < wl ? LW[b0.x + e] : RW[b0.y + e - wl];
            const bool ins = e < wl + wr && (w & INS_BIT);
            const unsigned bal = __ballot_sync(0xffffffffu, ins);
            if (ins) {
                const int slot = base_ins + run + __popc(bal & ((1u << tid) - 1u));
                const int r = (int)(w & RANK_MASK);
                sRK[slot] = r;
                sPt[slot] = a.pts.P[r];
                sb.smap[r] = slot;
            }
            run += __popc(bal);
        }
    }
    __syncthreads();
    // rank -> slot: binary search in the child's start hull, else an inserted point
    auto find = [&](int r, int child) -> int {
        if (r < 0) return NIL;
        int f = child ? aL : 0, l = child ? aL + aR : aL;
        while (f < l) {
            int c = (f + l) >> 1;
            if (sRK[c] < r) f = c + 1; else l = c;
        }
        if (f < (child ? aL + aR : aL) && sRK[f] == r) return f;
        const int sl = sb.smap[r];
        if (sl >= base_ins && sl < base_ins + nins && sRK[sl] == r) return sl;
        s_bad = 1;
        return NIL;
    };
    for (int i = tid; i < nins; i += SEG_THREADS) {
        const int slot = base_ins + i;
        const int r = sRK[slot];
        const int child = r >= (int)mid ? 1 : 0;
        const int2 l = pb.lk[r];  // neighbours at its insertion
        sLk[slot] = make_int2(find(l.x, child), find(l.y, child));
    }
    for (int e = tid; e < wl + wr; e += SEG_THREADS) {
        const bool left = e < wl;
        const unsigned w = left ? LW[b0.x + e] : RW[b0.y + e - wl];
        sIn[e] = (unsigned)find((int)(w & RANK_MASK), left ? 0 : 1) | (w & INS_BIT);
    }
    __syncthreads();
    if (!s_bad) {
        CPts cp{ sPt, sRK };
        CLinks lk{ sLk };
        Tri at;
        at.s = 0;
        const int tb = base_ins + nins;
        if (s > 0) {  // the window starts just after the latest child event before it
            if (tid == 0) {
                GPts gp{ a.pts.P };
                const int *A = pb.A[src], *B = pb.B[src];
                int eb;  // index of that event in the source buffer
                if (b0.x > 0 && b0.y > 0) {
                    Tri tl, tr;
                    ev_tri(gp, pb.W[src], A, B, (int)(2 * lo) + b0.x - 1, tl);
                    ev_tri(gp, pb.W[src], A, B, (int)(2 * mid) + b0.y - 1, tr);
                    eb = tri_cmp(gp, tl, tr, upper) > 0 ? (int)(2 * lo) + b0.x - 1 : (int)(2 * mid) + b0.y - 1;
                } else {
                    eb = b0.x > 0 ? (int)(2 * lo) + b0.x - 1 : (int)(2 * mid) + b0.y - 1;
                }
                const int rr[3] = { A[eb], (int)(pb.W[src][eb] & RANK_MASK), B[eb] };
                for (int q = 0; q < 3; q++) {
                    sRK[tb + q] = rr[q];
                    sPt[tb + q] = a.pts.P[rr[q]];
                    sLk[tb + q] = make_int2(NIL, NIL);
                }
            }
            __syncwarp();
            tri_make(cp, at, tb, tb + 1, tb + 2);
        }
        int u = aL - 1, v = aL;  // the inner x-extremes mid - 1 and mid
        bridge_walk_warp(cp, 0, aL + aR - 1, u, v, s > 0 ? &at : (const Tri *)nullptr, upper);
        if (s == 0 && tid == 0) sb.bridge0[m] = make_int2(sRK[u], sRK[v]);
        SegIn L{ sIn }, R{ sIn + wl };
        const int64_t ob = seg_out_base(G.level, G.smax, m, s, b0.x + b0.y);
        SegOut out{ sb.oW + ob, sb.oA + ob, sb.oB + ob, sRK };
        int err = 0;
        const int k = kinetic_forward_warp(cp, lk, u, v, at, s > 0, L, wl, R, wr, out, 2 * (wl + wr) + 256, upper,
                                           s + 1 < S, &err);
        if (tid == 0) {
            sb.ocnt[g] = k;
            if (err) s_bad = 1;
        }
    }
    __syncthreads();
    if (tid == 0 && s_bad) sb.nofit[m] = 1;
}

// ---- concat: one CTA per merge ------------------------------------------------
constexpr int CAT_THREADS = 256;

__device__ void seg_concat_one(const SegArgs &a, int pass, int64_t m);

__global__ void __launch_bounds__(CAT_THREADS) k_seg_concat(SegArgs a)
{
    if (*a.status) return;
    const int cnt = *a.nseg_merges;
    for (int it = blockIdx.x; it < cnt; it += gridDim.x) {
        const unsigned e = a.mlist[it];
        seg_concat_one(a, (int)(e >> 31), (int64_t)(e & 0x7fffffffu));
        __syncthreads();
    }
}

__device__ void seg_concat_one(const SegArgs &a, int pass, int64_t m)
{
    __shared__ int s_off[CAT_THREADS + 1];
    const SegGeom &G = a.geo;
    const int64_t half = 1ll << (G.level - 1);
    const int64_t lo = m << G.level;
    int64_t hi;
    if (!node_span(a.sp, G.level, lo, hi)) return;
    const int64_t mid = lo + half;
    if (mid >= hi) return;
    const PassBufs &pb = a.pb[pass];
    const SegBufs &sb = a.sb[pass];
    if (sb.nofit[m]) return;  // merged serially by k_seg_fallback
    const int dst = G.level & 1;
    const int S = sb.nseg[m];
    if (S == 0) return;  // merged by the compacted kernel
    unsigned *W = pb.W[dst] + 2 * lo;
    int *A = pb.A[dst] + 2 * lo, *B = pb.B[dst] + 2 * lo;
    int base = 0;
    for (int s0 = 0; s0 < S; s0 += CAT_THREADS) {
        // exclusive scan of this chunk's window counts
        const int s = s0 + threadIdx.x;
        const int c = s < S ? sb.ocnt[m * G.smax + s] : 0;
        s_off[threadIdx.x + 1] = c;
        if (threadIdx.x == 0) s_off[0] = 0;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int t = 1; t <= CAT_THREADS; t++) s_off[t] += s_off[t - 1];
        __syncthreads();
        const int chunk = min(CAT_THREADS, S - s0);
        for (int t = 0; t < chunk; t++) {
            const int64_t g = m * G.smax + s0 + t;
            const int2 bd = sb.bound[g];
            const int64_t ob = seg_out_base(G.level, G.smax, m, s0 + t, bd.x + bd.y);
            const int off = base + s_off[t];
            const int cnt = s_off[t + 1] - s_off[t];
            for (int e = threadIdx.x; e < cnt; e += CAT_THREADS) {
                const unsigned w = sb.oW[ob + e];
                const int aa = sb.oA[ob + e], bb = sb.oB[ob + e];
                W[off + e] = w;
                A[off + e] = aa;
                B[off + e] = bb;
                if (w & INS_BIT) pb.lk[w & RANK_MASK] = make_int2(aa, bb);  // event-time links of an insertion
            }
        }
        base += s_off[chunk];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pb.cnt[dst][lo] = base;
        const int2 br = sb.bridge0[m];  // join the two t = -inf hulls
        pb.lk[br.x].y = br.y;
        pb.lk[br.y].x = br.x;
        atomicAdd(pb.lev_events + G.level, (unsigned long long)base);
    }
}

// ---- fallback: serial merge of the merges that did not fit -------------------
__global__ void k_seg_fallback(SegArgs a)
{
    if (*a.status) return;
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= *a.nseg_merges) return;
    const unsigned e = a.mlist[it];
    const int pass = (int)(e >> 31);
    const SegGeom &G = a.geo;
    const int64_t m = (int64_t)(e & 0x7fffffffu);
    const int64_t half = 1ll << (G.level - 1);
    const int64_t lo = m << G.level;
    int64_t hi;
    if (!node_span(a.sp, G.level, lo, hi)) return;
    const int64_t mid = lo + half;
    if (mid >= hi) return;
    const PassBufs &pb = a.pb[pass];
    if (!a.sb[pass].nofit[m] || a.sb[pass].nseg[m] == 0) return;
    atomicAdd(a.nserial, 1);
    const int src = (G.level - 1) & 1, dst = G.level & 1;
    GPts gp{ a.pts.P };
    GLinks lk{ pb.lk };
    GEvIn L{ pb.W[src] + 2 * lo }, R{ pb.W[src] + 2 * mid };
    GEvOut out{ pb.W[dst] + 2 * lo, pb.A[dst] + 2 * lo, pb.B[dst] + 2 * lo };
    int err = 0;
    int k = kinetic_merge(gp, lk, (int)mid - 1, (int)mid, (int)mid, L, pb.cnt[src][lo], R, pb.cnt[src][mid], out,
                          (int)(2 * (hi - lo)), pass != 0, &err);
    pb.cnt[dst][lo] = k;
    if (err) seg_status(a.status, HULL3D_ERR_INTERNAL);
    atomicAdd(pb.lev_events + G.level, (unsigned long long)k);
}

void seg_kernel_attributes()
{
    cudaFuncSetAttribute(k_seg_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

size_t seg_smem_bytes(int scap, int K) { return (size_t)scap * (sizeof(int4) + sizeof(int2) + sizeof(int)) + 4 * (K + 1); }

void launch_seg_level(const Points &pts, const Span &sp, int level, PassBufs *passes, SegBufs *sbufs, uint64_t *pairs,
                      uint32_t *pair_vals, uint64_t *pairs_alt, uint32_t *vals_alt, unsigned long long *npairs,
                      int *overflow, int64_t pair_cap, int64_t S_cap, int64_t M_cap, int K, int Kmin, int scap,
                      int scap_big, int min_events, const SortScratch &ss, const SegTables &gt, int32_t *status,
                      cudaStream_t st, int64_t *launches)
{
    SegArgs a;
    a.pts = pts;
    a.sp = sp;
    const int64_t n = sp.n;  // the rank space
    a.geo.n = n;
    a.geo.level = level;
    a.geo.K = K;
    a.geo.Kmin = Kmin;
    a.geo.smax = (int)(((1ll << (level + 1)) + Kmin - 1) / Kmin);
    a.geo.scap = scap;
    a.geo.pair_cap = pair_cap;
    a.geo.min_events = min_events;
    a.pb[0] = passes[0];
    a.pb[1] = passes[1];
    a.sb[0] = sbufs[0];
    a.sb[1] = sbufs[1];
    a.npairs = npairs;
    a.overflow = overflow;
    a.S_cap = S_cap;
    a.M_cap = M_cap;
    a.rbits = 1;  // the ranks of the rank space: below n
    while ((1ll << a.rbits) < n) a.rbits++;
    a.status = status;
    const int64_t M = (n + (1ll << level) - 1) >> level;
    const int64_t G = M * a.geo.smax;
    a.nseg_merges = overflow + 1;
    a.wcount = overflow + 2;
    a.fcount = overflow + 3;
    a.gcount = overflow + 4;
    a.nserial = overflow + 5;
    a.refit = overflow + 6;
    a.wlist = sbufs[0].wlist;
    a.flist = sbufs[0].flist;
    a.flist2 = sbufs[0].flist2;
    a.f2count = overflow + 7;
    a.mlist = sbufs[0].mlist;
    a.glist = sbufs[0].glist;
    a.gtab = gt.base;
    a.gstride = gt.stride;
    a.gcap = gt.cap;
    cudaMemsetAsync(npairs, 0, sizeof(unsigned long long), st);
    a.pairs = pairs;
    a.pair_vals = pair_vals;
    k_seg_bounds<<<dim3((unsigned)((G + 127) / 128), 2), 128, 0, st>>>(a, 0);
    static int flat_grid = 0;
    if (!flat_grid) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        flat_grid = sms > 0 ? 4 * sms : 512;
    }
    int64_t fg = (2 * n + 255) / 256;
    if (fg > flat_grid) fg = flat_grid;
    k_seg_idx<<<(unsigned)fg, 256, 0, st>>>(a);
    k_seg_pairs<<<(unsigned)fg, 256, 0, st>>>(a, 0);
    // a second attempt with longer windows, run only when the start hulls overflowed
    k_seg_refit<<<1, 1, 0, st>>>(a);
    k_seg_bounds<<<dim3((unsigned)((G + 127) / 128), 2), 128, 0, st>>>(a, 1);
    k_seg_pairs<<<(unsigned)fg, 256, 0, st>>>(a, 1);
    *launches += 6;
    int key_bits = a.rbits;
    while ((1ll << (key_bits - a.rbits)) < 4 * S_cap) key_bits++;
    int which = radix_sort_pairs(pairs, pair_vals, pairs_alt, vals_alt, pair_cap, (const int64_t *)npairs, key_bits, ss,
                                 st, launches);
    a.pairs = which ? pairs_alt : pairs;
    a.pair_vals = which ? vals_alt : pair_vals;
    // persistent grids over the device work lists: up to 16 one-warp CTAs per
    // SM (small tables fit that many; registers allow about 9)
    const int wg = flat_grid * 4;
    k_seg_merge<<<wg, SEG_THREADS, seg_smem_bytes(scap, K), st>>>(a, 0, scap);
    const int mid = scap_big < SEG_SLOTS_MID ? scap_big : SEG_SLOTS_MID;
    k_seg_merge<<<flat_grid / 2 > 0 ? flat_grid / 2 : 1, SEG_THREADS, seg_smem_bytes(mid, SEG_EVCAP_BIG), st>>>(
        a, 1, mid);
    k_seg_merge<<<flat_grid / 4 > 0 ? flat_grid / 4 : 1, SEG_THREADS, seg_smem_bytes(scap_big, SEG_EVCAP_BIG), st>>>(
        a, 2, scap_big);
    *launches += 1;
    if (gt.base) {
        k_seg_merge<<<gt.ctas, SEG_THREADS, 0, st>>>(a, 3, gt.cap);
        *launches += 1;
    }
    k_seg_concat<<<flat_grid, CAT_THREADS, 0, st>>>(a);
    const int64_t fb_threads = 2 * M;
    k_seg_fallback<<<(unsigned)((fb_threads + 63) / 64), 64, 0, st>>>(a);
    *launches += 4;
}

}  // namespace hull3d
