// merge.cu -- the bottom-up merge levels (White & Wortman, Sec. 2 "movie array";
// Sec. 3 main loop and kernel index math) and the face emission.
//
// Layout (one pass; the lower and upper passes have separate copies):
//   links lk[rank] = (prev, next)            in-place, as in the paper's P[].prev/next
//   event buffers W/A/B[2][2n]               ping-pong per level (the paper's A and B)
//   counts cnt[2][n]                         movie length, indexed by the node's first rank
// The node of level l with first rank lo covers [lo, min(lo + 2^l, n)); its
// movie occupies entries [2 lo, 2 lo + 2 m) of buffer (l & 1) (the paper's
// eventListOffset = 2 * leftGroupIndex).  Nodes of one level touch disjoint
// rank ranges, so the in-place link updates never race.
#include <type_traits>

#include "internal.h"
#include "merge.cuh"

namespace hull3d {

__device__ __forceinline__ void set_status2(int32_t *status, int code) { atomicCAS(status, 0, code); }

size_t fused_smem_bytes(int l1);

// ---------------------------------------------------------------------------
// One level in global memory, one thread per merge.
// ---------------------------------------------------------------------------
// The event loop's candidates live in shared memory (cand_smem_bytes of
// dynamic shared memory) rather than in a per-thread local array.
// Adds the events of a level to its statistics counter, one atomic per group of
// converged threads (the merges of a level number in the millions).
__device__ __forceinline__ void count_events(unsigned long long *lev_events, int level, int k)
{
    const unsigned m = __activemask();
    const unsigned sum = __reduce_add_sync(m, (unsigned)k);
    if ((int)(threadIdx.x & 31) == __ffs(m) - 1 && sum) atomicAdd(lev_events + level, (unsigned long long)sum);
}

// ---------------------------------------------------------------------------
// Levels 1 and 2 in one launch: one thread per (pass, node of four ranks)
// links the node's pairs (the state after level 1) and merges them
// (kinetic_merge_pairs).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_level2(Points pts, Span sp, PassBufs p0, PassBufs p1, int ab_level,
                                                int32_t *status)
{
    if (*status) return;
    const int64_t lo = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) << 2;
    int64_t hi, end;
    if (!node_span(sp, 2, lo, hi, end)) return;
    const bool upper = blockIdx.y != 0;
    const PassBufs &pb = upper ? p1 : p0;
    const int m = (int)(hi - lo);
    const int r0 = (int)lo;
    int2 *glk = pb.lk;
    glk[r0] = make_int2(NIL, m > 1 ? r0 + 1 : NIL);
    if (m > 1) glk[r0 + 1] = make_int2(r0, NIL);
    if (m > 2) glk[r0 + 2] = make_int2(NIL, m > 3 ? r0 + 3 : NIL);
    if (m > 3) glk[r0 + 3] = make_int2(r0 + 2, NIL);
    int *cdst = pb.cnt[0];  // level 2 writes buffer 0
    if (m <= 2) {  // no right child: the pair's (or point's) empty movie passes through
        cdst[lo] = 0;
        return;
    }
    GPtsX gp;  // pairs of equal x are common here: no float filter
    gp.P = pts.P;
    GLinks lk{ glk };
    const bool keep_ab = 2 >= ab_level || hi == end;
    GEvOut out{ pb.W[0] + 2 * lo, keep_ab ? pb.A[0] + 2 * lo : nullptr, keep_ab ? pb.B[0] + 2 * lo : nullptr };
    int err = 0;
    const int k = kinetic_merge_pairs(gp, lk, r0, m, out, upper, &err);
    cdst[lo] = k;
    if (err) set_status2(status, HULL3D_ERR_INTERNAL);
    count_events(pb.lev_events, 2, k);
}

void launch_level2(const Points &pts, const Span &sp, PassBufs *passes, int ab_level, int32_t *status, cudaStream_t st)
{
    const int64_t nodes = (sp.n + 3) >> 2;
    k_level2<<<dim3((unsigned)((nodes + 127) / 128), 2), 128, 0, st>>>(pts, sp, passes[0], passes[1], ab_level,
                                                                      status);
}

// Merge order of one level: the (pass, node) entries sorted by the merge's
// child event count, longest first.  In x-order, neighbouring merges take
// quite different numbers of rounds and a warp runs as long as its longest
// merge (about 70% of the lanes busy on a uniform cube); sorted, the 32 merges
// of a warp take about as many rounds each.  With `typed`, merges are first
// grouped by how their points share x-values (the x-value changes along the
// node, up to three, and whether the two children meet on one x-value): where
// most points share x-values with others (the
// lowest levels of clouds with several points per x-value) the comparisons of
// such merges take the same tie tiers, so a warp of one kind diverges less.
__global__ void k_order_keys(Points pts, Span sp, int level, PassBufs p0, PassBufs p1, int64_t nodes, bool typed,
                             uint64_t *keys, uint32_t *vals)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 2 * nodes) return;
    const int pass = i >= nodes ? 1 : 0;
    const int64_t node = pass ? i - nodes : i;
    const int src = (level - 1) & 1;
    const int64_t lo = node << level, mid = lo + (1ll << (level - 1));
    unsigned work = 0;  // no node, or one without a right child: sorts last (k_level skips it)
    unsigned kind = 7;
    int64_t hi;
    if (node_span(sp, level, lo, hi) && mid < hi) {
        const int *c = (pass ? p1 : p0).cnt[src];
        const unsigned w = (unsigned)c[lo] + (unsigned)c[mid];
        work = (w < 0x1ffeu ? w : 0x1ffeu) + 1;
        kind = 0;
        if (typed) {  // x-value changes along the node (at most 3), and whether the children meet on one
            int changes = 0, xp = pts.P[lo].x;
            for (int64_t r = lo + 1; r < hi && changes < 3; r++) {
                const int x = pts.P[r].x;
                changes += x != xp;
                xp = x;
            }
            kind = (unsigned)changes * 2u + (pts.P[mid - 1].x == pts.P[mid].x ? 0u : 1u);
        }
    }
    keys[i] = (kind << 13) | (0x1fffu - work);
    vals[i] = ((uint32_t)pass << 31) | (uint32_t)node;
}

// order == nullptr: merge (pass = blockIdx.y, node = thread index); else the
// thread's entry of the sorted merge order.
// The event neighbours (A, B) of a parent movie are kept only from level
// ab_level on and for the node that ends at its cloud's end: the time-window
// kernels read them from the children of their merges, the faces from the
// root movie, and the last node of a level is the one a pass-through copy may
// carry upwards.
template <int MINB, bool FILT>
__global__ void __launch_bounds__(128, MINB) k_level(Points pts, Span sp, int level, PassBufs p0, PassBufs p1,
                                                     int max_events, const uint32_t *order, int64_t entries,
                                                     int ab_level, int32_t *status)
{
    if (*status) return;
    int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool upper = blockIdx.y != 0;
    if (order) {
        if (node >= entries) return;
        const uint32_t e = order[node];
        upper = (e >> 31) != 0;
        node = e & 0x7fffffffu;
    }
    const int64_t lo = node << level;
    int64_t hi, end;
    if (!node_span(sp, level, lo, hi, end)) return;
    const int src = (level - 1) & 1, dst = level & 1;
    const int64_t half = 1ll << (level - 1);
    const int64_t mid = lo + half;
    if (mid >= hi) return;  // pass-through nodes are copied by k_passthrough
    const int *csrc = upper ? p1.cnt[src] : p0.cnt[src];
    int *cdst = upper ? p1.cnt[dst] : p0.cnt[dst];
    const unsigned *Wsrc = upper ? p1.W[src] : p0.W[src];
    unsigned *Wdst = upper ? p1.W[dst] : p0.W[dst];
    int *Adst = upper ? p1.A[dst] : p0.A[dst], *Bdst = upper ? p1.B[dst] : p0.B[dst];
    int nl = csrc[lo], nr = csrc[mid];
    if (max_events >= 0 && nl + nr > max_events) return;  // left to the time-segment kernels
    typename std::conditional<FILT, GPts, GPtsX>::type gp;
    gp.P = pts.P;
    GLinks lk{ upper ? p1.lk : p0.lk };
    GEvIn L{ Wsrc + 2 * lo }, R{ Wsrc + 2 * mid };
    const bool keep_ab = level >= ab_level || hi == end;
    GEvOut out{ Wdst + 2 * lo, keep_ab ? Adst + 2 * lo : nullptr, keep_ab ? Bdst + 2 * lo : nullptr };
    int err = 0;
    extern __shared__ long long cand_sm[];  // the block's event-loop candidates
    const CandSmem cs{ (int *)(cand_sm + 3 * 6 * blockDim.x), cand_sm, (int)blockDim.x, (int)threadIdx.x };
    const int k = kinetic_merge_sm(gp, lk, (int)mid - 1, (int)mid, (int)mid, L, nl, R, nr, out, (int)(2 * (hi - lo)),
                                   upper, &err, cs);
    cdst[lo] = k;
    if (err) set_status2(status, HULL3D_ERR_INTERNAL);
    count_events(upper ? p1.lev_events : p0.lev_events, level, k);
}

// The last node of a cloud's level may have no right child: its movie is the
// child's.  bpc blocks per cloud copy it (grid.x = clouds x bpc, grid.y = pass).
__global__ void k_passthrough(Span sp, int ncl, int bpc, int level, PassBufs p0, PassBufs p1, int32_t *status)
{
    if (*status) return;
    const bool up = blockIdx.y != 0;
    const int src = (level - 1) & 1, dst = level & 1;
    const unsigned *Ws = up ? p1.W[src] : p0.W[src];
    const int *As = up ? p1.A[src] : p0.A[src], *Bs = up ? p1.B[src] : p0.B[src];
    unsigned *Wd = up ? p1.W[dst] : p0.W[dst];
    int *Ad = up ? p1.A[dst] : p0.A[dst], *Bd = up ? p1.B[dst] : p0.B[dst];
    const int *cs = up ? p1.cnt[src] : p0.cnt[src];
    int *cd = up ? p1.cnt[dst] : p0.cnt[dst];
    const int part = (int)blockIdx.x % bpc;
    for (int c = (int)blockIdx.x / bpc; c < ncl; c += (int)gridDim.x / bpc) {
        int64_t base = 0, end = sp.n;
        if (sp.blk) {
            if (sp.ctop[c] < level || sp.cstat[c]) continue;
            base = sp.cbase[c];
            end = sp.cend[c];
        }
        const int64_t lo = base + (((end - base - 1) >> level) << level);
        if (lo + (1ll << (level - 1)) < end) continue;  // the last node has a right child
        const int cnt = cs[lo];
        for (int64_t e = part * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)bpc * blockDim.x) {
            Wd[2 * lo + e] = Ws[2 * lo + e];
            Ad[2 * lo + e] = As[2 * lo + e];
            Bd[2 * lo + e] = Bs[2 * lo + e];
        }
        if (part == 0 && threadIdx.x == 0) cd[lo] = cnt;
    }
}

int launch_passthrough(const Span &sp, int ncl, int level, PassBufs *passes, int32_t *status, cudaStream_t st)
{
    if (!sp.blk) {  // one cloud: only when its last node has no right child
        const int64_t lo = ((sp.n - 1) >> level) << level;
        if (lo + (1ll << (level - 1)) < sp.n) return 0;
        int64_t blocks = (2 * (sp.n - lo) + 255) / 256;
        if (blocks > 1024) blocks = 1024;
        k_passthrough<<<dim3((unsigned)blocks, 2), 256, 0, st>>>(sp, 1, (int)blocks, level, passes[0], passes[1],
                                                                 status);
        return 1;
    }
    const int g = ncl < 4096 ? ncl : 4096;
    k_passthrough<<<dim3((unsigned)(g > 0 ? g : 1), 2), 256, 0, st>>>(sp, ncl, 1, level, passes[0], passes[1], status);
    return 1;
}

int launch_level(const Points &pts, const Span &sp, int level, PassBufs *passes, int npass, int32_t *status,
                 cudaStream_t st, int occupancy, int max_events, const LevelOrder *ord, int ab_level, bool filter)
{
    int launches = 0;
    const int64_t nodes = (sp.n + (1ll << level) - 1) >> level;
    dim3 g((unsigned)((nodes + 127) / 128), npass);
    const uint32_t *order = nullptr;
    int64_t entries = 0;
    if (ord && npass == 2) {
        entries = 2 * nodes;
        k_order_keys<<<(unsigned)((entries + 255) / 256), 256, 0, st>>>(pts, sp, level, passes[0], passes[1], nodes,
                                                                         ord->typed, ord->k0, ord->v0);
        int64_t sl = 0;
        const int which = radix_sort_pairs(ord->k0, ord->v0, ord->k1, ord->v1, entries, nullptr, 16, ord->ss, st, &sl);
        launches += 1 + (int)sl;
        order = which ? ord->v1 : ord->v0;
        g = dim3((unsigned)((entries + 127) / 128), 1);
    }
    const int sm = cand_smem_bytes(128, filter);
    const Points &P = pts;
    PassBufs &a = passes[0], &b = passes[npass - 1];
    const int ab = ab_level;
#define LEVEL_ARGS P, sp, level, a, b, max_events, order, entries, ab, status
    if (occupancy >= 4) {
        if (filter) k_level<4, true><<<g, 128, sm, st>>>(LEVEL_ARGS);
        else k_level<4, false><<<g, 128, sm, st>>>(LEVEL_ARGS);
    } else if (occupancy == 3) {
        if (filter) k_level<3, true><<<g, 128, sm, st>>>(LEVEL_ARGS);
        else k_level<3, false><<<g, 128, sm, st>>>(LEVEL_ARGS);
    } else if (occupancy == 2) {
        if (filter) k_level<2, true><<<g, 128, sm, st>>>(LEVEL_ARGS);
        else k_level<2, false><<<g, 128, sm, st>>>(LEVEL_ARGS);
    } else {
        if (filter) k_level<1, true><<<g, 128, sm, st>>>(LEVEL_ARGS);
        else k_level<1, false><<<g, 128, sm, st>>>(LEVEL_ARGS);
    }
#undef LEVEL_ARGS
    launches++;
    return launches;
}

// ---------------------------------------------------------------------------
// Upper levels: one warp per merge on a compacted copy in shared memory.
// The points a merge can touch are the event points of its two children plus
// the four x-extremes (lo, mid-1, mid, hi-1): an x-extreme of a child is on
// the child's hull at every time, every other hull vertex has an event, and
// the links of these points (t = -inf hull links, or event-time links) only
// lead to such points.  The warp gathers them -- child movies read
// coalesced -- into a slot table (a rank -> slot map in global scratch makes
// each point's slot unique), one lane runs the serial merge at shared-memory
// latency, and the warp writes the links and the parent movie back.
// ---------------------------------------------------------------------------
struct CEvIn {
    const unsigned *W;
    __device__ __forceinline__ unsigned w(int i) const { return W[i]; }
};
struct CEvOut {  // slots stay in shared memory (backward pass), ranks go to global memory
    unsigned *S, *W;
    int *A, *B;
    const int *RK;
    __device__ __forceinline__ void put(int k, unsigned w, int a, int b)
    {
        S[k] = w;
        W[k] = (unsigned)RK[w & RANK_MASK] | (w & INS_BIT);
        A[k] = RK[a];
        B[k] = RK[b];
    }
    __device__ __forceinline__ unsigned w(int k) const { return S[k]; }
};

constexpr int CMP_THREADS = 32;

// Merges with more than max_events child events are left to the time-segment
// kernels (max_events < 0: none).
__global__ void __launch_bounds__(CMP_THREADS) k_level_cmp(Points pts, Span sp, int level, PassBufs p0, PassBufs p1,
                                                           int scap, int max_events, int32_t *status)
{
    extern __shared__ int sm[];
    __shared__ int s_k, s_bad;
    if (*status) return;
    const bool upper = blockIdx.y != 0;
    const int64_t lo = (int64_t)blockIdx.x << level;
    int64_t hi;
    if (!node_span(sp, level, lo, hi)) return;
    const int64_t half = 1ll << (level - 1);
    const int64_t mid = lo + half;
    if (mid >= hi) return;  // pass-through nodes are copied by k_passthrough
    const int src = (level - 1) & 1, dst = level & 1;
    const int *csrc = upper ? p1.cnt[src] : p0.cnt[src];
    int *cdst = upper ? p1.cnt[dst] : p0.cnt[dst];
    const unsigned *Wsrc = upper ? p1.W[src] : p0.W[src];
    unsigned *Wdst = upper ? p1.W[dst] : p0.W[dst];
    int *Adst = upper ? p1.A[dst] : p0.A[dst], *Bdst = upper ? p1.B[dst] : p0.B[dst];
    int2 *glk = upper ? p1.lk : p0.lk;
    int *gmap = upper ? p1.gmap : p0.gmap;
    const int nl = csrc[lo], nr = csrc[mid];
    if (max_events >= 0 && nl + nr > max_events) return;
    const int ns = nl + nr + 4;
    const int tid = threadIdx.x;
    const int cap = (int)(2 * (hi - lo));
    if (ns > scap) {  // too big for the table: the plain global-memory merge
        if (tid == 0) {
            GPts gp{ pts.P };
            GLinks lk{ glk };
            GEvIn L{ Wsrc + 2 * lo }, R{ Wsrc + 2 * mid };
            GEvOut out{ Wdst + 2 * lo, Adst + 2 * lo, Bdst + 2 * lo };
            int err = 0;
            int k = kinetic_merge(gp, lk, (int)mid - 1, (int)mid, (int)mid, L, nl, R, nr, out, cap, upper, &err);
            cdst[lo] = k;
            if (err) set_status2(status, HULL3D_ERR_INTERNAL);
            atomicAdd((upper ? p1.lev_events : p0.lev_events) + level, (unsigned long long)k);
        }
        return;
    }
    int4 *sPt = (int4 *)sm;                   // slot -> (x, y, z, input index)
    int2 *sLk = (int2 *)(sPt + scap);         // slot -> (prev, next) slots
    int *sRK = (int *)(sLk + scap);           // slot -> rank
    unsigned *sIn = (unsigned *)(sRK + scap);  // the two child movies as slots (nl + nr <= scap)
    unsigned *sOut = sIn + scap;              // the parent movie as slots (<= 2 scap)
    const unsigned *Lw = Wsrc + 2 * lo, *Rw = Wsrc + 2 * mid;
    const int e0 = (int)lo, e1 = (int)mid - 1, e2 = (int)mid, e3 = (int)hi - 1;
    // entry e: 0..3 the x-extremes, then the left movie, then the right movie
    auto entry = [&](int e) -> unsigned {
        return e < 4 ? (unsigned)(e == 0 ? e0 : e == 1 ? e1 : e == 2 ? e2 : e3)
                     : (e < 4 + nl ? Lw[e - 4] : Rw[e - 4 - nl]);
    };
    if (tid == 0) s_bad = 0;
    for (int e = tid; e < ns; e += CMP_THREADS) gmap[entry(e) & RANK_MASK] = 0x7fffffff;
    __syncthreads();
    for (int e = tid; e < ns; e += CMP_THREADS) atomicMin(&gmap[entry(e) & RANK_MASK], e);
    __syncthreads();
    // slot of a linked rank, checked against the table (never indexes out of it)
    auto slot_of = [&](int r) -> int {
        if (r < 0) return NIL;
        int s = gmap[r];
        if (s < 0 || s >= ns || (int)(entry(s) & RANK_MASK) != r) { s_bad = 1; return NIL; }
        return s;
    };
    for (int e = tid; e < ns; e += CMP_THREADS) {
        unsigned raw = entry(e);
        int r = (int)(raw & RANK_MASK);
        int s = gmap[r];
        if (e >= 4) sIn[e - 4] = (unsigned)s | (raw & INS_BIT);
        if (s == e) {
            sPt[e] = pts.P[r];
            sRK[e] = r;
            int2 l = glk[r];
            sLk[e] = make_int2(slot_of(l.x), slot_of(l.y));
        }
    }
    __syncthreads();
    if (!s_bad) {
        CPts cp{ sPt, sRK };
        CLinks lk{ sLk };
        CEvIn L{ sIn }, R{ sIn + nl };
        CEvOut out{ sOut, Wdst + 2 * lo, Adst + 2 * lo, Bdst + 2 * lo, sRK };
        int err = 0;
        int u = gmap[e1], v = gmap[e2];
        if (tid == 0) bridge_walk(cp, lk, u, v, (const Tri *)nullptr, upper);  // follows links: serial
        u = __shfl_sync(0xffffffffu, u, 0);
        v = __shfl_sync(0xffffffffu, v, 0);
        Tri none;
        none.p = none.q = none.r = -2;
        none.s = 0;
        const int k = kinetic_forward_warp(cp, lk, u, v, none, false, L, nl, R, nr, out, min(cap, 2 * scap), upper,
                                           false, &err);
        if (tid == 0) {
            if (err) s_bad = 1;
            else kinetic_backward(cp, lk, u, v, (int)mid, out, k);
            s_k = k;
        }
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) set_status2(status, HULL3D_ERR_INTERNAL);
        return;
    }
    for (int e = tid; e < ns; e += CMP_THREADS) {
        int r = (int)(entry(e) & RANK_MASK);
        if (gmap[r] == e) {
            int2 l = sLk[e];
            glk[r] = make_int2(l.x < 0 ? NIL : sRK[l.x], l.y < 0 ? NIL : sRK[l.y]);
        }
    }
    if (tid == 0) {
        cdst[lo] = s_k;
        atomicAdd((upper ? p1.lev_events : p0.lev_events) + level, (unsigned long long)s_k);
    }
}

size_t cmp_smem_bytes(int scap) { return (size_t)scap * (sizeof(int4) + sizeof(int2) + 4 * sizeof(int)); }


void launch_level_cmp(const Points &pts, const Span &sp, int level, PassBufs *passes, int npass, int32_t *status,
                      cudaStream_t st, int scap, int max_events)
{
    const int64_t nodes = (sp.n + (1ll << level) - 1) >> level;
    dim3 g((unsigned)nodes, npass);
    k_level_cmp<<<g, CMP_THREADS, cmp_smem_bytes(scap), st>>>(pts, sp, level, passes[0], passes[npass - 1], scap,
                                                              max_events, status);
}

// ---------------------------------------------------------------------------
// Fused bottom levels: one CTA merges a block of 2^l1 ranks through levels
// 1..l1 in shared memory, for both passes, then writes the links and the
// level-l1 movies to global memory.
// ---------------------------------------------------------------------------
struct SEvIn {
    const unsigned *W;
    __device__ __forceinline__ unsigned w(int i) const { return W[i]; }
};
struct SEvOut {  // intermediate levels keep only the event points
    unsigned *W;
    __device__ __forceinline__ void put(int k, unsigned w, int, int) { W[k] = w; }
    __device__ __forceinline__ unsigned w(int k) const { return W[k]; }
};

constexpr int FUSED_THREADS = 256;

__global__ void __launch_bounds__(FUSED_THREADS) k_fused(Points pts, int64_t n, int l1, PassBufs p0, PassBufs p1,
                                                         int npass, int32_t *status)
{
    extern __shared__ int sm[];
    if (*status) return;
    const int Bcap = 1 << l1;
    const int64_t base = blockIdx.x * (int64_t)Bcap;
    const int B = (int)((base + Bcap <= n) ? Bcap : n - base);
    int4 *sPt = (int4 *)sm;
    int2 *sLk = (int2 *)(sPt + Bcap);
    unsigned *sW0 = (unsigned *)(sLk + Bcap), *sW1 = sW0 + 2 * Bcap;
    int *sC0 = (int *)(sW1 + 2 * Bcap), *sC1 = sC0 + Bcap;
    for (int i = threadIdx.x; i < B; i += blockDim.x) sPt[i] = pts.P[base + i];
    SPts sp{ sPt, (int)base };
    SLinks lk{ sLk, (int)base };
    __shared__ unsigned lev_cnt[2][16];
    if (threadIdx.x < 32) lev_cnt[threadIdx.x >> 4][threadIdx.x & 15] = 0;
    int err = 0;
    for (int pass = 0; pass < npass; pass++) {
        const bool upper = pass != 0;
        unsigned *gW = upper ? p1.W[l1 & 1] : p0.W[l1 & 1];
        int *gA = upper ? p1.A[l1 & 1] : p0.A[l1 & 1], *gB = upper ? p1.B[l1 & 1] : p0.B[l1 & 1];
        int *gcnt = upper ? p1.cnt[l1 & 1] : p0.cnt[l1 & 1];
        int2 *glk = upper ? p1.lk : p0.lk;
        __syncthreads();
        for (int i = threadIdx.x; i < B; i += blockDim.x) { sLk[i] = make_int2(NIL, NIL); sC0[i] = 0; }
        __syncthreads();
        // a partial last block stops at its own top level; the node above it
        // has no right child, so its movie is the same
        int top = 0;
        while ((1 << top) < B) top++;
        for (int level = 1; level <= top; level++) {
            unsigned *Wsrc = (level & 1) ? sW0 : sW1, *Wdst = (level & 1) ? sW1 : sW0;
            int *Csrc = (level & 1) ? sC0 : sC1, *Cdst = (level & 1) ? sC1 : sC0;
            const int half = 1 << (level - 1);
            const int nodes = (B + 2 * half - 1) / (2 * half);
            const bool last = level == top;  // then nodes == 1 and the node has a right child
            for (int t = threadIdx.x; t < nodes; t += blockDim.x) {
                int llo = t * 2 * half, lmid = llo + half, lhi = min(llo + 2 * half, B);
                int64_t glo = base + llo;
                if (lmid >= lhi) {  // no right child: pass the movie through
                    int c = Csrc[llo];
                    for (int e = 0; e < c; e++) Wdst[2 * llo + e] = Wsrc[2 * llo + e];
                    Cdst[llo] = c;
                    continue;
                }
                SEvIn L{ Wsrc + 2 * llo }, R{ Wsrc + 2 * lmid };
                int k;
                if (last) {
                    GEvOut out{ gW + 2 * glo, gA + 2 * glo, gB + 2 * glo };
                    k = kinetic_merge(sp, lk, (int)(base + lmid) - 1, (int)(base + lmid), (int)(base + lmid), L,
                                      Csrc[llo], R, Csrc[lmid], out, 2 * (lhi - llo), upper, &err);
                } else {
                    SEvOut out{ Wdst + 2 * llo };
                    k = kinetic_merge(sp, lk, (int)(base + lmid) - 1, (int)(base + lmid), (int)(base + lmid), L,
                                      Csrc[llo], R, Csrc[lmid], out, 2 * (lhi - llo), upper, &err);
                }
                Cdst[llo] = k;
                if (k) atomicAdd(&lev_cnt[pass][level], (unsigned)k);
            }
            __syncthreads();
        }
        // write back links and the level-l1 count of this block's node
        int *Cfin = (top & 1) ? sC1 : sC0;
        for (int i = threadIdx.x; i < B; i += blockDim.x) glk[base + i] = sLk[i];
        if (threadIdx.x == 0) gcnt[base] = Cfin[0];
    }
    if (err) set_status2(status, HULL3D_ERR_INTERNAL);
    __syncthreads();
    if (threadIdx.x < 32) {
        int ps = threadIdx.x >> 4, lv = threadIdx.x & 15;
        unsigned c = lev_cnt[ps][lv];
        if (c && ps < npass) atomicAdd((ps ? p1.lev_events : p0.lev_events) + lv, (unsigned long long)c);
    }
}

size_t fused_smem_bytes(int l1) { return (size_t)(1 << l1) * (sizeof(int4) + sizeof(int2) + 6 * sizeof(int)); }

void launch_fused(const Points &pts, int64_t n, int l0, int l1, PassBufs *passes, int npass, int32_t *status,
                  cudaStream_t st)
{
    (void)l0;
    int64_t blocks = (n + (1ll << l1) - 1) >> l1;
    size_t smem = fused_smem_bytes(l1);
    // one thread per bottom merge: 2^(l1-1) threads, at least a warp
    int threads = 1 << (l1 - 1);
    if (threads < 32) threads = 32;
    if (threads > FUSED_THREADS) threads = FUSED_THREADS;
    k_fused<<<(unsigned)blocks, threads, smem, st>>>(pts, n, l1, passes[0], passes[npass - 1], npass, status);
}

// ---------------------------------------------------------------------------
// Faces: each root event (a, w, b) is one face (Sec. 2: one event per face).
// ---------------------------------------------------------------------------
__global__ void k_face_keys(Points pts, int64_t n, int level, PassBufs p0, PassBufs p1, int fbits, uint64_t *keys,
                            uint32_t *vals, int64_t *d_nfaces, int32_t *status)
{
    const int buf = level & 1;
    const int kl = p0.cnt[buf][0], ku = p1.cnt[buf][0];
    // a closed triangulated surface on at most n vertices has at most 2n - 4 faces
    const bool bad = (int64_t)kl + ku > 2 * n - 4;
    if (blockIdx.x == 0 && threadIdx.x == 0 && blockIdx.y == 0) {
        if (bad) set_status2(status, HULL3D_ERR_INTERNAL);
        *d_nfaces = (*status || bad) ? 0 : (int64_t)kl + ku;
    }
    if (*status || bad) return;
    const bool upper = blockIdx.y != 0;
    const unsigned *W_ = upper ? p1.W[buf] : p0.W[buf];
    const int *A_ = upper ? p1.A[buf] : p0.A[buf], *B_ = upper ? p1.B[buf] : p0.B[buf];
    const int cnt = upper ? ku : kl;
    GPts gp{ pts.P };
    // the face count is known on the device only: a grid sized to the GPU strides over it
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
        int w = (int)(W_[e] & RANK_MASK), a = A_[e], b = B_[e];
        P3 A = gp.get(a), W = gp.get(w), Bp = gp.get(b);
        // lower faces are oriented with the normal (w - a) x (b - a) pointing down
        // (Y~ < 0), upper faces with it pointing up
        bool up = turn_sign(A, W, Bp) > 0;
        int f0 = A.id, f1, f2;
        if (up == upper) { f1 = W.id; f2 = Bp.id; } else { f1 = Bp.id; f2 = W.id; }
        // rotate min-first
        if (f1 < f0 && f1 < f2) { int t = f0; f0 = f1; f1 = f2; f2 = t; }
        else if (f2 < f0 && f2 < f1) { int t = f2; f2 = f1; f1 = f0; f0 = t; }
        int64_t o = upper ? kl + e : e;
        keys[o] = ((uint64_t)f0 << fbits) | (uint64_t)f1;
        vals[o] = (uint32_t)f2;
    }
}

// Delaunay triangles: the lower pass's root events (a, w, b) whose points are
// not collinear in the plane, counter-clockwise in the plane, rotated
// min-first; zero-area events (a sliver the perturbation makes of points on
// one edge of the convex hull) get the largest key and are not counted.
// *d_items = the lower event count (keys written), *d_ntris = the triangles.
__global__ void k_tri_keys(Points pts, int64_t n, int level, PassBufs p0, int fbits, uint64_t *keys, uint32_t *vals,
                           int64_t *d_items, int64_t *d_ntris, int32_t *status)
{
    const int buf = level & 1;
    const int kl = p0.cnt[buf][0];
    const bool bad = (int64_t)kl > 2 * n - 4;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (bad) set_status2(status, HULL3D_ERR_INTERNAL);
        *d_items = (*status || bad) ? 0 : kl;
    }
    if (*status || bad) return;
    GPts gp{ pts.P };
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < kl; e += (int64_t)gridDim.x * blockDim.x) {
        const P3 A = gp.get(p0.A[buf][e]), W = gp.get((int)(p0.W[buf][e] & RANK_MASK)), B = gp.get(p0.B[buf][e]);
        const long long area = (long long)(W.x - A.x) * (B.y - A.y) - (long long)(B.x - A.x) * (W.y - A.y);
        if (area == 0) {
            keys[e] = ~0ull;
            vals[e] = 0;
            continue;
        }
        int f0 = A.id, f1, f2;
        if (area > 0) { f1 = W.id; f2 = B.id; } else { f1 = B.id; f2 = W.id; }
        if (f1 < f0 && f1 < f2) { int t = f0; f0 = f1; f1 = f2; f2 = t; }
        else if (f2 < f0 && f2 < f1) { int t = f2; f2 = f1; f1 = f0; f0 = t; }
        keys[e] = ((uint64_t)f0 << fbits) | (uint64_t)f1;
        vals[e] = (uint32_t)f2;
        atomicAdd((unsigned long long *)d_ntris, 1ull);
    }
}

static int face_grid();

void launch_tri_keys(const Points &pts, int64_t n, int level, PassBufs *passes, uint64_t *keys, uint32_t *vals,
                     int64_t *d_items, int64_t *d_ntris, int32_t *status, cudaStream_t st)
{
    int fbits = 1;
    while ((1ll << fbits) < n) fbits++;
    const int64_t need = (n + 255) / 256;
    const unsigned gx = (unsigned)(need < face_grid() ? need : face_grid());
    k_tri_keys<<<gx, 256, 0, st>>>(pts, n, level, passes[0], fbits, keys, vals, d_items, d_ntris, status);
}

static int face_grid()
{
    static int g = 0;
    if (!g) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g = sms > 0 ? 4 * sms : 512;
    }
    return g;
}

void launch_face_keys(const Points &pts, int64_t n, int level, PassBufs *passes, uint64_t *keys, uint32_t *vals,
                      int64_t *d_nfaces, int32_t *status, cudaStream_t st)
{
    int fbits = 1;
    while ((1ll << fbits) < n) fbits++;
    const int64_t need = (n + 255) / 256;  // at most n faces per pass
    const unsigned gx = (unsigned)(need < face_grid() ? need : face_grid());
    k_face_keys<<<dim3(gx, 2), 256, 0, st>>>(pts, n, level, passes[0], passes[1], fbits, keys, vals, d_nfaces, status);
}

__global__ void k_face_out(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int fbits,
                           const int64_t *d_nfaces, int32_t *__restrict__ faces)
{
    const int64_t nf = *d_nfaces;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
        faces[3 * i] = (int32_t)(k >> fbits);
        faces[3 * i + 1] = (int32_t)(k & ((1ull << fbits) - 1));
        faces[3 * i + 2] = (int32_t)vals[i];
    }
}

void launch_face_out(const uint64_t *keys, const uint32_t *vals, int64_t cap, int fbits, const int64_t *d_nfaces,
                          int32_t *faces, cudaStream_t st)
{
    const int64_t need = (cap + 255) / 256;
    const unsigned g = (unsigned)(need < face_grid() ? need : face_grid());
    k_face_out<<<g > 0 ? g : 1, 256, 0, st>>>(keys, vals, fbits, d_nfaces, faces);
}

// Shared-memory limits of the kernels that need more than the default; set
// once, before any launch or stream capture.
void merge_kernel_attributes()
{
    cudaFuncSetAttribute(k_level_cmp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cmp_smem_bytes(4096));
    cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem_bytes(10));
}

}  // namespace hull3d
