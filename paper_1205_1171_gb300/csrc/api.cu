// api.cu -- the C ABI: plan (all scratch allocated up front), the level driver
// (the paper's host "main outer loop", Sec. 3, replayed without host syncs)
// and the entry points declared in include/hull3d.h.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <climits>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"
#include "segmerge.cuh"

using namespace hull3d;

namespace {

thread_local int g_last_cuda = 0;

int cuda_fail(cudaError_t e)
{
    g_last_cuda = (int)e;
    return HULL3D_ERR_CUDA;
}

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

// HULL3D_DEBUG_SYNC=1: synchronise after every step and name the failing one
// on stderr (a diagnostic mode; the default path never synchronises or prints).
bool debug_sync()
{
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("HULL3D_DEBUG_SYNC");
        v = (e && *e && *e != '0') ? 1 : 0;
    }
    return v == 1;
}

int step_check(cudaStream_t st, const char *what)
{
    if (!debug_sync()) return HULL3D_OK;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "hull3d: step '%s' failed: %s\n", what, cudaGetErrorString(e));
        return cuda_fail(e);
    }
    return HULL3D_OK;
}

#define STEP(what)                                  \
    do {                                            \
        int rc_ = step_check(st, what);             \
        if (rc_) return rc_;                        \
    } while (0)

int ceil_log2(int64_t n)
{
    int l = 0;
    while ((1ll << l) < n) l++;
    return l;
}

}  // namespace

struct hull3d_plan_s {
    int64_t max_n = 0, max_clouds = 0;
    hull3d_opts opts{};
    int device = 0;
    char *pool = nullptr;
    size_t pool_bytes = 0;
    // sort (capacity 2 max_n: also used for the face sort)
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr;
    SortScratch ss{};
    // rank-ordered points
    int4 *P4 = nullptr;
    PassBufs pass[2]{};
    int32_t *status = nullptr;
    int64_t *nfaces = nullptr;
    int64_t *items = nullptr;  // device count of a sort's items (Delaunay triangle keys)
    // the point sort's long runs of one x-value: [0] the full-sort count (0, or n when the runs do not fit),
    // [1] the number of long runs (as an int), then their starts and lengths
    int64_t *sortfb = nullptr;
    int32_t *stage_xyz = nullptr, *stage_faces = nullptr;
    // pinned host mirrors
    int64_t *h_nfaces = nullptr;
    int32_t *h_status = nullptr;
    int64_t last_launches = 0;
    unsigned long long *lev_stats = nullptr;  // [2][64]
    // time-segment-parallel levels
    SegBufs seg[2]{};
    uint64_t *pk0 = nullptr, *pk1 = nullptr;
    uint32_t *pv0 = nullptr, *pv1 = nullptr;
    unsigned long long *npairs = nullptr;
    int *overflow = nullptr;
    int64_t pair_cap = 0, S_cap = 0, M_cap = 0;
    SegTables gtab{};  // global-memory slot tables of the time windows too large for shared memory
    // phase profiling
    bool profile = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<int> marks;  // per recorded call: HULL3D_PHASES + 1 event indices
    std::vector<int> level_marks;  // per recorded level launch: (level, start event, end event)
    // CUDA graphs of the whole pipeline, keyed by the call's arguments
    struct GraphEntry {
        const void *xyz;
        int64_t n;
        void *faces, *nf, *status;
        cudaGraphExec_t exec;
        int64_t launches;
        uint64_t used;
    };
    static constexpr int kGraphs = 8;
    GraphEntry graphs[kGraphs]{};
    uint64_t graph_clock = 0;
    cudaStream_t cap_stream = nullptr;  // private stream the pipeline is captured on
    // batched clouds: per-cloud metadata uploaded for the persistent kernels
    int64_t *b_off = nullptr, *b_foff = nullptr;
    int32_t *b_order = nullptr;
    int *b_counter = nullptr;
    std::vector<int32_t> h_order;
    int sms = 0;
    // groups of large clouds hulled together (multi.cu)
    MultiTables mt{};
    int64_t mt_cap = 0;  // clouds per group
};

namespace {

// Shared-memory limits of every kernel that needs more than the default, for
// the current device; set before the first launch or stream capture there.
void kernel_attributes()
{
    merge_kernel_attributes();
    sort_kernel_attributes();
    seg_kernel_attributes();
    batch_kernel_attributes();
}

struct Bump {
    char *base;
    size_t off, cap;
    template <class T>
    T *take(int64_t count)
    {
        size_t bytes = ((size_t)count * sizeof(T) + 255) & ~(size_t)255;
        T *p = (T *)(base ? base + off : nullptr);
        off += bytes;
        return p;
    }
};

int default_seg_level(const hull3d_plan_s *p);
int default_seg_events(const hull3d_plan_s *p);
int default_seg_events_min(const hull3d_plan_s *p);
int default_seg_slots(const hull3d_plan_s *p);

// Lays out every buffer of the plan; with base == nullptr it only measures.
size_t layout(hull3d_plan_s *p, char *base)
{
    const int64_t N = p->max_n, N2 = 2 * p->max_n;
    Bump b{ base, 0, 0 };
    p->k0 = b.take<uint64_t>(N2);
    p->k1 = b.take<uint64_t>(N2);
    p->v0 = b.take<uint32_t>(N2);
    p->v1 = b.take<uint32_t>(N2);
    p->ss.max_tiles = (N2 + SORT_TILE - 1) / SORT_TILE;
    p->ss.hist = b.take<uint32_t>(256 * p->ss.max_tiles);
    p->ss.rowsum = b.take<uint32_t>(256);
    p->P4 = b.take<int4>(N);
    for (int s = 0; s < 2; s++) {
        PassBufs &pb = p->pass[s];
        for (int k = 0; k < 2; k++) {
            pb.W[k] = b.take<unsigned>(N2);
            pb.A[k] = b.take<int32_t>(N2);
            pb.B[k] = b.take<int32_t>(N2);
            pb.cnt[k] = b.take<int32_t>(N);
        }
        pb.lk = b.take<int2>(N);
        pb.gmap = b.take<int32_t>(N);
    }
    // time-segment-parallel levels: window scratch sized for the largest level
    {
        int Lmax = 0;
        while ((1ll << Lmax) < N) Lmax++;
        const int sl = default_seg_level(p), Kmin = default_seg_events_min(p);
        p->S_cap = p->M_cap = 0;
        for (int lv = sl > 2 ? sl : 2; lv <= Lmax; lv++) {
            const int64_t M = (N + (1ll << lv) - 1) >> lv;
            const int64_t smax = ((1ll << (lv + 1)) + Kmin - 1) / Kmin;
            if (M * smax > p->S_cap) p->S_cap = M * smax;
            if (M > p->M_cap) p->M_cap = M;
        }
        // window outputs (seg_out_base): 4 per rank of the padded level plus 256 per window
        const int64_t out_cap = 4 * (1ll << Lmax) + 256 * p->S_cap;
        // start-hull entries of one level: windows x (the two child hull sizes).
        // Points on a sphere are the worst case of the workloads: its child hulls
        // hold ~0.8 sqrt(m) points, so the top levels of a 2^20-point sphere need
        // ~4.7 n entries; beyond the budget a level's windowed merges run serially.
        p->pair_cap = p->S_cap ? 8 * N + 8 * p->S_cap : 0;
        for (int s = 0; s < 2 && p->S_cap; s++) {
            SegBufs &sb = p->seg[s];
            sb.bound = b.take<int2>(p->S_cap);
            sb.nseg = b.take<int>(p->M_cap);
            sb.ins_idx = b.take<int>(N);
            sb.del_idx = b.take<int>(N);
            sb.smap = b.take<int>(N);
            sb.oW = b.take<unsigned>(out_cap);
            sb.oA = b.take<int>(out_cap);
            sb.oB = b.take<int>(out_cap);
            sb.ocnt = b.take<int>(p->S_cap);
            sb.bridge0 = b.take<int2>(p->M_cap);
            sb.nofit = b.take<int>(p->M_cap);
            if (s == 0) {
                sb.wlist = b.take<unsigned>(2 * p->S_cap);
                sb.flist = b.take<unsigned>(2 * p->S_cap);
                sb.glist = b.take<unsigned>(2 * p->S_cap);
                sb.flist2 = b.take<unsigned>(2 * p->S_cap);
                sb.mlist = b.take<unsigned>(2 * p->M_cap);
            }
        }
        if (p->S_cap) {
            p->pk0 = b.take<uint64_t>(p->pair_cap);
            p->pk1 = b.take<uint64_t>(p->pair_cap);
            p->pv0 = b.take<uint32_t>(p->pair_cap);
            p->pv1 = b.take<uint32_t>(p->pair_cap);
            p->npairs = b.take<unsigned long long>(1);
            // per merge level, the window counters (SEG_STAT_STRIDE ints per level)
            p->overflow = b.take<int>(SEG_STAT_STRIDE * 64);
            // one global-memory slot table per SM for windows whose start hulls exceed the largest shared-memory
            // table (hull-heavy clouds of 2^22 points and more): 32768 slots, windows of up to 4096 child events
            p->gtab.cap = N >= (1 << 20) ? 32768 : 8192;
            p->gtab.ctas = p->sms > 0 ? p->sms : 132;
            p->gtab.stride = ((int64_t)seg_smem_bytes(p->gtab.cap, 4096) + 255) & ~(int64_t)255;
            p->gtab.base = b.take<char>(p->gtab.stride * p->gtab.ctas);
            // the pair sort needs histogram space for pair_cap items
            int64_t tiles = (p->pair_cap + SORT_TILE - 1) / SORT_TILE;
            if (tiles > p->ss.max_tiles) {
                p->ss.max_tiles = tiles;
                p->ss.hist = b.take<uint32_t>(256 * tiles);
            }
        }
    }
    // tables of a group of large clouds: blocks of at least 2^SPAN_SHIFT ranks
    p->mt_cap = (N >> SPAN_SHIFT) + 1;
    p->mt.blk = b.take<int32_t>(p->mt_cap);
    p->mt.cbase = b.take<int64_t>(p->mt_cap);
    p->mt.cend = b.take<int64_t>(p->mt_cap);
    p->mt.coff = b.take<int64_t>(p->mt_cap + 1);
    p->mt.ioff = b.take<int64_t>(p->mt_cap);
    p->mt.cfoff = b.take<int64_t>(p->mt_cap);
    p->mt.ctop = b.take<int32_t>(p->mt_cap);
    p->mt.cstat = b.take<int32_t>(p->mt_cap);
    p->mt.corig = b.take<int32_t>(p->mt_cap);
    p->mt.fcount = b.take<int64_t>(p->mt_cap);
    p->mt.fstart = b.take<int64_t>(p->mt_cap + 1);
    p->lev_stats = b.take<unsigned long long>(128);
    p->b_off = b.take<int64_t>(p->max_clouds + 1);
    p->b_foff = b.take<int64_t>(p->max_clouds + 1);
    p->b_order = b.take<int32_t>(p->max_clouds + 1);
    p->b_counter = b.take<int>(BATCH_CLASSES);
    p->pass[0].lev_events = p->lev_stats;
    p->pass[1].lev_events = p->lev_stats + 64;
    p->status = b.take<int32_t>(1);
    p->nfaces = b.take<int64_t>(1);
    p->items = b.take<int64_t>(1);
    p->sortfb = b.take<int64_t>(2 + TIE_SORT_LONG_CAP + TIE_SORT_LONG_CAP / 2);
    p->stage_xyz = b.take<int32_t>(3 * N);
    p->stage_faces = b.take<int32_t>(3 * N2);
    return b.off;
}

// The adjacency kernels' scratch, laid over the start of the plan's pool (the
// hull's buffers are free once its faces are written): keys and edge ids for
// 3 F <= 6 max_n directed edges, twice, and their sort histograms.  With
// base == nullptr it only measures.
size_t adj_layout(const hull3d_plan_s *p, char *base, AdjScratch *s)
{
    const int64_t E = 6 * p->max_n;
    Bump b{ base, 0, 0 };
    s->k0 = b.take<uint64_t>(E);
    s->k1 = b.take<uint64_t>(E);
    s->v0 = b.take<uint32_t>(E);
    s->v1 = b.take<uint32_t>(E);
    s->ss.max_tiles = (E + SORT_TILE - 1) / SORT_TILE;
    s->ss.hist = b.take<uint32_t>(256 * s->ss.max_tiles);
    s->ss.rowsum = b.take<uint32_t>(256);
    s->n3 = b.take<int64_t>(1);
    return b.off;
}

// Defaults from the measured level sweeps (2^24 cube and clipped Gaussian,
// GB300): no fused bottom kernel; the thread-per-merge kernel with 168
// registers (3 blocks per SM) at levels 6-8, 128 registers (4 blocks) at
// levels 2-5 and 9, and uncapped for levels 10-12.
int default_fused(const hull3d_plan_s *p) { return p->opts.fused_levels > 0 ? p->opts.fused_levels : 1; }
int default_occupancy(const hull3d_plan_s *p, int level)
{
    if (p->opts.level_occupancy > 0) return p->opts.level_occupancy;
    if (level >= 6 && level <= 8) return 3;
    return level <= 9 ? 4 : 1;
}
// First level of the compacted warp-per-merge kernel for a hull of 2^L points
// (L = ceil(log2 n)): one thread per merge pays while a level has enough merges
// to fill the GPU, one warp per merge after that.  log2(n) - 11, within [6, 13],
// was at or within 1% of the best cut-over measured for every n from 2^12 to
// 2^24 (cube, ball, sphere, clipped Gaussian).
int default_cmp_level(const hull3d_plan_s *p, int L)
{
    if (p->opts.cmp_level > 0) return p->opts.cmp_level;
    const int c = L - 11;
    return c < 6 ? 6 : (c > 13 ? 13 : c);
}
int default_cmp_slots(const hull3d_plan_s *p) { return p->opts.cmp_slots > 0 ? p->opts.cmp_slots : 1024; }
// The compacted kernel's table on a level whose merges above max_events child
// events go to time windows: a merge it takes needs at most max_events + 4
// slots, and a smaller table fits more blocks per SM (2^24 cube: levels 13-15
// 25% faster with 544 slots than with 1024).
int cmp_slots_at(const hull3d_plan_s *p, int max_events)
{
    const int d = default_cmp_slots(p);
    if (p->opts.cmp_slots > 0 || max_events < 0) return d;
    const int need = (max_events + 4 + 31) / 32 * 32;
    return need < d ? need : d;
}
int default_seg_level(const hull3d_plan_s *p) { return p->opts.seg_level > 0 ? p->opts.seg_level : 10; }
int default_seg_min_events(const hull3d_plan_s *p)
{
    return p->opts.seg_min_events > 0 ? p->opts.seg_min_events : 512;
}
// The threshold at one level of a hull of n points: where a level has few
// merges (at most 128 per pass), a merge's serial event chain is the level's
// critical path, so merges above 128 child events are cut into windows too
// (2^24 cube and Gaussian: the top levels 1.2 -> 0.6 ms each; at 256 merges per
// pass the warp kernel is still faster).
int seg_min_events_at(const hull3d_plan_s *p, int64_t n, int level)
{
    if (p->opts.seg_min_events > 0) return p->opts.seg_min_events;
    const int64_t merges = n >> level;
    return merges <= 128 ? 128 : 512;
}
// Thread-per-merge levels 3-8 run their merges longest first (measured on the
// 2^24 cube and clipped Gaussian: 3% per hull).  Level 2's merges of
// event-free pairs are all alike, and from level 9 on there are too few merges
// for the sort to pay.
const LevelOrder *level_order(const hull3d_plan_s *p, int level, LevelOrder *ord, bool typed)
{
    ord->typed = typed;
    return (p->opts.merge_order >= 0 && level >= 3 && level <= 8) ? ord : nullptr;
}
// Last level whose merge order groups the merges by how their points share
// x-values (k_order_keys), for clouds of up to 2^L points: levels up to
// L - 19 (3 to 5 at 2^24 points, eight per x-value: levels 3-5 of the cube
// 19.5 -> 18.6 ms, of the Gaussian 21.5 -> 20.6 ms; at level 6 and above the
// work order alone is faster).
int default_typed_level(int L, bool lifted)
{
    const int xbits = lifted ? 16 : 21;
    return L - xbits + 2;
}
int default_seg_events(const hull3d_plan_s *p) { return p->opts.seg_events > 0 ? p->opts.seg_events : 512; }
// Longest time window of a level.  A window starts from both child hulls,
// whose size grows as the square root of the merge's points, so the
// start-hull entries of a level of merges of m points grow as m^1.5 while the
// buffer for them is linear in n: from a size on the windows double per level
// (1024, 2048, then 4096 child events).  Points lifted to a paraboloid (2D
// Delaunay) all lie on the lower hull and need that from level 21 (a 2^22-point
// triangulation overflows the buffer with 512 and falls back to the serial
// merge: 18.7 s instead of 0.48 s); the hull of points on a sphere, the worst
// 3D case of the workloads, fits with 512 through level 22 (2^22 sphere: 376 ms
// with 512, 422 ms with the longer windows) and needs it from level 23.
int seg_events_at(const hull3d_plan_s *p, int level, bool lifted)
{
    if (p->opts.seg_events > 0) return p->opts.seg_events;
    const int from = lifted ? 21 : 23;
    if (level < from) return 512;
    return level >= from + 2 ? 4096 : 1024 << (level - from);
}
int default_seg_events_min(const hull3d_plan_s *p)
{
    const int K = default_seg_events(p);
    const int k = p->opts.seg_events_min > 0 ? p->opts.seg_events_min : 128;
    return k < K ? k : K;
}
int default_seg_slots(const hull3d_plan_s *p) { return p->opts.seg_slots > 0 ? p->opts.seg_slots : 1536; }
int seg_events_at(const hull3d_plan_s *p, int level, bool lifted);
// The first-round slot table of a level's time windows: its start hulls (two
// child hulls, at most ~1.45 sqrt(m) points each on the workloads, m = 2^(level-1)
// child points: points on a paraboloid; ~1.1 sqrt(m) on a sphere) plus the
// points a window inserts (at most its length, 2 sqrt(E) for E <= 2^(level+1)
// child events, within the level's limits).  4 sqrt(2^level) + that length
// leaves about twice the room the hulls need; a window that does not fit goes
// to the retry rounds.  Smaller tables put more windows on an SM (the register
// limit allows 9 one-warp CTAs): 288 slots at level 10 instead of 1536.
int seg_slots_at(const hull3d_plan_s *p, int level, bool lifted)
{
    const int d = default_seg_slots(p);
    if (p->opts.seg_slots > 0) return d;
    const int K = seg_events_at(p, level, lifted);
    const int Kmin = p->opts.seg_events_min > 0 ? std::min(p->opts.seg_events_min, K) : std::min(128, K);
    const double e = 2.0 * std::sqrt((double)(1ll << (level + 1)));
    const int kl = (int)std::min<double>(K, std::max<double>(Kmin, e));
    const int need = ((int)(4.0 * std::sqrt((double)(1ll << level))) + kl + 8 + 31) / 32 * 32;
    return need < d ? need : d;
}
int default_seg_slots_big(const hull3d_plan_s *p) { return p->opts.seg_slots_big > 0 ? p->opts.seg_slots_big : 6144; }
// Batch kernel: one thread per merge while a level of a cloud has at least 64
// merges, then one warp per merge (the tuner may pick another cut-over).
int default_batch_warp_nodes(const hull3d_plan_s *p)
{
    return p->opts.batch_warp_nodes > 0 ? p->opts.batch_warp_nodes : 64;
}
// Rank space of one group of large clouds: the plan's max_n, or less.
int64_t default_multi_ranks(const hull3d_plan_s *p)
{
    return (p->opts.multi_ranks > 0 && p->opts.multi_ranks < p->max_n) ? p->opts.multi_ranks : p->max_n;
}

// First level of the thread-per-merge kernel whose time comparisons try the
// float filter, for clouds of up to 2^L points.  A cloud spanning the
// coordinate range has 2^21 x-values (2^16 for lifted planar points); with
// several points per x-value the low levels' triples through equal-x points
// tie in Z/Y, where the filter only adds work (at 2^24 points, eight per
// x-value, it cost 2-4% at levels 2-6 and gained from level 9 on; at 2^20 it
// gained from level 4).
int default_filter_level(const hull3d_plan_s *p, int L, bool lifted)
{
    if (p->opts.filter_level > 0) return p->opts.filter_level;
    const int xbits = lifted ? 16 : 21;
    return L > xbits ? std::max(3, L - xbits + 6) : 3;
}

// Records a phase-boundary event when profiling (one per boundary per call).
int mark(hull3d_plan_s *p, cudaStream_t st, int *slot)
{
    if (!p->profile) return HULL3D_OK;
    if (p->ev_used == p->ev_pool.size()) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        p->ev_pool.push_back(e);
    }
    *slot = (int)p->ev_used++;
    CK(cudaEventRecord(p->ev_pool[*slot], st));
    return HULL3D_OK;
}

#define MARK(k)                                      \
    do {                                             \
        int rc_ = mark(p, st, &slots[k]);            \
        if (rc_) return rc_;                         \
    } while (0)

// Enqueues merge levels l1 + 1 .. L over the rank space sp (one cloud, or
// ncl clouds in aligned blocks): one launch sequence per level for every
// node of every cloud at that level, with no host synchronisation.
int enqueue_levels(hull3d_plan_s *p, const Points &pts, const Span &sp, int ncl, int L, int l1, int32_t *status,
                   cudaStream_t st, int64_t *launches, int *slots, bool *seg_marked, bool lifted = false)
{
    const int64_t R = sp.n;  // the rank space: thresholds follow the merges a level holds
    LevelOrder ord{ p->k0, p->k1, p->v0, p->v1, p->ss, false };
    const int typed_to = default_typed_level(L, lifted);
    // parent movies keep their event neighbours from the level below the
    // first time-window level (whose kernels read them) and at the roots
    const int ab_level = p->S_cap ? std::min(default_seg_level(p) - 1, L) : L;
    const int LR = ceil_log2(R);
    const int filter_from = default_filter_level(p, L, lifted);
    if (p->S_cap) CK(cudaMemsetAsync(p->overflow, 0, sizeof(int) * SEG_STAT_STRIDE * 64, st));
    for (int level = l1 + 1; level <= L; level++) {
        // level 2 merges event-free pairs: its own kernel, never time windows
        const bool seg = level >= default_seg_level(p) && p->S_cap && level > 2;
        if (seg && !*seg_marked) { MARK(3); *seg_marked = true; }
        int lv0 = -1, lv1 = -1;
        if (p->profile) { int r_ = mark(p, st, &lv0); if (r_) return r_; }
        if (level == 2) {
            launch_level2(pts, sp, p->pass, ab_level, status, st);
            *launches += 1;
        } else if (seg) {
            // small merges on this level's usual kernel, large ones in time windows
            const int min_ev = seg_min_events_at(p, R, level);
            if (level >= default_cmp_level(p, LR)) {
                launch_level_cmp(pts, sp, level, p->pass, 2, status, st, cmp_slots_at(p, min_ev), min_ev);
                *launches += 1;
            } else {
                *launches += launch_level(pts, sp, level, p->pass, 2, status, st, default_occupancy(p, level), min_ev,
                                          level_order(p, level, &ord, level <= typed_to), ab_level,
                                          level >= filter_from);
            }
            launch_seg_level(pts, sp, level, p->pass, p->seg, p->pk0, p->pv0, p->pk1, p->pv1, p->npairs,
                             p->overflow + SEG_STAT_STRIDE * level,
                             p->pair_cap, p->S_cap, p->M_cap, seg_events_at(p, level, lifted), default_seg_events_min(p),
                             seg_slots_at(p, level, lifted), default_seg_slots_big(p), min_ev, p->ss, p->gtab, status,
                             st, launches);
        } else if (level >= default_cmp_level(p, LR)) {
            launch_level_cmp(pts, sp, level, p->pass, 2, status, st, default_cmp_slots(p));
            *launches += 1;
        } else {
            *launches += launch_level(pts, sp, level, p->pass, 2, status, st, default_occupancy(p, level), -1,
                                      level_order(p, level, &ord, level <= typed_to), ab_level,
                                          level >= filter_from);
        }
        if (level > 2) *launches += launch_passthrough(sp, ncl, level, p->pass, status, st);
        if (p->profile) {
            int r_ = mark(p, st, &lv1);
            if (r_) return r_;
            p->level_marks.insert(p->level_marks.end(), { level, lv0, lv1 });
        }
        STEP("merge level");
    }
    return HULL3D_OK;
}

// Enqueues the whole single-hull pipeline.
int enqueue_hull(hull3d_plan_s *p, const int32_t *d_xyz, int64_t n, int32_t *d_faces, int64_t *nf, int32_t *status,
                 cudaStream_t st)
{
    int64_t launches = 0;
    int slots[HULL3D_PHASES + 1];
    STEP("entry");
    MARK(0);
    CK(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
    CK(cudaMemsetAsync(p->lev_stats, 0, 128 * sizeof(unsigned long long), st));
    int which = 0;
    if (n <= SMALL_SORT_MAX) {  // one CTA: keys, sort, decode
        launch_small_sort(d_xyz, n, p->P4, status, st);
        launches++;
        STEP("small sort");
    } else {
        launch_keys(d_xyz, n, p->k0, p->v0, status, st);
        launches++;
        STEP("keys");
        // by x only (bits 39-62: three passes), then each x-value's few points
        // by the whole key; a cloud with too many points on one x-value takes
        // the full 63-bit sort instead (its launches see a zero count otherwise)
        CK(cudaMemsetAsync(p->sortfb, 0, 2 * sizeof(int64_t), st));
        radix_sort_pairs(p->k0, p->v0, p->k1, p->v1, n, nullptr, 24, p->ss, st, &launches, 39);
        const TieRuns runs{ p->sortfb, (int *)(p->sortfb + 1), p->sortfb + 2, (int *)(p->sortfb + 2 + TIE_SORT_LONG_CAP) };
        launch_tie_sort(p->k1, p->v1, p->k0, p->v0, n, TIE_SORT_MAX_RUN, runs, st);
        launches += 2;
        // the full sort of the x-sorted keys ends in (k1, v1) after its even number of passes
        radix_sort_pairs(p->k1, p->v1, p->k0, p->v0, n, p->sortfb, 63, p->ss, st, &launches);
        STEP("point sort");
        launch_decode_either(p->k0, p->v0, p->k1, p->v1, p->sortfb, n, p->P4, status, st);
        launches++;
        STEP("decode");
    }
    MARK(1);
    if (n < 3) {
        CK(cudaMemsetAsync(nf, 0, sizeof(int64_t), st));
        for (int k = 2; k <= HULL3D_PHASES; k++) MARK(k);
        if (p->profile) p->marks.insert(p->marks.end(), slots, slots + HULL3D_PHASES + 1);
        p->last_launches = launches;
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? HULL3D_OK : cuda_fail(e);
    }
    Points pts{ p->P4 };
    const int L = ceil_log2(n);
    int l1 = default_fused(p);
    if (l1 > L) l1 = L;
    if (l1 > 10) l1 = 10;
    if (l1 > 1) {  // otherwise the pairs of level 1 are linked by the level-2 kernel
        launch_fused(pts, n, 0, l1, p->pass, 2, status, st);
        launches++;
    }
    STEP("fused levels");
    MARK(2);
    bool seg_marked = false;
    {
        int rc = enqueue_levels(p, pts, single_span(n), 1, L, l1, status, st, &launches, slots, &seg_marked);
        if (rc) return rc;
    }
    if (!seg_marked) MARK(3);
    MARK(4);
    int fbits = ceil_log2(n);
    if (fbits < 1) fbits = 1;
    launch_face_keys(pts, n, L, p->pass, p->k0, p->v0, nf, status, st);
    launches++;
    STEP("face keys");
    if (n <= SMALL_SORT_MAX) {  // at most 2n - 4 faces: one CTA sorts them
        launch_small_face_sort(p->k0, p->v0, fbits, nf, d_faces, st);
        launches++;
        STEP("small face sort");
    } else {
        which = radix_sort_pairs(p->k0, p->v0, p->k1, p->v1, 2 * n, nf, 2 * fbits, p->ss, st, &launches);
        STEP("face sort");
        launch_face_out(which ? p->k1 : p->k0, which ? p->v1 : p->v0, 2 * n, fbits, nf, d_faces, st);
        launches++;
        STEP("face out");
    }
    MARK(5);
    if (p->profile) p->marks.insert(p->marks.end(), slots, slots + HULL3D_PHASES + 1);
    p->last_launches = launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    return HULL3D_OK;
}

// Largest cloud the multi-cloud path takes (face keys need the cloud index
// and two vertex indices in 64 bits).
constexpr int64_t MULTI_MAX_CLOUD = 1ll << 24;

int64_t pow2_ceil(int64_t x)
{
    int64_t b = 1;
    while (b < x) b <<= 1;
    return b;
}

// Enqueues the hulls of the clouds group[0 .. C) (batch indices, decreasing
// size, each of more than 4096 points, their aligned blocks fitting the
// plan's max_n ranks) together: one sort, one launch sequence per merge
// level for all of them, one face sort.
int enqueue_multi(hull3d_plan_s *p, const int32_t *d_xyz, const int64_t *h_offsets, const int64_t *h_face_offsets,
                  const std::vector<int32_t> &group, int32_t *d_faces, int64_t *d_nfaces, int32_t *d_status,
                  cudaStream_t st, int64_t *launches)
{
    const int C = (int)group.size();
    std::vector<int64_t> cbase(C), cend(C), coff(C + 1), ioff(C), cfoff(C);
    std::vector<int32_t> ctop(C), corig(C);
    int64_t R = 0, total = 0, nmax = 0;
    int L = 0;
    for (int c = 0; c < C; c++) {
        const int32_t b = group[c];
        const int64_t nb = h_offsets[b + 1] - h_offsets[b];
        const int64_t blk = pow2_ceil(nb);  // blocks by decreasing size: each starts at a multiple of its size
        cbase[c] = R;
        cend[c] = R + nb;
        coff[c] = total;
        ioff[c] = h_offsets[b];
        cfoff[c] = h_face_offsets[b];
        ctop[c] = ceil_log2(nb);
        corig[c] = b;
        R += blk;
        total += nb;
        nmax = std::max(nmax, nb);
        L = std::max(L, ctop[c]);
    }
    coff[C] = total;
    std::vector<int32_t> blkmap((size_t)(R >> SPAN_SHIFT), -1);
    for (int c = 0; c < C; c++)
        for (int64_t r = cbase[c]; r < cbase[c] + pow2_ceil(cend[c] - cbase[c]); r += 1ll << SPAN_SHIFT)
            blkmap[(size_t)(r >> SPAN_SHIFT)] = c;
    MultiTables t = p->mt;
    t.ncl = C;
    CK(cudaMemcpyAsync(t.blk, blkmap.data(), sizeof(int32_t) * blkmap.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(t.cbase, cbase.data(), sizeof(int64_t) * C, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(t.cend, cend.data(), sizeof(int64_t) * C, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(t.coff, coff.data(), sizeof(int64_t) * (C + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(t.ioff, ioff.data(), sizeof(int64_t) * C, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(t.cfoff, cfoff.data(), sizeof(int64_t) * C, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(t.ctop, ctop.data(), sizeof(int32_t) * C, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(t.corig, corig.data(), sizeof(int32_t) * C, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(t.cstat, 0, sizeof(int32_t) * C, st));
    CK(cudaMemsetAsync(p->status, 0, sizeof(int32_t), st));
    CK(cudaMemsetAsync(p->lev_stats, 0, 128 * sizeof(unsigned long long), st));
    launch_multi_sort(d_xyz, t, C, total, p->P4, p->k0, p->v0, p->k1, p->v1, p->ss, p->sms, st, launches);
    const Points pts{ p->P4 };
    const Span sp{ R, t.blk, t.cbase, t.cend, t.ctop, t.cstat };
    // levels are timed when profiling; the per-call phase record belongs to single hulls
    int slots[HULL3D_PHASES + 1];
    bool seg_marked = false;
    int rc = enqueue_levels(p, pts, sp, C, L, 1, p->status, st, launches, slots, &seg_marked);
    if (rc) return rc;
    const int fbits = ceil_log2(nmax);
    launch_multi_faces(pts, t, C, fbits, p->pass, p->k0, p->v0, p->k1, p->v1, 2 * p->max_n, p->ss, p->status,
                       d_faces, d_nfaces, d_status, p->sms, st, launches);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HULL3D_OK : cuda_fail(e);
}

// Enqueues the Delaunay triangulation of n 2D points through the lifting
// map: lifted keys, the sort, every merge level (the lower pass gives the
// triangles), the triangles' canonical sort.
int enqueue_delaunay(hull3d_plan_s *p, const int32_t *d_xy, int64_t n, int32_t *d_tris, int64_t *nt, int32_t *status,
                     cudaStream_t st)
{
    int64_t launches = 0;
    CK(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
    CK(cudaMemsetAsync(nt, 0, sizeof(int64_t), st));
    CK(cudaMemsetAsync(p->lev_stats, 0, 128 * sizeof(unsigned long long), st));
    launch_keys_lifted(d_xy, n, p->k0, p->v0, status, st);
    int which = radix_sort_pairs(p->k0, p->v0, p->k1, p->v1, n, nullptr, 63, p->ss, st, &launches);
    launch_decode_lifted(which ? p->k1 : p->k0, which ? p->v1 : p->v0, n, p->P4, status, st);
    launches += 2;
    if (n >= 3) {
        const Points pts{ p->P4 };
        const int L = ceil_log2(n);
        // levels are timed when profiling; the per-call phase record belongs to hulls
        int slots[HULL3D_PHASES + 1];
        bool seg_marked = false;
        int rc = enqueue_levels(p, pts, single_span(n), 1, L, 1, status, st, &launches, slots, &seg_marked, true);
        if (rc) return rc;
        int fbits = ceil_log2(n);
        if (fbits < 1) fbits = 1;
        launch_tri_keys(pts, n, L, p->pass, p->k0, p->v0, p->items, nt, status, st);
        which = radix_sort_pairs(p->k0, p->v0, p->k1, p->v1, 2 * n, p->items, 2 * fbits, p->ss, st, &launches);
        launch_face_out(which ? p->k1 : p->k0, which ? p->v1 : p->v0, 2 * n, fbits, nt, d_tris, st);
        launches += 2;
    }
    p->last_launches = launches;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HULL3D_OK : cuda_fail(e);
}

bool use_graphs(const hull3d_plan_s *p) { return p->opts.use_graph >= 0 && !p->profile && !debug_sync(); }

// Enqueues the pipeline as a replay of a cached CUDA graph (captured on the
// plan's private stream on first use of these arguments).
int enqueue_hull_graph(hull3d_plan_s *p, const int32_t *d_xyz, int64_t n, int32_t *d_faces, int64_t *nf,
                       int32_t *status, cudaStream_t st)
{
    hull3d_plan_s::GraphEntry *hit = nullptr, *victim = &p->graphs[0];
    for (auto &g : p->graphs) {
        if (g.exec && g.xyz == d_xyz && g.n == n && g.faces == d_faces && g.nf == nf && g.status == status) hit = &g;
        if (!g.exec || g.used < victim->used) victim = &g;
    }
    if (!hit) {
        if (!p->cap_stream) CK(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_hull(p, d_xyz, n, d_faces, nf, status, p->cap_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(p->cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e);
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e);
        if (victim->exec) cudaGraphExecDestroy(victim->exec);
        *victim = hull3d_plan_s::GraphEntry{ d_xyz, n, d_faces, nf, status, exec, p->last_launches, 0 };
        hit = victim;
    }
    hit->used = ++p->graph_clock;
    CK(cudaGraphLaunch(hit->exec, st));
    p->last_launches = hit->launches;
    return HULL3D_OK;
}

int check_compute_args(hull3d_plan_s *p, const void *xyz, int64_t n, const void *faces, int64_t cap)
{
    if (!p || !xyz || n < 1 || n > p->max_n) return HULL3D_ERR_INVALID_ARG;
    if (n >= 3) {
        if (!faces) return HULL3D_ERR_INVALID_ARG;
        if (cap < 2 * n - 4) return HULL3D_ERR_CAPACITY;
    }
    return HULL3D_OK;
}

}  // namespace

extern "C" {

int hull3d_plan(hull3d_plan_t *out, int64_t max_n, int64_t max_clouds, const hull3d_opts *opts)
{
    if (!out) return HULL3D_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_n < 1 || max_n > HULL3D_MAX_N || max_clouds < 0) return HULL3D_ERR_INVALID_ARG;
    hull3d_plan_s *p = new (std::nothrow) hull3d_plan_s();
    if (!p) return HULL3D_ERR_OOM;
    p->max_n = max_n < 4 ? 4 : max_n;
    p->max_clouds = max_clouds;
    if (opts) p->opts = *opts;
    if (p->opts.float32_ablation < 0 || p->opts.float32_ablation > 1 || p->opts.fused_levels < 0 ||
        p->opts.fused_levels > 10 || p->opts.cmp_slots < 0 || p->opts.cmp_slots > 4096 || p->opts.seg_slots_big < 0 ||
        p->opts.seg_slots_big > 6144 || p->opts.filter_level < 0 ||
        p->opts.seg_slots < 0 || p->opts.seg_slots > 6144 || p->opts.seg_events < 0 || p->opts.seg_events > 4096 ||
        p->opts.seg_events_min < 0) {
        delete p;
        return HULL3D_ERR_INVALID_ARG;
    }
    cudaGetDevice(&p->device);
    kernel_attributes();
    cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
    {
        AdjScratch as{};
        p->pool_bytes = std::max(layout(p, nullptr), adj_layout(p, nullptr, &as));
    }
    cudaError_t e = cudaMalloc((void **)&p->pool, p->pool_bytes);
    if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        cudaGetLastError();
        delete p;
        return e == cudaErrorMemoryAllocation ? HULL3D_ERR_OOM : HULL3D_ERR_CUDA;
    }
    layout(p, p->pool);
    e = cudaMallocHost((void **)&p->h_nfaces, 64);
    if (e != cudaSuccess) {
        cudaFree(p->pool);
        delete p;
        return cuda_fail(e);
    }
    p->h_status = (int32_t *)(p->h_nfaces + 2);
    *out = p;
    return HULL3D_OK;
}

void hull3d_destroy(hull3d_plan_t p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    for (auto &g : p->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    cudaFree(p->pool);
    cudaFreeHost(p->h_nfaces);
    delete p;
}

int64_t hull3d_plan_bytes(hull3d_plan_t p) { return p ? (int64_t)p->pool_bytes : 0; }

int hull3d_plan_opts(hull3d_plan_t p, hull3d_opts *out)
{
    if (!p || !out) return HULL3D_ERR_INVALID_ARG;
    *out = p->opts;
    out->fused_levels = default_fused(p);
    out->level_occupancy = p->opts.level_occupancy;
    out->cmp_level = default_cmp_level(p, ceil_log2(p->max_n));
    out->cmp_slots = default_cmp_slots(p);
    out->seg_level = default_seg_level(p);
    out->seg_events = default_seg_events(p);
    out->seg_events_min = default_seg_events_min(p);
    out->seg_slots = default_seg_slots(p);
    out->seg_slots_big = default_seg_slots_big(p);
    out->filter_level = default_filter_level(p, ceil_log2(p->max_n), false);
    out->seg_min_events = default_seg_min_events(p);
    out->merge_order = p->opts.merge_order < 0 ? -1 : 1;
    out->batch_warp_nodes = default_batch_warp_nodes(p);
    out->multi_ranks = (int32_t)std::min<int64_t>(default_multi_ranks(p), INT32_MAX);
    return HULL3D_OK;
}

int64_t hull3d_last_launch_count(hull3d_plan_t p) { return p ? p->last_launches : 0; }

int hull3d_compute_async(hull3d_plan_t p, const int32_t *d_xyz, int64_t n, int32_t *d_faces, int64_t cap_faces,
                         int64_t *d_nfaces, int32_t *d_status, void *stream)
{
    int rc = check_compute_args(p, d_xyz, n, d_faces, cap_faces);
    if (rc) return rc;
    int64_t *nf = d_nfaces ? d_nfaces : p->nfaces;
    int32_t *status = d_status ? d_status : p->status;
    if (use_graphs(p)) return enqueue_hull_graph(p, d_xyz, n, d_faces, nf, status, (cudaStream_t)stream);
    return enqueue_hull(p, d_xyz, n, d_faces, nf, status, (cudaStream_t)stream);
}

int hull3d_compute(hull3d_plan_t p, const int32_t *d_xyz, int64_t n, int32_t *d_faces, int64_t cap_faces,
                   int64_t *h_nfaces, void *stream)
{
    int rc = check_compute_args(p, d_xyz, n, d_faces, cap_faces);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = use_graphs(p) ? enqueue_hull_graph(p, d_xyz, n, d_faces, p->nfaces, p->status, st)
                       : enqueue_hull(p, d_xyz, n, d_faces, p->nfaces, p->status, st);
    if (rc) return rc;
    CK(cudaMemcpyAsync(p->h_nfaces, p->nfaces, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(p->h_status, p->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_nfaces) *h_nfaces = *p->h_status ? 0 : *p->h_nfaces;
    return *p->h_status;
}

int hull3d_compute_host(hull3d_plan_t p, const int32_t *h_xyz, int64_t n, int32_t *h_faces, int64_t cap_faces,
                        int64_t *h_nfaces, void *stream)
{
    int rc = check_compute_args(p, h_xyz, n, h_faces, cap_faces);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(p->stage_xyz, h_xyz, (size_t)n * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    rc = use_graphs(p) ? enqueue_hull_graph(p, p->stage_xyz, n, p->stage_faces, p->nfaces, p->status, st)
                       : enqueue_hull(p, p->stage_xyz, n, p->stage_faces, p->nfaces, p->status, st);
    if (rc) return rc;
    CK(cudaMemcpyAsync(p->h_nfaces, p->nfaces, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(p->h_status, p->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int status = *p->h_status;
    int64_t nf = status ? 0 : *p->h_nfaces;
    if (nf > 0) {
        CK(cudaMemcpyAsync(h_faces, p->stage_faces, (size_t)nf * 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    if (h_nfaces) *h_nfaces = nf;
    return status;
}

int hull3d_batch_async(hull3d_plan_t p, const int32_t *d_xyz, const int64_t *h_offsets, int64_t B, int32_t *d_faces,
                       const int64_t *h_face_offsets, int64_t *d_nfaces, int32_t *d_status, void *stream)
{
    if (!p || !h_offsets || !h_face_offsets || B < 0 || (B > 0 && (!d_xyz || !d_faces || !d_nfaces || !d_status)))
        return HULL3D_ERR_INVALID_ARG;
    if (B > p->max_clouds) return HULL3D_ERR_INVALID_ARG;
    if (h_offsets[0] != 0 || h_face_offsets[0] != 0) return HULL3D_ERR_INVALID_ARG;
    const int small_max = batch_class_limit(BATCH_CLASSES - 1);
    for (int64_t b = 0; b < B; b++) {
        int64_t nb = h_offsets[b + 1] - h_offsets[b];
        int64_t cap = h_face_offsets[b + 1] - h_face_offsets[b];
        if (nb < 1 || cap < 0) return HULL3D_ERR_INVALID_ARG;
        if (nb > small_max && nb > p->max_n) return HULL3D_ERR_INVALID_ARG;
        if (nb >= 3 && cap < 2 * nb - 4) return HULL3D_ERR_CAPACITY;
    }
    if (B == 0) return HULL3D_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // size classes, largest clouds first inside each class
    std::vector<int32_t> &ord = p->h_order;
    ord.resize((size_t)B);
    int64_t cls_begin[BATCH_CLASSES + 1] = {};
    {
        std::vector<int32_t> idx((size_t)B);
        for (int64_t b = 0; b < B; b++) idx[b] = (int32_t)b;
        auto size = [&](int32_t b) { return h_offsets[b + 1] - h_offsets[b]; };
        std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t c) { return size(a) > size(c); });
        // idx is by decreasing size: big clouds, then class 2, 1, 0
        int64_t pos = 0;
        for (int c = BATCH_CLASSES; c >= 0; c--) {
            const int64_t lo_lim = c == 0 ? 0 : batch_class_limit(c - 1);
            const int64_t hi_lim = c == BATCH_CLASSES ? INT64_MAX : batch_class_limit(c);
            cls_begin[c] = pos;
            for (int32_t b : idx) {
                int64_t nb = size(b);
                if (nb > lo_lim && nb <= hi_lim) ord[pos++] = b;
            }
        }
    }
    CK(cudaMemcpyAsync(p->b_off, h_offsets, sizeof(int64_t) * (size_t)(B + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(p->b_foff, h_face_offsets, sizeof(int64_t) * (size_t)(B + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(p->b_order, ord.data(), sizeof(int32_t) * (size_t)B, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(p->b_counter, 0, sizeof(int) * BATCH_CLASSES, st));
    int64_t launches = 0;
    for (int c = 0; c < BATCH_CLASSES; c++) {
        // classes were laid out big, 2, 1, 0: class c starts at cls_begin[c]
        const int64_t begin = cls_begin[c];
        const int64_t end = c == 0 ? B : cls_begin[c - 1];
        const int count = (int)(end - begin);
        if (count <= 0) continue;
        launch_batch_class(c, d_xyz, p->b_off, p->b_foff, p->b_order + begin, count, p->b_counter + c, d_faces,
                           d_nfaces, d_status, p->sms, default_batch_warp_nodes(p), p->opts.float32_ablation == 1, st);
        launches++;
    }
    // clouds above the largest class (ord holds them by decreasing size):
    // hulled together, level by level, in groups whose aligned blocks fill
    // the plan's max_n ranks; a cloud whose block alone does not fit runs
    // the single-hull pipeline
    {
        std::vector<int32_t> group;
        int64_t used = 0;
        auto flush = [&]() -> int {
            if (group.empty()) return HULL3D_OK;
            int rc = enqueue_multi(p, d_xyz, h_offsets, h_face_offsets, group, d_faces, d_nfaces, d_status, st,
                                   &launches);
            group.clear();
            used = 0;
            return rc;
        };
        for (int64_t q = cls_begin[BATCH_CLASSES]; q < cls_begin[BATCH_CLASSES - 1]; q++) {
            const int32_t b = ord[q];
            const int64_t nb = h_offsets[b + 1] - h_offsets[b];
            const int64_t blk = pow2_ceil(nb);
            if (blk > p->max_n || nb > MULTI_MAX_CLOUD) {
                int rc = enqueue_hull(p, d_xyz + 3 * h_offsets[b], nb, d_faces + 3 * h_face_offsets[b], d_nfaces + b,
                                      d_status + b, st);
                if (rc) return rc;
                launches += p->last_launches;
                continue;
            }
            if (used + blk > default_multi_ranks(p) || (int64_t)group.size() + 1 > p->mt_cap) {
                int rc = flush();
                if (rc) return rc;
            }
            group.push_back(b);
            used += blk;
        }
        int rc = flush();
        if (rc) return rc;
    }
    p->last_launches = launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    return HULL3D_OK;
}

int hull3d_delaunay_async(hull3d_plan_t p, const int32_t *d_xy, int64_t n, int32_t *d_tris, int64_t cap_tris,
                          int64_t *d_ntris, int32_t *d_status, void *stream)
{
    if (!p || !d_xy || n < 1 || n > p->max_n) return HULL3D_ERR_INVALID_ARG;
    if (n >= 3) {
        if (!d_tris) return HULL3D_ERR_INVALID_ARG;
        if (cap_tris < 2 * n - 4) return HULL3D_ERR_CAPACITY;
    }
    return enqueue_delaunay(p, d_xy, n, d_tris, d_ntris ? d_ntris : p->nfaces, d_status ? d_status : p->status,
                            (cudaStream_t)stream);
}

int hull3d_adjacency_async(hull3d_plan_t p, const int32_t *d_faces, const int64_t *d_nfaces, int64_t cap_faces,
                           int64_t n, int32_t *d_nb, int64_t *d_star_off, int32_t *d_star, int32_t *d_status,
                           void *stream)
{
    if (!p || !d_nfaces || !d_star_off || !d_status || n < 1 || n > p->max_n || cap_faces < 0 ||
        cap_faces > 2 * p->max_n)
        return HULL3D_ERR_INVALID_ARG;
    if (cap_faces > 0 && (!d_faces || !d_nb || !d_star)) return HULL3D_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemsetAsync(d_status, 0, sizeof(int32_t), st));
    if (cap_faces == 0) {  // no faces: every star is empty
        CK(cudaMemsetAsync(d_star_off, 0, sizeof(int64_t) * (size_t)(n + 1), st));
        p->last_launches = 0;
        return HULL3D_OK;
    }
    AdjScratch as{};
    adj_layout(p, p->pool, &as);
    int64_t launches = 0;
    launch_adjacency(d_faces, d_nfaces, cap_faces, n, d_nb, d_star_off, d_star, d_status, as, p->sms, st, &launches);
    p->last_launches = launches;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HULL3D_OK : cuda_fail(e);
}

int hull3d_profile(hull3d_plan_t p, int enable)
{
    if (!p) return HULL3D_ERR_INVALID_ARG;
    p->profile = enable != 0;
    p->marks.clear();
    p->level_marks.clear();
    p->ev_used = 0;
    return HULL3D_OK;
}

int hull3d_profile_levels(hull3d_plan_t p, double *ms)
{
    if (!p || !ms) return HULL3D_ERR_INVALID_ARG;
    for (int k = 0; k < 64; k++) ms[k] = 0.0;
    if (!p->level_marks.empty()) CK(cudaEventSynchronize(p->ev_pool[p->level_marks.back()]));
    for (size_t i = 0; i + 3 <= p->level_marks.size(); i += 3) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, p->ev_pool[p->level_marks[i + 1]], p->ev_pool[p->level_marks[i + 2]]));
        ms[p->level_marks[i] & 63] += t;
    }
    return HULL3D_OK;
}

int hull3d_profile_read(hull3d_plan_t p, double *ms, int64_t *calls)
{
    if (!p || !ms) return HULL3D_ERR_INVALID_ARG;
    for (int k = 0; k < HULL3D_PHASES; k++) ms[k] = 0.0;
    const int per = HULL3D_PHASES + 1;
    int64_t nc = (int64_t)(p->marks.size() / per);
    if (nc > 0) CK(cudaEventSynchronize(p->ev_pool[p->marks.back()]));
    for (int64_t c = 0; c < nc; c++)
        for (int k = 0; k < HULL3D_PHASES; k++) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, p->ev_pool[p->marks[c * per + k]], p->ev_pool[p->marks[c * per + k + 1]]));
            ms[k] += t;
        }
    if (calls) *calls = nc;
    p->marks.clear();
    p->level_marks.clear();
    p->ev_used = 0;
    return HULL3D_OK;
}

int hull3d_level_events(hull3d_plan_t p, int64_t *out)
{
    if (!p || !out) return HULL3D_ERR_INVALID_ARG;
    unsigned long long tmp[128];
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(tmp, p->lev_stats, sizeof tmp, cudaMemcpyDeviceToHost));
    for (int k = 0; k < 128; k++) out[k] = (int64_t)tmp[k];
    return HULL3D_OK;
}

int hull3d_window_stats(hull3d_plan_t p, int64_t *out)
{
    if (!p || !out) return HULL3D_ERR_INVALID_ARG;
    for (int k = 0; k < HULL3D_WINDOW_STATS * 64; k++) out[k] = 0;
    if (!p->overflow) return HULL3D_OK;
    std::vector<int> tmp(SEG_STAT_STRIDE * 64);
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(tmp.data(), p->overflow, sizeof(int) * tmp.size(), cudaMemcpyDeviceToHost));
    for (int l = 0; l < 64; l++)
        for (int k = 0; k < HULL3D_WINDOW_STATS; k++) out[l * HULL3D_WINDOW_STATS + k] = tmp[l * SEG_STAT_STRIDE + k];
    return HULL3D_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entry point: the pipeline's scratch lives in one static
// device array (held by every GPU that loads the library until exit).
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_static_scratch[HULL3D_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
hull3d_plan_s g_static_plan[kMaxDevices];
bool g_static_ready[kMaxDevices] = {};

// Once per device, with that device current: look up the array's device
// address (in host code its name is only a host-side stand-in) and lay the
// plan's buffers out in it.
int static_plan_for_current_device(hull3d_plan_s **out)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return HULL3D_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_static_mu);
    hull3d_plan_s *p = &g_static_plan[dev];
    if (!g_static_ready[dev]) {
        kernel_attributes();  // this path may be the process's first use of the device
        void *base = nullptr;
        CK(cudaGetSymbolAddress(&base, g_static_scratch));
        p->max_n = HULL3D_STATIC_MAX_N;
        p->max_clouds = 0;
        p->device = dev;
        p->opts.seg_level = 64;  // n <= 2^14: no time-segment-parallel levels, no window scratch
        if (layout(p, nullptr) > (size_t)HULL3D_STATIC_SCRATCH_BYTES) return HULL3D_ERR_INTERNAL;
        p->pool = (char *)base;
        p->pool_bytes = layout(p, p->pool);
        g_static_ready[dev] = true;
    }
    *out = p;
    return HULL3D_OK;
}

}  // namespace

extern "C" {

int hull3d_compute_static(const int32_t *d_xyz, int64_t n, int32_t *d_faces, int64_t cap_faces, int64_t *d_nfaces,
                          int32_t *d_status, void *stream)
{
    if (!d_xyz || !d_nfaces || !d_status || n < 1) return HULL3D_ERR_INVALID_ARG;
    if (n > HULL3D_STATIC_MAX_N) return HULL3D_ERR_TOO_LARGE;
    if (n >= 3 && (!d_faces)) return HULL3D_ERR_INVALID_ARG;
    if (n >= 3 && cap_faces < 2 * n - 4) return HULL3D_ERR_CAPACITY;
    hull3d_plan_s *p = nullptr;
    int rc = static_plan_for_current_device(&p);
    if (rc) return rc;
    return enqueue_hull(p, d_xyz, n, d_faces, d_nfaces, d_status, (cudaStream_t)stream);
}

const char *hull3d_strerror(int code)
{
    switch (code) {
    case HULL3D_OK: return "ok";
    case HULL3D_ERR_INVALID_ARG: return "invalid argument";
    case HULL3D_ERR_COORD_RANGE: return "coordinate outside [-2^20, 2^20)";
    case HULL3D_ERR_DUPLICATE: return "duplicate point";
    case HULL3D_ERR_CAPACITY: return "output capacity below 2n - 4 faces";
    case HULL3D_ERR_OOM: return "device allocation failed";
    case HULL3D_ERR_BUDGET: return "request above the memory budget";
    case HULL3D_ERR_DEVICE_TIMEOUT: return "a bounded device wait ran out";
    case HULL3D_ERR_CUDA: return "CUDA runtime error";
    case HULL3D_ERR_INTERNAL: return "internal consistency check failed";
    case HULL3D_ERR_TOO_LARGE: return "n above HULL3D_STATIC_MAX_N for the allocation-free entry point";
    case HULL3D_ERR_NOT_CLOSED: return "faces are not a closed, consistently oriented surface";
    default: return "unknown error";
    }
}

int hull3d_last_cuda_error(void) { return g_last_cuda; }

}  // extern "C"
