// segmerge.cuh -- time-segment-parallel merge for the top levels.
//
// At the top of the bottom-up movie construction (White & Wortman, Sec. 2)
// there are too few merges to fill the GPU, and a merge's event loop is
// serial in time.  Here the parent's time line is cut into windows holding
// about K child events each (a merge-path split of the two child movies by
// event time), and every window is merged independently:
//   bounds  window s starts after kL_s left and kR_s right child events;
//   pairs   a child event point is on its child's hull over one interval of
//           that child's event indices, [first event, last event) (the
//           invariant the kinetic movie guarantees), so it belongs to the
//           start hull of every window whose start index falls in it; the
//           (window, child, rank) triples are emitted and radix-sorted, which
//           gives every window both start hulls in x-order;
//   merge   one warp per window: a slot table holds the start hulls (linked
//           in x-order) and the points the window inserts (linked through
//           their stored event-time neighbours); the start bridge is found
//           by walking in from the inner x-extremes with orientations taken
//           just after the window's first instant; then the same six-
//           candidate event loop runs until the window's child events are
//           consumed (the last window runs to t = +infinity);
//   concat  the window outputs are concatenated in order; the parent's links
//           for the next level are written in parallel: every insert event
//           (a, w, b) gives w the links (a, b), and the t = -infinity bridge
//           (u0, v0) joins the two children's t = -infinity hulls.
// A window too large for the shared-memory slot tables gets a table in global
// memory; a merge with a window that fits no table is merged serially.
//
// The phases are written as functions of (thread, thread count) so that the
// kernels call them between barriers.
#pragma once
#include "merge.cuh"

namespace hull3d {

// Per-pass scratch of one segment level.
struct SegBufs {
    int2 *bound;            // [S_cap]: child events before window g = (kL, kR)
    int *nseg;              // [M_cap]: windows of merge m
    int *ins_idx, *del_idx;  // [n]: index of a point's insert / delete event in its child movie
    int *smap;              // [n]: slot of a point inserted inside a window
    unsigned *oW;           // window outputs, at seg_out_base (see there)
    int *oA, *oB;
    int *ocnt;              // [S_cap]
    int2 *bridge0;          // [M_cap]: t = -inf bridge (u0, v0) as ranks
    int *nofit;             // [M_cap]: 1 when a window did not fit (merge serially)
    unsigned *wlist, *flist, *mlist;  // work lists (pass 0's copy holds both passes): [2 S_cap], [2 S_cap], [2 M_cap]
    unsigned *glist;                  // [2 S_cap]: windows for the global-memory slot tables
    unsigned *flist2;                 // [2 S_cap]: windows for the largest shared-memory table
};

// Geometry of one segment level (shared by both passes).
struct SegGeom {
    int64_t n;
    int level;     // parent level
    int K;         // longest time window, in child events
    int Kmin;      // shortest time window
    int smax;      // windows per merge reserved in the scratch (for Kmin)
    int scap;      // slot table capacity
    int64_t pair_cap;
    int min_events;  // merges with at most this many child events are not merged here
};

// Slots of the middle retry round's shared-memory table (two per SM), when
// the largest one is at least this large.
constexpr int SEG_SLOTS_MID = 3072;

// Child events a window of the retry rounds (the larger shared-memory tables and
// the global-memory tables) holds; the first round holds the level's longest
// window K.
constexpr int SEG_EVCAP_BIG = 4096;

// Per merge level, the window counters (HULL3D_WINDOW_STATS of them; a block
// of SEG_STAT_STRIDE ints per level): pair overflow, merges in windows,
// windows, windows to retry, windows for the global tables, merges run
// serially, the refit multiplier.
constexpr int SEG_STAT_STRIDE = 8;

// Window length of a merge with E child events: 2 sqrt(E) within [Kmin, K].
// A time window starts from the two child hulls at its first instant (their
// points become start-hull entries), so its setup grows with the hull size
// while its serial event chain grows with its length; the child hulls of the
// workloads hold at most ~0.8 sqrt(m) points (points on a sphere; m child
// points, about E child events), so windows of 2 sqrt(E) events keep both in
// proportion and the start-hull entries of a merge below its event count.
// Small hulls (a cube's, a ball's) take the shortest windows.  (Measured
// against sqrt(E) / 2 and sqrt(E): the same on the cube, ball and Gaussian,
// 3% faster on the 2^20 sphere.)
__host__ __device__ __forceinline__ int seg_window_len(int E, int K, int Kmin)
{
    const int r = (int)(2.0f * sqrtf((float)E));  // the same value in every thread of a merge
    return r < Kmin ? Kmin : (r > K ? K : r);
}

// First output entry of window s of merge m whose first event is the j-th of
// the merge's child events: merge m owns 2 E + 256 S entries from
// 4 lo + 256 m smax on (E <= 2 (hi - lo) child events in S <= smax windows), and
// window s holds at most 2 w + 256 events (w = its child events).
__host__ __device__ __forceinline__ int64_t seg_out_base(int level, int smax, int64_t m, int s, int j)
{
    return 4 * (m << level) + 256 * (m * smax + s) + 2 * (int64_t)j;
}

__host__ __device__ __forceinline__ int seg_count(int nl, int nr, int K, int smax)
{
    int s = (nl + nr + K - 1) / K;
    if (s < 1) s = 1;
    return s < smax ? s : smax;
}

// Key of a start-hull entry: pass, window, child, rank (sorted ascending);
// the rank takes the low rbits bits (ranks of the rank space are below 2^rbits).
__host__ __device__ __forceinline__ uint64_t seg_key(int pass, int64_t g, int child, int rank, int64_t S_cap, int rbits)
{
    return ((((uint64_t)pass * (uint64_t)S_cap + (uint64_t)g) * 2u + (uint64_t)child) << rbits) | (uint64_t)rank;
}

// The time of child event k of a movie (its triple, in ranks).
__device__ __forceinline__ void ev_tri(const GPts &gp, const unsigned *W, const int *A, const int *B, int k, Tri &t)
{
    tri_make(gp, t, A[k], (int)(W[k] & RANK_MASK), B[k]);
}

// Number of left-child events among the first j events of the merged order
// (merge path: binary search on exact event times).
__device__ __forceinline__ int merge_path(const GPts &gp, const unsigned *LW, const int *LA, const int *LB, int nl,
                                          const unsigned *RW, const int *RA, const int *RB, int nr, int j,
                                          bool upper)
{
    int lo = j - nr > 0 ? j - nr : 0, hi = j < nl ? j : nl;
    while (lo < hi) {
        int m = (lo + hi) >> 1;
        Tri a, b;
        ev_tri(gp, LW, LA, LB, m, a);
        ev_tri(gp, RW, RA, RB, j - 1 - m, b);
        if (tri_cmp(gp, a, b, upper) < 0) lo = m + 1;
        else hi = m;
    }
    return lo;
}

}  // namespace hull3d
