// internal.h -- launchers shared between the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hull3d.h"
#include "span.cuh"

namespace hull3d {

// Scratch for the LSD radix sort of (uint64 key, uint32 value) pairs.
struct SortScratch {
    uint32_t *hist;     // 256 x max_tiles
    uint32_t *rowsum;   // 256
    int64_t max_tiles;
};

constexpr int SORT_TILE = 4096;  // keys per CTA tile (256 threads x 16)

// Sorts keys/vals (n items, or *d_n items when d_n != NULL, n being the
// capacity) by bits [0, bits) of the key.  Ping-pongs between (k0, v0) and
// (k1, v1); returns 0 if the result ends in (k0, v0) and 1 otherwise.
int radix_sort_pairs(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t n, const int64_t *d_n,
                     int bits, const SortScratch &s, cudaStream_t st, int64_t *launches, int lo_bit = 0);
// Sorts each run of point keys with one x-value (bits 42-62) by the whole
// key, from (kin, vin) into (kout, vout): one thread per key of a run of at
// most max_run keys, one CTA per longer run (up to TIE_SORT_LONG_CAP runs of
// up to TIE_SORT_LONG_MAX keys); beyond that it stores n in *runs.fallback_n
// and leaves such runs out (the caller then sorts every key of kin in full).
// runs.fallback_n and runs.count start at zero (two launches).
constexpr int TIE_SORT_LONG_MAX = 4096;
constexpr int TIE_SORT_LONG_CAP = 256;
struct TieRuns {
    int64_t *fallback_n;
    int *count;
    int64_t *start;  // [TIE_SORT_LONG_CAP]
    int *len;        // [TIE_SORT_LONG_CAP]
};
void launch_tie_sort(const uint64_t *kin, const uint32_t *vin, uint64_t *kout, uint32_t *vout, int64_t n, int max_run,
                     const TieRuns &runs, cudaStream_t st);
// launch_decode from (keys_b, vals_b) instead where *use_b is nonzero.
void launch_decode_either(const uint64_t *keys, const uint32_t *vals, const uint64_t *keys_b, const uint32_t *vals_b,
                          const int64_t *use_b, int64_t n, int4 *P, int32_t *status, cudaStream_t st);

// A1 + A2 for n <= SMALL_SORT_MAX in one CTA (keys, bitonic sort in shared
// memory, decode, duplicates), and the canonical sort of such a hull's faces
// (keys and values as for launch_face_out; *d_nf <= 2 SMALL_SORT_MAX).
constexpr int SMALL_SORT_MAX = 4096;
// Longest run of points on one x-value the point sort orders in place after
// its x passes (larger runs: the full sort).
constexpr int TIE_SORT_MAX_RUN = 128;
constexpr int SMALL_SORT_THREADS = 1024;
void launch_small_sort(const int32_t *xyz, int64_t n, int4 *P, int32_t *status, cudaStream_t st);
void launch_small_face_sort(const uint64_t *keys, const uint32_t *vals, int fbits, const int64_t *d_nf,
                            int32_t *faces, cudaStream_t st);

// A1: range check and key build: key = (x + 2^20) << 42 | (z + 2^20) << 21 | (y + 2^20).
void launch_keys(const int32_t *xyz, int64_t n, uint64_t *keys, uint32_t *vals, int32_t *status, cudaStream_t st);

// After the sort: decode the sorted keys to rank-ordered points (x, y, z, input
// index) and flag duplicates.
void launch_decode(const uint64_t *keys, const uint32_t *vals, int64_t n, int4 *P, int32_t *status, cudaStream_t st);

// The same for 2D points (n x 2 int32, |x|, |y| < 2^15) lifted to
// (x, y, x^2 + y^2): key (x + 2^15) << 47 | z << 16 | (y + 2^15).
void launch_keys_lifted(const int32_t *xy, int64_t n, uint64_t *keys, uint32_t *vals, int32_t *status,
                        cudaStream_t st);
void launch_decode_lifted(const uint64_t *keys, const uint32_t *vals, int64_t n, int4 *P, int32_t *status,
                          cudaStream_t st);

// Event-list storage of one pass: two ping-pong buffers (W with the insert flag, A, B) and counts by node lo.
struct PassBufs {
    unsigned *W[2];
    int32_t *A[2], *B[2];
    int32_t *cnt[2];
    int2 *lk;                        // [n]: (prev, next) ranks, NIL = -1
    unsigned long long *lev_events;  // [64]: events written per level (statistics)
    int32_t *gmap;                   // [n]: rank -> slot scratch of the compacted merge
};

struct Points {
    const int4 *P;  // [n]: (x, y, z, input index) by rank
};

// Levels 1 and 2 for both passes: the pairs' links, then each node of four
// ranks merges its two pairs (movies in buffer 0; event neighbours kept from
// level ab_level on and for the last node).
void launch_level2(const Points &pts, const Span &sp, PassBufs *passes, int ab_level, int32_t *status, cudaStream_t st);

// Levels [l0 + 1, l1] fused in shared memory (block = 2^l1 ranks), reading level l0 from buffer l0 & 1.
void launch_fused(const Points &pts, int64_t n, int l0, int l1, PassBufs *passes, int npass, int32_t *status,
                  cudaStream_t st);

// Scratch for sorting a level's merges by their work (the point-sort buffers,
// free while the levels run).
struct LevelOrder {
    uint64_t *k0, *k1;
    uint32_t *v0, *v1;
    SortScratch ss;
    bool typed;  // group the merges by how their points share x-values first (k_order_keys)
};

// One level (>= 2), one thread per merge, global memory.  With max_events >= 0
// only merges of at most max_events child events are done (see launch_level_cmp).
// With ord, the merges of both passes run in order of decreasing child event
// count.  Parent movies keep their event neighbours (A, B) only from level
// ab_level on and for the last node of the level (see k_level).  Returns the
// number of kernel launches.
int launch_level(const Points &pts, const Span &sp, int level, PassBufs *passes, int npass, int32_t *status,
                 cudaStream_t st, int occupancy, int max_events = -1, const LevelOrder *ord = nullptr,
                 int ab_level = 0, bool filter = true);

// One level (>= 2), one warp per merge on a compacted shared-memory table of
// up to scap slots (merges that do not fit run the global-memory merge).
// With max_events >= 0 only merges of at most max_events child events are
// done (the others are left to the time-segment kernels).
void launch_level_cmp(const Points &pts, const Span &sp, int level, PassBufs *passes, int npass, int32_t *status,
                      cudaStream_t st, int scap, int max_events = -1);

// Copies the movie of each cloud's last node of a level when it has no right
// child (the span's ncl clouds; one cloud: only when needed).  Returns the
// number of launches.
int launch_passthrough(const Span &sp, int ncl, int level, PassBufs *passes, int32_t *status, cudaStream_t st);

struct SegBufs;
// Slot tables in global memory for time windows too large for shared memory:
// ctas regions of stride bytes, each holding cap slots (base null: none).
struct SegTables {
    char *base;
    int64_t stride;
    int cap, ctas;
};
// Bytes of a window's slot table of scap slots for windows of up to K child events.
size_t seg_smem_bytes(int scap, int K);

// One level merged time-segment-parallel (windows of Kmin .. K child events,
// see seg_window_len; shared-memory slot tables of scap, then scap_big points,
// then the global-memory tables gt); pairs/pair_vals and their alternates hold
// pair_cap sort items.
void launch_seg_level(const Points &pts, const Span &sp, int level, PassBufs *passes, SegBufs *sbufs, uint64_t *pairs,
                      uint32_t *pair_vals, uint64_t *pairs_alt, uint32_t *vals_alt, unsigned long long *npairs,
                      int *overflow, int64_t pair_cap, int64_t S_cap, int64_t M_cap, int K, int Kmin, int scap,
                      int scap_big, int min_events, const SortScratch &ss, const SegTables &gt, int32_t *status,
                      cudaStream_t st, int64_t *launches);

// Faces of the root movies of both passes (level L = ceil(log2 n) in buffer L & 1):
// orient, rotate min-first, build the sort key (f0 << 28 | f1) and value f2.
void launch_face_keys(const Points &pts, int64_t n, int level, PassBufs *passes, uint64_t *keys, uint32_t *vals,
                      int64_t *d_nfaces, int32_t *status, cudaStream_t st);

// Delaunay triangles of lifted points from the lower pass's root movie (see
// k_tri_keys): keys as launch_face_keys, *d_items keys written (zero-area
// ones with the largest key), *d_ntris the triangles (must start at 0).
void launch_tri_keys(const Points &pts, int64_t n, int level, PassBufs *passes, uint64_t *keys, uint32_t *vals,
                     int64_t *d_items, int64_t *d_ntris, int32_t *status, cudaStream_t st);

// Sorted face keys -> int32 x 3 output rows (key = f0 << fbits | f1, fbits = ceil(log2 n)).
void launch_face_out(const uint64_t *keys, const uint32_t *vals, int64_t cap, int fbits, const int64_t *d_nfaces,
                     int32_t *faces, cudaStream_t st);

// Shared memory of the fused kernel for blocks of 2^l1 ranks.
size_t fused_smem_bytes(int l1);

// Kernel attributes (shared-memory limits), set once per process before any launch.
void merge_kernel_attributes();
void sort_kernel_attributes();
void seg_kernel_attributes();
void batch_kernel_attributes();

// Scratch of the adjacency kernels: the directed-edge keys and edge ids
// (two ping-pong copies of 3 F entries), their radix-sort histograms and the
// device edge count 3 F.
struct AdjScratch {
    uint64_t *k0, *k1;
    uint32_t *v0, *v1;
    int64_t *n3;
    SortScratch ss;
};

// Face neighbours and vertex stars of the canonical face list faces[0, *d_nf)
// (cap rows) of a hull whose vertices are in [0, n): nb[3 f + k] is the face
// holding the edge f[(k + 1) % 3] -> f[k]; star[star_off[v] .. star_off[v + 1])
// are the faces around v, counter-clockwise from outside, starting from the
// smallest.  Returns 0 and the number of launches in *launches.
int launch_adjacency(const int32_t *faces, const int64_t *d_nf, int64_t cap, int64_t n, int32_t *nb,
                     int64_t *star_off, int32_t *star, int32_t *status, const AdjScratch &s, int sms,
                     cudaStream_t st, int64_t *launches);

// Device tables of a group of clouds hulled together (multi.cu): layout
// order c = 0 .. ncl - 1 (clouds by decreasing size, each in an aligned block
// of 2^L_c ranks), blk[] maps each 2^SPAN_SHIFT ranks to its cloud.
struct MultiTables {
    int ncl;
    int32_t *blk;                                 // [rank space >> SPAN_SHIFT]
    int64_t *cbase, *cend;                        // [ncl]: block start, block start + n_c
    int64_t *coff;                                // [ncl + 1]: start of cloud c among the group's points
    int64_t *ioff, *cfoff;                        // [ncl]: first input row, first output face row
    int32_t *ctop, *cstat, *corig;                // [ncl]: L_c, input status, index in the caller's batch
    int64_t *fcount, *fstart;                     // [ncl], [ncl + 1]: faces per cloud and their prefix
};

// Steps 1-3 of a group (see multi.cu): keys, the two stable sorts and the
// decode into the rank space (P); total = points of the group.
int launch_multi_sort(const int32_t *xyz, const MultiTables &t, int C, int64_t total, int4 *P, uint64_t *k0,
                      uint32_t *v0, uint64_t *k1, uint32_t *v1, const SortScratch &ss, int sms, cudaStream_t st,
                      int64_t *launches);

// Step 5: faces of every cloud of the group into the caller's rows, face
// counts and statuses by batch index (cap = face-key capacity of k0 .. v1).
int launch_multi_faces(const Points &pts, const MultiTables &t, int C, int fbits, PassBufs *passes, uint64_t *k0,
                       uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t cap, const SortScratch &ss,
                       const int32_t *status, int32_t *faces, int64_t *nfaces, int32_t *cstatus, int sms,
                       cudaStream_t st, int64_t *launches);

// Batched clouds: size class c (0 .. BATCH_CLASSES - 1) holds clouds of at most
// batch_class_limit(c) points; one persistent launch hulls `count` clouds
// listed in order[] (cloud indices into off/foff), pulling work from *counter.
constexpr int BATCH_CLASSES = 4;
int batch_class_limit(int c);
// Levels of a cloud with fewer than warp_nodes merges run one warp per merge.
// f32: the float32 predicate ablation instead of the exact predicates.
void launch_batch_class(int c, const int32_t *xyz, const int64_t *off, const int64_t *foff, const int32_t *order,
                        int count, int *counter, int32_t *faces, int64_t *nfaces, int32_t *status, int sms,
                        int warp_nodes, bool f32, cudaStream_t st);

}  // namespace hull3d
