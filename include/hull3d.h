/*
 * hull3d.h -- C ABI of the GB300 kinetic divide-and-conquer 3D convex hull.
 *
 * The problem (White & Wortman, Sec. 1): given n points in R^3, find the
 * faces of their convex hull.  The method (Sec. 2): sort the points by x,
 * recast the lower hull as a kinetic 2D hull whose "movie" is a chronological
 * list of insert/delete events, build those movies bottom-up by merging
 * adjacent blocks level by level (ceil(log2 n) merge steps, each merge
 * tracking the bridge between its two halves), and read the faces off the
 * root movie (each event is one face).  The upper hull is the same
 * computation on the z-mirrored set.
 *
 * Conventions shared by every entry point
 *   - Points are int32 triples (x, y, z), row-major n x 3, every coordinate in
 *     [-2^20, 2^20).  Duplicated points are an error.
 *   - Degenerate inputs (equal x, collinear or coplanar points) are resolved
 *     by one fixed symbolic perturbation:
 *       x~ = x + a z + a^2 y,  y~ = y + b z + eta_i,  z~ = z + gam_i
 *     (i = input index, a >> b >> gam_0 >> ... >> gam_{n-1} >> eta_0 >> ...),
 *     so the output is always a triangulated closed surface with
 *     F = 2V - 4 faces, V <= n.  All arithmetic is exact integer arithmetic.
 *   - Output faces are int32 triples of INPUT indices, counter-clockwise seen
 *     from outside, rotated so the smallest index comes first, and sorted
 *     lexicographically.  n <= 2 gives 0 faces, n = 3 gives the triangle's
 *     two sides.  At most 2n - 4 faces (n >= 3).
 *   - Device pointers are CUDA device (or managed) memory owned by the
 *     caller; the plan owns all scratch.  "stream" is a cudaStream_t (NULL =
 *     the legacy default stream).  Asynchronous entry points only enqueue
 *     work; their results are valid once the stream has reached them.
 *   - Return values: 0 on success, else a HULL3D_ERR_* code (see
 *     hull3d_strerror).  Nothing aborts, traps or prints.
 */
#ifndef HULL3D_H
#define HULL3D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HULL3D_OK 0
#define HULL3D_ERR_INVALID_ARG 1   /* null pointer, n < 1, n above the plan, bad offsets */
#define HULL3D_ERR_COORD_RANGE 2   /* a coordinate outside [-2^20, 2^20) */
#define HULL3D_ERR_DUPLICATE 3     /* two equal points */
#define HULL3D_ERR_CAPACITY 4      /* output capacity below 2n - 4 faces */
#define HULL3D_ERR_OOM 5           /* device allocation failed */
#define HULL3D_ERR_BUDGET 6        /* request above a memory budget */
#define HULL3D_ERR_DEVICE_TIMEOUT 7 /* a bounded device wait ran out */
#define HULL3D_ERR_CUDA 8          /* a CUDA runtime call failed (see hull3d_last_cuda_error) */
#define HULL3D_ERR_INTERNAL 9      /* an internal consistency check failed */
#define HULL3D_ERR_TOO_LARGE 10    /* n above HULL3D_STATIC_MAX_N (hull3d_compute_static only) */
#define HULL3D_ERR_NOT_CLOSED 11   /* faces are not a closed, consistently oriented surface (hull3d_adjacency_async) */

#define HULL3D_MAX_N (1 << 28)     /* largest n one plan accepts */

typedef struct hull3d_plan_s *hull3d_plan_t;

/* Tuning knobs; zero fields mean "automatic" (hull3d_plan_opts reports the
 * resolved values).  None of them changes the result, only its speed, except
 * float32_ablation, which exists to measure the paper's float arithmetic. */
typedef struct {
    int32_t fused_levels;    /* bottom levels merged in one shared-memory kernel (1 = none, up to 10) */
    int32_t seg_level;       /* first level merged time-segment-parallel (> log2 n: never) */
    int32_t seg_events;      /* longest time window of a segment-parallel merge, in child events */
    int32_t use_graph;       /* 1: replay the level sequence as a CUDA graph, -1: plain launches */
    int32_t level_occupancy; /* thread-per-merge kernel: 128-thread blocks per SM its register cap allows (1 = no cap .. 4;
                                automatic: 4 at levels 2-5 and 9, 3 at levels 6-8, 1 above) */
    int32_t cmp_level;       /* first level merged by the compacted warp-per-merge kernel (automatic:
                                log2 n - 11 within [6, 13] for a hull of n points) */
    int32_t cmp_slots;       /* its shared-memory table size in points (<= 4096; automatic: 1024, and on
                                time-window levels the 4 + seg_min_events points its largest merge needs) */
    int32_t seg_slots;       /* shared-memory table size of one time window in points (<= 6144) */
    int32_t seg_min_events;  /* from seg_level on, merges with fewer child events use the compacted kernel
                                (automatic: 128 on levels with at most 128 merges per pass, else 512) */
    int32_t merge_order;     /* thread-per-merge levels 3-8 run their merges longest first: 1 (default),
                                or in x-order: -1 */
    int32_t seg_events_min;  /* shortest time window; a merge of E child events gets 2 sqrt(E) within
                                [seg_events_min, seg_events] */
    int32_t batch_warp_nodes; /* batch kernel: levels of a cloud with fewer merges than this run one warp per
                                 merge, the others one thread per merge (automatic: 64) */
    int32_t multi_ranks;     /* batch calls: clouds above 4096 points are hulled together in groups whose
                                aligned blocks fill at most this many ranks (automatic and at most: max_n) */
    int32_t float32_ablation; /* 1: batch calls hull the clouds of at most 4096 points with the float32
                                 arithmetic of the paper's GPU kernel (Sec. 3: cl_float coordinates) instead
                                 of the exact predicates -- an ablation: the result need not be the hull,
                                 and is the only knob here that can change it.  0: exact (default) */
    int32_t seg_slots_big;   /* shared-memory table size of the third round of time windows (<= 6144, automatic:
                                6144; the second round's holds 3072, or this many if fewer); windows too large
                                for it get slot tables in global memory */
    int32_t filter_level;    /* first merge level of the thread-per-merge kernel whose time comparisons try a
                                float filter before the exact products (the result is the same; automatic: 3 up
                                to 2^21 points, log2(n) - 15 above, where points share x-values) */
} hull3d_opts;

/* Creates a plan for hulls of up to max_n points (hull3d_compute*) and for
 * batches of up to max_clouds clouds totalling up to max_n points
 * (hull3d_batch).  Allocates every scratch buffer up front on the current
 * device.  opts may be NULL.  On failure *out is NULL and the code is
 * HULL3D_ERR_INVALID_ARG or HULL3D_ERR_OOM.  Sec. 3: the point array P and
 * the two event arrays A and B of 2n entries are allocated once, before the
 * main loop; a plan holds those and every other buffer of the pipeline. */
int hull3d_plan(hull3d_plan_t *out, int64_t max_n, int64_t max_clouds, const hull3d_opts *opts);

/* Copies the plan's effective options (automatic fields resolved) into *out. */
int hull3d_plan_opts(hull3d_plan_t plan, hull3d_opts *out);

/* Frees the plan and its scratch (synchronises the device first). NULL is a no-op. */
void hull3d_destroy(hull3d_plan_t plan);

/* Bytes of device scratch the plan holds. */
int64_t hull3d_plan_bytes(hull3d_plan_t plan);

/* Enqueues the hull of n points on stream.
 *   d_xyz     device, n x 3 int32, read only
 *   d_faces   device, cap_faces x 3 int32, written with the canonical faces
 *   d_nfaces  device int64, written with the face count (may be NULL)
 *   d_status  device int32, written with 0 or a HULL3D_ERR_* code detected on
 *             the device (range, duplicate, internal) (may be NULL)
 * Host-detected argument errors are returned immediately and nothing is
 * enqueued.  Calls sharing a plan must be serialised on one stream (they
 * share its scratch).  Sec. 2 ("movie array" merge steps), Sec. 3 (act, time). */
int hull3d_compute_async(hull3d_plan_t plan, const int32_t *d_xyz, int64_t n, int32_t *d_faces,
                         int64_t cap_faces, int64_t *d_nfaces, int32_t *d_status, void *stream);

/* Synchronous form of hull3d_compute_async: enqueues, waits for the stream,
 * stores the face count in *h_nfaces (host, may be NULL) and returns the
 * device-detected status.  Sec. 2 and Sec. 3 as for hull3d_compute_async;
 * the blocking face-count readback is an addition of this library. */
int hull3d_compute(hull3d_plan_t plan, const int32_t *d_xyz, int64_t n, int32_t *d_faces, int64_t cap_faces,
                   int64_t *h_nfaces, void *stream);

/* End-to-end form on HOST buffers: copies h_xyz (n x 3 int32) to the device,
 * computes, copies the faces back to h_faces (cap_faces x 3 int32) and the
 * count to *h_nfaces, then returns the status.  Uses plan-owned device
 * staging buffers; the host buffers should be pinned for full copy speed.
 * Sec. 3: the host only uploads the points, runs every merge level on the
 * GPU without reading anything back in between, and reads the result once. */
int hull3d_compute_host(hull3d_plan_t plan, const int32_t *h_xyz, int64_t n, int32_t *h_faces, int64_t cap_faces,
                        int64_t *h_nfaces, void *stream);

/* Enqueues the hulls of B independent clouds concatenated in d_xyz.
 * Sec. 2 notes that the merges of a level are independent of one another;
 * hulling many independent clouds in one call is an addition of this library
 * (no paper counterpart).
 *   h_offsets       host int64 [B+1]: cloud b is rows [h_offsets[b], h_offsets[b+1]) of d_xyz
 *   d_faces         device int32 x 3: cloud b's faces start at row h_face_offsets[b]
 *   h_face_offsets  host int64 [B+1]: row capacity of cloud b is
 *                   h_face_offsets[b+1] - h_face_offsets[b] (needs max(0, 2 n_b - 4))
 *   d_nfaces        device int64 [B]: face count per cloud
 *   d_status        device int32 [B]: 0 or a HULL3D_ERR_* code per cloud
 * Faces are per-cloud canonical lists of indices local to the cloud.  Each
 * cloud may hold up to the plan's max_n points.  Host-detected argument
 * errors (bad offsets, capacity) are returned before anything is enqueued. */
int hull3d_batch_async(hull3d_plan_t plan, const int32_t *d_xyz, const int64_t *h_offsets, int64_t B,
                       int32_t *d_faces, const int64_t *h_face_offsets, int64_t *d_nfaces, int32_t *d_status,
                       void *stream);

/* 2D Delaunay triangulation through the lifting map: the points (x, y) are
 * lifted to (x, y, x^2 + y^2), whose lower hull projects to the Delaunay
 * triangulation, and the hull pipeline's lower pass (Sec. 2) computes it.
 * This is an application of the paper's method, not a part of the paper.
 *   d_xy      device, n x 2 int32, |x| and |y| < 2^15 (so x^2 + y^2 < 2^31)
 *   d_tris    device, cap_tris x 3 int32 (cap_tris >= 2n - 4 for n >= 3):
 *             triangles of input indices, counter-clockwise in the plane,
 *             rotated min-first, sorted; the lower faces of zero area (points
 *             on one edge of the convex hull) are not triangles and are left
 *             out, so n points with h on the hull boundary give 2n - h - 2
 *   d_ntris   device int64, the triangle count (may be NULL)
 *   d_status  device int32, 0 or HULL3D_ERR_COORD_RANGE / _DUPLICATE /
 *             _INTERNAL found on the device (may be NULL)
 * Four or more cocircular points get one consistent triangulation (the
 * perturbation of the hull decides).  Uses the plan's scratch; host-detected
 * argument errors are returned before anything is enqueued. */
int hull3d_delaunay_async(hull3d_plan_t plan, const int32_t *d_xy, int64_t n, int32_t *d_tris, int64_t cap_tris,
                          int64_t *d_ntris, int32_t *d_status, void *stream);

/* Adjacency of a hull: the arrangement structure (a doubly connected edge
 * list, in essence) that the paper names as the prerequisite for further
 * geometric algorithms on the GPU (Sec. 5), built from a canonical face list
 * such as hull3d_compute_async writes.
 *   d_faces     device int32 [cap_faces x 3]: outward counter-clockwise faces,
 *               rows [0, *d_nfaces) used, vertex indices in [0, n)
 *   d_nfaces    device int64: the face count F (0 <= F <= cap_faces)
 *   n           number of vertices (1 <= n <= the plan's max_n)
 *   cap_faces   at most 2 * max_n
 *   d_nb        device int32 [cap_faces x 3]: d_nb[3 f + k] is the face that
 *               holds the directed edge d_faces[f][(k + 1) % 3] -> d_faces[f][k]
 *               (the face across edge k of f)
 *   d_star_off  device int64 [n + 1], d_star device int32 [3 cap_faces]: the
 *               faces around vertex v are d_star[d_star_off[v] ..
 *               d_star_off[v + 1]), counter-clockwise seen from outside,
 *               starting from the smallest face index; a vertex on no face
 *               (an interior point) has none
 *   d_status    device int32: 0, or HULL3D_ERR_NOT_CLOSED when an edge has no
 *               opposite, is held twice, or the faces around a vertex do not
 *               form one cycle; HULL3D_ERR_INVALID_ARG when F > cap_faces
 * Stream-ordered; uses the plan's scratch (serialise it with the plan's
 * other calls on one stream).  Host-detected argument errors are returned
 * before anything is enqueued. */
int hull3d_adjacency_async(hull3d_plan_t plan, const int32_t *d_faces, const int64_t *d_nfaces, int64_t cap_faces,
                           int64_t n, int32_t *d_nb, int64_t *d_star_off, int32_t *d_star, int32_t *d_status,
                           void *stream);

/* Allocation-free form of hull3d_compute_async, for hulls of at most
 * HULL3D_STATIC_MAX_N points.  The paper has no counterpart: this is a
 * convenience of this library.
 *
 * It exists for callers that may not allocate device memory themselves:
 * code running inside a host framework that owns every byte of the device
 * (a fixed memory pool or a budget it must not exceed), and latency-critical
 * loops that cannot afford cudaMalloc/cudaFree, which may synchronise the
 * device.  Such callers pass their own input and output buffers; all
 * scratch comes from one static device array of HULL3D_STATIC_SCRATCH_BYTES
 * that this library defines, so every GPU that loads the library holds that
 * array until the process exits.  This entry point calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *
 *   d_xyz, n, d_faces, cap_faces, d_nfaces, d_status, stream: as for
 *   hull3d_compute_async (d_nfaces and d_status may not be NULL here).
 *   n > HULL3D_STATIC_MAX_N returns HULL3D_ERR_TOO_LARGE and enqueues nothing.
 *
 * The first call on a device looks up the device address of the static array
 * (with that device current); make that first call before any stream capture.
 * All calls share the one array: calls whose work may overlap on the GPU
 * (different streams, or different host threads) race and must be serialised
 * by the caller.  Every value the pipeline needs to start from zero is
 * cleared by each call, so the contents left by an earlier call do not matter. */
#define HULL3D_STATIC_MAX_N 16384
#define HULL3D_STATIC_SCRATCH_BYTES (4 << 20)
int hull3d_compute_static(const int32_t *d_xyz, int64_t n, int32_t *d_faces, int64_t cap_faces, int64_t *d_nfaces,
                          int32_t *d_status, void *stream);

/* Text for a HULL3D_* code. */
const char *hull3d_strerror(int code);

/* The last CUDA runtime error code seen by the library on this thread (0 if none). */
int hull3d_last_cuda_error(void);

/* Number of kernel launches the last call on this plan enqueued (graph nodes
 * count one each). */
int64_t hull3d_last_launch_count(hull3d_plan_t plan);

/* Phase timing.  With enable = 1, every later single-hull call records CUDA
 * events on its own stream at the boundaries of its phases
 *   0 sort   (range check, key build, radix sort, decode, duplicate check)
 *   1 fused  (bottom merge levels in shared memory)
 *   2 levels (merge levels in global memory)
 *   3 seg    (time-segment-parallel top levels)
 *   4 faces  (face emission and canonical sort)
 * hull3d_profile_read waits for the recorded events, writes the per-phase
 * milliseconds summed over the recorded calls into ms[HULL3D_PHASES] and the
 * number of calls into *calls, and clears the record.  enable = 0 stops
 * recording. */
#define HULL3D_PHASES 5
int hull3d_profile(hull3d_plan_t plan, int enable);
int hull3d_profile_read(hull3d_plan_t plan, double *ms, int64_t *calls);

/* Per merge level launched in global memory: ms[level] summed over the
 * recorded calls of hull3d_compute*, hull3d_batch_async and
 * hull3d_delaunay_async (call before hull3d_profile_read, which clears the
 * record). */
int hull3d_profile_levels(hull3d_plan_t plan, double *ms);

/* Movie lengths of the last single-hull call: out[pass * 64 + level] is the
 * total number of events written at that merge level (pass 0 lower, 1
 * upper).  Synchronises the device. */
int hull3d_level_events(hull3d_plan_t plan, int64_t *out);

/* Time-window counters of the last call (hull3d_compute*, the large clouds of
 * hull3d_batch_async, hull3d_delaunay_async), both passes together, for the
 * levels merged in windows (Sec. 3's segment-parallel merge at the top
 * levels): out[level * HULL3D_WINDOW_STATS + k] with k
 *   0 the level's start-hull entries overflowed their buffer (1/0: every
 *     windowed merge of the level then ran serially)
 *   1 merges cut into windows
 *   2 windows
 *   3 windows retried with the larger shared-memory tables (3072, then
 *     seg_slots_big slots)
 *   4 windows run with a slot table in global memory
 *   5 merges that fit no table and ran serially (one thread each)
 *   6 the window-length multiplier of a second attempt, taken when the
 *     first one's start-hull entries overflowed (0: none; counters 1-5
 *     then describe the second attempt)
 * for level = 0 .. 63 (zero where no windows ran).  out holds
 * 64 * HULL3D_WINDOW_STATS entries.  Synchronises the device. */
#define HULL3D_WINDOW_STATS 7
int hull3d_window_stats(hull3d_plan_t plan, int64_t *out);

#ifdef __cplusplus
}
#endif

#endif /* HULL3D_H */
