// sort.cu -- A1 (validate + key) and A2 (radix sort by the perturbed x-order).
//
// The paper presorts the points by x before the merge levels (Sec. 2; the
// `sort(P, n)` of the figure "Differences in list creation").  Under the
// symbolic perturbation x~ = x + a z + a^2 y the x-order is the lexicographic
// order of (x, z, y), so each point gets the 63-bit key
//   (x + 2^20) << 42 | (z + 2^20) << 21 | (y + 2^20)
// and a stable LSD radix sort (8-bit digits) orders the keys with the input
// index as payload.  The sorted keys decode back to the coordinates, so no
// gather of the input is needed afterwards; equal adjacent keys are duplicates.
#include "internal.h"

namespace hull3d {

__device__ __forceinline__ void set_status(int32_t *status, int code) { atomicCAS(status, 0, code); }

__global__ void k_keys(const int32_t *__restrict__ xyz, int64_t n, uint64_t *__restrict__ keys,
                       uint32_t *__restrict__ vals, int32_t *status)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    const int lo = -(1 << 20), hi = (1 << 20) - 1;
    bool ok = x >= lo && x <= hi && y >= lo && y <= hi && z >= lo && z <= hi;
    if (!ok) set_status(status, HULL3D_ERR_COORD_RANGE);
    uint64_t bx = (uint64_t)(x - lo) & 0x1fffff, by = (uint64_t)(y - lo) & 0x1fffff, bz = (uint64_t)(z - lo) & 0x1fffff;
    keys[i] = (bx << 42) | (bz << 21) | by;
    vals[i] = (uint32_t)i;
}

void launch_keys(const int32_t *xyz, int64_t n, uint64_t *keys, uint32_t *vals, int32_t *status, cudaStream_t st)
{
    if (n <= 0) return;
    k_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(xyz, n, keys, vals, status);
}

// (keys, vals), or (keys_b, vals_b) where *use_b is nonzero
__global__ void k_decode(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n,
                         int4 *__restrict__ P, int32_t *status, const uint64_t *keys_b, const uint32_t *vals_b,
                         const int64_t *use_b)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (use_b && *use_b) {
        keys = keys_b;
        vals = vals_b;
    }
    uint64_t k = keys[i];
    const int lo = -(1 << 20);
    P[i] = make_int4((int)((k >> 42) & 0x1fffff) + lo, (int)(k & 0x1fffff) + lo, (int)((k >> 21) & 0x1fffff) + lo,
                     (int32_t)vals[i]);
    if (i > 0 && keys[i - 1] == k) set_status(status, HULL3D_ERR_DUPLICATE);
}

void launch_decode(const uint64_t *keys, const uint32_t *vals, int64_t n, int4 *P, int32_t *status, cudaStream_t st)
{
    if (n <= 0) return;
    k_decode<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(keys, vals, n, P, status, nullptr, nullptr, nullptr);
}

void launch_decode_either(const uint64_t *keys, const uint32_t *vals, const uint64_t *keys_b, const uint32_t *vals_b,
                          const int64_t *use_b, int64_t n, int4 *P, int32_t *status, cudaStream_t st)
{
    if (n <= 0) return;
    k_decode<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(keys, vals, n, P, status, keys_b, vals_b, use_b);
}

// The point keys after a radix sort of their x bits (42-62) only: each run of
// equal x holds the points of one x-value in input order.  Each key of a run
// of at most max_run keys takes its place in the run by rank: the number of
// the run's keys below it, ties by position (equal keys are duplicate points,
// which the decode reports), and moves from (kin, vin) to (kout, vout) there.
// The threads only read the input, so the runs need no ordering among them.
// On uniform clouds a run holds the few points that share an x-value (eight
// on average at 2^24 points).  The first key of a longer run puts the run on
// the list that k_tie_sort_long sorts one per CTA (a clipped Gaussian puts
// hundreds of points on each clipping plane); a run longer than
// TIE_SORT_LONG_MAX, or more than TIE_SORT_LONG_CAP long runs, ask for the
// full sort instead.
constexpr int TIE_TILE = 2048;     // keys ranked per CTA
constexpr int TIE_THREADS = 256;
constexpr int TIE_HALO = 128;      // = TIE_SORT_MAX_RUN: a short run around the tile lies in the tile and its halos

__global__ void __launch_bounds__(TIE_THREADS) k_tie_sort(const uint64_t *__restrict__ kin,
                                                         const uint32_t *__restrict__ vin,
                                                         uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                         int64_t n, int max_run, TieRuns runs)
{
    // the tile's keys and max_run more on each side, in shared memory
    __shared__ uint64_t K[TIE_TILE + 2 * TIE_HALO];
    const int64_t t0 = (int64_t)blockIdx.x * TIE_TILE;
    const int64_t b0 = t0 - TIE_HALO;
    for (int t = threadIdx.x; t < TIE_TILE + 2 * TIE_HALO; t += TIE_THREADS) {
        const int64_t g = b0 + t;
        K[t] = (g >= 0 && g < n) ? kin[g] : ~0ull;  // outside: never on a run (x bits all ones are out of range)
    }
    __syncthreads();
    for (int u = threadIdx.x; u < TIE_TILE; u += TIE_THREADS) {
        const int64_t a = t0 + u;
        if (a >= n) break;
        const int ia = u + TIE_HALO;  // a's slot
        const uint64_t k = K[ia], x = k >> 42;
        int i = ia;  // the run's first key, looked for at most max_run back
        while (i > 0 && ia - i <= max_run && (K[i - 1] >> 42) == x) i--;
        if (ia - i > max_run) continue;  // in a long run: its first key registers it
        int e = ia + 1;
        while (e < TIE_TILE + 2 * TIE_HALO && e - i <= max_run && (K[e] >> 42) == x) e++;
        if (e - i > max_run) {
            if (i == ia) {  // the first key measures the run in global memory and registers it
                int64_t ge = a + (e - i);
                while (ge < n && ge - a <= TIE_SORT_LONG_MAX && (kin[ge] >> 42) == x) ge++;
                const int slot = ge - a <= TIE_SORT_LONG_MAX ? atomicAdd(runs.count, 1) : TIE_SORT_LONG_CAP;
                if (slot < TIE_SORT_LONG_CAP) {
                    runs.start[slot] = a;
                    runs.len[slot] = (int)(ge - a);
                } else {
                    *runs.fallback_n = n;
                }
            }
            continue;
        }
        int r = 0;
        for (int b = i; b < e; b++) {
            const uint64_t kb = K[b];
            r += (kb < k) | (kb == k && b < ia);
        }
        kout[a - (ia - i) + r] = k;
        vout[a - (ia - i) + r] = vin[a];
    }
}

// The long runs of k_tie_sort, one per CTA at a time: the run's keys in shared
// memory, padded to a power of two with the largest key, a bitonic sort, and
// the run written to the output buffer.
__global__ void __launch_bounds__(1024) k_tie_sort_long(const uint64_t *__restrict__ kin,
                                                        const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
                                                        uint32_t *__restrict__ vout, TieRuns runs);

void launch_tie_sort(const uint64_t *kin, const uint32_t *vin, uint64_t *kout, uint32_t *vout, int64_t n, int max_run,
                     const TieRuns &runs, cudaStream_t st)
{
    if (n <= 0) return;
    k_tie_sort<<<(unsigned)((n + TIE_TILE - 1) / TIE_TILE), TIE_THREADS, 0, st>>>(kin, vin, kout, vout, n,
                                                                                   max_run < TIE_HALO ? max_run : TIE_HALO,
                                                                                   runs);
    k_tie_sort_long<<<64, 1024, 0, st>>>(kin, vin, kout, vout, runs);
}

// ---------------------------------------------------------------------------
// Small clouds (n <= SMALL_SORT_MAX): the key build, the sort, the decode and
// the duplicate check in one CTA, the keys sorted by a bitonic network in
// shared memory; and the canonical face sort of such a hull (at most
// 2 SMALL_SORT_MAX - 4 faces) the same way.  Two launches instead of the
// radix sort's three per pass.
// ---------------------------------------------------------------------------
template <class V>
__device__ void bitonic_block(uint64_t *k, V *v, int m)
{
    for (int size = 2; size <= m; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (m >> 1); t += blockDim.x) {
                const int i = 2 * t - (t & (stride - 1)), j = i + stride;
                if ((k[i] > k[j]) == ((i & size) == 0)) {
                    const uint64_t tk = k[i]; k[i] = k[j]; k[j] = tk;
                    const V tv = v[i]; v[i] = v[j]; v[j] = tv;
                }
            }
            __syncthreads();
        }
}

__global__ void __launch_bounds__(1024) k_tie_sort_long(const uint64_t *__restrict__ kin,
                                                        const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
                                                        uint32_t *__restrict__ vout, TieRuns runs)
{
    __shared__ uint64_t K[TIE_SORT_LONG_MAX];
    __shared__ uint32_t V[TIE_SORT_LONG_MAX];
    const int cnt = min(*runs.count, TIE_SORT_LONG_CAP);
    for (int r = blockIdx.x; r < cnt; r += gridDim.x) {
        const int64_t s = runs.start[r];
        const int len = runs.len[r];
        int m = 1;
        while (m < len) m <<= 1;
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            K[t] = t < len ? kin[s + t] : ~0ull;
            V[t] = t < len ? vin[s + t] : 0u;
        }
        __syncthreads();
        bitonic_block(K, V, m);
        for (int t = threadIdx.x; t < len; t += blockDim.x) {
            kout[s + t] = K[t];
            vout[s + t] = V[t];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SMALL_SORT_THREADS) k_small_sort(const int32_t *__restrict__ xyz, int n,
                                                                    int4 *__restrict__ P, int32_t *status)
{
    __shared__ uint64_t K[SMALL_SORT_MAX];
    __shared__ unsigned short V[SMALL_SORT_MAX];
    int m = 1;
    while (m < n) m <<= 1;
    const int lo = -(1 << 20), hi = (1 << 20) - 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        if (i < n) {
            const int x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
            if (x < lo || x > hi || y < lo || y > hi || z < lo || z > hi) set_status(status, HULL3D_ERR_COORD_RANGE);
            K[i] = ((uint64_t)((x - lo) & 0x1fffff) << 42) | ((uint64_t)((z - lo) & 0x1fffff) << 21) |
                   (uint64_t)((y - lo) & 0x1fffff);
        } else {
            K[i] = ~0ull;
        }
        V[i] = (unsigned short)i;
    }
    __syncthreads();
    bitonic_block(K, V, m);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const uint64_t k = K[i];
        P[i] = make_int4((int)((k >> 42) & 0x1fffff) + lo, (int)(k & 0x1fffff) + lo, (int)((k >> 21) & 0x1fffff) + lo,
                         (int)V[i]);
        if (i > 0 && K[i - 1] == k) set_status(status, HULL3D_ERR_DUPLICATE);
    }
}

void launch_small_sort(const int32_t *xyz, int64_t n, int4 *P, int32_t *status, cudaStream_t st)
{
    k_small_sort<<<1, SMALL_SORT_THREADS, 0, st>>>(xyz, (int)n, P, status);
}

constexpr int SMALL_FACES = 2 * SMALL_SORT_MAX;
constexpr size_t SMALL_FACE_SMEM = (size_t)SMALL_FACES * (sizeof(uint64_t) + sizeof(uint32_t));

// keys f0 << fbits | f1 and values f2 of *d_nf faces -> sorted int32 x 3 rows
__global__ void __launch_bounds__(SMALL_SORT_THREADS) k_small_face_sort(const uint64_t *__restrict__ keys,
                                                                         const uint32_t *__restrict__ vals, int fbits,
                                                                         const int64_t *d_nf, int32_t *faces)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    uint64_t *K = (uint64_t *)fsm;
    uint32_t *V = (uint32_t *)(K + SMALL_FACES);
    const int nf = (int)min(*d_nf, (int64_t)SMALL_FACES);
    int m = 1;
    while (m < nf) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        K[i] = i < nf ? keys[i] : ~0ull;
        V[i] = i < nf ? vals[i] : 0u;
    }
    __syncthreads();
    bitonic_block(K, V, m);
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const uint64_t k = K[i];
        faces[3 * i] = (int32_t)(k >> fbits);
        faces[3 * i + 1] = (int32_t)(k & ((1ull << fbits) - 1));
        faces[3 * i + 2] = (int32_t)V[i];
    }
}

void launch_small_face_sort(const uint64_t *keys, const uint32_t *vals, int fbits, const int64_t *d_nf,
                            int32_t *faces, cudaStream_t st)
{
    k_small_face_sort<<<1, SMALL_SORT_THREADS, SMALL_FACE_SMEM, st>>>(keys, vals, fbits, d_nf, faces);
}

// ---------------------------------------------------------------------------
// 2D points lifted to the paraboloid (x, y, x^2 + y^2) for the Delaunay
// triangulation: |x|, |y| < 2^15, so z < 2^31 and the x-order key (x, z, y)
// packs into 16 + 31 + 16 bits.
// ---------------------------------------------------------------------------
constexpr int LIFT_LIM = (1 << 15) - 1;

__global__ void k_keys_lifted(const int32_t *__restrict__ xy, int64_t n, uint64_t *__restrict__ keys,
                              uint32_t *__restrict__ vals, int32_t *status)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = xy[2 * i], y = xy[2 * i + 1];
    if (x < -LIFT_LIM || x > LIFT_LIM || y < -LIFT_LIM || y > LIFT_LIM) {
        set_status(status, HULL3D_ERR_COORD_RANGE);
        keys[i] = 0;
    } else {
        const uint64_t z = (uint64_t)((int64_t)x * x + (int64_t)y * y);
        keys[i] = ((uint64_t)(x + (1 << 15)) << 47) | (z << 16) | (uint64_t)(y + (1 << 15));
    }
    vals[i] = (uint32_t)i;
}

void launch_keys_lifted(const int32_t *xy, int64_t n, uint64_t *keys, uint32_t *vals, int32_t *status,
                        cudaStream_t st)
{
    if (n <= 0) return;
    k_keys_lifted<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(xy, n, keys, vals, status);
}

__global__ void k_decode_lifted(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n,
                                int4 *__restrict__ P, int32_t *status)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t k = keys[i];
    P[i] = make_int4((int)(k >> 47) - (1 << 15), (int)(k & 0xffff) - (1 << 15), (int)((k >> 16) & 0x7fffffff),
                     (int32_t)vals[i]);
    if (i > 0 && keys[i - 1] == k) set_status(status, HULL3D_ERR_DUPLICATE);
}

void launch_decode_lifted(const uint64_t *keys, const uint32_t *vals, int64_t n, int4 *P, int32_t *status,
                          cudaStream_t st)
{
    if (n <= 0) return;
    k_decode_lifted<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(keys, vals, n, P, status);
}

// ---------------------------------------------------------------------------
// LSD radix sort, 8-bit digits, 3 kernels per pass:
//   hist    per-tile digit histogram -> hist[digit * T + tile]
//   rowscan per-digit exclusive scan over tiles, row totals -> rowsum[digit]
//   scatter stable per-tile ranking (warp match + per-warp bases), the tile
//           staged in shared memory in digit order, written out in runs
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = SORT_TILE / RS_THREADS;  // 16
constexpr int RS_WARPS = RS_THREADS / 32;

// items to sort: the capacity n, or a device count clamped to it
__device__ __forceinline__ int64_t count_of(int64_t n, const int64_t *d_n)
{
    if (!d_n) return n;
    int64_t c = *d_n;
    return c < n ? c : n;
}

// (grid-stride over the tiles in use, so a small device count costs little)
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t *__restrict__ keys, int64_t n,
                                                        const int64_t *d_n, int shift, uint32_t *hist, int64_t T)
{
    __shared__ uint32_t h[256];
    const int64_t cnt = count_of(n, d_n);
    const int64_t Tu = (cnt + SORT_TILE - 1) / SORT_TILE;
    for (int64_t tile = blockIdx.x; tile < Tu; tile += gridDim.x) {
        h[threadIdx.x] = 0;
        __syncthreads();
        const int64_t base = tile * SORT_TILE;
#pragma unroll 4
        for (int it = 0; it < RS_ITEMS; it++) {
            int64_t i = base + it * RS_THREADS + threadIdx.x;
            if (i < cnt) atomicAdd(&h[(keys[i] >> shift) & 0xff], 1u);
        }
        __syncthreads();
        hist[threadIdx.x * T + tile] = h[threadIdx.x];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_rs_rowscan(uint32_t *hist, int64_t T, const int64_t *d_n, int64_t n,
                                                     uint32_t *rowsum)
{
    __shared__ uint32_t wsum[32];
    int64_t cnt = count_of(n, d_n);
    int64_t Tu = (cnt + SORT_TILE - 1) / SORT_TILE;  // tiles in use
    uint32_t *row = hist + blockIdx.x * T;
    int per = (int)((Tu + 1023) / 1024);
    int64_t b0 = threadIdx.x * (int64_t)per;
    uint32_t s = 0;
    for (int k = 0; k < per; k++)
        if (b0 + k < Tu) s += row[b0 + k];
    // block exclusive scan of s
    uint32_t x = s;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;  // inclusive
    }
    __syncthreads();
    uint32_t run = x - s + (w ? wsum[w - 1] : 0);  // exclusive prefix of this thread's chunk
    for (int k = 0; k < per; k++)
        if (b0 + k < Tu) {
            uint32_t t = row[b0 + k];
            row[b0 + k] = run;
            run += t;
        }
    if (threadIdx.x == 1023) rowsum[blockIdx.x] = run;
}

// The tile is ranked stably (warp, then item, then lane), each item first goes
// to its position in the tile's digit-sorted order in shared memory, and the
// tile is then written out in that order, so consecutive threads write
// consecutive addresses of one digit's output run instead of 32 scattered
// buckets per store.  The kernel waits mostly on the shared-memory pipe (warp
// matches, staging stores), so three blocks per SM (80 registers, a few bytes
// spilled) hide more of it than two: the 2^24 point sort 2.5 -> 1.9 ms.
constexpr size_t RS_STAGE_BYTES = (size_t)SORT_TILE * (sizeof(uint64_t) + sizeof(uint32_t));

__global__ void __launch_bounds__(RS_THREADS, 3) k_rs_scatter(const uint64_t *__restrict__ kin,
                                                           const uint32_t *__restrict__ vin,
                                                           uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                           int64_t n, const int64_t *d_n, int shift,
                                                           const uint32_t *__restrict__ hist, int64_t T,
                                                           const uint32_t *__restrict__ rowsum)
{
    extern __shared__ __align__(16) unsigned char rs_stage[];
    uint64_t *sk = (uint64_t *)rs_stage;         // [SORT_TILE] keys in tile order by digit
    uint32_t *sv = (uint32_t *)(sk + SORT_TILE);  // [SORT_TILE] their values
    __shared__ uint32_t gofs[256];                // output index of tile position 0 of each digit's run
    __shared__ uint32_t wh[RS_WARPS][256];
    __shared__ uint32_t ws[RS_WARPS];
    const int64_t cnt = count_of(n, d_n);
    const int64_t Tu = (cnt + SORT_TILE - 1) / SORT_TILE;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t tile = blockIdx.x; tile < Tu; tile += gridDim.x) {
        const int64_t base = tile * SORT_TILE;
        const int nvalid = (int)(cnt - base < SORT_TILE ? cnt - base : SORT_TILE);

        // output base of digit tid for this tile: exclusive scan of the row
        // totals plus this tile's row prefix
        uint32_t obase;
        {
            const uint32_t v = rowsum[tid];
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) ws[w] = x;
            __syncthreads();
            uint32_t off = 0;
            for (int k = 0; k < w; k++) off += ws[k];
            obase = off + x - v + hist[tid * T + tile];
        }
#pragma unroll
        for (int k = 0; k < RS_WARPS; k++) wh[k][tid] = 0;
        __syncthreads();

        uint64_t kk[RS_ITEMS];
        uint32_t vv[RS_ITEMS];
        int dd[RS_ITEMS];
        const int64_t wbase = base + w * (32 * RS_ITEMS);
#pragma unroll
        for (int r = 0; r < RS_ITEMS; r++) {
            const int64_t i = wbase + r * 32 + lane;
            if (i < cnt) { kk[r] = kin[i]; vv[r] = vin[i]; dd[r] = (int)((kk[r] >> shift) & 0xff); }
            else { kk[r] = 0; vv[r] = 0; dd[r] = 256 + lane; }
        }
        // per-warp digit counts; each item's peer mask (the lanes holding the
        // same digit in its round) is kept for the ranking below
        unsigned pm[RS_ITEMS];
#pragma unroll
        for (int r = 0; r < RS_ITEMS; r++) {
            pm[r] = __match_any_sync(0xffffffffu, dd[r]);
            if (dd[r] < 256 && (pm[r] & lt) == 0) wh[w][dd[r]] += __popc(pm[r]);
            __syncwarp();
        }
        __syncthreads();
        {  // digit tid: tile-local start of its run, and each warp's start inside it
            uint32_t tot = 0;
#pragma unroll
            for (int k = 0; k < RS_WARPS; k++) tot += wh[k][tid];
            uint32_t x = tot;  // inclusive scan of the digit totals over the block
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            __syncthreads();  // every thread has read ws (output bases) above
            if (lane == 31) ws[w] = x;
            __syncthreads();
            uint32_t off = 0;
            for (int k = 0; k < w; k++) off += ws[k];
            uint32_t run = off + x - tot;  // exclusive: tile position of digit tid's first item
            gofs[tid] = obase - run;       // (mod 2^32) output index = gofs[d] + tile position
#pragma unroll
            for (int k = 0; k < RS_WARPS; k++) {
                const uint32_t t = wh[k][tid];
                wh[k][tid] = run;
                run += t;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RS_ITEMS; r++) {
            const unsigned peers = pm[r];
            uint32_t pos = 0;
            if (dd[r] < 256) pos = wh[w][dd[r]] + __popc(peers & lt);
            __syncwarp();
            if (dd[r] < 256 && (peers & lt) == 0) wh[w][dd[r]] += __popc(peers);
            __syncwarp();
            if (dd[r] < 256) { sk[pos] = kk[r]; sv[pos] = vv[r]; }
        }
        __syncthreads();
        for (int j = tid; j < nvalid; j += RS_THREADS) {
            const uint64_t k = sk[j];
            const uint32_t g = gofs[(int)((k >> shift) & 0xff)] + (uint32_t)j;
            kout[g] = k;
            vout[g] = sv[j];
        }
        __syncthreads();  // the stage and the tables are rewritten by the next tile
    }
}

void sort_kernel_attributes()
{
    cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RS_STAGE_BYTES);
    cudaFuncSetAttribute(k_small_face_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMALL_FACE_SMEM);
}

int radix_sort_pairs(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t n, const int64_t *d_n,
                     int bits, const SortScratch &s, cudaStream_t st, int64_t *launches, int lo_bit)
{
    if (n <= 0) return 0;
    int64_t T = (n + SORT_TILE - 1) / SORT_TILE;
    int passes = (bits + 7) / 8;
    static int grid_cap = 0;  // a few CTAs per SM: the kernels loop over the tiles in use
    if (!grid_cap) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid_cap = sms > 0 ? 8 * sms : 1024;
    }
    const unsigned G = (unsigned)(T < grid_cap ? T : grid_cap);
    uint64_t *ka = k0, *kb = k1;
    uint32_t *va = v0, *vb = v1;
    for (int p = 0; p < passes; p++) {
        int shift = lo_bit + 8 * p;
        k_rs_hist<<<G, RS_THREADS, 0, st>>>(ka, n, d_n, shift, s.hist, T);
        k_rs_rowscan<<<256, 1024, 0, st>>>(s.hist, T, d_n, n, s.rowsum);
        k_rs_scatter<<<G, RS_THREADS, RS_STAGE_BYTES, st>>>(ka, va, kb, vb, n, d_n, shift, s.hist, T, s.rowsum);
        if (launches) *launches += 3;
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    return (passes & 1) ? 1 : 0;
}

}  // namespace hull3d
