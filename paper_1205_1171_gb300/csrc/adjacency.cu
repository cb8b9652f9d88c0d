// adjacency.cu -- the hull's arrangement structure: the face across each
// directed edge and the faces around each vertex.  The paper names an
// arrangement structure such as a doubly connected edge list as what further
// geometric algorithms on the GPU need (Sec. 5); for a closed triangulated
// hull given as its canonical face list (outward counter-clockwise triples)
// it is fixed by these two relations.
//
//   1. Face f has the directed edges e = 3 f + k, from f[k] to f[(k + 1) % 3],
//      each keyed (source << b | target), b = ceil(log2 n).
//   2. A radix sort of the keys groups the edges by source vertex: the group
//      of v starts at off[v] and holds one edge for each face around v, so
//      off[] is also the CSR offset array of the vertex stars.
//   3. The face across (a, b) is the one holding (b, a): a binary search in
//      b's group.  A missing or repeated directed edge means the faces are not
//      a closed, consistently oriented surface (HULL3D_ERR_NOT_CLOSED).
//   4. Each vertex walks its star from its smallest face f = (v, x, y) (in its
//      rotation to v) to the face across y -> v, counter-clockwise seen from
//      outside, until it is back at the start after exactly deg(v) faces.
#include "internal.h"

namespace hull3d {

__device__ __forceinline__ void adj_status(int32_t *status, int code) { atomicCAS(status, 0, code); }

// edges in use: 3 F, F clamped to the capacity
__device__ __forceinline__ int64_t adj_edges(const int64_t *d_nf, int64_t cap)
{
    const int64_t f = *d_nf;
    return 3 * (f < 0 ? 0 : (f < cap ? f : cap));
}

__global__ void k_adj_keys(const int32_t *__restrict__ faces, const int64_t *d_nf, int64_t cap, int64_t n, int bits,
                           uint64_t *__restrict__ keys, uint32_t *__restrict__ vals, int64_t *d_n3, int32_t *status)
{
    const int64_t m = adj_edges(d_nf, cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *d_n3 = m;
        if (*d_nf < 0 || *d_nf > cap) adj_status(status, HULL3D_ERR_INVALID_ARG);
    }
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = e / 3;
        const int k = (int)(e - 3 * f);
        const int a = faces[3 * f + k], b = faces[3 * f + (k == 2 ? 0 : k + 1)];
        if (a < 0 || a >= n || b < 0 || b >= n || a == b) {
            adj_status(status, HULL3D_ERR_NOT_CLOSED);
            keys[e] = 0;
        } else {
            keys[e] = ((uint64_t)a << bits) | (uint64_t)b;
        }
        vals[e] = (uint32_t)e;
    }
}

// first position in the sorted keys [0, m) whose key is >= x
__device__ __forceinline__ int64_t adj_lower_bound(const uint64_t *keys, int64_t lo, int64_t hi, uint64_t x)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// off[v] for v in [0, n]: start of v's group of edges (off[n] = 3 F)
__global__ void k_adj_off(const uint64_t *__restrict__ keys, const int64_t *d_n3, int64_t n, int bits,
                          int64_t *__restrict__ off)
{
    const int64_t m = *d_n3;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x)
        off[v] = v == n ? m : adj_lower_bound(keys, 0, m, (uint64_t)v << bits);
}

// the face across every directed edge
__global__ void k_adj_nb(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, const int64_t *d_n3,
                         const int64_t *__restrict__ off, int bits, int32_t *__restrict__ nb, int32_t *status)
{
    const int64_t m = *d_n3;
    const uint64_t mask = (1ull << bits) - 1;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[j];
        if (j > 0 && keys[j - 1] == key) adj_status(status, HULL3D_ERR_NOT_CLOSED);  // an edge held twice
        const int64_t a = (int64_t)(key >> bits), b = (int64_t)(key & mask);
        const uint64_t want = ((uint64_t)b << bits) | (uint64_t)a;
        const int64_t q = adj_lower_bound(keys, off[b], off[b + 1], want);
        const uint32_t e = vals[j];
        if (q >= off[b + 1] || keys[q] != want) {  // no opposite edge
            adj_status(status, HULL3D_ERR_NOT_CLOSED);
            nb[e] = -1;
        } else {
            nb[e] = (int32_t)(vals[q] / 3);
        }
    }
}

// the faces around each vertex, counter-clockwise from its smallest face
__global__ void k_adj_star(const int32_t *__restrict__ faces, const int32_t *__restrict__ nb,
                           const uint32_t *__restrict__ vals, const int64_t *__restrict__ off, int64_t n,
                           int32_t *__restrict__ star, int32_t *status)
{
    if (*status) return;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = off[v], d = off[v + 1] - b;
        if (d == 0) continue;
        uint32_t first = 0xffffffffu;
        for (int64_t i = 0; i < d; i++) first = min(first, vals[b + i] / 3);
        int32_t f = (int32_t)first;
        for (int64_t i = 0; i < d; i++) {
            if (i > 0 && f == (int32_t)first) {  // back too early: more than one cycle of faces around v
                adj_status(status, HULL3D_ERR_NOT_CLOSED);
                break;
            }
            star[b + i] = f;
            const int kv = faces[3 * f] == v ? 0 : faces[3 * f + 1] == v ? 1 : faces[3 * f + 2] == v ? 2 : -1;
            const int32_t g = kv < 0 ? -1 : nb[3 * (int64_t)f + (kv == 0 ? 2 : kv - 1)];
            if (g < 0) {
                adj_status(status, HULL3D_ERR_NOT_CLOSED);
                break;
            }
            f = g;
        }
        if (f != (int32_t)first) adj_status(status, HULL3D_ERR_NOT_CLOSED);  // the walk does not close
    }
}

static unsigned adj_grid(int64_t items, int sms)
{
    const int64_t need = (items + 255) / 256;
    const int64_t cap = 8 * (int64_t)(sms > 0 ? sms : 132);
    return (unsigned)(need < 1 ? 1 : (need < cap ? need : cap));
}

int launch_adjacency(const int32_t *faces, const int64_t *d_nf, int64_t cap, int64_t n, int32_t *nb,
                     int64_t *star_off, int32_t *star, int32_t *status, const AdjScratch &s, int sms,
                     cudaStream_t st, int64_t *launches)
{
    int bits = 1;
    while ((1ll << bits) < n) bits++;
    const int64_t m = 3 * cap;
    k_adj_keys<<<adj_grid(m, sms), 256, 0, st>>>(faces, d_nf, cap, n, bits, s.k0, s.v0, s.n3, status);
    int64_t l = 1;
    const int which = radix_sort_pairs(s.k0, s.v0, s.k1, s.v1, m, s.n3, 2 * bits, s.ss, st, &l);
    const uint64_t *keys = which ? s.k1 : s.k0;
    const uint32_t *vals = which ? s.v1 : s.v0;
    k_adj_off<<<adj_grid(n + 1, sms), 256, 0, st>>>(keys, s.n3, n, bits, star_off);
    k_adj_nb<<<adj_grid(m, sms), 256, 0, st>>>(keys, vals, s.n3, star_off, bits, nb, status);
    k_adj_star<<<adj_grid(n, sms), 256, 0, st>>>(faces, nb, vals, star_off, n, star, status);
    l += 3;
    if (launches) *launches = l;
    return 0;
}

}  // namespace hull3d
