// multi.cu -- many clouds hulled together, level by level.
//
// Each merge of a level is independent of every other (Sec. 2), so the
// merges of different clouds can share a launch just as those of one cloud
// do.  The clouds of a group get aligned blocks of one rank space (span.cuh):
//   1. keys    every point of the group gets its (x, z, y) key (the perturbed
//              x-order, as for one hull) and its position q in the group;
//   2. sort    a radix sort by the key, then a stable one by cloud, leaves
//              each cloud's points contiguous and in x-order;
//   3. decode  the point of cloud c at sorted position j goes to rank
//              cbase[c] + (j - coff[c]); equal neighbours are duplicates;
//   4. levels  the merge levels of the single-hull pipeline over the whole
//              rank space (enqueue_levels);
//   5. faces   each cloud's root movies (level L_c) give its faces, written
//              compactly after a scan of the per-cloud counts, sorted once by
//              (cloud, a, b) and copied to each cloud's output rows.
// Input errors (a coordinate out of range, a duplicate point) mark only
// their cloud, whose nodes the level kernels then skip.
#include "internal.h"
#include "merge.cuh"

namespace hull3d {

__device__ __forceinline__ void multi_status(int32_t *st, int code) { atomicCAS(st, 0, code); }

// the cloud (layout order) holding sorted position q: coff is nondecreasing, coff[0] = 0
__device__ __forceinline__ int cloud_of(const int64_t *coff, int C, int64_t q)
{
    int lo = 0, hi = C - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (coff[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_multi_keys(const int32_t *__restrict__ xyz, MultiTables t, int C, int64_t total,
                             uint64_t *__restrict__ keys, uint32_t *__restrict__ vals)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int c = cloud_of(t.coff, C, q);
        const int64_t row = t.ioff[c] + (q - t.coff[c]);
        const int x = xyz[3 * row], y = xyz[3 * row + 1], z = xyz[3 * row + 2];
        const int lo = -(1 << 20), hi = (1 << 20) - 1;
        if (x < lo || x > hi || y < lo || y > hi || z < lo || z > hi) multi_status(t.cstat + c, HULL3D_ERR_COORD_RANGE);
        const uint64_t bx = (uint64_t)(x - lo) & 0x1fffff, by = (uint64_t)(y - lo) & 0x1fffff;
        const uint64_t bz = (uint64_t)(z - lo) & 0x1fffff;
        keys[q] = (bx << 42) | (bz << 21) | by;
        vals[q] = (uint32_t)q;
    }
}

// after the sort by point key: the cloud of each item becomes its key
__global__ void k_multi_cloud_keys(const uint32_t *__restrict__ vals, MultiTables t, int C, int64_t total,
                                   uint64_t *__restrict__ keys2, uint32_t *__restrict__ vals2)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t q = vals[j];
        keys2[j] = (uint64_t)cloud_of(t.coff, C, q);
        vals2[j] = q;
    }
}

__global__ void k_multi_decode(const int32_t *__restrict__ xyz, const uint64_t *__restrict__ keys2,
                               const uint32_t *__restrict__ vals2, MultiTables t, int64_t total, int4 *__restrict__ P)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total; j += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)keys2[j];
        const int64_t q = vals2[j], local = q - t.coff[c];
        const int64_t row = t.ioff[c] + local;
        const int x = xyz[3 * row], y = xyz[3 * row + 1], z = xyz[3 * row + 2];
        P[t.cbase[c] + (j - t.coff[c])] = make_int4(x, y, z, (int)local);
        if (j > t.coff[c]) {  // same cloud, previous in x-order: equal means a duplicate
            const int64_t prow = t.ioff[c] + ((int64_t)vals2[j - 1] - t.coff[c]);
            if (xyz[3 * prow] == x && xyz[3 * prow + 1] == y && xyz[3 * prow + 2] == z)
                multi_status(t.cstat + c, HULL3D_ERR_DUPLICATE);
        }
    }
}

// faces of each cloud: its root movies hold kl (lower) and ku (upper) events
__global__ void k_multi_face_count(MultiTables t, int C, PassBufs p0, PassBufs p1)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        int64_t f = 0;
        if (!t.cstat[c]) {
            const int buf = t.ctop[c] & 1;
            const int64_t base = t.cbase[c], m = t.cend[c] - base;
            f = (int64_t)p0.cnt[buf][base] + p1.cnt[buf][base];
            // a closed triangulated surface on at most m vertices has at most 2m - 4 faces
            if (f > 2 * m - 4) {
                multi_status(t.cstat + c, HULL3D_ERR_INTERNAL);
                f = 0;
            }
        }
        t.fcount[c] = f;
    }
}

// exclusive scan of the face counts (one block): fstart[c], fstart[C] = total
__global__ void k_multi_scan(MultiTables t, int C)
{
    __shared__ int64_t part[1024];
    const int T = blockDim.x, per = (C + T - 1) / T, b = threadIdx.x * per;
    int64_t s = 0;
    for (int i = 0; i < per && b + i < C; i++) s += t.fcount[b + i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int i = 0; i < T; i++) {
            const int64_t v = part[i];
            part[i] = run;
            run += v;
        }
        t.fstart[C] = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int i = 0; i < per && b + i < C; i++) {
        t.fstart[b + i] = run;
        run += t.fcount[b + i];
    }
}

// key (cloud << 2 fbits | a << fbits | b), value c of every face (a, b, c),
// oriented and rotated as for one hull; grid.x strides over clouds, grid.y = pass
__global__ void k_multi_face_keys(Points pts, MultiTables t, int C, PassBufs p0, PassBufs p1, int fbits,
                                  uint64_t *__restrict__ keys, uint32_t *__restrict__ vals)
{
    const bool upper = blockIdx.y != 0;
    const PassBufs &pb = upper ? p1 : p0;
    GPts gp{ pts.P };
    for (int c = blockIdx.x; c < C; c += gridDim.x) {
        if (t.cstat[c] || t.fcount[c] == 0) continue;
        const int buf = t.ctop[c] & 1;
        const int64_t base = t.cbase[c];
        const int kl = p0.cnt[buf][base];
        const int cnt = pb.cnt[buf][base];
        const int64_t o = t.fstart[c] + (upper ? kl : 0);
        const unsigned *W = pb.W[buf] + 2 * base;
        const int *A = pb.A[buf] + 2 * base, *B = pb.B[buf] + 2 * base;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const P3 Pa = gp.get(A[e]), Pw = gp.get((int)(W[e] & RANK_MASK)), Pb = gp.get(B[e]);
            const bool up = turn_sign(Pa, Pw, Pb) > 0;  // lower faces face down, upper faces up
            int f0 = Pa.id, f1, f2;
            if (up == upper) { f1 = Pw.id; f2 = Pb.id; }
            else { f1 = Pb.id; f2 = Pw.id; }
            if (f1 < f0 && f1 < f2) { const int x = f0; f0 = f1; f1 = f2; f2 = x; }
            else if (f2 < f0 && f2 < f1) { const int x = f2; f2 = f1; f1 = f0; f0 = x; }
            keys[o + e] = ((uint64_t)c << (2 * fbits)) | ((uint64_t)f0 << fbits) | (uint64_t)f1;
            vals[o + e] = (uint32_t)f2;
        }
    }
}

__global__ void k_multi_face_out(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, MultiTables t,
                                 int fbits, int32_t *__restrict__ faces)
{
    const int64_t total = t.fstart[t.ncl];
    const uint64_t mask = (1ull << fbits) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        const int c = (int)(k >> (2 * fbits));
        const int64_t row = t.cfoff[c] + (i - t.fstart[c]);
        faces[3 * row] = (int32_t)((k >> fbits) & mask);
        faces[3 * row + 1] = (int32_t)(k & mask);
        faces[3 * row + 2] = (int32_t)vals[i];
    }
}

// per cloud: its face count and status in the caller's arrays (batch order)
__global__ void k_multi_finish(MultiTables t, int C, const int32_t *status, int64_t *nfaces, int32_t *cstatus)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        const int b = t.corig[c];
        const int s = t.cstat[c] ? t.cstat[c] : *status;
        cstatus[b] = s;
        nfaces[b] = s ? 0 : t.fcount[c];
    }
}

static unsigned multi_grid(int64_t items, int sms)
{
    const int64_t need = (items + 255) / 256;
    const int64_t cap = 8 * (int64_t)(sms > 0 ? sms : 132);
    return (unsigned)(need < 1 ? 1 : (need < cap ? need : cap));
}

int launch_multi_sort(const int32_t *xyz, const MultiTables &t, int C, int64_t total, int4 *P, uint64_t *k0,
                      uint32_t *v0, uint64_t *k1, uint32_t *v1, const SortScratch &ss, int sms, cudaStream_t st,
                      int64_t *launches)
{
    k_multi_keys<<<multi_grid(total, sms), 256, 0, st>>>(xyz, t, C, total, k0, v0);
    int which = radix_sort_pairs(k0, v0, k1, v1, total, nullptr, 63, ss, st, launches);
    uint64_t *ka = which ? k1 : k0, *kb = which ? k0 : k1;
    uint32_t *va = which ? v1 : v0, *vb = which ? v0 : v1;
    k_multi_cloud_keys<<<multi_grid(total, sms), 256, 0, st>>>(va, t, C, total, kb, vb);
    int cbits = 1;
    while ((1ll << cbits) < C) cbits++;
    // (kb, vb) -> sorted by cloud, stable
    which = radix_sort_pairs(kb, vb, ka, va, total, nullptr, cbits, ss, st, launches);
    const uint64_t *keys2 = which ? ka : kb;
    const uint32_t *vals2 = which ? va : vb;
    k_multi_decode<<<multi_grid(total, sms), 256, 0, st>>>(xyz, keys2, vals2, t, total, P);
    *launches += 3;
    return 0;
}

int launch_multi_faces(const Points &pts, const MultiTables &t, int C, int fbits, PassBufs *passes, uint64_t *k0,
                       uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t cap, const SortScratch &ss,
                       const int32_t *status, int32_t *faces, int64_t *nfaces, int32_t *cstatus, int sms,
                       cudaStream_t st, int64_t *launches)
{
    const unsigned cg = (unsigned)((C + 255) / 256);
    k_multi_face_count<<<cg, 256, 0, st>>>(t, C, passes[0], passes[1]);
    k_multi_scan<<<1, 1024, 0, st>>>(t, C);
    const unsigned fg = (unsigned)(C < 4096 ? C : 4096);
    k_multi_face_keys<<<dim3(fg, 2), 256, 0, st>>>(pts, t, C, passes[0], passes[1], fbits, k0, v0);
    int cbits = 1;
    while ((1ll << cbits) < C) cbits++;
    const int which = radix_sort_pairs(k0, v0, k1, v1, cap, t.fstart + C, cbits + 2 * fbits, ss, st, launches);
    k_multi_face_out<<<multi_grid(cap, sms), 256, 0, st>>>(which ? k1 : k0, which ? v1 : v0, t, fbits, faces);
    k_multi_finish<<<cg, 256, 0, st>>>(t, C, status, nfaces, cstatus);
    *launches += 6;
    return 0;
}

}  // namespace hull3d
