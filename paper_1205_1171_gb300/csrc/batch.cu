// batch.cu -- many independent clouds in one persistent launch.
//
// The bottom-up movie construction of White & Wortman (Sec. 2) for one small
// cloud fits in one CTA's shared memory, so a batch of clouds needs no level
// sequence of launches at all: every CTA of a persistent grid takes clouds
// from an atomic work counter (largest first) and, for each,
//   1. loads it and builds the sort keys (x, z, y) with the range check;
//   2. sorts them by a bitonic network in shared memory, flags duplicates;
//   3. runs every merge level of both passes: one thread per merge while
//      there are many merges, one warp per merge (warp-cooperative event
//      rounds) near the top;
//   4. at the root, writes each face as a canonical key into the cloud's own
//      output rows (used as staging);
//   5. sorts the face keys in shared memory and writes the faces out.
// Clouds are split into size classes (one template instance per class) so
// that small clouds do not reserve a large cloud's shared memory.
#include "internal.h"
#include "merge.cuh"

namespace hull3d {

constexpr int BATCH_THREADS = 128;
// Threads per CTA of a size class: six warps for the largest (two such CTAs
// per SM still fit 168 registers a thread, and the extra warps take the
// merges of its middle levels; batch of 65,536 clouds 435.6 -> 419.9 ms, 256
// threads 433.3 ms at 128 registers), four for the others (more would force
// their four CTAs per SM below 128 registers).
template <int NMAX>
constexpr int batch_threads()
{
    return NMAX >= 4096 ? 192 : BATCH_THREADS;
}

// A cloud lives in shared memory in 26 bytes per point, so that two clouds of
// the largest class share an SM: each point as its 63-bit sort key (the biased
// x, z, y fields) and a 16-bit input index, links as two 16-bit ranks (0xffff
// for none), movie entries as a 15-bit rank with the insertion flag in bit 15.
constexpr unsigned short BNIL = 0xffff;

struct BPts {
    const uint64_t *K;
    const unsigned short *ID;
    __device__ __forceinline__ P3 get(int r) const
    {
        const uint64_t k = K[r];
        const int lo = -(1 << 20);
        return P3{ (int)((k >> 42) & 0x1fffff) + lo, (int)(k & 0x1fffff) + lo, (int)((k >> 21) & 0x1fffff) + lo,
                   (int)ID[r], r };
    }
    __device__ __forceinline__ int rk(int r) const { return r; }
};

// A cloud of at most 4096 points on 2^21 x-values rarely has three points on
// one x, so the batch kernel leaves out the equal-x index tier (its code alone
// cost the 65,536-cloud batch 2%).
template <>
struct EqxTier<BPts> {
    static constexpr bool on = false;
};

// The same points under the float32 predicates of the paper's GPU kernel
// (an ablation: how often float arithmetic gives a wrong hull).
struct BPtsF : BPts {
};
template <>
struct F32Pred<BPtsF> {
    static constexpr bool on = true;
};
template <>
struct EqxTier<BPtsF> {
    static constexpr bool on = false;
};

struct BLinks {
    ushort2 *L;
    __device__ __forceinline__ static int un(unsigned short v) { return v == BNIL ? NIL : (int)v; }
    __device__ __forceinline__ static unsigned short pk(int v) { return v < 0 ? BNIL : (unsigned short)v; }
    __device__ __forceinline__ int2 get(int r) const
    {
        const ushort2 l = L[r];
        return make_int2(un(l.x), un(l.y));
    }
    __device__ __forceinline__ int prv(int r) const { return un(L[r].x); }
    __device__ __forceinline__ int nxt(int r) const { return un(L[r].y); }
    __device__ __forceinline__ void set(int r, int2 v) { L[r] = make_ushort2(pk(v.x), pk(v.y)); }
    __device__ __forceinline__ void set_prv(int r, int v) { L[r].x = pk(v); }
    __device__ __forceinline__ void set_nxt(int r, int v) { L[r].y = pk(v); }
};

__device__ __forceinline__ unsigned bw_un(unsigned short s) { return (unsigned)(s & 0x7fffu) | ((s & 0x8000u) ? INS_BIT : 0u); }
__device__ __forceinline__ unsigned short bw_pk(unsigned w)
{
    return (unsigned short)((w & RANK_MASK) | ((w & INS_BIT) ? 0x8000u : 0u));
}

struct BEvIn {
    const unsigned short *W;
    __device__ __forceinline__ unsigned w(int i) const { return bw_un(W[i]); }
};
struct BEvOut {
    unsigned short *W;
    __device__ __forceinline__ void put(int k, unsigned w, int, int) { W[k] = bw_pk(w); }
    __device__ __forceinline__ unsigned w(int k) const { return bw_un(W[k]); }
};

// Root merge output: each event (a, w, b) is a face; it is oriented (lower
// faces face down, upper faces up), rotated min-first and written as the key
// f0 << 26 | f1 << 13 | f2 (local indices below 2^13), staged as two 32-bit
// halves in the cloud's output rows (which are only 4-byte aligned).
struct FaceKeyOut {
    BPts P;
    unsigned *keys;
    int base;
    bool upper;
    __device__ __forceinline__ void put(int k, unsigned w, int a, int b)
    {
        const int wi = (int)(w & RANK_MASK);
        const P3 A = P.get(a), W = P.get(wi), B = P.get(b);
        const bool up = turn_sign(A, W, B) > 0;
        int f0 = A.id, f1, f2;
        if (up == upper) { f1 = W.id; f2 = B.id; } else { f1 = B.id; f2 = W.id; }
        if (f1 < f0 && f1 < f2) { int t = f0; f0 = f1; f1 = f2; f2 = t; }
        else if (f2 < f0 && f2 < f1) { int t = f2; f2 = f1; f1 = f0; f0 = t; }
        const uint64_t key = ((uint64_t)f0 << 26) | ((uint64_t)f1 << 13) | (uint64_t)f2;
        keys[2 * (base + k)] = (unsigned)key;
        keys[2 * (base + k) + 1] = (unsigned)(key >> 32);
    }
    __device__ __forceinline__ unsigned w(int) const { return 0; }
};

// Bitonic sort of m (a power of two) keys with a 16-bit payload.
__device__ void bitonic_kv(uint64_t *k, unsigned short *v, int m)
{
    for (int size = 2; size <= m; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (m >> 1); t += blockDim.x) {
                const int i = 2 * t - (t & (stride - 1));
                const int j = i + stride;
                const bool asc = (i & size) == 0;
                if ((k[i] > k[j]) == asc) {
                    uint64_t tk = k[i]; k[i] = k[j]; k[j] = tk;
                    if (v) { unsigned short tv = v[i]; v[i] = v[j]; v[j] = tv; }
                }
            }
            __syncthreads();
        }
}

__device__ __forceinline__ int pow2_at_least(int x)
{
    int m = 1;
    while (m < x) m <<= 1;
    return m;
}

// Shared memory per class, 26 bytes per point: the points (sort keys, sorted
// in place with their input indices), the links, and region A with the two
// movie buffers (2 NMAX entries each) and their counts.  After the last merge
// the face keys are sorted over the whole of it.
template <int NMAX>
struct BatchSmem {
    static constexpr size_t K_OFF = 0;                    // uint64 [NMAX]
    static constexpr size_t ID_OFF = 8 * (size_t)NMAX;    // uint16 [NMAX]
    static constexpr size_t LK_OFF = 10 * (size_t)NMAX;   // ushort2 [NMAX]
    static constexpr size_t A_OFF = 14 * (size_t)NMAX;    // uint16 [2 NMAX] x 2, uint16 [NMAX] x 2
    static constexpr size_t bytes = 26 * (size_t)NMAX;
    static_assert(16 * NMAX <= 26 * NMAX, "face keys: at most 2 NMAX of 8 bytes");
};

// CTAs of a class that fit in an SM's 228 KB of shared memory (at most 4):
// the register cap follows, so a class that cannot have more resident CTAs
// does not pay for a tighter cap with spills.
template <int NMAX>
constexpr int batch_ctas_per_sm()
{
    return (int)((233472 / (BatchSmem<NMAX>::bytes + 1024)) < 4 ? (233472 / (BatchSmem<NMAX>::bytes + 1024)) : 4);
}

template <int NMAX, class PTS>
__global__ void __launch_bounds__(batch_threads<NMAX>(), batch_ctas_per_sm<NMAX>()) k_batch(const int32_t *__restrict__ xyz,
                                                         const int64_t *__restrict__ off,
                                                         const int64_t *__restrict__ foff,
                                                         const int32_t *__restrict__ order, int count, int *counter,
                                                         int32_t *faces, int64_t *nfaces, int32_t *status,
                                                         int warp_nodes)
{
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ int s_cloud, s_err, s_kl;
    uint64_t *K = (uint64_t *)(bsm + BatchSmem<NMAX>::K_OFF);
    unsigned short *ID = (unsigned short *)(bsm + BatchSmem<NMAX>::ID_OFF);
    ushort2 *LK = (ushort2 *)(bsm + BatchSmem<NMAX>::LK_OFF);
    unsigned char *regA = bsm + BatchSmem<NMAX>::A_OFF;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) s_cloud = atomicAdd(counter, 1);
        __syncthreads();
        const int slot = s_cloud;
        __syncthreads();
        if (slot >= count) return;
        const int b = order[slot];
        const int64_t o = off[b];
        const int n = (int)(off[b + 1] - o);
        int32_t *fout = faces + 3 * foff[b];
        unsigned *fkeys = (unsigned *)fout;  // staging: 2n - 4 rows of 12 bytes hold 2n - 4 keys of 8
        if (tid == 0) s_err = 0;
        __syncthreads();
        // 1. keys
        const int m = pow2_at_least(n);
        unsigned short *V = ID;
        for (int i = tid; i < m; i += blockDim.x) {
            if (i < n) {
                const int x = xyz[3 * (o + i)], y = xyz[3 * (o + i) + 1], z = xyz[3 * (o + i) + 2];
                const int lo = -(1 << 20), hi = (1 << 20) - 1;
                if (x < lo || x > hi || y < lo || y > hi || z < lo || z > hi) s_err = HULL3D_ERR_COORD_RANGE;
                K[i] = ((uint64_t)((x - lo) & 0x1fffff) << 42) | ((uint64_t)((z - lo) & 0x1fffff) << 21) |
                       (uint64_t)((y - lo) & 0x1fffff);
                V[i] = (unsigned short)i;
            } else {
                K[i] = ~0ull;
                V[i] = 0xffff;
            }
        }
        __syncthreads();
        // 2. sort in place (the sorted keys are the points), duplicates
        bitonic_kv(K, V, m);
        for (int i = tid; i < n; i += blockDim.x)
            if (i > 0 && K[i - 1] == K[i]) s_err = HULL3D_ERR_DUPLICATE;
        __syncthreads();
        int nf = 0;
        if (!s_err && n >= 3) {
            // 3. merge levels; region A now holds the movie buffers and counts
            unsigned short *W0 = (unsigned short *)regA, *W1 = W0 + 2 * NMAX;
            unsigned short *C0 = W1 + 2 * NMAX, *C1 = C0 + NMAX;
            int L = 0;
            while ((1 << L) < n) L++;
            PTS sp_;
            sp_.K = K;
            sp_.ID = ID;
            const PTS &sp = sp_;
            BLinks lk{ LK };
            for (int pass = 0; pass < 2; pass++) {
                const bool upper = pass != 0;
                for (int i = tid; i < n; i += blockDim.x) {
                    LK[i] = make_ushort2(BNIL, BNIL);
                    C0[i] = 0;
                }
                __syncthreads();
                for (int level = 1; level <= L; level++) {
                    unsigned short *Wsrc = (level & 1) ? W0 : W1, *Wdst = (level & 1) ? W1 : W0;
                    unsigned short *Csrc = (level & 1) ? C0 : C1, *Cdst = (level & 1) ? C1 : C0;
                    const int half = 1 << (level - 1);
                    const int nodes = (n + 2 * half - 1) / (2 * half);
                    const bool root = level == L;
                    if (nodes >= warp_nodes) {  // one thread per merge
                        for (int t = tid; t < nodes; t += blockDim.x) {
                            const int llo = t * 2 * half, lmid = llo + half, lhi = min(llo + 2 * half, n);
                            if (lmid >= lhi) {
                                const int c = Csrc[llo];
                                for (int e = 0; e < c; e++) Wdst[2 * llo + e] = Wsrc[2 * llo + e];
                                Cdst[llo] = (unsigned short)c;
                                continue;
                            }
                            BEvIn Lm{ Wsrc + 2 * llo }, Rm{ Wsrc + 2 * lmid };
                            BEvOut out{ Wdst + 2 * llo };
                            int err = 0;
                            const int k = kinetic_merge(sp, lk, lmid - 1, lmid, lmid, Lm, Csrc[llo], Rm, Csrc[lmid],
                                                        out, 2 * (lhi - llo), upper, &err);
                            Cdst[llo] = (unsigned short)k;
                            if (err) s_err = HULL3D_ERR_INTERNAL;
                        }
                    } else {  // one warp per merge, warp-cooperative rounds
                        for (int t = warp; t < nodes; t += batch_threads<NMAX>() / 32) {
                            const int llo = t * 2 * half, lmid = llo + half, lhi = min(llo + 2 * half, n);
                            if (lmid >= lhi) {
                                const int c = Csrc[llo];
                                for (int e = lane; e < c; e += 32) Wdst[2 * llo + e] = Wsrc[2 * llo + e];
                                if (lane == 0) Cdst[llo] = (unsigned short)c;
                                continue;
                            }
                            BEvIn Lm{ Wsrc + 2 * llo }, Rm{ Wsrc + 2 * lmid };
                            int u = lmid - 1, v = lmid;
                            if (lane == 0) bridge_walk(sp, lk, u, v, (const Tri *)nullptr, upper);
                            u = __shfl_sync(0xffffffffu, u, 0);
                            v = __shfl_sync(0xffffffffu, v, 0);
                            Tri none;
                            none.p = none.q = none.r = -2;
                            none.s = 0;
                            int err = 0;
                            if (root) {
                                const int base = pass ? s_kl : 0;
                                FaceKeyOut fo{ sp, fkeys, base, upper };
                                // the staging rows hold 12 (2n - 4) bytes = 3n - 6 keys of 8 bytes
                                const int room = 3 * n - 6 - base > 0 ? 3 * n - 6 - base : 0;
                                const int k = kinetic_forward_warp(sp, lk, u, v, none, false, Lm, Csrc[llo], Rm,
                                                                   Csrc[lmid], fo, room, upper, false, &err);
                                if (lane == 0) {
                                    if (pass == 0) s_kl = k;
                                    else Cdst[llo] = (unsigned short)k;  // upper count
                                }
                            } else {
                                BEvOut out{ Wdst + 2 * llo };
                                const int k = kinetic_forward_warp(sp, lk, u, v, none, false, Lm, Csrc[llo], Rm,
                                                                   Csrc[lmid], out, 2 * (lhi - llo), upper, false,
                                                                   &err);
                                if (lane == 0) {
                                    if (!err) kinetic_backward(sp, lk, u, v, lmid, out, k);
                                    Cdst[llo] = (unsigned short)k;
                                }
                            }
                            if (err && lane == 0) s_err = HULL3D_ERR_INTERNAL;
                            __syncwarp();
                        }
                    }
                    __syncthreads();
                }
            }
            nf = s_kl + ((L & 1) ? C1 : C0)[0];
            if (nf > 2 * n - 4) s_err = HULL3D_ERR_INTERNAL;
            __syncthreads();
            // 5. canonical order: sort the face keys (over the whole shared region,
            // the points and links being no longer needed) and write the faces
            if (!s_err) {
                uint64_t *FK = (uint64_t *)bsm;
                const int mf = pow2_at_least(nf);
                for (int i = tid; i < mf; i += blockDim.x)
                    FK[i] = i < nf ? ((uint64_t)fkeys[2 * i + 1] << 32) | fkeys[2 * i] : ~0ull;
                __syncthreads();
                bitonic_kv(FK, nullptr, mf);
                for (int i = tid; i < nf; i += blockDim.x) {
                    const uint64_t k = FK[i];
                    fout[3 * i] = (int32_t)(k >> 26);
                    fout[3 * i + 1] = (int32_t)((k >> 13) & 0x1fff);
                    fout[3 * i + 2] = (int32_t)(k & 0x1fff);
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            status[b] = s_err;
            nfaces[b] = s_err ? 0 : nf;
        }
        __syncthreads();
    }
}

template <int NMAX, class PTS>
static void launch_class(const int32_t *xyz, const int64_t *off, const int64_t *foff, const int32_t *order, int count,
                         int *counter, int32_t *faces, int64_t *nfaces, int32_t *status, int sms, int warp_nodes,
                         cudaStream_t st)
{
    if (count <= 0) return;
    const size_t smem = BatchSmem<NMAX>::bytes;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<NMAX, PTS>, batch_threads<NMAX>(), smem);
    if (per_sm < 1) per_sm = 1;
    int grid = sms * per_sm;
    if (grid > count) grid = count;
    k_batch<NMAX, PTS><<<grid, batch_threads<NMAX>(), smem, st>>>(xyz, off, foff, order, count, counter, faces,
                                                                  nfaces, status, warp_nodes);
}

template <class PTS>
static void batch_attributes()
{
    cudaFuncSetAttribute(k_batch<256, PTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BatchSmem<256>::bytes);
    cudaFuncSetAttribute(k_batch<1024, PTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BatchSmem<1024>::bytes);
    cudaFuncSetAttribute(k_batch<2048, PTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BatchSmem<2048>::bytes);
    cudaFuncSetAttribute(k_batch<4096, PTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BatchSmem<4096>::bytes);
}

void batch_kernel_attributes()
{
    batch_attributes<BPts>();
    batch_attributes<BPtsF>();
}

int batch_class_limit(int c) { return c == 0 ? 256 : c == 1 ? 1024 : c == 2 ? 2048 : 4096; }

template <class PTS>
static void launch_batch_pts(int c, const int32_t *xyz, const int64_t *off, const int64_t *foff, const int32_t *order,
                             int count, int *counter, int32_t *faces, int64_t *nfaces, int32_t *status, int sms,
                             int w, cudaStream_t st)
{
    if (c == 0) launch_class<256, PTS>(xyz, off, foff, order, count, counter, faces, nfaces, status, sms, w, st);
    else if (c == 1) launch_class<1024, PTS>(xyz, off, foff, order, count, counter, faces, nfaces, status, sms, w, st);
    else if (c == 2) launch_class<2048, PTS>(xyz, off, foff, order, count, counter, faces, nfaces, status, sms, w, st);
    else launch_class<4096, PTS>(xyz, off, foff, order, count, counter, faces, nfaces, status, sms, w, st);
}

void launch_batch_class(int c, const int32_t *xyz, const int64_t *off, const int64_t *foff, const int32_t *order,
                        int count, int *counter, int32_t *faces, int64_t *nfaces, int32_t *status, int sms,
                        int warp_nodes, bool f32, cudaStream_t st)
{
    if (f32)
        launch_batch_pts<BPtsF>(c, xyz, off, foff, order, count, counter, faces, nfaces, status, sms, warp_nodes, st);
    else
        launch_batch_pts<BPts>(c, xyz, off, foff, order, count, counter, faces, nfaces, status, sms, warp_nodes, st);
}

}  // namespace hull3d
