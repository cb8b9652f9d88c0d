// merge.cu -- the bottom-up merge levels (White & Wortman, Sec. 2 "movie array";
// Sec. 3 main loop and kernel index math) and the face emission.
//
// Layout (one pass; the lower and upper passes have separate copies):
//   links prv/nxt[rank]                      in-place, as in the paper's P[].prev/next
//   event buffers W/A/B[2][2n]               ping-pong per level (the paper's A and B)
//   counts cnt[2][n]                         movie length, indexed by the node's first rank
// The node of level l with first rank lo covers [lo, min(lo + 2^l, n)); its
// movie occupies entries [2 lo, 2 lo + 2 m) of buffer (l & 1) (the paper's
// eventListOffset = 2 * leftGroupIndex).  Nodes of one level touch disjoint
// rank ranges, so the in-place link updates never race.
#include "internal.h"
#include "merge.cuh"

namespace hull3d {

__device__ __forceinline__ void set_status2(int32_t *status, int code) { atomicCAS(status, 0, code); }

// ---------------------------------------------------------------------------
// Level 1: pairs.  A pair's hull is its segment at every time: no events.
// ---------------------------------------------------------------------------
__global__ void k_level1(int64_t n, PassBufs p0, PassBufs p1, int32_t *status)
{
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const bool up = blockIdx.y != 0;
    int *prv = up ? p1.prv : p0.prv, *nxt = up ? p1.nxt : p0.nxt, *cnt = up ? p1.cnt[1] : p0.cnt[1];
    if ((r & 1) == 0) {
        prv[r] = NIL;
        nxt[r] = (r + 1 < n) ? (int)(r + 1) : NIL;
        cnt[r] = 0;
    } else {
        prv[r] = (int)(r - 1);
        nxt[r] = NIL;
    }
}

void launch_level1(int64_t n, PassBufs *passes, int npass, int32_t *status, cudaStream_t st)
{
    dim3 g((unsigned)((n + 255) / 256), npass);
    k_level1<<<g, 256, 0, st>>>(n, passes[0], passes[npass - 1], status);
}

// ---------------------------------------------------------------------------
// One level in global memory, one thread per merge.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_level(Points pts, int64_t n, int level, PassBufs p0, PassBufs p1,
                                               int32_t *status)
{
    if (*status) return;
    int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t lo = node << level;
    if (lo >= n) return;
    const bool upper = blockIdx.y != 0;
    const int src = (level - 1) & 1, dst = level & 1;
    const int64_t half = 1ll << (level - 1);
    const int64_t mid = lo + half, hi = (lo + 2 * half < n) ? lo + 2 * half : n;
    if (mid >= hi) return;  // pass-through nodes are copied by k_passthrough
    const int *csrc = upper ? p1.cnt[src] : p0.cnt[src];
    int *cdst = upper ? p1.cnt[dst] : p0.cnt[dst];
    const unsigned *Wsrc = upper ? p1.W[src] : p0.W[src];
    unsigned *Wdst = upper ? p1.W[dst] : p0.W[dst];
    int *Adst = upper ? p1.A[dst] : p0.A[dst], *Bdst = upper ? p1.B[dst] : p0.B[dst];
    int nl = csrc[lo], nr = csrc[mid];
    GPts gp{ pts.X, pts.Y, pts.Z, pts.ID };
    GLinks lk{ upper ? p1.prv : p0.prv, upper ? p1.nxt : p0.nxt };
    GEvIn L{ Wsrc + 2 * lo }, R{ Wsrc + 2 * mid };
    GEvOut out{ Wdst + 2 * lo, Adst + 2 * lo, Bdst + 2 * lo };
    int err = 0;
    int k = kinetic_merge(gp, lk, (int)mid, L, nl, R, nr, out, (int)(2 * (hi - lo)), upper, &err);
    cdst[lo] = k;
    if (err) set_status2(status, HULL3D_ERR_INTERNAL);
}

// The last node of a level may have no right child: its movie is the child's.
__global__ void k_passthrough(int64_t lo, int level, PassBufs p0, PassBufs p1, int32_t *status)
{
    if (*status) return;
    const bool up = blockIdx.y != 0;
    const int src = (level - 1) & 1, dst = level & 1;
    const unsigned *Ws = up ? p1.W[src] : p0.W[src];
    const int *As = up ? p1.A[src] : p0.A[src], *Bs = up ? p1.B[src] : p0.B[src];
    unsigned *Wd = up ? p1.W[dst] : p0.W[dst];
    int *Ad = up ? p1.A[dst] : p0.A[dst], *Bd = up ? p1.B[dst] : p0.B[dst];
    int c = (up ? p1.cnt[src] : p0.cnt[src])[lo];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < c; e += (int64_t)gridDim.x * blockDim.x) {
        Wd[2 * lo + e] = Ws[2 * lo + e];
        Ad[2 * lo + e] = As[2 * lo + e];
        Bd[2 * lo + e] = Bs[2 * lo + e];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) (up ? p1.cnt[dst] : p0.cnt[dst])[lo] = c;
}

void launch_level(const Points &pts, int64_t n, int level, PassBufs *passes, int npass, int32_t *status,
                  cudaStream_t st)
{
    int64_t nodes = (n + (1ll << level) - 1) >> level;
    dim3 g((unsigned)((nodes + 127) / 128), npass);
    k_level<<<g, 128, 0, st>>>(pts, n, level, passes[0], passes[npass - 1], status);
    int64_t lo = (nodes - 1) << level;
    if (lo + (1ll << (level - 1)) >= n) {
        int64_t cap = 2 * (n - lo);
        unsigned blocks = (unsigned)((cap + 255) / 256);
        if (blocks > 1024) blocks = 1024;
        k_passthrough<<<dim3(blocks, npass), 256, 0, st>>>(lo, level, passes[0], passes[npass - 1], status);
    }
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
    int *sX = sm, *sY = sX + Bcap, *sZ = sY + Bcap, *sID = sZ + Bcap;
    int *sP = sID + Bcap, *sN = sP + Bcap;
    unsigned *sW0 = (unsigned *)(sN + Bcap), *sW1 = sW0 + 2 * Bcap;
    int *sC0 = (int *)(sW1 + 2 * Bcap), *sC1 = sC0 + Bcap;
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        sX[i] = pts.X[base + i]; sY[i] = pts.Y[base + i]; sZ[i] = pts.Z[base + i]; sID[i] = pts.ID[base + i];
    }
    SPts sp{ sX, sY, sZ, sID, (int)base };
    SLinks lk{ sP, sN, (int)base };
    int err = 0;
    for (int pass = 0; pass < npass; pass++) {
        const bool upper = pass != 0;
        unsigned *gW = upper ? p1.W[l1 & 1] : p0.W[l1 & 1];
        int *gA = upper ? p1.A[l1 & 1] : p0.A[l1 & 1], *gB = upper ? p1.B[l1 & 1] : p0.B[l1 & 1];
        int *gcnt = upper ? p1.cnt[l1 & 1] : p0.cnt[l1 & 1];
        int *gprv = upper ? p1.prv : p0.prv, *gnxt = upper ? p1.nxt : p0.nxt;
        __syncthreads();
        for (int i = threadIdx.x; i < B; i += blockDim.x) { sP[i] = NIL; sN[i] = NIL; sC0[i] = 0; }
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
                    k = kinetic_merge(sp, lk, (int)(base + lmid), L, Csrc[llo], R, Csrc[lmid], out,
                                      2 * (lhi - llo), upper, &err);
                } else {
                    SEvOut out{ Wdst + 2 * llo };
                    k = kinetic_merge(sp, lk, (int)(base + lmid), L, Csrc[llo], R, Csrc[lmid], out,
                                      2 * (lhi - llo), upper, &err);
                }
                Cdst[llo] = k;
            }
            __syncthreads();
        }
        // write back links and the level-l1 count of this block's node
        int *Cfin = (top & 1) ? sC1 : sC0;
        for (int i = threadIdx.x; i < B; i += blockDim.x) { gprv[base + i] = sP[i]; gnxt[base + i] = sN[i]; }
        if (threadIdx.x == 0) gcnt[base] = Cfin[0];
    }
    if (err) set_status2(status, HULL3D_ERR_INTERNAL);
}

size_t fused_smem_bytes(int l1) { return (size_t)(1 << l1) * sizeof(int) * 12; }

void launch_fused(const Points &pts, int64_t n, int l0, int l1, PassBufs *passes, int npass, int32_t *status,
                  cudaStream_t st)
{
    (void)l0;
    int64_t blocks = (n + (1ll << l1) - 1) >> l1;
    size_t smem = fused_smem_bytes(l1);
    // the attribute is per kernel: raise it once to the largest depth's need
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem_bytes(10));
        attr_set = true;
    }
    k_fused<<<(unsigned)blocks, FUSED_THREADS, smem, st>>>(pts, n, l1, passes[0], passes[npass - 1], npass, status);
}

// ---------------------------------------------------------------------------
// Faces: each root event (a, w, b) is one face (Sec. 2: one event per face).
// ---------------------------------------------------------------------------
__global__ void k_face_keys(Points pts, int64_t n, int level, PassBufs p0, PassBufs p1, int fbits, uint64_t *keys,
                            uint32_t *vals, int64_t *d_nfaces, int32_t *status)
{
    const int buf = level & 1;
    const int kl = p0.cnt[buf][0], ku = p1.cnt[buf][0];
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // a closed triangulated surface on at most n vertices has at most 2n - 4 faces
    const bool bad = (int64_t)kl + ku > 2 * n - 4;
    if (e == 0) {
        if (bad) set_status2(status, HULL3D_ERR_INTERNAL);
        *d_nfaces = (*status || bad) ? 0 : (int64_t)kl + ku;
    }
    if (*status || bad) return;
    const bool upper = blockIdx.y != 0;
    if (e >= (upper ? ku : kl)) return;
    const unsigned *W_ = upper ? p1.W[buf] : p0.W[buf];
    const int *A_ = upper ? p1.A[buf] : p0.A[buf], *B_ = upper ? p1.B[buf] : p0.B[buf];
    int w = (int)(W_[e] & RANK_MASK), a = A_[e], b = B_[e];
    GPts gp{ pts.X, pts.Y, pts.Z, pts.ID };
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

void launch_face_keys(const Points &pts, int64_t n, int level, PassBufs *passes, uint64_t *keys, uint32_t *vals,
                      int64_t *d_nfaces, int32_t *status, cudaStream_t st)
{
    int fbits = 1;
    while ((1ll << fbits) < n) fbits++;
    int64_t cap = 2 * n;
    dim3 g((unsigned)((cap + 255) / 256), 2);
    k_face_keys<<<g, 256, 0, st>>>(pts, n, level, passes[0], passes[1], fbits, keys, vals, d_nfaces, status);
}

__global__ void k_face_out(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int fbits,
                           const int64_t *d_nfaces, int32_t *__restrict__ faces)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= *d_nfaces) return;
    uint64_t k = keys[i];
    faces[3 * i] = (int32_t)(k >> fbits);
    faces[3 * i + 1] = (int32_t)(k & ((1ull << fbits) - 1));
    faces[3 * i + 2] = (int32_t)vals[i];
}

void launch_face_out(const uint64_t *keys, const uint32_t *vals, int64_t cap, int fbits, const int64_t *d_nfaces,
                          int32_t *faces, cudaStream_t st)
{
    k_face_out<<<(unsigned)((cap + 255) / 256), 256, 0, st>>>(keys, vals, fbits, d_nfaces, faces);
}

}  // namespace hull3d
