// Host compile of the device merge header, for a CPU regression test (test
// infrastructure; no product code calls it).  The merges of the header hull a
// point set level by level exactly as the device driver orders them (aligned
// blocks, both passes, faces from the root movies):
//   form 0: kinetic_merge, the loop the batch kernel and the serial fallback run;
//   form 1: kinetic_merge_pairs at level 2 and kinetic_merge_sm above it, the
//           loops of the level kernels, with the candidates in a one-thread
//           CandSmem slice and event neighbours kept only at the root and for
//           the last node of each level (the rule of the level kernels when no
//           time windows read them);
// and, from cmp_level on (> 0), the compacted slot-table form of the
// warp-per-merge kernel.  tests/test_merge_header_host.py compares the faces
// with the oracle's.
//
//   int merge_header_hull(const int32_t *xyz, int64_t n, int form, int cmp_level,
//                         int32_t *faces, int64_t *nfaces)
// xyz: n x 3 int32 in [-2^20, 2^20); faces: room for 2n triples.  Returns 0,
// or 2 (range), 3 (duplicate point), 10 + merge error.
#define __device__
#define __forceinline__ inline
#define __noinline__
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

struct int4 {
    int x, y, z, w;
};
struct int2 {
    int x, y;
};
static inline int2 make_int2(int a, int b) { return int2{ a, b }; }
static inline int __ffs(unsigned v) { return __builtin_ffs((int)v); }
static inline unsigned __float_as_uint(float f)
{
    unsigned u;
    std::memcpy(&u, &f, sizeof u);
    return u;
}
static inline float __uint_as_float(unsigned u)
{
    float f;
    std::memcpy(&f, &u, sizeof f);
    return f;
}
static inline float __int_as_float(int i) { return __uint_as_float((unsigned)i); }
static inline int __float_as_int(float f) { return (int)__float_as_uint(f); }
static inline float __fdividef(float a, float b) { return a / b; }

#include "../../paper_1205_1171_gb300/csrc/merge.cuh"

using namespace hull3d;

namespace {

// Output of the compacted form: slots stay for the backward pass, ranks go out.
struct SlotOut {
    unsigned *S, *W;
    int *A, *B;
    const int *RK;
    void put(int k, unsigned w, int a, int b)
    {
        S[k] = w;
        W[k] = (unsigned)RK[w & RANK_MASK] | (w & INS_BIT);
        A[k] = RK[a];
        B[k] = RK[b];
    }
    unsigned w(int k) const { return S[k]; }
};

struct SlotIn {
    const unsigned *W;
    unsigned w(int i) const { return W[i]; }
};

// One merge through a compacted table: the child event points and the four
// x-extremes, each rank once, linked slot to slot; links go back by rank.
int slot_merge(const int4 *P, std::vector<int2> &lk, const unsigned *Lw, int nl, const unsigned *Rw, int nr,
               int64_t lo, int64_t mid, int64_t hi, unsigned *Wd, int *Ad, int *Bd, bool upper, int *err)
{
    const int ex[4] = { (int)lo, (int)mid - 1, (int)mid, (int)hi - 1 };
    std::vector<int> rk;  // slot -> rank
    for (int e = 0; e < 4; e++) rk.push_back(ex[e]);
    for (int i = 0; i < nl; i++) rk.push_back((int)(Lw[i] & RANK_MASK));
    for (int i = 0; i < nr; i++) rk.push_back((int)(Rw[i] & RANK_MASK));
    std::sort(rk.begin(), rk.end());
    rk.erase(std::unique(rk.begin(), rk.end()), rk.end());
    const int ns = (int)rk.size();
    auto slot = [&](int r) -> int {
        if (r < 0) return NIL;
        auto it = std::lower_bound(rk.begin(), rk.end(), r);
        return (it != rk.end() && *it == r) ? (int)(it - rk.begin()) : -2;
    };
    std::vector<int4> sp(ns);
    std::vector<int2> sl(ns);
    for (int s = 0; s < ns; s++) {
        sp[s] = P[rk[s]];
        const int2 l = lk[rk[s]];
        sl[s] = make_int2(slot(l.x), slot(l.y));
        if (sl[s].x == -2 || sl[s].y == -2) { *err = 3; return 0; }  // a link leaves the table
    }
    std::vector<unsigned> in(nl + nr), so(2 * (nl + nr) + 8);
    for (int i = 0; i < nl; i++) in[i] = (unsigned)slot((int)(Lw[i] & RANK_MASK)) | (Lw[i] & INS_BIT);
    for (int i = 0; i < nr; i++) in[nl + i] = (unsigned)slot((int)(Rw[i] & RANK_MASK)) | (Rw[i] & INS_BIT);
    CPts cp{ sp.data(), rk.data() };
    CLinks cl{ sl.data() };
    SlotIn L{ in.data() }, R{ in.data() + nl };
    SlotOut out{ so.data(), Wd, Ad, Bd, rk.data() };
    const int cap = (int)std::min<int64_t>(2 * (hi - lo), (int64_t)so.size());
    const int k = kinetic_merge(cp, cl, slot(ex[1]), slot(ex[2]), (int)mid, L, nl, R, nr, out, cap, upper, err);
    for (int s = 0; s < ns; s++) {
        const int2 l = sl[s];
        lk[rk[s]] = make_int2(l.x < 0 ? NIL : rk[l.x], l.y < 0 ? NIL : rk[l.y]);
    }
    return k;
}

}  // namespace

extern "C" int merge_header_hull(const int32_t *xyz, int64_t n, int form, int cmp_level, int32_t *faces,
                                 int64_t *nfaces)
{
    *nfaces = 0;
    const int bias = 1 << 20;
    std::vector<uint64_t> key(n);
    std::vector<int> idx(n);
    for (int64_t i = 0; i < n; i++) {
        for (int c = 0; c < 3; c++)
            if (xyz[3 * i + c] < -bias || xyz[3 * i + c] >= bias) return 2;
        const uint64_t bx = xyz[3 * i] + bias, by = xyz[3 * i + 1] + bias, bz = xyz[3 * i + 2] + bias;
        key[i] = (bx << 42) | (bz << 21) | by;  // the perturbed x-order: (x, z, y)
        idx[i] = (int)i;
    }
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return key[a] < key[b]; });
    std::vector<int4> P(n);
    for (int64_t r = 0; r < n; r++) {
        const int i = idx[r];
        if (r && key[idx[r - 1]] == key[i]) return 3;
        P[r] = int4{ xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], i };
    }
    if (n < 3) return 0;
    int L = 0;
    while ((1ll << L) < n) L++;
    int fbits = L < 1 ? 1 : L;
    std::vector<uint64_t> fk;
    std::vector<int32_t> fv;
    GPts gp{ P.data() };
    int cand_i[5 * 6];        // CandSmem of one thread: p, q, r, s, tf of six candidates
    long long cand_q[3 * 6];  // and their Z, Y, Nx
    const CandSmem cs{ cand_i, cand_q, 1, 0 };
    for (int pass = 0; pass < 2; pass++) {
        const bool upper = pass != 0;
        std::vector<int2> lk(n, make_int2(NIL, NIL));
        std::vector<unsigned> W[2];
        std::vector<int> A[2], B[2], C[2];
        for (int b = 0; b < 2; b++) {
            W[b].assign(2 * n, 0);
            A[b].assign(2 * n, 0);
            B[b].assign(2 * n, 0);
            C[b].assign(n, 0);
        }
        GLinks gl{ lk.data() };
        for (int level = 1; level <= L; level++) {
            const int src = (level - 1) & 1, dst = level & 1;
            const int64_t half = 1ll << (level - 1);
            for (int64_t lo = 0; lo < n; lo += 2 * half) {
                const int64_t mid = lo + half, hi = std::min<int64_t>(lo + 2 * half, n);
                const int nl = C[src][lo];
                if (mid >= hi) {  // no right child: the movie passes through
                    for (int e = 0; e < nl; e++) {
                        W[dst][2 * lo + e] = W[src][2 * lo + e];
                        A[dst][2 * lo + e] = A[src][2 * lo + e];
                        B[dst][2 * lo + e] = B[src][2 * lo + e];
                    }
                    C[dst][lo] = nl;
                    continue;
                }
                const int nr = C[src][mid];
                int err = 0, k;
                if (cmp_level > 0 && level >= cmp_level) {
                    k = slot_merge(P.data(), lk, W[src].data() + 2 * lo, nl, W[src].data() + 2 * mid, nr, lo, mid,
                                   hi, W[dst].data() + 2 * lo, A[dst].data() + 2 * lo, B[dst].data() + 2 * lo, upper,
                                   &err);
                } else {
                    GEvIn Lv{ W[src].data() + 2 * lo }, Rv{ W[src].data() + 2 * mid };
                    GEvOut out{ W[dst].data() + 2 * lo, A[dst].data() + 2 * lo, B[dst].data() + 2 * lo };
                    if (form == 1 && level < L && hi != n) out.A = out.B = nullptr;  // the level kernel's rule
                    if (form == 1 && level == 2)
                        k = kinetic_merge_pairs(gp, gl, (int)lo, (int)(hi - lo), out, upper, &err);
                    else if (form == 1)
                        k = kinetic_merge_sm(gp, gl, (int)mid - 1, (int)mid, (int)mid, Lv, nl, Rv, nr, out,
                                             (int)(2 * (hi - lo)), upper, &err, cs);
                    else
                        k = kinetic_merge(gp, gl, (int)mid - 1, (int)mid, (int)mid, Lv, nl, Rv, nr, out,
                                          (int)(2 * (hi - lo)), upper, &err);
                }
                if (err) return 10 + err;
                C[dst][lo] = k;
            }
        }
        // one face per root event: (a, w, b) oriented outward, rotated min-first
        const int root = L & 1;
        for (int e = 0; e < C[root][0]; e++) {
            const P3 Ap = gp.get(A[root][e]), Wp = gp.get((int)(W[root][e] & RANK_MASK)), Bp = gp.get(B[root][e]);
            const bool up = turn_sign(Ap, Wp, Bp) > 0;
            int f0 = Ap.id, f1, f2;
            if (up == upper) { f1 = Wp.id; f2 = Bp.id; }
            else { f1 = Bp.id; f2 = Wp.id; }
            if (f1 < f0 && f1 < f2) { const int t = f0; f0 = f1; f1 = f2; f2 = t; }
            else if (f2 < f0 && f2 < f1) { const int t = f2; f2 = f1; f1 = f0; f0 = t; }
            fk.push_back(((uint64_t)f0 << fbits) | (uint64_t)f1);
            fv.push_back(f2);
        }
    }
    std::vector<size_t> o(fk.size());
    for (size_t i = 0; i < o.size(); i++) o[i] = i;
    std::sort(o.begin(), o.end(), [&](size_t a, size_t b) { return fk[a] != fk[b] ? fk[a] < fk[b] : fv[a] < fv[b]; });
    for (size_t i = 0; i < o.size(); i++) {
        faces[3 * i] = (int32_t)(fk[o[i]] >> fbits);
        faces[3 * i + 1] = (int32_t)(fk[o[i]] & ((1ull << fbits) - 1));
        faces[3 * i + 2] = fv[o[i]];
    }
    *nfaces = (int64_t)o.size();
    return 0;
}
