// merge.cuh -- one kinetic movie merge (White & Wortman, Sec. 2 "merge step"; the
// act() and time() figures of Sec. 3), templated over where the points, links
// and event lists live (global memory or a CTA's shared memory).
//
// A node covers the ranks [lo, hi) with children [lo, mid) and [mid, hi).  On
// entry the links hold both children's t = -inf hulls and every child event
// point's links are its neighbours at its event; the children's movies are
// (L, nl) and (R, nr).  The merge
//   1. finds the t = -inf bridge (u, v) by walking in from the inner x-extremes;
//   2. repeatedly takes the earliest of six candidate events strictly after the
//      last one -- the next event of either child, or one of the four bridge
//      moves (u -> u.next, u -> u.prev, v -> v.prev, v -> v.next) -- appends it
//      to the parent movie when it is visible there, and applies it;
//   3. walks the parent movie backwards from the t = +inf bridge to restore the
//      parent's t = -inf hull and the event-time links of its event points.
// Each output event records the event point (bit 31 set for an insertion) and
// its left/right neighbours at the event, i.e. one face of the node's hull.
#pragma once
#include "predicates.cuh"

namespace hull3d {

constexpr int NIL = -1;
constexpr unsigned INS_BIT = 0x80000000u;
constexpr unsigned RANK_MASK = 0x7fffffffu;

// A candidate event: a triple of ranks with its cached Z, Y and sign(Y~).
struct Tri {
    int p, q, r;
    long long Z, Y;
    int s;
    bool fin;  // false: a member is NIL (time +inf)
};

template <class PT>
__device__ __forceinline__ void tri_make(const PT &pt, Tri &t, int p, int q, int r)
{
    t.p = p; t.q = q; t.r = r;
    t.fin = (p >= 0) & (q >= 0) & (r >= 0);
    if (!t.fin) return;
    P3 P = pt.get(p), Q = pt.get(q), R = pt.get(r);
    zy3(P, Q, R, t.Z, t.Y);
    t.s = t.Y ? sgn64(t.Y) : turn_slow(P, Q, R);
}

// sign(t(a) - t(b)) in the pass's time direction, both finite.
template <class PT>
__device__ __forceinline__ int tri_cmp(const PT &pt, const Tri &a, const Tri &b, bool upper)
{
    i128 D0 = (i128)a.Z * b.Y - (i128)b.Z * a.Y;
    int s;
    if (D0 != 0) {
        s = sgn128(D0) * a.s * b.s;
    } else if (a.p == b.p && a.q == b.q && a.r == b.r) {
        s = 0;
    } else {
        P3 A[3] = { pt.get(a.p), pt.get(a.q), pt.get(a.r) };
        P3 B[3] = { pt.get(b.p), pt.get(b.q), pt.get(b.r) };
        s = time_cmp_slow(A, B, a.s, b.s);
    }
    return upper ? -s : s;
}

template <class PT>
__device__ __forceinline__ int turn3(const PT &pt, int p, int q, int r)
{
    return turn_sign(pt.get(p), pt.get(q), pt.get(r));
}

// act(): insert w between its stored neighbours if it is not linked in, else unlink it.
template <class LK>
__device__ __forceinline__ void act(LK &lk, int w)
{
    int pw = lk.prv(w), nw = lk.nxt(w);
    if (lk.nxt(pw) != w) {
        lk.set_nxt(pw, w);
        lk.set_prv(nw, w);
    } else {
        lk.set_nxt(pw, nw);
        lk.set_prv(nw, pw);
    }
}

// Returns the number of parent events written to `out` (at most cap); on an
// overflow (impossible for valid input) sets *err and returns cap.
template <class PT, class LK, class EIN, class EOUT>
__device__ int kinetic_merge(const PT &pt, LK &lk, int mid, const EIN &L, int nl, const EIN &R, int nr, EOUT &out,
                             int cap, bool upper, int *err)
{
    // 1. bridge at t = -inf; u only moves left and v only right, so this ends
    int u = mid - 1, v = mid;
    for (;;) {
        int vn = lk.nxt(v);
        if (vn != NIL && turn3(pt, u, v, vn) < 0) { v = vn; continue; }
        int up = lk.prv(u);
        if (up != NIL && turn3(pt, up, u, v) < 0) { u = up; continue; }
        break;
    }

    // 2. forward pass
    Tri c[6];
    bool valid[6];
#pragma unroll
    for (int l = 0; l < 6; l++) { c[l].p = c[l].q = c[l].r = -2; c[l].fin = false; valid[l] = false; }
    Tri old;
    bool have_old = false;
    int i = 0, j = 0, k = 0;
    for (;;) {
        int tp[6], tq[6], tr[6];
        if (i < nl) { int e = (int)(L.w(i) & RANK_MASK); tp[0] = lk.prv(e); tq[0] = e; tr[0] = lk.nxt(e); }
        else { tp[0] = tq[0] = tr[0] = NIL; }
        if (j < nr) { int e = (int)(R.w(j) & RANK_MASK); tp[1] = lk.prv(e); tq[1] = e; tr[1] = lk.nxt(e); }
        else { tp[1] = tq[1] = tr[1] = NIL; }
        int un = lk.nxt(u), upv = lk.prv(u), vp = lk.prv(v), vn = lk.nxt(v);
        tp[2] = u;   tq[2] = un; tr[2] = v;
        tp[3] = upv; tq[3] = u;  tr[3] = v;
        tp[4] = u;   tq[4] = vp; tr[4] = v;
        tp[5] = u;   tq[5] = v;  tr[5] = vn;
        // refresh the candidates whose triple changed; an unchanged candidate
        // keeps its validity (it was later than the previous event, hence
        // later than the one just taken, which had a different triple)
#pragma unroll
        for (int l = 0; l < 6; l++) {
            if (tp[l] != c[l].p || tq[l] != c[l].q || tr[l] != c[l].r) {
                tri_make(pt, c[l], tp[l], tq[l], tr[l]);
                valid[l] = c[l].fin && (!have_old || tri_cmp(pt, c[l], old, upper) > 0);
            }
        }
        int best = -1;
        Tri bt;
#pragma unroll
        for (int l = 0; l < 6; l++)
            if (valid[l] && (best < 0 || tri_cmp(pt, c[l], bt, upper) < 0)) { best = l; bt = c[l]; }
        if (best < 0) break;
        if (k >= cap) { *err = 1; return cap; }
        switch (best) {
        case 0: {
            int e = tq[0];
            i++;
            if (e < u) out.put(k++, (unsigned)e | (lk.nxt(tp[0]) != e ? INS_BIT : 0u), tp[0], tr[0]);
            act(lk, e);
            break;
        }
        case 1: {
            int e = tq[1];
            j++;
            if (e > v) out.put(k++, (unsigned)e | (lk.nxt(tp[1]) != e ? INS_BIT : 0u), tp[1], tr[1]);
            act(lk, e);
            break;
        }
        case 2: out.put(k++, (unsigned)un | INS_BIT, u, v); u = un; break;
        case 3: out.put(k++, (unsigned)u, upv, v); u = upv; break;
        case 4: out.put(k++, (unsigned)vp | INS_BIT, u, v); v = vp; break;
        default: out.put(k++, (unsigned)v, u, vn); v = vn; break;
        }
        old = bt;
        have_old = true;
#pragma unroll
        for (int l = 0; l < 6; l++) valid[l] = valid[l] && (l != best);  // static indices keep c[] in registers
    }

    // 3. backward pass from the t = +inf bridge
    lk.set_nxt(u, v);
    lk.set_prv(v, u);
    for (int kk = k - 1; kk >= 0; kk--) {
        int w = (int)(out.w(kk) & RANK_MASK);
        if (w <= u || w >= v) {
            act(lk, w);
            if (w == u) u = lk.prv(u);
            else if (w == v) v = lk.nxt(v);
        } else {
            lk.set_nxt(u, w); lk.set_prv(w, u);
            lk.set_prv(v, w); lk.set_nxt(w, v);
            if (w < mid) u = w; else v = w;
        }
    }
    return k;
}

// ---- storage adapters -------------------------------------------------------

struct GPts {  // sorted SoA in global memory, indexed by rank
    const int *X, *Y, *Z, *ID;
    __device__ __forceinline__ P3 get(int r) const { return P3{ X[r], Y[r], Z[r], ID[r], r }; }
};

struct GLinks {
    int *P, *N;
    __device__ __forceinline__ int prv(int r) const { return P[r]; }
    __device__ __forceinline__ int nxt(int r) const { return N[r]; }
    __device__ __forceinline__ void set_prv(int r, int v) { P[r] = v; }
    __device__ __forceinline__ void set_nxt(int r, int v) { N[r] = v; }
};

struct GEvIn {  // a movie in global memory
    const unsigned *W;
    __device__ __forceinline__ unsigned w(int i) const { return W[i]; }
};

struct GEvOut {
    unsigned *W;
    int *A, *B;
    __device__ __forceinline__ void put(int k, unsigned w, int a, int b) { W[k] = w; A[k] = a; B[k] = b; }
    __device__ __forceinline__ unsigned w(int k) const { return W[k]; }
};

// Shared-memory variants: arrays hold one block of ranks starting at `base`.
struct SPts {
    const int *X, *Y, *Z, *ID;
    int base;
    __device__ __forceinline__ P3 get(int r) const
    {
        int i = r - base;
        return P3{ X[i], Y[i], Z[i], ID[i], r };
    }
};

struct SLinks {
    int *P, *N;
    int base;
    __device__ __forceinline__ int prv(int r) const { return P[r - base]; }
    __device__ __forceinline__ int nxt(int r) const { return N[r - base]; }
    __device__ __forceinline__ void set_prv(int r, int v) { P[r - base] = v; }
    __device__ __forceinline__ void set_nxt(int r, int v) { N[r - base] = v; }
};

}  // namespace hull3d
