// merge.cuh -- one kinetic movie merge (White & Wortman, Sec. 2 "merge step"; the
// act() and time() figures of Sec. 3), templated over where the points, links
// and event lists live (global memory, a CTA's shared memory, or a compacted
// slot table).
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
//
// The event loop is written for a small instruction footprint: the six
// candidates live in a short array walked by non-unrolled loops with one call
// site for the time comparison (unrolling it overflowed the instruction cache).
#pragma once
#include "predicates.cuh"

namespace hull3d {

constexpr int NIL = -1;
constexpr unsigned INS_BIT = 0x80000000u;
constexpr unsigned RANK_MASK = 0x7fffffffu;

// A candidate event: a triple of point indices with its normal N = (q-p) x (r-p)
// cached as Z = -N.y, Y = N.z and Nx = N.x, and s = sign(Y~).
struct Tri {
    int p, q, r;
    int s;  // 0: a member is NIL (time +inf)
    long long Z, Y, Nx;
    float tf;  // Z / Y in float (NaN when Y = 0): the filter of tri_cmp
};

// Filter of the time comparison.  tf = fl(fl(Z) / fl(Y)) with the fast
// division (__fdividef, at most 2 ulp off for |Y| < 2^126; here |Y| < 2^49):
// the two conversions round to nearest, so |tf - Z/Y| < 2^-21 |Z/Y|.  When
// fl(tf_a - tf_b) exceeds 2^-19 (|tf_a| + |tf_b|) the true difference of the
// times has its sign, and the exact products are not needed; nearer times
// (and every tie) go to the exact tiers.
constexpr float TF_MARGIN = 1.0f / 524288.0f;

// Whether the triples of points of type PT carry tf and tri_cmp tries the
// filter first.  Where most comparisons tie in Z/Y (triples through points of
// equal x: the lowest merge levels of clouds with several points per x-value)
// the filter only adds work; a point type opts out by specialising this.
template <class PT>
struct TimeFilter {
    static constexpr bool on = true;
};

// Whether the predicates for points of type PT are the float32 arithmetic of
// the paper's GPU kernel (cl_float coordinates, Sec. 3) instead of the exact
// perturbed ones: an ablation only, whose results need not be a hull.  A
// point type opts in by specialising this.
template <class PT>
struct F32Pred {
    static constexpr bool on = false;
};

__device__ __forceinline__ int sgnf(float v) { return (v > 0.f) - (v < 0.f); }

template <class PT>
__device__ __forceinline__ void tri_make(const PT &pt, Tri &t, int p, int q, int r)
{
    t.p = p; t.q = q; t.r = r;
    if ((p | q | r) < 0) { t.s = 0; return; }
    P3 P = pt.get(p), Q = pt.get(q), R = pt.get(r);
    if constexpr (F32Pred<PT>::on) {
        // the time of the triple as the float quotient Z / Y of float cross
        // products; Y == 0 (collinear in the -infinity view) has no event
        const float ax = (float)Q.x - (float)P.x, ay = (float)Q.y - (float)P.y, az = (float)Q.z - (float)P.z;
        const float bx = (float)R.x - (float)P.x, by = (float)R.y - (float)P.y, bz = (float)R.z - (float)P.z;
        const float Z = ax * bz - bx * az, Y = ax * by - bx * ay;
        t.s = sgnf(Y);
        t.Z = (long long)__float_as_uint(t.s ? Z / Y : 0.f);
        t.Y = t.Nx = 0;
        t.tf = __uint_as_float(0x7fc00000u);
        return;
    }
    long long ax = Q.x - P.x, ay = Q.y - P.y, az = Q.z - P.z;
    long long bx = R.x - P.x, by = R.y - P.y, bz = R.z - P.z;
    t.Z = ax * bz - bx * az;
    t.Y = ax * by - bx * ay;
    t.Nx = ay * bz - az * by;
    if constexpr (TimeFilter<PT>::on) t.tf = t.Y ? __fdividef((float)t.Z, (float)t.Y) : __uint_as_float(0x7fc00000u);
    // sign(Y~) = first nonzero of (N.z, -N.x, -N.y), else the eta tier
    if (t.Y) t.s = sgn64(t.Y);
    else if (t.Nx) t.s = -sgn64(t.Nx);
    else if (t.Z) t.s = sgn64(t.Z);  // -N.y = Z
    else t.s = turn_slow(P, Q, R);
}

// Whether tri_cmp gives two triples that each lie on one x-value their own
// index-tier comparison (time_cmp_eqx) for points of type PT.  A point type
// opts out by specialising this; the general index tier gives the same sign.
template <class PT>
struct EqxTier {
    static constexpr bool on = true;
};

// sign(t(a) - t(b)) in the pass's time direction, both finite: the
// unperturbed value, then the tie tiers in the perturbation's order (equal
// triples; the shear terms -c.z and -c.y; the index tiers).  At 2^24 points on
// 2^21 x-values, triples through equal-x pairs tie often, so every tier is
// inline: a call would make the caller save its registers to local memory.
template <class PT>
__device__ __forceinline__ int tri_cmp(const PT &pt, const Tri &a, const Tri &b, bool upper)
{
    int s;
    if constexpr (F32Pred<PT>::on) {  // float times, equal times compare equal
        const float ta = __uint_as_float((unsigned)a.Z), tb = __uint_as_float((unsigned)b.Z);
        s = (ta > tb) - (ta < tb);
        return upper ? -s : s;
    }
    if constexpr (TimeFilter<PT>::on) {
        // both Y nonzero: sign(D0) a.s b.s is the sign of Z_a/Y_a - Z_b/Y_b
        const float df = a.tf - b.tf;
        if (fabsf(df) > TF_MARGIN * (fabsf(a.tf) + fabsf(b.tf))) {  // false for NaN
            s = df > 0.f ? 1 : -1;
            return upper ? -s : s;
        }
    }
    const i128 D0 = (i128)a.Z * b.Y - (i128)b.Z * a.Y;
    if (D0 != 0) s = sgn128(D0) * a.s * b.s;
    else if (a.p == b.p && a.q == b.q && a.r == b.r) s = 0;
    else {
        const i128 cz = (i128)a.Z * b.Nx - (i128)a.Nx * b.Z;
        if (cz != 0) s = -sgn128(cz) * a.s * b.s;
        else {
            const i128 cy = (i128)a.Y * b.Nx - (i128)a.Nx * b.Y;
            if (cy != 0) s = -sgn128(cy) * a.s * b.s;
            else if (EqxTier<PT>::on && (a.Z | a.Y | b.Z | b.Y) == 0 && a.Nx != 0 && b.Nx != 0)  // one x each
                s = time_cmp_eqx(pt, a.p, a.q, a.r, b.p, b.q, b.r, a.Nx, b.Nx, a.s * b.s);
            else s = time_cmp_index(pt, a.p, a.q, a.r, b.p, b.q, b.r, a.s * b.s);
        }
    }
    return upper ? -s : s;
}

template <class PT>
__device__ __forceinline__ int turn3(const PT &pt, int p, int q, int r)
{
    if constexpr (F32Pred<PT>::on) {  // float cross product of the (x, y) projection
        const P3 P = pt.get(p), Q = pt.get(q), R = pt.get(r);
        const float ax = (float)Q.x - (float)P.x, ay = (float)Q.y - (float)P.y;
        const float bx = (float)R.x - (float)P.x, by = (float)R.y - (float)P.y;
        return sgnf(ax * by - bx * ay);
    }
    return turn_sign(pt.get(p), pt.get(q), pt.get(r));
}

// act(): insert w between its stored neighbours if it is not linked in, else unlink it.
template <class LK>
__device__ __forceinline__ void act(LK &lk, int w)
{
    int2 lw = lk.get(w);
    if (lk.nxt(lw.x) != w) {
        lk.set_nxt(lw.x, w);
        lk.set_prv(lw.y, w);
    } else {
        lk.set_nxt(lw.x, lw.y);
        lk.set_prv(lw.y, lw.x);
    }
}

// Points are addressed by an index that is either the rank itself or a slot
// of a compacted table; pt.rk(i) gives the rank (the perturbed x-order).

// Orientation of (p, q, r) just after the event `at` in the pass's time
// frame (at == nullptr: t = -infinity): sign(Y~) times the sign of
// (time(p, q, r) - time(at)), the kinetic turn Z~ - t Y~ = Y~ (t_pqr - t).
template <class PT>
__device__ __forceinline__ int turn_after(const PT &pt, int p, int q, int r, const Tri *at, bool upper)
{
    if (!at) return turn3(pt, p, q, r);
    Tri t;
    tri_make(pt, t, p, q, r);
    return tri_cmp(pt, t, *at, upper) > 0 ? t.s : -t.s;
}

// The bridge of the two child hulls just after `at`: walks in from the inner
// x-extremes u (left) and v (right); u only moves left and v only right.
template <class PT, class LK>
__device__ void bridge_walk(const PT &pt, const LK &lk, int &u, int &v, const Tri *at, bool upper)
{
    for (;;) {
        int vn = lk.nxt(v);
        if (vn != NIL && turn_after(pt, u, v, vn, at, upper) < 0) { v = vn; continue; }
        int up = lk.prv(u);
        if (up != NIL && turn_after(pt, up, u, v, at, upper) < 0) { u = up; continue; }
        break;
    }
}

// Forward pass (step 2) from the bridge (u, v), after the event `old` when
// have_old.  Consumes the child movies (L, nl) and (R, nr) and appends the
// visible events to `out`.  With stop_at_end it stops once both child movies
// are consumed (a time window that does not reach t = +infinity).  Returns
// the number of events written; u and v are left at the final bridge.
template <class PT, class LK, class EIN, class EOUT>
__device__ int kinetic_forward(const PT &pt, LK &lk, int &u, int &v, Tri old, bool have_old, const EIN &L, int nl,
                               const EIN &R, int nr, EOUT &out, int cap, bool upper, bool stop_at_end, int *err)
{
    Tri c[6];
    unsigned valid = 0;  // bit l: candidate l is finite and later than the last event
#pragma unroll
    for (int l = 0; l < 6; l++) { c[l].p = c[l].q = c[l].r = -2; c[l].s = 0; }
    int i = 0, j = 0, k = 0;
    for (;;) {
        if (stop_at_end && i >= nl && j >= nr) break;
        const int e0 = i < nl ? (int)(L.w(i) & RANK_MASK) : NIL;
        const int e1 = j < nr ? (int)(R.w(j) & RANK_MASK) : NIL;
        const int2 l0 = e0 >= 0 ? lk.get(e0) : make_int2(NIL, NIL);
        const int2 l1 = e1 >= 0 ? lk.get(e1) : make_int2(NIL, NIL);
        const int2 lu = lk.get(u), lv = lk.get(v);
        // refresh the candidates whose triple changed; an unchanged candidate
        // keeps its validity (it was later than the previous event, hence
        // later than the one just taken, which had a different triple).  The
        // changed ones are collected first, so that threads of a warp working
        // on different merges rebuild only their own.
        //   0: next event of the left child   1: next event of the right child
        //   2: u advances to u.next           3: u retreats to u.prev
        //   4: v retreats to v.prev           5: v advances to v.next
        auto trip = [&](int l, int &tp, int &tq, int &tr) {
            tp = l == 0 ? l0.x : l == 1 ? l1.x : l == 3 ? lu.x : u;
            tq = l == 0 ? e0 : l == 1 ? e1 : l == 2 ? lu.y : l == 3 ? u : l == 4 ? lv.x : v;
            tr = l == 0 ? l0.y : l == 1 ? l1.y : l == 5 ? lv.y : v;
        };
        unsigned chg = 0;
#pragma unroll
        for (int l = 0; l < 6; l++) {
            int tp, tq, tr;
            trip(l, tp, tq, tr);
            if (tp != c[l].p || tq != c[l].q || tr != c[l].r) chg |= 1u << l;
        }
        while (chg) {
            const int l = __ffs(chg) - 1;
            chg &= chg - 1;
            int tp, tq, tr;
            trip(l, tp, tq, tr);
            tri_make(pt, c[l], tp, tq, tr);
            bool ok = c[l].s != 0 && (!have_old || tri_cmp(pt, c[l], old, upper) > 0);
            valid = ok ? (valid | (1u << l)) : (valid & ~(1u << l));
        }
        int best = -1;
#pragma unroll 1
        for (int l = 0; l < 6; l++)
            if (((valid >> l) & 1u) && (best < 0 || tri_cmp(pt, c[l], c[best], upper) < 0)) best = l;
        if (best < 0) break;
        if (k >= cap) { *err = 1; return cap; }
        const Tri t = c[best];
        // apply the event (its triple t is: left neighbour, point, right neighbour)
        if (best <= 1) {
            const int e = t.q;
            bool vis;
            if (best == 0) { i++; vis = pt.rk(e) < pt.rk(u); }
            else { j++; vis = pt.rk(e) > pt.rk(v); }
            if (vis) out.put(k++, (unsigned)e | (lk.nxt(t.p) != e ? INS_BIT : 0u), t.p, t.r);
            act(lk, e);
        } else {
            // bridge events: c2 and c4 insert the new bridge end, c3 and c5 delete the old one
            const bool ins = (best == 2) | (best == 4);
            out.put(k++, (unsigned)t.q | (ins ? INS_BIT : 0u), t.p, t.r);
            if (best == 2) u = t.q;
            else if (best == 3) u = t.p;
            else if (best == 4) v = t.q;
            else v = t.r;
        }
        old = t;
        have_old = true;
        valid &= ~(1u << best);
    }
    return k;
}

// The same forward pass with the six candidates in a CTA's shared memory
// instead of a per-thread array.  The loop indexes the candidates at run
// time, so an array lives in local memory, and with hundreds of resident
// threads per SM those accesses miss L1 and become most of the kernel's
// memory traffic; a shared-memory slice per thread, field-major so that the
// threads of a warp hit distinct banks, keeps them on chip.
struct CandSmem {
    int *I;        // [5][6][T]: p, q, r, s, tf (bits)
    long long *Q;  // [3][6][T]: Z, Y, Nx
    int T, t;
    __device__ __forceinline__ int &fi(int f, int l) const { return I[(f * 6 + l) * T + t]; }
    __device__ __forceinline__ long long &fq(int f, int l) const { return Q[(f * 6 + l) * T + t]; }
    template <bool TF>
    __device__ __forceinline__ Tri get(int l) const
    {
        Tri x;
        x.p = fi(0, l); x.q = fi(1, l); x.r = fi(2, l); x.s = fi(3, l);
        if constexpr (TF) x.tf = __int_as_float(fi(4, l));
        x.Z = fq(0, l); x.Y = fq(1, l); x.Nx = fq(2, l);
        return x;
    }
    template <bool TF>
    __device__ __forceinline__ void set(int l, const Tri &x) const
    {
        fi(0, l) = x.p; fi(1, l) = x.q; fi(2, l) = x.r; fi(3, l) = x.s;
        if constexpr (TF) fi(4, l) = __float_as_int(x.tf);
        fq(0, l) = x.Z; fq(1, l) = x.Y; fq(2, l) = x.Nx;
    }
};
// shared-memory bytes of CandSmem for a CTA of T threads (tf: with the float
// filter's field)
constexpr int cand_smem_bytes(int T, bool tf = true) { return T * 6 * ((tf ? 5 : 4) * 4 + 3 * 8); }

template <class PT, class LK, class EIN, class EOUT>
__device__ int kinetic_forward_sm(const PT &pt, LK &lk, int &u, int &v, const EIN &L, int nl, const EIN &R, int nr,
                                  EOUT &out, int cap, bool upper, int *err, const CandSmem &c)
{
    unsigned valid = 0;  // bit l: candidate l is finite and later than the last event
#pragma unroll
    for (int l = 0; l < 6; l++) c.fi(0, l) = c.fi(1, l) = c.fi(2, l) = -2;  // no triple yet
    Tri old;
    old.p = old.q = old.r = -2;
    bool have_old = false;
    int i = 0, j = 0, k = 0;
    for (;;) {
        const int e0 = i < nl ? (int)(L.w(i) & RANK_MASK) : NIL;
        const int e1 = j < nr ? (int)(R.w(j) & RANK_MASK) : NIL;
        const int2 l0 = e0 >= 0 ? lk.get(e0) : make_int2(NIL, NIL);
        const int2 l1 = e1 >= 0 ? lk.get(e1) : make_int2(NIL, NIL);
        const int2 lu = lk.get(u), lv = lk.get(v);
        // refresh the candidates whose triple changed (as in kinetic_forward).
        // Each lane first collects its changed candidates in a mask and then
        // rebuilds only those: the threads of a warp, each on its own merge,
        // change different candidates, and a loop over the six fixed slots
        // would make the warp rebuild every slot some lane needs.
        auto trip = [&](int l, int &tp, int &tq, int &tr) {
            tp = l == 0 ? l0.x : l == 1 ? l1.x : l == 3 ? lu.x : u;
            tq = l == 0 ? e0 : l == 1 ? e1 : l == 2 ? lu.y : l == 3 ? u : l == 4 ? lv.x : v;
            tr = l == 0 ? l0.y : l == 1 ? l1.y : l == 5 ? lv.y : v;
        };
        unsigned chg = 0;
#pragma unroll
        for (int l = 0; l < 6; l++) {
            int tp, tq, tr;
            trip(l, tp, tq, tr);
            if (tp != c.fi(0, l) || tq != c.fi(1, l) || tr != c.fi(2, l)) chg |= 1u << l;
        }
        while (chg) {
            const int l = __ffs(chg) - 1;
            chg &= chg - 1;
            int tp, tq, tr;
            trip(l, tp, tq, tr);
            if (tp == old.p && tq == old.q && tr == old.r) {
                // the reverse of the bridge move just applied: the same triple
                // as the last event, never strictly after it.  Only its
                // triple is kept (for the change test); it stays invalid
                // until its triple changes, which rebuilds it.
                c.fi(0, l) = tp; c.fi(1, l) = tq; c.fi(2, l) = tr;
                valid &= ~(1u << l);
                continue;
            }
            Tri t;
            tri_make(pt, t, tp, tq, tr);
            c.template set<TimeFilter<PT>::on>(l, t);
            // a child's next event changes only right after an event of that
            // child was taken (act rewrites links inside one child only), and
            // a child's movie is in time order: it is always later than the
            // last event, so only the bridge moves need the comparison
            bool ok = t.s != 0 && (l <= 1 || !have_old || tri_cmp(pt, t, old, upper) > 0);
            valid = ok ? (valid | (1u << l)) : (valid & ~(1u << l));
        }
        int best = -1;
        Tri t;
#pragma unroll 1
        for (int l = 0; l < 6; l++) {
            if (!((valid >> l) & 1u)) continue;
            const Tri cl = c.template get<TimeFilter<PT>::on>(l);
            if (best < 0 || tri_cmp(pt, cl, t, upper) < 0) { best = l; t = cl; }
        }
        if (best < 0) break;
        if (k >= cap) { *err = 1; return cap; }
        if (best <= 1) {
            const int e = t.q;
            bool vis;
            if (best == 0) { i++; vis = pt.rk(e) < pt.rk(u); }
            else { j++; vis = pt.rk(e) > pt.rk(v); }
            if (vis) out.put(k++, (unsigned)e | (lk.nxt(t.p) != e ? INS_BIT : 0u), t.p, t.r);
            act(lk, e);
        } else {
            const bool ins = (best == 2) | (best == 4);
            out.put(k++, (unsigned)t.q | (ins ? INS_BIT : 0u), t.p, t.r);
            if (best == 2) u = t.q;
            else if (best == 3) u = t.p;
            else if (best == 4) v = t.q;
            else v = t.r;
        }
        old = t;
        have_old = true;
        valid &= ~(1u << best);
    }
    return k;
}

#ifdef __CUDACC__
__device__ __forceinline__ Tri shfl_tri(const Tri &t, int src, unsigned mask = 0xffffffffu)
{
    Tri r;
    r.p = __shfl_sync(mask, t.p, src);
    r.q = __shfl_sync(mask, t.q, src);
    r.r = __shfl_sync(mask, t.r, src);
    r.s = __shfl_sync(mask, t.s, src);
    r.Z = __shfl_sync(mask, t.Z, src);
    r.Y = __shfl_sync(mask, t.Y, src);
    r.Nx = __shfl_sync(mask, t.Nx, src);
    r.tf = __shfl_sync(mask, t.tf, src);
    return r;
}

// Warp-cooperative forward pass: the same loop as kinetic_forward, entered
// by all 32 lanes with identical arguments.  Lane l < 6 owns candidate l and
// refreshes it in parallel with the others; a three-step shuffle reduction
// finds the earliest valid candidate; lane 0 applies the event to the shared
// links and the output while every lane advances the (identical) loop state.
template <class PT, class LK, class EIN, class EOUT>
__device__ int kinetic_forward_warp(const PT &pt, LK &lk, int &u, int &v, Tri old, bool have_old, const EIN &L,
                                    int nl, const EIN &R, int nr, EOUT &out, int cap, bool upper, bool stop_at_end,
                                    int *err)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    Tri c;
    c.p = c.q = c.r = -2;
    c.s = 0;
    bool valid = false;
    int i = 0, j = 0, k = 0;
    for (;;) {
        if (stop_at_end && i >= nl && j >= nr) break;
        // every lane reads the same few links (broadcast loads, no branch per
        // candidate), then lane l < 6 picks its triple
        const int e0 = i < nl ? (int)(L.w(i) & RANK_MASK) : NIL;
        const int e1 = j < nr ? (int)(R.w(j) & RANK_MASK) : NIL;
        const int2 lu = lk.get(u), lv = lk.get(v);
        const int2 l0 = e0 >= 0 ? lk.get(e0) : make_int2(NIL, NIL);
        const int2 l1 = e1 >= 0 ? lk.get(e1) : make_int2(NIL, NIL);
        if (lane < 6) {
            const int tp = lane == 0 ? l0.x : lane == 1 ? l1.x : lane == 3 ? lu.x : u;
            const int tq = lane == 0 ? e0 : lane == 1 ? e1 : lane == 2 ? lu.y : lane == 3 ? u : lane == 4 ? lv.x : v;
            const int tr = lane == 0 ? l0.y : lane == 1 ? l1.y : lane == 5 ? lv.y : v;
            if (tp != c.p || tq != c.q || tr != c.r) {
                tri_make(pt, c, tp, tq, tr);
                // a child's next event is always later than the last event
                // (its movie is in time order and it changes only after one of
                // its events was taken): only the bridge moves are compared
                valid = c.s != 0 && (lane <= 1 || !have_old || tri_cmp(pt, c, old, upper) > 0);
            }
        }
        // all 15 pairs at once: lane k < 15 compares candidates (i, j) = pair k;
        // the earliest valid candidate is the one that beats the other five
        // (equal triples: the lower index wins, as in the serial scan)
        const int pk = lane < 15 ? lane : 0;
        const int pi = pk < 5 ? 0 : pk < 9 ? 1 : pk < 12 ? 2 : pk < 14 ? 3 : 4;
        const int pj = pk - (pi == 0 ? -1 : pi == 1 ? 3 : pi == 2 ? 6 : pi == 3 ? 8 : 9);
        const bool vi = __shfl_sync(FULL, valid, pi) != 0, vj = __shfl_sync(FULL, valid, pj) != 0;
        bool ibeats;
        if constexpr (TimeFilter<PT>::on) {
            // the float times first; the whole triples move only when some
            // pair is too close for them to decide
            const float fi = __shfl_sync(FULL, c.tf, pi), fj = __shfl_sync(FULL, c.tf, pj);
            const float df = fi - fj;
            int dec = fabsf(df) > TF_MARGIN * (fabsf(fi) + fabsf(fj)) ? (df > 0.f ? 1 : -1) : 0;  // 0: NaN or near
            if (upper) dec = -dec;
            const bool both = lane < 15 && vi && vj;
            if (__any_sync(FULL, both && dec == 0)) {
                const Tri ti = shfl_tri(c, pi), tj = shfl_tri(c, pj);
                ibeats = lane < 15 && vi && (!vj || (dec != 0 ? dec < 0 : tri_cmp(pt, ti, tj, upper) <= 0));
            } else {
                ibeats = lane < 15 && vi && (!vj || dec < 0);
            }
        } else {
            const Tri ti = shfl_tri(c, pi), tj = shfl_tri(c, pj);
            ibeats = lane < 15 && vi && (!vj || tri_cmp(pt, ti, tj, upper) <= 0);
        }
        const unsigned win = __ballot_sync(FULL, ibeats);
        const unsigned vmask = __ballot_sync(FULL, lane < 6 && valid) & 0x3fu;
        int best = -1;
        if (vmask) {
            // pair bits where candidate x is the first (I) or second (J) member
            constexpr unsigned IM[6] = { 0x001fu, 0x01e0u, 0x0e00u, 0x3000u, 0x4000u, 0x0000u };
            constexpr unsigned JM[6] = { 0x0000u, 0x0001u, 0x0022u, 0x0244u, 0x1488u, 0x6910u };
#pragma unroll
            for (int x = 0; x < 6; x++)
                if (((vmask >> x) & 1u) && (win & IM[x]) == IM[x] && (win & JM[x]) == 0) best = x;
        }
        if (best < 0) break;
        const Tri t = shfl_tri(c, best);
        if (k >= cap) { *err = 1; return cap; }
        if (best <= 1) {
            const int e = t.q;
            const bool vis = best == 0 ? pt.rk(e) < pt.rk(u) : pt.rk(e) > pt.rk(v);
            if (best == 0) i++; else j++;
            if (lane == 0) {
                if (vis) out.put(k, (unsigned)e | (lk.nxt(t.p) != e ? INS_BIT : 0u), t.p, t.r);
                act(lk, e);
            }
            k += vis ? 1 : 0;
        } else {
            const bool ins = (best == 2) | (best == 4);
            if (lane == 0) out.put(k, (unsigned)t.q | (ins ? INS_BIT : 0u), t.p, t.r);
            k++;
            if (best == 2) u = t.q;
            else if (best == 3) u = t.p;
            else if (best == 4) v = t.q;
            else v = t.r;
        }
        __syncwarp();
        old = t;
        have_old = true;
        if (lane == best) valid = false;
    }
    return k;
}

// Warp-parallel version of bridge_walk for two chains stored as consecutive
// slots (left chain ends at slot u, right chain starts at slot v, lengths
// given by u_first and v_last): each step tests 32 consecutive chain links at
// once and jumps to the first one that stops the serial walk, so it ends at
// the serial walk's bridge.
template <class PT>
__device__ void bridge_walk_warp(const PT &pt, int u_first, int v_last, int &u, int &v, const Tri *at, bool upper)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (;;) {
        // advance v while (u, v, v.next) turns right, 32 links per step
        for (;;) {
            const int a = v + lane;
            const bool right = a + 1 <= v_last && turn_after(pt, u, a, a + 1, at, upper) < 0;
            const unsigned bal = __ballot_sync(FULL, right);
            const int run = bal == FULL ? 32 : __ffs(~bal) - 1;  // consecutive right turns from v
            v += run;
            if (run < 32) break;
        }
        // then move u back one step if (u.prev, u, v) turns right, and retry v
        if (u > u_first && turn_after(pt, u - 1, u, v, at, upper) < 0) {
            u -= 1;
            continue;
        }
        break;
    }
}
#endif

// Backward pass (step 3): from the t = +infinity bridge (u, v) undo the
// parent's k events in reverse, leaving the parent's t = -infinity hull and
// the event-time links of its event points.
template <class PT, class LK, class EOUT>
__device__ void kinetic_backward(const PT &pt, LK &lk, int u, int v, int mid, const EOUT &out, int k)
{
    lk.set_nxt(u, v);
    lk.set_prv(v, u);
    for (int kk = k - 1; kk >= 0; kk--) {
        int w = (int)(out.w(kk) & RANK_MASK);
        const int rw = pt.rk(w);
        if (rw <= pt.rk(u) || rw >= pt.rk(v)) {
            act(lk, w);
            if (w == u) u = lk.prv(u);
            else if (w == v) v = lk.nxt(v);
        } else {
            lk.set_nxt(u, w);
            lk.set(w, make_int2(u, v));
            lk.set_prv(v, w);
            if (rw < mid) u = w; else v = w;
        }
    }
}

// The whole merge of one node.  u0 and v0 address the ranks mid - 1 and mid.
// Returns the number of parent events written to `out` (at most cap); on an
// overflow (impossible for valid input) sets *err and returns cap.
template <class PT, class LK, class EIN, class EOUT>
__device__ int kinetic_merge(const PT &pt, LK &lk, int u0, int v0, int mid, const EIN &L, int nl, const EIN &R,
                             int nr, EOUT &out, int cap, bool upper, int *err)
{
    int u = u0, v = v0;
    bridge_walk(pt, lk, u, v, (const Tri *)nullptr, upper);  // 1. bridge at t = -inf
    Tri none;
    none.p = none.q = none.r = -2;
    none.s = 0;
    int k = kinetic_forward(pt, lk, u, v, none, false, L, nl, R, nr, out, cap, upper, false, err);  // 2.
    if (k >= cap && *err) return k;
    kinetic_backward(pt, lk, u, v, mid, out, k);  // 3.
    return k;
}

// kinetic_merge with the candidates of the event loop in shared memory.
template <class PT, class LK, class EIN, class EOUT>
__device__ int kinetic_merge_sm(const PT &pt, LK &lk, int u0, int v0, int mid, const EIN &L, int nl, const EIN &R,
                                int nr, EOUT &out, int cap, bool upper, int *err, const CandSmem &cs)
{
    int u = u0, v = v0;
    bridge_walk(pt, lk, u, v, (const Tri *)nullptr, upper);
    int k = kinetic_forward_sm(pt, lk, u, v, L, nl, R, nr, out, cap, upper, err, cs);
    if (k >= cap && *err) return k;
    kinetic_backward(pt, lk, u, v, mid, out, k);
    return k;
}

// The merge of a level-2 node: ranks r0 .. r0 + m - 1 (m = 3 or 4), children
// the pair (r0, r0 + 1) and the pair (r0 + 2, r0 + 3) (a single point when
// m = 3), linked as such on entry.  A pair's hull is its segment at every
// time, so neither child has an event and of the six candidates of the merge
// step only the two bridge triples remain: (r0, r0 + 1, v) for u stepping
// between r0 and r0 + 1, and (u, r0 + 2, r0 + 3) for v stepping between
// r0 + 2 and r0 + 3.  Same steps and output as kinetic_merge (at most
// 2 m - 5 = 3 events).
template <class PT, class LK, class EOUT>
__device__ int kinetic_merge_pairs(const PT &pt, LK &lk, int r0, int m, EOUT &out, bool upper, int *err)
{
    int u = r0 + 1, v = r0 + 2;
    bridge_walk(pt, lk, u, v, (const Tri *)nullptr, upper);  // 1. bridge at t = -inf
    const bool has3 = m > 3;
    Tri tu, tv, old;
    old.p = old.q = old.r = -2;
    bool have_old = false, vu = false, vv = false, new_u = true, new_v = true;
    int k = 0;
    for (;;) {  // 2. forward pass
        // a triple is rebuilt only when the other bridge end moved; the one
        // just applied stays invalid (its time is the last event's)
        if (new_u) {
            tri_make(pt, tu, r0, r0 + 1, v);
            vu = !have_old || tri_cmp(pt, tu, old, upper) > 0;
            new_u = false;
        }
        if (new_v) {
            vv = false;
            if (has3) {
                tri_make(pt, tv, u, r0 + 2, r0 + 3);
                vv = !have_old || tri_cmp(pt, tv, old, upper) > 0;
            }
            new_v = false;
        }
        const bool take_u = vu && (!vv || tri_cmp(pt, tu, tv, upper) < 0);
        if (!take_u && !vv) break;
        if (k >= 2 * m) { *err = 1; return k; }
        if (take_u) {  // r0 + 1 joins the bridge (u advances) or leaves it (u retreats)
            const bool ins = u == r0;
            out.put(k++, (unsigned)(r0 + 1) | (ins ? INS_BIT : 0u), r0, v);
            u = ins ? r0 + 1 : r0;
            old = tu;
            vu = false;
            new_v = true;
        } else {  // r0 + 2 joins the bridge (v retreats) or leaves it (v advances)
            const bool ins = v == r0 + 3;
            out.put(k++, (unsigned)(r0 + 2) | (ins ? INS_BIT : 0u), u, r0 + 3);
            v = ins ? r0 + 2 : r0 + 3;
            old = tv;
            vv = false;
            new_u = true;
        }
        have_old = true;
    }
    kinetic_backward(pt, lk, u, v, r0 + 2, out, k);  // 3.
    return k;
}

// ---- storage adapters -------------------------------------------------------
// Points are packed as int4 (x, y, z, input index); links as int2 (prev, next).

struct GPts {  // rank-ordered points in global memory
    const int4 *P;
    __device__ __forceinline__ P3 get(int r) const
    {
        int4 p = P[r];
        return P3{ p.x, p.y, p.z, p.w, r };
    }
    __device__ __forceinline__ int rk(int r) const { return r; }
};

// The same points, compared without the float filter.
struct GPtsX : GPts {
};
template <>
struct TimeFilter<GPtsX> {
    static constexpr bool on = false;
};

struct GLinks {
    int2 *L;
    __device__ __forceinline__ int2 get(int r) const { return L[r]; }
    __device__ __forceinline__ int prv(int r) const { return L[r].x; }
    __device__ __forceinline__ int nxt(int r) const { return L[r].y; }
    __device__ __forceinline__ void set(int r, int2 v) { L[r] = v; }
    __device__ __forceinline__ void set_prv(int r, int v) { L[r].x = v; }
    __device__ __forceinline__ void set_nxt(int r, int v) { L[r].y = v; }
};

struct GEvIn {  // a movie in global memory
    const unsigned *W;
    __device__ __forceinline__ unsigned w(int i) const { return W[i]; }
};

struct GEvOut {  // A == nullptr: the neighbours are not kept (no later reader)
    unsigned *W;
    int *A, *B;
    __device__ __forceinline__ void put(int k, unsigned w, int a, int b)
    {
        W[k] = w;
        if (A) { A[k] = a; B[k] = b; }
    }
    __device__ __forceinline__ unsigned w(int k) const { return W[k]; }
};

// Shared-memory variants: arrays hold one block of ranks starting at `base`.
struct SPts {
    const int4 *P;
    int base;
    __device__ __forceinline__ P3 get(int r) const
    {
        int4 p = P[r - base];
        return P3{ p.x, p.y, p.z, p.w, r };
    }
    __device__ __forceinline__ int rk(int r) const { return r; }
};

struct SLinks {
    int2 *L;
    int base;
    __device__ __forceinline__ int2 get(int r) const { return L[r - base]; }
    __device__ __forceinline__ int prv(int r) const { return L[r - base].x; }
    __device__ __forceinline__ int nxt(int r) const { return L[r - base].y; }
    __device__ __forceinline__ void set(int r, int2 v) { L[r - base] = v; }
    __device__ __forceinline__ void set_prv(int r, int v) { L[r - base].x = v; }
    __device__ __forceinline__ void set_nxt(int r, int v) { L[r - base].y = v; }
};

// Compacted table in shared memory: slot -> point, with its rank.
struct CPts {
    const int4 *P;
    const int *RK;
    __device__ __forceinline__ P3 get(int s) const
    {
        int4 p = P[s];
        return P3{ p.x, p.y, p.z, p.w, RK[s] };
    }
    __device__ __forceinline__ int rk(int s) const { return RK[s]; }
};

struct CLinks {  // links between slots
    int2 *L;
    __device__ __forceinline__ int2 get(int s) const { return L[s]; }
    __device__ __forceinline__ int prv(int s) const { return L[s].x; }
    __device__ __forceinline__ int nxt(int s) const { return L[s].y; }
    __device__ __forceinline__ void set(int s, int2 v) { L[s] = v; }
    __device__ __forceinline__ void set_prv(int s, int v) { L[s].x = v; }
    __device__ __forceinline__ void set_nxt(int s, int v) { L[s].y = v; }
};

}  // namespace hull3d
