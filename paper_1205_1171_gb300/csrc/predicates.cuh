// predicates.cuh -- exact, perturbed geometric predicates for the kinetic merge.
//
// Kinetic recast (White & Wortman, Sec. 2): at time t the point (x, y, z) sits
// at (x, z - t*y).  For a triple (p, q, r) with N = (q-p) x (r-p):
//   turn at t = -inf       sign(Y),   Y = N.z
//   event time (time())    t = Z / Y, Z = -N.y   (figure "time calculations")
//
// Degeneracies are resolved by the symbolic perturbation
//   x~ = x + a z + a^2 y,  y~ = y + b z + eta_i,  z~ = z + gam_i   (i = input index)
// with a >> b >> gam_0 >> ... >> gam_{n-1} >> eta_0 >> ... >> eta_{n-1}; the sign
// of a predicate is the sign of its largest monomial, monomials ordered
// lexicographically from the smallest variable up.  Expanding by hand:
//   Y~ = N.z - a N.x - b N.y + a^2 b N.x + sum_i eta_i w_i
//   Z~ = -N.y + a^2 N.x + sum_i gam_i w_i
// where, for (p, q, r), w_p = x~_r - x~_q, w_q = x~_p - x~_r, w_r = x~_q - x~_p and
// x~_s - x~_t = dx + a dz + a^2 dy.  sign(x~_s - x~_t) is the rank order.
// The time comparison sign(t1 - t2) = sign(D) sign(Y~1) sign(Y~2) with
// D = Z~1 Y~2 - Z~2 Y~1, whose monomials come in this order:
//   1, a, a^2            : -c.x, -c.z, -c.y with c = N1 x N2
//   gam_i (i ascending)   : (w_i^1 Y~2 - w_i^2 Y~1) without eta, as a polynomial in a, b
//   gam_i eta_j (j, then i): w_i^1 w_j^2 - w_i^2 w_j^1   (reached only if N1 = N2 = 0)
//
// Widths: coordinate differences < 2^21; N components < 2^43 (int64); products
// of two N components or of a difference and an N component < 2^87 (__int128).
#pragma once
#include <stdint.h>

namespace hull3d {

typedef __int128 i128;

struct P3 {
    int x, y, z;  // coordinates
    int id;       // input index (picks gam_id, eta_id)
    int rk;       // rank in the perturbed x-order
};

__device__ __forceinline__ int sgn64(long long v) { return (v > 0) - (v < 0); }
__device__ __forceinline__ int sgn128(i128 v) { return (v > 0) - (v < 0); }

__device__ __forceinline__ void normal3(const P3 &p, const P3 &q, const P3 &r, long long &nx, long long &ny,
                                        long long &nz)
{
    long long ax = q.x - p.x, ay = q.y - p.y, az = q.z - p.z;
    long long bx = r.x - p.x, by = r.y - p.y, bz = r.z - p.z;
    nx = ay * bz - az * by;
    ny = az * bx - ax * bz;
    nz = ax * by - ay * bx;
}

// Z and Y of a triple (the unperturbed numerator and denominator of its time).
__device__ __forceinline__ void zy3(const P3 &p, const P3 &q, const P3 &r, long long &Z, long long &Y)
{
    long long ax = q.x - p.x, ay = q.y - p.y, az = q.z - p.z;
    long long bx = r.x - p.x, by = r.y - p.y, bz = r.z - p.z;
    Z = ax * bz - bx * az;
    Y = ax * by - bx * ay;
}

// sign of Y~(p, q, r): nonzero for distinct points.  Inline: three points with
// equal x (frequent at 2^24 points on 2^21 x-values) reach it in every bridge
// walk over them.
__device__ __forceinline__ int turn_slow(const P3 &p, const P3 &q, const P3 &r)
{
    long long nx, ny, nz;
    normal3(p, q, r, nx, ny, nz);
    if (nz) return sgn64(nz);
    if (nx) return -sgn64(nx);
    if (ny) return -sgn64(ny);
    // collinear in 3D: the eta term of the smallest input index decides
    if (p.id < q.id && p.id < r.id) return (r.rk > q.rk) - (r.rk < q.rk);
    if (q.id < r.id) return (p.rk > r.rk) - (p.rk < r.rk);
    return (q.rk > p.rk) - (q.rk < p.rk);
}

__device__ __forceinline__ int turn_sign(const P3 &p, const P3 &q, const P3 &r)
{
    long long nz = (long long)(q.x - p.x) * (r.y - p.y) - (long long)(r.x - p.x) * (q.y - p.y);
    if (nz) return sgn64(nz);
    return turn_slow(p, q, r);
}

// Coefficients (of 1, a, a^2) of w_id for triple T, zero if id is not in T.
__device__ __forceinline__ void wcoef(const P3 *T, int id, long long w[3])
{
    int k = (T[0].id == id) ? 0 : (T[1].id == id) ? 1 : (T[2].id == id) ? 2 : -1;
    if (k < 0) { w[0] = w[1] = w[2] = 0; return; }
    // w_p = x~_r - x~_q, w_q = x~_p - x~_r, w_r = x~_q - x~_p
    const P3 &s = (k == 0) ? T[2] : (k == 1) ? T[0] : T[1];
    const P3 &t = (k == 0) ? T[1] : (k == 1) ? T[2] : T[0];
    w[0] = (long long)s.x - t.x;
    w[1] = (long long)s.z - t.z;
    w[2] = (long long)s.y - t.y;
}

// Coefficient m of w * (N.z - a N.x - b N.y + a^2 b N.x), monomials in the order
// 1, a, a^2, a^3, a^4, b, ab, a^2b, a^3b, a^4b.
__device__ __forceinline__ i128 wy_coef(const long long w[3], long long nx, long long ny, long long nz, int m)
{
    const long long dx = w[0], dz = w[1], dy = w[2];
    switch (m) {
    case 0: return (i128)dx * nz;
    case 1: return (i128)dz * nz - (i128)dx * nx;
    case 2: return (i128)dy * nz - (i128)dz * nx;
    case 3: return -(i128)dy * nx;
    case 4: return 0;
    case 5: return -(i128)dx * ny;
    case 6: return -(i128)dz * ny;
    case 7: return (i128)dx * nx - (i128)dy * ny;
    case 8: return (i128)dz * nx;
    default: return (i128)dy * nx;
    }
}

// Coefficient of a^m in the product of two w polynomials.
__device__ __forceinline__ long long ww_coef(const long long u[3], const long long v[3], int m)
{
    switch (m) {
    case 0: return u[0] * v[0];
    case 1: return u[0] * v[1] + u[1] * v[0];
    case 2: return u[0] * v[2] + u[1] * v[1] + u[2] * v[0];
    case 3: return u[1] * v[2] + u[2] * v[1];
    default: return u[2] * v[2];
    }
}

// The index tiers of sign(t~(A) - t~(B)) for two triples whose constant, a and
// a^2 coefficients of D vanished (their normals are parallel or zero): the
// gam_i then gam_i eta_j coefficients, indices ascending.  ss = sign(Y~A) sign(Y~B).
// Returns 0 only for equal point sets.  Inlined into the time comparison: at
// 2^24 points on 2^21 x-values, triples of three equal-x points are common and
// compare with each other only here (about half the comparisons of merge
// levels 3-4 on the clipped Gaussian); out of line, every call made the caller
// save its registers to local memory.
template <class PT>
__device__ __forceinline__ int time_cmp_index(PT pt, int a0, int a1, int a2, int b0, int b1, int b2, int ss)
{
    const P3 A[3] = { pt.get(a0), pt.get(a1), pt.get(a2) };
    const P3 B[3] = { pt.get(b0), pt.get(b1), pt.get(b2) };
    {
        int m = 0;
        for (int i = 0; i < 3; i++)
            m += (A[i].id == B[0].id) | (A[i].id == B[1].id) | (A[i].id == B[2].id);
        if (m == 3) return 0;
    }
    long long n1x, n1y, n1z, n2x, n2y, n2z;
    normal3(A[0], A[1], A[2], n1x, n1y, n1z);
    normal3(B[0], B[1], B[2], n2x, n2y, n2z);
    // the input indices involved, ascending, visited by repeated minimum search
    int prev = -1;
    for (int t = 0; t < 6; t++) {
        int id = 0x7fffffff;
        for (int i = 0; i < 3; i++) {
            if (A[i].id > prev && A[i].id < id) id = A[i].id;
            if (B[i].id > prev && B[i].id < id) id = B[i].id;
        }
        if (id == 0x7fffffff) break;
        prev = id;
        long long w1[3], w2[3];
        wcoef(A, id, w1);
        wcoef(B, id, w2);
        for (int m = 0; m < 10; m++) {
            i128 c = wy_coef(w1, n2x, n2y, n2z, m) - wy_coef(w2, n1x, n1y, n1z, m);
            if (c) return sgn128(c) * ss;
        }
    }
    // gam_i eta_j: both triples collinear in 3D; j ascending, then i ascending
    int pj = -1;
    for (int tj = 0; tj < 6; tj++) {
        int jd = 0x7fffffff;
        for (int i = 0; i < 3; i++) {
            if (A[i].id > pj && A[i].id < jd) jd = A[i].id;
            if (B[i].id > pj && B[i].id < jd) jd = B[i].id;
        }
        if (jd == 0x7fffffff) break;
        pj = jd;
        long long u1[3], u2[3];
        wcoef(A, jd, u1);
        wcoef(B, jd, u2);
        int pi = -1;
        for (int ti = 0; ti < 6; ti++) {
            int id = 0x7fffffff;
            for (int i = 0; i < 3; i++) {
                if (A[i].id > pi && A[i].id < id) id = A[i].id;
                if (B[i].id > pi && B[i].id < id) id = B[i].id;
            }
            if (id == 0x7fffffff) break;
            pi = id;
            long long w1[3], w2[3];
            wcoef(A, id, w1);
            wcoef(B, id, w2);
            for (int m = 0; m < 5; m++) {
                long long c = ww_coef(w1, u2, m) - ww_coef(w2, u1, m);
                if (c) return sgn64(c) * ss;
            }
        }
    }
    return 0;  // unreachable for distinct sets
}

// time_cmp_index for two triples that each lie on one x-value (Z = Y = 0 and
// Nx != 0, so dx = 0 in every w and N = (Nx, 0, 0)).  Then the gam_id
// coefficient of D has no 1, a or b terms: its a^2 and a^3 coefficients are
//   -(w1.dz n2x - w2.dz n1x)   and   -(w1.dy n2x - w2.dy n1x)
// and the a^3 b, a^4 b ones repeat them negated.  The smallest id in only one
// triple has w = 0 in the other and a nonzero (dz, dy) in its own (the other
// two points of that triple are distinct on one x), so an unequal pair is
// always decided in the gam tiers.  n1x, n2x are the triples' cached Nx.
template <class PT>
__device__ __forceinline__ int time_cmp_eqx(PT pt, int a0, int a1, int a2, int b0, int b1, int b2, long long n1x,
                                            long long n2x, int ss)
{
    const P3 A[3] = { pt.get(a0), pt.get(a1), pt.get(a2) };
    const P3 B[3] = { pt.get(b0), pt.get(b1), pt.get(b2) };
    int prev = -1;
    for (int t = 0; t < 6; t++) {
        int id = 0x7fffffff;
        for (int i = 0; i < 3; i++) {
            if (A[i].id > prev && A[i].id < id) id = A[i].id;
            if (B[i].id > prev && B[i].id < id) id = B[i].id;
        }
        if (id == 0x7fffffff) break;
        prev = id;
        long long w1[3], w2[3];
        wcoef(A, id, w1);
        wcoef(B, id, w2);
        i128 c = (i128)w1[1] * n2x - (i128)w2[1] * n1x;
        if (c) return -sgn128(c) * ss;
        c = (i128)w1[2] * n2x - (i128)w2[2] * n1x;
        if (c) return -sgn128(c) * ss;
    }
    return 0;  // equal point sets
}

}  // namespace hull3d
