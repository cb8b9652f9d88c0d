/*
 * hull3d_oracle.c -- CPU oracle for the kinetic divide-and-conquer 3D hull.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code with the CUDA path.
 *
 * What it computes (White & Wortman, "Divide-and-Conquer 3D Convex Hulls on
 * the GPU", Sec. 2, which adapts Chan's minimalist algorithm):
 *   - points are sorted by x (Sec. 2);
 *   - the 3D lower hull is recast as a kinetic 2D problem: at time t the point
 *     (x, y, z) sits at (x, z - t*y); a lower face of the 3D hull is an
 *     instant at which three points of the 2D lower hull become collinear,
 *     i.e. a point is inserted into or deleted from the kinetic hull (Sec. 2);
 *   - the "movie" of a point set is the chronological list of those events;
 *     the movie of a node is obtained by recursing on the two halves and
 *     merging their movies by tracking the bridge (u, v) between them
 *     (Sec. 2, "Graham-scan-like O(n) merging");
 *   - the act() toggle and the time() of a triple are those of the figures
 *     "Differences in act() functions" and "Differences in time calculations"
 *     (Sec. 3), restated here on arrays of ranks;
 *   - the upper hull is the same computation on the z-mirrored point set.
 *
 * Exactness and degeneracies (the paper assumes general position; the reading
 * used here is one fixed symbolic perturbation, applied identically by the
 * CUDA path):
 *   coordinates are int32 in [-2^20, 2^20); the perturbed point i is
 *     x~ = x + a*z + a^2*y,   y~ = y + b*z + eta_i,   z~ = z + gam_i
 *   with infinitesimals a >> b >> gam_0 >> ... >> gam_{n-1} >> eta_0 >> ...
 *   (i = input index).  A predicate is a polynomial in these; its sign is the
 *   sign of the coefficient of its largest monomial, monomials being compared
 *   lexicographically from the smallest variable upwards (smaller exponent
 *   wins).  The constant term is the unperturbed value, so whenever it is
 *   nonzero it decides; otherwise the full polynomial is built by the small
 *   sparse-polynomial engine below and its leading term decides.
 *
 * Arithmetic widths: coordinate differences < 2^21, 2D cross products < 2^43
 * (int64), products of two cross products < 2^87 (__int128), orient3d < 2^66.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>

typedef __int128 i128;

#define NIL (-1)
#define COORD_LO (-(1 << 20))
#define COORD_HI ((1 << 20) - 1)

enum { OK = 0, E_INVALID = 1, E_RANGE = 2, E_DUP = 3, E_CAP = 4, E_NOMEM = 5 };

static int sgn64(int64_t v) { return (v > 0) - (v < 0); }
static int sgn128(i128 v) { return (v > 0) - (v < 0); }

/* ------------------------------------------------------------------------ */
/* Sparse polynomials over the infinitesimals a, b, gam_i, eta_i.            */
/* A term is coeff * a^ea * b^eb * gam_g * eta_h (g, h = index or -1).        */
/* Every predicate used here has at most one gam and one eta factor per term. */
/* ------------------------------------------------------------------------ */
typedef struct { int ea, eb, g, h; i128 c; } Term;
#define MAXT 1024
typedef struct { int n; Term t[MAXT]; } Poly;

static void poly_die(const char *why)
{
    fprintf(stderr, "hull3d oracle: polynomial engine: %s\n", why);
    abort();
}

static void poly_add_term(Poly *p, int ea, int eb, int g, int h, i128 c)
{
    if (c == 0) return;
    for (int i = 0; i < p->n; i++) {
        Term *t = &p->t[i];
        if (t->ea == ea && t->eb == eb && t->g == g && t->h == h) { t->c += c; return; }
    }
    if (p->n >= MAXT) poly_die("too many terms");
    p->t[p->n++] = (Term){ ea, eb, g, h, c };
}

/* r = p - q */
static void poly_sub(Poly *r, const Poly *p, const Poly *q)
{
    r->n = 0;
    for (int i = 0; i < p->n; i++) poly_add_term(r, p->t[i].ea, p->t[i].eb, p->t[i].g, p->t[i].h, p->t[i].c);
    for (int i = 0; i < q->n; i++) poly_add_term(r, q->t[i].ea, q->t[i].eb, q->t[i].g, q->t[i].h, -q->t[i].c);
}

/* r = p * q */
static void poly_mul(Poly *r, const Poly *p, const Poly *q)
{
    r->n = 0;
    for (int i = 0; i < p->n; i++)
        for (int j = 0; j < q->n; j++) {
            const Term *a = &p->t[i], *b = &q->t[j];
            if (a->g >= 0 && b->g >= 0) poly_die("two gamma factors");
            if (a->h >= 0 && b->h >= 0) poly_die("two eta factors");
            poly_add_term(r, a->ea + b->ea, a->eb + b->eb, a->g >= 0 ? a->g : b->g,
                          a->h >= 0 ? a->h : b->h, a->c * b->c);
        }
}

/* Monomial order: m1 is larger than m2 when, reading exponents from the
 * smallest variable (eta_{n-1}) upwards to a, m1 has the smaller exponent at
 * the first difference.  With one eta and one gam at most this is the
 * ascending lexicographic order of (h, g, eb, ea) with "absent" = -1. */
static int mono_less_key(const Term *x, const Term *y) /* 1 if x is the LARGER monomial */
{
    if (x->h != y->h) return x->h < y->h;
    if (x->g != y->g) return x->g < y->g;
    if (x->eb != y->eb) return x->eb < y->eb;
    return x->ea < y->ea;
}

static int poly_lead_sign(const Poly *p)
{
    const Term *best = NULL;
    for (int i = 0; i < p->n; i++) {
        if (p->t[i].c == 0) continue;
        if (!best || mono_less_key(&p->t[i], best)) best = &p->t[i];
    }
    return best ? sgn128(best->c) : 0;
}

/* ------------------------------------------------------------------------ */
/* Points.                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t x, y, z; int id; } Pt;

static void pt_xt(Poly *r, const Pt *p) /* x~ = x + a z + a^2 y */
{
    r->n = 0;
    poly_add_term(r, 0, 0, -1, -1, p->x);
    poly_add_term(r, 1, 0, -1, -1, p->z);
    poly_add_term(r, 2, 0, -1, -1, p->y);
}
static void pt_yt(Poly *r, const Pt *p) /* y~ = y + b z + eta_id */
{
    r->n = 0;
    poly_add_term(r, 0, 0, -1, -1, p->y);
    poly_add_term(r, 0, 1, -1, -1, p->z);
    poly_add_term(r, 0, 0, -1, p->id, 1);
}
static void pt_zt(Poly *r, const Pt *p) /* z~ = z + gam_id */
{
    r->n = 0;
    poly_add_term(r, 0, 0, -1, -1, p->z);
    poly_add_term(r, 0, 0, p->id, -1, 1);
}

/* The pure-a part of a predicate: set b, every gam and every eta to zero, so
 * that x~ = x + a z + a^2 y is a polynomial in a alone (coefficients (x, z, y))
 * while y~ = y and z~ = z.  The 2D cross product (q-p) x (r-p) of the
 * (x~, w) projections is then a polynomial of degree 2 in a; out[k] is its
 * coefficient of a^k (|out[k]| < 2^43). */
static void cross2_a(int64_t out[3], const Pt *p, const Pt *q, const Pt *r, int w_is_z)
{
    const int64_t dxq[3] = { q->x - p->x, q->z - p->z, q->y - p->y };
    const int64_t dxr[3] = { r->x - p->x, r->z - p->z, r->y - p->y };
    const int64_t dwq = w_is_z ? q->z - p->z : q->y - p->y;
    const int64_t dwr = w_is_z ? r->z - p->z : r->y - p->y;
    for (int k = 0; k < 3; k++) out[k] = dxq[k] * dwr - dxr[k] * dwq;
}

typedef void (*coord_fn)(Poly *, const Pt *);

/* 2D cross product of the (x~, w~) projections: (q-p) x (r-p), w~ = y~ or z~ */
static void poly_cross2(Poly *out, const Pt *p, const Pt *q, const Pt *r, coord_fn wf)
{
    static _Thread_local Poly xp, xq, xr, wp, wq, wr, dxq, dxr, dwq, dwr, m1, m2;
    pt_xt(&xp, p); pt_xt(&xq, q); pt_xt(&xr, r);
    wf(&wp, p); wf(&wq, q); wf(&wr, r);
    poly_sub(&dxq, &xq, &xp); poly_sub(&dxr, &xr, &xp);
    poly_sub(&dwq, &wq, &wp); poly_sub(&dwr, &wr, &wp);
    poly_mul(&m1, &dxq, &dwr);
    poly_mul(&m2, &dxr, &dwq);
    poly_sub(out, &m1, &m2);
}

/* sign of Y~(p,q,r) = (x~q-x~p)(y~r-y~p) - (x~r-x~p)(y~q-y~p): the turn of
 * the triple in the t = -infinity view (Sec. 2's kinetic recast). */
static int turn_sign(const Pt *p, const Pt *q, const Pt *r)
{
    int64_t nz = (q->x - p->x) * (r->y - p->y) - (r->x - p->x) * (q->y - p->y);
    if (nz) return sgn64(nz);
    /* Lazy evaluation of the same polynomial: setting b, gam, eta to zero keeps
     * exactly its pure-a monomials, and any of those outranks every monomial
     * that contains b, a gam or an eta (smaller powers of a rank higher); so
     * when that part is not zero its lowest nonzero coefficient decides. */
    int64_t ya[3];
    cross2_a(ya, p, q, r, 0);
    for (int k = 1; k < 3; k++)
        if (ya[k]) return sgn64(ya[k]);
    static _Thread_local Poly Yt;
    poly_cross2(&Yt, p, q, r, pt_yt);
    return poly_lead_sign(&Yt);
}

/* Unperturbed Z and Y of a triple: time = Z / Y (figure "time calculations"). */
static void cross_zy(const Pt *p, const Pt *q, const Pt *r, int64_t *Z, int64_t *Y)
{
    int64_t ax = q->x - p->x, ay = q->y - p->y, az = q->z - p->z;
    int64_t bx = r->x - p->x, by = r->y - p->y, bz = r->z - p->z;
    *Z = ax * bz - bx * az;
    *Y = ax * by - bx * ay;
}

static int same_set(const Pt *a[3], const Pt *b[3])
{
    int m = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            if (a[i]->id == b[j]->id) { m++; break; }
    return m == 3;
}

/* sign(t~(T1) - t~(T2)) with t~ = Z~/Y~, i.e. sign(Z~1 Y~2 - Z~2 Y~1) * sign(Y~1) * sign(Y~2). */
static int time_cmp_pts(const Pt *T1[3], const Pt *T2[3])
{
    if (same_set(T1, T2)) return 0;
    int s1 = turn_sign(T1[0], T1[1], T1[2]);
    int s2 = turn_sign(T2[0], T2[1], T2[2]);
    int64_t Z1, Y1, Z2, Y2;
    cross_zy(T1[0], T1[1], T1[2], &Z1, &Y1);
    cross_zy(T2[0], T2[1], T2[2], &Z2, &Y2);
    i128 D0 = (i128)Z1 * Y2 - (i128)Z2 * Y1;
    if (D0) return sgn128(D0) * s1 * s2;
    /* the pure-a part of D first (see turn_sign): with Z~ and Y~ of degree 2 in
     * a, D = Z~1 Y~2 - Z~2 Y~1 has degree 4 (|coefficients| < 2^88); its
     * lowest nonzero coefficient decides unless all of them are zero */
    {
        int64_t z1[3], y1[3], z2[3], y2[3];
        cross2_a(z1, T1[0], T1[1], T1[2], 1);
        cross2_a(y1, T1[0], T1[1], T1[2], 0);
        cross2_a(z2, T2[0], T2[1], T2[2], 1);
        cross2_a(y2, T2[0], T2[1], T2[2], 0);
        for (int k = 1; k <= 4; k++) {
            i128 d = 0;
            for (int i = 0; i <= 2; i++) {
                int j = k - i;
                if (j < 0 || j > 2) continue;
                d += (i128)z1[i] * y2[j] - (i128)z2[i] * y1[j];
            }
            if (d) return sgn128(d) * s1 * s2;
        }
    }
    static _Thread_local Poly Zt1, Yt1, Zt2, Yt2, m1, m2, D;
    poly_cross2(&Zt1, T1[0], T1[1], T1[2], pt_zt);
    poly_cross2(&Yt1, T1[0], T1[1], T1[2], pt_yt);
    poly_cross2(&Zt2, T2[0], T2[1], T2[2], pt_zt);
    poly_cross2(&Yt2, T2[0], T2[1], T2[2], pt_yt);
    poly_mul(&m1, &Zt1, &Yt2);
    poly_mul(&m2, &Zt2, &Yt1);
    poly_sub(&D, &m1, &m2);
    int sd = poly_lead_sign(&D);
    if (sd == 0) poly_die("distinct triples with equal perturbed times");
    return sd * s1 * s2;
}

/* orient3d(a,b,c,d) = det[b-a; c-a; d-a] of the perturbed points. */
static int orient3d_sign(const Pt *a, const Pt *b, const Pt *c, const Pt *d)
{
    int64_t m[3][3] = {
        { b->x - a->x, b->y - a->y, b->z - a->z },
        { c->x - a->x, c->y - a->y, c->z - a->z },
        { d->x - a->x, d->y - a->y, d->z - a->z },
    };
    i128 det = (i128)m[0][0] * ((i128)m[1][1] * m[2][2] - (i128)m[1][2] * m[2][1])
             - (i128)m[0][1] * ((i128)m[1][0] * m[2][2] - (i128)m[1][2] * m[2][0])
             + (i128)m[0][2] * ((i128)m[1][0] * m[2][1] - (i128)m[1][1] * m[2][0]);
    if (det) return sgn128(det);
    static _Thread_local Poly P[4][3], E[3][3], t1, t2, t3, acc, tmp;
    const Pt *pts[4] = { a, b, c, d };
    for (int i = 0; i < 4; i++) { pt_xt(&P[i][0], pts[i]); pt_yt(&P[i][1], pts[i]); pt_zt(&P[i][2], pts[i]); }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) poly_sub(&E[i][j], &P[i + 1][j], &P[0][j]);
    /* cofactor expansion along the first row */
    acc.n = 0;
    static const int cols[3][2] = { { 1, 2 }, { 0, 2 }, { 0, 1 } };
    for (int j = 0; j < 3; j++) {
        int c0 = cols[j][0], c1 = cols[j][1];
        poly_mul(&t1, &E[1][c0], &E[2][c1]);
        poly_mul(&t2, &E[1][c1], &E[2][c0]);
        poly_sub(&t3, &t1, &t2);
        poly_mul(&tmp, &E[0][j], &t3);
        for (int k = 0; k < tmp.n; k++)
            poly_add_term(&acc, tmp.t[k].ea, tmp.t[k].eb, tmp.t[k].g, tmp.t[k].h,
                          (j == 1) ? -tmp.t[k].c : tmp.t[k].c);
    }
    int s = poly_lead_sign(&acc);
    if (s == 0) poly_die("degenerate perturbed orient3d");
    return s;
}

/* ------------------------------------------------------------------------ */
/* Sorting by the perturbed x-order: sign(x~a - x~b) = lex compare (x, z, y). */
/* ------------------------------------------------------------------------ */
static int xcmp_pt(const Pt *a, const Pt *b)
{
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    if (a->z != b->z) return a->z < b->z ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    return 0;
}
static int qsort_pt(const void *a, const void *b) { return xcmp_pt((const Pt *)a, (const Pt *)b); }

/* Loads points, checks range, sorts, checks duplicates.  P[r] is the point of rank r. */
static int load_sorted(const int32_t *xyz, int64_t n, Pt **out)
{
    if (n < 0 || (n > 0 && !xyz)) return E_INVALID;
    Pt *P = (Pt *)malloc(sizeof(Pt) * (size_t)(n > 0 ? n : 1));
    if (!P) return E_NOMEM;
    for (int64_t i = 0; i < n; i++) {
        int32_t x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        if (x < COORD_LO || x > COORD_HI || y < COORD_LO || y > COORD_HI || z < COORD_LO || z > COORD_HI) {
            free(P);
            return E_RANGE;
        }
        P[i] = (Pt){ x, y, z, (int)i };
    }
    qsort(P, (size_t)n, sizeof(Pt), qsort_pt);
    for (int64_t i = 1; i < n; i++)
        if (xcmp_pt(&P[i - 1], &P[i]) == 0) { free(P); return E_DUP; }
    *out = P;
    return OK;
}

/* ------------------------------------------------------------------------ */
/* The kinetic merge (Sec. 2 and the act()/time() figures of Sec. 3).       */
/* All indices below are ranks in the sorted order; NIL = -1.                */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t w, a, b; int8_t ins; } Ev; /* event point, its neighbours, insert flag */

typedef struct {
    const Pt *P;
    int32_t *prv, *nxt;
    int upper;        /* 1: the z-mirrored pass, every finite time comparison negated */
    int aligned;      /* 1: split at the largest power of two < m (bottom-up blocks) */
} Ctx;

/* A candidate time: a triple of ranks with its unperturbed Z and Y and the
 * sign of its perturbed Y~ cached, or one of the two infinities. */
typedef struct { int32_t p, q, r; int inf; int64_t Z, Y; int s; } Tm; /* inf: -1 = -inf, +1 = +inf, 0 = finite */

static Tm mk_time(const Ctx *c, int32_t p, int32_t q, int32_t r)
{
    Tm t = { p, q, r, 0, 0, 0, 0 };
    if (p == NIL || q == NIL || r == NIL) { t.inf = 1; return t; }
    const Pt *P = c->P;
    cross_zy(&P[p], &P[q], &P[r], &t.Z, &t.Y);
    t.s = t.Y ? sgn64(t.Y) : turn_sign(&P[p], &P[q], &P[r]);
    return t;
}

/* sign(t1 - t2) in the current pass's time direction. */
static int tcmp(const Ctx *c, const Tm *t1, const Tm *t2)
{
    if (t1->inf || t2->inf) return (t1->inf > t2->inf) - (t1->inf < t2->inf);
    int s;
    i128 D0 = (i128)t1->Z * t2->Y - (i128)t2->Z * t1->Y;
    if (D0) { /* the unperturbed value decides; equal sets always give D0 = 0 */
        s = sgn128(D0) * t1->s * t2->s;
    } else {
        const Pt *A[3] = { &c->P[t1->p], &c->P[t1->q], &c->P[t1->r] };
        const Pt *B[3] = { &c->P[t2->p], &c->P[t2->q], &c->P[t2->r] };
        s = time_cmp_pts(A, B);
    }
    return c->upper ? -s : s;
}

static int turn_r(const Ctx *c, int32_t p, int32_t q, int32_t r)
{
    return turn_sign(&c->P[p], &c->P[q], &c->P[r]);
}

/* act(): insert the point between its stored neighbours if it is not in the
 * list, else unlink it (its own links are kept). */
static void act(Ctx *c, int32_t w)
{
    int32_t *prv = c->prv, *nxt = c->nxt;
    if (nxt[prv[w]] != w) {
        nxt[prv[w]] = w;
        prv[nxt[w]] = w;
    } else {
        nxt[prv[w]] = nxt[w];
        prv[nxt[w]] = prv[w];
    }
}

static int64_t split_size(const Ctx *c, int64_t m)
{
    if (!c->aligned) return m / 2;
    int64_t s = 1;
    while (s * 2 < m) s *= 2;
    return s;
}

/* Movie of the ranks [lo, lo+m): its events go to A (count returned), B is
 * scratch for the children; on return the links hold the t = -infinity hull
 * of the node, and every event point's links are its neighbours at its event. */
static int64_t movie(Ctx *c, int32_t lo, int64_t m, Ev *A, Ev *B)
{
    int32_t *prv = c->prv, *nxt = c->nxt;
    if (m == 1) { prv[lo] = nxt[lo] = NIL; return 0; }
    int64_t ml = split_size(c, m);
    int32_t mid = lo + (int32_t)ml;
    int64_t nl = movie(c, lo, ml, B, A);
    int64_t nr = movie(c, mid, m - ml, B + 2 * ml, A + 2 * ml);
    const Ev *L = B, *R = B + 2 * ml;

    /* initial bridge at t = -infinity: walk in from the inner x-extremes */
    int32_t u = mid - 1, v = mid;
    for (;;) {
        if (nxt[v] != NIL && turn_r(c, u, v, nxt[v]) < 0) v = nxt[v];
        else if (prv[u] != NIL && turn_r(c, prv[u], u, v) < 0) u = prv[u];
        else break;
    }

    /* forward pass: the earliest of six candidate events after the last one */
    int64_t i = 0, j = 0, k = 0;
    Tm old = { 0, 0, 0, -1, 0, 0, 0 };
    for (;;) {
        Tm t[6];
        t[0] = (i < nl) ? mk_time(c, prv[L[i].w], L[i].w, nxt[L[i].w]) : mk_time(c, NIL, NIL, NIL);
        t[1] = (j < nr) ? mk_time(c, prv[R[j].w], R[j].w, nxt[R[j].w]) : mk_time(c, NIL, NIL, NIL);
        t[2] = mk_time(c, u, nxt[u], v);
        t[3] = mk_time(c, prv[u], u, v);
        t[4] = mk_time(c, u, prv[v], v);
        t[5] = mk_time(c, u, v, nxt[v]);
        int best = -1;
        for (int l = 0; l < 6; l++) {
            if (t[l].inf) continue;
            if (tcmp(c, &t[l], &old) <= 0) continue;
            if (best < 0 || tcmp(c, &t[l], &t[best]) < 0) best = l;
        }
        if (best < 0) break;
        int32_t e;
        switch (best) {
        case 0:
            e = L[i++].w;
            if (e < u) A[k++] = (Ev){ e, prv[e], nxt[e], (int8_t)(nxt[prv[e]] != e) };
            act(c, e);
            break;
        case 1:
            e = R[j++].w;
            if (e > v) A[k++] = (Ev){ e, prv[e], nxt[e], (int8_t)(nxt[prv[e]] != e) };
            act(c, e);
            break;
        case 2: { int32_t a = u; u = nxt[u]; A[k++] = (Ev){ u, a, v, 1 }; break; }
        case 3: A[k++] = (Ev){ u, prv[u], v, 0 }; u = prv[u]; break;
        case 4: { int32_t b = v; v = prv[v]; A[k++] = (Ev){ v, u, b, 1 }; break; }
        case 5: A[k++] = (Ev){ v, u, nxt[v], 0 }; v = nxt[v]; break;
        }
        old = t[best];
    }

    /* backward pass: from the t = +infinity bridge, undo the node's events in
     * reverse, splicing bridge events back, to reach the t = -infinity state */
    nxt[u] = v;
    prv[v] = u;
    for (int64_t kk = k - 1; kk >= 0; kk--) {
        int32_t w = A[kk].w;
        if (w <= u || w >= v) {
            act(c, w);
            if (w == u) u = prv[u];
            else if (w == v) v = nxt[v];
        } else {
            nxt[u] = w; prv[w] = u;
            prv[v] = w; nxt[w] = v;
            if (w < mid) u = w; else v = w;
        }
    }
    return k;
}

/* ------------------------------------------------------------------------ */
/* Faces.                                                                    */
/* ------------------------------------------------------------------------ */
static void canon_face(int32_t f[3])
{
    /* rotate so the smallest index comes first (orientation kept) */
    while (!(f[0] < f[1] && f[0] < f[2])) {
        int32_t t = f[0]; f[0] = f[1]; f[1] = f[2]; f[2] = t;
    }
}

static int qsort_face(const void *a, const void *b)
{
    const int32_t *x = (const int32_t *)a, *y = (const int32_t *)b;
    for (int i = 0; i < 3; i++)
        if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    return 0;
}

/* Runs one pass over all n points; replays the root movie from the -infinity
 * hull and writes its faces, outward-oriented, as input indices. */
static int64_t pass_faces(Ctx *c, int64_t n, Ev *A, Ev *B, int32_t *faces, int *consistent)
{
    int64_t k = movie(c, 0, n, A, B);
    for (int64_t e = 0; e < k; e++) {
        int32_t w = A[e].w, p = c->prv[w], r = c->nxt[w];
        if (p != A[e].a || r != A[e].b) *consistent = 0;
        int up = turn_r(c, p, w, r) > 0; /* Y~ > 0: normal (q-p)x(r-p) points up */
        int32_t f[3];
        /* lower faces face down, upper faces face up */
        if (up == c->upper) { f[0] = c->P[p].id; f[1] = c->P[w].id; f[2] = c->P[r].id; }
        else { f[0] = c->P[p].id; f[1] = c->P[r].id; f[2] = c->P[w].id; }
        canon_face(f);
        memcpy(faces + 3 * e, f, sizeof f);
        act(c, w);
    }
    return k;
}

static int run_hull(const int32_t *xyz, int64_t n, int aligned, int32_t *faces, int64_t cap, int64_t *nfaces)
{
    if (!nfaces) return E_INVALID;
    *nfaces = 0;
    if (n < 1 || !xyz) return E_INVALID;
    Pt *P;
    int rc = load_sorted(xyz, n, &P);
    if (rc) return rc;
    if (n < 3) { free(P); return OK; }
    int64_t need = 2 * n - 4;
    if (cap < need || !faces) { free(P); return E_CAP; }
    int32_t *prv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    Ev *A = (Ev *)malloc(sizeof(Ev) * (size_t)(2 * n));
    Ev *B = (Ev *)malloc(sizeof(Ev) * (size_t)(2 * n));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(2 * n));
    if (!prv || !nxt || !A || !B || !tmp) {
        free(P); free(prv); free(nxt); free(A); free(B); free(tmp);
        return E_NOMEM;
    }
    int consistent = 1;
    Ctx c = { P, prv, nxt, 0, aligned };
    int64_t nf = pass_faces(&c, n, A, B, tmp, &consistent);
    c.upper = 1;
    nf += pass_faces(&c, n, A, B, tmp + 3 * nf, &consistent);
    qsort(tmp, (size_t)nf, 3 * sizeof(int32_t), qsort_face);
    rc = OK;
    if (!consistent) rc = E_INVALID; /* replayed faces must equal the recorded ones */
    if (nf > cap) rc = E_CAP;
    else memcpy(faces, tmp, sizeof(int32_t) * 3 * (size_t)nf);
    *nfaces = nf;
    free(P); free(prv); free(nxt); free(A); free(B); free(tmp);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Exported API (ctypes).                                                    */
/* ------------------------------------------------------------------------ */

/* Canonical face list of the hull of n points (xyz: n x 3 int32, row-major).
 * Faces are outward-CCW triples of input indices, rotated min-first, sorted.
 * split_mode 0: Chan's top-down split at floor(m/2); 1: aligned power-of-two
 * blocks as in the bottom-up movie array (Sec. 2).  Returns 0 or an error. */
int oracle_hull(const int32_t *xyz, int64_t n, int split_mode, int32_t *faces, int64_t cap, int64_t *nfaces)
{
    return run_hull(xyz, n, split_mode == 1, faces, cap, nfaces);
}

/* order[r] = input index of the point of rank r (sorted by x, then z, then y). */
int oracle_sort_order(const int32_t *xyz, int64_t n, int32_t *order)
{
    Pt *P;
    int rc = load_sorted(xyz, n, &P);
    if (rc) return rc;
    for (int64_t r = 0; r < n; r++) order[r] = P[r].id;
    free(P);
    return OK;
}

/* Event list of the node holding the sorted ranks [lo, hi), for one pass.
 * ev_w/ev_a/ev_b are ranks (the event point and its two neighbours in the
 * node's hull at the event), ev_ins is 1 for an insertion.  Also returns the
 * node's t = -infinity hull as a rank list in neg_hull (may be NULL). */
int oracle_node_events(const int32_t *xyz, int64_t n, int64_t lo, int64_t hi, int upper,
                       int32_t *ev_w, int32_t *ev_a, int32_t *ev_b, int8_t *ev_ins, int64_t cap,
                       int64_t *nev, int32_t *neg_hull, int64_t *nneg)
{
    if (!nev || lo < 0 || hi > n || lo >= hi) return E_INVALID;
    Pt *P;
    int rc = load_sorted(xyz, n, &P);
    if (rc) return rc;
    int64_t m = hi - lo;
    int32_t *prv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    Ev *A = (Ev *)malloc(sizeof(Ev) * (size_t)(2 * m));
    Ev *B = (Ev *)malloc(sizeof(Ev) * (size_t)(2 * m));
    if (!prv || !nxt || !A || !B) { free(P); free(prv); free(nxt); free(A); free(B); return E_NOMEM; }
    Ctx c = { P, prv, nxt, upper != 0, 0 };
    int64_t k = movie(&c, (int32_t)lo, m, A, B);
    *nev = k;
    if (k > cap) rc = E_CAP;
    else
        for (int64_t e = 0; e < k; e++) {
            ev_w[e] = A[e].w; ev_a[e] = A[e].a; ev_b[e] = A[e].b; ev_ins[e] = A[e].ins;
        }
    if (nneg) {
        int64_t cnt = 0;
        for (int32_t w = (int32_t)lo; w != NIL; w = nxt[w]) {
            if (neg_hull) neg_hull[cnt] = w;
            cnt++;
        }
        *nneg = cnt;
    }
    free(P); free(prv); free(nxt); free(A); free(B);
    return rc;
}

/* Brute force: a triple is a face iff every other point lies strictly on one
 * side of its perturbed plane.  O(n^4); for tiny n only. */
int oracle_brute_faces(const int32_t *xyz, int64_t n, int32_t *faces, int64_t cap, int64_t *nfaces)
{
    if (!nfaces) return E_INVALID;
    *nfaces = 0;
    if (n < 1 || !xyz) return E_INVALID;
    Pt *P;
    int rc = load_sorted(xyz, n, &P);
    if (rc) return rc;
    /* work in input-index order so that the result does not depend on the sort */
    Pt *Q = (Pt *)malloc(sizeof(Pt) * (size_t)n);
    for (int64_t i = 0; i < n; i++) Q[P[i].id] = P[i];
    free(P);
    int64_t nf = 0;
    if (n == 3) {
        /* a lone triangle: both of its sides are faces */
        if (cap < 2) { free(Q); *nfaces = 2; return E_CAP; }
        int32_t f1[3] = { 0, 1, 2 }, f2[3] = { 0, 2, 1 };
        memcpy(faces, f1, sizeof f1);
        memcpy(faces + 3, f2, sizeof f2);
        nf = 2;
    }
    for (int64_t i = 0; i < n && n > 3; i++)
        for (int64_t j = i + 1; j < n; j++)
            for (int64_t k = j + 1; k < n; k++) {
                int side = 0, ok = 1;
                for (int64_t l = 0; l < n && ok; l++) {
                    if (l == i || l == j || l == k) continue;
                    int s = orient3d_sign(&Q[i], &Q[j], &Q[k], &Q[l]);
                    if (side == 0) side = s;
                    else if (s != side) ok = 0;
                }
                if (!ok) continue;
                /* every other point on the negative side of n = (j-i)x(k-i): (i,j,k) faces out */
                int32_t f[3];
                if (side < 0) { f[0] = (int32_t)i; f[1] = (int32_t)j; f[2] = (int32_t)k; }
                else { f[0] = (int32_t)i; f[1] = (int32_t)k; f[2] = (int32_t)j; }
                canon_face(f);
                if (nf + 1 > cap) { free(Q); *nfaces = nf + 1; return E_CAP; }
                memcpy(faces + 3 * nf, f, sizeof f);
                nf++;
            }
    qsort(faces, (size_t)nf, 3 * sizeof(int32_t), qsort_face);
    *nfaces = nf;
    free(Q);
    return OK;
}

/* ------------------------------------------------------------------------ */
/* 2D Delaunay triangulation through the lifting map.                         */
/* ------------------------------------------------------------------------ */
/* The points (x, y) lifted to (x, y, x^2 + y^2) lie on a paraboloid; a triple
 * is a lower face of their 3D hull exactly when no other point lies inside
 * the triple's circumcircle, so the lower hull projects to the Delaunay
 * triangulation.  Here the lower pass of the method above (Sec. 2) runs on
 * the lifted points, with the same perturbation (so four cocircular points
 * get one consistent diagonal).  Coordinates are limited to |x|, |y| < 2^15:
 * the lifted z < 2^31, coordinate differences < 2^31, 2D cross products of
 * the (x, z) and (x, y) projections < 2^48 (int64), their products < 2^97
 * (__int128), orient3d < 2^66 -- the widths of the 3D hull above still hold.
 * A lower face whose three points are collinear in the plane (points on one
 * edge of the convex hull, which the perturbation may turn into a sliver) has
 * zero area and is not a triangle of the triangulation: it is left out.  The
 * triangles are written counter-clockwise in the plane, rotated min-first and
 * sorted. */
#define LIFT_LIM ((1 << 15) - 1)

int oracle_delaunay(const int32_t *xy, int64_t n, int32_t *tris, int64_t cap, int64_t *ntris)
{
    if (!ntris) return E_INVALID;
    *ntris = 0;
    if (n < 1 || !xy) return E_INVALID;
    Pt *P = (Pt *)malloc(sizeof(Pt) * (size_t)n);
    if (!P) return E_NOMEM;
    for (int64_t i = 0; i < n; i++) {
        const int64_t x = xy[2 * i], y = xy[2 * i + 1];
        if (x < -LIFT_LIM || x > LIFT_LIM || y < -LIFT_LIM || y > LIFT_LIM) { free(P); return E_RANGE; }
        P[i] = (Pt){ x, y, x * x + y * y, (int)i };
    }
    qsort(P, (size_t)n, sizeof(Pt), qsort_pt);
    for (int64_t i = 1; i < n; i++)
        if (xcmp_pt(&P[i - 1], &P[i]) == 0) { free(P); return E_DUP; }
    if (n < 3) { free(P); return OK; }
    int32_t *prv = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    Ev *A = (Ev *)malloc(sizeof(Ev) * (size_t)(2 * n));
    Ev *B = (Ev *)malloc(sizeof(Ev) * (size_t)(2 * n));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(2 * n));
    if (!prv || !nxt || !A || !B || !tmp) {
        free(P); free(prv); free(nxt); free(A); free(B); free(tmp);
        return E_NOMEM;
    }
    Ctx c = { P, prv, nxt, 0, 0 };
    int64_t k = movie(&c, 0, n, A, B); /* the lower pass only */
    int rc = OK;
    int64_t nt = 0;
    for (int64_t e = 0; e < k; e++) { /* replay the root movie: one face per event */
        int32_t w = A[e].w, p = c.prv[w], r = c.nxt[w];
        if (p != A[e].a || r != A[e].b) rc = E_INVALID;
        const int64_t area = (P[w].x - P[p].x) * (P[r].y - P[p].y) - (P[r].x - P[p].x) * (P[w].y - P[p].y);
        if (area != 0) {
            int32_t f[3];
            /* counter-clockwise in the plane */
            if (area > 0) { f[0] = P[p].id; f[1] = P[w].id; f[2] = P[r].id; }
            else { f[0] = P[p].id; f[1] = P[r].id; f[2] = P[w].id; }
            canon_face(f);
            memcpy(tmp + 3 * nt, f, sizeof f);
            nt++;
        }
        act(&c, w);
    }
    qsort(tmp, (size_t)nt, 3 * sizeof(int32_t), qsort_face);
    if (!rc && nt > cap) rc = E_CAP;
    else if (!rc) memcpy(tris, tmp, sizeof(int32_t) * 3 * (size_t)nt);
    *ntris = nt;
    free(P); free(prv); free(nxt); free(A); free(B); free(tmp);
    return rc;
}

/* Predicates on explicit points, for the predicate tests.  pts: k x 3 int32,
 * ids: k input indices (they pick the gam/eta infinitesimals). */
int oracle_turn_sign(const int32_t *pts, const int32_t *ids)
{
    Pt a = { pts[0], pts[1], pts[2], ids[0] }, b = { pts[3], pts[4], pts[5], ids[1] },
       c = { pts[6], pts[7], pts[8], ids[2] };
    return turn_sign(&a, &b, &c);
}

int oracle_time_cmp(const int32_t *pts, const int32_t *ids)
{
    Pt q[6];
    for (int i = 0; i < 6; i++) q[i] = (Pt){ pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], ids[i] };
    const Pt *A[3] = { &q[0], &q[1], &q[2] }, *B[3] = { &q[3], &q[4], &q[5] };
    return time_cmp_pts(A, B);
}

int oracle_orient3d_sign(const int32_t *pts, const int32_t *ids)
{
    Pt q[4];
    for (int i = 0; i < 4; i++) q[i] = (Pt){ pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], ids[i] };
    return orient3d_sign(&q[0], &q[1], &q[2], &q[3]);
}
