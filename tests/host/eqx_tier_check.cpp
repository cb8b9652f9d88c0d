// Host compile of the device predicate header (test only): checks that the
// short index-tier comparison of two triples that each lie on one x-value
// (time_cmp_eqx) gives the sign of the general index tier (time_cmp_index) for
// the same pair, on seeded random triples with shared points, both
// orientations, coordinates over the full 21-bit range and over a few values.
// Prints "checked <pairs> mismatches <count>".
#define __device__
#define __forceinline__ inline
#define __noinline__
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1205_1171_gb300/csrc/predicates.cuh"

using namespace hull3d;

struct Pts {  // point table: slot -> P3 (rank = slot)
    const std::vector<P3> *v;
    P3 get(int s) const { return (*v)[s]; }
};

static uint64_t rng_state = 0x9e3779b97f4a7c15ull;
static uint64_t next_u64()
{  // splitmix64
    uint64_t z = (rng_state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
static int uniform(int lo, int hi) { return lo + (int)(next_u64() % (uint64_t)(hi - lo)); }

static long long nx_of(const P3 &p, const P3 &q, const P3 &r)
{
    long long ax = q.x - p.x, ay = q.y - p.y, az = q.z - p.z;
    long long bx = r.x - p.x, by = r.y - p.y, bz = r.z - p.z;
    (void)ax; (void)bx;
    return ay * bz - az * by;
}

int main(int argc, char **argv)
{
    const long pairs = argc > 1 ? atol(argv[1]) : 200000;
    long checked = 0, bad = 0;
    for (long it = 0; it < pairs; it++) {
        // a handful of points on two x-values, small or full-range y and z
        const bool small = (it & 1) != 0;
        const int span = small ? 4 : (1 << 20);
        const int x0 = uniform(-(1 << 20), 1 << 20), x1 = (it % 3 == 0) ? x0 : uniform(-(1 << 20), 1 << 20);
        std::vector<P3> pts;
        const int m = 6;
        for (int i = 0; i < m; i++) {
            P3 p;
            p.x = i < m / 2 ? x0 : x1;
            p.y = uniform(-span, span);
            p.z = uniform(-span, span);
            p.id = uniform(0, 1 << 24);
            p.rk = i;
            bool dup = false;
            for (const P3 &o : pts) dup |= (o.x == p.x && o.y == p.y && o.z == p.z) || o.id == p.id;
            if (dup) { i--; continue; }
            pts.push_back(p);
        }
        // two triples, each of three points on one x-value; they may share points
        int a[3], b[3];
        for (int k = 0; k < 3; k++) a[k] = k;  // the x0 points
        const int base_b = (it % 3 == 0) ? 0 : 3;
        for (int k = 0; k < 3; k++) b[k] = (it % 3 == 0) ? uniform(0, m) : base_b + k;
        if (b[0] == b[1] || b[1] == b[2] || b[0] == b[2]) continue;
        if (next_u64() & 1) { int t = a[1]; a[1] = a[2]; a[2] = t; }  // either orientation
        if (next_u64() & 1) { int t = b[0]; b[0] = b[1]; b[1] = t; }
        const long long n1 = nx_of(pts[a[0]], pts[a[1]], pts[a[2]]);
        const long long n2 = nx_of(pts[b[0]], pts[b[1]], pts[b[2]]);
        if (pts[b[0]].x != pts[b[1]].x || pts[b[1]].x != pts[b[2]].x) continue;
        if (n1 == 0 || n2 == 0) continue;  // collinear: not the short form's case
        const int ss = ((n1 < 0) ? 1 : -1) * ((n2 < 0) ? 1 : -1);  // sign(Y~) = -sign(Nx) here
        Pts pt{ &pts };
        const int want = time_cmp_index(pt, a[0], a[1], a[2], b[0], b[1], b[2], ss);
        const int got = time_cmp_eqx(pt, a[0], a[1], a[2], b[0], b[1], b[2], n1, n2, ss);
        checked++;
        if (want != got) {
            if (bad < 5)
                printf("mismatch: want %d got %d (triples %d %d %d / %d %d %d)\n", want, got, a[0], a[1], a[2], b[0],
                       b[1], b[2]);
            bad++;
        }
    }
    printf("checked %ld mismatches %ld\n", checked, bad);
    return bad ? 1 : 0;
}
