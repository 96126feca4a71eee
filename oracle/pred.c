/*
 * Geometric predicates and fixed-order FP64 geometry for the oracle.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Compile with -ffp-contract=off:
 * the FP64 formulas below (quality test, circumcentre, midpoint) are the
 * specification that the CUDA path must reproduce bit for bit, so no fused
 * multiply-add may change their rounding.
 *
 * Predicates are exact (Sec. 7 set-up: exact arithmetic + simulation of
 * simplicity).  Each is written as the determinant it is defined by:
 *   orient(a,b,c)    = det [ax ay 1; bx by 1; cx cy 1]                 (> 0: CCW)
 *   incircle(a,b,c,d)= det [x y x^2+y^2 1] over rows a,b,c,d          (> 0: d inside
 *                      the circle through CCW a,b,c)
 *   dot(a,b;p)       = (a-p).(b-p)   (< 0: p strictly inside the diametral circle
 *                      of ab, i.e. p encroaches ab -- Sec. 4.2, Ruppert's rule)
 *   lens(a,b;p)      = p strictly inside the diametral lens of ab (Chew's rule,
 *                      Sec. 4.2): 3 ((a-p).(b-p))^2 > ((a-p) x (b-p))^2 with a
 *                      negative dot product
 * A floating-point value with a forward error bound answers when it can;
 * otherwise the monomial expansion of the determinant is summed exactly.
 */
#include "oracle.h"

#include <math.h>
#include <string.h>

static int g_filter = 1;
void or_set_filter(int enabled) { g_filter = enabled; }

/* unit roundoff of binary64 */
#define U_RND (1.1102230246251565e-16)
/* below this magnitude the relative error model may fail (underflow): go exact */
#define TINY (1e-250)

static void mono2(or_mono* m, int s, double a, double b) {
    m->sign = s; m->k = 2; m->f[0] = a; m->f[1] = b;
}
static void mono4(or_mono* m, int s, double a, double b, double c, double d) {
    m->sign = s; m->k = 4; m->f[0] = a; m->f[1] = b; m->f[2] = c; m->f[3] = d;
}

/* the six monomials of det [ax ay 1; bx by 1; cx cy 1], scaled by sign s */
static int orient_monos(or_mono* m, int s, double ax, double ay, double bx, double by,
                        double cx, double cy) {
    mono2(m + 0, s, ax, by);
    mono2(m + 1, -s, ax, cy);
    mono2(m + 2, -s, ay, bx);
    mono2(m + 3, s, ay, cx);
    mono2(m + 4, s, bx, cy);
    mono2(m + 5, -s, by, cx);
    return 6;
}

static int orient_exact(double ax, double ay, double bx, double by, double cx, double cy) {
    or_mono m[6];
    orient_monos(m, 1, ax, ay, bx, by, cx, cy);
    return or_exact_sign(m, 6);
}

int or_orient(double ax, double ay, double bx, double by, double cx, double cy) {
    if (g_filter) {
        /* l - r with l = (ax-cx)(by-cy), r = (ay-cy)(bx-cx): each product carries
         * at most three roundings (two differences, one product), the final
         * subtraction one more; |err| <= (3u + u + O(u^2)) (|l|+|r|).  5u covers
         * the higher-order terms and the rounding of the bound itself. */
        double l = (ax - cx) * (by - cy);
        double r = (ay - cy) * (bx - cx);
        double det = l - r;
        double perm = fabs(l) + fabs(r);
        double bound = 5.0 * U_RND * perm;
        if (perm > TINY) {
            if (det > bound) return 1;
            if (-det > bound) return -1;
        }
    }
    return orient_exact(ax, ay, bx, by, cx, cy);
}

/* incircle as the lifted 4x4 determinant, Laplace-expanded along the lift column:
 *   + z_a*orient(b,c,d) - z_b*orient(a,c,d) + z_c*orient(a,b,d) - z_d*orient(a,b,c)
 * with z = x^2 + y^2; 48 monomials of degree 4. */
static int incircle_exact(double ax, double ay, double bx, double by, double cx, double cy,
                          double dx, double dy) {
    const double px[4] = {ax, bx, cx, dx}, py[4] = {ay, by, cy, dy};
    or_mono m[48];
    int n = 0;
    for (int i = 0; i < 4; ++i) {
        int s = (i % 2 == 0) ? 1 : -1;
        double q[6];
        int k = 0;
        for (int j = 0; j < 4; ++j) if (j != i) { q[k++] = px[j]; q[k++] = py[j]; }
        or_mono o[6];
        orient_monos(o, s, q[0], q[1], q[2], q[3], q[4], q[5]);
        for (int t = 0; t < 6; ++t) {
            mono4(&m[n++], o[t].sign, px[i], px[i], o[t].f[0], o[t].f[1]);
            mono4(&m[n++], o[t].sign, py[i], py[i], o[t].f[0], o[t].f[1]);
        }
    }
    return or_exact_sign(m, n);
}

int or_incircle(double ax, double ay, double bx, double by, double cx, double cy,
                double dx, double dy) {
    if (g_filter) {
        double adx = ax - dx, ady = ay - dy, bdx = bx - dx, bdy = by - dy;
        double cdx = cx - dx, cdy = cy - dy;
        double p1 = bdx * cdy, p2 = cdx * bdy, al = adx * adx + ady * ady;
        double p3 = cdx * ady, p4 = adx * cdy, bl = bdx * bdx + bdy * bdy;
        double p5 = adx * bdy, p6 = bdx * ady, cl = cdx * cdx + cdy * cdy;
        double det = al * (p1 - p2) + bl * (p3 - p4) + cl * (p5 - p6);
        double perm = (fabs(p1) + fabs(p2)) * al + (fabs(p3) + fabs(p4)) * bl +
                      (fabs(p5) + fabs(p6)) * cl;
        /* per term: lift <= 4 roundings, each cross product <= 3, their
         * difference 1, the product 1; two more for the sum of three terms:
         * about 11u * perm to first order.  14u leaves room for the rest. */
        double bound = 14.0 * U_RND * perm;
        if (perm > TINY) {
            if (det > bound) return 1;
            if (-det > bound) return -1;
        }
    }
    return incircle_exact(ax, ay, bx, by, cx, cy, dx, dy);
}

int or_lex_less(double ax, double ay, double bx, double by) {
    return (ax < bx) || (ax == bx && ay < by);
}

/* Simulation of simplicity for incircle: the lift of each point is raised by
 * an infinitesimal eps_i, with eps_i >> eps_j whenever point i is
 * lexicographically (x, then y) larger than point j.  The perturbed
 * determinant is det + sum_i eps_i * C_i where C_i is the cofactor of the lift
 * entry of row i, i.e. C_a = orient(b,c,d), C_b = -orient(a,c,d),
 * C_c = orient(a,b,d), C_d = -orient(a,b,c).  A zero determinant therefore
 * takes the sign of the first non-zero cofactor in decreasing lexicographic
 * order of the points.  The ranking uses coordinates, not vertex ids, so that
 * any two triangulators agree whatever ids they give their vertices. */
int or_incircle_sos(double ax, double ay, double bx, double by, double cx, double cy,
                    double dx, double dy) {
    int s = or_incircle(ax, ay, bx, by, cx, cy, dx, dy);
    if (s != 0) return s;
    const double px[4] = {ax, bx, cx, dx}, py[4] = {ay, by, cy, dy};
    int ord[4] = {0, 1, 2, 3};
    /* sort indices by decreasing (x, y) */
    for (int i = 1; i < 4; ++i) {
        int v = ord[i], j = i - 1;
        while (j >= 0 && or_lex_less(px[ord[j]], py[ord[j]], px[v], py[v])) {
            ord[j + 1] = ord[j];
            --j;
        }
        ord[j + 1] = v;
    }
    for (int r = 0; r < 4; ++r) {
        int i = ord[r];
        double q[6];
        int k = 0;
        for (int j = 0; j < 4; ++j) if (j != i) { q[k++] = px[j]; q[k++] = py[j]; }
        int o = or_orient(q[0], q[1], q[2], q[3], q[4], q[5]);
        if (o != 0) return (i % 2 == 0) ? o : -o;
    }
    return 0;
}

int or_dot_sign(double ax, double ay, double bx, double by, double px, double py) {
    if (g_filter) {
        double d1 = (ax - px) * (bx - px);
        double d2 = (ay - py) * (by - py);
        double s = d1 + d2;
        double perm = fabs(d1) + fabs(d2);
        double bound = 5.0 * U_RND * perm;
        if (perm > TINY) {
            if (s > bound) return 1;
            if (-s > bound) return -1;
        }
    }
    /* (ax-px)(bx-px) + (ay-py)(by-py), expanded */
    or_mono m[8];
    mono2(m + 0, 1, ax, bx);
    mono2(m + 1, -1, ax, px);
    mono2(m + 2, -1, px, bx);
    mono2(m + 3, 1, px, px);
    mono2(m + 4, 1, ay, by);
    mono2(m + 5, -1, ay, py);
    mono2(m + 6, -1, py, by);
    mono2(m + 7, 1, py, py);
    return or_exact_sign(m, 8);
}

/* lens(a,b;p): p strictly inside the diametral lens of ab, the encroachment
 * region of Chew's rule (Sec. 4.2).  The lens is the set of points from which
 * the segment subtends an angle above 120 degrees: the intersection of the two
 * disks through a and b whose centres lie on each other's circles, its apexes
 * seeing the segment's ends at 30 degrees.  With u = a-p, w = b-p, D = u.w and
 * C = u x w, Lagrange's identity |u|^2 |w|^2 = D^2 + C^2 turns
 * cos(angle) < -1/2 into: D < 0 and 3 D^2 - C^2 > 0.
 * Returns -1 inside, 0 on the boundary (a, b themselves), +1 outside. */
static int lens_monos(or_mono* m, double ax, double ay, double bx, double by, double px, double py) {
    /* D and C as signed degree-2 monomials in the raw coordinates */
    const double dd[8][2] = {{ax, bx}, {ax, px}, {px, bx}, {px, px},
                             {ay, by}, {ay, py}, {py, by}, {py, py}};
    const int ds[8] = {1, -1, -1, 1, 1, -1, -1, 1};
    const double cc[8][2] = {{ax, by}, {ax, py}, {px, by}, {px, py},
                             {ay, bx}, {ay, px}, {py, bx}, {py, px}};
    const int cs[8] = {1, -1, -1, 1, -1, 1, 1, -1};
    int n = 0;
    for (int r = 0; r < 3; ++r)            /* 3 D^2 */
        for (int i = 0; i < 8; ++i)
            for (int j = 0; j < 8; ++j)
                mono4(m + n++, ds[i] * ds[j], dd[i][0], dd[i][1], dd[j][0], dd[j][1]);
    for (int i = 0; i < 8; ++i)            /* - C^2 */
        for (int j = 0; j < 8; ++j)
            mono4(m + n++, -cs[i] * cs[j], cc[i][0], cc[i][1], cc[j][0], cc[j][1]);
    return n;
}

int or_lens_sign(double ax, double ay, double bx, double by, double px, double py) {
    const int d = or_dot_sign(ax, ay, bx, by, px, py);
    if (d > 0) return 1;
    if (d == 0) return ((px == ax && py == ay) || (px == bx && py == by)) ? 0 : 1;
    if (g_filter) {
        /* D and C with forward error bounds, then 3 D^2 - C^2 over the intervals */
        const double ux = ax - px, uy = ay - py, wx = bx - px, wy = by - py;
        const double D = ux * wx + uy * wy, Cr = ux * wy - uy * wx;
        const double eD = 4.0 * U_RND * (fabs(ux * wx) + fabs(uy * wy)) + 4.0 * U_RND * (fabs(ux) + fabs(uy)) * (fabs(wx) + fabs(wy));
        const double eC = 4.0 * U_RND * (fabs(ux * wy) + fabs(uy * wx)) + 4.0 * U_RND * (fabs(ux) + fabs(uy)) * (fabs(wx) + fabs(wy));
        const double aD = fabs(D), aC = fabs(Cr);
        if (aD > TINY && aD > eD) {
            const double dlo = aD - eD, dhi = aD + eD;
            const double clo = aC > eC ? aC - eC : 0.0, chi = aC + eC;
            const double lo = 3.0 * dlo * dlo * (1 - 8 * U_RND) - chi * chi * (1 + 8 * U_RND);
            const double hi = 3.0 * dhi * dhi * (1 + 8 * U_RND) - clo * clo * (1 - 8 * U_RND);
            if (lo > 0) return -1;
            if (hi < 0) return 1;
        }
    }
    or_mono m[256];
    const int n = lens_monos(m, ax, ay, bx, by, px, py);
    const int s = or_exact_sign(m, n);
    return s > 0 ? -1 : (s < 0 ? 1 : 0);
}

/* ---------------- fixed-order FP64 geometry ----------------
 * Canonical form: the triangle's vertices are rotated (keeping CCW order) so
 * that a is the lexicographically smallest.  All quantities below are then
 * evaluated in exactly this order, in binary64 with round-to-nearest and no
 * contraction. */
static void canon3(double ax, double ay, double bx, double by, double cx, double cy,
                   double* o) {
    int k = 0;
    if (or_lex_less(bx, by, ax, ay)) k = 1;
    double kx = k ? bx : ax, ky = k ? by : ay;
    if (or_lex_less(cx, cy, kx, ky)) k = 2;
    const double x[3] = {ax, bx, cx}, y[3] = {ay, by, cy};
    for (int i = 0; i < 3; ++i) {
        o[2 * i] = x[(k + i) % 3];
        o[2 * i + 1] = y[(k + i) % 3];
    }
}

typedef struct { double ax, ay, dx, dy, ex, ey, la, lb, lc, cr; } tri_terms;

static void terms(double ax, double ay, double bx, double by, double cx, double cy,
                  tri_terms* t) {
    double p[6];
    canon3(ax, ay, bx, by, cx, cy, p);
    t->ax = p[0]; t->ay = p[1];
    t->dx = p[2] - p[0]; t->dy = p[3] - p[1];       /* b - a */
    t->ex = p[4] - p[0]; t->ey = p[5] - p[1];       /* c - a */
    double fx = p[4] - p[2], fy = p[5] - p[3];      /* c - b */
    t->la = t->dx * t->dx + t->dy * t->dy;          /* |ab|^2 */
    t->lb = t->ex * t->ex + t->ey * t->ey;          /* |ac|^2 */
    t->lc = fx * fx + fy * fy;                      /* |bc|^2 */
    t->cr = t->dx * t->ey - t->dy * t->ex;          /* twice the signed area */
}

/* Bad triangle (C1 reading of Sec. 4.1 with the radius-edge bound of Sec. 5.1):
 *   R / l_min > B  <=>  la*lb*lc > 4 B^2 l_min^2 (2A)^2  since R = |ab||bc||ca| / (4A). */
int or_is_bad(double ax, double ay, double bx, double by, double cx, double cy, double B2) {
    tri_terms t;
    terms(ax, ay, bx, by, cx, cy, &t);
    double lmin = t.la;
    if (t.lb < lmin) lmin = t.lb;
    if (t.lc < lmin) lmin = t.lc;
    double lhs = (t.la * t.lb) * t.lc;
    double rhs = ((4.0 * B2) * lmin) * (t.cr * t.cr);
    return lhs > rhs;
}

/* Edge-length criterion (Sec. 4.1: besides the angle bound, an edge length
 * bound l): the longest edge is longer than l, i.e. max(|ab|^2, |bc|^2,
 * |ca|^2) > L2 = l^2 with the squared lengths of the quality test above. */
int or_is_long(double ax, double ay, double bx, double by, double cx, double cy, double L2) {
    tri_terms t;
    terms(ax, ay, bx, by, cx, cy, &t);
    double lmax = t.la;
    if (t.lb > lmax) lmax = t.lb;
    if (t.lc > lmax) lmax = t.lc;
    return lmax > L2;
}

/* (R / l_min)^2 * 4, used only to order the oracle's queue of bad triangles */
double or_ratio_key(double ax, double ay, double bx, double by, double cx, double cy) {
    tri_terms t;
    terms(ax, ay, bx, by, cx, cy, &t);
    double lmin = t.la;
    if (t.lb < lmin) lmin = t.lb;
    if (t.lc < lmin) lmin = t.lc;
    return ((t.la * t.lb) * t.lc) / (lmin * (t.cr * t.cr));
}

/* circumcentre relative to the canonical vertex a (C5):
 *   c = a + ( ey*la - dy*lb , dx*lb - ex*la ) / (2*cr) */
void or_circumcenter(double ax, double ay, double bx, double by, double cx, double cy,
                     double* ox, double* oy) {
    tri_terms t;
    terms(ax, ay, bx, by, cx, cy, &t);
    double den = 2.0 * t.cr;
    double nx = t.ey * t.la - t.dy * t.lb;
    double ny = t.dx * t.lb - t.ex * t.la;
    *ox = t.ax + nx / den;
    *oy = t.ay + ny / den;
}

/* midpoint (C4): ((ax+bx)*0.5, (ay+by)*0.5), symmetric in a and b */
void or_midpoint(double ax, double ay, double bx, double by, double* ox, double* oy) {
    *ox = (ax + bx) * 0.5;
    *oy = (ay + by) * 0.5;
}

/* priority measure bits (C7): float32 of a non-negative value, sign bit dropped;
 * the bit patterns of non-negative floats increase with the value. */
uint32_t or_measure_bits(double v) {
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    return u & 0x7fffffffu;
}

/* triangle measure: twice its area, |cr| in canonical form */
double or_tri_measure(double ax, double ay, double bx, double by, double cx, double cy) {
    tri_terms t;
    terms(ax, ay, bx, by, cx, cy, &t);
    return fabs(t.cr);
}

/* subsegment measure: squared length, endpoints in lexicographic order */
double or_seg_measure(double ax, double ay, double bx, double by) {
    if (or_lex_less(bx, by, ax, ay)) {
        double tx = ax, ty = ay;
        ax = bx; ay = by; bx = tx; by = ty;
    }
    double dx = bx - ax, dy = by - ay;
    return dx * dx + dy * dy;
}
