/*
 * Sequential Ruppert refinement (the oracle for Algorithm 1 of Sec. 4).
 * TEST INFRASTRUCTURE ONLY.
 *
 * Loop (Sec. 4.2 rules, applied one point at a time):
 *   1. while a subsegment is encroached -- a vertex strictly inside its
 *      diametral circle (Ruppert's rule) or its diametral lens (Chew's rule,
 *      or_refine_mode with lens != 0) -- split it (midpoint, or a
 *      concentric-shell point next to a small input angle);
 *   2. otherwise take the worst bad triangle and compute its circumcentre c:
 *      - if the walk from the triangle to c crosses a subsegment, split that
 *        subsegment instead (Sec. 4.3, point location);
 *      - if c would encroach a subsegment on its cavity boundary, split those
 *        subsegments instead (Sec. 4.2: midpoints take priority over
 *        circumcentres; such a circumcentre is redundant);
 *      - else insert c by Bowyer-Watson;
 *   3. stop when nothing is encroached and no triangle is bad (bad triangles
 *      whose shortest edge joins two segments meeting at a small input angle
 *      are accepted, Sec. 4.1).
 */
#include "mesh_int.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- small input angles ---------------- */
typedef struct {
    int64_t* off;   /* CSR over input vertices: incident input segments */
    int32_t* adj;
} seg_adj;

static void build_adj(const or_mesh* M, seg_adj* A) {
    A->off = (int64_t*)calloc((size_t)M->n_in + 1, sizeof(int64_t));
    A->adj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * M->nseg + 1));
    for (int64_t s = 0; s < M->nseg; ++s) {
        A->off[M->seg[2 * s] + 1]++;
        A->off[M->seg[2 * s + 1] + 1]++;
    }
    for (int64_t v = 0; v < M->n_in; ++v) A->off[v + 1] += A->off[v];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(M->n_in + 1));
    memcpy(fill, A->off, sizeof(int64_t) * (size_t)(M->n_in + 1));
    for (int64_t s = 0; s < M->nseg; ++s) {
        A->adj[fill[M->seg[2 * s]]++] = (int32_t)s;
        A->adj[fill[M->seg[2 * s + 1]]++] = (int32_t)s;
    }
    free(fill);
}

/* C6/C10: the angle at a shared endpoint o between the directions to p and q
 * is below 60 degrees iff cos > 1/2, i.e. 2 (u.w) > |u| |w| with u = p - o,
 * w = q - o, evaluated in FP64 in this order (no contraction).  This only
 * selects where the small-angle rules of Sec. 4.1 apply. */
int or_small_angle(double ox, double oy, double px, double py, double qx, double qy) {
    double ux = px - ox, uy = py - oy;
    double wx = qx - ox, wy = qy - oy;
    double dot = ux * wx + uy * wy;
    double nn = sqrt(ux * ux + uy * uy) * sqrt(wx * wx + wy * wy);
    return 2.0 * dot > nn;
}

/* two distinct input segments meeting at a shared endpoint at less than 60 degrees */
static int small_pair_seg(const double* x, const double* y, const int32_t* seg, int64_t s1, int64_t s2) {
    if (s1 == s2 || s1 < 0 || s2 < 0) return 0;
    const int32_t* a = seg + 2 * s1;
    const int32_t* b = seg + 2 * s2;
    int64_t o = -1, p = -1, q = -1;
    for (int i = 0; i < 2 && o < 0; ++i)
        for (int j = 0; j < 2; ++j)
            if (a[i] == b[j]) { o = a[i]; p = a[1 - i]; q = b[1 - j]; break; }
    if (o < 0) return 0;
    return or_small_angle(x[o], y[o], x[p], y[p], x[q], y[q]);
}

/* the segments a vertex lies on: the incident segments of an input vertex,
 * the segment a Steiner vertex was placed on (vseg), else none */
static int segs_of(const seg_adj* A, int64_t n_in, const int32_t* vseg, int64_t v, int32_t* out,
                   int cap) {
    if (v < n_in) {
        int n = 0;
        for (int64_t k = A->off[v]; k < A->off[v + 1] && n < cap; ++k) out[n++] = A->adj[k];
        return n;
    }
    if (vseg[v] >= 0) { out[0] = vseg[v]; return 1; }
    return 0;
}

/* C10: a bad triangle (a, b, c) is accepted when its shortest edge joins
 * vertices on two segments that meet at a small input angle.  Where several
 * edges are equally short each one is tried, so the decision does not depend
 * on the order of a, b, c. */
static int exempt_abc(const double* x, const double* y, const int32_t* seg, int64_t nseg,
                      const seg_adj* A, int64_t n_in, const int32_t* vseg, const int64_t v[3]) {
    if (nseg < 2) return 0;
    double l[3];
    for (int e = 0; e < 3; ++e) {
        int64_t a = v[(e + 1) % 3], b = v[(e + 2) % 3];
        double dx = x[b] - x[a], dy = y[b] - y[a];
        l[e] = dx * dx + dy * dy;
    }
    double best = l[0];
    if (l[1] < best) best = l[1];
    if (l[2] < best) best = l[2];
    for (int e = 0; e < 3; ++e) {
        if (l[e] != best) continue;
        int64_t u = v[(e + 1) % 3], w = v[(e + 2) % 3];
        int32_t su[64], sw[64];
        int nu = segs_of(A, n_in, vseg, u, su, 64), nw = segs_of(A, n_in, vseg, w, sw, 64);
        for (int i = 0; i < nu; ++i)
            for (int j = 0; j < nw; ++j)
                if (small_pair_seg(x, y, seg, su[i], sw[j])) return 1;
    }
    return 0;
}

static int exempt(const or_mesh* M, const seg_adj* A, int64_t t) {
    const int32_t* tv = M->tv + 3 * t;
    int64_t v[3] = {tv[0], tv[1], tv[2]};
    return exempt_abc(M->x, M->y, M->seg, M->nseg, A, M->n_in, M->vseg, v);
}

/* vertex ids as in or_export (the enclosing vertices left out) */
int or_exempt_query(const or_mesh* M, int64_t a, int64_t b, int64_t c) {
    int64_t v[3] = {a, b, c};
    for (int k = 0; k < 3; ++k) {
        if (v[k] < 0 || v[k] >= M->nv - 3) return -1;
        if (v[k] >= M->super0) v[k] += 3;
    }
    seg_adj A;
    build_adj(M, &A);
    int r = exempt_abc(M->x, M->y, M->seg, M->nseg, &A, M->n_in, M->vseg, v);
    free(A.off);
    free(A.adj);
    return r;
}

/* per triangle of a mesh given as arrays: 1 if it is bad (C1) and exempt
 * (C10).  The segment a Steiner vertex lies on is read off the subsegments
 * it ends (sub: (u, v, input segment id) triples). */
void or_eval_exempt(const double* xy, int64_t nv, const int32_t* tri, int64_t nt, const int32_t* sub,
                    int64_t ns, const int32_t* seg_in, int64_t m, int64_t n_in, double B2, int32_t* out) {
    double* x = (double*)malloc(sizeof(double) * (size_t)(nv + 1));
    double* y = (double*)malloc(sizeof(double) * (size_t)(nv + 1));
    int32_t* vseg = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nv + 1));
    for (int64_t k = 0; k < nv; ++k) { x[k] = xy[2 * k]; y[k] = xy[2 * k + 1]; vseg[k] = -1; }
    for (int64_t i = 0; i < ns; ++i)
        for (int k = 0; k < 2; ++k)
            if (sub[3 * i + k] >= n_in) vseg[sub[3 * i + k]] = sub[3 * i + 2];
    or_mesh tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.n_in = n_in;
    tmp.nseg = m;
    tmp.seg = (int32_t*)seg_in;
    seg_adj A;
    build_adj(&tmp, &A);
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t* tv = tri + 3 * t;
        int64_t v[3] = {tv[0], tv[1], tv[2]};
        out[t] = or_is_bad(x[v[0]], y[v[0]], x[v[1]], y[v[1]], x[v[2]], y[v[2]], B2) &&
                 exempt_abc(x, y, seg_in, m, &A, n_in, vseg, v);
    }
    free(A.off);
    free(A.adj);
    free(x);
    free(y);
    free(vseg);
}

/* C6: split point of subsegment ab.  If exactly one endpoint is an input
 * vertex where segments meet at a small angle (apex_a / apex_b), the point
 * sits at the power-of-two distance d from it nearest to half the length L
 * in ratio (concentric shells): with L/2 = m 2^e, m in [1/2, 1), d = 2^(e-1)
 * when m^2 < 1/2 (then L/2 is nearer 2^(e-1) than 2^e in ratio), else 2^e.
 * Otherwise the midpoint. */
void or_split_point(double ax, double ay, double bx, double by, int apex_a, int apex_b, double* px,
                    double* py) {
    if ((apex_a != 0) == (apex_b != 0)) {
        or_midpoint(ax, ay, bx, by, px, py);
        return;
    }
    double ox = apex_a ? ax : bx, oy = apex_a ? ay : by;
    double qx = apex_a ? bx : ax, qy = apex_a ? by : ay;
    double dx = qx - ox, dy = qy - oy;
    double L = sqrt(dx * dx + dy * dy);
    int e;
    double m = frexp(0.5 * L, &e);
    double d = (m * m < 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
    double r = d / L;
    *px = ox + dx * r;
    *py = oy + dy * r;
}

static void split_point(const or_mesh* M, int64_t u, int64_t v, double* px, double* py) {
    int au = (u < M->n_in) && M->apex && M->apex[u];
    int av = (v < M->n_in) && M->apex && M->apex[v];
    or_split_point(M->x[u], M->y[u], M->x[v], M->y[v], au, av, px, py);
}

/* ---------------- work queues ---------------- */
typedef struct { double key; int64_t t; int32_t v[3]; } hent;
typedef struct { hent* a; int64_t n, cap; } heap;

static void hpush(heap* h, hent e) {
    if (h->n + 1 > h->cap) {
        h->cap = h->cap ? 2 * h->cap : 1024;
        h->a = (hent*)realloc(h->a, sizeof(hent) * (size_t)h->cap);
    }
    int64_t i = h->n++;
    h->a[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h->a[p].key >= h->a[i].key) break;
        hent t = h->a[p];
        h->a[p] = h->a[i];
        h->a[i] = t;
        i = p;
    }
}

static hent hpop(heap* h) {
    hent top = h->a[0];
    h->a[0] = h->a[--h->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < h->n && h->a[l].key > h->a[m].key) m = l;
        if (r < h->n && h->a[r].key > h->a[m].key) m = r;
        if (m == i) break;
        hent t = h->a[m];
        h->a[m] = h->a[i];
        h->a[i] = t;
        i = m;
    }
    return top;
}

typedef struct { int64_t u, v; int forced; } sent;
typedef struct { sent* a; int64_t head, n, cap; } fifo;

static void qpush(fifo* q, int64_t u, int64_t v, int forced) {
    if (q->n + 1 > q->cap) {
        int64_t nc = q->cap ? 2 * q->cap : 1024;
        sent* na = (sent*)malloc(sizeof(sent) * (size_t)nc);
        for (int64_t i = 0; i < q->n; ++i) na[i] = q->a[(q->head + i) % q->cap];
        free(q->a);
        q->a = na;
        q->cap = nc;
        q->head = 0;
    }
    q->a[(q->head + q->n) % q->cap] = (sent){u, v, forced};
    ++q->n;
}

static sent qpop(fifo* q) {
    sent s = q->a[q->head];
    q->head = (q->head + 1) % q->cap;
    --q->n;
    return s;
}

typedef struct {
    or_mesh* M;
    seg_adj A;
    double B2;
    double L2;   /* edge-length bound squared, 0 = none */
    int lens;    /* encroachment region: 0 diametral circle (Ruppert), 1 diametral lens (Chew) */
    int order;
    int64_t seq;
    heap H;
    fifo Q;
    int64_t* nt_buf;
    int64_t nt_cap;
} rstate;

static void consider_tri(rstate* S, int64_t t) {
    or_mesh* M = S->M;
    const int32_t* v = M->tv + 3 * t;
    double ax = M->x[v[0]], ay = M->y[v[0]], bx = M->x[v[1]], by = M->y[v[1]];
    double cx = M->x[v[2]], cy = M->y[v[2]];
    const int lng = S->L2 > 0 && or_is_long(ax, ay, bx, by, cx, cy, S->L2);
    if (!lng) {
        if (!or_is_bad(ax, ay, bx, by, cx, cy, S->B2)) return;
        if (exempt(M, &S->A, t)) return;
    }
    hent e;
    e.t = t;
    e.v[0] = v[0];
    e.v[1] = v[1];
    e.v[2] = v[2];
    if (S->order == 0) e.key = or_ratio_key(ax, ay, bx, by, cx, cy);
    else if (S->order == 1) e.key = -(double)(S->seq++);
    else e.key = or_tri_measure(ax, ay, bx, by, cx, cy);
    hpush(&S->H, e);
}

/* new triangles: queue the bad ones and re-check their subsegments */
static void after_insert(rstate* S, int64_t nn) {
    or_mesh* M = S->M;
    for (int64_t i = 0; i < nn; ++i) {
        int64_t t = S->nt_buf[i];
        consider_tri(S, t);
        const int32_t* v = M->tv + 3 * t;
        for (int e = 0; e < 3; ++e) {
            int64_t a = v[(e + 1) % 3], b = v[(e + 2) % 3];
            if (or_is_sub(M, a, b)) qpush(&S->Q, a, b, 0);
        }
    }
}

/* p strictly inside the encroachment region of ab: the diametral circle
 * (Ruppert's rule, C2) or the diametral lens (Chew's rule, C22), Sec. 4.2 */
static int inside_region(const rstate* S, double ax, double ay, double bx, double by, double px,
                         double py) {
    return S->lens ? or_lens_sign(ax, ay, bx, by, px, py) < 0 : or_dot_sign(ax, ay, bx, by, px, py) < 0;
}

/* C2: encroached iff the apex of an adjacent triangle is strictly inside the
 * encroachment region */
static int encroached(const rstate* S, int64_t u, int64_t v) {
    const or_mesh* M = S->M;
    int64_t ts[2] = {or_map_get(&M->edges, or_dkey(u, v)), or_map_get(&M->edges, or_dkey(v, u))};
    for (int k = 0; k < 2; ++k) {
        int64_t t = ts[k];
        if (t < 0) continue;
        const int32_t* tv = M->tv + 3 * t;
        for (int j = 0; j < 3; ++j) {
            int64_t w = tv[j];
            if (w == u || w == v) continue;
            if (inside_region(S, M->x[u], M->y[u], M->x[v], M->y[v], M->x[w], M->y[w])) return 1;
        }
    }
    return 0;
}

static int split_sub(rstate* S, int64_t u, int64_t v) {
    or_mesh* M = S->M;
    double px, py;
    split_point(M, u, v, &px, &py);
    int32_t sid = (int32_t)or_map_get(&M->subs, or_ukey(u, v));
    int64_t p = or_add_vertex(M, px, py, sid);
    int64_t nn = or_insert_vertex(M, p, -1, u, v, &S->nt_buf, &S->nt_cap);
    if (nn < 0) { M->nv--; return OR_INTERNAL; }
    M->n_steiner++;
    after_insert(S, nn);
    return OR_OK;
}

int or_refine(or_mesh* M, double B, int64_t max_steiner, int order) {
    return or_refine_len(M, B, 0.0, max_steiner, order);
}

int or_refine_len(or_mesh* M, double B, double l, int64_t max_steiner, int order) {
    return or_refine_mode(M, B, l, 0, max_steiner, order);
}

int or_refine_mode(or_mesh* M, double B, double l, int lens, int64_t max_steiner, int order) {
    rstate S;
    memset(&S, 0, sizeof(S));
    S.M = M;
    S.B2 = B * B;
    S.L2 = l > 0 ? l * l : 0.0;
    S.lens = lens ? 1 : 0;
    S.order = order;
    build_adj(M, &S.A);
    int status = OR_OK;
    for (int64_t i = 0; i < M->subs.cap; ++i) {
        if (M->subs.keys[i] == UINT64_MAX) continue;
        qpush(&S.Q, (int64_t)(M->subs.keys[i] >> 32), (int64_t)(M->subs.keys[i] & 0xffffffffu), 0);
    }
    for (int64_t t = 0; t < M->nt; ++t)
        if (M->alive[t]) consider_tri(&S, t);
    int64_t* ctris = NULL;
    int64_t ccap = 0, *cbnd = NULL, cbcap = 0;
    for (;;) {
        while (S.Q.n > 0) {
            sent s = qpop(&S.Q);
            if (!or_is_sub(M, s.u, s.v)) continue;
            if (!s.forced && !encroached(&S, s.u, s.v)) continue;
            if (M->n_steiner >= max_steiner) { status = OR_LIMIT; goto done; }
            status = split_sub(&S, s.u, s.v);
            if (status != OR_OK) goto done;
        }
        int64_t t = -1;
        while (S.H.n > 0) {
            hent e = hpop(&S.H);
            const int32_t* v = M->tv + 3 * e.t;
            if (!M->alive[e.t] || v[0] != e.v[0] || v[1] != e.v[1] || v[2] != e.v[2]) continue;
            t = e.t;
            break;
        }
        if (t < 0) break;
        if (M->n_steiner >= max_steiner) { status = OR_LIMIT; goto done; }
        const int32_t* v = M->tv + 3 * t;
        double cx, cy;
        or_circumcenter(M->x[v[0]], M->y[v[0]], M->x[v[1]], M->y[v[1]], M->x[v[2]], M->y[v[2]],
                        &cx, &cy);
        int64_t su = -1, sv = -1;
        int64_t tl = or_locate(M, t, cx, cy, 1, &su, &sv);
        if (tl == -2) { status = OR_INTERNAL; goto done; }
        if (tl < 0) {
            qpush(&S.Q, su, sv, 1);
            consider_tri(&S, t);
            continue;
        }
        int64_t nb = 0;
        or_cavity(M, cx, cy, tl, -1, &ctris, &ccap, &cbnd, &nb, &cbcap);
        int enc = 0;
        for (int64_t i = 0; i < nb; ++i) {
            int64_t a = cbnd[2 * i], b = cbnd[2 * i + 1];
            if (!or_is_sub(M, a, b)) continue;
            if (inside_region(&S, M->x[a], M->y[a], M->x[b], M->y[b], cx, cy)) {
                qpush(&S.Q, a, b, 1);
                enc = 1;
            }
        }
        if (enc) {
            consider_tri(&S, t);
            continue;
        }
        int64_t p = or_add_vertex(M, cx, cy, -1);
        int64_t nn = or_insert_vertex(M, p, tl, -1, -1, &S.nt_buf, &S.nt_cap);
        if (nn < 0) { M->nv--; status = OR_INTERNAL; goto done; }
        M->n_steiner++;
        after_insert(&S, nn);
    }
done:
    free(ctris);
    free(cbnd);
    free(S.H.a);
    free(S.Q.a);
    free(S.nt_buf);
    free(S.A.off);
    free(S.A.adj);
    return status;
}

/* ---------------- fixed batches (parity of the insertion kernels) ---------------- */
int or_insert_points(or_mesh* M, const double* xy, int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        double px = xy[2 * i], py = xy[2 * i + 1];
        int64_t t = or_locate(M, M->last_tri, px, py, 0, NULL, NULL);
        if (t < 0) return OR_INPUT;
        const int32_t* v = M->tv + 3 * t;
        for (int e = 0; e < 3; ++e) {
            int64_t a = v[(e + 1) % 3], b = v[(e + 2) % 3];
            if (M->x[v[e]] == px && M->y[v[e]] == py) return OR_INPUT;
            if (or_is_sub(M, a, b) &&
                or_orient(M->x[a], M->y[a], M->x[b], M->y[b], px, py) == 0)
                return OR_INPUT;
        }
        int64_t p = or_add_vertex(M, px, py, -1);
        if (or_insert_vertex(M, p, t, -1, -1, NULL, NULL) < 0) { M->nv--; return OR_INTERNAL; }
        M->n_steiner++;
    }
    return OR_OK;
}

int or_split_subsegments(or_mesh* M, const double* abxy, int64_t n) {
    or_map pos;
    or_map_init(&pos, 2 * M->nv + 16);
    for (int64_t v = 0; v < M->nv; ++v) {
        uint64_t kx, ky;
        memcpy(&kx, &M->x[v], 8);
        memcpy(&ky, &M->y[v], 8);
        or_map_put(&pos, kx * 0x9e3779b97f4a7c15ULL ^ ky, v);
    }
    int st = OR_OK;
    for (int64_t i = 0; i < n && st == OR_OK; ++i) {
        int64_t ids[2];
        for (int k = 0; k < 2; ++k) {
            uint64_t kx, ky;
            memcpy(&kx, &abxy[4 * i + 2 * k], 8);
            memcpy(&ky, &abxy[4 * i + 2 * k + 1], 8);
            ids[k] = or_map_get(&pos, kx * 0x9e3779b97f4a7c15ULL ^ ky);
        }
        for (int k = 0; k < 2; ++k)
            if (ids[k] >= 0 && (M->x[ids[k]] != abxy[4 * i + 2 * k] ||
                                M->y[ids[k]] != abxy[4 * i + 2 * k + 1]))
                ids[k] = -1;
        if (ids[0] < 0 || ids[1] < 0 || !or_is_sub(M, ids[0], ids[1])) { st = OR_INPUT; break; }
        double px, py;
        split_point(M, ids[0], ids[1], &px, &py);
        int32_t sid = (int32_t)or_map_get(&M->subs, or_ukey(ids[0], ids[1]));
        int64_t p = or_add_vertex(M, px, py, sid);
        uint64_t kx, ky;
        memcpy(&kx, &px, 8);
        memcpy(&ky, &py, 8);
        or_map_put(&pos, kx * 0x9e3779b97f4a7c15ULL ^ ky, p);
        if (or_insert_vertex(M, p, -1, ids[0], ids[1], NULL, NULL) < 0) { M->nv--; st = OR_INTERNAL; }
        else M->n_steiner++;
    }
    or_map_free(&pos);
    return st;
}
