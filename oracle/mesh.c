/*
 * Oracle triangulation: storage, point location, Bowyer-Watson insertion,
 * segment insertion and construction of the CDT.  TEST INFRASTRUCTURE ONLY.
 *
 * CDT (Sec. 4): a triangulation of the PSLG whose triangles' circumcircles
 * contain no vertex visible from the triangle.  Construction (one plain
 * method among many; the CDT is unique under the simulation of simplicity):
 *   1. all points inserted by Bowyer-Watson into an enclosing triangle,
 *   2. each segment inserted by deleting the triangles it crosses and
 *      re-triangulating the two pseudo-polygons on its sides,
 *   3. triangles reachable from the enclosing triangle without crossing a
 *      segment are removed (the domain is what the segments enclose).
 */
#include "mesh_int.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- hash map: open addressing, linear probing ---------------- */
#define EMPTY_KEY UINT64_MAX

static uint64_t hmix(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

void or_map_init(or_map* m, int64_t cap) {
    int64_t c = 16;
    while (c < cap) c <<= 1;
    m->cap = c;
    m->size = 0;
    m->keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)c);
    m->vals = (int64_t*)malloc(sizeof(int64_t) * (size_t)c);
    for (int64_t i = 0; i < c; ++i) m->keys[i] = EMPTY_KEY;
}

void or_map_free(or_map* m) {
    free(m->keys);
    free(m->vals);
    m->keys = NULL;
    m->vals = NULL;
}

static void map_grow(or_map* m) {
    or_map n;
    or_map_init(&n, m->cap * 2);
    for (int64_t i = 0; i < m->cap; ++i)
        if (m->keys[i] != EMPTY_KEY) or_map_put(&n, m->keys[i], m->vals[i]);
    or_map_free(m);
    *m = n;
}

void or_map_put(or_map* m, uint64_t k, int64_t v) {
    if ((m->size + 1) * 2 > m->cap) map_grow(m);
    uint64_t mask = (uint64_t)m->cap - 1, i = hmix(k) & mask;
    while (m->keys[i] != EMPTY_KEY && m->keys[i] != k) i = (i + 1) & mask;
    if (m->keys[i] == EMPTY_KEY) { m->keys[i] = k; ++m->size; }
    m->vals[i] = v;
}

int64_t or_map_get(const or_map* m, uint64_t k) {
    uint64_t mask = (uint64_t)m->cap - 1, i = hmix(k) & mask;
    while (m->keys[i] != EMPTY_KEY) {
        if (m->keys[i] == k) return m->vals[i];
        i = (i + 1) & mask;
    }
    return -1;
}

/* deletion with backward shift, so no tombstones are needed */
void or_map_del(or_map* m, uint64_t k) {
    uint64_t mask = (uint64_t)m->cap - 1, i = hmix(k) & mask;
    while (m->keys[i] != EMPTY_KEY && m->keys[i] != k) i = (i + 1) & mask;
    if (m->keys[i] == EMPTY_KEY) return;
    --m->size;
    uint64_t j = i;
    for (;;) {
        j = (j + 1) & mask;
        if (m->keys[j] == EMPTY_KEY) break;
        uint64_t h = hmix(m->keys[j]) & mask;
        /* can the entry at j move to the hole at i? (h cyclically outside (i, j]) */
        int move = (i <= j) ? (h <= i || h > j) : (h <= i && h > j);
        if (move) {
            m->keys[i] = m->keys[j];
            m->vals[i] = m->vals[j];
            i = j;
        }
    }
    m->keys[i] = EMPTY_KEY;
}

/* ---------------- storage ---------------- */
#define GROW(ptr, cap, need, type)                                              \
    do {                                                                        \
        if ((need) > (cap)) {                                                   \
            int64_t nc = (cap) ? (cap) : 64;                                    \
            while (nc < (need)) nc *= 2;                                        \
            ptr = (type*)realloc(ptr, sizeof(type) * (size_t)nc);               \
            cap = nc;                                                           \
        }                                                                       \
    } while (0)

int64_t or_add_vertex(or_mesh* M, double x, double y, int32_t seg) {
    if (M->nv + 1 > M->capv) {
        int64_t nc = M->capv ? 2 * M->capv : 64;
        M->x = (double*)realloc(M->x, sizeof(double) * (size_t)nc);
        M->y = (double*)realloc(M->y, sizeof(double) * (size_t)nc);
        M->vseg = (int32_t*)realloc(M->vseg, sizeof(int32_t) * (size_t)nc);
        M->vtri = (int64_t*)realloc(M->vtri, sizeof(int64_t) * (size_t)nc);
        M->capv = nc;
    }
    M->x[M->nv] = x;
    M->y[M->nv] = y;
    M->vseg[M->nv] = seg;
    M->vtri[M->nv] = -1;
    return M->nv++;
}

int64_t or_tri_add(or_mesh* M, int64_t a, int64_t b, int64_t c) {
    int64_t t;
    if (M->nfree > 0) {
        t = M->freel[--M->nfree];
    } else {
        if (M->nt + 1 > M->capt) {
            int64_t nc = M->capt ? 2 * M->capt : 64;
            M->tv = (int32_t*)realloc(M->tv, sizeof(int32_t) * 3 * (size_t)nc);
            M->alive = (uint8_t*)realloc(M->alive, (size_t)nc);
            M->stamp = (int64_t*)realloc(M->stamp, sizeof(int64_t) * (size_t)nc);
            M->capt = nc;
        }
        t = M->nt++;
        M->stamp[t] = 0;
    }
    M->tv[3 * t] = (int32_t)a;
    M->tv[3 * t + 1] = (int32_t)b;
    M->tv[3 * t + 2] = (int32_t)c;
    M->alive[t] = 1;
    or_map_put(&M->edges, or_dkey(a, b), t);
    or_map_put(&M->edges, or_dkey(b, c), t);
    or_map_put(&M->edges, or_dkey(c, a), t);
    M->vtri[a] = t;
    M->vtri[b] = t;
    M->vtri[c] = t;
    M->last_tri = t;
    return t;
}

void or_tri_del(or_mesh* M, int64_t t) {
    int32_t* v = M->tv + 3 * t;
    or_map_del(&M->edges, or_dkey(v[0], v[1]));
    or_map_del(&M->edges, or_dkey(v[1], v[2]));
    or_map_del(&M->edges, or_dkey(v[2], v[0]));
    M->alive[t] = 0;
    GROW(M->freel, M->capfree, M->nfree + 1, int64_t);
    M->freel[M->nfree++] = t;
}

/* edge e of t is (v[e+1], v[e+2]), the edge opposite vertex e */
int64_t or_nbr(const or_mesh* M, int64_t t, int e) {
    const int32_t* v = M->tv + 3 * t;
    return or_map_get(&M->edges, or_dkey(v[(e + 2) % 3], v[(e + 1) % 3]));
}

int or_is_sub(const or_mesh* M, int64_t u, int64_t v) {
    return or_map_get(&M->subs, or_ukey(u, v)) >= 0;
}

int or_orient_v(const or_mesh* M, int64_t a, int64_t b, int64_t c) {
    return or_orient(M->x[a], M->y[a], M->x[b], M->y[b], M->x[c], M->y[c]);
}

int or_incircle_v(const or_mesh* M, int64_t t, double px, double py) {
    const int32_t* v = M->tv + 3 * t;
    return or_incircle_sos(M->x[v[0]], M->y[v[0]], M->x[v[1]], M->y[v[1]], M->x[v[2]],
                           M->y[v[2]], px, py);
}

/* ---------------- point location ---------------- */
int64_t or_locate(or_mesh* M, int64_t t, double px, double py, int stop_at_sub,
                  int64_t* su, int64_t* sv) {
    int64_t steps = 0, limit = 4 * M->nt + 100;
    for (;;) {
        if (++steps > limit) return -2;
        const int32_t* v = M->tv + 3 * t;
        int blocked_e = -1;
        int64_t next = -1;
        for (int e = 0; e < 3 && next < 0; ++e) {
            int64_t a = v[(e + 1) % 3], b = v[(e + 2) % 3];
            if (or_orient(M->x[a], M->y[a], M->x[b], M->y[b], px, py) < 0) {
                if (stop_at_sub && or_is_sub(M, a, b)) {
                    if (blocked_e < 0) blocked_e = e;
                    continue;
                }
                int64_t n = or_nbr(M, t, e);
                if (n < 0) {
                    if (blocked_e < 0) blocked_e = e;
                    continue;
                }
                next = n;
            }
        }
        if (next >= 0) { t = next; continue; }
        if (blocked_e >= 0) {
            if (su) *su = v[(blocked_e + 1) % 3];
            if (sv) *sv = v[(blocked_e + 2) % 3];
            return -1;
        }
        return t;
    }
}

/* ---------------- Bowyer-Watson cavity ---------------- */
int64_t or_cavity(or_mesh* M, double px, double py, int64_t t, int64_t t2,
                  int64_t** tris, int64_t* capt, int64_t** bnd, int64_t* nb,
                  int64_t* capb) {
    int64_t n = 0, nbd = 0;
    ++M->cur_stamp;
    GROW(*tris, *capt, 2, int64_t);
    (*tris)[n++] = t;
    M->stamp[t] = M->cur_stamp;
    if (t2 >= 0) {
        (*tris)[n++] = t2;
        M->stamp[t2] = M->cur_stamp;
    }
    for (int64_t q = 0; q < n; ++q) {
        int64_t c = (*tris)[q];
        const int32_t* v = M->tv + 3 * c;
        for (int e = 0; e < 3; ++e) {
            int64_t a = v[(e + 1) % 3], b = v[(e + 2) % 3];
            int64_t nb_t = or_nbr(M, c, e);
            int inside = 0;
            if (nb_t >= 0 && M->stamp[nb_t] == M->cur_stamp) continue;  /* interior edge */
            if (nb_t >= 0 && !or_is_sub(M, a, b))
                inside = or_incircle_v(M, nb_t, px, py) > 0;
            if (inside) {
                GROW(*tris, *capt, n + 1, int64_t);
                (*tris)[n++] = nb_t;
                M->stamp[nb_t] = M->cur_stamp;
            } else {
                GROW(*bnd, *capb, 2 * (nbd + 1), int64_t);
                (*bnd)[2 * nbd] = a;
                (*bnd)[2 * nbd + 1] = b;
                ++nbd;
            }
        }
    }
    *nb = nbd;
    return n;
}

int64_t or_insert_vertex(or_mesh* M, int64_t p, int64_t t, int64_t sa, int64_t sb,
                         int64_t** new_tris, int64_t* cap_new) {
    int64_t t2 = -1;
    if (sa >= 0) {
        /* the subsegment's two triangles both contain p */
        int64_t ta = or_map_get(&M->edges, or_dkey(sa, sb));
        int64_t tb = or_map_get(&M->edges, or_dkey(sb, sa));
        t = ta >= 0 ? ta : tb;
        t2 = (ta >= 0) ? tb : -1;
    }
    static int64_t* tris = NULL;
    static int64_t capt = 0;
    static int64_t* bnd = NULL;
    static int64_t capb = 0;
    int64_t nb = 0;
    int64_t k = or_cavity(M, M->x[p], M->y[p], t, t2, &tris, &capt, &bnd, &nb, &capb);
    /* every fan triangle must be strictly CCW */
    for (int64_t i = 0; i < nb; ++i) {
        int64_t a = bnd[2 * i], b = bnd[2 * i + 1];
        if (sa >= 0 && ((a == sa && b == sb) || (a == sb && b == sa))) continue;
        if (or_orient_v(M, a, b, p) <= 0) return -OR_INTERNAL;
    }
    for (int64_t i = 0; i < k; ++i) or_tri_del(M, tris[i]);
    int64_t nn = 0;
    for (int64_t i = 0; i < nb; ++i) {
        int64_t a = bnd[2 * i], b = bnd[2 * i + 1];
        if (sa >= 0 && ((a == sa && b == sb) || (a == sb && b == sa))) continue;
        int64_t nt = or_tri_add(M, p, a, b);
        if (new_tris) {
            GROW(*new_tris, *cap_new, nn + 1, int64_t);
            (*new_tris)[nn] = nt;
        }
        ++nn;
    }
    if (sa >= 0) {
        int64_t sid = or_map_get(&M->subs, or_ukey(sa, sb));
        or_map_del(&M->subs, or_ukey(sa, sb));
        or_map_put(&M->subs, or_ukey(sa, p), sid);
        or_map_put(&M->subs, or_ukey(p, sb), sid);
    }
    return nn;
}

/* ---------------- segment insertion ---------------- */

/* Re-triangulate the pseudo-polygon with base u->w and chain c[0..n) (all
 * left of u->w, ordered from u to w): pick the chain vertex whose circle
 * through u, w holds no other chain vertex, emit (u, w, c) and recurse on
 * both sides (the usual recursive CDT of a pseudo-polygon). */
static void tri_pseudo(or_mesh* M, int64_t u, int64_t w, const int64_t* c, int64_t n) {
    if (n <= 0) return;
    int64_t best = 0;
    for (int64_t i = 1; i < n; ++i) {
        int64_t b = c[best];
        if (or_incircle_sos(M->x[u], M->y[u], M->x[w], M->y[w], M->x[b], M->y[b], M->x[c[i]],
                            M->y[c[i]]) > 0)
            best = i;
    }
    or_tri_add(M, u, w, c[best]);
    tri_pseudo(M, u, c[best], c, best);
    tri_pseudo(M, c[best], w, c + best + 1, n - best - 1);
}

int or_insert_segment(or_mesh* M, int64_t a, int64_t b, int32_t sid) {
    if (or_map_get(&M->edges, or_dkey(a, b)) >= 0 || or_map_get(&M->edges, or_dkey(b, a)) >= 0) {
        or_map_put(&M->subs, or_ukey(a, b), sid);
        return OR_OK;
    }
    double ax = M->x[a], ay = M->y[a], bx = M->x[b], by = M->y[b];
    /* find the triangle around a whose opposite edge the segment crosses:
     * rotate around a through the edge map */
    int64_t t0 = M->vtri[a];
    if (t0 < 0 || !M->alive[t0]) return OR_INTERNAL;
    int64_t t = t0, start = -1;
    for (int64_t guard = 0; guard < M->nt + 3; ++guard) {
        const int32_t* v = M->tv + 3 * t;
        int i = (v[0] == a) ? 0 : (v[1] == a) ? 1 : 2;
        int64_t u = v[(i + 1) % 3], w = v[(i + 2) % 3];
        int o1 = or_orient(ax, ay, M->x[u], M->y[u], bx, by);   /* b left of a->u ? */
        int o2 = or_orient(ax, ay, M->x[w], M->y[w], bx, by);
        if (o1 == 0 && or_dot_sign(M->x[u] - ax, M->y[u] - ay, bx - ax, by - ay, 0, 0) > 0)
            return OR_INPUT;                     /* segment runs through vertex u */
        if (o1 > 0 && o2 < 0) { start = t; break; }
        /* next triangle clockwise around a: across edge (a, u) */
        int64_t n = or_map_get(&M->edges, or_dkey(u, a));
        if (n < 0) return OR_INTERNAL;
        t = n;
        if (t == t0) break;
    }
    if (start < 0) return OR_INTERNAL;
    /* walk along a->b collecting crossed triangles and the two chains */
    int64_t *cross = NULL, ncross = 0, capc = 0;
    int64_t *up = NULL, nup = 0, capu = 0, *lo = NULL, nlo = 0, capl = 0;
    t = start;
    {
        const int32_t* v = M->tv + 3 * t;
        int i = (v[0] == a) ? 0 : (v[1] == a) ? 1 : 2;
        int64_t u = v[(i + 1) % 3], w = v[(i + 2) % 3];
        /* u is right of a->b, w is left */
        GROW(lo, capl, nlo + 1, int64_t);
        lo[nlo++] = u;
        GROW(up, capu, nup + 1, int64_t);
        up[nup++] = w;
        GROW(cross, capc, ncross + 1, int64_t);
        cross[ncross++] = t;
        /* crossing edge (u, w) seen from t is u->w; next triangle has w->u */
        int64_t ru = u, lw = w;
        for (int64_t guard = 0; guard < M->nt + 3; ++guard) {
            int64_t n = or_map_get(&M->edges, or_dkey(lw, ru));
            if (n < 0) { free(cross); free(up); free(lo); return OR_INTERNAL; }
            GROW(cross, capc, ncross + 1, int64_t);
            cross[ncross++] = n;
            const int32_t* nv = M->tv + 3 * n;
            int j = (nv[0] == lw) ? 0 : (nv[1] == lw) ? 1 : 2;
            /* n = (lw, ru, z) in CCW order */
            int64_t z = nv[(j + 2) % 3];
            if (z == b) break;
            int o = or_orient(ax, ay, bx, by, M->x[z], M->y[z]);
            if (o == 0) { free(cross); free(up); free(lo); return OR_INPUT; }
            if (o > 0) {
                GROW(up, capu, nup + 1, int64_t);
                up[nup++] = z;
                lw = z;
            } else {
                GROW(lo, capl, nlo + 1, int64_t);
                lo[nlo++] = z;
                ru = z;
            }
        }
    }
    for (int64_t i = 0; i < ncross; ++i) or_tri_del(M, cross[i]);
    /* upper chain lies left of a->b, ordered from a to b */
    tri_pseudo(M, a, b, up, nup);
    /* lower chain lies left of b->a; order it from b to a */
    for (int64_t i = 0; i < nlo / 2; ++i) {
        int64_t tmp = lo[i];
        lo[i] = lo[nlo - 1 - i];
        lo[nlo - 1 - i] = tmp;
    }
    tri_pseudo(M, b, a, lo, nlo);
    or_map_put(&M->subs, or_ukey(a, b), sid);
    free(cross);
    free(up);
    free(lo);
    return OR_OK;
}

/* ---------------- construction ---------------- */

static void mark_apexes(or_mesh* M) {
    M->apex = (uint8_t*)calloc((size_t)M->n_in + 1, 1);
    /* per input vertex, every pair of incident segments is compared; the
     * angle at the shared vertex is below 60 degrees iff cos > 1/2
     * (or_small_angle) -- decided in FP64, this only selects where the
     * small-angle rules apply. */
    int64_t* deg = (int64_t*)calloc((size_t)M->n_in + 1, sizeof(int64_t));
    for (int64_t s = 0; s < M->nseg; ++s) {
        deg[M->seg[2 * s]]++;
        deg[M->seg[2 * s + 1]]++;
    }
    for (int64_t s = 0; s < M->nseg; ++s) {
        for (int end = 0; end < 2; ++end) {
            int64_t o = M->seg[2 * s + end], p = M->seg[2 * s + 1 - end];
            if (deg[o] < 2) continue;
            for (int64_t r = s + 1; r < M->nseg; ++r) {
                int64_t q = -1;
                if (M->seg[2 * r] == o) q = M->seg[2 * r + 1];
                else if (M->seg[2 * r + 1] == o) q = M->seg[2 * r];
                if (q < 0) continue;
                if (or_small_angle(M->x[o], M->y[o], M->x[p], M->y[p], M->x[q], M->y[q])) M->apex[o] = 1;
            }
        }
    }
    free(deg);
}

/* visit order for point insertion: rows of a coarse grid, alternating
 * direction, so consecutive points are close (the walk stays short).  The
 * resulting CDT does not depend on the order. */
static int64_t* grid_order(const double* xy, int64_t n) {
    double x0 = xy[0], x1 = xy[0], y0 = xy[1], y1 = xy[1];
    for (int64_t i = 1; i < n; ++i) {
        if (xy[2 * i] < x0) x0 = xy[2 * i];
        if (xy[2 * i] > x1) x1 = xy[2 * i];
        if (xy[2 * i + 1] < y0) y0 = xy[2 * i + 1];
        if (xy[2 * i + 1] > y1) y1 = xy[2 * i + 1];
    }
    int64_t g = (int64_t)sqrt((double)n / 2.0) + 1;
    int64_t* cnt = (int64_t*)calloc((size_t)(g * g + 1), sizeof(int64_t));
    int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    double wx = (x1 - x0) > 0 ? (x1 - x0) : 1, wy = (y1 - y0) > 0 ? (y1 - y0) : 1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t cx = (int64_t)((xy[2 * i] - x0) / wx * (double)g);
        int64_t cy = (int64_t)((xy[2 * i + 1] - y0) / wy * (double)g);
        if (cx >= g) cx = g - 1;
        if (cy >= g) cy = g - 1;
        if (cx < 0) cx = 0;
        if (cy < 0) cy = 0;
        if (cy % 2) cx = g - 1 - cx;
        cell[i] = cy * g + cx;
        cnt[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < g * g; ++c) cnt[c + 1] += cnt[c];
    int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) ord[cnt[cell[i]]++] = i;
    free(cnt);
    free(cell);
    return ord;
}

void or_destroy(or_mesh* M) {
    if (!M) return;
    free(M->x);
    free(M->y);
    free(M->vseg);
    free(M->vtri);
    free(M->tv);
    free(M->alive);
    free(M->freel);
    free(M->stamp);
    free(M->seg);
    free(M->apex);
    or_map_free(&M->edges);
    or_map_free(&M->subs);
    free(M);
}

or_mesh* or_cdt_create(const double* xy, int64_t n, const int32_t* seg, int64_t m,
                       int* status) {
    *status = OR_OK;
    if (n < 3) { *status = OR_INPUT; return NULL; }
    for (int64_t i = 0; i < 2 * n; ++i)
        if (!isfinite(xy[i])) { *status = OR_INPUT; return NULL; }
    for (int64_t s = 0; s < 2 * m; ++s)
        if (seg[s] < 0 || seg[s] >= n) { *status = OR_INPUT; return NULL; }
    for (int64_t s = 0; s < m; ++s)
        if (seg[2 * s] == seg[2 * s + 1]) { *status = OR_INPUT; return NULL; }
    or_mesh* M = (or_mesh*)calloc(1, sizeof(or_mesh));
    or_map_init(&M->edges, 8 * n + 64);
    or_map_init(&M->subs, 4 * m + 64);
    M->n_in = n;
    for (int64_t i = 0; i < n; ++i) or_add_vertex(M, xy[2 * i], xy[2 * i + 1], -1);
    M->nseg = m;
    M->seg = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m + 2));
    memcpy(M->seg, seg, sizeof(int32_t) * (size_t)(2 * m));
    /* enclosing triangle, far outside the bounding box */
    double x0 = xy[0], x1 = xy[0], y0 = xy[1], y1 = xy[1];
    for (int64_t i = 1; i < n; ++i) {
        x0 = fmin(x0, xy[2 * i]);
        x1 = fmax(x1, xy[2 * i]);
        y0 = fmin(y0, xy[2 * i + 1]);
        y1 = fmax(y1, xy[2 * i + 1]);
    }
    double cx = 0.5 * (x0 + x1), cy = 0.5 * (y0 + y1);
    double D = fmax(x1 - x0, y1 - y0);
    if (!(D > 0)) D = 1;
    M->super0 = M->nv;
    or_add_vertex(M, cx - 64 * D, cy - 64 * D, -1);
    or_add_vertex(M, cx + 64 * D, cy - 64 * D, -1);
    or_add_vertex(M, cx, cy + 64 * D, -1);
    or_tri_add(M, M->super0, M->super0 + 1, M->super0 + 2);
    /* 1. points */
    int64_t* ord = grid_order(xy, n);
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = ord[k];
        int64_t t = or_locate(M, M->last_tri, M->x[i], M->y[i], 0, NULL, NULL);
        if (t < 0) { free(ord); or_destroy(M); *status = OR_INTERNAL; return NULL; }
        /* duplicate point? */
        const int32_t* v = M->tv + 3 * t;
        for (int j = 0; j < 3; ++j)
            if (M->x[v[j]] == M->x[i] && M->y[v[j]] == M->y[i]) {
                free(ord);
                or_destroy(M);
                *status = OR_INPUT;
                return NULL;
            }
        if (or_insert_vertex(M, i, t, -1, -1, NULL, NULL) < 0) {
            free(ord);
            or_destroy(M);
            *status = OR_INTERNAL;
            return NULL;
        }
    }
    free(ord);
    /* 2. segments (crossing input segments show up as a failed walk or a
     * segment that runs through a vertex) */
    for (int64_t s = 0; s < m; ++s) {
        int64_t a = seg[2 * s], b = seg[2 * s + 1];
        if (or_is_sub(M, a, b)) { *status = OR_INPUT; or_destroy(M); return NULL; }
        int st = or_insert_segment(M, a, b, (int32_t)s);
        if (st != OR_OK) { or_destroy(M); *status = OR_INPUT; return NULL; }
    }
    /* a segment crossing an earlier one would have removed its subsegment */
    for (int64_t s = 0; s < m; ++s) {
        int64_t a = seg[2 * s], b = seg[2 * s + 1];
        if (or_map_get(&M->edges, or_dkey(a, b)) < 0 && or_map_get(&M->edges, or_dkey(b, a)) < 0) {
            or_destroy(M);
            *status = OR_INPUT;
            return NULL;
        }
        if (or_map_get(&M->subs, or_ukey(a, b)) != s) { or_destroy(M); *status = OR_INPUT; return NULL; }
    }
    /* 3. exterior: flood from triangles touching the enclosing vertices */
    int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)(M->nt + 1));
    uint8_t* ext = (uint8_t*)calloc((size_t)M->nt + 1, 1);
    int64_t ns = 0;
    for (int64_t t = 0; t < M->nt; ++t) {
        if (!M->alive[t]) continue;
        const int32_t* v = M->tv + 3 * t;
        if (v[0] >= M->super0 || v[1] >= M->super0 || v[2] >= M->super0) {
            ext[t] = 1;
            stack[ns++] = t;
        }
    }
    while (ns > 0) {
        int64_t t = stack[--ns];
        const int32_t* v = M->tv + 3 * t;
        for (int e = 0; e < 3; ++e) {
            int64_t a = v[(e + 1) % 3], b = v[(e + 2) % 3];
            if (or_is_sub(M, a, b)) continue;
            int64_t nb_t = or_nbr(M, t, e);
            if (nb_t >= 0 && !ext[nb_t]) {
                ext[nb_t] = 1;
                stack[ns++] = nb_t;
            }
        }
    }
    for (int64_t t = 0; t < M->nt; ++t)
        if (M->alive[t] && ext[t]) or_tri_del(M, t);
    free(stack);
    free(ext);
    for (int64_t v = 0; v < M->nv; ++v) M->vtri[v] = -1;
    int64_t live = 0;
    for (int64_t t = 0; t < M->nt; ++t) {
        if (!M->alive[t]) continue;
        ++live;
        M->last_tri = t;
        for (int j = 0; j < 3; ++j) M->vtri[M->tv[3 * t + j]] = t;
    }
    if (live == 0) { or_destroy(M); *status = OR_INPUT; return NULL; }
    mark_apexes(M);
    return M;
}

int64_t or_n_vertices(const or_mesh* M) { return M->nv - 3; }
int64_t or_n_triangles(const or_mesh* M) {
    int64_t c = 0;
    for (int64_t t = 0; t < M->nt; ++t) c += M->alive[t];
    return c;
}
int64_t or_n_subsegments(const or_mesh* M) { return M->subs.size; }
int64_t or_n_steiner(const or_mesh* M) { return M->n_steiner; }

/* export ids: input points keep 0..n_in-1, the enclosing vertices are
 * dropped, Steiner points follow in insertion order */
static int64_t ex_id(const or_mesh* M, int64_t v) { return v < M->super0 ? v : v - 3; }

void or_export(const or_mesh* M, double* xy, int32_t* tri, int32_t* sub) {
    if (xy) {
        int64_t k = 0;
        for (int64_t v = 0; v < M->nv; ++v) {
            if (v >= M->super0 && v < M->super0 + 3) continue;
            xy[2 * k] = M->x[v];
            xy[2 * k + 1] = M->y[v];
            ++k;
        }
    }
    if (tri) {
        int64_t k = 0;
        for (int64_t t = 0; t < M->nt; ++t) {
            if (!M->alive[t]) continue;
            for (int j = 0; j < 3; ++j) tri[3 * k + j] = (int32_t)ex_id(M, M->tv[3 * t + j]);
            ++k;
        }
    }
    if (sub) {
        int64_t k = 0;
        for (int64_t i = 0; i < M->subs.cap; ++i) {
            if (M->subs.keys[i] == UINT64_MAX) continue;
            int64_t u = (int64_t)(M->subs.keys[i] >> 32), v = (int64_t)(M->subs.keys[i] & 0xffffffffu);
            sub[3 * k] = (int32_t)ex_id(M, u);
            sub[3 * k + 1] = (int32_t)ex_id(M, v);
            sub[3 * k + 2] = (int32_t)M->subs.vals[i];
            ++k;
        }
    }
}
