/*
 * Internal mesh representation of the oracle.  TEST INFRASTRUCTURE ONLY.
 *
 * Deliberately simple: a triangle is three CCW vertex ids; adjacency is not
 * stored but looked up in a hash map from directed edges (u,v) to the
 * triangle that contains u->v.  Subsegments (Sec. 4: edges of the
 * triangulation that lie on an input segment) live in a second map from the
 * undirected edge to the input segment id.
 */
#ifndef GDP_ORACLE_MESH_INT_H
#define GDP_ORACLE_MESH_INT_H

#include <stdint.h>
#include "oracle.h"

typedef struct {
    uint64_t* keys;
    int64_t* vals;
    int64_t cap;   /* power of two */
    int64_t size;
} or_map;

void    or_map_init(or_map* m, int64_t cap);
void    or_map_free(or_map* m);
void    or_map_put(or_map* m, uint64_t k, int64_t v);
int64_t or_map_get(const or_map* m, uint64_t k);   /* -1 if absent */
void    or_map_del(or_map* m, uint64_t k);

static inline uint64_t or_dkey(int64_t u, int64_t v) {
    return ((uint64_t)(uint32_t)u << 32) | (uint32_t)v;
}
static inline uint64_t or_ukey(int64_t u, int64_t v) {
    return u < v ? or_dkey(u, v) : or_dkey(v, u);
}

struct or_mesh {
    /* vertices */
    double* x;
    double* y;
    int64_t nv, capv;
    int64_t n_in;        /* input points: ids 0..n_in-1 */
    int64_t super0;      /* ids super0..super0+2: enclosing triangle (removed) */
    int32_t* vseg;       /* input segment a Steiner vertex lies on, else -1 */
    int64_t* vtri;       /* some live triangle incident to the vertex */
    /* triangles */
    int32_t* tv;         /* 3 per triangle */
    uint8_t* alive;
    int64_t nt, capt;
    int64_t* freel;      /* free triangle slots */
    int64_t nfree, capfree;
    or_map edges;        /* directed edge -> triangle */
    or_map subs;         /* undirected subsegment -> input segment id */
    /* input segments */
    int32_t* seg;        /* 2 per segment */
    int64_t nseg;
    /* small input angles (C6/C10): per input vertex, 1 if two segments meet
     * there at less than 60 degrees */
    uint8_t* apex;
    /* scratch */
    int64_t* stamp;      /* per triangle, cavity membership stamp */
    int64_t cur_stamp;
    int64_t last_tri;    /* hint for point location */
    int64_t n_steiner;
};

/* mesh.c */
int64_t or_add_vertex(or_mesh* M, double x, double y, int32_t seg);
int64_t or_tri_add(or_mesh* M, int64_t a, int64_t b, int64_t c);
void    or_tri_del(or_mesh* M, int64_t t);
int64_t or_nbr(const or_mesh* M, int64_t t, int e);     /* triangle across edge e */
int     or_is_sub(const or_mesh* M, int64_t u, int64_t v);
int     or_orient_v(const or_mesh* M, int64_t a, int64_t b, int64_t c);
int     or_incircle_v(const or_mesh* M, int64_t t, double px, double py);

/* point location: walk from t towards (px,py).
 * stop_at_sub: a step that would cross a subsegment stops the walk and
 * reports that subsegment in (*su,*sv).  Returns the triangle containing the
 * point (closed), or -1 when blocked / outside. */
int64_t or_locate(or_mesh* M, int64_t t, double px, double py, int stop_at_sub,
                  int64_t* su, int64_t* sv);

/* Bowyer-Watson insertion of vertex p (already added) whose location is t.
 * If (sa,sb) >= 0 the point splits the subsegment (sa,sb), which is then
 * replaced by (sa,p),(p,sb).  The cavity is grown by the exact incircle test
 * (with simulation of simplicity) and never crosses a subsegment.
 * new_tris (optional) receives the created triangles. Returns their count or
 * a negative status. */
int64_t or_insert_vertex(or_mesh* M, int64_t p, int64_t t, int64_t sa, int64_t sb,
                         int64_t** new_tris, int64_t* cap_new);

/* cavity of a point not yet added: fills tris (cavity triangles) and bnd
 * (boundary edges as directed vertex pairs), returns #triangles */
int64_t or_cavity(or_mesh* M, double px, double py, int64_t t, int64_t t2,
                  int64_t** tris, int64_t* capt, int64_t** bnd, int64_t* nb,
                  int64_t* capb);

int  or_insert_segment(or_mesh* M, int64_t a, int64_t b, int32_t sid);

#endif
