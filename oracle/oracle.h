/*
 * Sequential CPU oracle for constrained Delaunay refinement (gDP2d, Sec. 4).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this code: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code with the CUDA path.
 *
 * What it computes, and where the paper defines it:
 *   - PSLG, triangulation, subsegment, CDT ........ Sec. 4 (definitions)
 *   - bad triangle (radius-edge ratio form) ....... Sec. 4.1 / Sec. 5.1
 *   - encroachment (diametral circle, Ruppert;
 *     diametral lens, Chew) ...................... Sec. 4.2
 *   - splitting points (midpoint / circumcentre) .. Sec. 4.2, Algorithm 1
 *   - priorities (midpoint first, larger first) ... Sec. 4.3
 *   - exact predicates + simulation of simplicity . Sec. 7 (set-up)
 *   - cavity (Bowyer-Watson) insertion ............ Sec. 5.2
 * The refinement loop is plain sequential Ruppert: encroached subsegments
 * first (FIFO), then one bad triangle at a time (worst ratio first).
 */
#ifndef GDP_ORACLE_H
#define GDP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (same meaning as the library's, but defined independently) */
enum { OR_OK = 0, OR_INPUT = 1, OR_NOMEM = 2, OR_LIMIT = 3, OR_INTERNAL = 5 };

/* ---------------- exact arithmetic (exact.c) ---------------- */
/* One monomial: sign * f[0] * ... * f[k-1], 1 <= k <= 4. */
typedef struct { int sign; int k; double f[4]; } or_mono;
/* Exact sign (-1, 0, +1) of a sum of monomials, by big-integer evaluation. */
int or_exact_sign(const or_mono* m, int n);

/* ---------------- predicates (pred.c) ---------------- */
void or_set_filter(int enabled);             /* 1 = float filter first (default) */
int  or_orient(double ax, double ay, double bx, double by, double cx, double cy);
int  or_incircle(double ax, double ay, double bx, double by, double cx, double cy,
                 double dx, double dy);
int  or_incircle_sos(double ax, double ay, double bx, double by, double cx, double cy,
                     double dx, double dy);
int  or_dot_sign(double ax, double ay, double bx, double by, double px, double py);
/* -1: p strictly inside the diametral lens of ab (the segment subtends more
 * than 120 degrees at p; Chew's rule, Sec. 4.2), 0: p is a or b, +1: outside */
int  or_lens_sign(double ax, double ay, double bx, double by, double px, double py);
int  or_lex_less(double ax, double ay, double bx, double by);

/* ---------------- FP64 geometry with a fixed evaluation order (pred.c) ---- */
int    or_is_bad(double ax, double ay, double bx, double by, double cx, double cy,
                 double B2);
int    or_is_long(double ax, double ay, double bx, double by, double cx, double cy,
                  double L2);
double or_ratio_key(double ax, double ay, double bx, double by, double cx, double cy);
void   or_circumcenter(double ax, double ay, double bx, double by, double cx, double cy,
                       double* ox, double* oy);
void   or_midpoint(double ax, double ay, double bx, double by, double* ox, double* oy);
uint32_t or_measure_bits(double v);          /* top 31 bits of float32(v), v >= 0 */
double or_tri_measure(double ax, double ay, double bx, double by, double cx, double cy);
double or_seg_measure(double ax, double ay, double bx, double by);

/* ---------------- mesh (mesh.c, cdt.c, ruppert.c) ---------------- */
typedef struct or_mesh or_mesh;

or_mesh* or_cdt_create(const double* xy, int64_t n, const int32_t* seg, int64_t m,
                       int* status);
void     or_destroy(or_mesh*);
/* order: 0 = worst ratio first, 1 = FIFO, 2 = largest area first */
int      or_refine(or_mesh*, double B, int64_t max_steiner, int order);
/* the same with the edge-length bound l of Sec. 4.1 as well (l <= 0: none):
 * a triangle whose longest edge exceeds l is refined like a bad one (the
 * small-angle exemption covers only the radius-edge test) */
int      or_refine_len(or_mesh*, double B, double l, int64_t max_steiner, int order);
/* the same with the encroachment region chosen: lens = 0 the diametral circle
 * (Ruppert's rule), lens != 0 the diametral lens (Chew's rule), Sec. 4.2 */
int      or_refine_mode(or_mesh*, double B, double l, int lens, int64_t max_steiner, int order);
/* C6: split point of subsegment ab -- the midpoint, or, when exactly one
 * endpoint is an apex (an input vertex where segments meet below 60 degrees),
 * the point at the power-of-two distance from it nearest to half the length
 * in ratio (concentric shells) */
void     or_split_point(double ax, double ay, double bx, double by, int apex_a, int apex_b,
                        double* px, double* py);
/* 1 iff the angle at o between the directions to p and q is below 60 degrees */
int      or_small_angle(double ox, double oy, double px, double py, double qx, double qy);
/* C10 on vertices a, b, c of a mesh (ids as in or_export, not necessarily a
 * triangle of it): 1 if the shortest edge -- each of them on a tie -- joins
 * vertices on two segments meeting at a small input angle; -1 bad id */
int      or_exempt_query(const or_mesh*, int64_t a, int64_t b, int64_t c);
/* per triangle of a mesh given as arrays (sub: (u, v, input segment) triples,
 * seg_in over the first n_in vertices): 1 if bad (C1) and exempt (C10) */
void     or_eval_exempt(const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
                        const int32_t* sub, int64_t ns, const int32_t* seg_in, int64_t m,
                        int64_t n_in, double B2, int32_t* out);
/* insert free points (strictly inside the domain, not on a subsegment) */
int      or_insert_points(or_mesh*, const double* xy, int64_t n);
/* split the subsegments given by endpoint coordinates (ax,ay,bx,by) at their
 * split points (or_split_point: midpoint, or a concentric-shell point next to
 * a small input angle) */
int      or_split_subsegments(or_mesh*, const double* abxy, int64_t n);
/* bad list of the current mesh: per live triangle / subsegment (see C API) */
int64_t  or_n_vertices(const or_mesh*);
int64_t  or_n_triangles(const or_mesh*);
int64_t  or_n_subsegments(const or_mesh*);
int64_t  or_n_steiner(const or_mesh*);
/* vertex ids in export: input points 0..n-1, then Steiner points in order */
void     or_export(const or_mesh*, double* xy, int32_t* tri, int32_t* sub);

/* ---------------- invariant checker (check.c) ---------------- */
typedef struct {
    int64_t n_tri, n_vert, n_sub;
    int64_t bad_orient;        /* triangles not strictly CCW (exact) */
    int64_t bad_adjacency;     /* directed edge used twice, or edge in > 2 triangles */
    int64_t open_not_sub;      /* boundary edges that are not subsegments */
    int64_t sub_not_edge;      /* subsegments that are not mesh edges */
    int64_t seg_not_covered;   /* input segments not a chain of subsegments */
    int64_t not_locally_cd;    /* non-constrained interior edges failing incircle (SoS) */
    int64_t bf_cd_violations;  /* brute force: visible vertex inside a circumcircle */
    int64_t bad_quality;       /* non-exempt triangles with ratio above B */
    int64_t exempt_bad;        /* bad triangles exempted by the small-angle rule */
    int64_t encroached;        /* subsegments with a visible vertex strictly inside */
    int64_t euler_defect;      /* V - E + F - 1 (0 for a disk) */
    int64_t inputs_missing;    /* input points not found at their ids */
    double  min_angle_deg;     /* over non-exempt triangles */
    double  area_sum;          /* sum of triangle areas */
    double  bad_area;          /* area of bad triangles (all) */
} or_report;

/* tri: 3*nt CCW vertex ids; sub: 2*ns vertex ids; seg_in: 2*m input segments
 * over the first n_in vertices.  B2 <= 0 skips the quality checks.
 * brute != 0 adds the O(T*V) empty-circumcircle and encroachment checks. */
int or_check(const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
             const int32_t* sub, int64_t ns, const int32_t* seg_in, int64_t m,
             int64_t n_in, double B2, int brute, or_report* rep);
/* the same with encroachment tested against the diametral lens when lens != 0 */
int or_check_mode(const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
                  const int32_t* sub, int64_t ns, const int32_t* seg_in, int64_t m,
                  int64_t n_in, double B2, int brute, int lens, or_report* rep);

#ifdef __cplusplus
}
#endif
#endif
