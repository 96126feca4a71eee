/*
 * Vectorised helpers for the parity tests: per-element results of the
 * scan / splitting-point steps of Algorithm 1 (Sec. 4.3) evaluated on a
 * mesh given as arrays.  TEST INFRASTRUCTURE ONLY.
 */
#include "mesh_int.h"

#include <stdlib.h>

/* per triangle: bad flag (C1), circumcentre (C5) and priority measure bits (C7) */
void or_eval_tris(const double* xy, const int32_t* tri, int64_t nt, double B2, int32_t* bad,
                  double* cc, uint32_t* meas) {
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t* v = tri + 3 * t;
        double ax = xy[2 * v[0]], ay = xy[2 * v[0] + 1], bx = xy[2 * v[1]], by = xy[2 * v[1] + 1];
        double cx = xy[2 * v[2]], cy = xy[2 * v[2] + 1];
        bad[t] = or_is_bad(ax, ay, bx, by, cx, cy, B2);
        or_circumcenter(ax, ay, bx, by, cx, cy, &cc[2 * t], &cc[2 * t + 1]);
        meas[t] = or_measure_bits(or_tri_measure(ax, ay, bx, by, cx, cy));
    }
}

/* per subsegment (u,v): encroached by an adjacent triangle's apex (C2),
 * midpoint (C4) and measure bits (C7) */
void or_eval_subs_mode(const double* xy, const int32_t* tri, int64_t nt, const int32_t* sub,
                       int64_t ns, int lens, int32_t* enc, double* mid, uint32_t* meas);

void or_eval_subs(const double* xy, const int32_t* tri, int64_t nt, const int32_t* sub,
                  int64_t ns, int32_t* enc, double* mid, uint32_t* meas) {
    or_eval_subs_mode(xy, tri, nt, sub, ns, 0, enc, mid, meas);
}

/* the same with encroachment by the diametral lens when lens != 0 (Chew) */
void or_eval_subs_mode(const double* xy, const int32_t* tri, int64_t nt, const int32_t* sub,
                       int64_t ns, int lens, int32_t* enc, double* mid, uint32_t* meas) {
    or_map dir;
    or_map_init(&dir, 6 * nt + 16);
    for (int64_t t = 0; t < nt; ++t)
        for (int j = 0; j < 3; ++j)
            or_map_put(&dir, or_dkey(tri[3 * t + j], tri[3 * t + (j + 1) % 3]),
                       tri[3 * t + (j + 2) % 3]);
    for (int64_t i = 0; i < ns; ++i) {
        int64_t u = sub[3 * i], v = sub[3 * i + 1];
        int e = 0;
        int64_t ap[2] = {or_map_get(&dir, or_dkey(u, v)), or_map_get(&dir, or_dkey(v, u))};
        for (int k = 0; k < 2; ++k)
            if (ap[k] >= 0 &&
                (lens ? or_lens_sign(xy[2 * u], xy[2 * u + 1], xy[2 * v], xy[2 * v + 1], xy[2 * ap[k]],
                                     xy[2 * ap[k] + 1])
                      : or_dot_sign(xy[2 * u], xy[2 * u + 1], xy[2 * v], xy[2 * v + 1], xy[2 * ap[k]],
                                    xy[2 * ap[k] + 1])) < 0)
                e = 1;
        enc[i] = e;
        or_midpoint(xy[2 * u], xy[2 * u + 1], xy[2 * v], xy[2 * v + 1], &mid[2 * i], &mid[2 * i + 1]);
        meas[i] = or_measure_bits(or_seg_measure(xy[2 * u], xy[2 * u + 1], xy[2 * v], xy[2 * v + 1]));
    }
    or_map_free(&dir);
}
