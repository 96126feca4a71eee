/*
 * Invariant checker for any triangulation given as plain arrays (the
 * oracle's own output or the CUDA path's export).  TEST INFRASTRUCTURE ONLY.
 *
 * Checked properties (Sec. 4 definitions and the termination state of
 * Algorithm 1):
 *   - every triangle strictly CCW (exact orient);
 *   - a manifold: each directed edge used once, open edges are subsegments;
 *   - every input segment is the union of a chain of subsegments;
 *   - constrained Delaunay: every non-subsegment interior edge is locally
 *     Delaunay (exact incircle with simulation of simplicity) and, with
 *     brute != 0, no vertex visible from a triangle lies inside its circle;
 *   - quality: no triangle has radius-edge ratio above B, except those whose
 *     shortest edge joins two segments meeting at a small input angle;
 *   - no subsegment is encroached (apex of an adjacent triangle strictly
 *     inside its diametral circle);
 *   - Euler characteristic of a disk.
 */
#include "mesh_int.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int crosses(const double* xy, int64_t p, int64_t q, double gx, double gy, int64_t w) {
    /* proper crossing of segment (g,w) with segment (p,q) */
    double px = xy[2 * p], py = xy[2 * p + 1], qx = xy[2 * q], qy = xy[2 * q + 1];
    double wx = xy[2 * w], wy = xy[2 * w + 1];
    int o1 = or_orient(gx, gy, wx, wy, px, py), o2 = or_orient(gx, gy, wx, wy, qx, qy);
    int o3 = or_orient(px, py, qx, qy, gx, gy), o4 = or_orient(px, py, qx, qy, wx, wy);
    return o1 * o2 < 0 && o3 * o4 < 0;
}

static int small_pair_xy(const double* xy, const int32_t* seg, int64_t s1, int64_t s2) {
    if (s1 == s2) return 0;
    const int32_t* a = seg + 2 * s1;
    const int32_t* b = seg + 2 * s2;
    int64_t o = -1, p = -1, q = -1;
    for (int i = 0; i < 2 && o < 0; ++i)
        for (int j = 0; j < 2; ++j)
            if (a[i] == b[j]) { o = a[i]; p = a[1 - i]; q = b[1 - j]; break; }
    if (o < 0) return 0;
    double ux = xy[2 * p] - xy[2 * o], uy = xy[2 * p + 1] - xy[2 * o + 1];
    double wx = xy[2 * q] - xy[2 * o], wy = xy[2 * q + 1] - xy[2 * o + 1];
    double dot = ux * wx + uy * wy;
    double nn = sqrt(ux * ux + uy * uy) * sqrt(wx * wx + wy * wy);
    return 2.0 * dot > nn;
}

int or_check(const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
             const int32_t* sub, int64_t ns, const int32_t* seg_in, int64_t m,
             int64_t n_in, double B2, int brute, or_report* rep) {
    return or_check_mode(xy, nv, tri, nt, sub, ns, seg_in, m, n_in, B2, brute, 0, rep);
}

int or_check_mode(const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
                  const int32_t* sub, int64_t ns, const int32_t* seg_in, int64_t m,
                  int64_t n_in, double B2, int brute, int lens, or_report* rep) {
    memset(rep, 0, sizeof(*rep));
    rep->n_tri = nt;
    rep->n_vert = nv;
    rep->n_sub = ns;
    rep->min_angle_deg = 180.0;
    or_map dir, und, subs;
    or_map_init(&dir, 6 * nt + 16);
    or_map_init(&und, 6 * nt + 16);
    or_map_init(&subs, 2 * ns + 16);
    for (int64_t i = 0; i < ns; ++i) or_map_put(&subs, or_ukey(sub[3 * i], sub[3 * i + 1]), sub[3 * i + 2]);
    uint8_t* used = (uint8_t*)calloc((size_t)nv + 1, 1);
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t* v = tri + 3 * t;
        for (int j = 0; j < 3; ++j) {
            if (v[j] < 0 || v[j] >= nv) { rep->bad_adjacency++; continue; }
            used[v[j]] = 1;
        }
        if (or_orient(xy[2 * v[0]], xy[2 * v[0] + 1], xy[2 * v[1]], xy[2 * v[1] + 1], xy[2 * v[2]],
                      xy[2 * v[2] + 1]) <= 0)
            rep->bad_orient++;
        for (int j = 0; j < 3; ++j) {
            uint64_t k = or_dkey(v[j], v[(j + 1) % 3]);
            if (or_map_get(&dir, k) >= 0) rep->bad_adjacency++;
            or_map_put(&dir, k, t * 3 + (j + 2) % 3);   /* value: tri*3 + opposite corner */
            or_map_put(&und, or_ukey(v[j], v[(j + 1) % 3]), 1);
        }
        double ax = xy[2 * v[0]], ay = xy[2 * v[0] + 1], bx = xy[2 * v[1]], by = xy[2 * v[1] + 1];
        double cx = xy[2 * v[2]], cy = xy[2 * v[2] + 1];
        rep->area_sum += 0.5 * ((bx - ax) * (cy - ay) - (by - ay) * (cx - ax));
    }
    for (int64_t i = 0; i < n_in && i < nv; ++i)
        if (!used[i]) rep->inputs_missing++;
    int64_t vused = 0;
    for (int64_t i = 0; i < nv; ++i) vused += used[i];
    rep->euler_defect = vused - und.size + nt - 1;
    /* subsegments must be edges */
    for (int64_t i = 0; i < ns; ++i)
        if (or_map_get(&und, or_ukey(sub[3 * i], sub[3 * i + 1])) < 0) rep->sub_not_edge++;
    /* incident subsegments per vertex (for the segment chains) */
    int64_t* off = (int64_t*)calloc((size_t)nv + 2, sizeof(int64_t));
    int64_t* adj = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * ns + 1));
    for (int64_t i = 0; i < ns; ++i) { off[sub[3 * i] + 1]++; off[sub[3 * i + 1] + 1]++; }
    for (int64_t v = 0; v < nv; ++v) off[v + 1] += off[v];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nv + 1));
    memcpy(fill, off, sizeof(int64_t) * (size_t)(nv + 1));
    for (int64_t i = 0; i < ns; ++i) { adj[fill[sub[3 * i]]++] = i; adj[fill[sub[3 * i + 1]]++] = i; }
    free(fill);
    for (int64_t s = 0; s < m; ++s) {
        int64_t a = seg_in[2 * s], b = seg_in[2 * s + 1], cur = a, prev_sub = -1, steps = 0;
        int ok = 0;
        while (steps++ <= ns) {
            int64_t next_sub = -1;
            for (int64_t k = off[cur]; k < off[cur + 1]; ++k) {
                int64_t i = adj[k];
                if (i != prev_sub && sub[3 * i + 2] == s) { next_sub = i; break; }
            }
            if (next_sub < 0) break;
            cur = (sub[3 * next_sub] == cur) ? sub[3 * next_sub + 1] : sub[3 * next_sub];
            prev_sub = next_sub;
            if (cur == b) { ok = 1; break; }
        }
        if (!ok) rep->seg_not_covered++;
    }
    /* per-edge checks */
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t* v = tri + 3 * t;
        for (int j = 0; j < 3; ++j) {
            int64_t u = v[j], w = v[(j + 1) % 3], apex = v[(j + 2) % 3];
            int is_sub = or_map_get(&subs, or_ukey(u, w)) >= 0;
            int64_t o = or_map_get(&dir, or_dkey(w, u));
            if (o < 0) {
                if (!is_sub) rep->open_not_sub++;
            } else if (!is_sub && u < w) {
                int64_t other = tri[o];   /* value encodes tri*3+corner; tri[] is flat */
                if (or_incircle_sos(xy[2 * v[0]], xy[2 * v[0] + 1], xy[2 * v[1]], xy[2 * v[1] + 1],
                                    xy[2 * v[2]], xy[2 * v[2] + 1], xy[2 * other],
                                    xy[2 * other + 1]) > 0)
                    rep->not_locally_cd++;
            }
            if (is_sub &&
                (lens ? or_lens_sign(xy[2 * u], xy[2 * u + 1], xy[2 * w], xy[2 * w + 1], xy[2 * apex],
                                     xy[2 * apex + 1])
                      : or_dot_sign(xy[2 * u], xy[2 * u + 1], xy[2 * w], xy[2 * w + 1], xy[2 * apex],
                                    xy[2 * apex + 1])) < 0)
                rep->encroached++;
        }
    }
    /* quality with the small-angle exemption */
    if (B2 > 0) {
        /* input vertex -> incident input segments */
        int64_t* soff = (int64_t*)calloc((size_t)n_in + 2, sizeof(int64_t));
        int64_t* sadj = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
        for (int64_t s = 0; s < m; ++s) { soff[seg_in[2 * s] + 1]++; soff[seg_in[2 * s + 1] + 1]++; }
        for (int64_t v = 0; v < n_in; ++v) soff[v + 1] += soff[v];
        int64_t* sf = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_in + 1));
        memcpy(sf, soff, sizeof(int64_t) * (size_t)(n_in + 1));
        for (int64_t s = 0; s < m; ++s) { sadj[sf[seg_in[2 * s]]++] = s; sadj[sf[seg_in[2 * s + 1]]++] = s; }
        free(sf);
        /* Steiner vertex -> its segment, from the subsegments it ends */
        int32_t* vseg = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nv + 1));
        for (int64_t v = 0; v < nv; ++v) vseg[v] = -1;
        for (int64_t i = 0; i < ns; ++i)
            for (int k = 0; k < 2; ++k)
                if (sub[3 * i + k] >= n_in) vseg[sub[3 * i + k]] = sub[3 * i + 2];
        for (int64_t t = 0; t < nt; ++t) {
            const int32_t* v = tri + 3 * t;
            double ax = xy[2 * v[0]], ay = xy[2 * v[0] + 1], bx = xy[2 * v[1]], by = xy[2 * v[1] + 1];
            double cx = xy[2 * v[2]], cy = xy[2 * v[2] + 1];
            int bad = or_is_bad(ax, ay, bx, by, cx, cy, B2);
            int ex = 0;
            if (bad) {
                rep->bad_area += 0.5 * fabs((bx - ax) * (cy - ay) - (by - ay) * (cx - ax));
                double best = -1;
                int be = 0;
                for (int e = 0; e < 3; ++e) {
                    int64_t a = v[(e + 1) % 3], b = v[(e + 2) % 3];
                    double dx = xy[2 * b] - xy[2 * a], dy = xy[2 * b + 1] - xy[2 * a + 1];
                    double l = dx * dx + dy * dy;
                    if (best < 0 || l < best) { best = l; be = e; }
                }
                int64_t ends[2] = {v[(be + 1) % 3], v[(be + 2) % 3]};
                int64_t ss[2][64];
                int nn[2] = {0, 0};
                for (int k = 0; k < 2; ++k) {
                    int64_t q = ends[k];
                    if (q < n_in) {
                        for (int64_t j = soff[q]; j < soff[q + 1] && nn[k] < 64; ++j) ss[k][nn[k]++] = sadj[j];
                    } else if (vseg[q] >= 0) {
                        ss[k][nn[k]++] = vseg[q];
                    }
                }
                for (int i = 0; i < nn[0] && !ex; ++i)
                    for (int j = 0; j < nn[1] && !ex; ++j)
                        if (small_pair_xy(xy, seg_in, ss[0][i], ss[1][j])) ex = 1;
                if (ex) rep->exempt_bad++;
                else rep->bad_quality++;
            }
            if (!ex) {
                /* smallest angle, from the law of cosines */
                double L[3];
                for (int e = 0; e < 3; ++e) {
                    int64_t a = v[(e + 1) % 3], b = v[(e + 2) % 3];
                    double dx = xy[2 * b] - xy[2 * a], dy = xy[2 * b + 1] - xy[2 * a + 1];
                    L[e] = sqrt(dx * dx + dy * dy);
                }
                for (int e = 0; e < 3; ++e) {
                    double c = (L[(e + 1) % 3] * L[(e + 1) % 3] + L[(e + 2) % 3] * L[(e + 2) % 3] -
                                L[e] * L[e]) / (2 * L[(e + 1) % 3] * L[(e + 2) % 3]);
                    if (c > 1) c = 1;
                    if (c < -1) c = -1;
                    double ang = acos(c) * 180.0 / M_PI;
                    if (ang < rep->min_angle_deg) rep->min_angle_deg = ang;
                }
            }
        }
        free(soff);
        free(sadj);
        free(vseg);
    }
    /* brute force: no vertex visible from a triangle inside its circumcircle */
    if (brute) {
        for (int64_t t = 0; t < nt; ++t) {
            const int32_t* v = tri + 3 * t;
            double ax = xy[2 * v[0]], ay = xy[2 * v[0] + 1], bx = xy[2 * v[1]], by = xy[2 * v[1] + 1];
            double cx = xy[2 * v[2]], cy = xy[2 * v[2] + 1];
            double gx = (ax + bx + cx) / 3.0, gy = (ay + by + cy) / 3.0;
            for (int64_t w = 0; w < nv; ++w) {
                if (!used[w] || w == v[0] || w == v[1] || w == v[2]) continue;
                if (or_incircle_sos(ax, ay, bx, by, cx, cy, xy[2 * w], xy[2 * w + 1]) <= 0) continue;
                int blocked = 0;
                for (int64_t i = 0; i < ns && !blocked; ++i)
                    if (crosses(xy, sub[3 * i], sub[3 * i + 1], gx, gy, w)) blocked = 1;
                if (!blocked) rep->bf_cd_violations++;
            }
        }
    }
    free(off);
    free(adj);
    free(used);
    or_map_free(&dir);
    or_map_free(&und);
    or_map_free(&subs);
    return 0;
}
