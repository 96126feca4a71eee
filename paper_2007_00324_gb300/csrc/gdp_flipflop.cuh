// Flip-Flop insertion: the insertion step of Algorithm 1 as the paper's gDP2d
// does it (Sec. 4.3), the alternative to cavity re-triangulation
// (GDP_REFINE_FLIPFLOP).
//
// The splitting points that survive the cavity filter (the same growth and
// priority marks as the cavity insertion, Sec. 4.3's filtering step) are all
// put into the triangulation at once -- a free point splits its triangle in
// three, a point on an edge (a subsegment's midpoint) splits the two
// triangles of that edge in four -- without the Delaunay-dependence check.
// Then, in parallel passes:
//   * a flip replaces two triangles abc, acd forming a convex quadrilateral by
//     abd, dbc; it is done where an edge is not locally Delaunay (the sum of
//     the opposite angles exceeds pi, i.e. incircle > 0), and to lower the
//     degree of a redundant point;
//   * a flop replaces the three triangles around a point of degree three by
//     one, removing the point; a redundant midpoint whose two sides are down
//     to two triangles each is removed the same way (four triangles to two,
//     the subsegment restored);
//   * a point inserted in this iteration is redundant when it is joined by an
//     edge to another one of higher priority (Sec. 4.2: no two Steiner points
//     of one iteration may form an edge -- they are Delaunay dependent); after
//     the passes settle, the check is repeated, until the triangulation is a
//     CDT with no redundant point.
// Circumcentres that encroach a subsegment on their cavity boundary are
// replaced by that subsegment's split point during the filter (as in the
// cavity insertion), so no inserted free point is redundant for that reason.
//
// Passes work on a list of triangles like the construction's flip passes:
// proposals mark the triangles they need with 64-bit keys (atomicMax), the
// owners rewrite them in place and record where each outer edge went, and a
// link pass repairs the neighbour references.  Removal proposals outrank
// Lawson flips, and of two adjacent redundant points the one with the lower
// key is removed first, so every pass removes or reduces something.
#pragma once
#include "gdp_cdt.cuh"

namespace gdp {

// operation kinds (Pool::fop), FF_EXEC once done
constexpr int FF_NONE = -1, FF_FLIP = 0, FF_FLOP = 1, FF_UNSPLIT = 2, FF_RETRI = 3, FF_EXEC = 16;
constexpr int FF_RETRI_MAX = 6;   // stars up to this size are removed by re-triangulation
constexpr int FF_DEG_MAX = 64;    // star walks are bounded (a larger star waits)

__device__ __forceinline__ unsigned long long ff_key(const Pool& P, int step, int cls, int t, int x) {
  const int lt = t - P.mi[P.T[t].w >> 4].tri_base;
  return ((unsigned long long)step << 44) | ((unsigned long long)cls << 42) |
         ((unsigned long long)(hash32((uint32_t)lt) & 0x3ffu) << 32) | (unsigned)((lt << 2) | (x & 3));
}

__device__ __forceinline__ int pos_of(const int4& T4, int v) {
  return T4.x == v ? 0 : (T4.y == v ? 1 : (T4.z == v ? 2 : -1));
}
__device__ __forceinline__ bool live(const int4& T4) { return T4.w >= 0 && !(T4.w & INFO_DEAD); }
__device__ __forceinline__ int cbit(const int4& T4, int e) { return (T4.w >> e) & 1; }

// a vertex inserted in this iteration and not removed
__device__ __forceinline__ bool ff_new(const Pool& P, const MeshInfo& M, int v) {
  return v >= M.vert_base + M.ff_v0 && v < M.vert_base + M.vert_count && !(P.vred[v] & 2);
}
__device__ __forceinline__ bool ff_redundant(const Pool& P, int v) { return (P.vred[v] & 3) == 1; }

// position in T4 of its redundant point with the lowest key, -1 if none
__device__ __forceinline__ int ff_first_redundant(const Pool& P, const int4& T4) {
  int j = -1;
  unsigned long long best = 0ull;
  for (int q = 0; q < 3; ++q) {
    const int x = comp(T4, q);
    if (!ff_redundant(P, x)) continue;
    const unsigned long long k = P.vkey[x];
    if (j < 0 || k < best) { j = q; best = k; }
  }
  return j;
}

// ---------------------------------------------------------------- insertion
// per surviving candidate: how it goes in (c_loc = t << 2 | e: split edge e
// of t; e = 3: split t in three) and its new slots (c_extra), with block sums
// for k_offsets; every mesh records where this iteration's vertices start
__global__ void __launch_bounds__(BS) k_ff_prep(Pool P, int trace) {
  __shared__ int sm[33];
  const int n = P.ctrl->n_cand;
  {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    for (int m = gt; m < P.n_mesh; m += gs) P.mi[m].ff_v0 = P.mi[m].vert_count;
  }
  const Chunk ch = chunk_of(n);
  int se = 0, sv = 0;
  for (int i = ch.b0 + threadIdx.x; i < ch.b1; i += BS) {
    bool fin = P.c_state[i] == C_SURV;
    int extra = 0, code = -1;
    if (fin) {
      const int t0 = cav_of(P, i)[0];
      const int4 T4 = P.T[t0];
      const int4 N4 = P.N[t0];
      const int2 sub = P.c_sub[i];
      int e = -1;
      if (sub.x >= 0) {   // a split point on subsegment sub: the edge of t0 it lies on
        for (int k = 0; k < 3 && e < 0; ++k) {
          const int u = comp(T4, mod3(k + 1)), v = comp(T4, mod3(k + 2));
          if ((u == sub.x && v == sub.y) || (u == sub.y && v == sub.x)) e = k;
        }
      } else {            // a free point: inside t0, or on one of its edges
        const P2 p{P.c_pt[i], P.c_ptf[i]};
        int zero = -1, nz = 0, neg = 0;
        for (int k = 0; k < 3; ++k) {
          const int o = orient(pt(P, comp(T4, mod3(k + 1))), pt(P, comp(T4, mod3(k + 2))), p);
          if (o == 0) { zero = k; ++nz; }
          if (o < 0) ++neg;
        }
        if (neg == 0 && nz == 0) e = 3;
        else if (neg == 0 && nz == 1 && !cbit(T4, zero) && comp(N4, zero) >= 0) e = zero;
      }
      if (e < 0) {   // cannot happen for a located, filtered point
        set_err(P.ctrl, S_INTERNAL);
        atomicCAS(&P.ctrl->dbg, 0, 1);
        if (trace) {
          const double2 p = P.c_pt[i];
          printf("ff prep: candidate %d elem %d t0=%d (%d %d %d w=%x) N=(%d %d %d) sub=(%d %d) p=(%.17g %.17g) "
                 "o=(%d %d %d) big=%d\n", i, P.c_elem[i], t0, T4.x, T4.y, T4.z, T4.w, N4.x, N4.y, N4.z, sub.x,
                 sub.y, p.x, p.y,
                 orient(pt(P, T4.y), pt(P, T4.z), P2{p, P.c_ptf[i]}),
                 orient(pt(P, T4.z), pt(P, T4.x), P2{p, P.c_ptf[i]}),
                 orient(pt(P, T4.x), pt(P, T4.y), P2{p, P.c_ptf[i]}), P.c_big[i]);
        }
        fin = false;
      } else {
        code = (t0 << 2) | e;
        extra = (e == 3 || comp(N4, e) >= 0) ? 2 : 1;
      }
    }
    P.c_final[i] = fin;
    P.c_extra[i] = extra;
    P.c_loc[i] = code;
    se += extra;
    sv += fin ? 1 : 0;
  }
  se = block_sum(se, sm);
  sv = block_sum(sv, sm);
  if (threadIdx.x == 0) {
    P.blk[blockIdx.x] = se;
    P.blk[gridDim.x + blockIdx.x] = sv;
  }
}

__device__ __forceinline__ void ff_touch(const Pool& P, int s, int step) {
  P.tstamp[s] = step;
  P.dirty[s] = 1;
  fl_push(P, P.fl_nxt, s, step + 1);
}

// Every surviving point goes in.  Free point p in t = (a0, a1, a2):
// T_e = (p, a[e+1], a[e+2]) keeps edge e of t as its edge 0.  Point p on edge
// (u1, u2) of t = (u0, u1, u2) with t1 = (d, u2, u1) across it (none on the
// hull): (p, u0, u1) and (p, u2, u0) in t and a new slot, (p, d, u2) and
// (p, u1, d) in t1 and a new slot; both halves of a split subsegment stay
// subsegments.  Outer edges go to newref for the link kernel.
__global__ void __launch_bounds__(BS) k_ff_split(Pool P) {
  const int n = P.ctrl->n_cand;
  const int step = P.ctrl->step;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int i = gt; i < n; i += gs) {
    const int m = P.c_mesh[i];
    const MeshInfo& M = P.mi[m];
    const int f = M.first_cand, l = M.last_cand;
    int totE, totV;
    mesh_totals(P, f, l, totE, totV);
    const bool ok = M.tri_count + totE <= M.tri_cap && M.vert_count + totV <= M.vert_cap;
    if (i == f) {
      P.mi[m].ins_ok = ok ? 1 : 0;
      if (!ok) no_room<0>(P, m);
    }
    if (!P.c_final[i] || !ok) continue;
    const int base = M.tri_base + M.tri_count + (P.c_offT[i] - P.c_offT[f]);
    const int vid = M.vert_base + M.vert_count + (P.c_offV[i] - P.c_offV[f]);
    P.c_base[i] = base;
    P.V[vid] = P.c_pt[i];
    P.Vf[vid] = P.c_ptf[i];
    P.vseg[vid] = P.c_vseg[i];
    P.vkey[vid] = P.c_key[i];
    P.vred[vid] = 0;
    const int code = P.c_loc[i], t = code >> 2, e = code & 3;
    P.vtri[vid] = t;
    const int4 T4 = P.T[t];
    const int4 N4 = P.N[t];
    const int info = m << 4;
    if (e == 3) {
      const int s[3] = {t, base, base + 1};
      for (int k = 0; k < 3; ++k) {
        P.T[s[k]] = make_int4(vid, comp(T4, mod3(k + 1)), comp(T4, mod3(k + 2)), info | cbit(T4, k));
        P.N[s[k]] = make_int4(comp(N4, k), (s[mod3(k + 1)] << 2) | 2, (s[mod3(k + 2)] << 2) | 1, 0);
        P.newref[(t << 2) | k] = s[k] << 2;
        ff_touch(P, s[k], step);
      }
      continue;
    }
    const int u0 = comp(T4, e), u1 = comp(T4, mod3(e + 1)), u2 = comp(T4, mod3(e + 2));
    const int c0 = cbit(T4, e), c1 = cbit(T4, mod3(e + 1)), c2 = cbit(T4, mod3(e + 2));
    const int n01 = comp(N4, mod3(e + 2)), n20 = comp(N4, mod3(e + 1)), r = comp(N4, e);
    const int S0 = t, S1 = base;
    if (r < 0) {   // hull edge (always a subsegment)
      P.T[S0] = make_int4(vid, u0, u1, info | c2 | (c0 << 1));
      P.N[S0] = make_int4(n01, -1, (S1 << 2) | 1, 0);
      P.T[S1] = make_int4(vid, u2, u0, info | c1 | (c0 << 2));
      P.N[S1] = make_int4(n20, (S0 << 2) | 2, -1, 0);
      P.newref[(t << 2) | mod3(e + 2)] = S0 << 2;
      P.newref[(t << 2) | mod3(e + 1)] = S1 << 2;
      ff_touch(P, S0, step);
      ff_touch(P, S1, step);
      continue;
    }
    const int t1 = r >> 2, e1 = r & 3;
    const int4 U4 = P.T[t1];
    const int4 M4 = P.N[t1];
    const int d = comp(U4, e1);
    const int d1 = cbit(U4, mod3(e1 + 1)), d2 = cbit(U4, mod3(e1 + 2));   // (u1, d), (d, u2)
    const int n1d = comp(M4, mod3(e1 + 1)), nd2 = comp(M4, mod3(e1 + 2));
    const int S2 = t1, S3 = base + 1;
    P.T[S0] = make_int4(vid, u0, u1, info | c2 | (c0 << 1));
    P.N[S0] = make_int4(n01, (S3 << 2) | 2, (S1 << 2) | 1, 0);
    P.T[S1] = make_int4(vid, u2, u0, info | c1 | (c0 << 2));
    P.N[S1] = make_int4(n20, (S0 << 2) | 2, (S2 << 2) | 1, 0);
    P.T[S2] = make_int4(vid, d, u2, info | d2 | (c0 << 1));
    P.N[S2] = make_int4(nd2, (S1 << 2) | 2, (S3 << 2) | 1, 0);
    P.T[S3] = make_int4(vid, u1, d, info | d1 | (c0 << 2));
    P.N[S3] = make_int4(n1d, (S2 << 2) | 2, (S0 << 2) | 1, 0);
    P.newref[(t << 2) | mod3(e + 2)] = S0 << 2;
    P.newref[(t << 2) | mod3(e + 1)] = S1 << 2;
    P.newref[(t1 << 2) | mod3(e1 + 2)] = S2 << 2;
    P.newref[(t1 << 2) | mod3(e1 + 1)] = S3 << 2;
    ff_touch(P, S0, step);
    ff_touch(P, S1, step);
    ff_touch(P, S2, step);
    ff_touch(P, S3, step);
  }
}

// outer neighbours of the split triangles (edge 0 of each), then per-mesh counts
__global__ void __launch_bounds__(BS) k_ff_split_link(Pool P) {
  const int n = P.ctrl->n_cand;
  const int step = P.ctrl->step;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  int ins = 0;
  for (int i = gt; i < n; i += gs) {
    const int m = P.c_mesh[i];
    const MeshInfo& M = P.mi[m];
    const bool ok = M.ins_ok;
    if (P.c_final[i] && ok) {
      ++ins;
      const int code = P.c_loc[i], t = code >> 2, e = code & 3, base = P.c_base[i];
      int s[4], ns = 0;
      s[ns++] = t;
      s[ns++] = base;
      if (e == 3) {
        s[ns++] = base + 1;
      } else {
        const int r = P.N[base].z;   // (p, u2, u0): its edge 2 leads to (p, d, u2) in t1
        if (r >= 0) {
          s[ns++] = r >> 2;
          s[ns++] = base + 1;
        }
      }
      for (int k = 0; k < ns; ++k) flip_fix(P, s[k], 0, step);
    }
    if (i == M.last_cand && ok) {
      int totE, totV;
      mesh_totals(P, M.first_cand, i, totE, totV);
      P.mi[m].tri_count = M.tri_count + totE;
      P.mi[m].vert_count = M.vert_count + totV;
      P.mi[m].steiner = M.steiner + totV;
    }
  }
  for (int o = 16; o; o >>= 1) ins += __shfl_xor_sync(0xffffffffu, ins, o);
  if ((threadIdx.x & 31) == 0 && ins) {
    atomicAdd(&P.ctrl->n_ins, (unsigned long long)ins);
    atomicAdd(&P.ctrl->tot_ins, (unsigned long long)ins);
  }
}

// ---------------------------------------------------------------- stars
// Triangle s holds v at position j.  Its edge after v is (v, comp(s, j+1))
// (edge index j+2), the edge before v is (comp(s, j+2), v) (edge index j+1).
struct Corner {
  int t, j;
};
__device__ __forceinline__ int after_edge(int j) { return mod3(j + 2); }
__device__ __forceinline__ int before_edge(int j) { return mod3(j + 1); }

// step around v across the edge after it (clockwise) or before it; -1 at a
// subsegment (when stop_cons) or the hull.  The position j of v in the next
// triangle is -1 only in a broken mesh; callers check it before using it.
__device__ __forceinline__ Corner step_around(const Pool& P, Corner c, int v, bool after, bool stop_cons) {
  if (c.j < 0) return {-1, -1};
  const int4 T4 = P.T[c.t];
  const int e = after ? after_edge(c.j) : before_edge(c.j);
  const int r = comp(P.N[c.t], e);
  if (r < 0 || (stop_cons && cbit(T4, e))) return {-1, -1};
  const int t2 = r >> 2;
  return {t2, pos_of(P.T[t2], v)};
}

// ---------------------------------------------------------------- proposals
// The triangle t holds the redundant point v (position j).  A free point of
// degree three is flopped (proposed by the lowest slot of its star); a
// midpoint whose sides are down to two triangles each is unsplit (the lowest
// slot of the four, or two on the hull); otherwise t proposes to flip its
// edge after v when the quadrilateral is strictly convex (a star of any size).
// Order among adjacent redundant points: an operation of v never rewrites a
// triangle that holds a redundant point of lower key -- a flop or unsplit
// waits while any vertex of its (small) star is one, a flip while a vertex of
// its two triangles is one -- so the point of lowest key in any group always
// proceeds and the passes end.  Returns the kind proposed (fprop[k] = the
// slot that carries it out).
__device__ __forceinline__ bool ff_blocks(const Pool& P, int x, unsigned long long kv) {
  return ff_redundant(P, x) && P.vkey[x] < kv;
}

__device__ int ff_propose_removal(const Pool& P, int k, int t, int j, int v, int step) {
  const unsigned long long kv = P.vkey[v];
  // the star (one side of it for a midpoint), as far as FF_DEG_MAX triangles:
  // after-v edges clockwise, then before-v edges
  int side[FF_DEG_MAX], ns = 0;
  bool closed = false, wait = false;
  side[ns++] = t;
  Corner c{t, j};
  for (int s = 0; s < FF_DEG_MAX - 1; ++s) {
    const int4 T4 = P.T[c.t];
    if (ff_blocks(P, comp(T4, mod3(c.j + 1)), kv)) wait = true;
    c = step_around(P, c, v, true, true);
    if (c.t < 0) break;
    if (c.t == t) { closed = true; break; }
    side[ns++] = c.t;
  }
  Corner first{t, j};
  bool whole = closed;   // the walk saw the whole star (or the whole side)
  if (!closed && ns < FF_DEG_MAX) {
    Corner b{t, j};
    for (int s = 0; s < FF_DEG_MAX && ns < FF_DEG_MAX; ++s) {
      const int4 T4 = P.T[b.t];
      if (ff_blocks(P, comp(T4, mod3(b.j + 2)), kv)) wait = true;
      const Corner nb = step_around(P, b, v, false, true);
      if (nb.t < 0) { whole = true; break; }
      b = nb;
      side[ns++] = b.t;
    }
    first = b;   // the end whose before-v edge is a subsegment (or the hull)
  }
  if (whole && closed && ns > 3 && ns <= FF_RETRI_MAX) {   // a small star: re-triangulated
    if (wait) return FF_NONE;
    int tmin = side[0];
    for (int q = 1; q < ns; ++q) tmin = min(tmin, side[q]);
    if (t != tmin) return FF_NONE;
    const unsigned long long key = ff_key(P, step, 2, tmin, 3);
    for (int q = 0; q < ns; ++q) atomicMax(&P.ffmark[side[q]], key);
    P.fprop[k] = tmin;
    return FF_RETRI;
  }
  if (whole && closed && ns == 3) {   // flop of a free point of degree three
    if (wait) return FF_NONE;
    int tmin = side[0];
    for (int q = 1; q < 3; ++q) tmin = min(tmin, side[q]);
    if (t != tmin) return FF_NONE;
    const unsigned long long key = ff_key(P, step, 2, tmin, 3);
    for (int q = 0; q < 3; ++q) atomicMax(&P.ffmark[side[q]], key);
    P.fprop[k] = tmin;
    return FF_FLOP;
  }
  if (whole && !closed && ns == 2) {   // a midpoint: unsplit once both sides have two triangles
    const int e = before_edge(first.j);
    const int r = comp(P.N[first.t], e);
    int other[4], no = 0;
    if (r >= 0) {
      // (v, p2, d) across the subsegment, then counter-clockwise to (v, d, p1)
      Corner o{r >> 2, pos_of(P.T[r >> 2], v)};
      other[no++] = o.t;
      for (int s = 0; s < 3; ++s) {
        if (ff_blocks(P, comp(P.T[o.t], mod3(o.j + 1)), kv) || ff_blocks(P, comp(P.T[o.t], mod3(o.j + 2)), kv))
          wait = true;
        o = step_around(P, o, v, false, true);
        if (o.t < 0) break;
        if (no == 4) { no = 5; break; }
        other[no++] = o.t;
      }
    }
    // a side of two triangles cannot lose another edge: it waits for the other
    if (no != 0 && no != 2) return FF_NONE;
    if (wait) return FF_NONE;
    int tmin = min(side[0], side[1]);
    for (int q = 0; q < no; ++q) tmin = min(tmin, other[q]);
    if (t != tmin) return FF_NONE;
    const unsigned long long key = ff_key(P, step, 2, tmin, 3);
    atomicMax(&P.ffmark[side[0]], key);
    atomicMax(&P.ffmark[side[1]], key);
    for (int q = 0; q < no; ++q) atomicMax(&P.ffmark[other[q]], key);
    P.fprop[k] = tmin;
    return FF_UNSPLIT;
  }
  // degree reduction: flip the edge after v, (v, x), with (v, w, x) across it
  const int4 T4 = P.T[t];
  const int ea = after_edge(j);
  if (cbit(T4, ea)) return FF_NONE;
  const int r = comp(P.N[t], ea);
  if (r < 0) return FF_NONE;
  const int x = comp(T4, mod3(j + 1)), y = comp(T4, mod3(j + 2));
  const int4 U4 = P.T[r >> 2];
  const int w = comp(U4, r & 3);
  if (ff_blocks(P, x, kv) || ff_blocks(P, y, kv) || ff_blocks(P, w, kv)) return FF_NONE;
  // The flip makes (y, v, w) and (y, w, x).  Neither may get the two halves of
  // a split subsegment as two of its edges (a sliver through a split point a
  // rounding error off its segment): not at v (edges (y, v) and (v, w)), not
  // at x when x is a split point (edges (x, y) and (w, x)).
  const int jw = pos_of(U4, v);
  if (jw < 0) return FF_NONE;
  const bool c_yv = cbit(T4, before_edge(j)), c_vw = cbit(U4, after_edge(jw));
  const bool c_xy = cbit(T4, j), c_wx = cbit(U4, jw);
  if (c_yv && c_vw) return FF_NONE;
  if (P.vseg[x] >= 0 && c_xy && c_wx) return FF_NONE;
  if (orient(pt(P, y), pt(P, v), pt(P, w)) <= 0 || orient(pt(P, y), pt(P, w), pt(P, x)) <= 0) return FF_NONE;
  const unsigned long long key = ff_key(P, step, 1, t, ea);
  atomicMax(&P.ffmark[t], key);
  atomicMax(&P.ffmark[r >> 2], key);
  P.fprop[k] = (t << 2) | ea;
  return FF_FLIP | 4;   // a flip of class 1
}

__global__ void __launch_bounds__(BS) k_ff_propose(Pool P) {
  const int n = P.ctrl->n_fl;
  const int step = P.ctrl->step;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int k = gt; k < n; k += gs) {
    const int t = P.fl_cur[k];
    const int4 T4 = P.T[t];
    P.fop[k] = FF_NONE;
    if (!live(T4)) continue;
    // the redundant point of t with the lowest key, if any: the one whose
    // removal goes first (the others wait for it)
    const int j = ff_first_redundant(P, T4);
    const int v = j >= 0 ? comp(T4, j) : -1;
    if (v >= 0) {
      P.fop[k] = ff_propose_removal(P, k, t, j, v, step);
      continue;
    }
    // Lawson: the first edge whose opposite vertex lies in the circumcircle
    const int4 N4 = P.N[t];
    const P2 a = pt(P, T4.x), b = pt(P, T4.y), c = pt(P, T4.z);
    for (int e = 0; e < 3; ++e) {
      const int r = comp(N4, e);
      if (r < 0 || cbit(T4, e)) continue;
      const int4 U4 = P.T[r >> 2];
      if (ff_redundant(P, U4.x) || ff_redundant(P, U4.y) || ff_redundant(P, U4.z)) continue;
      if (incircle(a, b, c, pt(P, comp(U4, r & 3))) > 0) {
        const unsigned long long key = ff_key(P, step, 0, t, e);
        atomicMax(&P.ffmark[t], key);
        atomicMax(&P.ffmark[r >> 2], key);
        P.fprop[k] = (t << 2) | e;
        P.fop[k] = FF_FLIP;
        break;
      }
    }
  }
}

// ---------------------------------------------------------------- operations
// flip edge e of t = (a, b, c), t2 = (d, c, b) across it, keeping the
// subsegment bits of the four outer edges: (a, b, d) + (a, d, c)
__device__ void ff_flip(const Pool& P, int t, int e, int step) {
  const int4 T4 = P.T[t];
  const int4 N4 = P.N[t];
  const int r = comp(N4, e);
  const int t2 = r >> 2, e2 = r & 3;
  const int4 U4 = P.T[t2];
  const int4 M4 = P.N[t2];
  const int a = comp(T4, e), b = comp(T4, mod3(e + 1)), c = comp(T4, mod3(e + 2));
  const int d = comp(U4, e2);
  const int nab = comp(N4, mod3(e + 2)), nca = comp(N4, mod3(e + 1));
  const int nbd = comp(M4, mod3(e2 + 1)), ndc = comp(M4, mod3(e2 + 2));
  const int cab = cbit(T4, mod3(e + 2)), cca = cbit(T4, mod3(e + 1));
  const int cbd = cbit(U4, mod3(e2 + 1)), cdc = cbit(U4, mod3(e2 + 2));
  const int info = T4.w & ~15;
  P.T[t] = make_int4(a, b, d, info | cbd | (cab << 2));
  P.N[t] = make_int4(nbd, (t2 << 2) | 2, nab, 0);
  P.T[t2] = make_int4(a, d, c, info | cdc | (cca << 1));
  P.N[t2] = make_int4(ndc, nca, (t << 2) | 1, 0);
  P.newref[(t << 2) | mod3(e + 2)] = (t << 2) | 2;     // ab
  P.newref[(t << 2) | mod3(e + 1)] = (t2 << 2) | 1;    // ca
  P.newref[(t2 << 2) | mod3(e2 + 1)] = t << 2;         // bd
  P.newref[(t2 << 2) | mod3(e2 + 2)] = t2 << 2;        // dc
  ff_touch(P, t, step);
  ff_touch(P, t2, step);
  P.vtri[a] = t;
  P.vtri[b] = t;
  P.vtri[d] = t;
  P.vtri[c] = t2;
}

__device__ __forceinline__ void ff_kill(const Pool& P, int s, int step) {
  P.T[s].w = (P.T[s].w & ~15) | INFO_DEAD;
  P.flag[s] = 0;
  P.dirty[s] = 0;
  P.tstamp[s] = step;
}

__device__ __forceinline__ void ff_removed(const Pool& P, int v, int m) {
  P.vred[v] = 3;
  atomicSub(&P.mi[m].steiner, 1);
  atomicAdd(&P.ctrl->ff_removed, 1ull);
}

// The three triangles (v, x0, x1), (v, x1, x2), (v, x2, x0) around v, found
// counter-clockwise from t, become (x0, x1, x2) in slot t.  Every triangle of
// the star is owned (key) before it is read.  False when one is not.
__device__ bool ff_flop(const Pool& P, int t, int v, unsigned long long key, int step) {
  int s[3], j[3];
  Corner c{t, pos_of(P.T[t], v)};
  for (int q = 0; q < 3; ++q) {
    if (c.t < 0 || __ldcg(&P.ffmark[c.t]) != key) return false;
    if (c.j < 0) {   // v not in a triangle of its own star: the mesh is broken
      set_err(P.ctrl, S_INTERNAL);
      atomicCAS(&P.ctrl->dbg, 0, 2);
      return false;
    }
    s[q] = c.t;
    j[q] = c.j;
    if (q < 2) c = step_around(P, c, v, false, false);
  }
  int x[3], nr[3], cb[3];
  for (int q = 0; q < 3; ++q) {
    const int4 T4 = P.T[s[q]];
    x[q] = comp(T4, mod3(j[q] + 1));   // s[q] = (v, x_q, x_{q+1})
    nr[q] = comp(P.N[s[q]], j[q]);     // its edge opposite v
    cb[q] = cbit(T4, j[q]);
  }
  const int m = P.T[t].w >> 4;
  // (x0, x1, x2): edge 0 = (x1, x2) of s[1], edge 1 = (x2, x0) of s[2], edge 2 = (x0, x1) of s[0]
  const int ne[3] = {2, 0, 1};
  for (int q = 0; q < 3; ++q) P.newref[(s[q] << 2) | j[q]] = (t << 2) | ne[q];
  for (int q = 0; q < 3; ++q)
    if (s[q] != t) ff_kill(P, s[q], step);
  P.T[t] = make_int4(x[0], x[1], x[2], (m << 4) | cb[1] | (cb[2] << 1) | (cb[0] << 2));
  P.N[t] = make_int4(nr[1], nr[2], nr[0], 0);
  ff_touch(P, t, step);
  for (int q = 0; q < 3; ++q) P.vtri[x[q]] = t;
  ff_removed(P, v, m);
  atomicAdd(&P.ctrl->ff_flops, 1ull);
  return true;
}

// A midpoint v on subsegment (p2, p1) whose sides are down to two triangles:
// E1 = (v, p1, c), E2 = (v, c, p2) and, across the subsegment, F = (v, d, p1),
// G = (v, p2, d) become (p2, p1, c) in E1 and (p1, p2, d) in G, joined by the
// restored subsegment (on the hull only the first).  Returns E1, -1 when a
// triangle is not owned.
__device__ int ff_unsplit(const Pool& P, int t, int v, unsigned long long key, int step) {
  if (__ldcg(&P.ffmark[t]) != key) return -1;
  Corner e1{t, pos_of(P.T[t], v)};
  if (e1.j < 0) {
    set_err(P.ctrl, S_INTERNAL);
    atomicCAS(&P.ctrl->dbg, 0, 3);
    return -1;
  }
  if (!cbit(P.T[t], after_edge(e1.j))) {
    e1 = step_around(P, e1, v, true, true);
    if (e1.t < 0 || __ldcg(&P.ffmark[e1.t]) != key) return -1;
  }
  const Corner e2 = step_around(P, e1, v, false, true);
  if (e2.t < 0 || __ldcg(&P.ffmark[e2.t]) != key) return -1;
  if (e1.j < 0 || e2.j < 0) {
    set_err(P.ctrl, S_INTERNAL);
    atomicCAS(&P.ctrl->dbg, 0, 3);
    return -1;
  }
  const int4 A4 = P.T[e1.t], B4 = P.T[e2.t];
  const int p1 = comp(A4, mod3(e1.j + 1)), c = comp(A4, mod3(e1.j + 2));
  const int p2 = comp(B4, mod3(e2.j + 2));
  const int rA = comp(P.N[e1.t], e1.j), rB = comp(P.N[e2.t], e2.j);
  const int cA = cbit(A4, e1.j), cB = cbit(B4, e2.j);
  const int m = A4.w >> 4;
  const int across = comp(P.N[e1.t], after_edge(e1.j));
  int G = -1;
  if (across >= 0) {
    Corner f{across >> 2, -1};
    if (__ldcg(&P.ffmark[f.t]) != key) return -1;
    f.j = pos_of(P.T[f.t], v);
    if (f.j < 0) {
      set_err(P.ctrl, S_INTERNAL);
      atomicCAS(&P.ctrl->dbg, 0, 3);
      return -1;
    }
    const Corner g = step_around(P, f, v, true, true);
    if (g.t < 0 || __ldcg(&P.ffmark[g.t]) != key) return -1;
    if (g.j < 0) {
      set_err(P.ctrl, S_INTERNAL);
      atomicCAS(&P.ctrl->dbg, 0, 3);
      return -1;
    }
    const int4 F4 = P.T[f.t], G4 = P.T[g.t];
    const int d = comp(F4, mod3(f.j + 1));
    const int rF = comp(P.N[f.t], f.j), rG = comp(P.N[g.t], g.j);
    const int cF = cbit(F4, f.j), cG = cbit(G4, g.j);
    G = g.t;
    P.newref[(g.t << 2) | g.j] = G << 2;
    P.newref[(f.t << 2) | f.j] = (G << 2) | 1;
    ff_kill(P, f.t, step);
    P.T[G] = make_int4(p1, p2, d, (m << 4) | cG | (cF << 1) | 4);
    P.N[G] = make_int4(rG, rF, (e1.t << 2) | 2, 0);
    ff_touch(P, G, step);
    P.vtri[d] = G;
  }
  P.newref[(e1.t << 2) | e1.j] = e1.t << 2;
  P.newref[(e2.t << 2) | e2.j] = (e1.t << 2) | 1;
  ff_kill(P, e2.t, step);
  P.T[e1.t] = make_int4(p2, p1, c, (m << 4) | cA | (cB << 1) | 4);
  P.N[e1.t] = make_int4(rA, rB, G >= 0 ? (G << 2) | 2 : -1, 0);
  ff_touch(P, e1.t, step);
  P.vtri[p1] = e1.t;
  P.vtri[p2] = e1.t;
  P.vtri[c] = e1.t;
  ff_removed(P, v, m);
  atomicAdd(&P.ctrl->ff_flops, 1ull);
  return e1.t;
}

// The star of free point v (4 to FF_RETRI_MAX triangles, found
// counter-clockwise from t, each owned) is removed with v and its link
// polygon triangulated by ear clipping: an ear is a strictly convex corner
// whose triangle holds no other polygon vertex, inside or on its edges
// (exact orient), so collinear link vertices -- split points along a
// subsegment -- are handled where no flip is strictly convex.  In general
// position this gives a triangulation that flips and a flop also reach; the
// Lawson flips that follow make it Delaunay.  The new triangles take the
// lowest slots of the star; the two highest die and keep, for the link pass,
// the list of new slots (T.x = count, T.y, T.z, N.x, N.y of the first dead
// slot).  Returns that slot, or -1 when a triangle is not owned.
__device__ int ff_retri(const Pool& P, int t, int v, unsigned long long key, int step) {
  int st[FF_RETRI_MAX], sj[FF_RETRI_MAX], ns = 0;
  Corner c{t, pos_of(P.T[t], v)};
  for (int q = 0; q < FF_RETRI_MAX; ++q) {
    if (c.t < 0 || __ldcg(&P.ffmark[c.t]) != key) return -1;
    if (c.j < 0) {
      set_err(P.ctrl, S_INTERNAL);
      atomicCAS(&P.ctrl->dbg, 0, 6);
      return -1;
    }
    st[ns] = c.t;
    sj[ns] = c.j;
    ++ns;
    c = step_around(P, c, v, false, false);
    if (c.t == t) break;
  }
  if (c.t != t || ns < 4) return -1;
  // link polygon x[0..ns) counter-clockwise; edge i = (x_i, x_{i+1}) is the
  // edge opposite v in st[i]: its outer ref, subsegment bit and origin
  int x[FF_RETRI_MAX], er[FF_RETRI_MAX], ec[FF_RETRI_MAX], eo[FF_RETRI_MAX];
  for (int q = 0; q < ns; ++q) {
    x[q] = comp(P.T[st[q]], mod3(sj[q] + 1));
    er[q] = comp(P.N[st[q]], sj[q]);
    ec[q] = cbit(P.T[st[q]], sj[q]);
    eo[q] = (st[q] << 2) | sj[q];   // where the outside refers to this edge
  }
  const int m = P.T[t].w >> 4;
  int slot[FF_RETRI_MAX];
  for (int q = 0; q < ns; ++q) slot[q] = st[q];
  for (int a = 1; a < ns; ++a)   // ascending slots
    for (int b = a; b > 0 && slot[b] < slot[b - 1]; --b) {
      const int tmp = slot[b];
      slot[b] = slot[b - 1];
      slot[b - 1] = tmp;
    }
  // polygon edges: outer (internal = -1) or an edge (s << 2 | e) of a new triangle
  int in_e[FF_RETRI_MAX], nxt[FF_RETRI_MAX], prv[FF_RETRI_MAX];
  for (int q = 0; q < ns; ++q) {
    in_e[q] = -1;
    nxt[q] = q + 1 < ns ? q + 1 : 0;
    prv[q] = q > 0 ? q - 1 : ns - 1;
  }
  int4 NT[FF_RETRI_MAX - 2], NN[FF_RETRI_MAX - 2];
  int used = 0, left = ns, start = 0;
  // set edge e of new triangle u from polygon edge i
  auto put = [&](int u, int e, int i) {
    int* nref = comp_ptr(&NN[u], e);
    if (in_e[i] < 0) {
      *nref = er[i];
      NT[u].w |= ec[i] << e;
      P.newref[eo[i]] = (slot[u] << 2) | e;
    } else {
      *nref = in_e[i];
      const int ou = in_e[i] >> 2, oe = in_e[i] & 3;   // ou: index of a new triangle
      *comp_ptr(&NN[ou], oe) = (slot[u] << 2) | e;
      *nref = (slot[ou] << 2) | oe;
    }
  };
  int guard = 0;
  while (left > 3 && guard++ < 64) {
    int b = start, found = -1;
    for (int r = 0; r < left; ++r, b = nxt[b]) {
      const int a = prv[b], cc = nxt[b];
      if (orient(pt(P, x[a]), pt(P, x[b]), pt(P, x[cc])) <= 0) continue;
      bool ear = true;
      for (int q = nxt[cc]; q != a && ear; q = nxt[q]) {
        const P2 pq = pt(P, x[q]);
        if (orient(pt(P, x[a]), pt(P, x[b]), pq) >= 0 && orient(pt(P, x[b]), pt(P, x[cc]), pq) >= 0 &&
            orient(pt(P, x[cc]), pt(P, x[a]), pq) >= 0)
          ear = false;
      }
      if (ear) { found = b; break; }
    }
    if (found < 0) {   // a star-shaped polygon always has an ear
      set_err(P.ctrl, S_INTERNAL);
      atomicCAS(&P.ctrl->dbg, 0, 7);
      return -1;
    }
    const int a = prv[found], cc = nxt[found];
    const int u = used++;
    // ear (x_a, x_b, x_c): edge 0 = (x_b, x_c) polygon edge found, edge 1 = (x_c, x_a)
    // the new diagonal, edge 2 = (x_a, x_b) polygon edge a
    NT[u] = make_int4(x[a], x[found], x[cc], m << 4);
    NN[u] = make_int4(-1, -1, -1, 0);
    put(u, 0, found);
    put(u, 2, a);
    in_e[a] = (u << 2) | 1;   // the diagonal is now polygon edge a
    nxt[a] = cc;
    prv[cc] = a;
    start = cc;
    --left;
  }
  {
    const int a = start, b = nxt[a], cc = nxt[b];
    const int u = used++;
    NT[u] = make_int4(x[a], x[b], x[cc], m << 4);
    NN[u] = make_int4(-1, -1, -1, 0);
    put(u, 0, b);
    put(u, 1, cc);
    put(u, 2, a);
  }
  for (int q = 0; q < ns; ++q) P.tstamp[st[q]] = step;
  for (int u = 0; u < used; ++u) {
    P.T[slot[u]] = NT[u];
    P.N[slot[u]] = NN[u];
    ff_touch(P, slot[u], step);
    for (int e = 0; e < 3; ++e) P.vtri[comp(NT[u], e)] = slot[u];
  }
  const int d1 = slot[ns - 2], d2 = slot[ns - 1];
  ff_kill(P, d1, step);
  ff_kill(P, d2, step);
  // the record of the new slots for the link pass, in the first dead slot
  P.T[d1] = make_int4(used, used > 0 ? slot[0] : -1, used > 1 ? slot[1] : -1, (m << 4) | INFO_DEAD);
  P.N[d1] = make_int4(used > 2 ? slot[2] : -1, used > 3 ? slot[3] : -1, -1, 0);
  ff_removed(P, v, m);
  atomicAdd(&P.ctrl->ff_flops, 1ull);
  return d1;
}

// the triangle t of list entry k goes to the next pass unless its work is done
__device__ __forceinline__ void ff_retry(const Pool& P, int t, int step) {
  const int4 T4 = P.T[t];
  if (live(T4)) fl_push(P, P.fl_nxt, t, step + 1);
}

__global__ void __launch_bounds__(BS) k_ff_do(Pool P) {
  const int n = P.ctrl->n_fl;
  const int step = P.ctrl->step;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int k = gt; k < n; k += gs) {
    const int op = P.fop[k];
    const int t = P.fl_cur[k];
    if (op == FF_NONE) {   // a star waiting for its turn stays listed
      const int4 T4 = P.T[t];
      if (live(T4) && (ff_redundant(P, T4.x) || ff_redundant(P, T4.y) || ff_redundant(P, T4.z)))
        ff_retry(P, t, step);
      continue;
    }
    const int kind = op & 3;
    if (kind == FF_FLIP) {
      const int prop = P.fprop[k], tt = prop >> 2, e = prop & 3;
      const unsigned long long key = ff_key(P, step, (op & 4) ? 1 : 0, tt, e);
      if (__ldcg(&P.ffmark[tt]) != key) { ff_retry(P, t, step); continue; }
      const int r = comp(P.N[tt], e);
      if (r < 0 || __ldcg(&P.ffmark[r >> 2]) != key) { ff_retry(P, t, step); continue; }
      ff_flip(P, tt, e, step);
      atomicAdd(&P.ctrl->ff_flips, 1ull);
      P.fop[k] = op | FF_EXEC;
      continue;
    }
    // flop / unsplit of the redundant point of t that proposed it
    const int4 T4 = P.T[t];
    const int jr = ff_first_redundant(P, T4);
    const int v = jr >= 0 ? comp(T4, jr) : -1;
    const unsigned long long key = ff_key(P, step, 2, t, 3);
    if (kind == FF_FLOP) {
      if (v >= 0 && ff_flop(P, t, v, key, step)) P.fop[k] = op | FF_EXEC;
      else ff_retry(P, t, step);
    } else if (kind == FF_RETRI) {
      const int d1 = v >= 0 ? ff_retri(P, t, v, key, step) : -1;
      if (d1 >= 0) {
        P.fprop[k] = d1;
        P.fop[k] = op | FF_EXEC;
      } else {
        ff_retry(P, t, step);
      }
    } else {
      const int up = v >= 0 ? ff_unsplit(P, t, v, key, step) : -1;
      if (up >= 0) {
        P.fprop[k] = up;
        P.fop[k] = op | FF_EXEC;
      } else {
        ff_retry(P, t, step);
      }
    }
  }
}

// outer neighbours of the rewritten triangles
__global__ void __launch_bounds__(BS) k_ff_link(Pool P) {
  const int n = P.ctrl->n_fl;
  const int step = P.ctrl->step;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int k = gt; k < n; k += gs) {
    const int op = P.fop[k];
    if (op == FF_NONE || !(op & FF_EXEC)) continue;
    const int kind = op & 3;
    if (kind == FF_FLIP) {
      const int t = P.fprop[k] >> 2;
      const int t2 = P.N[t].y >> 2;
      flip_fix(P, t, 0, step);
      flip_fix(P, t, 2, step);
      flip_fix(P, t2, 0, step);
      flip_fix(P, t2, 1, step);
    } else if (kind == FF_FLOP) {
      const int t = P.fl_cur[k];
      for (int e = 0; e < 3; ++e) flip_fix(P, t, e, step);
    } else if (kind == FF_RETRI) {
      // the new slots from the record in the first dead slot; edges between
      // two of them were linked by the operation itself
      const int d1 = P.fprop[k];
      const int4 R = P.T[d1];
      const int4 R2 = P.N[d1];
      const int ns[4] = {R.y, R.z, R2.x, R2.y};
      const int cnt = min(R.x, 4);
      for (int u = 0; u < cnt; ++u) {
        const int su = ns[u];
        for (int e = 0; e < 3; ++e) {
          const int r = comp(P.N[su], e);
          bool inner = false;
          for (int q = 0; q < cnt; ++q) inner |= (r >= 0 && (r >> 2) == ns[q]);
          if (!inner) flip_fix(P, su, e, step);
        }
      }
    } else {
      const int up = P.fprop[k];
      flip_fix(P, up, 0, step);
      flip_fix(P, up, 1, step);
      const int r = P.N[up].z;
      if (r >= 0) {
        flip_fix(P, r >> 2, 0, step);
        flip_fix(P, r >> 2, 1, step);
      }
    }
  }
}

// GDP_TRACE: the first entries of a list that does not empty (a star that no
// proposal can reduce), printed from the device
__global__ void k_ff_debug(Pool P, int limit) {
  const int n = min(P.ctrl->n_fl, limit);
  for (int k = 0; k < n; ++k) {
    const int t = P.fl_cur[k];
    const int4 T4 = P.T[t];
    const int4 N4 = P.N[t];
    printf("ff list %d: t=%d (%d %d %d w=%x) N=(%d %d %d) vred=(%d %d %d) vseg=(%d %d %d) key=(%llx %llx %llx) fop=%d\n",
           k, t, T4.x, T4.y, T4.z, T4.w, N4.x, N4.y, N4.z, P.vred[T4.x], P.vred[T4.y], P.vred[T4.z],
           P.vseg[T4.x], P.vseg[T4.y], P.vseg[T4.z], P.vkey[T4.x], P.vkey[T4.y], P.vkey[T4.z], P.fop[k]);
  }
}

// ---------------------------------------------------------------- redundancy check
// Of two points inserted in this iteration that are joined by an edge, the
// one with the lower key is redundant (Sec. 4.2).  Every triangle that holds
// a point of this iteration was written in it, so the check reads the
// triangles marked dirty.  Counts the new marks in ctrl->ff_marked.
__global__ void __launch_bounds__(BS) k_ff_check(Pool P) {
  const int ns = scan_slots(P);
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  int marked = 0;
  for (int t = gt; t < ns; t += gs) {
    if (!P.dirty[t]) continue;
    const int4 T4 = P.T[t];
    if (!live(T4)) continue;
    const MeshInfo& M = P.mi[T4.w >> 4];
    for (int e = 0; e < 3; ++e) {
      const int u = comp(T4, mod3(e + 1)), w = comp(T4, mod3(e + 2));
      if (!ff_new(P, M, u) || !ff_new(P, M, w)) continue;
      const int lo = P.vkey[u] < P.vkey[w] ? u : w;
      if (!(atomicOr(&P.vred[lo], 1) & 1)) ++marked;
    }
  }
  for (int o = 16; o; o >>= 1) marked += __shfl_xor_sync(0xffffffffu, marked, o);
  if ((threadIdx.x & 31) == 0 && marked) atomicAdd(&P.ctrl->ff_marked, marked);
}

// every triangle around a redundant point goes into the next pass's list
__global__ void __launch_bounds__(BS) k_ff_push_stars(Pool P) {
  const int ns = scan_slots(P);
  const int step = P.ctrl->step;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int t = gt; t < ns; t += gs) {
    if (!P.dirty[t]) continue;
    const int4 T4 = P.T[t];
    if (!live(T4)) continue;
    if (ff_redundant(P, T4.x) || ff_redundant(P, T4.y) || ff_redundant(P, T4.z))
      fl_push(P, P.fl_nxt, t, step + 1);
  }
}

// ---------------------------------------------------------------- compaction
// The removed points leave holes in this iteration's vertex range; the points
// kept move down in order (one block per mesh), the triangles written in this
// iteration take the new ids, and vert_count shrinks.  Everything that refers
// to a vertex id by then lives in those triangles and the vertex arrays.
constexpr int FF_CT = 1024;   // threads of the per-mesh compaction blocks

__global__ void __launch_bounds__(FF_CT) k_ff_vmap(Pool P) {
  __shared__ int sm[33];
  for (int m = blockIdx.x; m < P.n_mesh; m += gridDim.x) {
    const MeshInfo& M = P.mi[m];
    const int v0 = M.vert_base + M.ff_v0, v1 = M.vert_base + M.vert_count;
    int off = 0;
    for (int base = v0; base < v1; base += FF_CT) {
      const int v = base + threadIdx.x;
      const int alive = (v < v1 && !(P.vred[v] & 2)) ? 1 : 0;
      int tot;
      const int r = block_excl_scan(alive, sm, tot);
      if (v < v1) P.vmap[v] = alive ? v0 + off + r : -1;
      off += tot;
    }
    if (threadIdx.x == 0) P.mi[m].tmp = (v1 - v0) - off;   // points removed
    __syncthreads();
  }
}

__global__ void __launch_bounds__(BS) k_ff_rename(Pool P) {
  const int ns = scan_slots(P);
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int t = gt; t < ns; t += gs) {
    if (!P.dirty[t]) continue;
    int4 T4 = P.T[t];
    if (!live(T4)) continue;
    const MeshInfo& M = P.mi[T4.w >> 4];
    if (!M.tmp) continue;
    const int v0 = M.vert_base + M.ff_v0, v1 = M.vert_base + M.vert_count;
    bool ch = false;
    for (int q = 0; q < 3; ++q) {
      int* x = comp_ptr(&T4, q);
      if (*x >= v0 && *x < v1) {
        *x = P.vmap[*x];
        ch = true;
      }
    }
    if (ch) P.T[t] = T4;
  }
}

__global__ void __launch_bounds__(FF_CT) k_ff_move(Pool P) {
  if (blockIdx.x == 0 && threadIdx.x == 0) P.ctrl->need_eval = 1;   // evaluate the written triangles
  for (int m = blockIdx.x; m < P.n_mesh; m += gridDim.x) {
    const MeshInfo& M = P.mi[m];
    const int v0 = M.vert_base + M.ff_v0, v1 = M.vert_base + M.vert_count;
    const int removed = M.tmp;
    __syncthreads();
    if (removed) {
      // chunks in order: a chunk is read whole before it is written, and its
      // targets lie below its sources, so no later chunk is overwritten
      for (int base = v0; base < v1; base += FF_CT) {
        const int v = base + threadIdx.x;
        const int to = v < v1 ? P.vmap[v] : -1;
        double2 V = make_double2(0, 0);
        float4 Vf = make_float4(0, 0, 0, 0);
        int vs = -1, vt = -1;
        if (to >= 0) {
          V = P.V[v];
          Vf = P.Vf[v];
          vs = P.vseg[v];
          vt = P.vtri[v];
        }
        __syncthreads();
        if (to >= 0) {
          P.V[to] = V;
          P.Vf[to] = Vf;
          P.vseg[to] = vs;
          P.vtri[to] = vt;
          P.vred[to] = 0;
        }
        __syncthreads();
      }
    }
    if (threadIdx.x == 0) {
      P.mi[m].vert_count = M.vert_count - removed;
      P.mi[m].tmp = 0;
    }
    __syncthreads();
  }
}

}  // namespace gdp
