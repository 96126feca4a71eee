// The initial CDT on the GPU (Algorithm 1 line 1).
//
// 1. Point insertion in parallel rounds into one enclosing triangle per mesh.
//    Every pending point walks to the triangle containing it; each triangle
//    keeps the point with the largest (round, hash) key (at most one
//    splitting point per triangle, Sec. 4.3); those points go through the same
//    cavity kernels as refinement (grow, marks, dependence check, fan).
// 2. Segment recovery: each missing segment collects the triangles it
//    crosses, claims them and their neighbours with a 64-bit atomicMax mark,
//    and the owner flips crossing edges until the segment is an edge, then
//    restores the constrained Delaunay property inside its region by Lawson
//    flips (the paper's flip criterion: an edge is flipped when the opposite
//    angles sum to more than pi, i.e. incircle > 0).
// 3. Triangles reachable from the enclosing vertices without crossing a
//    segment are removed and the survivors are compacted per mesh.
#pragma once
#include "gdp_kernels.cuh"

namespace gdp {

// one block per mesh: bounding box, enclosing triangle, pending point list
__global__ void k_cdt_init(Pool P) {
  const int m = blockIdx.x;
  MeshInfo& M = P.mi[m];
  __shared__ double sx0[BS], sx1[BS], sy0[BS], sy1[BS];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
  for (int k = threadIdx.x; k < M.n_in; k += blockDim.x) {
    const int v = M.vert_base + k;
    const double2 p = P.V[v];
    if (!isfinite(p.x) || !isfinite(p.y)) bad = 1;
    x0 = fmin(x0, p.x); x1 = fmax(x1, p.x);
    y0 = fmin(y0, p.y); y1 = fmax(y1, p.y);
    P.loc[v] = M.tri_base;
    P.vseg[v] = -1;
    P.pts[M.pts_base + k] = v;
  }
  sx0[threadIdx.x] = x0; sx1[threadIdx.x] = x1; sy0[threadIdx.x] = y0; sy1[threadIdx.x] = y1;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sx0[threadIdx.x] = fmin(sx0[threadIdx.x], sx0[threadIdx.x + s]);
      sx1[threadIdx.x] = fmax(sx1[threadIdx.x], sx1[threadIdx.x + s]);
      sy0[threadIdx.x] = fmin(sy0[threadIdx.x], sy0[threadIdx.x + s]);
      sy1[threadIdx.x] = fmax(sy1[threadIdx.x], sy1[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (bad || M.n_in < 3) {
      M.status = S_INPUT;
      M.active = 0;
    }
    const double cx = 0.5 * (sx0[0] + sx1[0]), cy = 0.5 * (sy0[0] + sy1[0]);
    double D = fmax(sx1[0] - sx0[0], sy1[0] - sy0[0]);
    if (!(D > 0)) D = 1.0;
    M.lo = make_double2(sx0[0], sy0[0]);
    M.hi = make_double2(sx1[0], sy1[0]);
    M.org = make_double2(cx, cy);
    const int s0 = M.vert_base + M.n_in;
    P.V[s0] = make_double2(cx - 64 * D, cy - 64 * D);
    P.V[s0 + 1] = make_double2(cx + 64 * D, cy - 64 * D);
    P.V[s0 + 2] = make_double2(cx, cy + 64 * D);
    for (int k = 0; k < 3; ++k) {
      P.vseg[s0 + k] = -1;
      P.vtri[s0 + k] = M.tri_base;
    }
    const double d = 0.5 * D;
    P.V[s0 + 3] = make_double2(sx0[0] - d, sy0[0] - d);
    P.V[s0 + 4] = make_double2(sx1[0] + d, sy0[0] - d);
    P.V[s0 + 5] = make_double2(sx1[0] + d, sy1[0] + d);
    P.V[s0 + 6] = make_double2(sx0[0] - d, sy1[0] + d);
    for (int k = 3; k < N_AUX; ++k) {
      P.vseg[s0 + k] = -1;
      P.loc[s0 + k] = M.tri_base;
      P.pts[M.pts_base + M.n_in + k - 3] = s0 + k;
    }
    for (int k = 0; k < N_AUX; ++k) P.Vf[s0 + k] = to_f(P.V[s0 + k], M.org);
    P.T[M.tri_base] = make_int4(s0, s0 + 1, s0 + 2, m << 4);
    P.N[M.tri_base] = make_int4(-1, -1, -1, 0);
    M.tri_count = 1;
    M.vert_count = M.n_in + N_AUX;
  }
  __syncthreads();
  const double2 org = M.org;
  for (int k = threadIdx.x; k < M.n_in; k += blockDim.x) {
    const int v = M.vert_base + k;
    P.Vf[v] = to_f(P.V[v], org);
  }
}

// every pending point walks to its triangle and bids for it
__global__ void __launch_bounds__(BS) k_cdt_locate(Pool P, int round, int stop_cons) {
  const int n = P.ctrl->n_pts;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int k = gt; k < n; k += gs) {
    const int v = P.pts[k];
    const double2 p = P.V[v];
    int bt, be;
    const int t = walk(P, P.loc[v], pt(P, v), false, bt, be);
    if (t < 0) {
      set_err(P.ctrl, t == -2 ? S_WALK : S_INTERNAL);
      continue;
    }
    P.loc[v] = t;
    const int4 T4 = P.T[t];
    const int m = T4.w >> 4;
    bool dup = false;
    for (int e = 0; e < 3; ++e) {
      const double2 q = P.V[comp(T4, e)];
      dup |= (q.x == p.x && q.y == p.y);
    }
    if (stop_cons) {
      // inserted points must not lie on a subsegment
      for (int e = 0; e < 3; ++e)
        if (((T4.w >> e) & 1) &&
            orient(pt(P, comp(T4, mod3(e + 1))), pt(P, comp(T4, mod3(e + 2))), pt(P, v)) == 0)
          dup = true;
    }
    if (dup) {
      P.mi[m].status = S_INPUT;
      set_err(P.ctrl, S_INPUT);
      continue;
    }
    const unsigned long long key = ((unsigned long long)round << 52) |
                                   ((unsigned long long)(insert_prio(P.mi[m], v) >> 12) << 32) |
                                   (unsigned)v;
    atomicMax(&P.tbest[t], key);
  }
}

// stable compaction of the winners of their triangle into the candidate list
__global__ void __launch_bounds__(BS) k_cdt_pick_count(Pool P, int round) {
  __shared__ int sm[33];
  const Chunk ch = chunk_of(P.ctrl->n_pts);
  int cnt = 0;
  for (int k = ch.b0 + threadIdx.x; k < ch.b1; k += BS) {
    const int v = P.pts[k];
    const unsigned long long tb = P.tbest[P.loc[v]];
    cnt += ((int)(unsigned)(tb & 0xffffffffull) == v && (int)(tb >> 52) == round) ? 1 : 0;
  }
  cnt = block_sum(cnt, sm);
  if (threadIdx.x == 0) P.blk[blockIdx.x] = cnt;
}

__global__ void __launch_bounds__(BS) k_cdt_pick_write(Pool P, int round) {
  __shared__ int sm[33];
  const Chunk ch = chunk_of(P.ctrl->n_pts);
  int off = block_prefix(P.blk, blockIdx.x, sm);
  const int cap = P.cap_cand;
  for (int base = ch.b0; base < ch.b1; base += BS) {
    const int k = base + threadIdx.x;
    int win = 0, v = -1;
    if (k < ch.b1) {
      v = P.pts[k];
      const unsigned long long tb = P.tbest[P.loc[v]];
      win = ((int)(unsigned)(tb & 0xffffffffull) == v && (int)(tb >> 52) == round) ? 1 : 0;
    }
    int tot;
    const int r = block_excl_scan(win, sm, tot);
    if (win && off + r < cap) {
      P.c_elem[off + r] = v;
      P.c_loc[off + r] = P.loc[v];
    }
    off += tot;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    const int n = min(off, cap);
    P.ctrl->n_cand = n;
    P.ctrl->prev_cand = n;
  }
}

// drop inserted points from the pending list (stable)
__global__ void __launch_bounds__(BS) k_cdt_keep_count(Pool P) {
  __shared__ int sm[33];
  const Chunk ch = chunk_of(P.ctrl->n_pts);
  int cnt = 0;
  for (int k = ch.b0 + threadIdx.x; k < ch.b1; k += BS) cnt += P.loc[P.pts[k]] >= 0 ? 1 : 0;
  cnt = block_sum(cnt, sm);
  if (threadIdx.x == 0) P.blk[blockIdx.x] = cnt;
}

__global__ void __launch_bounds__(BS) k_cdt_keep_write(Pool P) {
  __shared__ int sm[33];
  const Chunk ch = chunk_of(P.ctrl->n_pts);
  int off = block_prefix(P.blk, blockIdx.x, sm);
  for (int base = ch.b0; base < ch.b1; base += BS) {
    const int k = base + threadIdx.x;
    int keep = 0, v = -1;
    if (k < ch.b1) {
      v = P.pts[k];
      keep = P.loc[v] >= 0 ? 1 : 0;
    }
    int tot;
    const int r = block_excl_scan(keep, sm, tot);
    if (keep) P.pts2[off + r] = v;
    off += tot;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) P.ctrl->n_pts = off;
}

// ---------------------------------------------------------------- segment recovery
__device__ __forceinline__ int idx_of(const int4& T4, int v) {
  return T4.x == v ? 0 : (T4.y == v ? 1 : (T4.z == v ? 2 : -1));
}

__device__ __forceinline__ void set_nb(const Pool& P, int ref, int val) {
  if (ref >= 0) *comp_ptr(&P.N[ref >> 2], ref & 3) = val;
}

// Flip edge e1 of t1 (shared with t2): quad p1,u,o,v (CCW) gets the diagonal p1-o.
// t1 = (p1,u,v) -> (p1,u,o);  t2 = (o,v,u) -> (p1,o,v).  Outside neighbours are
// re-pointed; subsegment bits move with their edges.
__device__ void flip(const Pool& P, int t1, int e1) {
  const int4 A = P.T[t1], NA = P.N[t1];
  const int ref = comp(NA, e1);
  const int t2 = ref >> 2, e2 = ref & 3;
  const int4 B = P.T[t2], NB = P.N[t2];
  const int p1 = comp(A, e1), u = comp(A, mod3(e1 + 1)), v = comp(A, mod3(e1 + 2));
  const int o = comp(B, e2);
  const int m = A.w >> 4;
  // outer edges: (p1,u) = A opp v [e1+2]; (v,p1) = A opp u [e1+1];
  //              (u,o)  = B opp v [e2+1]; (o,v)  = B opp u [e2+2]
  const int r_pu = comp(NA, mod3(e1 + 2)), r_vp = comp(NA, mod3(e1 + 1));
  const int r_uo = comp(NB, mod3(e2 + 1)), r_ov = comp(NB, mod3(e2 + 2));
  const int c_pu = (A.w >> mod3(e1 + 2)) & 1, c_vp = (A.w >> mod3(e1 + 1)) & 1;
  const int c_uo = (B.w >> mod3(e2 + 1)) & 1, c_ov = (B.w >> mod3(e2 + 2)) & 1;
  // t1' = (p1, u, o): e0 = (u,o), e1 = (o,p1) -> t2' e2, e2 = (p1,u)
  // t2' = (p1, o, v): e0 = (o,v), e1 = (v,p1), e2 = (p1,o) -> t1' e1
  P.T[t1] = make_int4(p1, u, o, (m << 4) | c_uo | (c_pu << 2));
  P.N[t1] = make_int4(r_uo, (t2 << 2) | 2, r_pu, 0);
  P.T[t2] = make_int4(p1, o, v, (m << 4) | c_ov | (c_vp << 1));
  P.N[t2] = make_int4(r_ov, r_vp, (t1 << 2) | 1, 0);
  set_nb(P, r_uo, (t1 << 2) | 0);
  set_nb(P, r_pu, (t1 << 2) | 2);
  set_nb(P, r_ov, (t2 << 2) | 0);
  set_nb(P, r_vp, (t2 << 2) | 1);
}

__device__ __forceinline__ bool crosses_seg(const Pool& P, int a, int b, int u, int v) {
  if (u == a || u == b || v == a || v == b) return false;
  const P2 A = pt(P, a), B = pt(P, b), U = pt(P, u), W = pt(P, v);
  return orient(A, B, U) * orient(A, B, W) < 0 && orient(U, W, A) * orient(U, W, B) < 0;
}

__device__ __forceinline__ unsigned long long seg_key(int round, int s, int k) {
  return ((unsigned long long)(round + 1) << 48) |
         ((unsigned long long)(hash32((uint32_t)s) & 0xffffu) << 32) | (unsigned)k;
}

// reg_n[k]: > 0 crossed triangles collected; -1 recovered; -2 error
__global__ void __launch_bounds__(BS) k_seg_find(Pool P, int round) {
  const int n = min(P.ctrl->n_segs, P.cap_segq);
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int k = gt; k < n; k += gs) {
    const int s = P.segq[k];
    const int a = P.seg[s].x, b = P.seg[s].y;
    if (a == b) {   // rejected at input (its mesh carries the status)
      P.reg_n[k] = -1;
      continue;
    }
    int t = P.vtri[a];
    const int m = P.T[t].w >> 4;
    int start = -1, ia = -1, status = 0;
    for (int it = 0; it < 4096 && start < 0 && status == 0; ++it) {
      const int4 T4 = P.T[t];
      const int i = idx_of(T4, a);
      if (i < 0) { status = S_INTERNAL; break; }
      const int u = comp(T4, mod3(i + 1)), w = comp(T4, mod3(i + 2));
      if (u == b || w == b) {
        const int e = (u == b) ? mod3(i + 2) : mod3(i + 1);
        atomicOr(&P.T[t].w, 1 << e);
        const int nb = comp(P.N[t], e);
        if (nb >= 0) atomicOr(&P.T[nb >> 2].w, 1 << (nb & 3));
        status = -1;
        break;
      }
      const P2 A = pt(P, a), B = pt(P, b);
      const int o1 = orient(A, pt(P, u), B), o2 = orient(A, pt(P, w), B);
      if (o1 == 0 && dot_sign(pt(P, u), B, A) > 0) { status = S_INPUT; break; }
      if (o1 > 0 && o2 < 0) { start = t; ia = i; break; }
      const int nb = comp(P.N[t], mod3(i + 2));   // clockwise: across (a, u)
      if (nb < 0) { status = S_INTERNAL; break; }
      t = nb >> 2;
    }
    if (status == 0 && start < 0) status = S_INTERNAL;
    if (status != 0) {
      if (status > 0) {
        P.mi[m].status = status;
        set_err(P.ctrl, status);
        P.reg_n[k] = -2;
      } else {
        P.reg_n[k] = -1;
      }
      continue;
    }
    int* R = P.reg + (size_t)k * KMAX;
    int cnt = 0;
    R[cnt++] = start;
    const int4 S4 = P.T[start];
    int l = comp(S4, mod3(ia + 2)), r = comp(S4, mod3(ia + 1));
    int ref = comp(P.N[start], ia);
    if ((S4.w >> ia) & 1) status = S_INPUT;
    for (; status == 0;) {
      if (ref < 0) { status = S_INTERNAL; break; }
      if (cnt == KMAX) { status = S_CAPACITY; break; }
      const int tn = ref >> 2, ee = ref & 3;
      if ((P.T[tn].w >> ee) & 1) { status = S_INPUT; break; }   // crosses a recovered segment
      R[cnt++] = tn;
      const int4 T4 = P.T[tn];
      const int z = comp(T4, ee);
      if (z == b) break;
      const int o = orient(pt(P, a), pt(P, b), pt(P, z));
      if (o == 0) { status = S_INPUT; break; }
      if (o > 0) {
        ref = comp(P.N[tn], idx_of(T4, l));
        l = z;
      } else {
        ref = comp(P.N[tn], idx_of(T4, r));
        r = z;
      }
    }
    if (status != 0) {
      P.mi[m].status = status;
      set_err(P.ctrl, status);
      P.reg_n[k] = -2;
      continue;
    }
    P.reg_n[k] = cnt;
    const unsigned long long key = seg_key(round, s, k);
    for (int j = 0; j < cnt; ++j) {
      atomicMax(&P.segmark[R[j]], key);
      const int4 N4 = P.N[R[j]];
      for (int e = 0; e < 3; ++e) {
        const int nb = comp(N4, e);
        if (nb >= 0) atomicMax(&P.segmark[nb >> 2], key);
      }
    }
  }
}

__device__ int region_find_edge(const Pool& P, const int* R, int cnt, int u, int v, int& e) {
  for (int j = 0; j < cnt; ++j) {
    const int4 T4 = P.T[R[j]];
    for (int q = 0; q < 3; ++q)
      if (comp(T4, mod3(q + 1)) == u && comp(T4, mod3(q + 2)) == v) { e = q; return R[j]; }
  }
  return -1;
}

__device__ __forceinline__ bool in_region(const int* R, int cnt, int t) {
  for (int j = 0; j < cnt; ++j)
    if (R[j] == t) return true;
  return false;
}

// the owner of a region makes the segment an edge by flips, then restores the
// constrained Delaunay property inside the region
__global__ void __launch_bounds__(BS) k_seg_apply(Pool P, int round, int2* work) {
  const int n = min(P.ctrl->n_segs, P.cap_segq);
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int k = gt; k < n; k += gs) {
    const int cnt = P.reg_n[k];
    if (cnt <= 0) continue;
    const int s = P.segq[k];
    const unsigned long long key = seg_key(round, s, k);
    const int* R = P.reg + (size_t)k * KMAX;
    bool own = true;
    for (int j = 0; j < cnt && own; ++j) {
      own = P.segmark[R[j]] == key;
      const int4 N4 = P.N[R[j]];
      for (int e = 0; e < 3 && own; ++e) {
        const int nb = comp(N4, e);
        if (nb >= 0) own = P.segmark[nb >> 2] == key;
      }
    }
    if (!own) continue;
    const int a = P.seg[s].x, b = P.seg[s].y;
    const int m = P.T[R[0]].w >> 4;
    // crossing edges, as vertex pairs, in a circular queue
    int2* Q = work + (size_t)k * KMAX;
    int qh = 0, qn = 0;
    for (int j = 0; j + 1 < cnt; ++j) {
      const int4 T4 = P.T[R[j]];
      const int4 N4 = P.N[R[j]];
      for (int e = 0; e < 3; ++e)
        if (comp(N4, e) >= 0 && (comp(N4, e) >> 2) == R[j + 1]) {
          Q[qn++] = make_int2(comp(T4, mod3(e + 1)), comp(T4, mod3(e + 2)));
          break;
        }
    }
    int status = 0;
    long long steps = 0;
    const long long limit = 64ll * cnt * cnt + 256;
    while (qn > 0 && status == 0) {
      if (++steps > limit) { status = S_INTERNAL; break; }
      const int2 ed = Q[qh];
      qh = (qh + 1) % KMAX;
      --qn;
      int e1 = -1;
      int t1 = region_find_edge(P, R, cnt, ed.x, ed.y, e1);
      if (t1 < 0) { status = S_INTERNAL; break; }
      const int4 A = P.T[t1];
      const int ref = comp(P.N[t1], e1);
      if (ref < 0) { status = S_INTERNAL; break; }
      const int4 B = P.T[ref >> 2];
      const int p1 = comp(A, e1), u = comp(A, mod3(e1 + 1)), v = comp(A, mod3(e1 + 2));
      const int o = comp(B, ref & 3);
      if (orient(pt(P, p1), pt(P, u), pt(P, o)) > 0 && orient(pt(P, p1), pt(P, o), pt(P, v)) > 0) {
        flip(P, t1, e1);
        if (crosses_seg(P, a, b, p1, o)) {
          Q[(qh + qn) % KMAX] = make_int2(p1, o);
          ++qn;
        }
      } else {
        Q[(qh + qn) % KMAX] = ed;
        ++qn;
      }
    }
    if (status == 0) {
      int e = -1;
      int t = region_find_edge(P, R, cnt, a, b, e);
      if (t < 0) t = region_find_edge(P, R, cnt, b, a, e);
      if (t < 0) {
        status = S_INTERNAL;
      } else {
        P.T[t].w |= 1 << e;
        const int nb = comp(P.N[t], e);
        if (nb >= 0) P.T[nb >> 2].w |= 1 << (nb & 3);
      }
    }
    // Lawson flips on the region's interior, non-subsegment edges
    for (int pass = 0; status == 0; ++pass) {
      if (pass > 4 * cnt + 16) { status = S_INTERNAL; break; }
      bool any = false;
      for (int j = 0; j < cnt; ++j) {
        const int t = R[j];
        for (int e = 0; e < 3; ++e) {
          const int4 T4 = P.T[t];
          const int ref = comp(P.N[t], e);
          if (ref < 0 || ((T4.w >> e) & 1)) continue;
          const int t2 = ref >> 2;
          if (!in_region(R, cnt, t2)) continue;
          const int o = comp(P.T[t2], ref & 3);
          if (incircle(pt(P, T4.x), pt(P, T4.y), pt(P, T4.z), pt(P, o)) > 0) {
            const int p1 = comp(T4, e), u = comp(T4, mod3(e + 1)), v = comp(T4, mod3(e + 2));
            if (orient(pt(P, p1), pt(P, u), pt(P, o)) > 0 && orient(pt(P, p1), pt(P, o), pt(P, v)) > 0) {
              flip(P, t, e);
              any = true;
            }
          }
        }
      }
      if (!any) break;
    }
    if (status != 0) {
      P.mi[m].status = status;
      set_err(P.ctrl, status);
      P.reg_n[k] = -2;
      continue;
    }
    for (int j = 0; j < cnt; ++j) {
      const int4 T4 = P.T[R[j]];
      P.vtri[T4.x] = R[j];
      P.vtri[T4.y] = R[j];
      P.vtri[T4.z] = R[j];
    }
    P.reg_n[k] = -1;
  }
}

// keep segments that still need work (stable); the rest of the list beyond
// the per-round capacity is kept as is
__global__ void __launch_bounds__(BS) k_seg_keep_count(Pool P) {
  __shared__ int sm[33];
  const int n = P.ctrl->n_segs, na = min(n, P.cap_segq);
  const Chunk ch = chunk_of(n);
  int cnt = 0;
  for (int k = ch.b0 + threadIdx.x; k < ch.b1; k += BS) cnt += (k >= na || P.reg_n[k] >= 0) ? 1 : 0;
  cnt = block_sum(cnt, sm);
  if (threadIdx.x == 0) P.blk[blockIdx.x] = cnt;
}

__global__ void __launch_bounds__(BS) k_seg_keep_write(Pool P) {
  __shared__ int sm[33];
  const int n = P.ctrl->n_segs, na = min(n, P.cap_segq);
  const Chunk ch = chunk_of(n);
  int off = block_prefix(P.blk, blockIdx.x, sm);
  for (int base = ch.b0; base < ch.b1; base += BS) {
    const int k = base + threadIdx.x;
    int keep = 0;
    if (k < ch.b1) keep = (k >= na || P.reg_n[k] >= 0) ? 1 : 0;
    int tot;
    const int r = block_excl_scan(keep, sm, tot);
    if (keep) P.segq2[off + r] = P.segq[k];
    off += tot;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) P.ctrl->n_segs = off;
}

// ---------------------------------------------------------------- exterior + compaction
__device__ __forceinline__ int mesh_of_slot(const Pool& P, int t) {
  int lo = 0, hi = P.n_mesh - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.mi[mid].tri_base <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ext: 0 inside, 1 exterior, 2 unused slot
__global__ void __launch_bounds__(BS) k_ext_init(Pool P) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int t = gt; t < P.n_slots; t += gs) {
    const int4 T4 = P.T[t];
    if (T4.w < 0) { P.ext[t] = 2; continue; }
    const MeshInfo& M = P.mi[T4.w >> 4];
    P.ext[t] = (is_aux(M, T4.x) || is_aux(M, T4.y) || is_aux(M, T4.z)) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(BS) k_ext_step(Pool P) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  int changed = 0;
  for (int t = gt; t < P.n_slots; t += gs) {
    if (P.ext[t] != 0) continue;
    const int4 T4 = P.T[t], N4 = P.N[t];
    for (int e = 0; e < 3; ++e) {
      const int nb = comp(N4, e);
      if (nb >= 0 && !((T4.w >> e) & 1) && P.ext[nb >> 2] == 1) {
        P.ext[t] = 1;
        changed = 1;
        break;
      }
    }
  }
  if (changed) P.ctrl->changed = 1;
}

// remap[t]: exclusive count of interior slots before t (all slots, stable)
__global__ void __launch_bounds__(BS) k_live_count(Pool P) {
  __shared__ int sm[33];
  const Chunk ch = chunk_of(P.n_slots);
  int cnt = 0;
  for (int t = ch.b0 + threadIdx.x; t < ch.b1; t += BS) cnt += P.ext[t] == 0 ? 1 : 0;
  cnt = block_sum(cnt, sm);
  if (threadIdx.x == 0) P.blk[blockIdx.x] = cnt;
}

__global__ void __launch_bounds__(BS) k_live_write(Pool P) {
  __shared__ int sm[33];
  const Chunk ch = chunk_of(P.n_slots);
  int off = block_prefix(P.blk, blockIdx.x, sm);
  for (int base = ch.b0; base < ch.b1; base += BS) {
    const int t = base + threadIdx.x;
    const int live = (t < ch.b1 && P.ext[t] == 0) ? 1 : 0;
    int tot;
    const int r = block_excl_scan(live, sm, tot);
    if (t < ch.b1) P.remap[t] = off + r;
    off += tot;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) P.remap[P.n_slots] = off;
}

__device__ __forceinline__ int new_slot(const Pool& P, int t) {
  const int m = P.T[t].w >> 4;
  const int b = P.mi[m].tri_base;
  return b + P.remap[t] - P.remap[b];
}

__global__ void __launch_bounds__(BS) k_compact_move(Pool P, int4* T2, int4* N2) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int t = gt; t < P.n_slots; t += gs) {
    if (P.ext[t] != 0) continue;
    const int4 T4 = P.T[t], N4 = P.N[t];
    int nn[3];
    for (int e = 0; e < 3; ++e) {
      const int r = comp(N4, e);
      nn[e] = (r >= 0 && P.ext[r >> 2] == 0) ? ((new_slot(P, r >> 2) << 2) | (r & 3)) : -1;
    }
    const int ns = new_slot(P, t);
    T2[ns] = T4;
    N2[ns] = make_int4(nn[0], nn[1], nn[2], 0);
  }
}

// per mesh: new triangle count; every slot: copy back, clear, mark dirty
__global__ void __launch_bounds__(BS) k_compact_finish(Pool P, const int4* T2, const int4* N2) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int m = gt; m < P.n_mesh; m += gs) {
    const int b = P.mi[m].tri_base;
    const int e = b + P.mi[m].tri_cap;
    P.mi[m].tmp = P.remap[e] - P.remap[b];   // staged count, applied below
  }
  for (int t = gt; t < P.n_slots; t += gs) {
    const int m = mesh_of_slot(P, t);
    const int b = P.mi[m].tri_base;
    const int cnt = P.remap[b + P.mi[m].tri_cap] - P.remap[b];
    if (t - b < cnt) {
      P.T[t] = T2[t];
      P.N[t] = N2[t];
      P.dirty[t] = 1;
    } else {
      P.T[t] = make_int4(-1, -1, -1, -1);
      P.N[t] = make_int4(-1, -1, -1, -1);
      P.dirty[t] = 0;
    }
    P.mark[t] = 0ull;
  }
}

__global__ void k_compact_counts(Pool P) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int m = gt; m < P.n_mesh; m += gs) {
    P.mi[m].tri_count = P.mi[m].tmp;
    if (P.mi[m].tri_count == 0 && P.mi[m].status == S_OK) P.mi[m].status = S_INPUT;
  }
}

}  // namespace gdp
