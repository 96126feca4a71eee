// The initial CDT on the GPU (the first step of Algorithm 1).
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

// Construction set-up, per mesh over a 2D grid (x: blocks of one mesh, y:
// meshes).  k_cdt_bbox: partial bounding boxes (4 doubles per block) and the
// pending point list; k_cdt_init (one block per mesh): the box, the enclosing
// triangle and the frame; k_cdt_vf: the float copies of the input points.
__global__ void __launch_bounds__(BS) k_cdt_bbox(Pool P, double* part) {
  __shared__ double sx0[BS], sx1[BS], sy0[BS], sy1[BS];
  for (int m = blockIdx.y; m < P.n_mesh; m += gridDim.y) {
    MeshInfo& M = P.mi[m];
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (int k = blockIdx.x * BS + threadIdx.x; k < M.n_in; k += gridDim.x * BS) {
      const int v = M.vert_base + k;
      const double2 p = P.V[v];
      if (!isfinite(p.x) || !isfinite(p.y)) M.status = S_INPUT;
      x0 = fmin(x0, p.x); x1 = fmax(x1, p.x);
      y0 = fmin(y0, p.y); y1 = fmax(y1, p.y);
      P.loc[v] = M.tri_base;
      P.vseg[v] = -1;
      P.pts[M.pts_base + k] = v;
    }
    sx0[threadIdx.x] = x0; sx1[threadIdx.x] = x1; sy0[threadIdx.x] = y0; sy1[threadIdx.x] = y1;
    __syncthreads();
    for (int s = BS / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        sx0[threadIdx.x] = fmin(sx0[threadIdx.x], sx0[threadIdx.x + s]);
        sx1[threadIdx.x] = fmax(sx1[threadIdx.x], sx1[threadIdx.x + s]);
        sy0[threadIdx.x] = fmin(sy0[threadIdx.x], sy0[threadIdx.x + s]);
        sy1[threadIdx.x] = fmax(sy1[threadIdx.x], sy1[threadIdx.x + s]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double* q = part + 4 * ((size_t)m * gridDim.x + blockIdx.x);
      q[0] = sx0[0]; q[1] = sx1[0]; q[2] = sy0[0]; q[3] = sy1[0];
    }
    __syncthreads();
  }
}

__global__ void k_cdt_init(Pool P, const double* part, int bx, double frame) {
  const int m = blockIdx.x;
  MeshInfo& M = P.mi[m];
  if (threadIdx.x == 0) {
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (int b = 0; b < bx; ++b) {
      const double* q = part + 4 * ((size_t)m * bx + b);
      x0 = fmin(x0, q[0]); x1 = fmax(x1, q[1]);
      y0 = fmin(y0, q[2]); y1 = fmax(y1, q[3]);
    }
    if (M.status == S_INPUT || M.n_in < 3) {
      M.status = S_INPUT;
      M.active = 0;
    }
    const double cx = 0.5 * (x0 + x1), cy = 0.5 * (y0 + y1);
    double D = fmax(x1 - x0, y1 - y0);
    if (!(D > 0)) D = 1.0;
    M.lo = make_double2(x0, y0);
    M.hi = make_double2(x1, y1);
    M.org = make_double2(cx, cy);
    const int s0 = M.vert_base + M.n_in;
    P.V[s0] = make_double2(cx - 64 * D, cy - 64 * D);
    P.V[s0 + 1] = make_double2(cx + 64 * D, cy - 64 * D);
    P.V[s0 + 2] = make_double2(cx, cy + 64 * D);
    for (int k = 0; k < 3; ++k) {
      P.vseg[s0 + k] = -1;
      P.vtri[s0 + k] = M.tri_base;
    }
    // frame 16 D out (inside the enclosing triangle): far enough that few
    // Delaunay edges from interior points to the frame cross the input's
    // hull, so boundary segments are mostly edges already
    const double d = frame * D;
    P.V[s0 + 3] = make_double2(x0 - d, y0 - d);
    P.V[s0 + 4] = make_double2(x1 + d, y0 - d);
    P.V[s0 + 5] = make_double2(x1 + d, y1 + d);
    P.V[s0 + 6] = make_double2(x0 - d, y1 + d);
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
}

__global__ void __launch_bounds__(BS) k_cdt_vf(Pool P) {
  for (int m = blockIdx.y; m < P.n_mesh; m += gridDim.y) {
    const MeshInfo& M = P.mi[m];
    const double2 org = M.org;
    for (int k = blockIdx.x * BS + threadIdx.x; k < M.n_in; k += gridDim.x * BS) {
      const int v = M.vert_base + k;
      P.Vf[v] = to_f(P.V[v], org);
    }
  }
}

// every pending point walks to its triangle and bids for it
// Which pending point a triangle takes this round (20 bits, larger first):
// the frame vertices, then the point nearest the triangle's circumcentre.
// A point there tends to lie in no neighbour's circumcircle, so its cavity
// is often the triangle alone and neighbouring candidates rarely collide.
// Any deterministic choice gives the same triangulation; FP32 is enough.
__device__ __forceinline__ uint32_t pick_measure(const Pool& P, const MeshInfo& M, int v,
                                                 const int4& T4) {
  if (is_aux(M, v)) return 0xfffffu;
  const float4 a = P.Vf[T4.x], b = P.Vf[T4.y], c = P.Vf[T4.z], q = P.Vf[v];
  const float dx = b.x - a.x, dy = b.y - a.y, ex = c.x - a.x, ey = c.y - a.y;
  const float d2 = dx * dx + dy * dy, e2 = ex * ex + ey * ey;
  const float D = 2.0f * (dx * ey - dy * ex);
  const float rx = q.x - a.x - (ey * d2 - dy * e2) / D;
  const float ry = q.y - a.y - (dx * e2 - ex * d2) / D;
  const float r2 = rx * rx + ry * ry;
  const uint32_t bits = (r2 >= 0.0f && r2 < INFINITY) ? __float_as_uint(r2) : 0x7f800000u;
  return 0xffffeu - min(bits >> 11, 0xffffeu);
}

// split: points on an edge of their triangle take no part in the pick (the
// split rounds insert only points strictly inside a triangle)
// resident blocks per SM the register allocation of k_cdt_locate aims at (the
// walks are latency-bound: more resident warps hide more of it)
#ifndef GDP_LOCATE_BLOCKS
#define GDP_LOCATE_BLOCKS 2
#endif
__global__ void __launch_bounds__(BS, GDP_LOCATE_BLOCKS) k_cdt_locate(Pool P, int stop_cons, int split) {
  const unsigned FULL = 0xffffffffu;
  const int n = P.ctrl->n_pts;
  const int round = P.ctrl->round;
  const int lane = threadIdx.x & 31;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int k0 = gt - lane; k0 < n; k0 += gs) {   // whole warps: the bids are combined per warp
    const int k = k0 + lane;
    bool bid = false;
    int t = -1;
    unsigned long long key = 0ull;
    if (k < n) {
      const int v = P.pts[k];
      const P2 pv = pt(P, v);
      int bt, be;
      int steps = 0;
      t = walk(P, P.loc[v], pv, false, bt, be, steps);
      if (t < 0) {
        set_err(P.ctrl, t == -2 ? S_WALK : S_INTERNAL);
      } else {
        P.loc[v] = t;
        const int4 T4 = P.T[t];
        const int m = T4.w >> 4;
        // a duplicate of a vertex of its triangle: equal points have equal
        // two-float copies (the walk has just read them), so the FP64
        // coordinates are compared only when those match
        bool dup = false;
        for (int e = 0; e < 3; ++e) {
          const int w = comp(T4, e);
          const float4 qf = P.Vf[w];
          if (qf.x == pv.f.x && qf.y == pv.f.y && qf.z == pv.f.z && qf.w == pv.f.w) {
            const double2 q = P.V[w];
            dup |= (q.x == pv.d.x && q.y == pv.d.y);
          }
        }
        if (stop_cons) {
          // inserted points must not lie on a subsegment
          for (int e = 0; e < 3; ++e)
            if (((T4.w >> e) & 1) && orient_ids(P, comp(T4, mod3(e + 1)), comp(T4, mod3(e + 2)), pv) == 0)
              dup = true;
        }
        bool edge = false;
        if (dup) {
          P.mi[m].status = S_INPUT;
          set_err(P.ctrl, S_INPUT);
        } else if (split) {
          for (int e = 0; e < 3; ++e) edge |= orient_ids(P, comp(T4, mod3(e + 1)), comp(T4, mod3(e + 2)), pv) == 0;
        }
        if (!dup && !edge) {
          bid = true;
          key = ((unsigned long long)round << 52) |
                ((unsigned long long)pick_measure(P, P.mi[m], v, T4) << 32) | (unsigned)v;
        }
      }
    }
    // the largest bid per triangle among the warp's lanes, then one atomic per
    // triangle: in the first rounds a million points bid for a few triangles,
    // and same-address atomics serialise
    const unsigned peers = __match_any_sync(FULL, bid ? t : -1 - lane);
    const unsigned hi = __reduce_max_sync(peers, (unsigned)(key >> 32));
    const unsigned lo = __reduce_max_sync(peers, (unsigned)(key >> 32) == hi ? (unsigned)key : 0u);
    if (bid && lane == __ffs(peers) - 1) atomicMax(&P.tbest[t], ((unsigned long long)hi << 32) | lo);
  }
}

// stable compaction of the winners of their triangle into the candidate list
__global__ void __launch_bounds__(BS) k_cdt_pick_count(Pool P) {
  __shared__ int sm[33];
  const int round = P.ctrl->round;
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

__global__ void __launch_bounds__(BS) k_cdt_pick_write(Pool P) {
  __shared__ int sm[33];
  const int round = P.ctrl->round;
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
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) P.ctrl->n_pts_next = off;
}

// end of a round (one thread): the next round's count and number.  Every
// block of the round's kernels read n_pts and round at its start, so they
// change only here, between kernels.
__global__ void k_cdt_next(Pool P) {
  if (P.ctrl->n_pts > 0) ++P.ctrl->round;
  P.ctrl->n_pts = P.ctrl->n_pts_next;
}

// ---------------------------------------------------------------- split + flip rounds
// Point insertion for the initial CDT, before any segment is inserted: every
// triangle that holds pending points is split in three at one of them (no
// two splits touch the same triangle, so all candidates go in), and parallel
// Lawson flips of edges that fail the incircle test (with simulation of
// simplicity) restore the Delaunay triangulation, which is unique.  Each
// pass rewrites whole triangles in place and records where every outer edge
// went (newref, indexed by the old slot and edge); a link kernel then
// repairs the neighbour references across edges whose other side was also
// rewritten (tstamp == pass) and writes back the others.

// push t for the next flip pass once (pass = the pass that will read it)
__device__ __forceinline__ void fl_push(const Pool& P, int* list, int t, int pass) {
  if (atomicMax(&P.lstamp[t], pass) < pass) list[atomicAdd(&P.ctrl->n_fl_next, 1)] = t;
}

// per-mesh candidate ranges and slot counts (two new triangles per split),
// laid out like k_depend's block sums so that k_offsets can scan them
__global__ void __launch_bounds__(BS) k_split_prep(Pool P) {
  __shared__ int sm[33];
  const int n = P.ctrl->n_cand;
  const Chunk ch = chunk_of(n);
  int se = 0;
  for (int i = ch.b0 + threadIdx.x; i < ch.b1; i += BS) {
    const int v = P.c_elem[i], t = P.c_loc[i];
    const int4 T4 = P.T[t];
    const int m = T4.w >> 4;
    const P2 q = pt(P, v);
    const bool in = orient(pt(P, T4.y), pt(P, T4.z), q) > 0 && orient(pt(P, T4.z), pt(P, T4.x), q) > 0 &&
                    orient(pt(P, T4.x), pt(P, T4.y), q) > 0;
    P.c_mesh[i] = m;
    P.c_vid[i] = v;
    P.c_final[i] = in;
    P.c_extra[i] = in ? 2 : 0;
    if (i == 0 || (P.T[P.c_loc[i - 1]].w >> 4) != m) P.mi[m].first_cand = i;
    if (i == n - 1 || (P.T[P.c_loc[i + 1]].w >> 4) != m) P.mi[m].last_cand = i;
    se += in ? 2 : 0;
  }
  se = block_sum(se, sm);
  if (threadIdx.x == 0) {
    P.blk[blockIdx.x] = se;
    P.blk[gridDim.x + blockIdx.x] = 0;
  }
}

// triangle t = (a0, a1, a2) split at p: T_e = (p, a[e+1], a[e+2]) keeps the
// old edge e as its edge 0; T_0 reuses the slot of t
__global__ void __launch_bounds__(BS) k_split(Pool P) {
  const int n = P.ctrl->n_cand;
  const int step = P.ctrl->step;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int i = gt; i < n; i += gs) {
    const int m = P.c_mesh[i];
    const MeshInfo& M = P.mi[m];
    const int f = M.first_cand, l = M.last_cand;
    int totE, totV;
    mesh_totals(P, f, l, totE, totV);
    const bool ok = M.tri_count + totE <= M.tri_cap;
    if (i == f) {
      P.mi[m].ins_ok = ok ? 1 : 0;
      if (!ok) P.mi[m].status = S_NOMEM;
    }
    if (!P.c_final[i] || !ok) continue;
    const int t = P.c_loc[i], v = P.c_vid[i];
    const int base = M.tri_base + M.tri_count + (P.c_offT[i] - P.c_offT[f]);
    P.c_base[i] = base;   // k_split_link must not recompute it: tri_count moves there
    const int4 T4 = P.T[t];
    const int4 N4 = P.N[t];
    const int s[3] = {t, base, base + 1};
    for (int e = 0; e < 3; ++e) {
      P.T[s[e]] = make_int4(v, comp(T4, mod3(e + 1)), comp(T4, mod3(e + 2)), m << 4);
      P.N[s[e]] = make_int4(comp(N4, e), (s[mod3(e + 1)] << 2) | 2, (s[mod3(e + 2)] << 2) | 1, 0);
      P.newref[(t << 2) | e] = s[e] << 2;
      P.tstamp[s[e]] = step;
      fl_push(P, P.fl_nxt, s[e], step + 1);
    }
    P.loc[v] = -1;
  }
}

// outer neighbours of the split triangles, then per-mesh counts
__global__ void __launch_bounds__(BS) k_split_link(Pool P) {
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
      const int t = P.c_loc[i];
      const int base = P.c_base[i];
      for (int e = 0; e < 3; ++e) {
        const int s = e == 0 ? t : base + e - 1;
        const int r = P.N[s].x;
        if (r < 0) continue;
        if (P.tstamp[r >> 2] == step) P.N[s].x = P.newref[r];
        else *comp_ptr(&P.N[r >> 2], r & 3) = s << 2;
      }
    }
    if (i == M.last_cand && ok) {
      int totE, totV;
      mesh_totals(P, M.first_cand, i, totE, totV);
      P.mi[m].tri_count = M.tri_count + totE;
    }
  }
  for (int o = 16; o; o >>= 1) ins += __shfl_xor_sync(0xffffffffu, ins, o);
  if ((threadIdx.x & 31) == 0 && ins) atomicAdd(&P.ctrl->n_ins, (unsigned long long)ins);
}

// flip priority from mesh-local slot numbers, so that a mesh flips the same
// way alone and in a batch (keys of earlier passes compare lower)
__device__ __forceinline__ unsigned long long flip_key(const Pool& P, int step, int t, int prop) {
  const int lt = t - P.mi[P.T[t].w >> 4].tri_base;   // the mesh bits of a slot never change
  return ((unsigned long long)step << 44) | ((unsigned long long)(hash32((uint32_t)lt) & 0xfffu) << 32) |
         (unsigned)((lt << 2) | (prop & 3));
}

// each listed triangle proposes its first edge whose opposite vertex lies in
// its circumcircle; the proposal marks both triangles (atomicMax)
__device__ __forceinline__ void flip_propose_one(const Pool& P, const int* cur, int k, int step) {
  const int t = cur[k];
  const int4 T4 = P.T[t];
  const int4 N4 = P.N[t];
  int prop = -1, t2 = -1;
  const P2 a = pt(P, T4.x), b = pt(P, T4.y), c = pt(P, T4.z);
  for (int e = 0; e < 3 && prop < 0; ++e) {
    const int r = comp(N4, e);
    if (r < 0) continue;
    const int d = comp(P.T[r >> 2], r & 3);
    if (incircle(a, b, c, pt(P, d)) > 0) {
      prop = (t << 2) | e;
      t2 = r >> 2;
    }
  }
  P.fprop[k] = prop;
  if (prop >= 0) {
    const unsigned long long key = flip_key(P, step, t, prop);
    atomicMax(&P.mark[t], key);
    atomicMax(&P.mark[t2], key);
  }
}

// proposals that own both marks flip; the others try again next pass
__device__ __forceinline__ void flip_do_one(const Pool& P, int* nxt, int k, int step) {
  const int prop = P.fprop[k];
  if (prop < 0) return;
  const int t = prop >> 2, e = prop & 3;
  const unsigned long long key = flip_key(P, step, t, prop);
  // t and t2 are read only once this proposal owns them: a triangle whose
  // mark another proposal holds may be rewritten by it meanwhile
  if (__ldcg(&P.mark[t]) != key) {
    fl_push(P, nxt, t, step + 1);
    return;
  }
  const int4 T4 = P.T[t];
  const int4 N4 = P.N[t];
  const int r = comp(N4, e);
  const int t2 = r >> 2, e2 = r & 3;
  if (__ldcg(&P.mark[t2]) != key) {
    fl_push(P, nxt, t, step + 1);
    return;
  }
  const int4 U4 = P.T[t2];
  const int4 M4 = P.N[t2];
  const int a = comp(T4, e), b = comp(T4, mod3(e + 1)), c = comp(T4, mod3(e + 2));
  const int d = comp(U4, e2);
  const int nab = comp(N4, mod3(e + 2)), nca = comp(N4, mod3(e + 1));
  const int nbd = comp(M4, mod3(e2 + 1)), ndc = comp(M4, mod3(e2 + 2));
  const int info = T4.w & ~15;
  // (a, b, c) + (d, c, b) -> (a, b, d) + (a, d, c)
  P.T[t] = make_int4(a, b, d, info);
  P.N[t] = make_int4(nbd, (t2 << 2) | 2, nab, 0);
  P.T[t2] = make_int4(a, d, c, info);
  P.N[t2] = make_int4(ndc, nca, (t << 2) | 1, 0);
  P.newref[(t << 2) | mod3(e + 2)] = (t << 2) | 2;      // ab
  P.newref[(t << 2) | mod3(e + 1)] = (t2 << 2) | 1;     // ca
  P.newref[(t2 << 2) | mod3(e2 + 1)] = t << 2;          // bd
  P.newref[(t2 << 2) | mod3(e2 + 2)] = t2 << 2;         // dc
  P.tstamp[t] = step;
  P.tstamp[t2] = step;
  P.fprop[k] = -2 - prop;
  fl_push(P, nxt, t, step + 1);
  fl_push(P, nxt, t2, step + 1);
}

__device__ __forceinline__ void flip_fix(const Pool& P, int x, int idx, int step) {
  const int r = comp(P.N[x], idx);
  if (r < 0) return;
  if (P.tstamp[r >> 2] == step) *comp_ptr(&P.N[x], idx) = P.newref[r];
  else *comp_ptr(&P.N[r >> 2], r & 3) = (x << 2) | idx;
}

// outer neighbours of a flipped pair
__device__ __forceinline__ void flip_link_one(const Pool& P, int k, int step) {
  const int f = P.fprop[k];
  if (f > -2) return;
  const int t = (-2 - f) >> 2;
  const int t2 = P.N[t].y >> 2;
  flip_fix(P, t, 0, step);
  flip_fix(P, t, 2, step);
  flip_fix(P, t2, 0, step);
  flip_fix(P, t2, 1, step);
}

__global__ void __launch_bounds__(BS) k_flip_propose(Pool P) {
  const int n = P.ctrl->n_fl;
  const int step = P.ctrl->step;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int k = gt; k < n; k += gs) flip_propose_one(P, P.fl_cur, k, step);
}

__global__ void __launch_bounds__(BS) k_flip_do(Pool P) {
  const int n = P.ctrl->n_fl;
  const int step = P.ctrl->step;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int k = gt; k < n; k += gs) flip_do_one(P, P.fl_nxt, k, step);
}

__global__ void __launch_bounds__(BS) k_flip_link(Pool P) {
  const int n = P.ctrl->n_fl;
  const int step = P.ctrl->step;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int k = gt; k < n; k += gs) flip_link_one(P, k, step);
}

// The last flip passes of a round in one block: while the list is short, a
// pass costs three block barriers instead of four kernel launches.  Passes
// go in pairs (P.fl_cur -> P.fl_nxt -> P.fl_cur), so the list ends where the
// launched passes expect it; a list that grows past FLIP_TAIL meanwhile is
// still finished here, and after FLIP_TAIL_PAIRS pairs the launched passes
// and the loop's condition (bounded) take over.  Same keys, marks and steps
// as the launched passes, so the same flips.
constexpr int FLIP_TAIL = 4096;
constexpr int FLIP_TAIL_THREADS = 512;
constexpr int FLIP_TAIL_PAIRS = 64;
__global__ void __launch_bounds__(FLIP_TAIL_THREADS) k_flip_tail(Pool P) {
  __shared__ int s_n, s_step;
  Ctrl* C = P.ctrl;
  if (threadIdx.x == 0) {
    s_n = C->n_fl;
    s_step = C->step;
  }
  __syncthreads();
  if (s_n == 0 || s_n > FLIP_TAIL) return;
  for (int pass = 0; pass < 2 * FLIP_TAIL_PAIRS; ++pass) {
    const int n = s_n, step = s_step;
    if (n == 0 && (pass & 1) == 0) break;
    const int* cur = (pass & 1) ? P.fl_nxt : P.fl_cur;
    int* nxt = (pass & 1) ? P.fl_cur : P.fl_nxt;
    for (int k = threadIdx.x; k < n; k += FLIP_TAIL_THREADS) flip_propose_one(P, cur, k, step);
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += FLIP_TAIL_THREADS) flip_do_one(P, nxt, k, step);
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += FLIP_TAIL_THREADS) flip_link_one(P, k, step);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int nn = atomicExch(&C->n_fl_next, 0);
      C->n_fl = nn;
      C->step = step + 1;
      s_n = nn;
      s_step = step + 1;
    }
    __syncthreads();
  }
}

// between passes (one thread): the list just built becomes the current one
__global__ void k_fl_next(Pool P) {
  P.ctrl->n_fl = P.ctrl->n_fl_next;
  P.ctrl->n_fl_next = 0;
  ++P.ctrl->step;
}

// start of a construction round (one thread): this round's counters
__global__ void k_round_begin(Pool P) {
  P.ctrl->n_ins = 0ull;
  P.ctrl->n_surv = 0ull;
}

// Conditions of the device-side loops of the construction graph (one
// thread).  Both loops are bounded: past the limit the kernel records an
// internal error and ends the loop.
constexpr int GUARD_ROUND_PAIRS = 1000;   // 2000 rounds (12-bit round keys)
constexpr int GUARD_FLIP = 1 << 17;

__global__ void k_flip_cond(Pool P, cudaGraphConditionalHandle h) {
  Ctrl* C = P.ctrl;
  bool go = C->n_fl > 0 && C->err == 0;
  if (go && ++C->guard_f > GUARD_FLIP) {
    set_err(C, S_INTERNAL);
    go = false;
  }
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_round_cond(Pool P, cudaGraphConditionalHandle h) {
  Ctrl* C = P.ctrl;
  bool go = C->n_pts > 0 && C->n_cand > 0 && C->err == 0;
  if (go && ++C->guard_r > GUARD_ROUND_PAIRS) {
    set_err(C, S_INTERNAL);
    go = false;
  }
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

// a triangle at every vertex (the segment walks start there)
__global__ void __launch_bounds__(BS) k_vtri(Pool P) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int t = gt; t < P.n_slots; t += gs) {
    const int4 T4 = P.T[t];
    if (T4.w < 0 || (T4.w & INFO_DEAD) || T4.x < 0) continue;
    P.vtri[T4.x] = t;
    P.vtri[T4.y] = t;
    P.vtri[T4.z] = t;
  }
}

// ---------------------------------------------------------------- segment recovery
// A missing segment ab is recovered by deleting the triangles it crosses and
// re-triangulating the two pseudo-polygons on its sides (upper chain left of
// a->b, lower chain right of it): for a base edge the chain vertex whose
// circle with the base holds no other chain vertex (exact incircle) forms a
// triangle, and both sides recurse.  The result is the constrained Delaunay
// triangulation of the region, so no flips are needed afterwards.  The region
// and its one-ring are claimed with 64-bit atomicMax marks so that segments
// whose regions touch are recovered in different rounds.
//
// Per-segment work space (capacity K crossed edges): crossed triangles
// R[K+1]; upper and lower chains U[K+2], L[K+2] (vertex ids, a first, b
// last); the outside neighbour and subsegment bit of each chain edge UR[K+2],
// LR[K+2] (as int2); an explicit recursion stack ST[K+2] (int4); NR[2(K+2)].
//
// A chain can run out and back along one edge: a vertex v between the
// segment and a chain vertex x makes the boundary ..., x, v, x, ...  Such
// twin edges (the same edge seen from both sides, possibly nested like
// parentheses) are interior to the new triangulation: their two new
// triangles are linked to each other, not to the old crossed triangles.
struct SegWork {
  int kcap;             // crossed edges that fit
  int* R;
  int* U;
  int* L;
  int2* UR;
  int2* LR;
  int4* ST;
  int* NR;              // 2 (K+2): new triangle refs of twin chain edges (upper, lower)
  int* list;            // segment ids to process
  int n_list;           // entries in list (host-set)
  int* state;           // per list entry: >= 0 crossings, -1 done, -2 error, -3 too long
};

__device__ __forceinline__ int idx_of(const int4& T4, int v) {
  return T4.x == v ? 0 : (T4.y == v ? 1 : (T4.z == v ? 2 : -1));
}

__device__ __forceinline__ void set_nb(const Pool& P, int ref, int val) {
  if (ref >= 0) *comp_ptr(&P.N[ref >> 2], ref & 3) = val;
}

// s is the segment's id within its mesh, so that a mesh's segments compete
// the same way alone and in a batch
__device__ __forceinline__ unsigned long long seg_key(int round, int s, int k) {
  return ((unsigned long long)(round + 1) << 48) |
         ((unsigned long long)(hash32((uint32_t)s) & 0xffffu) << 32) | (unsigned)k;
}

// walk a -> b, collecting the crossed triangles and both chains; claim the
// region and its one-ring
__global__ void __launch_bounds__(BS) k_seg_find(Pool P, SegWork W, int round) {
  const int n = W.n_list;
  const int K = W.kcap;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int k = gt; k < n; k += gs) {
    const int s = W.list[k];
    const int a = P.seg[s].x, b = P.seg[s].y;
    if (a == b) {   // rejected at input (its mesh carries the status)
      W.state[k] = -1;
      continue;
    }
    int t = P.vtri[a];
    const int m = P.T[t].w >> 4;
    int start = -1, ia = -1, status = 0;
    const P2 A = pt(P, a), B = pt(P, b);
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
      const int o1 = orient(A, pt(P, u), B), o2 = orient(A, pt(P, w), B);
      if (o1 == 0 && dot_sign(A, B, pt(P, u)) < 0) { status = S_INPUT; break; }
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
        W.state[k] = -2;
      } else {
        W.state[k] = -1;
      }
      continue;
    }
    int* R = W.R + (size_t)k * (K + 1);
    int* U = W.U + (size_t)k * (K + 2);
    int* L = W.L + (size_t)k * (K + 2);
    int2* UR = W.UR + (size_t)k * (K + 2);
    int2* LR = W.LR + (size_t)k * (K + 2);
    const int4 S4 = P.T[start];
    const int4 SN = P.N[start];
    // start = (a, r, l): lower boundary a->r (opposite l), upper boundary l->a (opposite r)
    int r = comp(S4, mod3(ia + 1)), l = comp(S4, mod3(ia + 2));
    int cnt = 0, nu = 0, nl = 0;
    R[cnt++] = start;
    U[nu++] = a; L[nl++] = a;
    UR[0] = make_int2(comp(SN, mod3(ia + 1)), (S4.w >> mod3(ia + 1)) & 1);
    LR[0] = make_int2(comp(SN, mod3(ia + 2)), (S4.w >> mod3(ia + 2)) & 1);
    U[nu++] = l; L[nl++] = r;
    int ref = comp(SN, ia);
    if ((S4.w >> ia) & 1) status = S_INPUT;   // crosses a recovered segment
    while (status == 0) {
      if (ref < 0) { status = S_INTERNAL; break; }
      if (cnt == K + 1) { status = 1000; break; }   // too long for this tier
      const int tn = ref >> 2, ee = ref & 3;
      const int4 T4 = P.T[tn];
      const int4 N4 = P.N[tn];
      if ((T4.w >> ee) & 1) { status = S_INPUT; break; }
      R[cnt++] = tn;
      // tn = (z, l, r) with entry edge l->r opposite z
      const int z = comp(T4, ee);
      if (z == b) {
        UR[nu - 1] = make_int2(comp(N4, mod3(ee + 2)), (T4.w >> mod3(ee + 2)) & 1);   // b->l
        LR[nl - 1] = make_int2(comp(N4, mod3(ee + 1)), (T4.w >> mod3(ee + 1)) & 1);   // r->b
        U[nu++] = b;
        L[nl++] = b;
        break;
      }
      const int o = orient(A, B, pt(P, z));
      if (o == 0) { status = S_INPUT; break; }
      if (o > 0) {   // z upper: boundary z->l (opposite r), exit r->z (opposite l)
        UR[nu - 1] = make_int2(comp(N4, mod3(ee + 2)), (T4.w >> mod3(ee + 2)) & 1);
        U[nu++] = z;
        ref = comp(N4, mod3(ee + 1));
        l = z;
      } else {       // z lower: boundary r->z (opposite l), exit z->l (opposite r)
        LR[nl - 1] = make_int2(comp(N4, mod3(ee + 1)), (T4.w >> mod3(ee + 1)) & 1);
        L[nl++] = z;
        ref = comp(N4, mod3(ee + 2));
        r = z;
      }
    }
#ifdef GDP_DIAG
    for (int i = 0; i < cnt && status == 0; ++i)
      for (int j = i + 1; j < cnt; ++j)
        if (R[i] == R[j]) printf("seg %d: walk revisits slot %d (cnt %d)\n", s, R[i], cnt);
#endif
    if (status == 1000) {
      W.state[k] = -3;
      continue;
    }
    if (status != 0) {
      P.mi[m].status = status;
      set_err(P.ctrl, status);
      W.state[k] = -2;
      continue;
    }
    W.state[k] = cnt;
    const unsigned long long key = seg_key(round, s - P.mi[m].seg_base, k);
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

// subsegment bit of a chain edge: read from the outside triangle now, since a
// segment found to be an edge already may have flagged it during the walk
__device__ __forceinline__ int out_cons(const Pool& P, int2 e) {
  return e.x >= 0 ? ((P.T[e.x >> 2].w >> (e.x & 3)) & 1) : e.y;
}

// chain accessors: the upper polygon uses U in order (base a->b); the lower
// one uses L reversed (base b->a).  Boundary edge j joins chain vertices j, j+1.
struct Chain {
  const int* v;
  int2* r;
  int* nr;        // new refs of twin edges, indexed like r
  int n;          // vertices
  bool rev;
  __device__ __forceinline__ int vert(int j) const { return rev ? v[n - 1 - j] : v[j]; }
  __device__ __forceinline__ int idx(int j) const { return rev ? n - 2 - j : j; }
  __device__ __forceinline__ int2 edge(int j) const { return r[idx(j)]; }
};

// mark twin edges: r[idx].x = -2 - (twin's chain index), r[idx].y = the
// subsegment bit, read from the old triangles before anything is rewritten
__device__ void mark_twins(const Pool& P, Chain& C) {
  int* stk = C.nr;   // nr is free until the re-triangulation
  int sp = 0;
  for (int j = 0; j + 1 < C.n; ++j) {
    const int u = C.vert(j), v = C.vert(j + 1);
    if (sp > 0) {
      const int t = stk[sp - 1];
      if (C.vert(t) == v && C.vert(t + 1) == u) {
        --sp;
        int2& ej = C.r[C.idx(j)];
        int2& et = C.r[C.idx(t)];
        const int cb = out_cons(P, ej) | out_cons(P, et) | ej.y | et.y;
        ej = make_int2(-2 - t, cb);
        et = make_int2(-2 - j, cb);
        continue;
      }
    }
    stk[sp++] = j;
  }
}

// link the new triangles on both sides of every twin edge
__device__ void link_twins(const Pool& P, const Chain& C) {
  for (int j = 0; j + 1 < C.n; ++j) {
    const int2 e = C.edge(j);
    if (e.x > -2) continue;
    const int t = -2 - e.x;
    if (t < j) continue;
    const int a = C.nr[C.idx(j)], b = C.nr[C.idx(t)];
    set_nb(P, a, b);
    set_nb(P, b, a);
  }
}

// re-triangulate one pseudo-polygon; returns the root triangle's slot or -1
__device__ int tri_pseudo(const Pool& P, Chain& C, int m, const int* R, int& next, int4* ST) {
  int sp = 0, root = -1;
  ST[sp++] = make_int4(0, C.n - 1, -1, 0);
  while (sp > 0) {
    const int4 tk = ST[--sp];
    const int lo = tk.x, hi = tk.y;
    const int u = C.vert(lo), w = C.vert(hi);
    const P2 pu = pt(P, u), pw = pt(P, w);
    int best = lo + 1;
    P2 pb = pt(P, C.vert(best));
    for (int j = lo + 2; j < hi; ++j) {
      const P2 pj = pt(P, C.vert(j));
      if (incircle(pu, pw, pb, pj) > 0) { best = j; pb = pj; }
    }
    const int c = C.vert(best);
    const int sl = R[next++];
    // (u, w, c): edge 0 = (w -> c), edge 1 = (c -> u), edge 2 = (u -> w) = base
    int cons = 0, n0 = -1, n1 = -1;
    if (hi == best + 1) {
      const int2 e = C.edge(best);
      if (e.x <= -2) {          // twin edge: linked after the re-triangulation
        cons |= e.y;
        C.nr[C.idx(best)] = (sl << 2) | 0;
      } else {
        n0 = e.x;
        cons |= out_cons(P, e);
        set_nb(P, e.x, (sl << 2) | 0);
      }
    } else {
      ST[sp++] = make_int4(best, hi, (sl << 2) | 0, 0);
    }
    if (best == lo + 1) {
      const int2 e = C.edge(lo);
      if (e.x <= -2) {
        cons |= e.y << 1;
        C.nr[C.idx(lo)] = (sl << 2) | 1;
      } else {
        n1 = e.x;
        cons |= out_cons(P, e) << 1;
        set_nb(P, e.x, (sl << 2) | 1);
      }
    } else {
      ST[sp++] = make_int4(lo, best, (sl << 2) | 1, 0);
    }
    const int n2 = tk.z;
    P.T[sl] = make_int4(u, w, c, (m << 4) | cons);
    P.N[sl] = make_int4(n0, n1, n2, 0);
    if (n2 >= 0) set_nb(P, n2, (sl << 2) | 2);
    else root = sl;
  }
  return root;
}

__global__ void __launch_bounds__(BS) k_seg_apply(Pool P, SegWork W, int round) {
  const int n = W.n_list;
  const int K = W.kcap;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int k = gt; k < n; k += gs) {
    const int cnt = W.state[k];
    if (cnt <= 0) continue;
    const int s = W.list[k];
    const int* R = W.R + (size_t)k * (K + 1);
    const unsigned long long key = seg_key(round, s - P.mi[P.T[R[0]].w >> 4].seg_base, k);
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
    const int m = P.T[R[0]].w >> 4;
    const int* U = W.U + (size_t)k * (K + 2);
    const int* L = W.L + (size_t)k * (K + 2);
    int nu = 0, nl = 0;
    const int b = P.seg[s].y;
    while (U[nu] != b) ++nu;
    while (L[nl] != b) ++nl;
    ++nu;
    ++nl;
    int* NR = W.NR + (size_t)k * 2 * (K + 2);
    Chain CU{U, W.UR + (size_t)k * (K + 2), NR, nu, false};
    Chain CL{L, W.LR + (size_t)k * (K + 2), NR + (K + 2), nl, true};
    mark_twins(P, CU);
    mark_twins(P, CL);
    int4* ST = W.ST + (size_t)k * (K + 2);
    int next = 0;
#ifdef GDP_DIAG
    if (nu + nl - 4 != cnt) printf("seg %d: nu %d nl %d cnt %d\n", s, nu, nl, cnt);
#endif
    const int ru = tri_pseudo(P, CU, m, R, next, ST);
    const int rl = tri_pseudo(P, CL, m, R, next, ST);
#ifdef GDP_DIAG
    if (next != cnt) printf("seg %d: created %d triangles for %d slots\n", s, next, cnt);
    if (cnt > 60) printf("seg %d: long region cnt %d nu %d nl %d\n", s, cnt, nu, nl);
#endif
    link_twins(P, CU);
    link_twins(P, CL);
    // the two roots share the segment (edge 2 of both), now a subsegment
    P.N[ru].z = (rl << 2) | 2;
    P.N[rl].z = (ru << 2) | 2;
    P.T[ru].w |= 4;
    P.T[rl].w |= 4;
    for (int j = 0; j < cnt; ++j) {
      const int4 T4 = P.T[R[j]];
      P.vtri[T4.x] = R[j];
      P.vtri[T4.y] = R[j];
      P.vtri[T4.z] = R[j];
    }
    W.state[k] = -1;
  }
}

// Keep the list entries that still need work (stable): not yet recovered
// (state >= 0), too long for the tier (state -3), or beyond the processed
// prefix.  ctrl->n_segs receives the kept count and ctrl->changed the number
// of kept entries that the current tier can still handle.
__global__ void __launch_bounds__(BS) k_seg_keep_count(Pool P, SegWork W, int n_total) {
  __shared__ int sm[33];
  const Chunk ch = chunk_of(n_total);
  int cnt = 0, shortc = 0;
  for (int k = ch.b0 + threadIdx.x; k < ch.b1; k += BS) {
    const int st = k < W.n_list ? W.state[k] : 0;
    cnt += (st >= 0 || st == -3) ? 1 : 0;
    shortc += st >= 0 ? 1 : 0;
  }
  cnt = block_sum(cnt, sm);
  shortc = block_sum(shortc, sm);
  if (threadIdx.x == 0) {
    P.blk[blockIdx.x] = cnt;
    P.blk[gridDim.x + blockIdx.x] = shortc;
  }
}

__global__ void __launch_bounds__(BS) k_seg_keep_write(Pool P, SegWork W, int n_total, int* out) {
  __shared__ int sm[33];
  const Chunk ch = chunk_of(n_total);
  int off = block_prefix(P.blk, blockIdx.x, sm);
  for (int base = ch.b0; base < ch.b1; base += BS) {
    const int k = base + threadIdx.x;
    int keep = 0;
    if (k < ch.b1) {
      const int st = k < W.n_list ? W.state[k] : 0;
      keep = (st >= 0 || st == -3) ? 1 : 0;
    }
    int tot;
    const int r = block_excl_scan(keep, sm, tot);
    if (keep) out[off + r] = W.list[k];
    off += tot;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    int sh = 0;
    for (int k = 0; k < (int)gridDim.x; ++k) sh += P.blk[gridDim.x + k];
    P.ctrl->n_segs = off;
    P.ctrl->changed = sh;
  }
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
    P.flag[t] = 0;
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
