// Kernels of the parallel refinement loop (Algorithm 1) and of the GPU CDT.
//
// One refinement iteration of Algorithm 1 is a fixed sequence of launches,
// all over the whole pool (every mesh of a batch at once, Rule 4):
//   k_scan_eval / _count / _write the scan: changed triangles are checked for
//                                 encroached subsegments and bad quality and the
//                                 hits are compacted, in slot order, into the
//                                 candidate list (block counts + block scans;
//                                 the compaction is stable so the run is
//                                 deterministic)
//   k_grow                        splitting point and priority,
//                                 point location by walking, cavity growth by
//                                 incircle blocked at subsegments, then one
//                                 64-bit atomicMax mark per cavity triangle
//   k_survive                     a point survives iff it owns every mark
//   k_depend                      Delaunay-dependence check on shared cavity
//                                 boundary edges (Sec. 5.2): the lower priority
//                                 point of a dependent pair is dropped
//   k_offsets                     stable prefix sums for new slots / vertex ids
//   k_insert / k_link             insertion: cavity re-triangulation as a fan,
//                                 neighbour fix-up, then links between adjacent
//                                 cavities
// The same cavity kernels insert the input points of the initial CDT; the
// CDT is finished by segment recovery (flips) and removal of the exterior.
#pragma once
#include <cstdint>

#include "gdp_core.cuh"
#include "gdp_pred.cuh"

namespace gdp {

// ---------------------------------------------------------------- small helpers
__device__ __forceinline__ int comp(const int4& a, int i) {
  return i == 0 ? a.x : (i == 1 ? a.y : a.z);
}
__device__ __forceinline__ int* comp_ptr(int4* p, int i) { return reinterpret_cast<int*>(p) + i; }
__device__ __forceinline__ int mod3(int i) { return i >= 3 ? i - 3 : i; }

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

__device__ __forceinline__ void set_err(Ctrl* C, int code) { atomicCAS(&C->err, 0, code); }

// Index checks of a checking build (-DGDP_CHECKS) on the growth and insertion
// paths: an index outside its array is recorded (the first failing site's
// code in ctrl->dbg, GDP_ERR_INTERNAL) and replaced by 0, so that the access
// stays in bounds.  A plain build compiles them away.
#ifdef GDP_CHECKS
__device__ __forceinline__ long long cidx_(Ctrl* C, long long x, long long lim, int site) {
  if (x >= 0 && x < lim) return x;
  atomicCAS(&C->dbg, 0, site);
  set_err(C, S_INTERNAL);
  return 0;
}
#define CI(x, lim, site) cidx_(P.ctrl, (long long)(x), (long long)(lim), (site))
#else
#define CI(x, lim, site) (x)
#endif

__device__ __forceinline__ int block_sum(int v, int* sm) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sm[w] = v;
  __syncthreads();
  if (w == 0) {
    int r = l < nw ? sm[l] : 0;
    for (int o = 16; o; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (l == 0) sm[32] = r;
  }
  __syncthreads();
  int r = sm[32];
  __syncthreads();
  return r;
}

// exclusive scan over the block; total receives the block sum
__device__ __forceinline__ int block_excl_scan(int v, int* sm, int& total) {
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (l >= o) x += y;
  }
  __syncthreads();
  if (l == 31) sm[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = l < nw ? sm[l] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (l >= o) s += y;
    }
    if (l < nw) sm[l] = s;
  }
  __syncthreads();
  int base = w ? sm[w - 1] : 0;
  total = sm[nw - 1];
  __syncthreads();
  return base + x - v;
}

// sum of blk[0..b), computed by the whole block
__device__ __forceinline__ int block_prefix(const int* blk, int b, int* sm) {
  int s = 0;
  for (int k = threadIdx.x; k < b; k += blockDim.x) s += blk[k];
  return block_sum(s, sm);
}

struct Chunk {
  int b0, b1;
};
// contiguous index range of this block (stable compactions use fixed chunks)
__device__ __forceinline__ Chunk chunk_of(int n) {
  int c = (n + gridDim.x - 1) / gridDim.x;
  int b0 = min(n, (int)blockIdx.x * c);
  return {b0, min(n, b0 + c)};
}

__device__ __forceinline__ P2 pt(const Pool& P, int v) { return P2{P.V[v], P.Vf[v]}; }

// Predicates on mesh vertices given by id.  The FP32 two-float filter reads
// only Vf; when it cannot decide, the FP64 coordinates are read and the FP64
// and exact stages run in separate, non-inlined functions, so that the common
// path neither loads nor holds FP64 coordinates.
static __device__ __noinline__ int orient_v64(const double2* V, int a, int b, double cx, double cy) {
  return orient(V[a], V[b], make_double2(cx, cy));
}
static __device__ __noinline__ int incircle_v64(const double2* V, int a, int b, int c, double dx, double dy) {
  return incircle(V[a], V[b], V[c], make_double2(dx, dy));
}
// circle (p, u, v) against the point of candidate j (Delaunay dependence)
static __device__ __noinline__ int incircle_dep64(const double2* V, const double2* cpt, double px, double py,
                                                  int u, int v, int j) {
  return incircle(make_double2(px, py), V[u], V[v], cpt[j]);
}
__device__ __forceinline__ int orient_ids(const Pool& P, int a, int b, const P2& c) {
  a = CI(a, P.n_verts, 127);
  b = CI(b, P.n_verts, 127);
  const int s = orient_f32(P.Vf[a], P.Vf[b], c.f);
  GDP_DIAG_ADD(9);
  if (!s) GDP_DIAG_ADD(12);
  return s ? s : orient_v64(P.V, a, b, c.d.x, c.d.y);
}
__device__ __forceinline__ int incircle_ids(const Pool& P, int a, int b, int c, const P2& d) {
  a = CI(a, P.n_verts, 105);
  b = CI(b, P.n_verts, 105);
  c = CI(c, P.n_verts, 105);
  const int s = incircle_f32(P.Vf[a], P.Vf[b], P.Vf[c], d.f);
  GDP_DIAG_ADD(10);
  if (!s) GDP_DIAG_ADD(13);
  return s ? s : incircle_v64(P.V, a, b, c, d.d.x, d.d.y);
}
__device__ __forceinline__ int incircle_dep(const Pool& P, const P2& p, int u, int v, int j) {
  const int s = incircle_f32(p.f, P.Vf[u], P.Vf[v], P.c_ptf[j]);
  GDP_DIAG_ADD(10);
  if (!s) GDP_DIAG_ADD(13);
  return s ? s : incircle_dep64(P.V, P.c_pt, p.d.x, p.d.y, u, v, j);
}
// the two-float copy of p - org (see the FP32 filter stage of the predicates)
__device__ __forceinline__ float4 to_f(double2 p, double2 org) {
  const double tx = __dsub_rn(p.x, org.x), ty = __dsub_rn(p.y, org.y);
  const float hx = __double2float_rn(tx), hy = __double2float_rn(ty);
  return make_float4(hx, hy, __double2float_rn(__dsub_rn(tx, (double)hx)),
                     __double2float_rn(__dsub_rn(ty, (double)hy)));
}

// ---------------------------------------------------------------- mesh queries
// Auxiliary vertices of every mesh, right after its input points: three
// enclosing vertices, then four frame vertices around the bounding box (16
// times its size out).  The
// frame is inserted first, so every input point lies inside the triangulated
// region from then on and points never queue up outside a growing hull.  All
// seven lie outside the segment-bounded domain and are removed with the
// exterior, so they do not change the CDT.
constexpr int N_AUX = 7;
__device__ __forceinline__ bool is_aux(const MeshInfo& M, int v) {
  const int s = M.vert_base + M.n_in;
  return v >= s && v < s + N_AUX;
}

// insertion priority of a construction point: frame vertices first, then a hash
__device__ __forceinline__ uint32_t insert_prio(const MeshInfo& M, int v) {
  if (is_aux(M, v)) return 0xffffffffu;
  return hash32((uint32_t)(v - M.vert_base)) | 1u;
}

__device__ __forceinline__ bool is_input(const MeshInfo& M, int v) {
  return v >= M.vert_base && v < M.vert_base + M.n_in;
}

// the input segment a subsegment (u,v) belongs to
__device__ int seg_of_sub(const Pool& P, const MeshInfo& M, int u, int v) {
  int s = P.vseg[u];
  if (s >= 0) return s;
  s = P.vseg[v];
  if (s >= 0) return s;
  if (!is_input(M, u)) return -1;
  const int lu = u - M.vert_base;
  for (int k = P.adj_off[M.adj_base + lu]; k < P.adj_off[M.adj_base + lu + 1]; ++k) {
    const int g = P.adj[k];
    const int2 e = P.seg[g];
    if ((e.x == u && e.y == v) || (e.x == v && e.y == u)) return g;
  }
  return -1;
}

// two distinct input segments sharing an endpoint at less than 60 degrees:
// cos > 1/2, i.e. 2 (u.w) > |u| |w| for the two directions u, w from the
// shared vertex.  Every operation is rounded on its own (no contraction), so
// the decision is the same bit for bit wherever this formula is evaluated in
// this order; it is symmetric in the two segments.
__device__ bool small_pair(const Pool& P, int s1, int s2) {
  if (s1 == s2 || s1 < 0 || s2 < 0) return false;
  const int2 a = P.seg[s1], b = P.seg[s2];
  int o, p, q;
  if (a.x == b.x) { o = a.x; p = a.y; q = b.y; }
  else if (a.x == b.y) { o = a.x; p = a.y; q = b.x; }
  else if (a.y == b.x) { o = a.y; p = a.x; q = b.y; }
  else if (a.y == b.y) { o = a.y; p = a.x; q = b.x; }
  else return false;
  const double2 O = P.V[o], A = P.V[p], B = P.V[q];
  const double ux = __dsub_rn(A.x, O.x), uy = __dsub_rn(A.y, O.y);
  const double wx = __dsub_rn(B.x, O.x), wy = __dsub_rn(B.y, O.y);
  const double dot = __dadd_rn(__dmul_rn(ux, wx), __dmul_rn(uy, wy));
  const double nn = __dmul_rn(__dsqrt_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy))),
                              __dsqrt_rn(__dadd_rn(__dmul_rn(wx, wx), __dmul_rn(wy, wy))));
  return __dmul_rn(2.0, dot) > nn;
}

// the k-th input segment vertex v lies on (an input vertex: its incident
// segments; a Steiner vertex: the segment it was placed on), and how many
__device__ __forceinline__ int n_segs_of(const Pool& P, const MeshInfo& M, int v) {
  if (is_input(M, v)) {
    const int l = v - M.vert_base;
    return P.adj_off[M.adj_base + l + 1] - P.adj_off[M.adj_base + l];
  }
  return P.vseg[v] >= 0 ? 1 : 0;
}
__device__ __forceinline__ int seg_at(const Pool& P, const MeshInfo& M, int v, int k) {
  if (is_input(M, v)) return P.adj[P.adj_off[M.adj_base + (v - M.vert_base)] + k];
  return P.vseg[v];
}

// Bad triangles whose shortest edge joins two segments meeting at a small
// input angle are accepted in the output (Sec. 4.1).  When several edges
// are shortest, each is tried, so the decision does not depend on where the
// triangle's vertex list starts.
__device__ bool exempt(const Pool& P, const MeshInfo& M, const int4& T4) {
  if (!M.has_apex) return false;
  double l[3];
  for (int e = 0; e < 3; ++e) {
    const double2 a = P.V[comp(T4, mod3(e + 1))], b = P.V[comp(T4, mod3(e + 2))];
    const double dx = __dsub_rn(b.x, a.x), dy = __dsub_rn(b.y, a.y);
    l[e] = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  }
  const double best = fmin(l[0], fmin(l[1], l[2]));
  for (int e = 0; e < 3; ++e) {
    if (l[e] != best) continue;
    const int u = comp(T4, mod3(e + 1)), w = comp(T4, mod3(e + 2));
    const int nu = n_segs_of(P, M, u), nw = n_segs_of(P, M, w);
    for (int i = 0; i < nu; ++i) {
      const int su = seg_at(P, M, u, i);
      for (int j = 0; j < nw; ++j)
        if (small_pair(P, su, seg_at(P, M, w, j))) return true;
    }
  }
  return false;
}

// Splitting point of subsegment (u,v): the midpoint, or -- when exactly one
// endpoint is an input vertex with a small input angle -- the point at the
// power-of-two distance d from it nearest to half the length L in ratio
// (concentric shells): with L/2 = m 2^e, m in [1/2, 1), d = 2^(e-1) when
// m^2 < 1/2, else 2^e.  Each operation rounded on its own (no contraction).
__device__ double2 split_point(const Pool& P, const MeshInfo& M, int u, int v) {
  const bool au = is_input(M, u) && P.apex[u];
  const bool av = is_input(M, v) && P.apex[v];
  if (au == av) return midpoint(P.V[u], P.V[v]);
  const int o = au ? u : v, q = au ? v : u;
  const double2 O = P.V[o], Q = P.V[q];
  const double dx = __dsub_rn(Q.x, O.x), dy = __dsub_rn(Q.y, O.y);
  const double L = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
  int e;
  const double m = frexp(__dmul_rn(0.5, L), &e);
  const double d = (__dmul_rn(m, m) < 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
  const double r = __ddiv_rn(d, L);
  return make_double2(__dadd_rn(O.x, __dmul_rn(dx, r)), __dadd_rn(O.y, __dmul_rn(dy, r)));
}

// ---------------------------------------------------------------- scan
// 0: nothing; 1..3: encroached subsegment on edge 0..2 (longest); 4: bad triangle
__device__ int eval_tri(const Pool& P, int t) {
  const int4 T4 = P.T[t];
  if (T4.w < 0 || (T4.w & INFO_DEAD)) return 0;
  const MeshInfo& M = P.mi[T4.w >> 4];
  if (!M.active) return 0;
  const int cons = T4.w & 7;
  if (cons) {
    int best = -1;
    double bl = -1.0;
    for (int e = 0; e < 3; ++e) {
      if (!((cons >> e) & 1)) continue;
      const P2 u = pt(P, comp(T4, mod3(e + 1))), v = pt(P, comp(T4, mod3(e + 2)));
      if (encroaches(u, v, pt(P, comp(T4, e)), M.lens)) {
        const double l = seg_measure(u.d, v.d);
        if (l > bl) { bl = l; best = e; }
      }
    }
    if (best >= 0) return 1 + best;
  }
  if (M.L2 > 0) {   // edge-length bound: a longest edge above l is refined, exempt or not
    const TriTerms tt = tri_terms(P.V[T4.x], P.V[T4.y], P.V[T4.z]);
    if (fmax(tt.la, fmax(tt.lb, tt.lc)) > M.L2) return 4;
  }
  const int q = bad_f32(P.Vf[T4.x], P.Vf[T4.y], P.Vf[T4.z], M.B2f);
  const bool bad = q > 0 || (q == 0 && is_bad(tri_terms(P.V[T4.x], P.V[T4.y], P.V[T4.z]), M.B2));
  if (bad && !exempt(P, M, T4)) return 4;
  return 0;
}

// Priority bucket of a flagged element for the per-mesh cap: [class bit |
// the top 9 bits (exponent + 1 mantissa bit) of float32 length^2 (subsegment)
// or |2A| (triangle)], from the float copies -- a scheduling heuristic, so
// FP32 is enough; it only has to be deterministic.
__device__ __forceinline__ int cap_bucket(const Pool& P, const int4& T4, int code) {
  float v;
  if (code == 4) {
    const float4 a = P.Vf[T4.x], b = P.Vf[T4.y], c = P.Vf[T4.z];
    v = fabsf((b.x - a.x) * (c.y - a.y) - (b.y - a.y) * (c.x - a.x));
  } else {
    const float4 u = P.Vf[comp(T4, mod3(code))], w = P.Vf[comp(T4, mod3(code + 1))];
    v = (w.x - u.x) * (w.x - u.x) + (w.y - u.y) * (w.y - u.y);
  }
  const uint32_t b = (v >= 0.0f && v < INFINITY) ? (__float_as_uint(v) >> 22) : 0x1ffu;
  return (code == 4 ? 0 : 512) | (int)min(b, 0x1ffu);
}

// slots the refinement scan covers (a resident pool scans up to its highest
// occupied region only)
__device__ __forceinline__ int scan_slots(const Pool& P) {
  const int h = P.ctrl->scan_hi;
  return (h > 0 && h < P.n_slots) ? h : P.n_slots;
}

// cavity work space of candidate i: its own slot, or its spill arena region
__device__ __forceinline__ int* cav_of(const Pool& P, int i) {
  const int o = P.c_big[i];
  return o < 0 ? P.c_cav + (size_t)i * CMAX : P.big_cav + o;
}

__device__ __forceinline__ int4* bnd_of(const Pool& P, int i) {
  const int o = P.c_big[i];
  return o < 0 ? P.c_bnd + (size_t)i * BMAX : P.big_bnd + o;
}

// Clears the marks of the previous iteration's cavities: one thread per
// candidate, the whole warp for a spill-tier cavity.  Called by all threads.
__device__ __forceinline__ void clear_prev_marks(const Pool& P) {
  const unsigned FULL = 0xffffffffu;
  const int prev = P.ctrl->prev_cand;
  const int lane = threadIdx.x & 31;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int i0 = gt - lane; i0 < prev; i0 += gs) {
    const int i = i0 + lane;
    const int n = i < prev ? P.c_ncav[i] : 0;
    const bool big = n > CMAX;
    if (!big) {
      const int* cav = cav_of(P, i);
      for (int j = 0; j < n; ++j) P.mark[cav[j]] = 0ull;
    }
    // the refinement pre-pass's marks (entries 0 when the last iteration ran no pre-pass)
    const int np = i < prev ? P.c_npre[i] : 0;
    for (int j = 0; j < np; ++j) {
      const int t = P.c_pre[(size_t)i * PRE_MAX + j];
      if ((unsigned)t < (unsigned)P.n_slots) P.pmark[t] = 0ull;
    }
    unsigned bm = __ballot_sync(FULL, big);
    while (bm) {
      const int src = __ffs(bm) - 1;
      bm &= bm - 1;
      const int ib = __shfl_sync(FULL, i, src), nb = __shfl_sync(FULL, n, src);
      const int* cav = cav_of(P, ib);
      for (int j = lane; j < nb; j += 32) P.mark[cav[j]] = 0ull;
    }
  }
}

__global__ void __launch_bounds__(BS) k_clear_marks(Pool P) { clear_prev_marks(P); }

// Evaluation of the changed triangles, interleaved over the whole grid (new
// triangles sit together at the end of a mesh's slots, so contiguous chunks
// would leave their evaluation to a few blocks); every slot's flag is written.
// Flags persist from one iteration to the next: a triangle's code depends on
// its vertices and on fixed per-mesh data only, and the insertion kernels
// evaluate every triangle they create.  This pass evaluates the triangles
// marked dirty by the construction or a relocation (Ctrl::need_eval, cleared
// by k_scan_count) and otherwise only clears the last iteration's marks.
__global__ void __launch_bounds__(BS) k_scan_eval(Pool P) {
  clear_prev_marks(P);
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int m = gt; m < P.n_mesh; m += gs) {
    P.mi[m].first_cand = -1;
    P.mi[m].last_cand = -1;
    P.mi[m].pending = 0;
  }
  if (!P.ctrl->need_eval) return;
  const int ns = scan_slots(P);
  for (int t = gt; t < ns; t += gs) {
    if (!P.dirty[t]) continue;
    P.dirty[t] = 0;
    P.flag[t] = (uint8_t)eval_tri(P, t);
  }
}

// start of a refinement: every slot is evaluated with this call's bounds
__global__ void __launch_bounds__(BS) k_mark_all(Pool P) {
  const int ns = scan_slots(P);
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int t = gt; t < ns; t += gs) P.dirty[t] = 1;
}

// The compaction's chunk of this block: whole groups of eight slots (flags
// are read eight at a time), the last chunk ending at ns.
__device__ __forceinline__ Chunk scan_chunk(int ns) {
  const int ngr = (ns + 7) >> 3;
  const int c = (ngr + gridDim.x - 1) / gridDim.x;
  const int g0 = min(ngr, (int)blockIdx.x * c);
  return {min(ns, 8 * g0), min(ns, 8 * (g0 + c))};
}

// flags of the eight slots from t0 (a multiple of 8), zero from ns on
__device__ __forceinline__ uint2 flags8(const Pool& P, int t0, int ns) {
  if (t0 + 8 <= ns) return reinterpret_cast<const uint2*>(P.flag)[t0 >> 3];
  unsigned lo = 0u, hi = 0u;
  for (int k = 0; t0 + k < ns; ++k) {
    const unsigned f = P.flag[t0 + k];
    if (k < 4) lo |= f << (8 * k);
    else hi |= f << (8 * (k - 4));
  }
  return make_uint2(lo, hi);
}

__device__ __forceinline__ int nz_bytes(unsigned w) { return __popc(__vcmpne4(w, 0u)) >> 3; }

// flagged slots per block chunk (the stable compaction's block counts)
// (capped: also the priority buckets and per-mesh histograms of the flagged
// slots of meshes with a cap)
__global__ void __launch_bounds__(BS) k_scan_count(Pool P, int capped) {
  __shared__ int sm[33];
  if (blockIdx.x == 0 && threadIdx.x == 0) P.ctrl->need_eval = 0;   // k_scan_eval has run
  const int ns = scan_slots(P);
  const Chunk ch = scan_chunk(ns);
  int cnt = 0;
  for (int t0 = ch.b0 + 8 * threadIdx.x; t0 < ch.b1; t0 += 8 * BS) {
    const uint2 f = flags8(P, t0, ns);
    cnt += nz_bytes(f.x) + nz_bytes(f.y);
    if (!capped || (f.x | f.y) == 0u) continue;
    for (int k = 0; k < 8; ++k) {
      const int code = (int)(((k < 4 ? f.x : f.y) >> (8 * (k & 3))) & 0xffu);
      if (!code) continue;
      const int t = t0 + k;
      const int4 T4 = P.T[t];
      const int m = T4.w >> 4;
      if (P.mi[m].cand_cap <= 0) continue;
      const int b = cap_bucket(P, T4, code);
      P.cbucket[t] = (uint16_t)b;
      atomicAdd(&P.cap_hist[(size_t)m * CAP_BUCKETS + b], 1);
    }
  }
  cnt = block_sum(cnt, sm);
  if (threadIdx.x == 0) P.blk[blockIdx.x] = cnt;
}

// per mesh with a cap: the lowest bucket such that all flagged elements at or
// above it fit in the cap (the top non-empty bucket is always taken); the
// histogram is cleared for the next iteration
__global__ void __launch_bounds__(BS) k_cap_select(Pool P) {
  for (int m = blockIdx.x; m < P.n_mesh; m += gridDim.x) {
    const int K = P.mi[m].cand_cap;
    if (K <= 0) continue;
    int* h = P.cap_hist + (size_t)m * CAP_BUCKETS;
    if (threadIdx.x == 0) {
      int acc = 0, thr = CAP_BUCKETS;
      for (int b = CAP_BUCKETS - 1; b >= 0; --b) {
        if (!h[b]) continue;
        if (thr < CAP_BUCKETS && acc + h[b] > K) break;
        acc += h[b];
        thr = b;
      }
      P.cap_thr[m] = thr;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < CAP_BUCKETS; b += blockDim.x) h[b] = 0;
    __syncthreads();
  }
}

// capped meshes: flagged elements below the threshold wait for a later
// iteration (k_scan_write skips them too); block counts for k_scan_write
__global__ void __launch_bounds__(BS) k_cap_count(Pool P) {
  __shared__ int sm[33];
  const Chunk ch = scan_chunk(scan_slots(P));
  int cnt = 0;
  for (int t = ch.b0 + threadIdx.x; t < ch.b1; t += BS) {
    if (!P.flag[t]) continue;
    const int m = P.T[t].w >> 4;
    if (P.mi[m].cand_cap > 0 && P.cbucket[t] < P.cap_thr[m]) {
      P.mi[m].pending = 1;   // stays flagged for a later iteration
      continue;
    }
    ++cnt;
  }
  cnt = block_sum(cnt, sm);
  if (threadIdx.x == 0) P.blk[blockIdx.x] = cnt;
}

__device__ __forceinline__ bool cap_skipped(const Pool& P, int t) {
  const int m = P.T[t].w >> 4;
  return P.mi[m].cand_cap > 0 && P.cbucket[t] < P.cap_thr[m];
}

__global__ void __launch_bounds__(BS) k_scan_write(Pool P, int capped) {
  __shared__ int sm[33];
  const int ns = scan_slots(P);
  const Chunk ch = scan_chunk(ns);
  int off = block_prefix(P.blk, blockIdx.x, sm);
  const int cap = P.cap_cand;
  for (int base = ch.b0; base < ch.b1; base += 8 * BS) {
    const int t0 = base + 8 * threadIdx.x;
    uint2 f = t0 < ch.b1 ? flags8(P, t0, ns) : make_uint2(0u, 0u);
    if (capped && (f.x | f.y) != 0u) {   // drop the slots the cap defers
      for (int k = 0; k < 8; ++k) {
        const int sh = 8 * (k & 3);
        if (((k < 4 ? f.x : f.y) >> sh) & 0xffu && cap_skipped(P, t0 + k)) {
          if (k < 4) f.x &= ~(0xffu << sh);
          else f.y &= ~(0xffu << sh);
        }
      }
    }
    const int c = nz_bytes(f.x) + nz_bytes(f.y);
    int tot;
    const int r = block_excl_scan(c, sm, tot);
    if (c) {
      int rank = off + r;
      for (int k = 0; k < 8; ++k) {
        const int code = (int)(((k < 4 ? f.x : f.y) >> (8 * (k & 3))) & 0xffu);
        if (!code) continue;
        const int t = t0 + k;
        if (rank < cap) {
          P.c_elem[rank] = (t << 2) | (code == 4 ? 3 : code - 1);
        } else {
          P.mi[P.T[t].w >> 4].pending = 1;   // over the per-iteration capacity: stays flagged
        }
        ++rank;
      }
    }
    off += tot;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    const int n = min(off, cap);
    Ctrl* C = P.ctrl;
    C->n_raw = off;
    C->n_cand = n;
    C->prev_cand = n;
    C->n_ins = 0;
    if (n > 0) {
      C->tot_cand += n;
      C->iters += 1;
    }
  }
}

// ---------------------------------------------------------------- locate + grow
// Visibility walk from t towards p.  Returns the triangle containing p
// (closed), -1 when the next step would cross a subsegment (stop_cons) or the
// hull -- (bt, be) is that edge -- or -2 at the step limit.  In a CDT every
// step across a locally Delaunay edge lowers the power of p with respect to
// the current circumcircle, so the walk cannot cycle.
__device__ int walk(const Pool& P, int t, const P2& p, bool stop_cons, int& bt, int& be, int& steps) {
  int from = -1;
#ifdef GDP_DIAG
  const long long c0 = clock64();
#endif
  for (int s = 0; s < WALK_MAX; ++s) {
#ifdef GDP_DIAG
    if (s > 0 && (s & 7) == 0) atomicMax(&g_diag[5], (unsigned long long)s);
#endif
    const int4 T4 = P.T[CI(t, P.n_slots, 122)];
    const int4 N4 = P.N[CI(t, P.n_slots, 122)];
    int next = -1, nfrom = -1, blk = -1;
    for (int e = 0; e < 3 && next < 0; ++e) {
      const int nb = comp(N4, e);
      if (nb >= 0 && (nb >> 2) == from) continue;   // p is on this side of the entry edge
      if (orient_ids(P, comp(T4, mod3(e + 1)), comp(T4, mod3(e + 2)), p) < 0) {
        if ((stop_cons && ((T4.w >> e) & 1)) || nb < 0) {
          if (blk < 0) blk = e;
        } else {
          next = nb >> 2;
          nfrom = t;
        }
      }
    }
    if (next >= 0) {
      from = nfrom;
      t = next;
      ++steps;
      continue;
    }
#ifdef GDP_DIAG
    atomicMax(&g_diag[7], (unsigned long long)(clock64() - c0));
#endif
    if (blk >= 0) {
      bt = t;
      be = blk;
      return -1;
    }
    return t;
  }
  return -2;
}

enum { G_OK = 0, G_OVF = 1, G_CONV = 2, G_LOSE = 3 };

// Bowyer-Watson cavity of p from t0 (and t1): breadth-first over triangles
// whose circumcircle holds p (exact incircle with simulation of simplicity),
// never across a subsegment (visibility).  Boundary edges are recorded as
// (u, v, outside ref, inside ref | subsegment bit).  With conv, meeting a
// subsegment that p encroaches stops the growth (G_CONV) so that the
// subsegment is split instead (Sec. 4.2: such a circumcentre is redundant).
// Cavity work space.  Every candidate first grows in its own slot (CMAX
// triangles, linear membership test).  One that outgrows it asks for a lane
// of spill tier A (CAP_A triangles), and from there for a lane of tier B
// (CMAX_BIG); a lane carries an open-addressing hash set for the membership
// test.  A lane goes, for one round, to the smallest candidate index mapped
// to it, so which candidates get one never depends on timing; the others
// fail this round and are retried in a later one.
struct CavBuf {
  int* cav;
  int4* bnd;     // capacity cap + 2
  int* hash;     // nullptr: linear membership test
  int cap;
  int hmask;     // hash set size - 1 (at least 2 cap - 1)
};

// is t in the cavity?  With a hash set a miss leaves in h the empty entry
// where t goes.  The set is never more than half full, so the probe always
// meets an empty entry; the loop is bounded all the same.
__device__ __forceinline__ bool cav_has(const CavBuf& B, int k, int t, int& h) {
  if (!B.hash) {
    for (int r = 0; r < k; ++r)
      if (B.cav[r] == t) return true;
    return false;
  }
  h = (int)(hash32((uint32_t)t) & (uint32_t)B.hmask);
  for (int s = 0; s <= B.hmask; ++s) {
    const int x = B.hash[h];
    if (x == t) return true;
    if (x < 0) return false;
    h = (h + 1) & B.hmask;
  }
  return true;   // unreachable: treat as present so nothing is overwritten
}

__device__ __forceinline__ bool cav_add(const CavBuf& B, int& k, int t) {
  int h = 0;
  if (cav_has(B, k, t, h)) return true;
  if (k == B.cap) return false;
  B.cav[k++] = t;
  if (B.hash) B.hash[h] = t;
  return true;
}

__device__ int grow(const Pool& P, const CavBuf& B, const P2& p, int t0, int t1, bool conv, bool lens,
                    int& nc, int& nb, int& ct, int& ce) {
  if (B.hash)
    for (int j = 0; j <= B.hmask; ++j) B.hash[j] = -1;
  int k = 0, b = 0;
  cav_add(B, k, t0);
  if (t1 >= 0) cav_add(B, k, t1);
  for (int q = 0; q < k; ++q) {
    const int t = B.cav[q];
    const int4 T4 = P.T[CI(t, P.n_slots, 131)];
    const int4 N4 = P.N[CI(t, P.n_slots, 131)];
    for (int e = 0; e < 3; ++e) {
      const int ref = comp(N4, e);
      const int cons = (T4.w >> e) & 1;
      int h = 0;
      if (ref >= 0 && cav_has(B, k, ref >> 2, h)) continue;
      const int u = comp(T4, mod3(e + 1)), v = comp(T4, mod3(e + 2));
      bool inside = false;
      if (!cons && ref >= 0) {
        const int4 Tn = P.T[CI(ref >> 2, P.n_slots, 132)];
        inside = incircle_ids(P, Tn.x, Tn.y, Tn.z, p) > 0;
      } else if (cons && conv && encroaches(pt(P, CI(u, P.n_verts, 133)), pt(P, CI(v, P.n_verts, 133)), p, lens)) {
        ct = t;
        ce = e;
        return G_CONV;
      }
      if (inside) {
        if (k == B.cap) return G_OVF;
        B.cav[k++] = ref >> 2;
        if (B.hash) B.hash[h] = ref >> 2;
      } else {
        if (b == B.cap + 2) return G_OVF;
        B.bnd[b++] = make_int4(u, v, ref, (int)(((unsigned)cons << 31) | (unsigned)((t << 2) | e)));
      }
    }
  }
  nc = k;
  nb = b;
  return G_OK;
}

__device__ __forceinline__ bool is_split_edge(const int4& rec, int2 sub) {
  return sub.x >= 0 && rec.z < 0 &&
         ((rec.x == sub.x && rec.y == sub.y) || (rec.x == sub.y && rec.y == sub.x));
}

// One candidate: its splitting point, its cavity in B, and its priority marks.
// MODE 0: refinement candidates (element = triangle << 2 | edge, 3 = the triangle);
// MODE 1: given points (element = vertex id, c_loc = located triangle).
// Returns G_OVF when the cavity does not fit B, else G_OK (c_state tells
// whether the candidate was grown).
// work of the grown candidates, summed per thread (see k_grow)
// (32-bit per thread: a thread's share of one launch stays far below 2^32;
// the warp sums are taken in 64 bits)
struct GrowAcc {
  unsigned grown = 0, cav = 0, bnd = 0, walk = 0, setup = 0;
};

__device__ __forceinline__ void acc_flush(const Pool& P, const GrowAcc& a, int timed = 0) {
  unsigned long long grown = a.grown, cav = a.cav, bnd = a.bnd, walk = a.walk, setup = a.setup;
  for (int o = 16; o; o >>= 1) {
    grown += __shfl_xor_sync(0xffffffffu, grown, o);
    cav += __shfl_xor_sync(0xffffffffu, cav, o);
    bnd += __shfl_xor_sync(0xffffffffu, bnd, o);
    walk += __shfl_xor_sync(0xffffffffu, walk, o);
    setup += __shfl_xor_sync(0xffffffffu, setup, o);
  }
  if ((threadIdx.x & 31) == 0 && grown + walk + setup) {
    atomicAdd(&P.ctrl->n_grown, grown);
    atomicAdd(&P.ctrl->sum_cav, cav);
    atomicAdd(&P.ctrl->sum_bnd, bnd);
    atomicAdd(&P.ctrl->sum_walk, walk);
    atomicAdd(&P.ctrl->n_setup, setup);
    if (timed) {
      atomicAdd(&P.ctrl->t_grown, grown);
      atomicAdd(&P.ctrl->t_cav, cav);
      atomicAdd(&P.ctrl->t_bnd, bnd);
      atomicAdd(&P.ctrl->t_walk, walk);
      atomicAdd(&P.ctrl->t_setup, setup);
    }
  }
}

// Splitting point, priority key and start triangles of candidate i
// (Algorithm 1).  MODE 0: refinement candidates (element =
// triangle << 2 | edge, 3 = the triangle); MODE 1: given points (element =
// vertex id, c_loc = located triangle).  False when the walk failed.
struct CandSetup {
  double2 p;
  float4 pf;
  unsigned long long key;
  int t0, t1, m, vid;
  int2 sub;
  // the first level of the growth as the pre-pass found it: bit 3q + e says
  // that the neighbour across edge e of start triangle q has the point in
  // its circumcircle (for the tuples the growth tests); -1: not known
  int pre_in;
  bool conv;
};

// the predicates of incircle_ids / orient_ids with the candidate's point
// read from its CandSetup slot (the FP64 point only on the fallback path)
__device__ __forceinline__ int incircle_cs(const Pool& P, int a, int b, int c, const CandSetup* ws) {
  a = CI(a, P.n_verts, 105);
  b = CI(b, P.n_verts, 105);
  c = CI(c, P.n_verts, 105);
  const int s = incircle_f32(P.Vf[a], P.Vf[b], P.Vf[c], ws->pf);
  GDP_DIAG_ADD(10);
  if (!s) GDP_DIAG_ADD(13);
  return s ? s : incircle_v64(P.V, a, b, c, ws->p.x, ws->p.y);
}
__device__ __forceinline__ int orient_cs(const Pool& P, int a, int b, const CandSetup* ws) {
  a = CI(a, P.n_verts, 127);
  b = CI(b, P.n_verts, 127);
  const int s = orient_f32(P.Vf[a], P.Vf[b], ws->pf);
  GDP_DIAG_ADD(9);
  if (!s) GDP_DIAG_ADD(12);
  return s ? s : orient_v64(P.V, a, b, ws->p.x, ws->p.y);
}

template <int MODE>
__device__ __noinline__ bool cand_setup(const Pool& P, int i, CandSetup& s, GrowAcc& acc) {
  P.c_ncav[i] = 0;
  P.c_nbnd[i] = 0;
  P.c_state[i] = C_FAIL;
  P.c_final[i] = 0;
  const int elem = P.c_elem[i];
  s.t1 = -1;
  s.vid = -1;
  s.pre_in = -1;
  s.conv = false;
  s.sub = make_int2(-1, -1);
  if (MODE == 1) {
    P.c_npre[i] = 0;   // no pre-marks (the pre-pass is refinement's)
    s.vid = CI(elem, P.n_verts, 126);
    s.t0 = CI(P.c_loc[i], P.n_slots, 125);
    s.m = P.T[s.t0].w >> 4;
    s.p = P.V[s.vid];
    s.key = ((unsigned long long)insert_prio(P.mi[s.m], s.vid) << 32) | (unsigned)i;
  } else {
    const int t = CI(elem >> 2, P.n_slots, 120), k = elem & 3;
    const int4 T4 = P.T[t];
    s.m = T4.w >> 4;
    const MeshInfo& M = P.mi[s.m];
    if (k == 3) {
      const TriTerms tt = tri_terms(P.V[CI(T4.x, P.n_verts, 121)], P.V[CI(T4.y, P.n_verts, 121)],
                                    P.V[CI(T4.z, P.n_verts, 121)]);
      s.p = circumcenter(tt);
      s.key = ((unsigned long long)measure_bits(fabs(tt.cr)) << 32) | (unsigned)i;
      int bt = -1, be = -1;
      int steps = 0;
      const int r = walk(P, t, P2{s.p, to_f(s.p, M.org)}, true, bt, be, steps);
      acc.walk += steps;
      if (r == -2) {
        P.c_mesh[i] = s.m;
        set_err(P.ctrl, S_WALK);
        return false;
      }
      if (r == -1) {
        // the walk meets a subsegment: split it instead (Sec. 4.3)
        const int4 B4 = P.T[CI(bt, P.n_slots, 123)];
        const int u = CI(comp(B4, mod3(be + 1)), P.n_verts, 124), v = CI(comp(B4, mod3(be + 2)), P.n_verts, 124);
        s.p = split_point(P, M, u, v);
        s.key = KEY_MID | ((unsigned long long)measure_bits(seg_measure(P.V[u], P.V[v])) << 32) |
                (unsigned)i;
        s.t0 = bt;
        const int nr = comp(P.N[bt], be);
        s.t1 = nr >= 0 ? nr >> 2 : -1;
        s.sub = make_int2(u, v);
      } else {
        s.t0 = r;
        s.conv = true;
      }
    } else {
      const int u = comp(T4, mod3(k + 1)), v = comp(T4, mod3(k + 2));
      s.p = split_point(P, M, u, v);
      s.key = KEY_MID | ((unsigned long long)measure_bits(seg_measure(P.V[u], P.V[v])) << 32) |
              (unsigned)i;
      s.t0 = t;
      const int nr = comp(P.N[t], k);
      s.t1 = nr >= 0 ? nr >> 2 : -1;
      s.sub = make_int2(u, v);
    }
  }
  P.c_mesh[i] = s.m;
  s.pf = MODE == 1 ? P.Vf[s.vid] : to_f(s.p, P.mi[s.m].org);
  return true;
}

// the circumcentre encroaches subsegment edge ce of triangle ct on its
// cavity boundary: that subsegment's split point replaces it (Sec. 4.2)
__device__ void cand_conv(const Pool& P, int i, CandSetup& s, int ct, int ce) {
  ct = CI(ct, P.n_slots, 128);
  const int4 B4 = P.T[ct];
  const int u = comp(B4, mod3(ce + 1)), v = comp(B4, mod3(ce + 2));
  s.p = split_point(P, P.mi[s.m], u, v);
  s.key = KEY_MID | ((unsigned long long)measure_bits(seg_measure(P.V[u], P.V[v])) << 32) | (unsigned)i;
  s.sub = make_int2(u, v);
  s.pf = to_f(s.p, P.mi[s.m].org);
  const int nr = comp(P.N[ct], ce);
  s.t0 = ct;
  s.t1 = nr >= 0 ? nr >> 2 : -1;
  s.pre_in = -1;
  s.conv = false;
}

// the grown candidate's record: point, priority, cavity sizes
__device__ void cand_record(const Pool& P, int i, const CandSetup& s, int nc, int nb, GrowAcc& acc) {
  P.c_pt[i] = s.p;
  P.c_ptf[i] = s.pf;
  P.c_key[i] = s.key;
  P.c_ncav[i] = nc;
  P.c_nbnd[i] = nb;
  P.c_sub[i] = s.sub;
  P.c_vid[i] = s.vid;
  P.c_vseg[i] = (s.sub.x >= 0) ? seg_of_sub(P, P.mi[s.m], s.sub.x, s.sub.y) : -1;
  P.c_state[i] = C_GROWN;
  acc.grown += 1;
  acc.cav += nc;
  acc.bnd += nb;
}

// ---------------------------------------------------------------- refinement pre-pass
// Every refinement candidate is set up once, one per lane, before any cavity
// grows: its splitting point, key, walk and start triangles go to c_setup[i].
// The candidate then puts its key (atomicMax, Sec. 5.2) on the part of its
// cavity that is known without growing it: the start triangles and, across
// their non-subsegment edges, the neighbours whose circumcircles contain the
// point -- the first level of the breadth-first growth, in the same order.
// These marks go to their own array, pmark.  A candidate that finds a larger
// key than its own on one of its pre-marked triangles shares a cavity
// triangle with a candidate of higher priority, so it would lose that
// triangle's growth mark as well; growth skips it (it stays a candidate for
// the next iteration).  Skipped candidates place no growth marks, so the
// lower-priority candidates near them are no longer blocked by candidates
// that lose anyway: fewer cavities are grown and no fewer points inserted.
// Growth reads pmark only after k_pre has finished, and pmark is never
// written during growth, so which candidates grow depends only on the set of
// keys: the outcome is deterministic and the same for a mesh alone and in a
// batch.  (A candidate whose circumcentre gives way to a subsegment during
// growth keeps the decision made for its circumcentre.)
// 128 registers: no spills (96, the compiler's choice, spilled and was 10% slower; 80: 15%)
#ifndef GDP_PRE_REGS
#define GDP_PRE_REGS 128
#endif
__global__ void __maxnreg__(GDP_PRE_REGS) k_pre(Pool P, int timed) {
  __shared__ CandSetup ws[128];
  const int n = P.ctrl->n_cand;
  GrowAcc acc;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    P.c_big[i] = -1;
    CandSetup& s = ws[threadIdx.x];
    int np = 0;
    if (cand_setup<0>(P, i, s, acc)) {
      acc.setup += 1;
      int pre[PRE_MAX];
      pre[np++] = s.t0;
      if (s.t1 >= 0 && s.t1 != s.t0) pre[np++] = s.t1;
      const int ns = P.no_prepass ? 0 : np;
      int pin = 0;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (q >= ns) break;
        const int t = CI(pre[q], P.n_slots, 140);
        const int4 T4 = P.T[t];
        const int4 N4 = P.N[t];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          const int ref = comp(N4, e);
          if (((T4.w >> e) & 1) || ref < 0) continue;
          const int tn = ref >> 2;
          bool dup = false;
#pragma unroll
          for (int r = 0; r < PRE_MAX; ++r) dup |= r < np && pre[r] == tn;
          if (dup) continue;
          const int4 Tn = P.T[CI(tn, P.n_slots, 141)];
          if (incircle_cs(P, Tn.x, Tn.y, Tn.z, &s) > 0) {
#pragma unroll
            for (int r = 0; r < PRE_MAX; ++r)
              if (r == np) pre[r] = tn;
            ++np;
            pin |= 1 << (3 * q + e);
          }
        }
      }
      s.pre_in = P.no_prepass ? -1 : pin;
      int* out = P.c_pre + (size_t)i * PRE_MAX;
#pragma unroll
      for (int r = 0; r < PRE_MAX; ++r)
        if (r < np) {
          out[r] = pre[r];
          if (!P.no_prepass) atomicMax(&P.pmark[pre[r]], s.key);
        }
      P.c_setup[i] = s;
    }
    P.c_npre[i] = np;
  }
  acc_flush(P, acc, timed);
}

// The set-up of candidate i for growth: MODE 1 computes it; MODE 0 takes the
// pre-pass's and is false when the candidate lost one of its pre-marks.
template <int MODE>
__device__ __forceinline__ bool cand_load(const Pool& P, int i, CandSetup& s, GrowAcc& acc) {
  if (MODE == 1) return cand_setup<1>(P, i, s, acc);
  const int np = P.c_npre[i];
  if (np <= 0) return false;
  s = P.c_setup[i];
  if (P.no_prepass) return true;
  const int* pre = P.c_pre + (size_t)i * PRE_MAX;
  for (int r = 0; r < np; ++r)
    if (P.pmark[pre[r]] != s.key) return false;
  return true;
}

// One candidate, one thread (the spill tiers; any cavity size up to the
// buffer's capacity).  Returns G_OVF when the cavity does not fit B, else
// G_OK (c_state tells whether the candidate was grown).
template <int MODE>
__device__ int grow_cand(const Pool& P, int i, const CavBuf& B, GrowAcc& acc) {
  CandSetup s;
  if (!cand_load<MODE>(P, i, s, acc)) return G_OK;
  P2 pp{s.p, s.pf};
  int nc = 0, nb = 0, ct = -1, ce = -1;
#ifdef GDP_DIAG
  const long long gc0 = clock64();
#endif
  const bool lens = P.mi[s.m].lens != 0;
  int g = grow(P, B, pp, s.t0, s.t1, s.conv, lens, nc, nb, ct, ce);
#ifdef GDP_DIAG
  atomicMax(&g_diag[6], (unsigned long long)(clock64() - gc0));
#endif
  if (g == G_CONV) {
    cand_conv(P, i, s, ct, ce);
    pp = P2{s.p, s.pf};
    g = grow(P, B, pp, s.t0, s.t1, false, lens, nc, nb, ct, ce);
  }
  if (g == G_OVF) return G_OVF;
  bool ok = true;
  for (int r = 0; r < nb && ok; ++r) {
    const int4 rec = B.bnd[r];
    if (is_split_edge(rec, s.sub)) continue;
    if (orient_ids(P, rec.x, rec.y, pp) <= 0) ok = false;
  }
  if (!ok) return G_OK;
  for (int j = 0; j < nc; ++j) atomicMax(&P.mark[B.cav[j]], s.key);
  cand_record(P, i, s, nc, nb, acc);
  return G_OK;
}

// ---------------------------------------------------------------- cooperative growth
// The cavity of one candidate grown by a group of W lanes (W = 32: a whole
// warp; W = 8: a quarter warp), level by level: the lanes test the (cavity
// triangle, edge) tuples of a level in parallel, W at a time (the tuple-list
// expansion of Sec. 5.3).  New triangles and boundary records are appended
// in (parent, edge) order, and a tuple sees the triangles that tuples before
// it added as cavity members, so the cavity list, the boundary records, the
// first encroached subsegment and the overflow point are those of the
// sequential breadth-first growth (grow) above, whatever W is.  Capacity
// CMAX = 32 triangles, BMAX boundary edges; the list of the cavity so far
// sits in shared memory (wc).
template <int W>
struct Group {
  int gl;          // lane within the group
  int gb;          // first warp lane of the group
  unsigned mask;   // the group's lanes in the warp
  __device__ __forceinline__ Group() {
    const int lane = threadIdx.x & 31;
    gl = lane & (W - 1);
    gb = lane - gl;
    mask = W == 32 ? 0xffffffffu : (((1u << W) - 1u) << gb);
  }
  // group-local bits (bit j = lane gb + j)
  __device__ __forceinline__ unsigned ballot(bool x) const { return __ballot_sync(mask, x) >> gb; }
  __device__ __forceinline__ unsigned match(int v) const { return __match_any_sync(mask, v) >> gb; }
  template <class X>
  __device__ __forceinline__ X shfl(X v, int src) const { return __shfl_sync(mask, v, gb + src); }
  __device__ __forceinline__ void sync() const { __syncwarp(mask); }
  __device__ __forceinline__ bool any(bool x) const { return ballot(x) != 0u; }
};

// The candidate (point, start triangles, conv) is read from its shared slot
// ws where it is used rather than held in registers for the whole growth.
template <int W>
__device__ int wgrow(const Pool& P, int* cav, int4* bnd, int* wc, const CandSetup* ws, bool lens, int& nc,
                     int& nb, int& ct, int& ce) {
  const Group<W> g;
  const int lane = g.gl;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int t0 = ws->t0, t1 = ws->t1;
  const int pin = ws->pre_in;   // the first level's incircle results, when the pre-pass has them
  int k = 1, b = 0;
  if (lane == 0) {
    wc[0] = t0;
    cav[0] = t0;
  }
  if (t1 >= 0 && t1 != t0) {
    if (lane == 0) {
      wc[1] = t1;
      cav[1] = t1;
    }
    k = 2;
  }
  g.sync();
  int lb = 0;
  while (lb < k) {
    const int le = k;
    for (int base = 3 * lb; base < 3 * le; base += W) {
      const int slot = base + lane;
      const bool act = slot < 3 * le;
      // the tuple as its boundary record would be: u, v, outside ref,
      // subsegment bit << 31 | t << 2 | e
      int tn = -1;
      bool cons = false;
      int4 rec = make_int4(-1, -1, -1, 0);
      if (act) {
        const int q = slot / 3;
        const int e = slot - 3 * q;
        const int t = wc[q];
        const int4 T4 = P.T[t];
        const int ref = comp(P.N[t], e);
        cons = (T4.w >> e) & 1;
        tn = ref >= 0 ? ref >> 2 : -1;
        rec = make_int4(comp(T4, mod3(e + 1)), comp(T4, mod3(e + 2)), ref,
                        (int)(((unsigned)cons << 31) | (unsigned)((t << 2) | e)));
      }
      bool member = false;
      for (int j = 0; j < k; ++j) member |= (wc[j] == tn);
      // one incircle test per distinct neighbour (the lowest lane's)
      const bool test = act && !member && tn >= 0 && !cons;
      const unsigned same = g.match(test ? tn : -2 - lane);
      const int leader = __ffs(same) - 1;
      bool in = false;
      if (test && lane == leader) {
        if (lb == 0 && pin >= 0) {
          in = (pin >> slot) & 1;
        } else {
          const int4 Tn = P.T[tn];
          in = incircle_cs(P, Tn.x, Tn.y, Tn.z, ws) > 0;
        }
      }
      in = g.shfl(in, leader);
      const unsigned adders = g.ballot(test && lane == leader && in);
      // a triangle added by an earlier tuple of this chunk is a cavity member
      const unsigned same_all = g.match((act && tn >= 0) ? tn : -2 - lane);
      if (act && tn >= 0 && (same_all & adders & lt_mask)) member = true;
      // 1 add, 2 boundary record, 3 encroached subsegment (the circumcentre gives way)
      int ev = 0;
      if (act && !member) {
        if (test) ev = (lane == leader && in) ? 1 : (in ? 0 : 2);
        else if (cons && ws->conv && encroaches(pt(P, rec.x), pt(P, rec.y), P2{ws->p, ws->pf}, lens)) ev = 3;
        else ev = 2;
      }
      const unsigned am = g.ballot(ev == 1);
      const unsigned rm = g.ballot(ev == 2);
      const unsigned cm = g.ballot(ev == 3);
      const int ar = __popc(am & lt_mask), rr = __popc(rm & lt_mask);
      const unsigned ovf = g.ballot((ev == 1 && k + ar >= CMAX) || (ev == 2 && b + rr >= BMAX));
      const int first_conv = cm ? __ffs(cm) - 1 : W;
      const int first_ovf = ovf ? __ffs(ovf) - 1 : W;
      if (first_conv < first_ovf) {
        const int te = g.shfl(rec.w & 0x7fffffff, first_conv);
        ct = te >> 2;
        ce = te & 3;
        return G_CONV;
      }
      if (first_ovf < W) return G_OVF;
      if (ev == 1) {
        wc[k + ar] = tn;
        cav[k + ar] = tn;
      } else if (ev == 2) {
        bnd[b + rr] = rec;
      }
      k += __popc(am);
      b += __popc(rm);
      g.sync();
    }
    lb = le;
  }
  nc = k;
  nb = b;
  return G_OK;
}

// One candidate grown by the group (all W lanes call it): splitting point,
// walk and key by the group's first lane, then the cavity, the visibility
// check of its boundary and the marks.  ws: the group's CandSetup slot.
// The growth of candidate i whose setup is in ws (all W lanes call it): the
// cavity, the visibility check of its boundary and the marks.
template <int MODE, int W>
__device__ __forceinline__ void group_grow_body(const Pool& P, int i, int* wc, CandSetup* ws, GrowAcc& acc) {
  const Group<W> g;
  int* cav = P.c_cav + (size_t)i * CMAX;
  int4* bnd = P.c_bnd + (size_t)i * BMAX;
  int nc = 0, nb = 0, ct = -1, ce = -1;
  const bool lens = P.mi[ws->m].lens != 0;
  int r = wgrow<W>(P, cav, bnd, wc, ws, lens, nc, nb, ct, ce);
  if (r == G_CONV) {
    if (g.gl == 0) cand_conv(P, i, *ws, ct, ce);   // clears ws->conv
    g.sync();
    r = wgrow<W>(P, cav, bnd, wc, ws, lens, nc, nb, ct, ce);
  }
  if (r == G_OVF) {
    if (g.gl == 0) atomicMin(&P.lane[i & (LANES_A - 1)], i);
    g.sync();
    return;
  }
  g.sync();
  const int2 sub = ws->sub;
  bool bad = false;
  for (int q = g.gl; q < nb; q += W) {
    const int4 rec = bnd[q];
    if (!is_split_edge(rec, sub) && orient_cs(P, rec.x, rec.y, ws) <= 0) bad = true;
  }
  if (g.any(bad)) return;
  const unsigned long long key = ws->key;
  for (int j = g.gl; j < nc; j += W) atomicMax(&P.mark[cav[j]], key);
  if (g.gl == 0) cand_record(P, i, *ws, nc, nb, acc);
  g.sync();
}

template <int MODE, int W>
__device__ __forceinline__ void group_grow_cand(const Pool& P, int i, int* wc, CandSetup* ws, GrowAcc& acc) {
  const Group<W> g;
  int ok = 1;
  if (g.gl == 0) {
    P.c_big[i] = -1;
    ok = cand_load<MODE>(P, i, *ws, acc) ? 1 : 0;
  }
  g.sync();
  if (!g.shfl(ok, 0)) return;
  group_grow_body<MODE, W>(P, i, wc, ws, acc);
}

// Cavity growth of the candidates in their own slots of CMAX triangles
// (larger cavities go to the spill tiers).  Up to P.warp_max candidates
// -- the usual, latency-bound case -- one warp grows each cavity (wgrow,
// k_grow_w); beyond that the launch is throughput-bound and one thread per
// candidate does less total work (grow, k_grow_t).  Both give the same
// cavities.
constexpr int WARP_GROW_MAX = 32768;   // default of Pool::warp_max

// timed: this launch is bracketed by CUDA events; its work is also counted apart
template <int MODE>
__global__ void __maxnreg__(128) k_grow_w(Pool P, int timed) {
  __shared__ int wcs[4][32];
  __shared__ CandSetup ws[4];
  const int wib = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int n = P.ctrl->n_cand;
  if (blockIdx.x == 0 && threadIdx.x == 0) P.ctrl->grow_next = 0;   // k_grow_t's counter
  if (n > P.warp_max) return;   // the per-group or per-thread kernel's case
  GrowAcc acc;
  for (int i = gw; i < n; i += nw) group_grow_cand<MODE, 32>(P, i, wcs[wib], &ws[wib], acc);
  if (MODE == 0) acc_flush(P, acc, timed);
}

// The same above P.warp_max candidates, where the launch is throughput-bound.
// A warp takes 32 candidates at a time: first their set-ups, one per lane
// (loaded from the pre-pass, with the first-ring check), then the cavities of
// the candidates that passed, a group of GROW_GROUP lanes per candidate, so
// that a level's few tuples keep most lanes busy.  The candidates that passed
// are dealt to the groups in turn (a list in shared memory), so that the
// groups of a warp have equal shares whatever the pattern of skipped ones.
#ifndef GDP_GROW_GROUP_W
#define GDP_GROW_GROUP_W 8
#endif
constexpr int GROW_GROUP = GDP_GROW_GROUP_W;   // lanes per candidate: 4, 8 or 16
static_assert(GROW_GROUP == 4 || GROW_GROUP == 8 || GROW_GROUP == 16, "a group is 4, 8 or 16 lanes");
#ifndef GDP_GROW_G_REGS
#define GDP_GROW_G_REGS 64
#endif
template <int MODE>
__global__ void __maxnreg__(GDP_GROW_G_REGS) k_grow_g(Pool P, int timed) {
  constexpr int GPB = 128 / GROW_GROUP;   // groups per 128-thread block
  constexpr int GPW = 32 / GROW_GROUP;    // groups per warp
  __shared__ int wcs[GPB][32];
  __shared__ CandSetup ws[128];           // the setups of a round, one per thread
  __shared__ int widx[4][32];             // per warp: the lanes whose candidate grows
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gib = threadIdx.x / GROW_GROUP;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int n = P.ctrl->n_cand;
  if (n <= P.warp_max) return;   // k_grow_w's case
  GrowAcc acc;
  for (int i0 = gw * 32; i0 < n; i0 += nw * 32) {
    // the setups of the warp's 32 candidates, one per lane, so that the FP64
    // circumcentre and key arithmetic and the walks keep the lanes busy
    const int i = i0 + lane;
    bool ok = false;
    if (i < n) {
      P.c_big[CI(i, P.cap_cand, 113)] = -1;
      ok = cand_load<MODE>(P, i, ws[threadIdx.x], acc);
    }
    const unsigned okm = __ballot_sync(0xffffffffu, ok);
    if (ok) widx[wib][__popc(okm & ((1u << lane) - 1u))] = lane;
    __syncwarp();
    // then every group grows one of them at a time
    const int na = __popc(okm);
    for (int r = 0; r < na; r += GPW) {
      const int k = r + lane / GROW_GROUP;
      if (k < na) {
        const int j = widx[wib][k];
        group_grow_body<MODE, GROW_GROUP>(P, i0 + j, wcs[gib], &ws[wib * 32 + j], acc);
      }
    }
    __syncwarp();   // the next round's setups overwrite the slots
  }
  if (MODE == 0) acc_flush(P, acc, timed);
}

// ---------------------------------------------------------------- warp-batched growth
// The same above P.warp_max candidates with GDP_GROW_GROUP=2: a warp grows the
// cavities of the (up to 32) candidates of a round together, level by level.
// The tuples of one level of every growing candidate form one list that the
// lanes take 32 at a time, so a lane's tuple may belong to any of them;
// matches, ballots and prefix counts are taken within each candidate's run of
// lanes.  Every lane runs every warp-wide step: the candidates share one
// instruction stream, where the four groups of k_grow_g diverge.  Per
// candidate the cavity list, the record order, the first encroached
// subsegment and the overflow point are those of the sequential
// breadth-first growth (the chunking does not matter, as in wgrow).
// Lane c keeps candidate c's set-up in ws and its cavity so far in cv[c]
// (shared memory); its counts, level start and state are in shared arrays that
// every lane reads for the candidate of its tuple.
// 128 registers: 7.2 ms per paper-shaped step against 9.7 ms at 64 (spills), 7.9 at 80, 8.2 at 96
#ifndef GDP_GROW_B_REGS
#define GDP_GROW_B_REGS 128
#endif
enum : int { B_NONE = 0, B_RUN = 1, B_OK = 2, B_CONV = 3, B_OVF = 4 };

__global__ void __maxnreg__(GDP_GROW_B_REGS) k_grow_b(Pool P, int timed) {
  const unsigned FULL = 0xffffffffu;
  __shared__ CandSetup ws[128];
  __shared__ int wcav[4][32][CMAX];
  __shared__ int sk[4][32], sb[4][32], slb[4][32], sst[4][32], sce[4][32];
  __shared__ int soff[4][33];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int n = P.ctrl->n_cand;
  if (n <= P.warp_max) return;   // k_grow_w's case
  GrowAcc acc;
  CandSetup* W = ws + wib * 32;
  int (*cv)[CMAX] = wcav[wib];
  for (int i0 = gw * 32; i0 < n; i0 += nw * 32) {
    const int i = i0 + lane;   // lane c owns candidate i0 + c
    bool ok = false;
    if (i < n) {
      P.c_big[CI(i, P.cap_cand, 114)] = -1;
      ok = cand_load<0>(P, i, W[lane], acc);
    }
    int st = ok ? B_RUN : B_NONE;
    sce[wib][lane] = 0;
    // pass 0: every candidate; pass 1: the ones whose circumcentre gave way to
    // a subsegment's split point (grown again from the subsegment's sides)
    for (int pass = 0; pass < 2; ++pass) {
      if (!__any_sync(FULL, st == B_RUN)) break;
      if (st == B_RUN) {
        const int t0 = W[lane].t0, t1 = W[lane].t1;
        cv[lane][0] = t0;
        P.c_cav[(size_t)i * CMAX] = t0;
        int k = 1;
        if (t1 >= 0 && t1 != t0) {
          cv[lane][1] = t1;
          P.c_cav[(size_t)i * CMAX + 1] = t1;
          k = 2;
        }
        sk[wib][lane] = k;
        sb[wib][lane] = 0;
        slb[wib][lane] = 0;
      }
      sst[wib][lane] = st;
      __syncwarp();
      while (__any_sync(FULL, sst[wib][lane] == B_RUN)) {
        // this level: tuples [3 lb, 3 le) of every running candidate
        const bool run = sst[wib][lane] == B_RUN;
        const int le = sk[wib][lane];
        const int T = run ? 3 * (le - slb[wib][lane]) : 0;
        int incl = T;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(FULL, incl, o);
          if (lane >= o) incl += y;
        }
        soff[wib][lane] = incl - T;
        if (lane == 31) soff[wib][32] = incl;
        __syncwarp();
        const int TT = soff[wib][32];
        for (int base = 0; base < TT; base += 32) {
          const int x = base + lane;
          bool act = x < TT;
          int c = 0;
          if (act) {   // the candidate of tuple x: the last c with soff[c] <= x
            int lo = 0, hi = 31;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (soff[wib][mid] <= x) lo = mid;
              else hi = mid - 1;
            }
            c = lo;
            act = sst[wib][c] == B_RUN;   // stopped earlier in this level: no more tuples
          }
          int slot = 0, t = -1, e = 0, tn = -1, kc = 0, bc = 0, lbc = 0;
          bool cons = false;
          int4 rec = make_int4(-1, -1, -1, 0);
          if (act) {
            lbc = slb[wib][c];
            kc = sk[wib][c];
            bc = sb[wib][c];
            slot = 3 * lbc + (x - soff[wib][c]);
            const int q = slot / 3;
            e = slot - 3 * q;
            t = cv[c][q];
            const int4 T4 = P.T[CI(t, P.n_slots, 115)];
            const int ref = comp(P.N[CI(t, P.n_slots, 115)], e);
            cons = (T4.w >> e) & 1;
            tn = ref >= 0 ? ref >> 2 : -1;
            rec = make_int4(comp(T4, mod3(e + 1)), comp(T4, mod3(e + 2)), ref,
                            (int)(((unsigned)cons << 31) | (unsigned)((t << 2) | e)));
          }
          bool member = false;
          for (int j = 0; j < kc; ++j) member |= (cv[c][j] == tn);
          const bool test = act && !member && tn >= 0 && !cons;
          // (candidate, neighbour) pairs; lane-unique values match nothing
          const unsigned long long uk = (unsigned long long)(64 + lane) << 32;
          const unsigned long long ck = ((unsigned long long)c << 32) | (unsigned)tn;
          const unsigned same = __match_any_sync(FULL, test ? ck : uk);
          const int leader = __ffs(same) - 1;
          bool in = false;
          if (test && lane == leader) {
            const CandSetup* sc = &W[c];
            if (lbc == 0 && sc->pre_in >= 0) {
              in = (sc->pre_in >> slot) & 1;
            } else {
              const int4 Tn = P.T[CI(tn, P.n_slots, 116)];
              in = incircle_cs(P, Tn.x, Tn.y, Tn.z, sc) > 0;
            }
          }
          in = __shfl_sync(FULL, in, leader);
          const unsigned adders = __ballot_sync(FULL, test && lane == leader && in);
          const unsigned same_all = __match_any_sync(FULL, (act && tn >= 0) ? ck : uk);
          if (act && tn >= 0 && (same_all & adders & lt_mask)) member = true;
          // 1 add, 2 boundary record, 3 encroached subsegment (the circumcentre gives way)
          int ev = 0;
          if (act && !member) {
            if (test) {
              ev = (lane == leader && in) ? 1 : (in ? 0 : 2);
            } else if (cons && W[c].conv &&
                       encroaches(pt(P, rec.x), pt(P, rec.y), P2{W[c].p, W[c].pf}, P.mi[W[c].m].lens != 0)) {
              ev = 3;
            } else {
              ev = 2;
            }
          }
          const unsigned seg = __match_any_sync(FULL, act ? c : 32 + lane);   // this candidate's lanes
          const unsigned am = __ballot_sync(FULL, ev == 1) & seg;
          const unsigned rm = __ballot_sync(FULL, ev == 2) & seg;
          const unsigned cm = __ballot_sync(FULL, ev == 3) & seg;
          const int ar = __popc(am & lt_mask), rr = __popc(rm & lt_mask);
          const unsigned ovf =
              __ballot_sync(FULL, (ev == 1 && kc + ar >= CMAX) || (ev == 2 && bc + rr >= BMAX)) & seg;
          const int first_conv = cm ? __ffs(cm) - 1 : 32;
          const int first_ovf = ovf ? __ffs(ovf) - 1 : 32;
          const bool head = act && lane == __ffs(seg) - 1;
          if (act) {
            if (first_conv < first_ovf) {
              if (lane == first_conv) {
                sst[wib][c] = B_CONV;
                sce[wib][c] = rec.w & 0x7fffffff;
              }
            } else if (first_ovf < 32) {
              if (head) sst[wib][c] = B_OVF;
            } else {
              const size_t ic = (size_t)(i0 + c);
              if (ev == 1) {
                cv[c][kc + ar] = tn;
                P.c_cav[ic * CMAX + kc + ar] = tn;
              } else if (ev == 2) {
                P.c_bnd[ic * BMAX + bc + rr] = rec;
              }
              if (head) {
                sk[wib][c] = kc + __popc(am);
                sb[wib][c] = bc + __popc(rm);
              }
            }
          }
          __syncwarp();
        }
        // the level is done; a level that added nothing ends the growth
        if (sst[wib][lane] == B_RUN) {
          slb[wib][lane] = le;
          if (sk[wib][lane] == le) sst[wib][lane] = B_OK;
        }
        __syncwarp();
      }
      st = sst[wib][lane];
      if (pass == 0 && st == B_CONV) {
        const int te = sce[wib][lane];
        cand_conv(P, i, W[lane], te >> 2, te & 3);
        sce[wib][lane] = 0;
        st = B_RUN;
      }
      __syncwarp();
    }
    if (st == B_OVF) atomicMin(&P.lane[i & (LANES_A - 1)], i);
    // visibility of the cavity boundaries from the points, records in parallel
    // (sce now flags a boundary edge that does not see the point)
    const int nbc = st == B_OK ? sb[wib][lane] : 0;
    int incl = nbc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    soff[wib][lane] = incl - nbc;
    if (lane == 31) soff[wib][32] = incl;
    __syncwarp();
    const int TR = soff[wib][32];
    for (int base = 0; base < TR; base += 32) {
      const int x = base + lane;
      if (x < TR) {
        int lo = 0, hi = 31;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (soff[wib][mid] <= x) lo = mid;
          else hi = mid - 1;
        }
        const int c = lo;
        const int4 rec = P.c_bnd[(size_t)(i0 + c) * BMAX + (x - soff[wib][c])];
        if (!is_split_edge(rec, W[c].sub) && orient_cs(P, rec.x, rec.y, &W[c]) <= 0) sce[wib][c] = 1;
      }
    }
    __syncwarp();
    if (st == B_OK && sce[wib][lane] == 0) {
      const int kc = sk[wib][lane];
      const unsigned long long key = W[lane].key;
      for (int j = 0; j < kc; ++j) atomicMax(&P.mark[cv[lane][j]], key);
      cand_record(P, i, W[lane], kc, sb[wib][lane], acc);
    }
    __syncwarp();   // the next round rewrites the set-ups and cavities
  }
  acc_flush(P, acc, timed);
}

// the same, one thread per candidate, when there are more than
// P.warp_max candidates (a separate kernel keeps each version's register
// allocation to itself).  Warps take runs of 32 candidates from a counter
// (reset by k_grow_w, launched just before), so that the uneven per-candidate
// work (walks, cavity sizes) does not leave SMs idle at the end.
#ifndef GDP_GROW_T_REGS
#define GDP_GROW_T_REGS 128
#endif
template <int MODE>
__global__ void __maxnreg__(GDP_GROW_T_REGS) k_grow_t(Pool P, int timed) {
  const int n = P.ctrl->n_cand;
  if (n <= P.warp_max) return;   // k_grow_w's case
  const int lane = threadIdx.x & 31;
  GrowAcc acc;
  for (;;) {
    int base = 0;
    if (lane == 0) base = atomicAdd(&P.ctrl->grow_next, 32);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n) break;
    const int i = base + lane;
    if (i >= n) continue;
    P.c_big[i] = -1;
    const CavBuf B{P.c_cav + (size_t)i * CMAX, P.c_bnd + (size_t)i * BMAX, nullptr, CMAX, 0};
    if (grow_cand<MODE>(P, i, B, acc) == G_OVF) atomicMin(&P.lane[i & (LANES_A - 1)], i);
  }
  if (MODE == 0) acc_flush(P, acc, timed);   // every thread of the block reaches this
}

// Cavity growth in a spill lane by one warp: the level-synchronous growth of
// wgrow with the lane's hash set for membership (any capacity).  Insertions
// into the set use atomicCAS, so lanes adding different triangles in the
// same step never overwrite each other; the list and record order, and so
// the result, are those of the sequential growth (grow).
__device__ __forceinline__ bool hash_has(const CavBuf& B, int t) {
  int h = (int)(hash32((uint32_t)t) & (uint32_t)B.hmask);
  for (int s = 0; s <= B.hmask; ++s) {
    const int x = B.hash[h];
    if (x == t) return true;
    if (x < 0) return false;
    h = (h + 1) & B.hmask;
  }
  return true;   // unreachable: the set is never more than half full
}

__device__ __forceinline__ void hash_put(const CavBuf& B, int t) {
  int h = (int)(hash32((uint32_t)t) & (uint32_t)B.hmask);
  for (int s = 0; s <= B.hmask; ++s) {
    const int prev = atomicCAS(&B.hash[h], -1, t);
    if (prev == -1 || prev == t) return;
    h = (h + 1) & B.hmask;
  }
}

// key > 0 (refinement): the growth gives up (G_LOSE) once it has taken a
// triangle on which the pre-pass put a larger key than its own (pmark).
// Such a triangle lies in the first ring of a candidate of higher priority,
// so this cavity would be lost unless that candidate was itself skipped;
// spill-tier cavities are large and seldom win, and their growth is the
// longest dependent chain of an iteration.  pmark is not written during
// growth, so the outcome is deterministic.
__device__ int wgrow_h(const Pool& P, const CavBuf& B, const P2& p, int t0, int t1, bool conv, bool lens,
                       unsigned long long key, int& nc, int& nb, int& ct, int& ce) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int j = lane; j <= B.hmask; j += 32) B.hash[j] = -1;
  __syncwarp();
  int k = 1, b = 0;
  if (lane == 0) {
    B.cav[0] = t0;
    hash_put(B, t0);
    if (t1 >= 0 && t1 != t0) {
      B.cav[1] = t1;
      hash_put(B, t1);
    }
  }
  if (t1 >= 0 && t1 != t0) k = 2;
  __syncwarp();
  int lb = 0;
  while (lb < k) {
    const int le = k;
    for (int base = 3 * lb; base < 3 * le; base += 32) {
      const int slot = base + lane;
      const bool act = slot < 3 * le;
      int e = 0, ref = -1, cons = 0, u = -1, v = -1, tn = -1, t = -1;
      if (act) {
        const int q = slot / 3;
        e = slot - 3 * q;
        t = B.cav[q];
        const int4 T4 = P.T[t];
        const int4 N4 = P.N[t];
        ref = comp(N4, e);
        cons = (T4.w >> e) & 1;
        u = comp(T4, mod3(e + 1));
        v = comp(T4, mod3(e + 2));
        tn = ref >= 0 ? ref >> 2 : -1;
      }
      bool member = act && tn >= 0 && hash_has(B, tn);
      const bool test = act && !member && tn >= 0 && !cons;
      const unsigned same = __match_any_sync(FULL, test ? tn : -2 - lane);
      const int leader = __ffs(same) - 1;
      bool in = false;
      if (test && lane == leader) {
        const int4 Tn = P.T[tn];
        in = incircle_ids(P, Tn.x, Tn.y, Tn.z, p) > 0;
      }
      in = __shfl_sync(FULL, in, leader);
      const unsigned adders = __ballot_sync(FULL, test && lane == leader && in);
      const unsigned same_all = __match_any_sync(FULL, (act && tn >= 0) ? tn : -2 - lane);
      if (act && tn >= 0 && (same_all & adders & lt_mask)) member = true;
      int ev = 0;
      if (act && !member) {
        if (test) ev = (lane == leader && in) ? 1 : (in ? 0 : 2);
        else if (cons && conv && encroaches(pt(P, u), pt(P, v), p, lens)) ev = 3;
        else ev = 2;
      }
      const unsigned am = __ballot_sync(FULL, ev == 1);
      const unsigned rm = __ballot_sync(FULL, ev == 2);
      const unsigned cm = __ballot_sync(FULL, ev == 3);
      const int ar = __popc(am & lt_mask), rr = __popc(rm & lt_mask);
      const unsigned ovf = __ballot_sync(FULL, (ev == 1 && k + ar >= B.cap) || (ev == 2 && b + rr >= B.cap + 2));
      const int first_conv = cm ? __ffs(cm) - 1 : 32;
      const int first_ovf = ovf ? __ffs(ovf) - 1 : 32;
      if (first_conv < first_ovf) {
        ct = __shfl_sync(FULL, t, first_conv);
        ce = __shfl_sync(FULL, e, first_conv);
        return G_CONV;
      }
      if (first_ovf < 32) return G_OVF;
      bool lose = false;
      if (ev == 1) {
        B.cav[k + ar] = tn;
        hash_put(B, tn);
        lose = key && P.pmark[tn] > key;
      } else if (ev == 2) {
        B.bnd[b + rr] = make_int4(u, v, ref, (int)(((unsigned)cons << 31) | (unsigned)((t << 2) | e)));
      }
      k += __popc(am);
      b += __popc(rm);
      __syncwarp();
      if (__any_sync(FULL, lose)) return G_LOSE;
    }
    lb = le;
  }
  nc = k;
  nb = b;
  return G_OK;
}

// Cavities that outgrew their slot (tier 0) or their tier-A lane (tier 1):
// one warp per lane; the lane is freed for the next round as it is read.
template <int MODE>
__global__ void __maxnreg__(128) k_grow_big(Pool P, int TIER) {
  __shared__ CandSetup ws[4];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int lanes = TIER ? LANES_B : LANES_A;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int l = gw; l < lanes; l += nw) {
    int* lp = P.lane + (TIER ? LANES_A : 0) + l;
    const int i = *lp;
    __syncwarp();
    if (i == LANE_FREE) continue;
    if (lane == 0) *lp = LANE_FREE;
    const int cap = TIER ? CAP_B : CAP_A;
    const size_t off = TIER ? (size_t)LANES_A * (CAP_A + 2) + (size_t)l * (CAP_B + 2)
                            : (size_t)l * (CAP_A + 2);
    const size_t hoff = TIER ? (size_t)LANES_A * 2 * CAP_A + (size_t)l * 2 * CAP_B
                             : (size_t)l * 2 * CAP_A;
    const CavBuf B{P.big_cav + off, P.big_bnd + off, P.big_hash + hoff, cap, 2 * cap - 1};
    GrowAcc acc;   // the work counters cover k_grow_w / k_grow_t only
    int ok = 1;
    if (lane == 0) {
      P.c_big[i] = (int)off;
      ok = cand_setup<MODE>(P, i, ws[wib], acc) ? 1 : 0;
    }
    __syncwarp();
    if (!__shfl_sync(FULL, ok, 0)) continue;
    CandSetup s = ws[wib];
    int nc = 0, nb = 0, ct = -1, ce = -1;
    const bool lens = P.mi[s.m].lens != 0;
    const unsigned long long lk = (MODE == 0 && !P.no_prepass) ? s.key : 0ull;
    int g = wgrow_h(P, B, P2{s.p, s.pf}, s.t0, s.t1, s.conv, lens, lk, nc, nb, ct, ce);
    if (g == G_CONV) {
      if (lane == 0) cand_conv(P, i, ws[wib], ct, ce);
      __syncwarp();
      s = ws[wib];
      g = wgrow_h(P, B, P2{s.p, s.pf}, s.t0, s.t1, false, lens, lk ? s.key : 0ull, nc, nb, ct, ce);
    }
    if (g == G_LOSE) {   // not grown: no marks, no record
      if (lane == 0) P.c_big[i] = -1;
      __syncwarp();
      continue;
    }
    if (g == G_OVF) {
      if (lane == 0) {
        P.c_big[i] = -1;
        if (TIER == 0) atomicMin(&P.lane[LANES_A + (i & (LANES_B - 1))], i);
        else set_err(P.ctrl, S_CAPACITY);
      }
      __syncwarp();
      continue;
    }
    __syncwarp();
    const P2 pp{s.p, s.pf};
    bool bad = false;
    for (int r = lane; r < nb; r += 32) {
      const int4 rec = B.bnd[r];
      if (!is_split_edge(rec, s.sub) && orient_ids(P, rec.x, rec.y, pp) <= 0) bad = true;
    }
    if (__any_sync(FULL, bad)) continue;
    for (int j = lane; j < nc; j += 32) atomicMax(&P.mark[B.cav[j]], s.key);
    if (lane == 0) cand_record(P, i, s, nc, nb, acc);
    __syncwarp();
  }
}

// lanes per survivor in k_depend and per final cavity in k_link
constexpr int DEP_W = 8;

// a point survives iff it still owns the mark of every cavity triangle
__global__ void __launch_bounds__(BS) k_survive(Pool P) {
  const unsigned FULL = 0xffffffffu;
  const int n = P.ctrl->n_cand;
  const int lane = threadIdx.x & 31;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int i0 = gt - lane; i0 < n; i0 += gs) {   // whole warps: spill-tier cavities below
    const int i = i0 + lane;
    bool big = false;
    if (i < n) {
      const int m = P.c_mesh[i];
      if (i == 0 || P.c_mesh[i - 1] != m) P.mi[m].first_cand = i;
      if (i == n - 1 || P.c_mesh[i + 1] != m) P.mi[m].last_cand = i;
      if (P.c_state[i] == C_GROWN) {
        const int nc = P.c_ncav[i];
        big = nc > CMAX;
        if (!big) {
          const unsigned long long key = P.c_key[i];
          const int* cav = cav_of(P, i);
          bool own = true;
          for (int j = 0; j < nc && own; ++j) own = P.mark[cav[j]] == key;
          P.c_state[i] = own ? C_SURV : C_LOST;
          if (own) atomicAdd(&P.ctrl->n_surv, 1ull);
        }
      }
    }
    unsigned bm = __ballot_sync(FULL, big);
    while (bm) {
      const int src = __ffs(bm) - 1;
      bm &= bm - 1;
      const int ib = __shfl_sync(FULL, i, src);
      const unsigned long long key = P.c_key[ib];
      const int* cav = cav_of(P, ib);
      const int nc = P.c_ncav[ib];
      bool own = true;
      for (int j0 = 0; j0 < nc; j0 += 32) {
        const int j = j0 + lane;
        own = __all_sync(FULL, j >= nc || P.mark[cav[j]] == key);
        if (!own) break;
      }
      if (lane == 0) {
        P.c_state[ib] = own ? C_SURV : C_LOST;
        if (own) atomicAdd(&P.ctrl->n_surv, 1ull);
      }
    }
  }
}

// Delaunay dependence (Sec. 5.2): survivors p, q whose cavities meet at a
// non-subsegment edge uv would need the edge pq if q lies inside the circle of
// p's new triangle (p,u,v); the lower priority one is dropped.  The test is
// symmetric (same four points), so both sides agree.
// A block takes its chunk BS candidates at a time; the survivors among them are
// listed in shared memory and each is checked by a group of DEP_W lanes, one
// boundary record per lane, so that the dependent loads of the records (mark,
// owner state and key, coordinates) overlap instead of running one after
// another in one thread.
__global__ void __launch_bounds__(BS) k_depend(Pool P) {
  __shared__ int sm[33];
  __shared__ int slist[BS];
  __shared__ int scount;
  const int n = P.ctrl->n_cand;
  const Chunk ch = chunk_of(n);
  const int gl = threadIdx.x & (DEP_W - 1);
  const int grp = threadIdx.x / DEP_W;
  const unsigned gmask = ((1u << DEP_W) - 1u) << ((threadIdx.x & 31) & ~(DEP_W - 1));
  int se = 0, sv = 0;
  for (int b0 = ch.b0; b0 < ch.b1; b0 += BS) {
    if (threadIdx.x == 0) scount = 0;
    __syncthreads();
    const int i = b0 + threadIdx.x;
    if (i < ch.b1) {
      if (P.c_state[i] == C_SURV) {
        slist[atomicAdd(&scount, 1)] = i;
      } else {
        P.c_final[i] = 0;
        P.c_extra[i] = 0;
      }
    }
    __syncthreads();
    const int ns = scount;
    for (int q = grp; q < ns; q += BS / DEP_W) {
      const int c = slist[q];
      const unsigned long long key = P.c_key[c];
      const P2 p{P.c_pt[c], P.c_ptf[c]};
      const int nb = P.c_nbnd[c];
      const int4* bnd = bnd_of(P, c);
      const int2 sub = P.c_sub[c];
      int eff = 0;
      bool lose = false;
      for (int r = gl; r < nb; r += DEP_W) {
        const int4 rec = bnd[r];
        if (!is_split_edge(rec, sub)) ++eff;
        if (rec.w < 0 || rec.z < 0) continue;
        const unsigned long long mo = P.mark[rec.z >> 2];
        if (!mo) continue;
        const int j = (int)(unsigned)(mo & 0xffffffffull);
        if (j == c || j >= n || P.c_state[j] != C_SURV || P.c_key[j] != mo) continue;
        if (key < mo && incircle_dep(P, p, rec.x, rec.y, j) > 0) lose = true;
      }
#pragma unroll
      for (int o = DEP_W / 2; o; o >>= 1) eff += __shfl_xor_sync(gmask, eff, o);
      lose = __ballot_sync(gmask, lose) != 0u;
      if (gl == 0) {
        const int extra = lose ? 0 : eff - P.c_ncav[c];
        P.c_final[c] = lose ? 0 : 1;
        P.c_extra[c] = extra;
        se += extra;
        sv += (!lose && P.c_vid[c] < 0) ? 1 : 0;
      }
    }
    __syncthreads();   // slist and scount are rewritten by the next step
  }
  se = block_sum(se, sm);
  sv = block_sum(sv, sm);
  if (threadIdx.x == 0) {
    P.blk[blockIdx.x] = se;
    P.blk[gridDim.x + blockIdx.x] = sv;
  }
}

__global__ void __launch_bounds__(BS) k_offsets(Pool P) {
  __shared__ int sm[33];
  const int n = P.ctrl->n_cand;
  const Chunk ch = chunk_of(n);
  int offE = block_prefix(P.blk, blockIdx.x, sm);
  int offV = block_prefix(P.blk + gridDim.x, blockIdx.x, sm);
  for (int base = ch.b0; base < ch.b1; base += BS) {
    const int i = base + threadIdx.x;
    const int e = i < ch.b1 ? P.c_extra[i] : 0;
    const int v = (i < ch.b1 && P.c_final[i] && P.c_vid[i] < 0) ? 1 : 0;
    int tE, tV;
    const int rE = block_excl_scan(e, sm, tE);
    const int rV = block_excl_scan(v, sm, tV);
    if (i < ch.b1) {
      P.c_offT[i] = offE + rE;
      P.c_offV[i] = offV + rV;
    }
    offE += tE;
    offV += tV;
  }
}

__device__ __forceinline__ void mesh_totals(const Pool& P, int f, int l, int& totE, int& totV) {
  const int nv_l = (P.c_final[l] && P.c_vid[l] < 0) ? 1 : 0;
  totE = P.c_offT[l] + P.c_extra[l] - P.c_offT[f];
  totV = P.c_offV[l] + nv_l - P.c_offV[f];
}

__device__ __forceinline__ bool replaced(const Pool& P, int ref, int n) {
  const unsigned long long mo = P.mark[ref >> 2];
  if (!mo) return false;
  const int j = (int)(unsigned)(mo & 0xffffffffull);
  return j < n && P.c_final[j] && P.c_key[j] == mo;
}

// A triangle made by an insertion: refinement evaluates it at once (the
// flag persists until its slot is rewritten); construction marks it dirty
// (the construction's end marks every triangle dirty anyway).
template <int MODE>
__device__ __forceinline__ void new_tri_code(const Pool& P, int s) {
  if (MODE == 0) P.flag[s] = (uint8_t)eval_tri(P, s);
  else P.dirty[s] = 1;
}

// A mesh whose insertions of this iteration do not fit its slots: in
// refinement the iteration inserts nothing for it (its elements stay flagged)
// and the host grows the pool after the graph replay; elsewhere it is out of
// memory.
template <int MODE>
__device__ __forceinline__ void no_room(const Pool& P, int m) {
  if (MODE == 0) {
    P.mi[m].need_grow = 2;
    atomicOr(&P.ctrl->grow, 1);
  } else {
    P.mi[m].status = S_NOMEM;
  }
}

// ---------------------------------------------------------------- spill-tier cavities, one warp each
// Cavities of the spill tiers have hundreds to tens of thousands of triangles.
// The thread-per-candidate kernels hand them to their whole warp (ballot, then
// one such candidate at a time), so no lane walks one alone.

// the fan map of the spill-tier region at offset off: keys (vertex ids) in
// big_hash, values in big_val, capacity twice the region's
struct BigMap {
  int* key;
  int2* val;
  int cap;
};
__device__ __forceinline__ BigMap big_map(const Pool& P, int off) {
  const int endA = LANES_A * (CAP_A + 2);
  if (off < endA) {
    const size_t h = (size_t)(off / (CAP_A + 2)) * 2 * CAP_A;
    return {P.big_hash + h, P.big_val + h, 2 * CAP_A};
  }
  const size_t h = (size_t)LANES_A * 2 * CAP_A + (size_t)((off - endA) / (CAP_B + 2)) * 2 * CAP_B;
  return {P.big_hash + h, P.big_val + h, 2 * CAP_B};
}

// slot of vertex v, inserted if absent (atomicCAS, linear probing); -1 only
// if the map were full, which it never is (at most half full)
__device__ __forceinline__ int map_slot(const BigMap& M, int mask, int v) {
  int h = (int)(hash32((uint32_t)v) & (uint32_t)mask);
  for (int s = 0; s <= mask; ++s) {
    const int prev = atomicCAS(&M.key[h], -1, v);
    if (prev == -1 || prev == v) return h;
    h = (h + 1) & mask;
  }
  return -1;
}

__device__ __forceinline__ int map_find(const BigMap& M, int mask, int v) {
  int h = (int)(hash32((uint32_t)v) & (uint32_t)mask);
  for (int s = 0; s <= mask; ++s) {
    const int x = __ldcg(&M.key[h]);
    if (x == v) return h;
    if (x < 0) return -1;
    h = (h + 1) & mask;
  }
  return -1;
}

// The fan of spill-tier cavity i, written by the calling warp (all lanes).
// The map gives per vertex the largest rank of a kept boundary record that
// starts (x) and that ends (y) there, so every record finds its two fan
// neighbours in O(1) -- the same ones as the quadratic search of the small
// cavities, which keeps the last match.
template <int MODE>
__device__ void fan_big(const Pool& P, int i, int m, int base, int vid, int n) {
  const unsigned FULL = 0xffffffffu;
  __syncwarp();   // the new vertex, written by one lane, is read by all
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int off = P.c_big[i];
  const BigMap M = big_map(P, off);
  const int4* bnd = P.big_bnd + off;
  const int* cav = P.big_cav + off;
  const int nc = P.c_ncav[i], nb = P.c_nbnd[i];
  const int2 sub = P.c_sub[i];
  const bool is_mid = sub.x >= 0;
  int hs = 64;
  while (hs < 2 * (nb + 1) && hs < M.cap) hs <<= 1;
  const int mask = hs - 1;
  for (int j = lane; j < hs; j += 32) {
    M.key[j] = -1;
    M.val[j] = make_int2(-1, -1);
  }
  __syncwarp();
  int done = 0;   // kept records before this chunk
  for (int r0 = 0; r0 < nb; r0 += 32) {
    const int r = r0 + lane;
    const int4 rec = r < nb ? bnd[r] : make_int4(-1, -1, -1, 0);
    const bool keep = r < nb && !is_split_edge(rec, sub);
    const unsigned km = __ballot_sync(FULL, keep);
    if (keep) {
      const int j = done + __popc(km & lt_mask);
      const int hu = map_slot(M, mask, rec.x), hv = map_slot(M, mask, rec.y);
      if (hu >= 0) atomicMax(&M.val[hu].x, j);
      if (hv >= 0) atomicMax(&M.val[hv].y, j);
    }
    done += __popc(km);
  }
  __syncwarp();
  done = 0;
  for (int r0 = 0; r0 < nb; r0 += 32) {
    const int r = r0 + lane;
    const int4 rec = r < nb ? bnd[r] : make_int4(-1, -1, -1, 0);
    const bool keep = r < nb && !is_split_edge(rec, sub);
    const unsigned km = __ballot_sync(FULL, keep);
    if (keep) {
      const int j = done + __popc(km & lt_mask);
      const int s = j < nc ? cav[j] : base + (j - nc);
      const int u = rec.x, v = rec.y;
      int cb = rec.w < 0 ? 1 : 0;
      if (is_mid && (v == sub.x || v == sub.y)) cb |= 2;
      if (is_mid && (u == sub.x || u == sub.y)) cb |= 4;
      const int hv = map_find(M, mask, v), hu = map_find(M, mask, u);
      const int a = hv >= 0 ? __ldcg(&M.val[hv].x) : -1;
      const int b = hu >= 0 ? __ldcg(&M.val[hu].y) : -1;
      const int n1 = a >= 0 ? ((a < nc ? cav[a] : base + (a - nc)) << 2) | 2 : -1;
      const int n2 = b >= 0 ? ((b < nc ? cav[b] : base + (b - nc)) << 2) | 1 : -1;
      int n0 = rec.z;
      if (n0 >= 0) {
        if (replaced(P, n0, n)) n0 = -1;   // linked by k_link
        else *comp_ptr(&P.N[n0 >> 2], n0 & 3) = s << 2;
      }
      P.T[s] = make_int4(vid, u, v, (m << 4) | cb);
      P.N[s] = make_int4(n0, n1, n2, 0);
      P.newref[rec.w & 0x7fffffff] = s << 2;
      new_tri_code<MODE>(P, s);
      P.vtri[u] = s;
      P.vtri[v] = s;
      P.vtri[vid] = s;
    }
    done += __popc(km);
  }
}

// Re-triangulate every surviving cavity as the fan from its point
// (Sec. 5.2 insertion + housekeeping).  Cavity slots are reused first, extra
// slots come from the mesh's bump region at stable prefix-sum offsets.
template <int MODE>
__global__ void __launch_bounds__(BS) k_insert_t(Pool P) {
  const unsigned FULL = 0xffffffffu;
  const int n = P.ctrl->n_cand;
  if (n <= P.warp_max) return;   // k_insert_w's case
  const int lane = threadIdx.x & 31;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int i0 = gt - lane; i0 < n; i0 += gs) {   // whole warps: spill-tier fans below
    const int i = i0 + lane;
    bool big = false;
    int m = 0, base = 0, vid = 0;
    if (i < n) {
      m = P.c_mesh[i];
      const MeshInfo& M = P.mi[m];
      const int f = M.first_cand, l = M.last_cand;
      int totE, totV;
      mesh_totals(P, f, l, totE, totV);
      const bool ok = M.tri_count + totE <= M.tri_cap && M.vert_count + totV <= M.vert_cap;
      if (i == f) {
        P.mi[m].ins_ok = ok ? 1 : 0;
        if (!ok) no_room<MODE>(P, m);
      }
      if (P.c_final[i] && ok) {
        base = M.tri_base + M.tri_count + (P.c_offT[i] - P.c_offT[f]);
        vid = (MODE == 1) ? P.c_vid[i] : M.vert_base + M.vert_count + (P.c_offV[i] - P.c_offV[f]);
        vid = CI(vid, P.n_verts, 217);
        P.c_base[i] = base;
        P.V[vid] = P.c_pt[i];
        P.Vf[vid] = P.c_ptf[i];
        P.vseg[vid] = P.c_vseg[i];
        if (MODE == 1) P.loc[vid] = -1;
        big = P.c_big[i] >= 0;
        if (!big) {
          const int4* bnd = P.c_bnd + (size_t)i * BMAX;
          const int* cav = P.c_cav + (size_t)i * CMAX;
          const int nc = CI(P.c_ncav[i], CMAX + 1, 211), nb = CI(P.c_nbnd[i], BMAX + 1, 211);
          const int2 sub = P.c_sub[i];
          const bool is_mid = sub.x >= 0;
          int j = 0;
          for (int r = 0; r < nb; ++r) {
            const int4 rec = bnd[r];
            if (is_split_edge(rec, sub)) continue;
            const int s = j < nc ? cav[j] : base + (j - nc);
            const int u = rec.x, v = rec.y;
            int cb = rec.w < 0 ? 1 : 0;
            if (is_mid && (v == sub.x || v == sub.y)) cb |= 2;
            if (is_mid && (u == sub.x || u == sub.y)) cb |= 4;
            int n1 = -1, n2 = -1, jj = 0;
            for (int r2 = 0; r2 < nb; ++r2) {
              const int4 q = bnd[r2];
              if (is_split_edge(q, sub)) continue;
              const int s2 = jj < nc ? cav[jj] : base + (jj - nc);
              if (q.x == v) n1 = (s2 << 2) | 2;
              if (q.y == u) n2 = (s2 << 2) | 1;
              ++jj;
            }
            int n0 = rec.z;
            if (n0 >= 0) {
              if (replaced(P, n0, n)) n0 = -1;   // linked by k_link
              else *comp_ptr(&P.N[n0 >> 2], n0 & 3) = s << 2;
            }
            P.T[s] = make_int4(vid, u, v, (m << 4) | cb);
            P.N[s] = make_int4(n0, n1, n2, 0);
            P.newref[rec.w & 0x7fffffff] = s << 2;
            new_tri_code<MODE>(P, s);
            P.vtri[u] = s;
            P.vtri[v] = s;
            P.vtri[vid] = s;
            ++j;
          }
        }
      }
    }
    unsigned bm = __ballot_sync(FULL, big);
    while (bm) {
      const int src = __ffs(bm) - 1;
      bm &= bm - 1;
      fan_big<MODE>(P, __shfl_sync(FULL, i, src), __shfl_sync(FULL, m, src), __shfl_sync(FULL, base, src),
              __shfl_sync(FULL, vid, src), n);
    }
  }
}

// The same, one warp per candidate up to P.warp_max candidates: the
// lanes take the cavity's boundary records (up to 64; larger spill-tier
// cavities go through fan_big), find the fan neighbours by shuffles and write
// the new triangles in parallel.  Identical output to k_insert_t.
template <int MODE>
__global__ void __launch_bounds__(128) k_insert_w(Pool P) {
  const unsigned FULL = 0xffffffffu;
  const int n = P.ctrl->n_cand;
  if (n > P.warp_max) return;   // k_insert_t's case
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = gw; i < n; i += nw) {
    const int m = P.c_mesh[i];
    const MeshInfo& M = P.mi[m];
    const int f = M.first_cand, l = M.last_cand;
    int totE, totV;
    mesh_totals(P, f, l, totE, totV);
    const bool ok = M.tri_count + totE <= M.tri_cap && M.vert_count + totV <= M.vert_cap;
    if (lane == 0 && i == f) {
      P.mi[m].ins_ok = ok ? 1 : 0;
      if (!ok) no_room<MODE>(P, m);
    }
    if (!P.c_final[i] || !ok) continue;
    const int base = M.tri_base + M.tri_count + (P.c_offT[i] - P.c_offT[f]);
    const int vid = (MODE == 1) ? P.c_vid[i] : M.vert_base + M.vert_count + (P.c_offV[i] - P.c_offV[f]);
    const int4* bnd = bnd_of(P, i);
    const int* cav = cav_of(P, i);
    const int nc = P.c_ncav[i], nb = P.c_nbnd[i];
    const int2 sub = P.c_sub[i];
    const bool is_mid = sub.x >= 0;
    if (lane == 0) {
      P.c_base[i] = base;
      P.V[vid] = P.c_pt[i];
      P.Vf[vid] = P.c_ptf[i];
      P.vseg[vid] = P.c_vseg[i];
      if (MODE == 1) P.loc[vid] = -1;
    }
    __syncwarp();   // the new vertex is read by every lane (new_tri_code)
    if (nb > 64) {   // a spill-tier cavity: the map-based fan
      fan_big<MODE>(P, i, m, base, vid, n);
      continue;
    }
    // records lane and lane + 32; j = rank among the records that are not the split edge
    int4 rec[2];
    bool keep[2];
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      rec[h] = r < nb ? bnd[r] : make_int4(-1, -1, -1, 0);
      keep[h] = r < nb && !is_split_edge(rec[h], sub);
    }
    const unsigned k0 = __ballot_sync(FULL, keep[0]), k1 = __ballot_sync(FULL, keep[1]);
    int slot[2];
    for (int h = 0; h < 2; ++h) {
      const int j = h == 0 ? __popc(k0 & lt_mask) : __popc(k0) + __popc(k1 & lt_mask);
      slot[h] = j < nc ? cav[j] : base + (j - nc);
    }
    // fan neighbours: the record starting where mine ends (edge 2), the one ending where mine starts (edge 1)
    int n1[2] = {-1, -1}, n2[2] = {-1, -1};
    for (int q = 0; q < nb; ++q) {
      const int h = q >> 5, src = q & 31;
      const int qx = __shfl_sync(FULL, h ? rec[1].x : rec[0].x, src);
      const int qy = __shfl_sync(FULL, h ? rec[1].y : rec[0].y, src);
      const int qs = __shfl_sync(FULL, h ? slot[1] : slot[0], src);
      const bool qk = ((h ? k1 : k0) >> src) & 1;
      if (!qk) continue;
      for (int g = 0; g < 2; ++g) {
        if (qx == rec[g].y) n1[g] = (qs << 2) | 2;
        if (qy == rec[g].x) n2[g] = (qs << 2) | 1;
      }
    }
    for (int h = 0; h < 2; ++h) {
      if (!keep[h]) continue;
      const int s = slot[h];
      const int u = rec[h].x, v = rec[h].y;
      int cb = rec[h].w < 0 ? 1 : 0;
      if (is_mid && (v == sub.x || v == sub.y)) cb |= 2;
      if (is_mid && (u == sub.x || u == sub.y)) cb |= 4;
      int n0 = rec[h].z;
      if (n0 >= 0) {
        if (replaced(P, n0, n)) n0 = -1;   // linked by k_link
        else *comp_ptr(&P.N[n0 >> 2], n0 & 3) = s << 2;
      }
      P.T[s] = make_int4(vid, u, v, (m << 4) | cb);
      P.N[s] = make_int4(n0, n1[h], n2[h], 0);
      P.newref[rec[h].w & 0x7fffffff] = s << 2;
      new_tri_code<MODE>(P, s);
      P.vtri[u] = s;
      P.vtri[v] = s;
      P.vtri[vid] = s;
    }
  }
}

// The same above P.warp_max candidates by groups of INSERT_GROUP lanes (eight
// candidates per warp at a time): a warp takes 32 candidates, one per lane for
// the room check, the slot bases and the new vertices, then deals the final
// ones to its groups in turn.  A group takes its cavity's boundary records (up
// to BMAX, ceil(BMAX / 4) per lane), finds the fan neighbours by shuffles
// within the group and writes and evaluates the new triangles in parallel.  A
// spill-tier cavity is written by the whole warp (fan_big) after the groups.
// Identical output to k_insert_t.
#ifndef GDP_INSERT_GROUP_W
#define GDP_INSERT_GROUP_W 4
#endif
constexpr int INSERT_GROUP = GDP_INSERT_GROUP_W;   // lanes per cavity: 4 or 8 (4 measured faster)
static_assert(INSERT_GROUP == 4 || INSERT_GROUP == 8, "an insertion group is 4 or 8 lanes");
#ifdef GDP_INSERT_REGS
#define GDP_INSERT_G_BOUNDS __maxnreg__(GDP_INSERT_REGS)
#else
#define GDP_INSERT_G_BOUNDS __launch_bounds__(128)
#endif
template <int MODE>
__global__ void GDP_INSERT_G_BOUNDS k_insert_g(Pool P) {
  constexpr int W = INSERT_GROUP;
  constexpr int GPW = 32 / W;
  constexpr int R = (BMAX + W - 1) / W;   // records per lane
  const unsigned FULL = 0xffffffffu;
  __shared__ int4 wq[4][32];   // per warp: the final candidates of a round (i, mesh, base, vid)
  const int n = P.ctrl->n_cand;
  if (n <= P.warp_max) return;   // k_insert_w's case
  const Group<W> g;
  const unsigned lt_mask = (1u << g.gl) - 1u;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int i0 = gw * 32; i0 < n; i0 += nw * 32) {
    // one candidate per lane: room check, slots and the new vertex
    const int i0l = i0 + lane;
    bool fin = false, big = false;
    int m = 0, base = 0, vid = 0;
    if (i0l < n) {
      m = P.c_mesh[i0l];
      const MeshInfo& M = P.mi[m];
      const int f = M.first_cand, l = M.last_cand;
      int totE, totV;
      mesh_totals(P, f, l, totE, totV);
      const bool ok = M.tri_count + totE <= M.tri_cap && M.vert_count + totV <= M.vert_cap;
      if (i0l == f) {
        P.mi[m].ins_ok = ok ? 1 : 0;
        if (!ok) no_room<MODE>(P, m);
      }
      if (P.c_final[i0l] && ok) {
        fin = true;
        base = M.tri_base + M.tri_count + (P.c_offT[i0l] - P.c_offT[f]);
        vid = (MODE == 1) ? P.c_vid[i0l] : M.vert_base + M.vert_count + (P.c_offV[i0l] - P.c_offV[f]);
        vid = CI(vid, P.n_verts, 207);
        P.c_base[i0l] = base;
        P.V[vid] = P.c_pt[i0l];
        P.Vf[vid] = P.c_ptf[i0l];
        P.vseg[vid] = P.c_vseg[i0l];
        if (MODE == 1) P.loc[vid] = -1;
        big = P.c_big[i0l] >= 0;
      }
    }
    const unsigned fm = __ballot_sync(FULL, fin && !big);
    if (fin && !big) wq[wib][__popc(fm & ((1u << lane) - 1u))] = make_int4(i0l, m, base, vid);
    __syncwarp();   // the new vertices (read by new_tri_code) and the list
    // then the groups write the small cavities' fans, the finals dealt in turn
    const int nf = __popc(fm);
    for (int r0 = 0; r0 < nf; r0 += GPW) {
      const int k = r0 + lane / W;
      if (k < nf) {
        const int4 e = wq[wib][k];
        const int i = e.x;
        const int mm = e.y, base = e.z, vid = e.w;
        const int4* bnd = P.c_bnd + (size_t)i * BMAX;
        const int* cav = P.c_cav + (size_t)i * CMAX;
        const int nc = CI(P.c_ncav[i], CMAX + 1, 201), nb = CI(P.c_nbnd[i], BMAX + 1, 201);
        const int2 sub = P.c_sub[i];
        const bool is_mid = sub.x >= 0;
        int4 rec[R];
        bool keep[R];
        int slot[R];
        int done = 0;   // kept records before chunk h
        for (int h = 0; h < R; ++h) {
          const int r = g.gl + W * h;
          rec[h] = r < nb ? bnd[r] : make_int4(-1, -1, -1, 0);
          keep[h] = r < nb && !is_split_edge(rec[h], sub);
          const unsigned km = g.ballot(keep[h]);
          const int j = done + __popc(km & lt_mask);
          slot[h] = j < nc ? cav[CI(j, CMAX, 202)] : base + (j - nc);
          done += __popc(km);
        }
        // fan neighbours: the record starting where mine ends (edge 2) and
        // the one ending where mine starts (edge 1); the last match wins
        int n1[R], n2[R];
        for (int h = 0; h < R; ++h) n1[h] = n2[h] = -1;
        for (int q = 0; q < nb; ++q) {
          const int hq = q / W, src = q - W * hq;
          int qx = -1, qy = -1, qs = -1, qk = 0;
          for (int h = 0; h < R; ++h)
            if (h == hq) { qx = rec[h].x; qy = rec[h].y; qs = slot[h]; qk = keep[h] ? 1 : 0; }
          qx = g.shfl(qx, src);
          qy = g.shfl(qy, src);
          qs = g.shfl(qs, src);
          qk = g.shfl(qk, src);
          if (!qk) continue;
          for (int h = 0; h < R; ++h) {
            if (qx == rec[h].y) n1[h] = (qs << 2) | 2;
            if (qy == rec[h].x) n2[h] = (qs << 2) | 1;
          }
        }
        for (int h = 0; h < R; ++h) {
          if (!keep[h]) continue;
          const int s = slot[h];
          const int u = rec[h].x, v = rec[h].y;
          int cb = rec[h].w < 0 ? 1 : 0;
          if (is_mid && (v == sub.x || v == sub.y)) cb |= 2;
          if (is_mid && (u == sub.x || u == sub.y)) cb |= 4;
          int n0 = rec[h].z;
          if (n0 >= 0) {
            if (replaced(P, CI(n0, 4ll * P.n_slots, 203), n)) n0 = -1;   // linked by k_link
            else *comp_ptr(&P.N[CI(n0 >> 2, P.n_slots, 203)], n0 & 3) = s << 2;
          }
          P.T[CI(s, P.n_slots, 204)] = make_int4(vid, u, v, (mm << 4) | cb);
          P.N[CI(s, P.n_slots, 204)] = make_int4(n0, n1[h], n2[h], 0);
          P.newref[CI(rec[h].w & 0x7fffffff, 4ll * P.n_slots, 205)] = s << 2;
          new_tri_code<MODE>(P, CI(s, P.n_slots, 204));
          P.vtri[CI(u, P.n_verts, 206)] = s;
          P.vtri[CI(v, P.n_verts, 206)] = s;
          P.vtri[CI(vid, P.n_verts, 206)] = s;
        }
      }
    }
    __syncwarp();   // wq is rewritten by the next round
    unsigned bm = __ballot_sync(FULL, fin && big);
    while (bm) {
      const int src = __ffs(bm) - 1;
      bm &= bm - 1;
      fan_big<MODE>(P, __shfl_sync(FULL, i0l, src), __shfl_sync(FULL, m, src), __shfl_sync(FULL, base, src),
                    __shfl_sync(FULL, vid, src), n);
    }
  }
}

// links between adjacent cavities, then per-mesh counters
template <int MODE>
__global__ void __launch_bounds__(BS) k_link(Pool P) {
  const unsigned FULL = 0xffffffffu;
  const int n = P.ctrl->n_cand;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  __shared__ int wl[BS / 32][32];
  const int wib = threadIdx.x >> 5;
  const int gl = lane & (DEP_W - 1);
  const unsigned gmask = ((1u << DEP_W) - 1u) << (lane & ~(DEP_W - 1));
  const unsigned glt = (1u << gl) - 1u;
  int ins = 0;
  for (int i0 = gt - lane; i0 < n; i0 += gs) {   // whole warps: spill-tier cavities below
    const int i = i0 + lane;
    bool big = false, small = false;
    if (i < n) {
      const int m = P.c_mesh[i];
      const MeshInfo& M = P.mi[m];
      const bool ok = M.ins_ok;
      if (P.c_final[i] && ok) {
        ++ins;
        big = P.c_big[i] >= 0;
        small = !big;
      }
      if (i == M.last_cand && ok) {
        int totE, totV;
        mesh_totals(P, M.first_cand, i, totE, totV);
        const int tc = M.tri_count + totE, vc = M.vert_count + totV;
        P.mi[m].tri_count = tc;
        P.mi[m].vert_count = vc;
        if (MODE == 0) {
          P.mi[m].steiner = M.steiner + totV;
          // under a quarter of the slots left: ask for more before they run out
          if (4ll * (M.tri_cap - tc) < M.tri_cap || 4ll * (M.vert_cap - vc) < M.vert_cap) {
            if (!M.need_grow) P.mi[m].need_grow = 1;
            atomicOr(&P.ctrl->grow, 1);
          }
        }
      }
    }
    // the small cavities' links, a group of DEP_W lanes per cavity (records in
    // parallel; the j-th kept record owns the j-th new slot)
    const unsigned sm_ = __ballot_sync(FULL, small);
    if (small) wl[wib][__popc(sm_ & lt_mask)] = i;
    __syncwarp();
    const int ns = __popc(sm_);
    for (int r0 = 0; r0 < ns; r0 += 32 / DEP_W) {
      const int k = r0 + lane / DEP_W;
      if (k < ns) {
        const int c = wl[wib][k];
        const int4* bnd = P.c_bnd + (size_t)c * BMAX;
        const int* cav = P.c_cav + (size_t)c * CMAX;
        const int nc = P.c_ncav[c], nb = P.c_nbnd[c], base = P.c_base[c];
        const int2 sub = P.c_sub[c];
        int done = 0;
        for (int h = 0; h < nb; h += DEP_W) {
          const int r = h + gl;
          const int4 rec = r < nb ? bnd[r] : make_int4(-1, -1, -1, 0);
          const bool keep = r < nb && !is_split_edge(rec, sub);
          const unsigned km = __ballot_sync(gmask, keep) >> (lane & ~(DEP_W - 1));
          if (keep && rec.z >= 0 && replaced(P, rec.z, n)) {
            const int j = done + __popc(km & glt);
            const int s = j < nc ? cav[j] : base + (j - nc);
            P.N[s].x = P.newref[rec.z];
          }
          done += __popc(km);
        }
      }
    }
    __syncwarp();   // wl is rewritten by the next round
    unsigned bm = __ballot_sync(FULL, big);
    while (bm) {
      const int src = __ffs(bm) - 1;
      bm &= bm - 1;
      const int ib = __shfl_sync(FULL, i, src);
      const int off = P.c_big[ib];
      const int4* bnd = P.big_bnd + off;
      const int* cav = P.big_cav + off;
      const int nc = P.c_ncav[ib], nb = P.c_nbnd[ib], base = P.c_base[ib];
      const int2 sub = P.c_sub[ib];
      int done = 0;   // kept records before this chunk
      for (int r0 = 0; r0 < nb; r0 += 32) {
        const int r = r0 + lane;
        const int4 rec = r < nb ? bnd[r] : make_int4(-1, -1, -1, 0);
        const bool keep = r < nb && !is_split_edge(rec, sub);
        const unsigned km = __ballot_sync(FULL, keep);
        if (keep && rec.z >= 0 && replaced(P, rec.z, n)) {
          const int j = done + __popc(km & lt_mask);
          const int s = j < nc ? cav[j] : base + (j - nc);
          P.N[s].x = P.newref[rec.z];
        }
        done += __popc(km);
      }
    }
  }
  for (int o = 16; o; o >>= 1) ins += __shfl_xor_sync(0xffffffffu, ins, o);
  if ((threadIdx.x & 31) == 0 && ins) {
    atomicAdd(&P.ctrl->n_ins, (unsigned long long)ins);
    atomicAdd(&P.ctrl->tot_ins, (unsigned long long)ins);
  }
}

// ---------------------------------------------------------------- export
// Mesh m in export numbering (input points first, the auxiliary vertices
// dropped, Steiner points after): its live triangles in slot order and its
// subsegments, each emitted once -- from the triangle with the smaller slot,
// or the only one on the hull -- with the input segment it lies on.
__device__ __forceinline__ int ex_id(const MeshInfo& M, int g) {
  const int l = g - M.vert_base;
  return l < M.n_in ? l : l - N_AUX;
}

__device__ __forceinline__ bool ex_sub(const Pool& P, int t, const int4& T4, int e) {
  if (!((T4.w >> e) & 1)) return false;
  const int nb = comp(P.N[t], e);
  return nb < 0 || (nb >> 2) > t;
}

__global__ void __launch_bounds__(BS) k_export_count(Pool P, int m) {
  __shared__ int sm[33];
  const MeshInfo& M = P.mi[m];
  const Chunk ch = chunk_of(M.tri_count);
  int nt = 0, ns = 0;
  for (int k = ch.b0 + threadIdx.x; k < ch.b1; k += BS) {
    const int t = M.tri_base + k;
    const int4 T4 = P.T[t];
    if (T4.w < 0 || (T4.w & INFO_DEAD)) continue;
    ++nt;
    for (int e = 0; e < 3; ++e) ns += ex_sub(P, t, T4, e) ? 1 : 0;
  }
  nt = block_sum(nt, sm);
  ns = block_sum(ns, sm);
  if (threadIdx.x == 0) {
    P.blk[blockIdx.x] = nt;
    P.blk[gridDim.x + blockIdx.x] = ns;
  }
}

// live triangles and subsegments of every mesh (a subsegment counted once,
// as the export emits it), for the statistics of a refine call; blocks on a
// 2D grid (x: blocks of one mesh, y: meshes)
__global__ void __launch_bounds__(BS) k_count_live(Pool P) {
  unsigned long long nt = 0, ns = 0;
  for (int m = blockIdx.y; m < P.n_mesh; m += gridDim.y) {
    const MeshInfo& M = P.mi[m];
    for (int k = blockIdx.x * BS + threadIdx.x; k < M.tri_count; k += gridDim.x * BS) {
      const int t = M.tri_base + k;
      const int4 T4 = P.T[t];
      if (T4.w < 0 || (T4.w & INFO_DEAD)) continue;
      ++nt;
      for (int e = 0; e < 3; ++e) ns += ex_sub(P, t, T4, e) ? 1 : 0;
    }
  }
  for (int o = 16; o; o >>= 1) {
    nt += __shfl_xor_sync(0xffffffffu, nt, o);
    ns += __shfl_xor_sync(0xffffffffu, ns, o);
  }
  if ((threadIdx.x & 31) == 0 && nt + ns) {
    atomicAdd(&P.ctrl->live_tri, nt);
    atomicAdd(&P.ctrl->live_sub, ns);
  }
}

__global__ void __launch_bounds__(BS) k_export_write(Pool P, int m, int* tri_out, int* sub_out) {
  __shared__ int sm[33];
  const MeshInfo& M = P.mi[m];
  const Chunk ch = chunk_of(M.tri_count);
  int ot = block_prefix(P.blk, blockIdx.x, sm);
  int os = block_prefix(P.blk + gridDim.x, blockIdx.x, sm);
  for (int base = ch.b0; base < ch.b1; base += BS) {
    const int k = base + threadIdx.x;
    int4 T4 = make_int4(-1, -1, -1, -1);
    const int t = M.tri_base + k;
    bool live = false;
    int es = 0;
    if (k < ch.b1) {
      T4 = P.T[t];
      live = !(T4.w < 0 || (T4.w & INFO_DEAD));
      if (live)
        for (int e = 0; e < 3; ++e) es += ex_sub(P, t, T4, e) ? 1 : 0;
    }
    int tt, ts;
    const int rt = block_excl_scan(live ? 1 : 0, sm, tt);
    const int rs = block_excl_scan(es, sm, ts);
    if (live) {
      int* o = tri_out + 3 * (size_t)(ot + rt);
      o[0] = ex_id(M, T4.x);
      o[1] = ex_id(M, T4.y);
      o[2] = ex_id(M, T4.z);
      int q = os + rs;
      for (int e = 0; e < 3; ++e) {
        if (!ex_sub(P, t, T4, e)) continue;
        const int u = comp(T4, mod3(e + 1)), v = comp(T4, mod3(e + 2));
        int sg = P.vseg[u];
        if (sg < 0) sg = P.vseg[v];
        if (sg < 0) {   // both ends are input points: the segment joining them
          const int lu = u - M.vert_base;
          for (int a = P.adj_off[M.adj_base + lu]; a < P.adj_off[M.adj_base + lu + 1] && sg < 0; ++a) {
            const int g = P.adj[a];
            const int2 s2 = P.seg[g];
            if ((s2.x == u && s2.y == v) || (s2.x == v && s2.y == u)) sg = g;
          }
        }
        int* w = sub_out + 3 * (size_t)q++;
        w[0] = ex_id(M, u);
        w[1] = ex_id(M, v);
        w[2] = sg < 0 ? -1 : sg - M.seg_base;
      }
    }
    ot += tt;
    os += ts;
  }
}

// ---------------------------------------------------------------- consistency (test hook)
// counts: [0] links that are not mutual, [1] links whose shared edge does not
// match, [2] subsegment bits that differ across an edge, [3] triangles not CCW
// (exact), [4] hull edges (no neighbour) that are not subsegments
__global__ void __launch_bounds__(BS) k_check(Pool P, unsigned long long* cnt) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int t = gt; t < P.n_slots; t += gs) {
    const int4 T4 = P.T[t];
    if (T4.w < 0 || (T4.w & INFO_DEAD)) continue;
    const int4 N4 = P.N[t];
    if (orient(pt(P, T4.x), pt(P, T4.y), pt(P, T4.z)) <= 0) atomicAdd(&cnt[3], 1ull);
    for (int e = 0; e < 3; ++e) {
      const int ref = comp(N4, e);
      const int u = comp(T4, mod3(e + 1)), v = comp(T4, mod3(e + 2));
      if (ref < 0) {
        if (!((T4.w >> e) & 1)) atomicAdd(&cnt[4], 1ull);
        continue;
      }
      const int t2 = ref >> 2, e2 = ref & 3;
      const int4 B4 = P.T[t2];
      bool badl = false;
      if (comp(P.N[t2], e2) != ((t << 2) | e)) { atomicAdd(&cnt[0], 1ull); badl = true; }
      if (comp(B4, mod3(e2 + 1)) != v || comp(B4, mod3(e2 + 2)) != u) {
        atomicAdd(&cnt[1], 1ull);
        badl = true;
      }
      if (badl) {   // keep the first four offenders (t << 2 | e) for diagnostics
        const unsigned long long k = atomicAdd(&cnt[5], 1ull);
        if (k < 4) cnt[6 + k] = (unsigned long long)((t << 2) | e);
      }
      if (((T4.w >> e) & 1) != ((B4.w >> e2) & 1)) atomicAdd(&cnt[2], 1ull);
    }
  }
}

// ---------------------------------------------------------------- scan report (test hook)
// Every live bad triangle (kind 0, or 2 when the small-angle exemption
// accepts it); every subsegment edge: encroachment by this triangle's apex
// (kind 1) with its split point.  Output order is not defined.
__global__ void __launch_bounds__(BS) k_scan_report(Pool P, double B2, int lens, int* kind, int* verts,
                                                    double2* spt, unsigned* meas, int cap,
                                                    int* count) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int t = gt; t < P.n_slots; t += gs) {
    const int4 T4 = P.T[t];
    if (T4.w < 0 || (T4.w & INFO_DEAD)) continue;
    const MeshInfo& M = P.mi[T4.w >> 4];
    const TriTerms tt = tri_terms(P.V[T4.x], P.V[T4.y], P.V[T4.z]);
    const int q = bad_f32(P.Vf[T4.x], P.Vf[T4.y], P.Vf[T4.z], __double2float_rn(B2));
    if (q > 0 || (q == 0 && is_bad(tt, B2))) {
      const int r = atomicAdd(count, 1);
      if (r < cap) {
        kind[r] = exempt(P, M, T4) ? 2 : 0;
        verts[3 * r] = T4.x; verts[3 * r + 1] = T4.y; verts[3 * r + 2] = T4.z;
        spt[r] = circumcenter(tt);
        meas[r] = measure_bits(fabs(tt.cr));
      }
    }
    for (int e = 0; e < 3; ++e) {
      if (!((T4.w >> e) & 1)) continue;
      const int u = comp(T4, mod3(e + 1)), v = comp(T4, mod3(e + 2));
      if (encroaches(pt(P, u), pt(P, v), pt(P, comp(T4, e)), lens != 0)) {
        const int r = atomicAdd(count, 1);
        if (r < cap) {
          kind[r] = 1;
          verts[3 * r] = u; verts[3 * r + 1] = v; verts[3 * r + 2] = -1;
          spt[r] = split_point(P, M, u, v);
          meas[r] = measure_bits(seg_measure(P.V[u], P.V[v]));
        }
      }
    }
  }
}

}  // namespace gdp
