// Host side of the library: pool layout and allocation, the CDT driver, the
// refinement loop (graph-captured iterations), export, and the C ABI of
// include/gdp.h.  The host only sizes buffers, launches kernels and reads a
// few counters; all mesh computation happens in the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "gdp.h"
#include "gdp_cdt.cuh"
#include "gdp_flipflop.cuh"

using namespace gdp;

namespace {

// ---------------------------------------------------------------- setup kernels
// per-mesh kernels over a 2D grid (x: blocks of one mesh, y: meshes)
__global__ void k_scatter_points(Pool P, const double2* src, const long long* pt_off) {
  for (int m = blockIdx.y; m < P.n_mesh; m += gridDim.y) {
    const MeshInfo& M = P.mi[m];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M.n_in; k += gridDim.x * blockDim.x)
      P.V[M.vert_base + k] = src[pt_off[m] + k];
  }
}

__global__ void k_scatter_segs(Pool P, const int2* src, const long long* seg_off, int* seg_mesh) {
  const int m = blockIdx.x;
  MeshInfo& M = P.mi[m];
  for (int k = threadIdx.x; k < M.n_seg; k += blockDim.x) {
    const int2 s = src[seg_off[m] + k];
    const int g = M.seg_base + k;
    seg_mesh[g] = m;
    if (s.x < 0 || s.x >= M.n_in || s.y < 0 || s.y >= M.n_in || s.x == s.y) {
      M.status = S_INPUT;
      P.seg[g] = make_int2(M.vert_base, M.vert_base);
      continue;
    }
    P.seg[g] = make_int2(M.vert_base + s.x, M.vert_base + s.y);
  }
}

__global__ void k_adj_count(Pool P, const int* seg_mesh, int n_seg_total, int* cnt) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int g = gt; g < n_seg_total; g += gs) {
    const MeshInfo& M = P.mi[seg_mesh[g]];
    const int2 s = P.seg[g];
    atomicAdd(&cnt[M.adj_base + (s.x - M.vert_base) + 1], 1);
    atomicAdd(&cnt[M.adj_base + (s.y - M.vert_base) + 1], 1);
  }
}

__global__ void k_adj_fill(Pool P, const int* seg_mesh, int n_seg_total, int* cursor) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int g = gt; g < n_seg_total; g += gs) {
    const MeshInfo& M = P.mi[seg_mesh[g]];
    const int2 s = P.seg[g];
    P.adj[atomicAdd(&cursor[M.adj_base + (s.x - M.vert_base)], 1)] = g;
    P.adj[atomicAdd(&cursor[M.adj_base + (s.y - M.vert_base)], 1)] = g;
  }
}

// inclusive scan of an int array in place (block counts, then block scans)
__global__ void __launch_bounds__(BS) k_iscan_count(int* a, int n, int* blk) {
  __shared__ int sm[33];
  const Chunk ch = chunk_of(n);
  int s = 0;
  for (int k = ch.b0 + threadIdx.x; k < ch.b1; k += BS) s += a[k];
  s = block_sum(s, sm);
  if (threadIdx.x == 0) blk[blockIdx.x] = s;
}

__global__ void __launch_bounds__(BS) k_iscan_write(int* a, int n, const int* blk) {
  __shared__ int sm[33];
  const Chunk ch = chunk_of(n);
  int off = block_prefix(blk, blockIdx.x, sm);
  for (int base = ch.b0; base < ch.b1; base += BS) {
    const int k = base + threadIdx.x;
    const int v = k < ch.b1 ? a[k] : 0;
    int tot;
    const int r = block_excl_scan(v, sm, tot);
    if (k < ch.b1) a[k] = off + r + v;
    off += tot;
  }
}

// ---------------------------------------------------------------- spatial order of the construction's points
// The construction inserts the pending points in the order of the pending list
// (each triangle takes one per round, chosen by its own key), and new triangles
// take slots in that order.  Listing each mesh's points by cell of a 2^L x 2^L
// grid over its box -- cells in Morton order, the points of a cell by id --
// puts triangles that are near in the plane near in memory, for the
// construction's walks and for every kernel after it.  The order depends only
// on the mesh's own points (a mesh is triangulated the same alone and in a
// batch), and the CDT does not depend on the order at all.  A mesh with a cell
// of more than CELL_SORT_MAX points (dense duplicates) keeps its input order.
constexpr int CELL_SORT_MAX = 256;

__device__ __forceinline__ uint32_t spread16(uint32_t v) {
  v &= 0xffffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

// the Morton index of p's cell; coordinates outside the box or not finite go
// to the nearest edge cell (such a mesh is rejected later anyway)
__device__ __forceinline__ int cell_of(const MeshInfo& M, double2 p, int L) {
  const double w = fmax(M.hi.x - M.lo.x, M.hi.y - M.lo.y);
  const int G = 1 << L;
  const double fx = w > 0 ? (p.x - M.lo.x) / w * G : 0.0;
  const double fy = w > 0 ? (p.y - M.lo.y) / w * G : 0.0;
  const int cx = (fx >= 0.0 && fx < G) ? (int)fx : (fx >= G ? G - 1 : 0);
  const int cy = (fy >= 0.0 && fy < G) ? (int)fy : (fy >= G ? G - 1 : 0);
  return (int)(spread16((uint32_t)cx) | (spread16((uint32_t)cy) << 1));
}

__global__ void k_cell_count(Pool P, const int* cbase, const int* lev, int* cnt) {
  for (int m = blockIdx.y; m < P.n_mesh; m += gridDim.y) {
    const MeshInfo& M = P.mi[m];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M.n_in; k += gridDim.x * blockDim.x)
      atomicAdd(&cnt[cbase[m] + cell_of(M, P.V[M.vert_base + k], lev[m])], 1);
  }
}

// end: inclusive prefix sums of cnt (a cell's points end there)
__global__ void k_cell_scatter(Pool P, const int* cbase, const int* lev, const int* end, const int* cnt,
                               int* fill, int* tmp, int* crowded) {
  for (int m = blockIdx.y; m < P.n_mesh; m += gridDim.y) {
    const MeshInfo& M = P.mi[m];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M.n_in; k += gridDim.x * blockDim.x) {
      const int c = cbase[m] + cell_of(M, P.V[M.vert_base + k], lev[m]);
      if (cnt[c] > CELL_SORT_MAX) crowded[m] = 1;
      tmp[end[c] - cnt[c] + atomicAdd(&fill[c], 1)] = M.vert_base + k;
    }
  }
}

// the points of each cell by id (insertion sort; crowded cells are skipped)
__global__ void k_cell_sort(int ncell, const int* end, const int* cnt, int* tmp) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int c = gt; c < ncell; c += gs) {
    const int n = cnt[c];
    if (n < 2 || n > CELL_SORT_MAX) continue;
    int* a = tmp + (end[c] - n);
    for (int i = 1; i < n; ++i) {
      const int x = a[i];
      int j = i - 1;
      while (j >= 0 && a[j] > x) {
        a[j + 1] = a[j];
        --j;
      }
      a[j + 1] = x;
    }
  }
}

__global__ void k_cell_put(Pool P, const int* cbase, const int* end, const int* cnt, const int* tmp,
                           const int* crowded) {
  for (int m = blockIdx.y; m < P.n_mesh; m += gridDim.y) {
    const MeshInfo& M = P.mi[m];
    if (crowded[m]) continue;
    const int first = end[cbase[m]] - cnt[cbase[m]];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M.n_in; k += gridDim.x * blockDim.x)
      P.pts[M.pts_base + k] = tmp[first + k];
  }
}

// input vertices where two segments meet at less than 60 degrees
__global__ void k_apex(Pool P) {
  for (int m = blockIdx.y; m < P.n_mesh; m += gridDim.y) {
    MeshInfo& M = P.mi[m];
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < M.n_in; l += gridDim.x * blockDim.x) {
      const int v = M.vert_base + l;
      P.apex[v] = 0;
      const int a0 = P.adj_off[M.adj_base + l], a1 = P.adj_off[M.adj_base + l + 1];
      for (int i = a0; i < a1 && !P.apex[v]; ++i)
        for (int j = i + 1; j < a1; ++j)
          if (small_pair(P, P.adj[i], P.adj[j])) { P.apex[v] = 1; M.has_apex = 1; break; }
    }
  }
}

__global__ void k_iota(int* a, int n) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int k = gt; k < n; k += gs) a[k] = k;
}

__global__ void k_set_loc(Pool P, const int* ids, int n, int t) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  const double2 org = P.mi[P.T[t].w >> 4].org;
  for (int k = gt; k < n; k += gs) {
    P.pts[k] = ids[k];
    P.loc[ids[k]] = t;
    P.Vf[ids[k]] = to_f(P.V[ids[k]], org);
  }
}

// Capacity growth: mesh m's triangles, vertices and links copied from the old
// pool O into the new layout Q (new bases in nb: x = triangle, y = vertex),
// every triangle and vertex id rebased; flags, dirty bits and priority buckets
// move with their slots.  Mesh-local slot order is unchanged, so the
// refinement continues exactly as it would have without the move.
__global__ void k_regrow(Pool Q, Pool O, const int2* nb) {
  for (int m = blockIdx.y; m < O.n_mesh; m += gridDim.y) {
    const MeshInfo& M = O.mi[m];
    const int ot = M.tri_base, ov = M.vert_base, qt = nb[m].x, qv = nb[m].y;
    const int dv = qv - ov, dt = qt - ot;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    for (int t = gt; t < M.tri_count; t += gs) {
      const int4 T4 = O.T[ot + t];
      const int4 N4 = O.N[ot + t];
      Q.T[qt + t] = T4.w < 0 ? T4 : make_int4(T4.x + dv, T4.y + dv, T4.z + dv, T4.w);
      int r[3] = {N4.x, N4.y, N4.z};
      for (int e = 0; e < 3; ++e)
        if (r[e] >= 0) r[e] = (((r[e] >> 2) + dt) << 2) | (r[e] & 3);
      Q.N[qt + t] = make_int4(r[0], r[1], r[2], N4.w);
      Q.dirty[qt + t] = O.dirty[ot + t];
      Q.flag[qt + t] = O.flag[ot + t];
      Q.cbucket[qt + t] = O.cbucket[ot + t];
    }
    for (int v = gt; v < M.vert_count; v += gs) {
      Q.V[qv + v] = O.V[ov + v];
      Q.Vf[qv + v] = O.Vf[ov + v];
      Q.vseg[qv + v] = O.vseg[ov + v];
      const int tv = O.vtri[ov + v];
      Q.vtri[qv + v] = tv >= 0 ? tv + dt : -1;
      const int lc = O.loc[ov + v];
      Q.loc[qv + v] = lc >= 0 ? lc + dt : -1;
      Q.apex[qv + v] = O.apex[ov + v];
    }
    // input segments hold vertex ids: rebase them in place (one thread per segment)
    for (int g = gt; g < M.n_seg; g += gs) {
      const int2 sg = O.seg[M.seg_base + g];
      Q.seg[M.seg_base + g] = make_int2(sg.x + dv, sg.y + dv);
    }
  }
}

// meshes taken out of the refinement (status set by the host): their flagged
// elements would keep producing candidates, so their flags are cleared
__global__ void k_drop_inactive(Pool P) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  for (int t = gt; t < P.n_slots; t += gs) {
    const int w = P.T[t].w;
    if (w >= 0 && !P.mi[w >> 4].active) P.flag[t] = 0;
  }
}

#define CK(x)                                                                         \
  do {                                                                                \
    cudaError_t e_ = (x);                                                             \
    if (e_ != cudaSuccess) {                                                          \
      if (std::getenv("GDP_DEBUG"))                                                   \
        std::fprintf(stderr, "gdp: %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return GDP_ERR_CUDA;                                                            \
    }                                                                                 \
  } while (0)

// every kernel launch of the library goes through LAUNCH: it is counted and,
// when profiling is on, bracketed by CUDA events on the launching stream
#define LAUNCH(h, kern, grid, ...)                                   \
  do {                                                               \
    (h).prof_begin(#kern);                                           \
    kern<<<(grid), BS, 0, (h).stream>>>(__VA_ARGS__);                \
    (h).prof_end();                                                  \
  } while (0)
// per-candidate kernels: small blocks over a wide grid, so that a few
// thousand latency-bound threads land on every SM instead of a few blocks
// (h).bs_cand threads per block (tunable), 1024 threads per SM in all
#define LAUNCH_C(h, kern, ...)                                       \
  do {                                                               \
    (h).prof_begin(#kern);                                           \
    kern<<<(h).Gc, (h).bs_cand, 0, (h).stream>>>(__VA_ARGS__);       \
    (h).prof_end();                                                  \
  } while (0)

// explicit launch shape (the spill-lane kernels: one thread per lane)
#define LAUNCH_B(h, kern, grid, block, ...)                          \
  do {                                                               \
    (h).prof_begin(#kern);                                           \
    kern<<<(grid), (block), 0, (h).stream>>>(__VA_ARGS__);           \
    (h).prof_end();                                                  \
  } while (0)
// candidate cavities (refinement: after the pre-pass k_pre): own slots,
// then the two spill tiers
// (above warp_max candidates: a group of lanes per candidate, or one thread
// per candidate with GDP_GROW_GROUP=0)
#define LAUNCH_GROW_PAIR(h, MODE, P, timed)                          \
  do {                                                               \
    if (MODE == 0) LAUNCH_B(h, k_pre, (h).n_sm * 16, 128, P, timed); \
    LAUNCH_B(h, k_grow_w<MODE>, (h).n_sm * 16, 128, P, timed);       \
    if ((h).grow_group == 2 && MODE == 0)                            \
      LAUNCH_B(h, k_grow_b, (h).n_sm * 16, 128, P, timed);           \
    else if ((h).grow_group)                                         \
      LAUNCH_B(h, k_grow_g<MODE>, (h).n_sm * 16, 128, P, timed);     \
    else                                                             \
      LAUNCH_C(h, k_grow_t<MODE>, P, timed);                         \
  } while (0)
#define LAUNCH_GROW(h, MODE, P)                                      \
  do {                                                               \
    LAUNCH_GROW_PAIR(h, MODE, P, 0);                                 \
    LAUNCH_B(h, k_grow_big<MODE>, LANES_A / 4, 128, P, 0);           \
    LAUNCH_B(h, k_grow_big<MODE>, LANES_B / 4, 128, P, 1);                 \
  } while (0)

double env_double(const char* name, double def) {
  const char* s = std::getenv(name);
  return s ? std::atof(s) : def;
}

}  // namespace

static void print_diag(const char* where) {
  if (!std::getenv("GDP_TRACE")) return;
  unsigned long long d[16];
  cudaDeviceSynchronize();
  if (cudaMemcpyFromSymbol(d, g_diag, sizeof(d)) != cudaSuccess) return;
  std::fprintf(stderr,
               "[%s] orient_exact %llu incircle_exact %llu (inexact diffs %llu, max %llu cyc) sos %llu "
               "dot_exact %llu | max walk steps %llu, max walk cyc %llu, max grow cyc %llu\n",
               where, d[0], d[1], d[4], d[8], d[2], d[3], d[5], d[7], d[6]);
  std::fprintf(stderr, "[%s] calls orient %llu incircle %llu dot %llu; past the FP32 filter: orient %llu incircle %llu dot %llu\n",
               where, d[9], d[10], d[11], d[12], d[13], d[14]);
  unsigned long long z[16] = {};
  cudaMemcpyToSymbol(g_diag, z, sizeof(z));
}

// stage-by-stage consistency report (GDP_TRACE)
static void trace_check(const Pool& P, cudaStream_t st, int G, const char* where) {
  if (!std::getenv("GDP_TRACE")) return;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 10 * sizeof(unsigned long long)) != cudaSuccess) return;
  cudaMemsetAsync(d, 0, 10 * sizeof(unsigned long long), st);
  k_check<<<G, BS, 0, st>>>(P, d);
  unsigned long long c[10] = {};
  cudaMemcpyAsync(c, d, sizeof(c), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  cudaFree(d);
  std::fprintf(stderr, "[check %s] not_mutual %llu edge_mismatch %llu flag_mismatch %llu not_ccw %llu open %llu\n",
               where, c[0], c[1], c[2], c[3], c[4]);
  for (unsigned long long k = 0; k < c[5] && k < 4; ++k) {
    const int t = (int)(c[6 + k] >> 2), e = (int)(c[6 + k] & 3);
    int4 T4, N4, T2, N2;
    cudaMemcpy(&T4, P.T + t, sizeof(int4), cudaMemcpyDeviceToHost);
    cudaMemcpy(&N4, P.N + t, sizeof(int4), cudaMemcpyDeviceToHost);
    const int r = e == 0 ? N4.x : (e == 1 ? N4.y : N4.z);
    cudaMemcpy(&T2, P.T + (r >> 2), sizeof(int4), cudaMemcpyDeviceToHost);
    cudaMemcpy(&N2, P.N + (r >> 2), sizeof(int4), cudaMemcpyDeviceToHost);
    std::fprintf(stderr, "  bad link t=%d e=%d T=(%d %d %d w=%x) N=(%d:%d %d:%d %d:%d) -> t2=%d e2=%d T2=(%d %d %d w=%x) N2=(%d:%d %d:%d %d:%d)\n",
                 t, e, T4.x, T4.y, T4.z, T4.w, N4.x >> 2, N4.x & 3, N4.y >> 2, N4.y & 3, N4.z >> 2, N4.z & 3,
                 r >> 2, r & 3, T2.x, T2.y, T2.z, T2.w, N2.x >> 2, N2.x & 3, N2.y >> 2, N2.y & 3, N2.z >> 2, N2.z & 3);
  }
}

// ---------------------------------------------------------------- memory
// Device buffers come from one stream-ordered memory pool per device that the
// library owns and never trims: a mesh's buffers are allocated and freed in
// stream order (no device-wide synchronisation on free), and later meshes
// reuse the same memory instead of going back to the driver.  The control
// blocks read by the host every round are pinned and recycled the same way.
namespace {
std::mutex g_mem_lock;
cudaMemPool_t g_pools[64] = {};
std::vector<Ctrl*> g_ctrl_free;

cudaMemPool_t device_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> g(g_mem_lock);
  if (!g_pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    unsigned long long keep = ~0ull;   // keep freed memory for reuse
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = p;
  }
  return g_pools[dev];
}

Ctrl* ctrl_get() {
  {
    std::lock_guard<std::mutex> g(g_mem_lock);
    if (!g_ctrl_free.empty()) {
      Ctrl* c = g_ctrl_free.back();
      g_ctrl_free.pop_back();
      return c;
    }
  }
  Ctrl* c = nullptr;
  if (cudaMallocHost(&c, sizeof(Ctrl)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return c;
}

void ctrl_put(Ctrl* c) {
  if (!c) return;
  std::lock_guard<std::mutex> g(g_mem_lock);
  g_ctrl_free.push_back(c);
}
}  // namespace

// ---------------------------------------------------------------- the pool
struct PoolHost {
  cudaStream_t stream = nullptr;
  int n_sm = 0, G = 0, Gc = 0;
  Pool P{};
  std::vector<MeshInfo> hmi;
  std::vector<int2> hseg;         // input segments, global vertex ids
  int n_mesh = 0;
  long long tot_in = 0, tot_seg = 0, pts_cap = 0;
  Ctrl* hctrl = nullptr;          // pinned
  std::vector<void*> allocs;
  gdp_stats stats{};
  // construction rounds replayed from CUDA graphs, each captured for the
  // pool layout it was recorded with (key) and a variant tag
  struct Cached {
    cudaGraphExec_t g = nullptr;
    Pool key{};
    int tag = -1;
    int kernels = 0;
  };
  Cached g_bw, g_split[2], g_flip, g_refine;
  bool capturing = false;
  int cdt_round = 0;              // last construction round used (device keys)
  int32_t* flA = nullptr;         // flip lists (construction only)
  int32_t* flB = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // per-kernel timing (profiling mode) and launch counting
  bool prof = false;
  long long launches = 0;
  struct Pending { const char* name; cudaEvent_t a, b; };
  std::vector<Pending> pend;
  std::vector<std::pair<std::string, std::pair<double, long long>>> ktimes;
  const char* cur_name = nullptr;
  cudaEvent_t cur_ev = nullptr;

  void prof_begin(const char* name) {
    ++launches;
    if (!prof) return;
    cur_name = name;
    cudaEventCreate(&cur_ev);
    cudaEventRecord(cur_ev, stream);
  }
  void prof_end() {
    if (!prof) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, stream);
    pend.push_back({cur_name, cur_ev, e});
  }
  void prof_flush() {
    if (pend.empty()) return;
    cudaStreamSynchronize(stream);
    for (auto& p : pend) {
      float ms = 0;
      cudaEventElapsedTime(&ms, p.a, p.b);
      bool found = false;
      for (auto& kv : ktimes)
        if (kv.first == p.name) { kv.second.first += ms; kv.second.second += 1; found = true; break; }
      if (!found) ktimes.push_back({p.name, {ms, 1}});
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    pend.clear();
  }

  ~PoolHost() {
    prof_flush();
    for (cudaEvent_t e : tg) cudaEventDestroy(e);
    if (split_graph) cudaGraphExecDestroy(split_graph);
    for (Cached* c : {&g_bw, &g_split[0], &g_split[1], &g_flip, &g_refine})
      if (c->g) cudaGraphExecDestroy(c->g);
    for (void* p : allocs) cudaFreeAsync(p, stream);
    if (!allocs.empty()) cudaStreamSynchronize(stream);   // hctrl may still be written
    ctrl_put(hctrl);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  }

  template <class X>
  int alloc(X** p, size_t n, int fill = 0) {
    void* q = nullptr;
    cudaMemPool_t mp = device_pool();
    if (!mp || cudaMallocFromPoolAsync(&q, std::max<size_t>(n, 1) * sizeof(X), mp, stream) != cudaSuccess) {
      cudaGetLastError();
      return GDP_ERR_NOMEM;
    }
    allocs.push_back(q);
    *p = reinterpret_cast<X*>(q);
    // fill < 0: scratch that every reader finds written first (no memset)
    if (fill >= 0 && cudaMemsetAsync(q, fill, std::max<size_t>(n, 1) * sizeof(X), stream) != cudaSuccess)
      return GDP_ERR_CUDA;
    return GDP_OK;
  }
  void release(void* p) {
    auto it = std::find(allocs.begin(), allocs.end(), p);
    if (it != allocs.end()) {
      cudaFreeAsync(p, stream);
      allocs.erase(it);
    }
  }

  bool err_reported = false;
  int sync_ctrl() {
    CK(cudaMemcpyAsync(hctrl, P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (hctrl->err && !err_reported && std::getenv("GDP_TRACE")) {
      std::fprintf(stderr, "[gdp] device error %d, first failing check site %d\n", hctrl->err, hctrl->dbg);
      err_reported = true;
    }
    return GDP_OK;
  }
  int pull_mi() {
    CK(cudaMemcpyAsync(hmi.data(), P.mi, sizeof(MeshInfo) * n_mesh, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    return GDP_OK;
  }
  int push_mi() {
    CK(cudaMemcpyAsync(P.mi, hmi.data(), sizeof(MeshInfo) * n_mesh, cudaMemcpyHostToDevice, stream));
    return GDP_OK;
  }
  int set_ctrl_field(size_t off, int v) {
    CK(cudaMemcpyAsync(reinterpret_cast<char*>(P.ctrl) + off, &v, sizeof(int), cudaMemcpyHostToDevice,
                       stream));
    CK(cudaStreamSynchronize(stream));
    return GDP_OK;
  }

  int setup(const double* xy, const long long* pt_off, const int32_t* seg, const long long* seg_off,
            int nm, bool on_device, void* s);
  int build_cdt();
  int spatial_order();
  bool cdt_done = false;          // build_cdt ran to the end (mesh statuses are final)
  int insert_rounds(int stop_cons, int* rounds_out, bool split);
  int launch_cdt_round(const Pool& Q, int stop_cons);
  int launch_split_round(const Pool& Q);
  int launch_split_kernels(const Pool& Q);
  int build_split_graph(cudaGraphExec_t* out);
  cudaGraphExec_t split_graph = nullptr;   // captured for split_key
  Pool split_key{};
  int launch_flip_passes();
  Pool flip_pool(bool a_to_b) const {
    Pool Q = P;
    Q.fl_cur = a_to_b ? flA : flB;
    Q.fl_nxt = a_to_b ? flB : flA;
    return Q;
  }
  // replays c, capturing body() first when the pool layout or tag changed
  template <class F>
  int replay(Cached& c, int tag, F&& body) {
    if (!c.g || c.tag != tag || std::memcmp(&c.key, &P, sizeof(Pool)) != 0) {
      if (c.g) cudaGraphExecDestroy(c.g);
      c.g = nullptr;
      cudaStream_t cs;
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaStream_t saved = stream;
      const long long saved_launches = launches;
      stream = cs;
      int st = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess ? GDP_OK
                                                                                           : GDP_ERR_CUDA;
      capturing = true;
      if (st == GDP_OK) st = body();
      capturing = false;
      c.kernels = (int)(launches - saved_launches);
      launches = saved_launches;
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(cs, &g);
      stream = saved;
      if (st == GDP_OK && e == cudaSuccess && cudaGraphInstantiate(&c.g, g, 0) != cudaSuccess) {
        c.g = nullptr;
        st = GDP_ERR_CUDA;
      }
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cs);
      if (st != GDP_OK || e != cudaSuccess || !c.g) {
        cudaGetLastError();
        return GDP_ERR_CUDA;
      }
      c.key = P;
      c.tag = tag;
    }
    CK(cudaGraphLaunch(c.g, stream));
    launches += c.kernels;
    return GDP_OK;
  }
  int refine(const double* B, const gdp_refine_opts* o);
  // capacity growth (refinement): meshes that asked for more slots get twice
  // their Steiner capacity in a new pool layout, at most grow_limit times
  int grow_meshes();
  int grow_steps = 0, grow_limit = 20;
  // Flip-Flop insertion (GDP_REFINE_FLIPFLOP): its arrays, sized for the pool
  bool ff_ready = false;
  int32_t *ffA = nullptr, *ffB = nullptr;   // the pass lists
  int ff_alloc();
  void ff_free();
  int ff_iteration();
  int launch_iteration(int k);
  dim3 mesh_grid = dim3(1, 1);    // per-mesh kernels: (blocks per mesh, meshes)
  int bs_cand = 64;               // per-candidate kernels: threads per block
  int grow_group = 2;   // above warp_max candidates: 2 k_grow_b (refinement), 1 k_grow_g, 0 k_grow_t
  bool capped = false;            // some mesh has a per-iteration candidate cap
  void set_cand_block(int b) {
    bs_cand = (b == 32 || b == 128 || b == 256) ? b : 64;
    Gc = n_sm * (1024 / bs_cand);
  }
  // GDP_REFINE_TIME_GROW: an event pair around the first growth launch of each replay
  bool time_grow = false;
  std::vector<cudaEvent_t> tg;
  int add_grow_times(int iters);
  int export_mesh(int m, double* xy, int64_t cap_pts, int32_t* tri, int64_t cap_tri, int32_t* sub,
                  int64_t cap_seg, int64_t* n_pts, int64_t* n_tri, int64_t* n_seg);
};

int PoolHost::setup(const double* xy, const long long* pt_off, const int32_t* seg,
                    const long long* seg_off, int nm, bool on_device, void* s) {
  stream = reinterpret_cast<cudaStream_t>(s);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return GDP_ERR_CUDA; }
  CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  G = 4 * n_sm;
  set_cand_block(64);
  prof = std::getenv("GDP_PROFILE") != nullptr;
  grow_group = (int)env_double("GDP_GROW_GROUP", 2.0);
  if (grow_group < 0 || grow_group > 2) grow_group = 1;
  grow_limit = (int)env_double("GDP_GROW_LIMIT", 20.0);
  if (!(hctrl = ctrl_get())) return GDP_ERR_NOMEM;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  n_mesh = nm;
  hmi.assign(nm, MeshInfo{});
  const double fp = env_double("GDP_STEINER_PER_POINT", 3.0);
  const double fs = env_double("GDP_STEINER_PER_SEGMENT", 64.0);
  long long tb = 0, vb = 0, sb = 0, ab = 0, pb = 0;
  for (int m = 0; m < nm; ++m) {
    const long long n_in = pt_off[m + 1] - pt_off[m];
    const long long n_seg = seg_off[m + 1] - seg_off[m];
    if (n_in < 3 || n_seg < 0) return GDP_ERR_INPUT;
    const long long steiner_cap = (long long)(fp * n_in + fs * n_seg) + 1024;
    const long long vcap = n_in + N_AUX + steiner_cap;
    const long long tcap = 2 * vcap + 16;
    MeshInfo& M = hmi[m];
    M.tri_base = (int)tb; M.tri_cap = (int)tcap;
    M.vert_base = (int)vb; M.vert_cap = (int)vcap;
    M.n_in = (int)n_in; M.seg_base = (int)sb; M.n_seg = (int)n_seg;
    M.adj_base = (int)ab; M.pts_base = (int)pb;
    M.status = S_OK; M.active = 0; M.first_cand = M.last_cand = -1;
    tb += tcap; vb += vcap; sb += n_seg; ab += n_in + 1; pb += n_in + 4;
    if (tb >= (1ll << 29) || vb >= (1ll << 31) - 1) return GDP_ERR_NOMEM;
  }
  tot_in = pb - 4 * nm;
  tot_seg = sb;
  P.n_mesh = nm;
  P.n_slots = (int)tb;
  P.n_verts = (int)vb;
  P.cap_cand = (int)std::min<long long>(std::max<long long>(tb / 4, 65536), 1 << 23);
  P.warp_max = (int)env_double("GDP_WARP_GROW_MAX", WARP_GROW_MAX);
  P.no_prepass = env_double("GDP_PREPASS", 1) == 0 ? 1 : 0;
  int st;
#define AL(ptr, n, fill) \
  if ((st = alloc(&(ptr), (size_t)(n), fill)) != GDP_OK) return st;
  AL(P.V, vb, 0);
  AL(P.Vf, vb, 0);
  AL(P.vseg, vb, 0xff);
  AL(P.vtri, vb, 0xff);
  AL(P.apex, vb, 0);
  AL(P.T, tb, 0xff);
  AL(P.N, tb, 0xff);
  AL(P.mark, tb, 0);
  AL(P.pmark, tb, 0);
  AL(P.newref, 4 * tb, 0xff);
  AL(P.dirty, tb, 0);
  AL(P.flag, tb, 0);
  AL(P.cbucket, tb, 0);
  AL(P.cap_hist, (size_t)nm * CAP_BUCKETS, 0);
  AL(P.cap_thr, nm, 0);
  AL(P.mi, nm, 0);
  AL(P.seg, sb, 0);
  AL(P.adj_off, ab + 1, 0);
  AL(P.adj, 2 * sb, 0);
  const size_t C = (size_t)P.cap_cand;
  AL(P.c_elem, C, 0); AL(P.c_loc, C, 0); AL(P.c_vid, C, 0); AL(P.c_mesh, C, 0);
  AL(P.c_vseg, C, 0); AL(P.c_sub, C, 0); AL(P.c_pt, C, 0); AL(P.c_ptf, C, 0); AL(P.c_key, C, 0);
  // cavity lists, boundary records and set-ups are written by the growth
  // kernels before any kernel reads them (only the counts start at zero)
  AL(P.c_ncav, C, 0); AL(P.c_nbnd, C, 0); AL(P.c_cav, C * CMAX, -1); AL(P.c_bnd, C * BMAX, -1);
  AL(P.c_big, C, 0xff); AL(P.big_cav, BIG_ENTRIES, -1); AL(P.big_bnd, BIG_ENTRIES, -1);
  AL(P.c_setup, C, -1); AL(P.c_pre, C * PRE_MAX, -1); AL(P.c_npre, C, 0);
  AL(P.big_hash, BIG_HASH, 0xff); AL(P.big_val, BIG_HASH, 0xff); AL(P.lane, LANES_A + LANES_B, 0x7f);
  AL(P.c_state, C, 0); AL(P.c_final, C, 0); AL(P.c_extra, C, 0); AL(P.c_offT, C, 0);
  AL(P.c_offV, C, 0); AL(P.c_base, C, 0);
  AL(P.blk, 2 * G, 0);
  AL(P.ctrl, 1, 0);
  AL(P.pts, pb, 0);
  AL(P.pts2, pb, 0);
  pts_cap = pb;
  AL(P.loc, vb, 0xff);
  AL(P.tbest, tb, 0);
  CK(cudaMemcpyAsync(P.mi, hmi.data(), sizeof(MeshInfo) * nm, cudaMemcpyHostToDevice, stream));
  // inputs
  double2* sxy = nullptr;
  int2* sseg = nullptr;
  long long *dpo = nullptr, *dso = nullptr;
  int* seg_mesh = nullptr;
  AL(sxy, tot_in, 0);
  AL(sseg, std::max<long long>(tot_seg, 1), 0);
  AL(dpo, nm + 1, 0);
  AL(dso, nm + 1, 0);
  AL(seg_mesh, std::max<long long>(tot_seg, 1), 0);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(sxy, xy, sizeof(double2) * tot_in, kind, stream));
  if (tot_seg) CK(cudaMemcpyAsync(sseg, seg, sizeof(int2) * tot_seg, kind, stream));
  CK(cudaMemcpyAsync(dpo, pt_off, sizeof(long long) * (nm + 1), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(dso, seg_off, sizeof(long long) * (nm + 1), cudaMemcpyHostToDevice, stream));
  {
    long long mx = 3;
    for (int m = 0; m < nm; ++m) mx = std::max<long long>(mx, hmi[m].n_in);
    const int bx = (int)std::min<long long>(64, std::max<long long>(1, (mx + 4095) / 4096));
    mesh_grid = dim3(bx, std::min(nm, 65535));
  }
  LAUNCH(*this, k_scatter_points, mesh_grid, P, sxy, dpo);
  LAUNCH(*this, k_scatter_segs, nm, P, sseg, dso, seg_mesh);
  if (tot_seg) {
    LAUNCH(*this, k_adj_count, G, P, seg_mesh, (int)tot_seg, P.adj_off);
    LAUNCH(*this, k_iscan_count, G, P.adj_off, (int)(ab + 1), P.blk);
    LAUNCH(*this, k_iscan_write, G, P.adj_off, (int)(ab + 1), P.blk);
    int* cursor = nullptr;
    AL(cursor, ab + 1, 0);
    CK(cudaMemcpyAsync(cursor, P.adj_off, sizeof(int) * (ab + 1), cudaMemcpyDeviceToDevice, stream));
    LAUNCH(*this, k_adj_fill, G, P, seg_mesh, (int)tot_seg, cursor);
    LAUNCH(*this, k_apex, mesh_grid, P);
    CK(cudaStreamSynchronize(stream));
    release(cursor);
  }
  CK(cudaGetLastError());
  hseg.resize(tot_seg);
  if (tot_seg)
    CK(cudaMemcpyAsync(hseg.data(), P.seg, sizeof(int2) * tot_seg, cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  release(sxy);
  release(sseg);
  release(dpo);
  release(dso);
  release(seg_mesh);
#undef AL
  return GDP_OK;
}

// One parallel insertion round of the pending points in Q.pts (the initial
// CDT of Algorithm 1 is built from them; the fixed-batch test hook inserts extra
// points the same way): locate, one point per triangle, cavities, marks,
// dependence, re-triangulation, and the points left go to Q.pts2.
int PoolHost::launch_cdt_round(const Pool& Q, int stop_cons) {
  CK(cudaMemsetAsync(&Q.ctrl->n_ins, 0, 2 * sizeof(unsigned long long), stream));
  LAUNCH(*this, k_clear_marks, G, Q);
  LAUNCH(*this, k_cdt_locate, G, Q, stop_cons, 0);
  LAUNCH(*this, k_cdt_pick_count, G, Q);
  LAUNCH(*this, k_cdt_pick_write, G, Q);
  LAUNCH_GROW(*this, 1, Q);
  LAUNCH_C(*this, k_survive, Q);
  LAUNCH(*this, k_depend, G, Q);
  LAUNCH(*this, k_offsets, G, Q);
  LAUNCH_B(*this, k_insert_w<1>, n_sm * 16, 128, Q);
  LAUNCH_C(*this, k_insert_t<1>, Q);
  LAUNCH_C(*this, k_link<1>, Q);
  LAUNCH(*this, k_cdt_keep_count, G, Q);
  LAUNCH(*this, k_cdt_keep_write, G, Q);
  LAUNCH_B(*this, k_cdt_next, 1, 1, Q);
  CK(cudaGetLastError());
  return GDP_OK;
}

constexpr int CDT_GRAPH_ROUNDS = 8;   // even: the pending list is back in P.pts after a launch
constexpr int CDT_FLIP_PASSES = 6;    // even: the flip list is back in flA after a launch

int PoolHost::launch_flip_passes() {
  for (int k = 0; k < CDT_FLIP_PASSES; ++k) {
    const Pool Q = flip_pool((k & 1) == 0);
    LAUNCH(*this, k_flip_propose, G, Q);
    LAUNCH(*this, k_flip_do, G, Q);
    LAUNCH(*this, k_flip_link, G, Q);
    LAUNCH_B(*this, k_fl_next, 1, 1, Q);
  }
  LAUNCH_B(*this, k_flip_tail, 1, FLIP_TAIL_THREADS, flip_pool(true));
  CK(cudaGetLastError());
  return GDP_OK;
}

// one split round on the pending points in Q.pts (the points left go to
// Q.pts2), then flip passes; the split triangles are listed in flA
int PoolHost::launch_split_kernels(const Pool& Q) {
  Pool S = Q;
  S.fl_nxt = flA;
  LAUNCH_B(*this, k_round_begin, 1, 1, S);
  LAUNCH(*this, k_cdt_locate, G, S, 0, 1);
  LAUNCH(*this, k_cdt_pick_count, G, S);
  LAUNCH(*this, k_cdt_pick_write, G, S);
  LAUNCH(*this, k_split_prep, G, S);
  LAUNCH(*this, k_offsets, G, S);
  LAUNCH_C(*this, k_split, S);
  LAUNCH_C(*this, k_split_link, S);
  LAUNCH(*this, k_cdt_keep_count, G, S);
  LAUNCH(*this, k_cdt_keep_write, G, S);
  LAUNCH_B(*this, k_cdt_next, 1, 1, S);
  LAUNCH_B(*this, k_fl_next, 1, 1, S);
  CK(cudaGetLastError());
  return GDP_OK;
}

int PoolHost::launch_split_round(const Pool& Q) {
  const int st = launch_split_kernels(Q);
  return st != GDP_OK ? st : launch_flip_passes();
}

// The split rounds as one CUDA graph with device-side loops (conditional
// WHILE nodes), so that the host waits once for the whole phase:
//   while (points pending and some triangle took one) {
//     split round (pts -> pts2); while (flip list) { two flip passes }
//     split round (pts2 -> pts); while (flip list) { two flip passes }
//   }
// The pending list is back in P.pts after every iteration.
int PoolHost::build_split_graph(cudaGraphExec_t* out) {
  *out = nullptr;
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaStream_t cs = nullptr, cs2 = nullptr;
  cudaStream_t saved = stream;
  const long long saved_launches = launches;
  int st = GDP_OK;
  auto fail = [&](int code) {
    if (st == GDP_OK) st = code;
  };
  auto add_while = [&](cudaGraph_t parent, cudaGraphConditionalHandle h, const cudaGraphNode_t* deps,
                       const cudaGraphEdgeData* ed, size_t nd, cudaGraphNode_t* node) -> cudaGraph_t {
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(node, parent, deps, ed, nd, &cp) != cudaSuccess) {
      fail(GDP_ERR_CUDA);
      return nullptr;
    }
    return cp.conditional.phGraph_out[0];
  };
  cudaGraphConditionalHandle hr;
  cudaGraphNode_t wr;
  cudaGraph_t body = nullptr;
  if (cudaGraphConditionalHandleCreate(&hr, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) fail(GDP_ERR_CUDA);
  if (st == GDP_OK) body = add_while(g, hr, nullptr, nullptr, 0, &wr);
  if (st == GDP_OK && (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking) != cudaSuccess))
    fail(GDP_ERR_CUDA);
  if (st == GDP_OK &&
      cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    fail(GDP_ERR_CUDA);
  if (st == GDP_OK) {
    capturing = true;
    stream = cs;
    Pool Q = P;
    std::swap(Q.pts, Q.pts2);
    for (int half = 0; half < 2 && st == GDP_OK; ++half) {
      st = launch_split_kernels(half ? Q : P);
      if (st != GDP_OK) break;
      cudaStreamCaptureStatus cst;
      cudaGraph_t cg = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      const cudaGraphEdgeData* ed = nullptr;
      size_t nd = 0;
      cudaGraphConditionalHandle hf;
      if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, &ed, &nd) != cudaSuccess ||
          cudaGraphConditionalHandleCreate(&hf, cg, 0, 0) != cudaSuccess) {
        fail(GDP_ERR_CUDA);
        break;
      }
      LAUNCH_B(*this, k_flip_cond, 1, 1, P, hf);
      if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, &ed, &nd) != cudaSuccess) {
        fail(GDP_ERR_CUDA);
        break;
      }
      cudaGraphNode_t wf;
      cudaGraph_t fbody = add_while(cg, hf, deps, ed, nd, &wf);
      if (st != GDP_OK ||
          cudaStreamUpdateCaptureDependencies(cs, &wf, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess) {
        fail(GDP_ERR_CUDA);
        break;
      }
      // the flip loop's body: two passes (the list ends in flA again), the
      // single-block tail for a short list, and the condition
      stream = cs2;
      if (cudaStreamBeginCaptureToGraph(cs2, fbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
          cudaSuccess) {
        stream = cs;
        fail(GDP_ERR_CUDA);
        break;
      }
      for (int k = 0; k < 2; ++k) {
        const Pool F = flip_pool(k == 0);
        LAUNCH(*this, k_flip_propose, G, F);
        LAUNCH(*this, k_flip_do, G, F);
        LAUNCH(*this, k_flip_link, G, F);
        LAUNCH_B(*this, k_fl_next, 1, 1, F);
      }
      LAUNCH_B(*this, k_flip_tail, 1, FLIP_TAIL_THREADS, flip_pool(true));
      LAUNCH_B(*this, k_flip_cond, 1, 1, P, hf);
      if (cudaStreamEndCapture(cs2, &fbody) != cudaSuccess) fail(GDP_ERR_CUDA);
      stream = cs;
    }
    LAUNCH_B(*this, k_round_cond, 1, 1, P, hr);
    if (cudaGetLastError() != cudaSuccess) fail(GDP_ERR_CUDA);
    if (cudaStreamEndCapture(cs, &body) != cudaSuccess) fail(GDP_ERR_CUDA);
    capturing = false;
  }
  stream = saved;
  launches = saved_launches;
  if (st == GDP_OK && cudaGraphInstantiate(out, g, 0) != cudaSuccess) {
    *out = nullptr;
    fail(GDP_ERR_CUDA);
  }
  cudaGetLastError();
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  if (cs2) cudaStreamDestroy(cs2);
  return st;
}

// Rounds until every pending point is in.  With split, the rounds first
// split triangles and flip (points strictly inside a triangle), and the
// cavity rounds take whatever is left (points on edges).  Rounds run from
// CUDA graphs (empty rounds and passes after the last point cost only their
// launches), one at a time when kernels are timed or traced.  The round
// number lives on the device and keeps counting across calls, so
// per-triangle pick keys left by earlier rounds always compare lower.
int PoolHost::insert_rounds(int stop_cons, int* rounds_out, bool split) {
  if (cdt_round + 4096 / 2 >= 4095) {   // round numbers have 12 bits in the pick keys
    CK(cudaMemsetAsync(P.tbest, 0, sizeof(unsigned long long) * (size_t)P.n_slots, stream));
    cdt_round = 0;
  }
  if (set_ctrl_field(offsetof(Ctrl, round), cdt_round + 1) != GDP_OK) return GDP_ERR_CUDA;
  if (sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
  const int first = hctrl->round;
  const bool trace = std::getenv("GDP_TRACE") != nullptr;
  const bool use_graph = !prof && !trace;
  int last = hctrl->n_pts, stall = 0;
  if (split && hctrl->n_pts > 0) {
    if (set_ctrl_field(offsetof(Ctrl, n_fl), 0) != GDP_OK ||
        set_ctrl_field(offsetof(Ctrl, n_fl_next), 0) != GDP_OK ||
        set_ctrl_field(offsetof(Ctrl, step), 1) != GDP_OK)
      return GDP_ERR_CUDA;
    int parity = 0;
    if (use_graph) {
      if (!split_graph || std::memcmp(&split_key, &P, sizeof(Pool)) != 0) {
        if (split_graph) cudaGraphExecDestroy(split_graph);
        split_graph = nullptr;
        const int st = build_split_graph(&split_graph);
        if (st != GDP_OK) return st;
        split_key = P;
      }
      if (set_ctrl_field(offsetof(Ctrl, guard_r), 0) != GDP_OK ||
          set_ctrl_field(offsetof(Ctrl, guard_f), 0) != GDP_OK)
        return GDP_ERR_CUDA;
      CK(cudaGraphLaunch(split_graph, stream));
      if (sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
      if (hctrl->err) return hctrl->err;
      // kernels run: 27 per round pair, 10 per flip loop iteration
      launches += 27LL * (hctrl->guard_r + 1) + 10LL * hctrl->guard_f;
      last = hctrl->n_pts;
    }
    while (!use_graph && hctrl->n_pts > 0) {
      Pool Q = P;
      if (parity) std::swap(Q.pts, Q.pts2);
      int st;
      if (use_graph) st = replay(g_split[parity], 0, [&] { return launch_split_round(Q); });
      else st = launch_split_round(Q);
      if (st != GDP_OK) return st;
      parity ^= 1;
      if (sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
      for (int guard = 0; hctrl->n_fl > 0 && !hctrl->err; ++guard) {
        if (guard > 4096) return GDP_ERR_INTERNAL;
        st = use_graph ? replay(g_flip, 0, [&] { return launch_flip_passes(); }) : launch_flip_passes();
        if (st != GDP_OK) return st;
        if (sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
      }
      if (trace)
        std::fprintf(stderr, "split round %d: pending %d cand %d inserted %llu flip passes %d\n",
                     hctrl->round - first, last, hctrl->n_cand, hctrl->n_ins, hctrl->step);
      if (hctrl->err) return hctrl->err;
      if (hctrl->round - first >= 4096 / 2 - CDT_GRAPH_ROUNDS) return GDP_ERR_INTERNAL;
      if (hctrl->n_cand == 0) break;   // the points left lie on edges
      stall = hctrl->n_pts == last ? stall + 1 : 0;
      if (stall > 64) return GDP_ERR_INTERNAL;
      last = hctrl->n_pts;
    }
    if (parity) std::swap(P.pts, P.pts2);
    // the cavity rounds start from clean marks and an empty candidate list
    CK(cudaMemsetAsync(P.mark, 0, sizeof(unsigned long long) * (size_t)P.n_slots, stream));
    CK(cudaMemsetAsync(P.pmark, 0, sizeof(unsigned long long) * (size_t)P.n_slots, stream));
    if (set_ctrl_field(offsetof(Ctrl, prev_cand), 0) != GDP_OK) return GDP_ERR_CUDA;
    if (sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
  }
  Pool Q = P;   // the odd rounds read pts2 and write pts
  std::swap(Q.pts, Q.pts2);
  int host_rounds = 0;
  stall = 0;
  while (hctrl->n_pts > 0) {
    int st;
    if (use_graph) {
      st = replay(g_bw, stop_cons, [&] {
        for (int k = 0; k < CDT_GRAPH_ROUNDS / 2; ++k) {
          int r = launch_cdt_round(P, stop_cons);
          if (r == GDP_OK) r = launch_cdt_round(Q, stop_cons);
          if (r != GDP_OK) return r;
        }
        return (int)GDP_OK;
      });
    } else {
      st = launch_cdt_round((host_rounds & 1) ? Q : P, stop_cons);
      ++host_rounds;
    }
    if (st != GDP_OK) return st;
    if (sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
    if (trace)
      std::fprintf(stderr, "round %d: pending %d cand %d marks-ok %llu inserted %llu\n",
                   hctrl->round - first, last, hctrl->n_cand, hctrl->n_surv, hctrl->n_ins);
    if (hctrl->err) return hctrl->err;
    if (hctrl->round - first >= 4096 / 2 - CDT_GRAPH_ROUNDS) return GDP_ERR_INTERNAL;
    if (hctrl->n_pts == last) {
      if (++stall > (use_graph ? 8 : 64)) return GDP_ERR_INTERNAL;
    } else {
      stall = 0;
    }
    last = hctrl->n_pts;
  }
  cdt_round = hctrl->round;
  if (rounds_out) *rounds_out = hctrl->round - first;
  return GDP_OK;
}

// the pending points of every mesh in cell (Morton) order, see k_cell_count
int PoolHost::spatial_order() {
  std::vector<int> lev(n_mesh), cbase(n_mesh + 1, 0);
  for (int m = 0; m < n_mesh; ++m) {
    int L = 0;   // 4^L >= n_in / 2: about two points per cell
    while (L < 15 && (1ll << (2 * L)) * 2 < (long long)hmi[m].n_in) ++L;
    lev[m] = L;
    cbase[m + 1] = cbase[m] + (1 << (2 * L));
  }
  const int ncell = cbase[n_mesh];
  int *d_lev = nullptr, *d_cbase = nullptr, *cnt = nullptr, *end = nullptr, *fill = nullptr, *tmp = nullptr,
      *crowded = nullptr;
  int st;
  if ((st = alloc(&d_lev, n_mesh)) != GDP_OK || (st = alloc(&d_cbase, n_mesh + 1)) != GDP_OK ||
      (st = alloc(&cnt, ncell, 0)) != GDP_OK || (st = alloc(&end, ncell, -1)) != GDP_OK ||
      (st = alloc(&fill, ncell, 0)) != GDP_OK || (st = alloc(&tmp, std::max<long long>(tot_in, 1), -1)) != GDP_OK ||
      (st = alloc(&crowded, n_mesh, 0)) != GDP_OK)
    return st;
  CK(cudaMemcpyAsync(d_lev, lev.data(), sizeof(int) * n_mesh, cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(d_cbase, cbase.data(), sizeof(int) * (n_mesh + 1), cudaMemcpyHostToDevice, stream));
  LAUNCH(*this, k_cell_count, mesh_grid, P, d_cbase, d_lev, cnt);
  CK(cudaMemcpyAsync(end, cnt, sizeof(int) * ncell, cudaMemcpyDeviceToDevice, stream));
  LAUNCH(*this, k_iscan_count, G, end, ncell, P.blk);
  LAUNCH(*this, k_iscan_write, G, end, ncell, P.blk);
  LAUNCH(*this, k_cell_scatter, mesh_grid, P, d_cbase, d_lev, end, cnt, fill, tmp, crowded);
  LAUNCH(*this, k_cell_sort, G, ncell, end, cnt, tmp);
  LAUNCH(*this, k_cell_put, mesh_grid, P, d_cbase, end, cnt, tmp, crowded);
  CK(cudaGetLastError());
  for (void* q : {(void*)d_lev, (void*)d_cbase, (void*)cnt, (void*)end, (void*)fill, (void*)tmp, (void*)crowded})
    release(q);
  return GDP_OK;
}

int PoolHost::build_cdt() {
  CK(cudaEventRecord(ev0, stream));
  double* part = nullptr;
  {
    const int st0 = alloc(&part, 4 * (size_t)mesh_grid.x * n_mesh);
    if (st0 != GDP_OK) return st0;
  }
  LAUNCH(*this, k_cdt_bbox, mesh_grid, P, part);
  LAUNCH(*this, k_cdt_init, n_mesh, P, part, (int)mesh_grid.x, env_double("GDP_FRAME_MARGIN", 16.0));
  LAUNCH(*this, k_cdt_vf, mesh_grid, P);
  release(part);
  if (env_double("GDP_SPATIAL_ORDER", 1) != 0) {
    const int so = spatial_order();
    if (so != GDP_OK) return so;
  }
  CK(cudaGetLastError());
  std::memset(hctrl, 0, sizeof(Ctrl));
  hctrl->n_pts = (int)(tot_in + 4 * n_mesh);
  CK(cudaMemcpyAsync(P.ctrl, hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, stream));
  int rounds = 0;
  int st;
  if ((st = alloc(&P.tstamp, (size_t)P.n_slots)) != GDP_OK) return st;
  if ((st = alloc(&P.lstamp, (size_t)P.n_slots)) != GDP_OK) return st;
  if ((st = alloc(&P.fprop, (size_t)P.n_slots)) != GDP_OK) return st;
  if ((st = alloc(&flA, (size_t)P.n_slots)) != GDP_OK) return st;
  if ((st = alloc(&flB, (size_t)P.n_slots)) != GDP_OK) return st;
  st = insert_rounds(0, &rounds, true);
  if (st != GDP_OK) return st;
  release(P.tstamp);
  release(P.lstamp);
  release(P.fprop);
  release(flA);
  release(flB);
  P.tstamp = P.lstamp = P.fprop = nullptr;
  flA = flB = nullptr;
  LAUNCH(*this, k_vtri, G, P);
  stats.cdt_rounds = rounds;
  trace_check(P, stream, G, "points");
  // segment recovery: short segments with a small work space per segment,
  // then the few long ones (e.g. boundary edges crossed by every point of the
  // outer layer) with a large one
  int st2;
  int* segq2 = nullptr;
  if ((st2 = alloc(&P.segq, std::max<long long>(tot_seg, 1))) != GDP_OK) return st2;
  if ((st2 = alloc(&segq2, std::max<long long>(tot_seg, 1))) != GDP_OK) return st2;
  if ((st2 = alloc(&P.segmark, (size_t)P.n_slots)) != GDP_OK) return st2;
  // three tiers of per-segment work space: all segments at once with room for
  // 64 crossed edges, then up to 16384 segments with 1024, then 8 with 32768
  constexpr int NT = 3;
  SegWork W[NT];
  const int kcap[NT] = {64, 1024, 1 << 15};
  const int lcap[NT] = {(int)std::max<long long>(tot_seg, 1),
                        (int)std::min<long long>(std::max<long long>(tot_seg, 1), 16384), 8};
  for (int tier = 0; tier < NT; ++tier) {
    const size_t n = lcap[tier], K = kcap[tier];
    W[tier].kcap = (int)K;
    if ((st2 = alloc(&W[tier].R, n * (K + 1))) != GDP_OK) return st2;
    if ((st2 = alloc(&W[tier].U, n * (K + 2))) != GDP_OK) return st2;
    if ((st2 = alloc(&W[tier].L, n * (K + 2))) != GDP_OK) return st2;
    if ((st2 = alloc(&W[tier].UR, n * (K + 2))) != GDP_OK) return st2;
    if ((st2 = alloc(&W[tier].LR, n * (K + 2))) != GDP_OK) return st2;
    if ((st2 = alloc(&W[tier].ST, n * (K + 2))) != GDP_OK) return st2;
    if ((st2 = alloc(&W[tier].NR, 2 * n * (K + 2))) != GDP_OK) return st2;
    if ((st2 = alloc(&W[tier].state, n)) != GDP_OK) return st2;
  }
  if (tot_seg) {
    LAUNCH(*this, k_iota, G, P.segq, (int)tot_seg);
    int n = (int)tot_seg, tier = 0, round = 0, stall = 0;
    while (n > 0) {
      SegWork w = W[tier];
      w.list = P.segq;
      w.n_list = std::min(n, lcap[tier]);
      if (std::getenv("GDP_SEG_SERIAL")) w.n_list = 1;
      LAUNCH(*this, k_seg_find, G, P, w, round);
      LAUNCH(*this, k_seg_apply, G, P, w, round);
      LAUNCH(*this, k_seg_keep_count, G, P, w, n);
      LAUNCH(*this, k_seg_keep_write, G, P, w, n, segq2);
      CK(cudaGetLastError());
      std::swap(P.segq, segq2);
      if (sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
      if (hctrl->err) return hctrl->err;
      const int n2 = hctrl->n_segs;
      if (std::getenv("GDP_TRACE")) {
        std::fprintf(stderr, "seg round %d tier %d: %d -> %d (tier-handled pending %d)\n", round, tier, n, n2,
                     hctrl->changed);
        trace_check(P, stream, G, "segment round");
      }
      if (hctrl->changed == 0 && n2 > 0) {
        // only segments too long for this tier are left
        if (++tier == NT) return GDP_ERR_CAPACITY;
      }
      stall = (n2 == n) ? stall + 1 : 0;
      if (stall > 64 || ++round > 60000) return GDP_ERR_INTERNAL;
      n = n2;
    }
  }
  for (int tier = 0; tier < NT; ++tier) {
    release(W[tier].R);
    release(W[tier].U);
    release(W[tier].L);
    release(W[tier].UR);
    release(W[tier].LR);
    release(W[tier].ST);
    release(W[tier].NR);
    release(W[tier].state);
  }
  release(segq2);
  // exterior
  if ((st2 = alloc(&P.ext, (size_t)P.n_slots)) != GDP_OK) return st2;
  if ((st2 = alloc(&P.remap, (size_t)P.n_slots + 1)) != GDP_OK) return st2;
  LAUNCH(*this, k_ext_init, G, P);
  for (int it = 0;; ++it) {
    if (set_ctrl_field(offsetof(Ctrl, changed), 0) != GDP_OK) return GDP_ERR_CUDA;
    LAUNCH(*this, k_ext_step, G, P);
    CK(cudaGetLastError());
    if (sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
    if (!hctrl->changed) break;
    if (it > 100000) return GDP_ERR_INTERNAL;
  }
  int4 *T2 = nullptr, *N2 = nullptr;
  if ((st2 = alloc(&T2, (size_t)P.n_slots, 0xff)) != GDP_OK) return st2;
  if ((st2 = alloc(&N2, (size_t)P.n_slots, 0xff)) != GDP_OK) return st2;
  LAUNCH(*this, k_live_count, G, P);
  LAUNCH(*this, k_live_write, G, P);
  LAUNCH(*this, k_compact_move, G, P, T2, N2);
  LAUNCH(*this, k_compact_finish, G, P, T2, N2);
  LAUNCH(*this, k_compact_counts, G, P);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ev1, stream));
  CK(cudaStreamSynchronize(stream));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, ev0, ev1));
  stats.cdt_ms = ms;
  release(T2);
  release(N2);
  release(P.segq);
  release(P.segmark);
  release(P.ext);
  release(P.remap);
  P.segq = P.remap = nullptr;
  P.segmark = nullptr;
  P.ext = nullptr;
  if (pull_mi() != GDP_OK) return GDP_ERR_CUDA;
  // marks and the candidate list start empty
  if (set_ctrl_field(offsetof(Ctrl, prev_cand), 0) != GDP_OK) return GDP_ERR_CUDA;
  stats.n_in_pts = tot_in;
  cdt_done = true;
  print_diag("cdt");
  int worst = GDP_OK;
  for (auto& M : hmi)
    if (M.status != S_OK && worst == GDP_OK) worst = M.status;
  return worst;
}

// one refinement iteration; k = its position in the graph (event pair)
int PoolHost::launch_iteration(int k) {
  LAUNCH(*this, k_scan_eval, G, P);
  LAUNCH(*this, k_scan_count, G, P, capped ? 1 : 0);
  if (capped) {
    LAUNCH(*this, k_cap_select, G, P);
    LAUNCH(*this, k_cap_count, G, P);
  }
  LAUNCH(*this, k_scan_write, G, P, capped ? 1 : 0);
  // the first iteration of each replay is timed (events in the graph stall
  // the pipeline, so not every one): its growth work is counted apart
  const unsigned rec = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  const int timed = (time_grow && k == 0) ? 1 : 0;
  if (timed) CK(cudaEventRecordWithFlags(tg[0], stream, rec));
  LAUNCH_GROW_PAIR(*this, 0, P, timed);
  if (timed) CK(cudaEventRecordWithFlags(tg[1], stream, rec));
  LAUNCH_B(*this, k_grow_big<0>, LANES_A / 4, 128, P, 0);
  LAUNCH_B(*this, k_grow_big<0>, LANES_B / 4, 128, P, 1);
  LAUNCH_C(*this, k_survive, P);
  LAUNCH(*this, k_depend, G, P);
  LAUNCH(*this, k_offsets, G, P);
  LAUNCH_B(*this, k_insert_w<0>, n_sm * 16, 128, P);
  if (grow_group) LAUNCH_B(*this, k_insert_g<0>, n_sm * 16, 128, P);
  else LAUNCH_C(*this, k_insert_t<0>, P);
  LAUNCH_C(*this, k_link<0>, P);
  return cudaGetLastError() == cudaSuccess ? GDP_OK : GDP_ERR_CUDA;
}

// after a synchronised replay: the timed growth launch's device time
int PoolHost::add_grow_times(int iters) {
  if (!time_grow || iters <= 0) return GDP_OK;
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, tg[0], tg[1]));
  stats.grow_ms += ms;
  stats.grow_launches += 1;
  return GDP_OK;
}

// ---------------------------------------------------------------- Flip-Flop insertion
void PoolHost::ff_free() {
  for (void* q : {(void*)P.tstamp, (void*)P.lstamp, (void*)P.fprop, (void*)P.fop, (void*)ffA, (void*)ffB,
                  (void*)P.ffmark, (void*)P.vkey, (void*)P.vred, (void*)P.vmap})
    if (q) release(q);
  P.tstamp = P.lstamp = P.fprop = P.fop = nullptr;
  ffA = ffB = nullptr;
  P.ffmark = P.vkey = nullptr;
  P.vred = P.vmap = nullptr;
  ff_ready = false;
}

int PoolHost::ff_alloc() {
  if (ff_ready) return GDP_OK;
  int st;
  const size_t T = (size_t)P.n_slots, V = (size_t)P.n_verts;
  if ((st = alloc(&P.tstamp, T)) != GDP_OK || (st = alloc(&P.lstamp, T)) != GDP_OK ||
      (st = alloc(&P.fprop, T)) != GDP_OK || (st = alloc(&P.fop, T)) != GDP_OK ||
      (st = alloc(&ffA, T)) != GDP_OK || (st = alloc(&ffB, T)) != GDP_OK ||
      (st = alloc(&P.ffmark, T)) != GDP_OK || (st = alloc(&P.vkey, V)) != GDP_OK ||
      (st = alloc(&P.vred, V)) != GDP_OK || (st = alloc(&P.vmap, V)) != GDP_OK) {
    ff_free();
    return st;
  }
  ff_ready = true;
  return GDP_OK;
}

// One iteration of Algorithm 1 with Flip-Flop insertion: the scan and the
// cavity filter as in launch_iteration, then every survivor split in, then
// passes of flips and flops until no edge is locally non-Delaunay and no
// point of this iteration is redundant, then the removed points compacted
// away.  Host-driven: the control block is read every four passes.
int PoolHost::ff_iteration() {
  const bool trace = std::getenv("GDP_TRACE") != nullptr;
  LAUNCH(*this, k_scan_eval, G, P);
  LAUNCH(*this, k_scan_count, G, P, capped ? 1 : 0);
  if (capped) {
    LAUNCH(*this, k_cap_select, G, P);
    LAUNCH(*this, k_cap_count, G, P);
  }
  LAUNCH(*this, k_scan_write, G, P, capped ? 1 : 0);
  LAUNCH_GROW_PAIR(*this, 0, P, 0);
  LAUNCH_B(*this, k_grow_big<0>, LANES_A / 4, 128, P, 0);
  LAUNCH_B(*this, k_grow_big<0>, LANES_B / 4, 128, P, 1);
  LAUNCH_C(*this, k_survive, P);
  LAUNCH(*this, k_ff_prep, G, P, trace ? 1 : 0);
  LAUNCH(*this, k_offsets, G, P);
  int32_t *cur = ffA, *nxt = ffB;
  Pool Q = P;
  Q.fl_cur = cur;
  Q.fl_nxt = nxt;
  LAUNCH_C(*this, k_ff_split, Q);
  LAUNCH_C(*this, k_ff_split_link, Q);
  LAUNCH_B(*this, k_fl_next, 1, 1, Q);
  std::swap(cur, nxt);
  CK(cudaGetLastError());
  int passes = 0;
  for (int check = 0;; ++check) {
    for (;;) {
      for (int k = 0; k < 4; ++k) {
        Q.fl_cur = cur;
        Q.fl_nxt = nxt;
        LAUNCH(*this, k_ff_propose, G, Q);
        LAUNCH(*this, k_ff_do, G, Q);
        LAUNCH(*this, k_ff_link, G, Q);
        LAUNCH_B(*this, k_fl_next, 1, 1, Q);
        std::swap(cur, nxt);
      }
      passes += 4;
      if (sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
      if (hctrl->err) return GDP_OK;   // the caller reads the error
      if (hctrl->n_fl == 0) break;
      if (trace && passes == 2000) {
        std::fprintf(stderr, "[ff] iteration %llu: list still %d after %d passes\n",
                     (unsigned long long)hctrl->iters, hctrl->n_fl, passes);
        Q.fl_cur = cur;
        LAUNCH_B(*this, k_ff_debug, 1, 1, Q, 12);
        CK(cudaStreamSynchronize(stream));
      }
      if (passes > 100000) {
        if (set_ctrl_field(offsetof(Ctrl, dbg), 4) != GDP_OK) return GDP_ERR_CUDA;
        return set_ctrl_field(offsetof(Ctrl, err), S_INTERNAL);
      }
    }
    // no edge left to flip: is any point of this iteration redundant?
    CK(cudaMemsetAsync(&P.ctrl->ff_marked, 0, sizeof(int), stream));
    Q.fl_cur = cur;
    Q.fl_nxt = nxt;
    LAUNCH(*this, k_ff_check, G, Q);
    LAUNCH(*this, k_ff_push_stars, G, Q);
    LAUNCH_B(*this, k_fl_next, 1, 1, Q);
    std::swap(cur, nxt);
    if (sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
    if (hctrl->err) return GDP_OK;
    if (trace)
      std::fprintf(stderr, "[ff] iteration %llu check %d: %d redundant, %d passes, flips %llu flops %llu\n",
                   (unsigned long long)hctrl->iters, check, hctrl->ff_marked, passes,
                   (unsigned long long)hctrl->ff_flips, (unsigned long long)hctrl->ff_flops);
    if (hctrl->ff_marked == 0) break;
    if (check > 10000) {
      if (set_ctrl_field(offsetof(Ctrl, dbg), 5) != GDP_OK) return GDP_ERR_CUDA;
      return set_ctrl_field(offsetof(Ctrl, err), S_INTERNAL);
    }
  }
  const int mb = std::min(n_mesh, 4096);
  LAUNCH_B(*this, k_ff_vmap, mb, FF_CT, P);
  LAUNCH(*this, k_ff_rename, G, P);
  LAUNCH_B(*this, k_ff_move, mb, FF_CT, P);
  return cudaGetLastError() == cudaSuccess ? GDP_OK : GDP_ERR_CUDA;
}

int PoolHost::grow_meshes() {
  if (pull_mi() != GDP_OK) return GDP_ERR_CUDA;
  std::vector<int> need(n_mesh);
  bool any = false;
  for (int m = 0; m < n_mesh; ++m) {
    need[m] = hmi[m].need_grow;
    hmi[m].need_grow = 0;
    any |= need[m] != 0;
  }
  // the new layout: twice the Steiner capacity for every mesh that asked
  std::vector<MeshInfo> nmi = hmi;
  long long tb = 0, vb = 0;
  for (int m = 0; m < n_mesh; ++m) {
    MeshInfo& M = nmi[m];
    if (need[m]) {
      const long long fixed = (long long)M.n_in + N_AUX;
      const long long vcap = fixed + 2 * ((long long)M.vert_cap - fixed);
      M.vert_cap = (int)std::min<long long>(vcap, (1ll << 30));
      M.tri_cap = (int)std::min<long long>(2ll * M.vert_cap + 16, (1ll << 29));
    }
    M.tri_base = (int)tb;
    M.vert_base = (int)vb;
    tb += M.tri_cap;
    vb += M.vert_cap;
  }
  Pool Q = P;
  std::vector<void*> fresh;
  int st = (any && grow_steps < grow_limit && tb < (1ll << 29) && vb < (1ll << 31) - 1) ? GDP_OK : GDP_ERR_NOMEM;
  auto take = [&](auto** ptr, size_t n, int fill) {
    if (st != GDP_OK) return;
    st = alloc(ptr, n, fill);
    if (st == GDP_OK) fresh.push_back((void*)*ptr);
  };
  take(&Q.V, vb, 0); take(&Q.Vf, vb, 0); take(&Q.vseg, vb, 0xff); take(&Q.vtri, vb, 0xff);
  take(&Q.apex, vb, 0); take(&Q.loc, vb, 0xff);
  take(&Q.T, tb, 0xff); take(&Q.N, tb, 0xff); take(&Q.mark, tb, 0); take(&Q.pmark, tb, 0); take(&Q.newref, 4 * (size_t)tb, 0xff);
  take(&Q.dirty, tb, 0); take(&Q.flag, tb, 0); take(&Q.cbucket, tb, 0); take(&Q.tbest, tb, 0);
  int2* nb = nullptr;
  take(&nb, n_mesh, 0);
  if (st != GDP_OK) {
    // no room for a larger pool (or the limit is reached): the meshes whose
    // insertions no longer fit stop with GDP_ERR_NOMEM and stay valid CDTs
    for (void* q : fresh) release(q);
    bool dropped = false;
    for (int m = 0; m < n_mesh; ++m)
      if (need[m] == 2) {
        hmi[m].status = S_NOMEM;
        hmi[m].active = 0;
        dropped = true;
      }
    if (push_mi() != GDP_OK) return GDP_ERR_CUDA;
    if (dropped) LAUNCH(*this, k_drop_inactive, G, P);
    return set_ctrl_field(offsetof(Ctrl, grow), 0);
  }
  std::vector<int2> hb(n_mesh);
  for (int m = 0; m < n_mesh; ++m) hb[m] = make_int2(nmi[m].tri_base, nmi[m].vert_base);
  CK(cudaMemcpyAsync(nb, hb.data(), sizeof(int2) * n_mesh, cudaMemcpyHostToDevice, stream));
  Q.n_slots = (int)tb;
  Q.n_verts = (int)vb;
  int most = 1;
  for (const MeshInfo& M : hmi) most = std::max(most, std::max(M.tri_count, M.vert_count));
  LAUNCH(*this, k_regrow, dim3(std::min(256, (most + 1023) / 1024), std::min(n_mesh, 65535)), Q, P, nb);
  CK(cudaGetLastError());
  for (void* q : {(void*)P.V, (void*)P.Vf, (void*)P.vseg, (void*)P.vtri, (void*)P.apex, (void*)P.loc,
                  (void*)P.T, (void*)P.N, (void*)P.mark, (void*)P.pmark, (void*)P.newref, (void*)P.dirty, (void*)P.flag,
                  (void*)P.cbucket, (void*)P.tbest})
    release(q);
  release(nb);
  P = Q;
  hmi = nmi;
  if (push_mi() != GDP_OK) return GDP_ERR_CUDA;
  if (ff_ready) {   // per-pass scratch only: a fresh set for the new sizes
    ff_free();
    const int fs = ff_alloc();
    if (fs != GDP_OK) return fs;
  }
  // the last iteration's marks were left behind in the old pool
  if (set_ctrl_field(offsetof(Ctrl, prev_cand), 0) != GDP_OK) return GDP_ERR_CUDA;
  if (set_ctrl_field(offsetof(Ctrl, grow), 0) != GDP_OK) return GDP_ERR_CUDA;
  ++grow_steps;
  stats.grow_steps = grow_steps;
  return GDP_OK;
}

int PoolHost::refine(const double* B, const gdp_refine_opts* o) {
  gdp_refine_opts d{};
  if (o) d = *o;
  if (!(d.B > 0)) d.B = std::sqrt(2.0);
  const long long max_iter = d.max_iter > 0 ? d.max_iter : 100000;
  const int giters = d.graph_iters == 0 ? 8 : d.graph_iters;
  if (pull_mi() != GDP_OK) return GDP_ERR_CUDA;
  for (int m = 0; m < n_mesh; ++m) {
    MeshInfo& M = hmi[m];
    const double b = B ? B[m] : d.B;
    if (!(b > 0.7072)) return GDP_ERR_INPUT;
    M.B2 = b * b;
    M.B2f = (float)M.B2;
    M.L2 = (d.max_len > 0 && std::isfinite(d.max_len)) ? d.max_len * d.max_len : 0.0;
    M.active = M.status == S_OK ? 1 : 0;
    M.steiner = 0;
    M.cand_cap = d.cand_cap;
    M.lens = (d.flags & GDP_REFINE_CHEW) ? 1 : 0;
    M.need_grow = 0;
  }
  if (push_mi() != GDP_OK) return GDP_ERR_CUDA;
  const bool ff = (d.flags & GDP_REFINE_FLIPFLOP) != 0;
  if (ff) {
    const int fs = ff_alloc();
    if (fs != GDP_OK) return fs;
    CK(cudaMemsetAsync(P.ffmark, 0, sizeof(unsigned long long) * (size_t)P.n_slots, stream));
    CK(cudaMemsetAsync(P.tstamp, 0, sizeof(int32_t) * (size_t)P.n_slots, stream));
    CK(cudaMemsetAsync(P.lstamp, 0, sizeof(int32_t) * (size_t)P.n_slots, stream));
  }
  std::memset(hctrl, 0, sizeof(Ctrl));
  hctrl->need_eval = 1;   // every triangle is evaluated with this call's bounds
  hctrl->step = 1;        // Flip-Flop passes: slot stamps start at 0, below every pass
  CK(cudaMemcpyAsync(P.ctrl, hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, stream));
  CK(cudaEventRecord(ev0, stream));
  // a call that stopped with candidates (iteration limit, error) leaves their
  // marks behind: the next call starts from clean marks
  CK(cudaMemsetAsync(P.mark, 0, sizeof(unsigned long long) * (size_t)P.n_slots, stream));
  CK(cudaMemsetAsync(P.pmark, 0, sizeof(unsigned long long) * (size_t)P.n_slots, stream));
  LAUNCH(*this, k_mark_all, G, P);
  int status = GDP_OK;
  time_grow = (d.flags & GDP_REFINE_TIME_GROW) != 0;
  capped = d.cand_cap > 0;
  set_cand_block(d.cand_block);
  stats.grow_ms = 0;
  stats.grow_launches = 0;
  if (time_grow) {
    while (tg.size() < 2) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      tg.push_back(e);
    }
  }
  if (ff) {
    for (;;) {
      if (ff_iteration() != GDP_OK) return GDP_ERR_CUDA;
      if (sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
      if (hctrl->err) {
        if (std::getenv("GDP_TRACE"))
          std::fprintf(stderr, "[ff] error %d at check site %d, iteration %llu\n", hctrl->err, hctrl->dbg,
                       (unsigned long long)hctrl->iters);
        status = hctrl->err;
        break;
      }
      if (hctrl->grow) {
        const int g = grow_meshes();
        if (g != GDP_OK) return g;
      }
      if (hctrl->n_cand == 0) break;
      if ((long long)hctrl->iters >= max_iter) { status = GDP_ERR_ITER_LIMIT; break; }
    }
  } else if (giters > 0 && !prof) {
    for (;;) {
      const int tag = ((giters * 2 + (time_grow ? 1 : 0)) * 2 + (capped ? 1 : 0)) * 512 + bs_cand;
      const int st = replay(g_refine, tag, [&] {
        for (int k = 0; k < giters; ++k) {
          const int r = launch_iteration(k);
          if (r != GDP_OK) return r;
        }
        return (int)GDP_OK;
      });
      if (st != GDP_OK) return st;
      if (sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
      if (add_grow_times(giters) != GDP_OK) return GDP_ERR_CUDA;
      if (hctrl->err) { status = hctrl->err; break; }
      if (hctrl->grow) {   // deferred insertions are retried in the next iterations
        const int g = grow_meshes();
        if (g != GDP_OK) return g;
      }
      if (hctrl->n_cand == 0) break;
      if ((long long)hctrl->iters >= max_iter) { status = GDP_ERR_ITER_LIMIT; break; }
    }
  } else {
    // GDP_TRACE_GROW: the running growth-work totals after every iteration
    // (to normalise per-launch profiler counters by the work of that launch)
    const bool trace_grow = std::getenv("GDP_TRACE_GROW") != nullptr;
    for (;;) {
      if (launch_iteration(0) != GDP_OK) return GDP_ERR_CUDA;
      if (sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
      if (trace_grow)
        std::fprintf(stderr, "[grow] iteration %llu grown %llu cavity_tris %llu walk_steps %llu\n",
                     (unsigned long long)hctrl->iters, (unsigned long long)hctrl->n_grown,
                     (unsigned long long)hctrl->sum_cav, (unsigned long long)hctrl->sum_walk);
      if (add_grow_times(1) != GDP_OK) return GDP_ERR_CUDA;
      if (hctrl->err) { status = hctrl->err; break; }
      if (hctrl->grow) {   // deferred insertions are retried in the next iterations
        const int g = grow_meshes();
        if (g != GDP_OK) return g;
      }
      if (hctrl->n_cand == 0) break;
      if ((long long)hctrl->iters >= max_iter) { status = GDP_ERR_ITER_LIMIT; break; }
    }
  }
  CK(cudaEventRecord(ev1, stream));
  // the refined meshes' live triangles and subsegments (after the timed region)
  CK(cudaMemsetAsync(&P.ctrl->live_tri, 0, 2 * sizeof(unsigned long long), stream));
  LAUNCH(*this, k_count_live, mesh_grid, P);
  CK(cudaMemcpyAsync(&hctrl->live_tri, &P.ctrl->live_tri, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                     stream));
  CK(cudaStreamSynchronize(stream));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, ev0, ev1));
  if (pull_mi() != GDP_OK) return GDP_ERR_CUDA;
  stats.refine_ms = ms;
  print_diag("refine");
  stats.iterations = (int64_t)hctrl->iters;
  stats.candidates = (int64_t)hctrl->tot_cand;
  stats.inserted = (int64_t)hctrl->tot_ins;
  stats.grown = (int64_t)hctrl->n_grown;
  stats.cavity_tris = (int64_t)hctrl->sum_cav;
  stats.cavity_edges = (int64_t)hctrl->sum_bnd;
  stats.walk_steps = (int64_t)hctrl->sum_walk;
  stats.timed_grown = (int64_t)hctrl->t_grown;
  stats.timed_cavity_tris = (int64_t)hctrl->t_cav;
  stats.timed_cavity_edges = (int64_t)hctrl->t_bnd;
  stats.timed_walk_steps = (int64_t)hctrl->t_walk;
  stats.setups = (int64_t)hctrl->n_setup;
  stats.timed_setups = (int64_t)hctrl->t_setup;
  stats.flips = (int64_t)hctrl->ff_flips;
  stats.flops = (int64_t)hctrl->ff_flops;
  stats.redundant_removed = (int64_t)hctrl->ff_removed;
  long long st = 0;
  for (auto& M : hmi) {
    st += M.steiner;
    if (M.status != S_OK && status == GDP_OK) status = M.status;
  }
  stats.n_steiner = st;
  stats.n_tris = (int64_t)hctrl->live_tri;
  stats.n_subsegs = (int64_t)hctrl->live_sub;
  return status;
}

// Export ids: input points 0..n_in-1, the auxiliary vertices dropped,
// Steiner points after.  Triangles and subsegments are gathered on the
// device (k_export_count / k_export_write) and copied out once.
int PoolHost::export_mesh(int m, double* xy, int64_t cap_pts, int32_t* tri, int64_t cap_tri,
                          int32_t* sub, int64_t cap_seg, int64_t* n_pts, int64_t* n_tri,
                          int64_t* n_seg) {
  if (m < 0 || m >= n_mesh) return GDP_ERR_INPUT;
  if (pull_mi() != GDP_OK) return GDP_ERR_CUDA;
  const MeshInfo& M = hmi[m];
  LAUNCH(*this, k_export_count, G, P, m);
  std::vector<int> blk(2 * G);
  CK(cudaMemcpyAsync(blk.data(), P.blk, sizeof(int) * 2 * G, cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  long long ntri = 0, nsub = 0;
  for (int b = 0; b < G; ++b) {
    ntri += blk[b];
    nsub += blk[G + b];
  }
  const long long npts = M.vert_count - N_AUX;
  if (n_pts) *n_pts = npts;
  if (n_tri) *n_tri = ntri;
  if (n_seg) *n_seg = nsub;
  if ((xy && cap_pts < npts) || (tri && cap_tri < ntri) || (sub && cap_seg < nsub)) return GDP_ERR_INPUT;
  if (xy) {
    CK(cudaMemcpyAsync(xy, P.V + M.vert_base, sizeof(double2) * M.n_in, cudaMemcpyDeviceToHost, stream));
    const long long rest = M.vert_count - M.n_in - N_AUX;
    if (rest > 0)
      CK(cudaMemcpyAsync(xy + 2 * (size_t)M.n_in, P.V + M.vert_base + M.n_in + N_AUX, sizeof(double2) * rest,
                         cudaMemcpyDeviceToHost, stream));
  }
  if (tri || sub) {
    int *dt = nullptr, *ds = nullptr;
    int st;
    if ((st = alloc(&dt, 3 * (size_t)std::max(ntri, 1LL))) != GDP_OK) return st;
    if ((st = alloc(&ds, 3 * (size_t)std::max(nsub, 1LL))) != GDP_OK) return st;
    LAUNCH(*this, k_export_write, G, P, m, dt, ds);
    CK(cudaGetLastError());
    if (tri && ntri) CK(cudaMemcpyAsync(tri, dt, sizeof(int) * 3 * ntri, cudaMemcpyDeviceToHost, stream));
    if (sub && nsub) CK(cudaMemcpyAsync(sub, ds, sizeof(int) * 3 * nsub, cudaMemcpyDeviceToHost, stream));
    release(dt);
    release(ds);
  }
  CK(cudaStreamSynchronize(stream));
  return GDP_OK;
}

// ---------------------------------------------------------------- C ABI
struct gdp_mesh {
  PoolHost h;
};
struct gdp_batch {
  PoolHost h;
};

static int create_common(PoolHost& h, const double* xy, int64_t n, const int32_t* seg, int64_t m,
                         bool dev, void* s) {
  long long po[2] = {0, (long long)n}, so[2] = {0, (long long)m};
  int st = h.setup(xy, po, seg, so, 1, dev, s);
  if (st != GDP_OK) return st;
  return h.build_cdt();
}

extern "C" {

const char* gdp_status_str(int s) {
  switch (s) {
    case GDP_OK: return "ok";
    case GDP_ERR_INPUT: return "invalid input";
    case GDP_ERR_NOMEM: return "out of memory";
    case GDP_ERR_ITER_LIMIT: return "iteration limit";
    case GDP_ERR_WALK_LIMIT: return "walk limit";
    case GDP_ERR_CUDA: return "CUDA error";
    case GDP_ERR_INTERNAL: return "internal error";
    case GDP_ERR_CAPACITY: return "work buffer capacity";
    default: return "unknown";
  }
}

int gdp_mesh_create(const double* xy, int64_t n_pts, const int32_t* seg, int64_t n_seg,
                    void* stream, gdp_mesh** out) {
  if (!out || !xy || n_pts < 3 || n_seg < 0 || (n_seg > 0 && !seg)) return GDP_ERR_INPUT;
  *out = nullptr;
  gdp_mesh* g = new gdp_mesh();
  const int st = create_common(g->h, xy, n_pts, seg, n_seg, false, stream);
  *out = g;
  return st;
}

int gdp_mesh_create_device(const double* xy, int64_t n_pts, const int32_t* seg, int64_t n_seg,
                           void* stream, gdp_mesh** out) {
  if (!out || !xy || n_pts < 3 || n_seg < 0 || (n_seg > 0 && !seg)) return GDP_ERR_INPUT;
  *out = nullptr;
  gdp_mesh* g = new gdp_mesh();
  const int st = create_common(g->h, xy, n_pts, seg, n_seg, true, stream);
  *out = g;
  return st;
}

int gdp_mesh_refine(gdp_mesh* g, const gdp_refine_opts* opts, gdp_stats* stats) {
  if (!g) return GDP_ERR_INPUT;
  const int st = g->h.refine(nullptr, opts);
  g->h.stats.launches = g->h.launches;
  if (stats) *stats = g->h.stats;
  return st;
}

int gdp_mesh_export(gdp_mesh* g, double* xy, int64_t cap_pts, int32_t* tri, int64_t cap_tri,
                    int32_t* sub, int64_t cap_seg, int64_t* n_pts, int64_t* n_tri, int64_t* n_seg) {
  if (!g) return GDP_ERR_INPUT;
  return g->h.export_mesh(0, xy, cap_pts, tri, cap_tri, sub, cap_seg, n_pts, n_tri, n_seg);
}

int gdp_mesh_stats(gdp_mesh* g, gdp_stats* s) {
  if (!g || !s) return GDP_ERR_INPUT;
  g->h.stats.launches = g->h.launches;
  *s = g->h.stats;
  return GDP_OK;
}

int gdp_mesh_insert_points(gdp_mesh* g, const double* xy, int64_t n) {
  if (!g || (n > 0 && !xy) || n < 0) return GDP_ERR_INPUT;
  if (n == 0) return GDP_OK;
  PoolHost& h = g->h;
  if (h.pull_mi() != GDP_OK) return GDP_ERR_CUDA;
  MeshInfo& M = h.hmi[0];
  if (M.vert_count + n > M.vert_cap || M.tri_count + 2 * n > M.tri_cap) return GDP_ERR_NOMEM;
  if (n > h.pts_cap) {   // grow the pending-point lists
    h.release(h.P.pts);
    h.release(h.P.pts2);
    int s2;
    if ((s2 = h.alloc(&h.P.pts, n)) != GDP_OK || (s2 = h.alloc(&h.P.pts2, n)) != GDP_OK) return s2;
    h.pts_cap = n;
  }
  const int first = M.vert_base + M.vert_count;
  CK(cudaMemcpyAsync(h.P.V + first, xy, sizeof(double2) * n, cudaMemcpyHostToDevice, h.stream));
  std::vector<int> ids(n);
  for (int64_t k = 0; k < n; ++k) ids[k] = first + (int)k;
  int* dids = nullptr;
  int st;
  if ((st = h.alloc(&dids, n)) != GDP_OK) return st;
  CK(cudaMemcpyAsync(dids, ids.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h.stream));
  // a live triangle to start the walks from
  LAUNCH(h, k_set_loc, h.G, h.P, dids, (int)n, M.tri_base);
  M.vert_count += (int)n;
  if (h.push_mi() != GDP_OK) return GDP_ERR_CUDA;
  std::memset(h.hctrl, 0, sizeof(Ctrl));
  h.hctrl->n_pts = (int)n;
  CK(cudaMemcpyAsync(h.P.ctrl, h.hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, h.stream));
  st = h.insert_rounds(1, nullptr, false);
  h.release(dids);
  if (st != GDP_OK) return st;
  if (h.pull_mi() != GDP_OK) return GDP_ERR_CUDA;
  h.hmi[0].steiner += (int)n;
  if (h.push_mi() != GDP_OK) return GDP_ERR_CUDA;
  if (h.set_ctrl_field(offsetof(Ctrl, prev_cand), 0) != GDP_OK) return GDP_ERR_CUDA;
  return GDP_OK;
}

int gdp_mesh_split_subsegments(gdp_mesh* g, const double* abxy, int64_t n) {
  if (!g || n < 0 || (n > 0 && !abxy)) return GDP_ERR_INPUT;
  PoolHost& h = g->h;
  std::vector<char> done(n, 0);
  for (int round = 0; round < 1000; ++round) {
    if (h.pull_mi() != GDP_OK) return GDP_ERR_CUDA;
    const MeshInfo& M = h.hmi[0];
    std::vector<int4> T(M.tri_count);
    std::vector<double2> V(M.vert_count);
    CK(cudaMemcpyAsync(T.data(), h.P.T + M.tri_base, sizeof(int4) * M.tri_count, cudaMemcpyDeviceToHost, h.stream));
    CK(cudaMemcpyAsync(V.data(), h.P.V + M.vert_base, sizeof(double2) * M.vert_count, cudaMemcpyDeviceToHost, h.stream));
    CK(cudaStreamSynchronize(h.stream));
    std::vector<int> elems;
    int left = 0;
    for (int64_t k = 0; k < n; ++k) {
      if (done[k]) continue;
      const double* q = abxy + 4 * k;
      int found = -1;
      for (int t = 0; t < M.tri_count && found < 0; ++t) {
        const int4 T4 = T[t];
        if (T4.w < 0) continue;
        const int vv[3] = {T4.x, T4.y, T4.z};
        for (int e = 0; e < 3; ++e) {
          if (!((T4.w >> e) & 1)) continue;
          const double2 a = V[vv[(e + 1) % 3] - M.vert_base], b = V[vv[(e + 2) % 3] - M.vert_base];
          if ((a.x == q[0] && a.y == q[1] && b.x == q[2] && b.y == q[3]) ||
              (a.x == q[2] && a.y == q[3] && b.x == q[0] && b.y == q[1])) {
            found = ((M.tri_base + t) << 2) | e;
            break;
          }
        }
      }
      if (found < 0) {
        if (round == 0) return GDP_ERR_INPUT;
        done[k] = 1;   // split in an earlier round
        continue;
      }
      ++left;
      elems.push_back(found);
    }
    if (left == 0) break;
    std::sort(elems.begin(), elems.end());
    if ((int)elems.size() > h.P.cap_cand) elems.resize(h.P.cap_cand);
    CK(cudaMemcpyAsync(h.P.c_elem, elems.data(), sizeof(int) * elems.size(), cudaMemcpyHostToDevice, h.stream));
    LAUNCH(h, k_clear_marks, h.G, h.P);
    const int nc = (int)elems.size();
    CK(cudaMemcpyAsync(&h.P.ctrl->n_cand, &nc, sizeof(int), cudaMemcpyHostToDevice, h.stream));
    CK(cudaMemcpyAsync(&h.P.ctrl->prev_cand, &nc, sizeof(int), cudaMemcpyHostToDevice, h.stream));
    for (auto& Mi : h.hmi) Mi.active = 1;
    LAUNCH_GROW(h, 0, h.P);
    LAUNCH_C(h, k_survive, h.P);
    LAUNCH(h, k_depend, h.G, h.P);
    LAUNCH(h, k_offsets, h.G, h.P);
    LAUNCH_B(h, k_insert_w<0>, h.n_sm * 16, 128, h.P);
    if (h.grow_group) LAUNCH_B(h, k_insert_g<0>, h.n_sm * 16, 128, h.P);
    else LAUNCH_C(h, k_insert_t<0>, h.P);
    LAUNCH_C(h, k_link<0>, h.P);
    CK(cudaGetLastError());
    if (h.sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
    if (h.hctrl->err) return h.hctrl->err;
  }
  return GDP_OK;
}

int gdp_mesh_scan(gdp_mesh* g, double B, int32_t* kind, int32_t* verts, double* pt, uint32_t* meas,
                  int64_t cap, int64_t* count) {
  return gdp_mesh_scan_mode(g, B, 0, kind, verts, pt, meas, cap, count);
}

int gdp_mesh_scan_mode(gdp_mesh* g, double B, int32_t flags, int32_t* kind, int32_t* verts, double* pt,
                       uint32_t* meas, int64_t cap, int64_t* count) {
  if (!g || !count || !(B > 0) || (flags & ~GDP_REFINE_CHEW)) return GDP_ERR_INPUT;
  PoolHost& h = g->h;
  if (h.pull_mi() != GDP_OK) return GDP_ERR_CUDA;
  const MeshInfo& M = h.hmi[0];
  const long long c = std::max<long long>(cap, 1);
  int *dk = nullptr, *dv = nullptr, *dc = nullptr;
  double2* dp = nullptr;
  unsigned* dm = nullptr;
  int st;
  if ((st = h.alloc(&dk, c)) || (st = h.alloc(&dv, 3 * c)) || (st = h.alloc(&dp, c)) ||
      (st = h.alloc(&dm, c)) || (st = h.alloc(&dc, 1)))
    return st;
  LAUNCH(h, k_scan_report, h.G, h.P, B * B, (flags & GDP_REFINE_CHEW) ? 1 : 0, dk, dv, dp, dm, (int)cap, dc);
  CK(cudaGetLastError());
  int cnt = 0;
  CK(cudaMemcpyAsync(&cnt, dc, sizeof(int), cudaMemcpyDeviceToHost, h.stream));
  CK(cudaStreamSynchronize(h.stream));
  *count = cnt;
  const long long k = std::min<long long>(cnt, cap);
  std::vector<int32_t> vv(3 * std::max<long long>(k, 1));
  if (kind && k) CK(cudaMemcpy(kind, dk, sizeof(int) * k, cudaMemcpyDeviceToHost));
  if (verts && k) {
    CK(cudaMemcpy(vv.data(), dv, sizeof(int) * 3 * k, cudaMemcpyDeviceToHost));
    for (long long i = 0; i < 3 * k; ++i) {
      const int gv = vv[i];
      if (gv < 0) { verts[i] = -1; continue; }
      const int l = gv - M.vert_base;
      verts[i] = l < M.n_in ? l : l - N_AUX;
    }
  }
  if (pt && k) CK(cudaMemcpy(pt, dp, sizeof(double2) * k, cudaMemcpyDeviceToHost));
  if (meas && k) CK(cudaMemcpy(meas, dm, sizeof(unsigned) * k, cudaMemcpyDeviceToHost));
  h.release(dk);
  h.release(dv);
  h.release(dp);
  h.release(dm);
  h.release(dc);
  return GDP_OK;
}

int gdp_mesh_check(gdp_mesh* g, int64_t counts[5]) {
  if (!g || !counts) return GDP_ERR_INPUT;
  PoolHost& h = g->h;
  unsigned long long* d = nullptr;
  int st;
  if ((st = h.alloc(&d, 5)) != GDP_OK) return st;
  LAUNCH(h, k_check, h.G, h.P, d);
  unsigned long long c[5];
  CK(cudaMemcpyAsync(c, d, sizeof(c), cudaMemcpyDeviceToHost, h.stream));
  CK(cudaStreamSynchronize(h.stream));
  h.release(d);
  for (int i = 0; i < 5; ++i) counts[i] = (int64_t)c[i];
  return GDP_OK;
}

int gdp_mesh_profile(gdp_mesh* g, int enable) {
  if (!g) return GDP_ERR_INPUT;
  g->h.prof_flush();
  g->h.ktimes.clear();
  g->h.prof = enable != 0;
  return GDP_OK;
}

int gdp_mesh_kernel_time(gdp_mesh* g, int32_t i, char* name, int64_t name_cap, double* total_ms,
                         int64_t* count) {
  if (!g) return GDP_ERR_INPUT;
  g->h.prof_flush();
  if (i < 0 || i >= (int32_t)g->h.ktimes.size()) return GDP_ERR_INPUT;
  const auto& kv = g->h.ktimes[i];
  if (name && name_cap > 0) {
    std::strncpy(name, kv.first.c_str(), (size_t)name_cap - 1);
    name[name_cap - 1] = 0;
  }
  if (total_ms) *total_ms = kv.second.first;
  if (count) *count = kv.second.second;
  return GDP_OK;
}

void gdp_mesh_destroy(gdp_mesh* g) { delete g; }

int gdp_batch_create(const double* xy, const int64_t* pt_off, const int32_t* seg,
                     const int64_t* seg_off, int32_t n_meshes, void* stream, gdp_batch** out) {
  if (!out || !xy || !pt_off || !seg_off || n_meshes <= 0) return GDP_ERR_INPUT;
  *out = nullptr;
  std::vector<long long> po(n_meshes + 1), so(n_meshes + 1);
  for (int m = 0; m <= n_meshes; ++m) {
    po[m] = pt_off[m];
    so[m] = seg_off[m];
    if (m && (po[m] - po[m - 1] < 3 || so[m] < so[m - 1])) return GDP_ERR_INPUT;
  }
  if (po[0] != 0 || so[0] != 0 || (so[n_meshes] > 0 && !seg)) return GDP_ERR_INPUT;
  gdp_batch* b = new gdp_batch();
  int st = b->h.setup(xy, po.data(), seg, so.data(), n_meshes, false, stream);
  if (st == GDP_OK) st = b->h.build_cdt();
  *out = b;
  return st;
}

int gdp_batch_refine(gdp_batch* b, const double* B, const gdp_refine_opts* opts, gdp_stats* stats) {
  if (!b) return GDP_ERR_INPUT;
  const int st = b->h.refine(B, opts);
  b->h.stats.launches = b->h.launches;
  if (stats) *stats = b->h.stats;
  return st;
}

int gdp_batch_info(gdp_batch* b, int32_t* status, int64_t* n_pts, int64_t* n_tri, int64_t* n_seg,
                   int64_t* n_steiner) {
  if (!b) return GDP_ERR_INPUT;
  if (b->h.pull_mi() != GDP_OK) return GDP_ERR_CUDA;
  for (int m = 0; m < b->h.n_mesh; ++m) {
    const MeshInfo& M = b->h.hmi[m];
    if (status) status[m] = M.status;
    if (n_pts) n_pts[m] = M.vert_count - N_AUX;
    if (n_tri) n_tri[m] = M.tri_count;
    if (n_seg) n_seg[m] = -1;
    if (n_steiner) n_steiner[m] = M.steiner;
  }
  return GDP_OK;
}

int gdp_batch_export(gdp_batch* b, int32_t mesh, double* xy, int64_t cap_pts, int32_t* tri,
                     int64_t cap_tri, int32_t* sub, int64_t cap_seg, int64_t* n_pts, int64_t* n_tri,
                     int64_t* n_seg) {
  if (!b) return GDP_ERR_INPUT;
  return b->h.export_mesh(mesh, xy, cap_pts, tri, cap_tri, sub, cap_seg, n_pts, n_tri, n_seg);
}

void gdp_batch_destroy(gdp_batch* b) { delete b; }

}  // extern "C"

#include "gdp_server.cuh"
#include "gdp_tune.cuh"
