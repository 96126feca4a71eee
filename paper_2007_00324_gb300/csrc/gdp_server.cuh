// Serving: a resident pool that refines many requests at once and admits new
// ones between refinement replays (continuous batching).  Included at the end
// of gdp.cu (it uses PoolHost).
//
// A step of the loop:
//   1. launch one graph replay of `iters` refinement iterations over every
//      resident mesh (main stream, asynchronous);
//   2. meanwhile build the CDT of waiting requests in staging pools (side
//      stream), as long as a region of the resident pool is free for them;
//   3. wait for the replay; retire the meshes that finished (no candidate in
//      the last iteration and nothing deferred), copy them out and free their
//      regions; move the staged CDTs into their regions (k_relocate) so that
//      they join the next replay.
// A mesh is refined by the same kernels with the same per-mesh keys alone and
// in the mix, so its result does not depend on the other requests.
#pragma once

#include <chrono>
#include <deque>
#include <map>
#include <memory>

// Copy mesh ms of a staging pool S (construction done, compacted) into the
// region of the resident pool D that starts at triangle dt, vertex dv,
// segment ds, adjacency row da, as mesh md.  Triangle and vertex ids, segment
// ids and CSR offsets are rebased; every triangle is marked dirty so that
// the first scan evaluates it.
__global__ void __launch_bounds__(BS) k_relocate(Pool D, Pool S, int ms, int md, int dt, int dv, int ds,
                                                 int da) {
  const MeshInfo& Ms = S.mi[ms];
  const int st = Ms.tri_base, sv0 = Ms.vert_base, ss = Ms.seg_base, sa = Ms.adj_base;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  if (gt == 0) D.ctrl->need_eval = 1;
  for (int t = gt; t < Ms.tri_count; t += gs) {
    const int4 T4 = S.T[st + t];
    const int4 N4 = S.N[st + t];
    const int sh = dv - sv0;
    D.T[dt + t] = make_int4(T4.x + sh, T4.y + sh, T4.z + sh, (md << 4) | (T4.w & 15));
    int r[3] = {N4.x, N4.y, N4.z};
    for (int e = 0; e < 3; ++e)
      if (r[e] >= 0) r[e] = (((r[e] >> 2) - st + dt) << 2) | (r[e] & 3);
    D.N[dt + t] = make_int4(r[0], r[1], r[2], 0);
    D.dirty[dt + t] = 1;
    D.flag[dt + t] = 0;
    D.mark[dt + t] = 0ull;
    D.pmark[dt + t] = 0ull;
  }
  for (int v = gt; v < Ms.vert_count; v += gs) {
    D.V[dv + v] = S.V[sv0 + v];
    D.Vf[dv + v] = S.Vf[sv0 + v];
    const int sg = S.vseg[sv0 + v];
    D.vseg[dv + v] = sg >= 0 ? sg - ss + ds : -1;
    const int tv = S.vtri[sv0 + v];
    D.vtri[dv + v] = tv >= 0 ? tv - st + dt : -1;
    D.apex[dv + v] = S.apex[sv0 + v];
  }
  for (int g = gt; g < Ms.n_seg; g += gs) {
    const int2 sg = S.seg[ss + g];
    D.seg[ds + g] = make_int2(sg.x - sv0 + dv, sg.y - sv0 + dv);
  }
  // the staging CSR is global: this mesh's entries start at 2 * its first segment
  for (int k = gt; k <= Ms.n_in; k += gs) D.adj_off[da + k] = S.adj_off[sa + k] - 2 * ss + 2 * ds;
  for (int j = gt; j < 2 * Ms.n_seg; j += gs) D.adj[2 * ds + j] = S.adj[2 * ss + j] - ss + ds;
}

// first-fit allocator of index ranges (triangle slots, vertices, segments,
// adjacency rows of the resident pool)
class RangeAlloc {
 public:
  void init(long long n) {
    free_.clear();
    if (n > 0) free_[0] = n;
    cap_ = n;
  }
  long long alloc(long long n) {
    if (n <= 0) n = 1;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const long long off = it->first, len = it->second;
      free_.erase(it);
      if (len > n) free_[off + n] = len - n;
      return off;
    }
    return -1;
  }
  void release(long long off, long long n) {
    if (n <= 0) n = 1;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  // end of the highest allocated range
  long long high() const {
    if (free_.empty()) return cap_;
    auto last = std::prev(free_.end());
    return last->first + last->second == cap_ ? last->first : cap_;
  }

 private:
  std::map<long long, long long> free_;
  long long cap_ = 0;
};

struct gdp_server {
  using clock = std::chrono::steady_clock;
  PoolHost h;                      // the resident pool
  cudaStream_t side = nullptr;     // staging CDT builds
  gdp_refine_opts opts{};
  int iters = 8;
  RangeAlloc tri, vert, seg, adj;
  std::vector<int> free_ids;
  clock::time_point t0 = clock::now();
  int64_t next_ticket = 1;

  struct Req {
    int64_t ticket;
    std::vector<double> xy;
    std::vector<int32_t> seg;
    double B;
    double t_submit;
  };
  struct Region {
    long long t, v, s, a;          // offsets
    long long nt, nv, ns, na;      // sizes
  };
  // the CDTs of several waiting requests, built together in one staging pool
  struct Staged {
    std::unique_ptr<PoolHost> S;
    std::vector<Req> r;
    std::vector<Region> g;
    int status = GDP_OK;           // of the whole build (CUDA, internal errors)
  };
  struct Live {
    int64_t ticket;
    Region g;
    double t_submit, t_admit;
    int64_t n_in;
  };
  struct Done {
    gdp_result_info info;
    std::vector<double> xy;
    std::vector<int32_t> tri, sub;
  };
  std::deque<Req> waiting;
  std::vector<Staged> staged;
  std::map<int, Live> live;        // by mesh id
  std::deque<Done> done;

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(clock::now() - t0).count();
  }
};

static void region_sizes(long long n_in, long long n_seg, gdp_server::Region& g) {
  // the capacities PoolHost::setup gives a single mesh
  const double fp = env_double("GDP_STEINER_PER_POINT", 3.0);
  const double fs = env_double("GDP_STEINER_PER_SEGMENT", 64.0);
  const long long steiner_cap = (long long)(fp * n_in + fs * n_seg) + 1024;
  g.nv = n_in + N_AUX + steiner_cap;
  g.nt = 2 * g.nv + 16;
  g.ns = n_seg;
  g.na = n_in + 1;
}

static void region_release(gdp_server* s, const gdp_server::Region& g) {
  s->tri.release(g.t, g.nt);
  s->vert.release(g.v, g.nv);
  if (g.ns > 0) s->seg.release(g.s, g.ns);
  s->adj.release(g.a, g.na);
}

static bool region_alloc(gdp_server* s, gdp_server::Region& g) {
  g.t = s->tri.alloc(g.nt);
  g.v = g.t < 0 ? -1 : s->vert.alloc(g.nv);
  g.s = g.v < 0 ? -1 : (g.ns > 0 ? s->seg.alloc(g.ns) : 0);
  g.a = g.s < 0 ? -1 : s->adj.alloc(g.na);
  if (g.a >= 0) return true;
  if (g.t >= 0) s->tri.release(g.t, g.nt);
  if (g.v >= 0) s->vert.release(g.v, g.nv);
  if (g.s >= 0 && g.ns > 0) s->seg.release(g.s, g.ns);
  return false;
}

// The resident pool: the refinement arrays of PoolHost::setup for the given
// capacities, every mesh entry free.
static int server_setup(gdp_server* s, long long tb, long long vb, long long sb, int nm, void* stream) {
  PoolHost& h = s->h;
  h.stream = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return GDP_ERR_CUDA; }
  CK(cudaDeviceGetAttribute(&h.n_sm, cudaDevAttrMultiProcessorCount, dev));
  h.G = 4 * h.n_sm;
  h.set_cand_block(s->opts.cand_block);
  h.prof = false;
  if (!(h.hctrl = ctrl_get())) return GDP_ERR_NOMEM;
  CK(cudaEventCreate(&h.ev0));
  CK(cudaEventCreate(&h.ev1));
  CK(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
  h.n_mesh = nm;
  h.hmi.assign(nm, MeshInfo{});
  for (auto& M : h.hmi) {
    M.status = S_OK;
    M.first_cand = M.last_cand = -1;
  }
  h.P.n_mesh = nm;
  h.P.n_slots = (int)tb;
  h.P.n_verts = (int)vb;
  h.P.cap_cand = (int)std::min<long long>(std::max<long long>(tb / 4, 65536), 1 << 23);
  h.P.warp_max = (int)env_double("GDP_WARP_GROW_MAX", WARP_GROW_MAX);
  h.P.no_prepass = env_double("GDP_PREPASS", 1) == 0 ? 1 : 0;
  const long long ab = vb + nm;   // adjacency rows: at most one per vertex plus one per mesh
  int st;
#define AL(ptr, n, fill) \
  if ((st = h.alloc(&(ptr), (size_t)(n), fill)) != GDP_OK) return st;
  PoolHost& H = h;
  AL(H.P.V, vb, 0);
  AL(H.P.Vf, vb, 0);
  AL(H.P.vseg, vb, 0xff);
  AL(H.P.vtri, vb, 0xff);
  AL(H.P.apex, vb, 0);
  AL(H.P.T, tb, 0xff);
  AL(H.P.N, tb, 0xff);
  AL(H.P.mark, tb, 0);
  AL(H.P.pmark, tb, 0);
  AL(H.P.newref, 4 * tb, 0xff);
  AL(H.P.dirty, tb, 0);
  AL(H.P.flag, tb, 0);
  AL(H.P.cbucket, tb, 0);
  AL(H.P.cap_hist, (size_t)nm * CAP_BUCKETS, 0);
  AL(H.P.cap_thr, nm, 0);
  AL(H.P.mi, nm, 0);
  AL(H.P.seg, std::max<long long>(sb, 1), 0);
  AL(H.P.adj_off, ab + 1, 0);
  AL(H.P.adj, 2 * std::max<long long>(sb, 1), 0);
  const size_t C = (size_t)H.P.cap_cand;
  AL(H.P.c_elem, C, 0); AL(H.P.c_loc, C, 0); AL(H.P.c_vid, C, 0); AL(H.P.c_mesh, C, 0);
  AL(H.P.c_vseg, C, 0); AL(H.P.c_sub, C, 0); AL(H.P.c_pt, C, 0); AL(H.P.c_ptf, C, 0);
  AL(H.P.c_key, C, 0); AL(H.P.c_ncav, C, 0); AL(H.P.c_nbnd, C, 0);
  AL(H.P.c_cav, C * CMAX, 0); AL(H.P.c_bnd, C * BMAX, 0);
  AL(H.P.c_big, C, 0xff); AL(H.P.big_cav, BIG_ENTRIES, 0); AL(H.P.big_bnd, BIG_ENTRIES, 0);
  AL(H.P.c_setup, C, 0); AL(H.P.c_pre, C * PRE_MAX, 0); AL(H.P.c_npre, C, 0);
  AL(H.P.big_hash, BIG_HASH, 0xff); AL(H.P.big_val, BIG_HASH, 0xff); AL(H.P.lane, LANES_A + LANES_B, 0x7f);
  AL(H.P.c_state, C, 0); AL(H.P.c_final, C, 0); AL(H.P.c_extra, C, 0); AL(H.P.c_offT, C, 0);
  AL(H.P.c_offV, C, 0); AL(H.P.c_base, C, 0);
  AL(H.P.blk, 2 * H.G, 0);
  AL(H.P.ctrl, 1, 0);
#undef AL
  h.hseg.assign((size_t)std::max<long long>(sb, 1), make_int2(0, 0));
  CK(cudaMemcpyAsync(h.P.mi, h.hmi.data(), sizeof(MeshInfo) * nm, cudaMemcpyHostToDevice, h.stream));
  std::memset(h.hctrl, 0, sizeof(Ctrl));
  h.hctrl->scan_hi = 1;   // nothing resident yet
  CK(cudaMemcpyAsync(h.P.ctrl, h.hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, h.stream));
  CK(cudaStreamSynchronize(h.stream));
  s->tri.init(tb);
  s->vert.init(vb);
  s->seg.init(std::max<long long>(sb, 1));
  s->adj.init(ab);
  for (int m = nm - 1; m >= 0; --m) s->free_ids.push_back(m);
  return GDP_OK;
}

// builds, in one staging pool on the side stream, the CDTs of the oldest
// waiting requests that fit in the resident pool (first come, first served;
// at most max_reqs requests or max_pts points per build)
static void server_stage(gdp_server* s, int max_reqs, long long max_pts) {
  gdp_server::Staged st;
  long long pts = 0;
  while (!s->waiting.empty() && (int)st.r.size() < max_reqs && (int)st.r.size() < (int)s->free_ids.size()) {
    gdp_server::Req& r = s->waiting.front();
    const long long n = (long long)r.xy.size() / 2, m = (long long)r.seg.size() / 2;
    if (!st.r.empty() && pts + n > max_pts) break;
    gdp_server::Region g;
    region_sizes(n, m, g);
    if (!region_alloc(s, g)) break;   // wait for room
    pts += n;
    st.g.push_back(g);
    st.r.push_back(std::move(r));
    s->waiting.pop_front();
  }
  if (st.r.empty()) return;
  const int k = (int)st.r.size();
  std::vector<long long> po(k + 1, 0), so(k + 1, 0);
  for (int i = 0; i < k; ++i) {
    po[i + 1] = po[i] + (long long)st.r[i].xy.size() / 2;
    so[i + 1] = so[i] + (long long)st.r[i].seg.size() / 2;
  }
  std::vector<double> xy((size_t)po[k] * 2);
  std::vector<int32_t> sg((size_t)std::max<long long>(so[k], 1) * 2);
  for (int i = 0; i < k; ++i) {
    std::copy(st.r[i].xy.begin(), st.r[i].xy.end(), xy.begin() + 2 * po[i]);
    std::copy(st.r[i].seg.begin(), st.r[i].seg.end(), sg.begin() + 2 * so[i]);
  }
  st.S.reset(new PoolHost());
  int rc = st.S->setup(xy.data(), po.data(), sg.data(), so.data(), k, false, s->side);
  if (rc == GDP_OK) rc = st.S->build_cdt();
  // a build that ran to the end reports per-mesh errors in the mesh statuses
  if (st.S->cdt_done) rc = GDP_OK;
  if (rc == GDP_OK && st.S->pull_mi() != GDP_OK) rc = GDP_ERR_CUDA;
  if (rc == GDP_ERR_INPUT && k > 1) {
    // an invalid input stopped the whole build (e.g. crossing segments):
    // build the requests one by one so that only the invalid ones fail
    st.S.reset();
    for (int i = 0; i < k; ++i) {
      gdp_server::Staged one;
      one.r.push_back(std::move(st.r[i]));
      one.g.push_back(st.g[i]);
      one.S.reset(new PoolHost());
      const gdp_server::Req& q = one.r[0];
      int r1 = create_common(*one.S, q.xy.data(), (long long)q.xy.size() / 2, q.seg.data(),
                             (long long)q.seg.size() / 2, false, s->side);
      if (one.S->cdt_done) r1 = GDP_OK;
      if (r1 == GDP_OK && one.S->pull_mi() != GDP_OK) r1 = GDP_ERR_CUDA;
      one.status = r1;
      s->staged.push_back(std::move(one));
    }
    return;
  }
  st.status = rc;
  s->staged.push_back(std::move(st));
}

static void server_fail(gdp_server* s, const gdp_server::Req& r, const gdp_server::Region& g, int status) {
  gdp_server::Done d{};
  d.info.ticket = r.ticket;
  d.info.status = status;
  d.info.n_in_pts = (int64_t)r.xy.size() / 2;
  d.info.t_submit_ms = r.t_submit;
  d.info.t_admit_ms = d.info.t_done_ms = s->now_ms();
  s->done.push_back(std::move(d));
  region_release(s, g);
}

// staged CDTs into their regions of the resident pool (main stream)
static int server_admit(gdp_server* s) {
  PoolHost& h = s->h;
  for (auto& st : s->staged) {
    for (size_t q = 0; q < st.r.size(); ++q) {
      const gdp_server::Req& r = st.r[q];
      const gdp_server::Region& g = st.g[q];
      if (st.status != GDP_OK) {
        server_fail(s, r, g, st.status);
        continue;
      }
      const MeshInfo& Ms = st.S->hmi[q];
      if (Ms.status != S_OK) {
        server_fail(s, r, g, Ms.status);
        continue;
      }
      const int md = s->free_ids.back();
      s->free_ids.pop_back();
      MeshInfo M = Ms;
      M.tri_base = (int)g.t;
      M.tri_cap = (int)g.nt;
      M.vert_base = (int)g.v;
      M.vert_cap = (int)g.nv;
      M.seg_base = (int)g.s;
      M.adj_base = (int)g.a;
      M.pts_base = 0;
      M.status = S_OK;
      M.active = 1;
      M.B2 = r.B * r.B;
      M.B2f = (float)M.B2;
      M.L2 = (s->opts.max_len > 0 && std::isfinite(s->opts.max_len)) ? s->opts.max_len * s->opts.max_len : 0.0;
      M.steiner = 0;
      M.cand_cap = s->opts.cand_cap;
      M.lens = (s->opts.flags & GDP_REFINE_CHEW) ? 1 : 0;
      M.first_cand = M.last_cand = -1;
      M.pending = 0;
      h.hmi[md] = M;
      for (int k = 0; k < Ms.n_seg; ++k) {
        const int2 e = st.S->hseg[Ms.seg_base + k];
        h.hseg[g.s + k] = make_int2(e.x - Ms.vert_base + (int)g.v, e.y - Ms.vert_base + (int)g.v);
      }
      CK(cudaMemcpyAsync(h.P.mi + md, &h.hmi[md], sizeof(MeshInfo), cudaMemcpyHostToDevice, h.stream));
      LAUNCH(h, k_relocate, h.G, h.P, st.S->P, (int)q, md, (int)g.t, (int)g.v, (int)g.s, (int)g.a);
      CK(cudaGetLastError());
      s->live[md] = gdp_server::Live{r.ticket, g, r.t_submit, s->now_ms(), (int64_t)r.xy.size() / 2};
    }
  }
  if (!s->staged.empty()) {
    // the staging pools are read by k_relocate: free them after it ran
    CK(cudaStreamSynchronize(h.stream));
    s->staged.clear();
  }
  const long long hi = std::max(1LL, s->tri.high());
  if (h.set_ctrl_field(offsetof(Ctrl, scan_hi), (int)hi) != GDP_OK) return GDP_ERR_CUDA;
  return GDP_OK;
}

// finished meshes out of the resident pool
static int server_retire(gdp_server* s) {
  PoolHost& h = s->h;
  if (s->live.empty()) return GDP_OK;
  if (h.pull_mi() != GDP_OK) return GDP_ERR_CUDA;
  std::vector<int> fin;
  for (auto& kv : s->live) {
    const MeshInfo& M = h.hmi[kv.first];
    // a request whose region ran out of slots (need_grow 2) ends with GDP_ERR_NOMEM:
    // resident regions are fixed, so the server does not grow them
    if (M.status != S_OK || M.need_grow == 2 || (M.first_cand < 0 && M.pending == 0)) fin.push_back(kv.first);
  }
  for (int md : fin) {
    gdp_server::Live L = s->live[md];
    gdp_server::Done d{};
    const MeshInfo M = h.hmi[md];
    d.info.ticket = L.ticket;
    d.info.status = (M.status == S_OK && M.need_grow == 2) ? S_NOMEM : M.status;
    d.info.n_in_pts = L.n_in;
    d.info.n_steiner = M.steiner;
    int64_t np = 0, nt = 0, ns = 0;
    int st = h.export_mesh(md, nullptr, 0, nullptr, 0, nullptr, 0, &np, &nt, &ns);
    if (st == GDP_OK) {
      d.xy.resize((size_t)np * 2);
      d.tri.resize((size_t)nt * 3);
      d.sub.resize((size_t)ns * 3);
      st = h.export_mesh(md, d.xy.data(), np, d.tri.data(), nt, d.sub.data(), ns, &np, &nt, &ns);
    }
    if (st != GDP_OK && d.info.status == GDP_OK) d.info.status = st;
    d.info.n_pts = np;
    d.info.n_tri = nt;
    d.info.n_subseg = ns;
    d.info.t_submit_ms = L.t_submit;
    d.info.t_admit_ms = L.t_admit;
    d.info.t_done_ms = s->now_ms();
    // free the region: dead slots, clean flags, a free mesh entry
    CK(cudaMemsetAsync(h.P.T + L.g.t, 0xff, sizeof(int4) * L.g.nt, h.stream));
    CK(cudaMemsetAsync(h.P.N + L.g.t, 0xff, sizeof(int4) * L.g.nt, h.stream));
    CK(cudaMemsetAsync(h.P.dirty + L.g.t, 0, L.g.nt, h.stream));
    CK(cudaMemsetAsync(h.P.flag + L.g.t, 0, L.g.nt, h.stream));
    MeshInfo F{};
    F.status = S_OK;
    F.first_cand = F.last_cand = -1;
    h.hmi[md] = F;
    CK(cudaMemcpyAsync(h.P.mi + md, &h.hmi[md], sizeof(MeshInfo), cudaMemcpyHostToDevice, h.stream));
    region_release(s, L.g);
    s->free_ids.push_back(md);
    s->live.erase(md);
    s->done.push_back(std::move(d));
  }
  if (!fin.empty()) CK(cudaStreamSynchronize(h.stream));
  return GDP_OK;
}

extern "C" {

int gdp_server_create(int64_t tri_slots, int64_t vert_slots, int64_t seg_slots, int32_t max_meshes,
                      const gdp_refine_opts* opts, void* stream, gdp_server** out) {
  if (!out || tri_slots < 64 || vert_slots < 64 || seg_slots < 0 || max_meshes < 1 ||
      tri_slots >= (1ll << 29) || vert_slots >= (1ll << 30) || max_meshes > (1 << 20))
    return GDP_ERR_INPUT;
  *out = nullptr;
  gdp_server* s = new gdp_server();
  if (opts) s->opts = *opts;
  if (!(s->opts.B > 0)) s->opts.B = std::sqrt(2.0);
  s->iters = s->opts.graph_iters > 0 ? s->opts.graph_iters : 8;
  const int st = server_setup(s, tri_slots, vert_slots, seg_slots, max_meshes, stream);
  *out = s;
  return st;
}

int gdp_server_submit(gdp_server* s, const double* xy, int64_t n_pts, const int32_t* seg, int64_t n_seg,
                      double B, int64_t* ticket) {
  if (!s || !xy || n_pts < 3 || n_seg < 0 || (n_seg > 0 && !seg) || !(B > 0.7072)) return GDP_ERR_INPUT;
  gdp_server::Region g;
  region_sizes(n_pts, n_seg, g);
  if (g.nt > s->h.P.n_slots || g.nv > s->h.P.n_verts) return GDP_ERR_NOMEM;   // could never fit
  gdp_server::Req r;
  r.ticket = s->next_ticket++;
  r.xy.assign(xy, xy + 2 * n_pts);
  if (n_seg) r.seg.assign(seg, seg + 2 * n_seg);
  r.B = B;
  r.t_submit = s->now_ms();
  if (ticket) *ticket = r.ticket;
  s->waiting.push_back(std::move(r));
  return GDP_OK;
}

int gdp_server_step(gdp_server* s, int32_t* n_waiting, int32_t* n_live, int32_t* n_done) {
  if (!s) return GDP_ERR_INPUT;
  PoolHost& h = s->h;
  const bool refine = !s->live.empty();
  if (refine) {
    h.time_grow = false;
    h.capped = s->opts.cand_cap > 0;
    const int tag = ((s->iters * 2) * 2 + (h.capped ? 1 : 0)) * 512 + h.bs_cand;
    const int st = h.replay(h.g_refine, tag, [&] {
      for (int k = 0; k < s->iters; ++k) {
        const int r = h.launch_iteration(k);
        if (r != GDP_OK) return r;
      }
      return (int)GDP_OK;
    });
    if (st != GDP_OK) return st;
  }
  // overlaps the replay: one staging build on the side stream
  server_stage(s, 256, 16ll << 20);
  if (refine) {
    if (h.sync_ctrl() != GDP_OK) return GDP_ERR_CUDA;
    if (h.hctrl->err) return h.hctrl->err;
    const int st = server_retire(s);
    if (st != GDP_OK) return st;
  }
  const int st = server_admit(s);
  if (st != GDP_OK) return st;
  if (n_waiting) *n_waiting = (int32_t)s->waiting.size();
  if (n_live) *n_live = (int32_t)s->live.size();
  if (n_done) *n_done = (int32_t)s->done.size();
  return GDP_OK;
}

int gdp_server_result(gdp_server* s, gdp_result_info* info, double* xy, int64_t cap_pts, int32_t* tri,
                      int64_t cap_tri, int32_t* sub, int64_t cap_sub) {
  if (!s || !info) return GDP_ERR_INPUT;
  if (s->done.empty()) return GDP_ERR_INPUT;
  gdp_server::Done& d = s->done.front();
  *info = d.info;
  if (!xy && !tri && !sub) return GDP_OK;   // peek
  if ((xy && cap_pts < d.info.n_pts) || (tri && cap_tri < d.info.n_tri) || (sub && cap_sub < d.info.n_subseg))
    return GDP_ERR_INPUT;
  if (xy) std::memcpy(xy, d.xy.data(), sizeof(double) * d.xy.size());
  if (tri) std::memcpy(tri, d.tri.data(), sizeof(int32_t) * d.tri.size());
  if (sub) std::memcpy(sub, d.sub.data(), sizeof(int32_t) * d.sub.size());
  s->done.pop_front();
  return GDP_OK;
}

void gdp_server_destroy(gdp_server* s) {
  if (!s) return;
  if (s->h.stream) cudaStreamSynchronize(s->h.stream);
  s->staged.clear();
  if (s->side) cudaStreamDestroy(s->side);
  delete s;
}

}  // extern "C"
