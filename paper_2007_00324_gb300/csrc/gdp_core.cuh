// Device-side data layout of the refinement pool (all meshes of a batch share it).
//
// Structure of arrays in HBM, one slot per triangle and per vertex:
//   T[t]   int4  (v0, v1, v2, info)   CCW vertex ids; info = mesh << 4 | cons bits 0..2
//                                     (edge e = (v[e+1], v[e+2]) is a subsegment) | DEAD bit 3
//   N[t]   int4  (n0, n1, n2, -)      neighbour across edge e as (tri << 2 | edge), -1 none
//   mark[t] u64                       cavity priority mark (Sec. 5.2 atomic marks)
//   pmark[t] u64                      the same for the refinement pre-pass (first rings)
//   newref[4t+e] int32                the new triangle that replaced edge e of t (this iteration)
//   dirty[t] u8                       triangle not yet evaluated (construction, relocation)
//   flag[t] u8                        its code: 0 good, 1-3 encroached edge + 1, 4 bad;
//                                     persists until the slot is rewritten
//   V[v]   double2                    vertex coordinates (FP64)
//   vseg[v] int32                     input segment a Steiner vertex lies on, else -1
// Per-candidate scratch (one candidate = one splitting point of Algorithm 1):
//   c_cav[i*CMAX + j]   cavity triangles;  c_bnd[i*BMAX + j]  cavity boundary edges
//   as int4 (u, v, outside ref, inside ref | subsegment << 31).
//   A cavity that outgrows its slot is grown again in a lane of a spill tier
//   (big_cav / big_bnd at offset c_big[i]): LANES_A lanes of CAP_A triangles,
//   then LANES_B lanes of CAP_B = CMAX_BIG; each lane has a hash set of twice
//   its capacity in big_hash (cavity membership while growing; the fan map
//   vertex -> boundary records, with big_val, while inserting).
//   Refinement sets every candidate up in a pre-pass (k_pre): c_setup[i]
//   holds its splitting point, key and start triangles, c_pre[i*PRE_MAX + j]
//   the c_npre[i] triangles of its cavity known before growth (0: the set-up
//   failed), on which it puts its key in pmark[].
#pragma once
#include <cstdint>

namespace gdp {

constexpr int CMAX = 32;            // cavity triangles per splitting point
constexpr int BMAX = CMAX + 2;      // boundary edges per cavity
constexpr int PRE_MAX = 6;          // start triangles + their first ring (pre-pass)
constexpr int CMAX_BIG = 1 << 16;   // largest cavity
constexpr int LANES_A = 4096, CAP_A = 512;       // spill tier A (powers of two)
constexpr int LANES_B = 16, CAP_B = CMAX_BIG;    // spill tier B
constexpr long long BIG_ENTRIES = (long long)LANES_A * (CAP_A + 2) + (long long)LANES_B * (CAP_B + 2);
constexpr long long BIG_HASH = 2ll * LANES_A * CAP_A + 2ll * LANES_B * CAP_B;
constexpr int LANE_FREE = 0x7f7f7f7f;            // byte fill 0x7f
constexpr int CAP_BUCKETS = 1024;   // per-mesh priority histogram (candidate cap)
constexpr int WALK_MAX = 1 << 16;   // point-location steps
constexpr int BS = 256;             // threads per block
constexpr int INFO_DEAD = 8;
constexpr unsigned long long KEY_MID = 1ull << 63;

struct CandSetup;   // a candidate's splitting point, key and start triangles

// candidate states
enum : uint8_t { C_NONE = 0, C_GROWN = 1, C_LOST = 2, C_SURV = 3, C_FAIL = 4 };

// status codes (mirror gdp_status)
enum : int32_t { S_OK = 0, S_INPUT = 1, S_NOMEM = 2, S_ITER = 3, S_WALK = 4, S_CUDA = 5,
                 S_INTERNAL = 6, S_CAPACITY = 7 };

struct MeshInfo {
  int32_t tri_base, tri_cap, tri_count;
  int32_t vert_base, vert_cap, vert_count;
  int32_t n_in;          // input points: vert_base .. vert_base + n_in - 1; 3 enclosing next
  int32_t seg_base, n_seg;
  int32_t adj_base;      // CSR of incident segments over the input points
  int32_t status;
  int32_t active;        // take part in refinement
  int32_t first_cand, last_cand;   // this iteration's candidate range
  int32_t ins_ok;        // this iteration's insertions fit the capacity
  int32_t pending;       // work left beyond the per-iteration cap
  int32_t steiner;       // Steiner points inserted by refinement
  int32_t has_apex;      // some input angle below 60 degrees
  int32_t cand_cap;      // per-iteration candidate cap (0 = none)
  int32_t lens;          // encroachment by the diametral lens (Chew), else the circle
  int32_t need_grow;     // refinement: 1 = under a quarter of the slots left, 2 = an
                         // iteration's insertions did not fit (the host grows the pool)
  int32_t ff_v0;         // Flip-Flop: vert_count at the start of this iteration (the
                         // vertices from here on were inserted in this iteration)
  int32_t pts_base;      // offset of this mesh's points in the construction list
  int32_t tmp;           // scratch for per-mesh reductions
  double B2;
  double L2;             // edge-length bound squared (Sec. 4.1), 0 = none
  double2 lo, hi;        // bounding box of the input points
  double2 org;           // origin of the float coordinate copies (box centre)
  float B2f;             // B^2 rounded to float (FP32 pre-checks)
};

struct Ctrl {
  int32_t n_cand;        // candidates this iteration / round
  int32_t prev_cand;     // candidates whose marks must be cleared
  int32_t n_raw;         // elements found by the last scan
  int32_t n_pts;         // CDT: points not yet inserted
  int32_t n_pts_next;    // CDT: points left after this round (moved to n_pts between rounds)
  int32_t n_segs;        // CDT: segments not yet recovered
  int32_t changed;       // flood fill progress
  int32_t err;           // first hard error (status code)
  int32_t round;         // CDT: insertion round (keys of earlier rounds compare lower)
  int32_t n_fl;          // CDT: triangles whose edges the current flip pass checks
  int32_t n_fl_next;     // CDT: triangles pushed for the next flip pass
  int32_t step;          // CDT: split / flip pass number (stamps, flip keys)
  int32_t scan_hi;       // refinement scans slots [0, scan_hi); 0 = all slots
  int32_t guard_r;       // CDT graph loops: round pairs run (bounded)
  int32_t guard_f;       // CDT graph loops: flip conditions evaluated (bounded)
  unsigned long long tot_cand, tot_ins, iters, n_ins, n_surv;
  // refinement work counters (algorithmic bytes of the cavity kernels)
  unsigned long long n_grown, sum_cav, sum_bnd, sum_walk;
  // the same for the launches timed with CUDA events (GDP_REFINE_TIME_GROW)
  unsigned long long t_grown, t_cav, t_bnd, t_walk;
  // candidates set up by the refinement pre-pass (all / in the timed launches)
  unsigned long long n_setup, t_setup;
  // live triangles and subsegments of all meshes after a refine call (k_count_live)
  unsigned long long live_tri, live_sub;
  int32_t grow_next;     // k_grow_t: next candidate to hand out
  int32_t need_eval;     // some triangles are marked dirty (construction, relocation)
  int32_t grow;          // some mesh asks for more slots (MeshInfo::need_grow)
  int32_t ff_marked;     // Flip-Flop: points found redundant by the last check
  int32_t dbg;           // which internal check failed first (GDP_TRACE reports it)
  unsigned long long ff_flips, ff_flops, ff_removed;   // Flip-Flop work counters
};

struct Pool {
  // mesh
  double2* V;
  float4* Vf;            // float copies of V - org (FP32 filter stage)
  int32_t* vseg;
  int32_t* vtri;
  uint8_t* apex;
  int4* T;
  int4* N;
  unsigned long long* mark;
  unsigned long long* pmark;   // pre-pass marks (first rings), cleared like mark
  int32_t* newref;
  uint8_t* dirty;
  uint8_t* flag;
  MeshInfo* mi;
  int32_t n_mesh;
  int32_t n_slots;       // triangle slots spanned by all meshes
  int32_t n_verts;       // vertex slots spanned by all meshes
  // input segments (global vertex ids) and per-input-vertex incident segments
  int2* seg;
  int32_t* adj_off;
  int32_t* adj;
  // candidates
  int32_t cap_cand;
  int32_t warp_max;      // up to this many candidates, one warp grows each cavity
  int32_t no_prepass;    // 1: the pre-pass sets candidates up but places no marks (ablation)
  int32_t* c_elem;
  int32_t* c_loc;
  int32_t* c_vid;
  int32_t* c_mesh;
  int32_t* c_vseg;
  int2* c_sub;
  double2* c_pt;
  float4* c_ptf;
  unsigned long long* c_key;
  int32_t* c_ncav;
  int32_t* c_nbnd;
  int32_t* c_cav;
  int4* c_bnd;
  // per-mesh candidate cap (Rule 2): priority bucket of each flagged slot,
  // per-mesh bucket histograms and the lowest bucket taken this iteration
  uint16_t* cbucket;
  int32_t* cap_hist;
  int32_t* cap_thr;
  int32_t* c_big;        // offset of the cavity in the spill tiers, -1 = own slot
  struct CandSetup* c_setup;   // refinement pre-pass: each candidate's set-up
  int32_t* c_pre;        // PRE_MAX per candidate: its pre-marked triangles
  int32_t* c_npre;       // how many (0: no set-up)
  int32_t* big_cav;      // BIG_ENTRIES
  int4* big_bnd;         // BIG_ENTRIES
  int32_t* big_hash;     // BIG_HASH
  int2* big_val;         // BIG_HASH: values of the fan map of a spill-tier cavity
  int32_t* lane;         // LANES_A + LANES_B owners (smallest candidate index)
  uint8_t* c_state;
  uint8_t* c_final;
  int32_t* c_extra;
  int32_t* c_offT;
  int32_t* c_offV;
  int32_t* c_base;
  int32_t* blk;          // block partial sums, 2 * G
  Ctrl* ctrl;
  // CDT construction
  int32_t* pts;
  int32_t* pts2;
  int32_t* loc;          // per vertex: containing triangle, -1 once inserted
  unsigned long long* tbest;
  // split + flip construction rounds
  int32_t* tstamp;       // per slot: the split / flip pass that last rewrote it
  int32_t* lstamp;       // per slot: the flip pass whose list holds it
  int32_t* fl_cur;       // triangles checked by this flip pass (ctrl->n_fl)
  int32_t* fl_nxt;       // triangles pushed for the next pass (ctrl->n_fl_next)
  int32_t* fprop;        // per list entry: proposed flip t << 2 | e, -1 none, -2 - prop done
  int32_t* segq;         // segments still to recover
  unsigned long long* segmark;
  uint8_t* ext;
  int32_t* remap;
  // Flip-Flop insertion (refinement with GDP_REFINE_FLIPFLOP; allocated on first use)
  unsigned long long* vkey;    // per vertex: priority key of a point inserted this iteration
  int32_t* vred;               // per vertex: bit 0 redundant, bit 1 removed
  int32_t* vmap;               // per vertex: id after the removed points are compacted away
  unsigned long long* ffmark;  // per slot: flip / flop ownership marks
  int32_t* fop;                // per list entry: operation kind of the proposal
};

}  // namespace gdp
