/*
 * gdp.h -- C ABI of the GB300 constrained Delaunay refinement library (gDP2d).
 *
 * The library turns a planar straight-line graph (PSLG: points P and
 * non-crossing segments E, Sec. 4 of the paper) into its constrained Delaunay
 * triangulation (CDT, the first step of Algorithm 1) and refines it (the loop of
 * Algorithm 1): Steiner points are inserted in parallel until no subsegment is
 * encroached (a vertex strictly inside its diametral circle, Sec. 4.2) and no
 * triangle has radius-edge ratio above B (the 3D bad-element measure of
 * Sec. 5.1, used here in 2D; B = sqrt 2 is a 20.7 degree angle bound).
 *
 * Everything between create and export runs on one GPU in CUDA kernels; the
 * host only launches them.  There is no CPU fallback: every call returns
 * GDP_ERR_CUDA when no usable device is present.
 *
 * Conventions for every entry point:
 *   - Host pointers unless the name says _device.  Input buffers are owned by
 *     the caller and copied; the library never keeps a caller pointer.
 *   - Meshes and batches are owned by the library from create to destroy.
 *   - Coordinates are FP64, points as interleaved (x, y) pairs; segments are
 *     pairs of 0-based indices into the points; triangles are CCW triples.
 *   - Every call returns a gdp_status.  After an error the object can still
 *     be destroyed; after GDP_ERR_NOMEM or GDP_ERR_ITER_LIMIT during refine
 *     the mesh is still a valid CDT and can be exported.
 *   - cuda_stream may be NULL (the legacy default stream) or a cudaStream_t;
 *     all work of the object is ordered on that stream.
 */
#ifndef GDP_H
#define GDP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GDP_OK = 0,
    GDP_ERR_INPUT = 1,       /* NaN/inf coordinate, duplicate point, bad index, crossing
                                segments, segment through a vertex, empty domain */
    GDP_ERR_NOMEM = 2,       /* device allocation failed, or a mesh ran out of slots and
                                could not be given more (see gdp_mesh_refine) */
    GDP_ERR_ITER_LIMIT = 3,  /* refinement hit max_iter */
    GDP_ERR_WALK_LIMIT = 4,  /* a point-location walk exceeded its step bound */
    GDP_ERR_CUDA = 5,        /* CUDA runtime error or no device */
    GDP_ERR_INTERNAL = 6,    /* an invariant check inside a kernel failed */
    GDP_ERR_CAPACITY = 7     /* a per-element work buffer overflowed: a cavity above 65536
                                triangles, or a segment crossing more than 32768 edges */
} gdp_status;

typedef struct gdp_mesh gdp_mesh;

/* Refinement options.  Zero-initialised fields take the defaults. */
typedef struct {
    double B;             /* radius-edge bound (> 0.70711; sqrt 2 default when 0) */
    double max_len;       /* edge-length bound l (Sec. 4.1): a triangle whose longest
                             edge exceeds l is refined as well; <= 0 or INF = off */
    int32_t max_iter;     /* parallel iterations (Algorithm 1 loop), 0 = 100000 */
    int32_t cand_cap;     /* candidates per iteration and mesh; 0 = no cap (Rule 2) */
    int32_t graph_iters;  /* iterations per CUDA-graph replay; 0 = 8, < 0 = no graph */
    int32_t flags;        /* GDP_REFINE_* bits, 0 = none */
    int32_t cand_block;   /* threads per block of the per-candidate kernels:
                             32, 64, 128 or 256; 0 = 64 */
} gdp_refine_opts;

typedef struct {
    int64_t n_in_pts;     /* input points */
    int64_t n_steiner;    /* Steiner points inserted by refinement */
    int64_t n_tris;       /* live triangles */
    int64_t n_subsegs;    /* subsegments */
    int64_t iterations;   /* refinement iterations executed */
    int64_t candidates;   /* splitting points considered, summed over iterations */
    int64_t inserted;     /* splitting points inserted, summed over iterations */
    int64_t cdt_rounds;   /* parallel insertion rounds of the initial CDT */
    double refine_ms;     /* device time of the refinement loop */
    double cdt_ms;        /* device time of the initial CDT */
    int64_t launches;     /* kernel launches of this object since creation */
    /* refinement work of the cavity kernel k_grow (candidates that fit in
     * their own slot), summed over iterations:                           */
    int64_t grown;        /* candidates whose cavity was grown */
    int64_t cavity_tris;  /* triangles in those cavities */
    int64_t cavity_edges; /* boundary edges of those cavities */
    int64_t walk_steps;   /* point-location steps of circumcentres */
    /* with GDP_REFINE_TIME_GROW: the cavity-growth launches of the first
     * iteration of every graph replay are bracketed by CUDA events inside
     * the graph; their device time, their number and their work:          */
    double grow_ms;
    int64_t grow_launches;
    int64_t timed_grown, timed_cavity_tris, timed_cavity_edges, timed_walk_steps;
    /* capacity growth: times the pool was re-laid out with more slots for the
     * meshes that ran short (each time doubling their Steiner capacity) */
    int64_t grow_steps;
    /* with GDP_REFINE_FLIPFLOP: flips, flops (point removals) and redundant
     * points removed, summed over the iterations */
    int64_t flips, flops, redundant_removed;
    /* refinement candidates set up by the pre-pass that precedes cavity
     * growth (splitting point, walk, first-ring marks); the ones that keep
     * all their first-ring marks are grown.  All iterations / the timed
     * launches. */
    int64_t setups, timed_setups;
} gdp_stats;

/* gdp_refine_opts.flags */
#define GDP_REFINE_TIME_GROW 1
/* Chew's rule (Sec. 4.2): a subsegment is encroached by a vertex or splitting
 * point strictly inside its diametral lens -- where the subsegment subtends
 * more than 120 degrees -- instead of its diametral circle (Ruppert's rule,
 * the default).  Only the encroachment region changes: split points, shells,
 * priorities and the quality test stay those of the default mode. */
#define GDP_REFINE_CHEW 2
/* Flip-Flop insertion (Sec. 4.3, the paper's gDP2d): the splitting points that
 * survive the cavity filter all go in by splitting their triangles, then
 * parallel flips restore the constrained Delaunay property, and of two points
 * of one iteration joined by an edge (Delaunay dependent, Sec. 4.2) the one
 * with the lower priority is removed again by flips and a flop; the default
 * is cavity (Bowyer-Watson) insertion with the dependence check before it.
 * Iterations are driven from the host (no CUDA graph). */
#define GDP_REFINE_FLIPFLOP 4

/* Build the CDT of a PSLG on the GPU (the first step of Algorithm 1).
 *   xy:  2*n_pts doubles, host;   seg: 2*n_seg int32 indices, host (may be NULL if 0)
 * The domain is the region enclosed by segments: triangles reachable from
 * outside without crossing a segment are removed, so the convex hull must be
 * covered by segments for the whole hull to be meshed.
 * Errors: GDP_ERR_INPUT for invalid input, GDP_ERR_NOMEM, GDP_ERR_CUDA. */
int gdp_mesh_create(const double* xy, int64_t n_pts, const int32_t* seg, int64_t n_seg,
                    void* cuda_stream, gdp_mesh** out);

/* Same, with xy and seg already in device memory (not modified, not kept). */
int gdp_mesh_create_device(const double* xy_device, int64_t n_pts, const int32_t* seg_device,
                           int64_t n_seg, void* cuda_stream, gdp_mesh** out);

/* Refine (the loop of Algorithm 1) until nothing is encroached and no
 * triangle is bad, bad triangles at small input angles excepted (Sec. 4.1).
 * opts may be NULL (defaults); stats may be NULL.  Blocks until done.
 * Slots: a mesh starts with room for 3 Steiner points per input point plus 64
 * per segment (GDP_STEINER_PER_POINT / _PER_SEGMENT).  When it has used three
 * quarters of them, or an iteration's insertions do not fit, the pool is laid
 * out again between graph replays with twice the Steiner capacity for that
 * mesh (at most 20 times, GDP_GROW_LIMIT); the deferred insertions are
 * retried, so the result does not depend on the starting capacity.  If the
 * larger pool cannot be allocated, the mesh stops with GDP_ERR_NOMEM and is
 * still a valid CDT that can be exported. */
int gdp_mesh_refine(gdp_mesh* mesh, const gdp_refine_opts* opts, gdp_stats* stats);

/* Copy the mesh out: the result of Algorithm 1 (the refined constrained
 * Delaunay triangulation) or, before gdp_mesh_refine, the initial CDT.  This
 * is the boundary's output side; the paper defines no interface for it.
 * Call with NULL buffers to get the sizes only.
 *   xy:     2*cap_pts doubles: input points keep ids 0..n_in-1, Steiner points follow
 *   tri:    3*cap_tri int32, CCW
 *   subseg: 3*cap_seg int32: (u, v, input segment id)
 * A buffer smaller than the size needed gives GDP_ERR_INPUT and copies nothing. */
int gdp_mesh_export(gdp_mesh* mesh, double* xy, int64_t cap_pts, int32_t* tri, int64_t cap_tri,
                    int32_t* subseg, int64_t cap_seg, int64_t* n_pts, int64_t* n_tri,
                    int64_t* n_seg);

/* Insert a fixed batch of free points (strictly inside the domain, not on a
 * subsegment, no duplicates) with the parallel cavity kernels (Sec. 5.2
 * cavity insertion, priority marks and the dependence check), in as many
 * parallel rounds as conflicts require.  The result is the CDT of the
 * enlarged vertex set. */
int gdp_mesh_insert_points(gdp_mesh* mesh, const double* xy, int64_t n);

/* Split the subsegments given by endpoint coordinates (4 doubles each:
 * ax, ay, bx, by) at their split points -- the midpoint, or the
 * concentric-shell point when exactly one end is an input vertex where two
 * segments meet below 60 degrees (Sec. 4.1 small input angles) -- with the
 * parallel cavity kernels, in as many rounds as conflicts require. */
int gdp_mesh_split_subsegments(gdp_mesh* mesh, const double* abxy, int64_t n);

/* One bad-element scan (Algorithm 1) plus splitting points and
 * priorities (before point location) of the current mesh.
 * Outputs per element, cap entries each (host buffers, NULL to skip):
 *   kind[i]:  0 = bad triangle, 1 = encroached subsegment, 2 = bad triangle
 *             accepted by the small-angle exemption (Sec. 4.1: its shortest
 *             edge joins two segments that meet below 60 degrees)
 *   verts[3i..3i+2]: the triangle's vertices (CCW), or the subsegment's two
 *             endpoints and -1
 *   pt[2i..2i+1]: circumcentre (C5 formula) or split point
 *   meas[i]: priority measure bits (float32 bits of 2*area or squared length)
 * *count receives the number of elements (all of them, even beyond cap). */
int gdp_mesh_scan(gdp_mesh* mesh, double B, int32_t* kind, int32_t* verts, double* pt,
                  uint32_t* meas, int64_t cap, int64_t* count);

/* The same with the encroachment region of flags (GDP_REFINE_CHEW: the
 * diametral lens, Sec. 4.2; 0: the diametral circle, as gdp_mesh_scan).
 * GDP_ERR_INPUT for B <= 0 or an unknown flag. */
int gdp_mesh_scan_mode(gdp_mesh* mesh, double B, int32_t flags, int32_t* kind, int32_t* verts,
                       double* pt, uint32_t* meas, int64_t cap, int64_t* count);

/* Consistency of the device mesh (a test hook): counts[0..4] receive the
 * number of neighbour links that are not mutual, links whose shared edge does
 * not match, subsegment flags that differ across an edge, triangles that are
 * not strictly CCW (exact orient), and hull edges that are not subsegments.
 * All zero for a valid mesh. */
int gdp_mesh_check(gdp_mesh* mesh, int64_t counts[5]);

/* Statistics of the last create/refine. */
int gdp_mesh_stats(gdp_mesh* mesh, gdp_stats* stats);

/* Per-kernel timing.  gdp_mesh_profile(mesh, 1) clears the table and brackets
 * every later kernel launch of the mesh with CUDA events on its stream
 * (refinement then runs without CUDA graphs); 0 turns it off.
 * gdp_mesh_kernel_time reads entry i of the table: the kernel's name (NUL
 * terminated, truncated to name_cap), its summed device time in ms and its
 * launch count.  Returns GDP_ERR_INPUT when i is past the end. */
int gdp_mesh_profile(gdp_mesh* mesh, int enable);
int gdp_mesh_kernel_time(gdp_mesh* mesh, int32_t i, char* name, int64_t name_cap, double* total_ms,
                         int64_t* count);

/* Free the mesh and every device allocation it holds (stream-ordered on its
 * stream).  NULL is ignored.  Housekeeping with no counterpart in the paper. */
void gdp_mesh_destroy(gdp_mesh* mesh);

/* ---------------- batches: many independent PSLGs in one pool ----------------
 * All meshes of a batch share device arrays; every kernel launch processes
 * all of them (one launch per step for the whole batch), and each mesh is
 * refined exactly as it would be alone.
 *   xy:      concatenated points, 2*sum(n_pts) doubles
 *   pt_off:  n_meshes+1 offsets into points (pt_off[0] = 0)
 *   seg:     concatenated segments, 2*sum(n_seg) int32, indices LOCAL to their mesh
 *   seg_off: n_meshes+1 offsets into segments */
typedef struct gdp_batch gdp_batch;

int gdp_batch_create(const double* xy, const int64_t* pt_off, const int32_t* seg,
                     const int64_t* seg_off, int32_t n_meshes, void* cuda_stream,
                     gdp_batch** out);
/* B: one bound per mesh (NULL: opts->B for all). */
int gdp_batch_refine(gdp_batch* b, const double* B, const gdp_refine_opts* opts,
                     gdp_stats* stats);
/* per-mesh status and sizes (arrays of n_meshes, NULL to skip) */
int gdp_batch_info(gdp_batch* b, int32_t* status, int64_t* n_pts, int64_t* n_tri,
                   int64_t* n_seg, int64_t* n_steiner);
int gdp_batch_export(gdp_batch* b, int32_t mesh, double* xy, int64_t cap_pts, int32_t* tri,
                     int64_t cap_tri, int32_t* subseg, int64_t cap_seg, int64_t* n_pts,
                     int64_t* n_tri, int64_t* n_seg);
void gdp_batch_destroy(gdp_batch* b);

/* ---------------- autotuning (Rule 2) ----------------
 * Not a step of Algorithm 1: picks the launch parameters of the refinement
 * for a workload.  For the PSLGs given (layout of gdp_batch_create; a sample
 * of the workload) it builds their CDT once per trial and refines with every
 * pair of cand_block in {32, 64, 128, 256} and cand_cap in
 * {0, 16384, 4096, 1024, 256}, starting from *base (may be NULL), and writes
 * to *best the options with the most Steiner points per second of refinement
 * device time.  trials (may be NULL): 4 doubles per trial (cand_block,
 * cand_cap, refine ms, Steiner points), up to trials_cap trials (20 in all).
 * B: one bound per mesh (NULL: base->B).  Errors as gdp_batch_create /
 * gdp_batch_refine. */
int gdp_autotune(const double* xy, const int64_t* pt_off, const int32_t* seg,
                 const int64_t* seg_off, int32_t n_meshes, const double* B,
                 const gdp_refine_opts* base, void* cuda_stream, gdp_refine_opts* best,
                 double* trials, int32_t trials_cap);

/* ---------------- serving (continuous batching) ----------------
 * Not in the paper: a request loop around Algorithm 1.  A server keeps one
 * resident device pool with room for tri_slots triangles, vert_slots vertices,
 * seg_slots input segments and max_meshes meshes (admission is by this
 * device memory).  Each gdp_server_step
 *   1. launches opts->graph_iters (0: 8) refinement iterations
 *      over every resident mesh at once (one CUDA-graph replay);
 *   2. while they run, builds the initial CDT of the oldest waiting
 *      requests in staging pools on a second stream, as long as a region of
 *      the resident pool is free for them (first come, first served);
 *   3. retires the meshes that finished (no candidate in the last iteration,
 *      nothing deferred), copying each result to host memory and freeing its
 *      region, and moves the new CDTs into their regions so that they join
 *      the next replay.
 * A request's result does not depend on the other requests: it is the same
 * mesh gdp_mesh_create + gdp_mesh_refine give for it alone.
 * The stream (may be NULL) is the one the refinement runs on.  opts: B is
 * unused (each request has its own), cand_cap / cand_block as for refine.
 * tri_slots < 2^29, vert_slots < 2^30, max_meshes <= 2^20.
 * Errors: GDP_ERR_INPUT, GDP_ERR_NOMEM (pool allocation), GDP_ERR_CUDA; on
 * error *out may still be set and must be destroyed. */
typedef struct gdp_server gdp_server;
typedef struct {
    int64_t ticket;        /* from gdp_server_submit */
    int32_t status;        /* gdp_status of this request */
    int64_t n_in_pts, n_steiner, n_pts, n_tri, n_subseg;
    double t_submit_ms;    /* server clock (ms since creation): submitted, */
    double t_admit_ms;     /* joined the resident pool, */
    double t_done_ms;      /* copied out */
} gdp_result_info;
int gdp_server_create(int64_t tri_slots, int64_t vert_slots, int64_t seg_slots, int32_t max_meshes,
                      const gdp_refine_opts* opts, void* cuda_stream, gdp_server** out);
/* Queue a request (host buffers, copied; same layout as gdp_mesh_create) with
 * bound B.  GDP_ERR_NOMEM when it could never fit the pool. */
int gdp_server_submit(gdp_server* s, const double* xy, int64_t n_pts, const int32_t* seg,
                      int64_t n_seg, double B, int64_t* ticket);
/* One scheduling step (blocking); counts after it (NULL to skip). */
int gdp_server_step(gdp_server* s, int32_t* n_waiting, int32_t* n_live, int32_t* n_done);
/* The oldest finished request.  With all buffers NULL: fills *info and keeps
 * it (sizes for the buffers); with buffers (layout of gdp_mesh_export): copies
 * it out and removes it.  GDP_ERR_INPUT when none is finished or a buffer is
 * too small. */
int gdp_server_result(gdp_server* s, gdp_result_info* info, double* xy, int64_t cap_pts,
                      int32_t* tri, int64_t cap_tri, int32_t* subseg, int64_t cap_seg);
void gdp_server_destroy(gdp_server* s);

/* ---------------- scan without device allocation ----------------
 * The paper has no counterpart to this entry point: it exists for callers
 * that must not allocate device memory (code running inside another
 * allocator's callbacks, processes whose device memory is fully pre-reserved
 * by a framework pool, real-time paths where an allocation could block).
 * It runs the same per-element tests as gdp_mesh_scan on a triangulation the
 * caller keeps in its own device buffers and writes into output buffers the
 * caller owns; it calls no cudaMalloc, cudaFree or allocating library routine.
 *
 *   xy_device:  2*n_vert doubles (x, y), 16-byte aligned
 *   tri_device: 4 int32 per triangle, 16-byte aligned: v0, v1, v2 (CCW) and a
 *               flags word whose bit e says that edge e = (v[e+1], v[e+2]) is a
 *               subsegment
 *   outputs (device, cap entries each, laid out as in gdp_mesh_scan):
 *               kind_device, verts_device (3 per entry), pt_device (2 doubles
 *               per entry, 16-byte aligned: the circumcentre, or for an
 *               encroached subsegment always its midpoint -- the call has no
 *               segment data, so no concentric-shell points and no small-angle
 *               exemption), meas_device
 *   *count (host): number of entries found, even beyond cap.  Entries come in
 *               triangle order: a bad triangle first, then its encroached edges.
 * Scratch: one file-scope device array of about 4.2 MB (per-triangle counts for
 * up to GDP_NOALLOC_MAX_TRIANGLES triangles plus block sums) that every GPU
 * which loads the library keeps until the process exits.  n_tri above
 * GDP_NOALLOC_MAX_TRIANGLES gives GDP_ERR_CAPACITY; a vertex id outside
 * [0, n_vert) or a misaligned buffer gives GDP_ERR_INPUT (before anything is
 * launched, for the alignment).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress), which may load the library's device code and so
 * allocate: make that first call as a warm-up, outside the context that must
 * not allocate and before any stream capture.  The address is kept for the
 * life of the process; resetting the device between calls is not supported.
 * All calls share the array, so calls that overlap on the GPU (for example
 * on two streams) race on it: issue them one after another.  The call blocks
 * until the count has been read back. */
#define GDP_NOALLOC_MAX_TRIANGLES (1 << 22)
int gdp_scan_noalloc(const double* xy_device, int64_t n_vert, const int32_t* tri_device,
                     int64_t n_tri, double B, int32_t* kind_device, int32_t* verts_device,
                     double* pt_device, uint32_t* meas_device, int64_t cap, int64_t* count,
                     void* cuda_stream);

/* ---------------- measurement ----------------
 * Not a step of the paper: the FP64 throughput of the current device, the
 * denominator of the FP64 roofline of the refinement kernels.  One kernel of
 * independent fused multiply-add chains (two flops each) over 8 blocks of 256
 * threads per SM, timed with CUDA events on cuda_stream (NULL: the legacy
 * default stream); *tflops receives the best of three timed launches after a
 * warm-up.  Allocates nothing.  Errors: GDP_ERR_INPUT (tflops NULL),
 * GDP_ERR_CUDA. */
int gdp_measure_fp64_peak(void* cuda_stream, double* tflops);

/* A static, human-readable name of a status code ("ok", "invalid input", ...);
 * unknown codes give "unknown".  Housekeeping with no counterpart in
 * the paper. */
const char* gdp_status_str(int status);

#ifdef __cplusplus
}
#endif
#endif
